"""Thin Python binding of the C ABI in ``include/lbe.h`` (ctypes).

Only argument marshalling happens here: every step of the LBE path runs in
the CUDA kernels of ``liblbe.so``.  If the library is missing or cannot be
loaded, ``load()`` raises -- there is no CPU fallback.  PyTorch provides
device buffers and the CUDA stream.

The functions keep the C names (``lbe_create``, ``lbe_step`` ...); ``Lattice``
wraps one handle for convenience.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbe.so")

LBE_OK = 0
LBE_ERR_ARG = -1
LBE_ERR_CUDA = -2
LBE_ERR_NOCONVERGE = -3
LBE_ERR_NONFINITE = -4
LBE_ERR_STATE = -5
LBE_ERR_GEOMETRY = -6
LBE_FP64, LBE_FP32 = 0, 1
LBE_RULE_MIDPLANE, LBE_RULE_NODE = 0, 1
LBE_MAX_SPECIES = 4
LBE_MAX_ELECTRODES = 16
FIELD_PHI, FIELD_N, FIELD_RHO, FIELD_U, FIELD_F, FIELD_QNODE = 0, 1, 2, 3, 4, 5
# order of the 19 populations in FIELD_F (as documented in lbe.h)
_HALF = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, -1, 0), (1, 0, 1), (1, 0, -1), (0, 1, 1), (0, 1, -1)]
VELOCITIES = [(0, 0, 0)] + _HALF + [(-a, -b, -c) for (a, b, c) in _HALF]

EXPORTED = ["lbe_default_params", "lbe_create", "lbe_destroy", "lbe_last_error", "lbe_set_geometry",
            "lbe_set_voltage", "lbe_init", "lbe_step", "lbe_induced_charge", "lbe_fields",
            "lbe_set_state", "lbe_save_state", "lbe_load_state", "lbe_get_stats",
            "lbe_profile_begin", "lbe_profile_end", "lbe_induced_charge_static",
            "lbe_batch_create", "lbe_batch_destroy", "lbe_batch_last_error", "lbe_batch_set_geometry",
            "lbe_batch_set_voltage", "lbe_batch_init", "lbe_batch_step", "lbe_batch_charge",
            "lbe_batch_fields", "lbe_batch_get_stats", "lbe_batch_tuning",
            "lbe_batch_profile_begin", "lbe_batch_profile_end",
            "lbe_adjoint_forward", "lbe_adjoint_forward_budget", "lbe_adjoint_backward"]
LBE_BATCH_MAX_ELECTRODES = 4
LBE_BATCH_TUNE_CANDIDATES = 6


class lbe_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("periodic", ctypes.c_int * 3), ("tau", ctypes.c_double), ("bjerrum", ctypes.c_double),
                ("nspecies", ctypes.c_int), ("z", ctypes.c_double * LBE_MAX_SPECIES),
                ("D", ctypes.c_double * LBE_MAX_SPECIES), ("rho_bulk", ctypes.c_double * LBE_MAX_SPECIES),
                ("e_app", ctypes.c_double * 3), ("flow", ctypes.c_int), ("precision", ctypes.c_int),
                ("poisson_tol", ctypes.c_double), ("poisson_max_iter", ctypes.c_int),
                ("boundary_rule", ctypes.c_int)]


class lbe_stats(ctypes.Structure):
    _fields_ = [("poisson_iters", ctypes.c_longlong), ("poisson_solves", ctypes.c_int),
                ("poisson_max_iters", ctypes.c_int), ("poisson_residual", ctypes.c_double)]


class lbe_profile(ctypes.Structure):
    _fields_ = [("sweep_ms", ctypes.c_double), ("sweep_launches", ctypes.c_longlong),
                ("advect_ms", ctypes.c_double), ("advect_launches", ctypes.c_longlong),
                ("poisson_ms", ctypes.c_double), ("poisson_solves", ctypes.c_longlong),
                ("poisson_iters", ctypes.c_longlong), ("kernel_launches", ctypes.c_longlong)]


class lbe_adjoint_grad(ctypes.Structure):
    _fields_ = [("dpsi", ctypes.c_double * LBE_MAX_ELECTRODES), ("drho_bulk", ctypes.c_double),
                ("dD", ctypes.c_double * LBE_MAX_SPECIES), ("poisson_iters", ctypes.c_longlong),
                ("recomputed_steps", ctypes.c_longlong), ("recompute_ms", ctypes.c_double),
                ("flux_ms", ctypes.c_double), ("solve_ms", ctypes.c_double)]


_lib = None


class LBEError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"LBE error {code}: {msg}")
        self.code = code


def load(path: str = LIB_PATH):
    """Load ``liblbe.so``; raises if it is missing (build it with build.py)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} not built: run paper_1907_04732_gb300/build.py")
    lib = ctypes.CDLL(path)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
    lib.lbe_default_params.argtypes = [ctypes.POINTER(lbe_params)]
    lib.lbe_default_params.restype = None
    lib.lbe_create.argtypes = [ctypes.POINTER(lbe_params), vp, ctypes.POINTER(vp)]
    lib.lbe_destroy.argtypes = [vp]
    lib.lbe_last_error.argtypes = [vp]
    lib.lbe_last_error.restype = ctypes.c_char_p
    lib.lbe_set_geometry.argtypes = [vp, vp, ip, ip]
    lib.lbe_set_voltage.argtypes = [vp, dp]
    lib.lbe_init.argtypes = [vp]
    lib.lbe_step.argtypes = [vp, ip]
    lib.lbe_induced_charge.argtypes = [vp, vp, ip]
    lib.lbe_fields.argtypes = [vp, ip, vp, ip]
    lib.lbe_set_state.argtypes = [vp, vp, vp, ip]
    lib.lbe_save_state.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_size_t)]
    lib.lbe_load_state.argtypes = [vp, vp, ctypes.c_size_t]
    lib.lbe_get_stats.argtypes = [vp, ctypes.POINTER(lbe_stats)]
    lib.lbe_profile_begin.argtypes = [vp]
    lib.lbe_profile_end.argtypes = [vp, ctypes.POINTER(lbe_profile)]
    lib.lbe_induced_charge_static.argtypes = [vp, vp, ip, ip, ip, ctypes.POINTER(ctypes.c_int), ctypes.c_double,
                                              ip, vp, vp]
    lib.lbe_batch_create.argtypes = [ctypes.POINTER(lbe_params), ip, vp, ctypes.POINTER(vp)]
    lib.lbe_batch_destroy.argtypes = [vp]
    lib.lbe_batch_last_error.argtypes = [vp]
    lib.lbe_batch_last_error.restype = ctypes.c_char_p
    lib.lbe_batch_set_geometry.argtypes = [vp, ip, vp, ip]
    lib.lbe_batch_set_voltage.argtypes = [vp, ip, dp]
    lib.lbe_batch_init.argtypes = [vp]
    lib.lbe_batch_step.argtypes = [vp, ip]
    lib.lbe_batch_charge.argtypes = [vp, vp, ip]
    lib.lbe_batch_fields.argtypes = [vp, ip, ip, vp, ip]
    lib.lbe_batch_get_stats.argtypes = [vp, ctypes.POINTER(lbe_stats)]
    lib.lbe_batch_tuning.argtypes = [vp, ctypes.POINTER(ctypes.c_int), dp]
    lib.lbe_adjoint_forward.argtypes = [vp, ip, ip, dp]
    lib.lbe_adjoint_forward_budget.argtypes = [vp, ip, ctypes.c_size_t, dp]
    lib.lbe_adjoint_backward.argtypes = [vp, dp, ip, ctypes.POINTER(lbe_adjoint_grad), vp, ip]
    lib.lbe_batch_profile_begin.argtypes = [vp]
    lib.lbe_batch_profile_end.argtypes = [vp, ctypes.POINTER(lbe_profile)]
    for name in EXPORTED:
        if name not in ("lbe_default_params", "lbe_last_error", "lbe_batch_last_error"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(h, rc):
    if rc != LBE_OK:
        msg = load().lbe_last_error(h)
        raise LBEError(rc, msg.decode() if msg else "")
    return rc


# --- C names -------------------------------------------------------------
def lbe_default_params() -> lbe_params:
    p = lbe_params()
    load().lbe_default_params(ctypes.byref(p))
    return p


def lbe_create(params: lbe_params, stream: int = 0) -> int:
    h = ctypes.c_void_p()
    rc = load().lbe_create(ctypes.byref(params), ctypes.c_void_p(stream or None), ctypes.byref(h))
    if rc != LBE_OK:
        raise LBEError(rc, "lbe_create failed (invalid parameters or CUDA error)")
    return h.value


def lbe_destroy(h: int) -> None:
    load().lbe_destroy(h)


def lbe_set_geometry(h, node_id_ptr: int, n_electrodes: int, on_device: bool):
    return _check(h, load().lbe_set_geometry(h, node_id_ptr, n_electrodes, int(on_device)))


def lbe_set_voltage(h, psi):
    arr = (ctypes.c_double * max(len(psi), 1))(*psi)
    return _check(h, load().lbe_set_voltage(h, arr))


def lbe_init(h):
    return _check(h, load().lbe_init(h))


def lbe_step(h, nsteps: int):
    return _check(h, load().lbe_step(h, int(nsteps)))


def lbe_induced_charge(h, out_ptr: int, on_device: bool):
    return _check(h, load().lbe_induced_charge(h, out_ptr, int(on_device)))


def lbe_fields(h, which: int, out_ptr: int, on_device: bool):
    return _check(h, load().lbe_fields(h, which, out_ptr, int(on_device)))


def lbe_set_state(h, n_ptr, phi_ptr, on_device: bool):
    return _check(h, load().lbe_set_state(h, n_ptr, phi_ptr, int(on_device)))


def lbe_save_state(h, blob_ptr, size: ctypes.c_size_t):
    return _check(h, load().lbe_save_state(h, blob_ptr, ctypes.byref(size)))


def lbe_load_state(h, blob_ptr, size: int):
    return _check(h, load().lbe_load_state(h, blob_ptr, size))


def lbe_get_stats(h) -> lbe_stats:
    s = lbe_stats()
    _check(h, load().lbe_get_stats(h, ctypes.byref(s)))
    return s


def lbe_profile_begin(h):
    return _check(h, load().lbe_profile_begin(h))


def lbe_profile_end(h) -> lbe_profile:
    out = lbe_profile()
    _check(h, load().lbe_profile_end(h, ctypes.byref(out)))
    return out


def lbe_induced_charge_static(phi_ptr: int, node_id_ptr: int, shape, periodic, bjerrum: float,
                              n_electrodes: int, q_out_ptr: int, stream: int = 0):
    """Induced charges from caller-owned device buffers; allocates nothing."""
    per = (ctypes.c_int * 3)(*[int(bool(p)) for p in periodic])
    rc = load().lbe_induced_charge_static(phi_ptr, node_id_ptr, int(shape[0]), int(shape[1]), int(shape[2]),
                                          per, float(bjerrum), int(n_electrodes), q_out_ptr,
                                          ctypes.c_void_p(stream or None))
    return _check(None, rc)


def lbe_adjoint_forward(h, nsteps: int, every: int, q_out=None):
    return _check(h, load().lbe_adjoint_forward(h, int(nsteps), int(every), q_out))


def lbe_adjoint_forward_budget(h, nsteps: int, device_bytes: int, q_out=None):
    return _check(h, load().lbe_adjoint_forward_budget(h, int(nsteps), int(device_bytes), q_out))


def lbe_adjoint_backward(h, dq, soft_electrode: int, dchi_ptr, dchi_on_device: bool) -> lbe_adjoint_grad:
    g = lbe_adjoint_grad()
    arr = (ctypes.c_double * max(len(dq), 1))(*[float(v) for v in dq])
    _check(h, load().lbe_adjoint_backward(h, arr, int(soft_electrode), ctypes.byref(g), dchi_ptr,
                                          int(dchi_on_device)))
    return g


def _bcheck(b, rc):
    if rc != LBE_OK:
        msg = load().lbe_batch_last_error(b)
        raise LBEError(rc, msg.decode() if msg else "")
    return rc


def lbe_batch_create(params_list, stream: int = 0) -> int:
    arr = (lbe_params * len(params_list))(*params_list)
    b = ctypes.c_void_p()
    rc = load().lbe_batch_create(arr, len(params_list), ctypes.c_void_p(stream or None), ctypes.byref(b))
    if rc != LBE_OK:
        raise LBEError(rc, "lbe_batch_create failed (invalid parameters or CUDA error)")
    return b.value


def lbe_batch_destroy(b):
    load().lbe_batch_destroy(b)


def lbe_batch_set_geometry(b, i: int, node_id_ptr: int, n_electrodes: int):
    return _bcheck(b, load().lbe_batch_set_geometry(b, i, node_id_ptr, n_electrodes))


def lbe_batch_set_voltage(b, i: int, psi):
    arr = (ctypes.c_double * max(len(psi), 1))(*psi)
    return _bcheck(b, load().lbe_batch_set_voltage(b, i, arr))


def lbe_batch_init(b):
    return _bcheck(b, load().lbe_batch_init(b))


def lbe_batch_step(b, nsteps: int):
    return _bcheck(b, load().lbe_batch_step(b, int(nsteps)))


def lbe_batch_charge(b, out_ptr: int, on_device: bool):
    return _bcheck(b, load().lbe_batch_charge(b, out_ptr, int(on_device)))


def lbe_batch_fields(b, i: int, which: int, out_ptr: int, on_device: bool):
    return _bcheck(b, load().lbe_batch_fields(b, i, which, out_ptr, int(on_device)))


def lbe_batch_get_stats(b) -> lbe_stats:
    s = lbe_stats()
    _bcheck(b, load().lbe_batch_get_stats(b, ctypes.byref(s)))
    return s


def lbe_batch_profile_begin(b):
    return _bcheck(b, load().lbe_batch_profile_begin(b))


def lbe_batch_profile_end(b) -> lbe_profile:
    out = lbe_profile()
    _bcheck(b, load().lbe_batch_profile_end(b, ctypes.byref(out)))
    return out


def lbe_batch_tuning(b):
    grid = ctypes.c_int(0)
    ms = (ctypes.c_double * LBE_BATCH_TUNE_CANDIDATES)()
    _bcheck(b, load().lbe_batch_tuning(b, ctypes.byref(grid), ms))
    return grid.value, list(ms)


# --- convenience wrapper ---------------------------------------------------
def params_for(workload, *, precision=LBE_FP64, tol=1e-13, maxit=100000, flow=None,
               rule=LBE_RULE_MIDPLANE) -> lbe_params:
    """lbe_params for a ``workloads.Workload`` (rule: lbe_params.boundary_rule)."""
    p = lbe_default_params()
    p.nx, p.ny, p.nz = workload.shape
    for a in range(3):
        p.periodic[a] = int(bool(workload.periodic[a]))
        p.e_app[a] = float(workload.e_app[a])
    p.tau = float(workload.tau)
    p.bjerrum = float(workload.bjerrum)
    p.nspecies = len(workload.z)
    for k in range(p.nspecies):
        p.z[k] = float(workload.z[k])
        p.D[k] = float(workload.D[k])
        p.rho_bulk[k] = float(workload.rho_bulk[k])
    p.flow = int(bool(workload.flow if flow is None else flow))
    p.precision = precision
    p.poisson_tol = tol
    p.poisson_max_iter = maxit
    p.boundary_rule = rule
    return p


class Lattice:
    """One LBE lattice on the GPU (owns an lbe handle)."""

    def __init__(self, params: lbe_params, stream: int | None = None):
        import torch
        self.p = params
        self.nx, self.ny, self.nz = params.nx, params.ny, params.nz
        self.N = self.nx * self.ny * self.nz
        self.ns = params.nspecies
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        self.h = lbe_create(params, stream)
        self.n_elec = 0

    @classmethod
    def from_workload(cls, w, **kw):
        lat = cls(params_for(w, **kw))
        lat.set_geometry(w.ids, w.n_elec)
        lat.set_voltage(w.psi)
        return lat

    def close(self):
        if getattr(self, "h", None):
            lbe_destroy(self.h)
            self.h = None

    __del__ = close

    def set_geometry(self, ids, n_electrodes: int):
        import torch
        if isinstance(ids, torch.Tensor):
            t = ids.contiguous().to(torch.uint8)
            assert t.numel() == self.N
            lbe_set_geometry(self.h, t.data_ptr(), n_electrodes, t.is_cuda)
        else:
            a = np.ascontiguousarray(np.asarray(ids).reshape(-1), dtype=np.uint8)
            assert a.size == self.N
            lbe_set_geometry(self.h, a.ctypes.data, n_electrodes, False)
        self.n_elec = n_electrodes

    def set_voltage(self, psi):
        lbe_set_voltage(self.h, [float(v) for v in psi])

    def init(self):
        lbe_init(self.h)

    def step(self, nsteps: int = 1):
        lbe_step(self.h, nsteps)

    def charge(self) -> np.ndarray:
        out = np.zeros(max(self.n_elec, 1))
        lbe_induced_charge(self.h, out.ctypes.data, False)
        return out[: self.n_elec]

    def charge_device(self, out):
        """Write the charges into a CUDA float64 tensor (stream-ordered)."""
        lbe_induced_charge(self.h, out.data_ptr(), True)
        return out

    def field(self, which: int, device: bool = False):
        import torch
        size = {FIELD_PHI: 1, FIELD_N: self.ns, FIELD_RHO: 1, FIELD_U: 3, FIELD_F: 19, FIELD_QNODE: 1}[which]
        shape = (self.nz, self.ny, self.nx) if size == 1 else (size, self.nz, self.ny, self.nx)
        if device:
            t = torch.empty(shape, dtype=torch.float64, device="cuda")
            lbe_fields(self.h, which, t.data_ptr(), True)
            return t
        out = np.zeros(shape)
        lbe_fields(self.h, which, out.ctypes.data, False)
        return out

    def phi(self):
        return self.field(FIELD_PHI)

    def n(self):
        return self.field(FIELD_N)

    def u(self):
        return self.field(FIELD_U)

    def rho(self):
        return self.field(FIELD_RHO)

    def populations(self):
        return self.field(FIELD_F)

    def charge_map(self):
        """Induced charge of every electrode node (0 on fluid nodes)."""
        return self.field(FIELD_QNODE)

    def set_state(self, n=None, phi=None):
        conv = lambda a: None if a is None else np.ascontiguousarray(np.asarray(a).reshape(-1), dtype=np.float64)
        n, phi = conv(n), conv(phi)
        lbe_set_state(self.h, n.ctypes.data if n is not None else None,
                      phi.ctypes.data if phi is not None else None, False)

    def save_state(self) -> bytes:
        size = ctypes.c_size_t(0)
        lbe_save_state(self.h, None, size)
        buf = ctypes.create_string_buffer(size.value)
        lbe_save_state(self.h, ctypes.addressof(buf), size)
        return buf.raw

    def load_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        lbe_load_state(self.h, ctypes.addressof(buf), len(blob))

    def stats(self) -> lbe_stats:
        return lbe_get_stats(self.h)

    def profile_begin(self):
        lbe_profile_begin(self.h)

    def profile_end(self) -> lbe_profile:
        return lbe_profile_end(self.h)

    def adjoint_forward(self, nsteps: int, every: int) -> np.ndarray:
        """lbe_init + nsteps steps with checkpoints; returns Q(T)."""
        q = np.zeros(max(self.n_elec, 1))
        lbe_adjoint_forward(self.h, nsteps, every, q.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return q[: self.n_elec]

    def adjoint_forward_budget(self, nsteps: int, device_bytes: int) -> np.ndarray:
        """lbe_init + nsteps steps with revolve checkpoints in device_bytes;
        returns Q(T)."""
        q = np.zeros(max(self.n_elec, 1))
        lbe_adjoint_forward_budget(self.h, nsteps, device_bytes, q.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return q[: self.n_elec]

    def adjoint_backward(self, dq, soft_electrode: int = 1, dchi=None):
        """Gradient of sum_e dq[e] Q_e(T); dchi: a CUDA float64 tensor of N
        values to receive the occupancy gradient (or None: returned as a host
        array)."""
        if dchi is None:
            out = np.zeros(self.N)
            g = lbe_adjoint_backward(self.h, dq, soft_electrode, out.ctypes.data, False)
            return g, out
        g = lbe_adjoint_backward(self.h, dq, soft_electrode, dchi.data_ptr(), True)
        return g, dchi


class Batch:
    """Many independent FP32 lattices advanced together (owns an lbe_batch)."""

    def __init__(self, workloads, *, tol=1e-12, maxit=100000, stream: int | None = None):
        import torch
        self.w = list(workloads)
        self.params = [params_for(w, precision=LBE_FP32, tol=tol, maxit=maxit) for w in self.w]
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        self.b = lbe_batch_create(self.params, stream)
        for i, w in enumerate(self.w):
            a = np.ascontiguousarray(np.asarray(w.ids).reshape(-1), dtype=np.uint8)
            lbe_batch_set_geometry(self.b, i, a.ctypes.data, w.n_elec)
            lbe_batch_set_voltage(self.b, i, [float(v) for v in w.psi])

    @property
    def n(self):
        return len(self.w)

    @property
    def nodes(self):
        return sum(w.nodes for w in self.w)

    def close(self):
        if getattr(self, "b", None):
            lbe_batch_destroy(self.b)
            self.b = None

    __del__ = close

    def init(self):
        lbe_batch_init(self.b)

    def step(self, nsteps: int = 1):
        lbe_batch_step(self.b, nsteps)

    def charge(self) -> np.ndarray:
        """[n, LBE_BATCH_MAX_ELECTRODES] induced charges (zero past n_elec)."""
        out = np.zeros((self.n, LBE_BATCH_MAX_ELECTRODES))
        lbe_batch_charge(self.b, out.ctypes.data, False)
        return out

    def charge_device(self, out):
        lbe_batch_charge(self.b, out.data_ptr(), True)
        return out

    def field(self, i: int, which: int) -> np.ndarray:
        nx, ny, nz = self.w[i].shape
        shape = (nz, ny, nx) if which == FIELD_PHI else (2, nz, ny, nx)
        out = np.zeros(shape)
        lbe_batch_fields(self.b, i, which, out.ctypes.data, False)
        return out

    def phi(self, i):
        return self.field(i, FIELD_PHI)

    def n_field(self, i):
        return self.field(i, FIELD_N)

    def stats(self) -> lbe_stats:
        return lbe_batch_get_stats(self.b)

    def tuning(self):
        return lbe_batch_tuning(self.b)

    def profile_begin(self):
        lbe_batch_profile_begin(self.b)

    def profile_end(self) -> lbe_profile:
        return lbe_batch_profile_end(self.b)
