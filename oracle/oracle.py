"""ctypes wrapper around the plain C FP64 oracle (``lbe_oracle.c``).

TEST INFRASTRUCTURE ONLY: used by the tests, by ``__graft_entry__.smoke()``
to check the CUDA path, and by the CPU-baseline leg of ``bench.py``.  It
shares no code with the CUDA library.

Conventions (lattice units, k_B T = e = 1): node index
``r = x + nx*(y + ny*z)``; species arrays are ``[k][r]``; vector fields are
``[a][r]``; geometry ``id[r]`` is 0 for fluid and ``e >= 1`` for electrode
``e``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbe_oracle.c")
_LIB = os.path.join(_HERE, "liblbe_oracle.so")
_lib = None

PHI, N_K, RHO, U, F = 0, 1, 2, 3, 4


def library_path() -> str:
    return _LIB


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, FP64, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-D_GNU_SOURCE", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    vp = ctypes.c_void_p
    lib.orc_create.restype = vp
    lib.orc_create.argtypes = [ctypes.c_int] * 3 + [ip, ctypes.c_double, ctypes.c_double,
                                                     ctypes.c_int, dp, dp, dp, dp,
                                                     ctypes.c_int, ctypes.c_double, ctypes.c_int]
    lib.orc_destroy.argtypes = [vp]
    lib.orc_set_geometry.argtypes = [vp, ctypes.POINTER(ctypes.c_uint8), ctypes.c_int]
    lib.orc_set_voltage.argtypes = [vp, dp]
    lib.orc_init.argtypes = [vp]
    lib.orc_step.argtypes = [vp, ctypes.c_int]
    lib.orc_charge.argtypes = [vp, dp]
    lib.orc_fields.argtypes = [vp, ctypes.c_int, dp]
    lib.orc_laplacian.argtypes = [vp, dp, dp]
    lib.orc_poisson.argtypes = [vp, dp]
    lib.orc_set_state.argtypes = [vp, dp, dp, dp]
    lib.orc_set_body_force.argtypes = [vp, dp]
    lib.orc_set_boundary_rule.argtypes = [vp, ctypes.c_int]
    lib.orc_force.argtypes = [vp, dp]
    lib.orc_advect.argtypes = [vp, dp, dp, dp]
    lib.orc_last_iters.argtypes = [vp]
    lib.orc_last_res.argtypes = [vp]
    lib.orc_last_res.restype = ctypes.c_double
    lib.orc_link_flux.restype = ctypes.c_double
    lib.orc_link_flux.argtypes = [ctypes.c_double] * 8
    _lib = lib
    return lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def link_flux(d, delta_len, zk, phi0, phi1, e_dot_c, n0, n1) -> float:
    """Single-link flux of Eq. LF2 (see ``lbe_oracle.c``)."""
    return _load().orc_link_flux(d, delta_len, zk, phi0, phi1, e_dot_c, n0, n1)


class Oracle:
    """One LBE lattice on the CPU in FP64."""

    def __init__(self, shape, periodic, *, tau=1.0, bjerrum=1.0, z=(1.0, -1.0),
                 D=(0.05, 0.05), rho_bulk=(0.01, 0.01), e_app=(0.0, 0.0, 0.0), flow=True,
                 tol=1e-14, maxit=200000):
        lib = _load()
        self.lib = lib
        self.nx, self.ny, self.nz = (int(s) for s in shape)
        self.N = self.nx * self.ny * self.nz
        self.ns = len(z)
        per = (ctypes.c_int * 3)(*[int(bool(p)) for p in periodic])
        arr = lambda v: np.ascontiguousarray(np.asarray(v, dtype=np.float64))
        self._z, self._D, self._rb, self._e = arr(z), arr(D), arr(rho_bulk), arr(e_app)
        self.h = lib.orc_create(self.nx, self.ny, self.nz, per, float(tau), float(bjerrum),
                                self.ns, _dp(self._z), _dp(self._D), _dp(self._rb),
                                _dp(self._e), int(bool(flow)), float(tol), int(maxit))
        if not self.h:
            raise ValueError("oracle: bad parameters")
        self.n_elec = 0

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.orc_destroy(h)
            self.h = None

    # -- set-up ---------------------------------------------------------
    def set_geometry(self, node_id: np.ndarray, n_electrodes: int):
        ids = np.ascontiguousarray(node_id.reshape(-1), dtype=np.uint8)
        assert ids.size == self.N
        rc = self.lib.orc_set_geometry(self.h, ids.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                       int(n_electrodes))
        if rc:
            raise ValueError(f"oracle: set_geometry rc={rc}")
        self.n_elec = int(n_electrodes)

    def set_voltage(self, psi):
        p = np.ascontiguousarray(np.asarray(psi, dtype=np.float64))
        assert p.size == self.n_elec
        self.lib.orc_set_voltage(self.h, _dp(p))

    def init(self):
        rc = self.lib.orc_init(self.h)
        if rc:
            raise RuntimeError(f"oracle: init rc={rc}")

    def step(self, nsteps=1):
        rc = self.lib.orc_step(self.h, int(nsteps))
        if rc:
            raise RuntimeError(f"oracle: step rc={rc}")

    # -- observables ----------------------------------------------------
    def charge(self) -> np.ndarray:
        q = np.zeros(max(self.n_elec, 1))
        self.lib.orc_charge(self.h, _dp(q))
        return q[: self.n_elec]

    def field(self, which: int) -> np.ndarray:
        size = {PHI: 1, N_K: self.ns, RHO: 1, U: 3, F: 19}[which]
        out = np.zeros(size * self.N)
        rc = self.lib.orc_fields(self.h, which, _dp(out))
        if rc:
            raise RuntimeError("oracle: fields")
        shape = (self.nz, self.ny, self.nx)
        return out.reshape(shape) if size == 1 else out.reshape((size,) + shape)

    def phi(self):
        return self.field(PHI)

    def n(self):
        return self.field(N_K)

    def u(self):
        return self.field(U)

    def rho(self):
        return self.field(RHO)

    def populations(self):
        return self.field(F)

    # -- pieces used by the pins ----------------------------------------
    def laplacian(self, phi: np.ndarray) -> np.ndarray:
        p = np.ascontiguousarray(phi.reshape(-1), dtype=np.float64)
        out = np.zeros(self.N)
        self.lib.orc_laplacian(self.h, _dp(p), _dp(out))
        return out.reshape(self.nz, self.ny, self.nx)

    def poisson(self, rho_el: np.ndarray) -> int:
        r = np.ascontiguousarray(rho_el.reshape(-1), dtype=np.float64)
        return self.lib.orc_poisson(self.h, _dp(r))

    def set_state(self, f=None, n=None, phi=None):
        conv = lambda a: None if a is None else np.ascontiguousarray(a.reshape(-1), dtype=np.float64)
        f, n, phi = conv(f), conv(n), conv(phi)
        nul = ctypes.POINTER(ctypes.c_double)()
        self.lib.orc_set_state(self.h, _dp(f) if f is not None else nul,
                               _dp(n) if n is not None else nul,
                               _dp(phi) if phi is not None else nul)

    def set_boundary_rule(self, node_rule: int):
        """0: the paper's rule (Eq. DiscreteLaplacianModif, the default); 1:
        the first-order rule it replaces (plain Laplacian, solid nodes held
        at their potential).  Call before init()."""
        self.lib.orc_set_boundary_rule(self.h, int(node_rule))

    def set_body_force(self, g):
        """Uniform external body force density on the solvent (3 values),
        added to the ion force; zero unless set."""
        self._g = np.ascontiguousarray(np.asarray(g, dtype=np.float64))
        assert self._g.size == 3
        self.lib.orc_set_body_force(self.h, _dp(self._g))

    def force(self) -> np.ndarray:
        out = np.zeros(3 * self.N)
        self.lib.orc_force(self.h, _dp(out))
        return out.reshape(3, self.nz, self.ny, self.nx)

    def advect(self, n: np.ndarray, u: np.ndarray) -> np.ndarray:
        a = np.ascontiguousarray(n.reshape(-1), dtype=np.float64)
        b = np.ascontiguousarray(u.reshape(-1), dtype=np.float64)
        out = np.zeros_like(a)
        self.lib.orc_advect(self.h, _dp(a), _dp(b), _dp(out))
        return out.reshape(n.shape)

    @property
    def last_iters(self) -> int:
        return self.lib.orc_last_iters(self.h)

    @property
    def last_res(self) -> float:
        return self.lib.orc_last_res(self.h)
