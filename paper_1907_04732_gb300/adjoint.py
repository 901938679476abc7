"""Gradients of the induced electrode charge after T steps, through the
library's hand-written adjoint of the LBE step (``lbe_adjoint_forward`` /
``lbe_adjoint_backward`` in include/lbe.h), as a torch.autograd.Function.

    spec = ChargeSpec.from_workload(w, steps=2000, every=100)
    q = induced_charge(psi, debye, D, chi, spec)      # Q_e(T), float64
    q[0].backward()                                    # psi.grad, debye.grad, D.grad, chi.grad

The solvent is at rest (the ions and the potential evolve; Sec. "Lattice
Boltzmann Electrokinetics" with the flow switched off, as in the
porous-electrode workload).  ``chi`` is the occupancy of the soft electrode
on every node: it must be 0 or 1 (the gradient is taken at that binary
geometry; include/lbe.h states the continuous reading it differentiates).
Nodes of the other electrodes come from ``spec.fixed_ids`` and must have
chi = 1.  The Debye length enters through the bulk concentration
rho_b = 1/(8 pi l_B lambda_D^2).

Only argument marshalling happens here; the forward steps, the
checkpointing and every backward step run in the CUDA library.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import lbe


@dataclass
class ChargeSpec:
    shape: tuple            # (nx, ny, nz)
    periodic: tuple
    fixed_ids: np.ndarray   # [z, y, x]: electrodes not described by chi (0 elsewhere)
    n_elec: int
    soft_electrode: int
    bjerrum: float
    steps: int
    every: int = 100
    tol: float = 1e-12
    e_app: tuple = (0.0, 0.0, 0.0)
    tau: float = 1.0
    extra: dict = field(default_factory=dict)

    @classmethod
    def from_workload(cls, w, *, steps=None, every=100, soft_electrode=1, tol=1e-12):
        fixed = np.where((w.ids != 0) & (w.ids != soft_electrode), w.ids, 0).astype(np.uint8)
        return cls(w.shape, tuple(w.periodic), fixed, w.n_elec, soft_electrode, w.bjerrum,
                   w.steps if steps is None else steps, every, tol, tuple(w.e_app), w.tau)

    def ids_for(self, chi: np.ndarray) -> np.ndarray:
        nx, ny, nz = self.shape
        c = np.asarray(chi, dtype=np.float64).reshape(nz, ny, nx)
        if not np.all((c == 0.0) | (c == 1.0)):
            raise ValueError("occupancy must be 0 or 1 (the gradient is taken at the binary geometry)")
        if np.any((self.fixed_ids != 0) & (c != 1.0)):
            raise ValueError("nodes of the fixed electrodes need chi = 1")
        ids = np.where(self.fixed_ids != 0, self.fixed_ids, np.where(c == 1.0, self.soft_electrode, 0))
        return ids.astype(np.uint8)


def _lattice(spec: ChargeSpec, psi, debye: float, D):
    rho_b = 1.0 / (8.0 * math.pi * spec.bjerrum * debye * debye)
    p = lbe.lbe_default_params()
    p.nx, p.ny, p.nz = spec.shape
    for a in range(3):
        p.periodic[a] = int(bool(spec.periodic[a]))
        p.e_app[a] = float(spec.e_app[a])
    p.tau = float(spec.tau)
    p.bjerrum = float(spec.bjerrum)
    p.nspecies = 2
    p.z[0], p.z[1] = 1.0, -1.0
    p.D[0], p.D[1] = float(D[0]), float(D[1])
    p.rho_bulk[0] = p.rho_bulk[1] = rho_b
    p.flow = 0
    p.precision = lbe.LBE_FP32
    p.poisson_tol = spec.tol
    p.poisson_max_iter = 100000
    return lbe.Lattice(p), rho_b


def _torch():
    import torch
    return torch


def _function_class():
    torch = _torch()

    class ChargeAfterSteps(torch.autograd.Function):
        """(psi, debye, D, chi) -> Q_e after spec.steps steps."""

        @staticmethod
        def forward(ctx, psi, debye, D, chi, spec):
            psi_h = psi.detach().cpu().double().numpy()
            D_h = D.detach().cpu().double().numpy()
            lam_d = float(debye.detach().cpu())
            ids = spec.ids_for(chi.detach().cpu().numpy())
            lat, rho_b = _lattice(spec, psi_h, lam_d, D_h)
            lat.set_geometry(ids, spec.n_elec)
            lat.set_voltage(psi_h)
            q = lat.adjoint_forward(spec.steps, spec.every)
            ctx.lat, ctx.spec, ctx.rho_b, ctx.lam_d = lat, spec, rho_b, lam_d
            ctx.chi_meta = (chi.shape, chi.device, chi.dtype)
            return torch.as_tensor(q, dtype=torch.float64, device=psi.device)

        @staticmethod
        def backward(ctx, gq):
            spec = ctx.spec
            g, dchi = ctx.lat.adjoint_backward(gq.detach().cpu().double().numpy(), spec.soft_electrode)
            shape, device, dtype = ctx.chi_meta
            dpsi = torch.tensor(list(g.dpsi)[: spec.n_elec], dtype=torch.float64)
            ddebye = torch.tensor(g.drho_bulk * (-2.0 * ctx.rho_b / ctx.lam_d), dtype=torch.float64)
            dD = torch.tensor(list(g.dD)[:2], dtype=torch.float64)
            dchi_t = torch.as_tensor(dchi, dtype=dtype).reshape(shape).to(device)
            ctx.stats = g
            return dpsi.to(gq.device), ddebye.to(gq.device), dD.to(gq.device), dchi_t, None

    return ChargeAfterSteps


_FN = None


def induced_charge(psi, debye, D, chi, spec: ChargeSpec):
    """Q_e(T) as a differentiable function of the electrode potentials psi
    (n_elec), the Debye length (scalar tensor), the diffusivities D (2) and
    the occupancy chi of the soft electrode (N values, 0 or 1)."""
    global _FN
    if _FN is None:
        _FN = _function_class()
    return _FN.apply(psi, debye, D, chi, spec)
