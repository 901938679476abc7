"""Plain FP64 CPU model of the LBE time step with a soft electrode
occupancy, and its forward-mode tangent by dual numbers.

TEST INFRASTRUCTURE ONLY: used by the tests (and the script that writes the
stored tangents under ``tests/golden/``) to check the GPU adjoint.  It
shares no code with the CUDA library.

The paper's electrodes are binary: a node is fluid or belongs to an
electrode (Sec. "Imposing conducting boundary conditions").  Gradients with
respect to the electrode shape need a continuous occupancy.  Every node r
carries chi_r in [0, 1] and a label l(r), the electrode it joins at
chi_r = 1.  With j = r + c_i and w_i = 1/3 (nearest) or 1/6 (next nearest):

  Laplacian     L phi(r) = sum_i w_i (1 + (chi_r - chi_j)^2) (phi_j - phi_r)
  Poisson       (1 - chi_r) (L phi(r) + 4 pi l_B rho_el(r)) + chi_r (psi_l(r) - phi_r) = 0
  ion link      Eq. LF2 flux times the openness (1 - chi_r)(1 - chi_j)
  initial ions  n_k = rho_b (1 - chi)
  charge        Q_e = -eps sum_{r: l(r)=e} chi_r sum_i (1 - chi_j) w_i (1 + (chi_r - chi_j)^2) (phi_j - phi_r)

At chi in {0, 1} each line is the paper's rule: the factor 1 + (chi_r -
chi_j)^2 is the doubling of fluid-solid links of Eq.
DiscreteLaplacianModif, solid nodes hold their electrode potential, no ion
crosses a fluid-solid link, and the charge is Eq. Qelec over the links from
electrode e to fluid.  The solvent is at rest (no populations, no
advection), as in the porous-electrode workload.

One step (Sec. "Lattice Boltzmann Electrokinetics", solvent at rest):
n <- n - sum_i J_i(n, phi), then phi <- Poisson(n); phi at t = 0 solves the
Poisson equation of the initial ions.  Q is evaluated after the last step.

The Poisson equation is linear in phi with a matrix M that depends on chi
only; its tangent is phi' = M^-1 (b' - M' phi).  Small boxes (or a
non-binary chi) use a sparse LU factorisation (scipy); larger boxes at a
binary chi eliminate the solid rows (phi_s = psi) and solve the symmetric
positive definite fluid block by Jacobi-preconditioned conjugate gradients
(scipy) to a relative residual of 1e-13, warm-started from the previous
step.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

A0 = 1.0 + 2.0 * math.sqrt(2.0)

# the 18 non-rest D3Q19 velocities
C18 = np.array([(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
                (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1),
                (1, 0, -1), (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)])
LEN = np.sqrt((C18 ** 2).sum(axis=1)).astype(np.float64)   # |c_i|
W = np.where((C18 ** 2).sum(axis=1) == 1, 1.0 / 3.0, 1.0 / 6.0)


# --- dual numbers ------------------------------------------------------------
class Dual:
    """a + b eps with eps^2 = 0; value and derivative arrays (or floats)."""
    __array_priority__ = 1000

    def __init__(self, v, d):
        self.v, self.d = v, d

    def __add__(self, o):
        o = lift(o)
        return Dual(self.v + o.v, self.d + o.d)

    __radd__ = __add__

    def __sub__(self, o):
        o = lift(o)
        return Dual(self.v - o.v, self.d - o.d)

    def __rsub__(self, o):
        return lift(o) - self

    def __mul__(self, o):
        o = lift(o)
        return Dual(self.v * o.v, self.d * o.v + self.v * o.d)

    __rmul__ = __mul__

    def __truediv__(self, o):
        o = lift(o)
        return Dual(self.v / o.v, (self.d * o.v - self.v * o.d) / (o.v * o.v))

    def __rtruediv__(self, o):
        return lift(o) / self

    def __neg__(self):
        return Dual(-self.v, -self.d)

    def __getitem__(self, idx):
        return Dual(self.v[idx], self.d[idx])

    def sum(self, axis=None):
        return Dual(np.sum(self.v, axis=axis), np.sum(self.d, axis=axis))


def lift(x):
    return x if isinstance(x, Dual) else Dual(x, 0.0)


def val(x):
    return x.v if isinstance(x, Dual) else x


def dexp(x):
    if isinstance(x, Dual):
        e = np.exp(x.v)
        return Dual(e, e * x.d)
    return np.exp(x)


def dsum(x, axis=None):
    return x.sum(axis=axis) if isinstance(x, Dual) else np.sum(x, axis=axis)


# --- geometry ----------------------------------------------------------------
class Geometry:
    """Neighbour tables of an nx x ny x nz box (arrays indexed [z, y, x],
    flattened r = x + nx (y + ny z)); links leaving a non-periodic face do
    not exist."""

    def __init__(self, shape, periodic):
        nx, ny, nz = shape
        self.shape, self.N = (nx, ny, nz), nx * ny * nz
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        x, y, z = x.ravel(), y.ravel(), z.ravel()
        nb = np.empty((18, self.N), dtype=np.int64)
        exist = np.ones((18, self.N), dtype=bool)
        for i, (cx, cy, cz) in enumerate(C18):
            X, Y, Z = x + cx, y + cy, z + cz
            for V, n, p in ((X, nx, periodic[0]), (Y, ny, periodic[1]), (Z, nz, periodic[2])):
                if p:
                    V %= n
                else:
                    exist[i] &= (V >= 0) & (V < n)
            X, Y, Z = np.clip(X, 0, nx - 1), np.clip(Y, 0, ny - 1), np.clip(Z, 0, nz - 1)
            nb[i] = X + nx * (Y + ny * Z)
        self.nb = np.where(exist, nb, np.arange(self.N)[None, :])
        self.exist = exist.astype(np.float64)


# --- the soft model ----------------------------------------------------------
class SoftLBE:
    """Soft-occupancy LBE (1:1 salt, z = +1, -1) on one box.

    label: int array [z, y, x], the electrode (1..M) each node joins at
    chi = 1; bjerrum l_B; e_app the applied field (reduced units)."""

    def __init__(self, shape, periodic, label, bjerrum, e_app=(0.0, 0.0, 0.0)):
        self.g = Geometry(shape, periodic)
        self.label = np.asarray(label).reshape(-1).astype(np.int64)
        self.bjerrum = float(bjerrum)
        self.eps = 1.0 / (4.0 * math.pi * self.bjerrum)
        self.e_dot_c = C18 @ np.asarray(e_app, dtype=np.float64)   # (18,)
        self.z = (1.0, -1.0)

    # Poisson matrix pieces: coefficient of each link, value and derivative
    def _link_coef(self, chi):
        g = self.g
        chi_j = chi[g.nb] if not isinstance(chi, Dual) else chi[g.nb]
        diff = lift(chi)[None] - chi_j if isinstance(chi, Dual) else chi[None, :] - chi_j
        return (1.0 + diff * diff) * (W[:, None] * g.exist)       # (18, N)

    def _assemble(self, coef, chi, part):
        """Sparse matrix of the Poisson rows from coefficient arrays (part =
        'v' or 'd' selects value or derivative of dual inputs)."""
        g, N = self.g, self.g.N
        c = coef if not isinstance(coef, Dual) else getattr(coef, part)
        x = chi if not isinstance(chi, Dual) else getattr(chi, part)
        if part == "v":
            one_m = 1.0 - x
            diag = -one_m * c.sum(axis=0) - x
            off = one_m[None, :] * c
        else:
            cv = val(coef)
            xv = val(chi)
            diag = x * cv.sum(axis=0) - (1.0 - xv) * c.sum(axis=0) - x
            off = -x[None, :] * cv + (1.0 - xv)[None, :] * c
        rows = np.concatenate([np.arange(N), np.repeat(np.arange(N)[None, :], 18, axis=0).ravel()])
        cols = np.concatenate([np.arange(N), g.nb.ravel()])
        data = np.concatenate([diag, off.ravel()])
        return sp.csc_matrix((data, (rows, cols)), shape=(N, N))

    def _rhs(self, n, chi, psi):
        rho = n[0] - n[1]
        psi_l = psi[self.label - 1] if not isinstance(psi, Dual) else psi[self.label - 1]
        return -(1.0 - chi) * (4.0 * math.pi * self.bjerrum) * rho - chi * psi_l

    LU_MAX = 6000  # larger boxes at a binary occupancy use conjugate gradients

    def _factor(self, chi_v, Mv):
        binary = bool(np.all((chi_v == 0.0) | (chi_v == 1.0)))
        if self.g.N <= self.LU_MAX or not binary:
            return {"lu": spla.splu(Mv)}
        fl = chi_v == 0.0
        Mr = Mv.tocsr()
        A = (-Mr[fl][:, fl]).tocsr()
        return {"fl": fl, "A": A, "C": Mr[fl][:, ~fl].tocsr(),
                "P": sp.diags(1.0 / A.diagonal()), "warm": {}}

    def _lin(self, fac, b, key):
        if "lu" in fac:
            return fac["lu"].solve(b)
        fl = fac["fl"]
        x = np.empty_like(b)
        xs = -b[~fl]
        x[~fl] = xs
        rhs = fac["C"] @ xs - b[fl]
        x0 = fac["warm"].get(key)
        xf, info = spla.cg(fac["A"], rhs, x0=x0, rtol=1e-13, atol=0.0, M=fac["P"], maxiter=50000)
        if info != 0:
            raise RuntimeError("soft oracle: CG did not converge")
        fac["warm"][key] = xf
        x[fl] = xf
        return x

    def _solve(self, fac, Md, rhs, dual):
        if not dual:
            return self._lin(fac, np.asarray(rhs, dtype=np.float64) * np.ones(self.g.N), "v")
        rhs = lift(rhs)
        pv = self._lin(fac, np.asarray(rhs.v, dtype=np.float64) * np.ones(self.g.N), "v")
        rd = np.asarray(rhs.d, dtype=np.float64) * np.ones(self.g.N)
        if Md is not None:
            rd = rd - Md @ pv
        return Dual(pv, self._lin(fac, rd, "d"))

    def _flux_step(self, n, phi, chi, d):
        g = self.g
        chi_j = chi[g.nb]
        open_ = (1.0 - lift(chi)[None] if isinstance(chi, Dual) else 1.0 - chi[None, :]) * (1.0 - chi_j) * g.exist
        phi_j = phi[g.nb]
        dphi = phi_j - (lift(phi)[None] if isinstance(phi, Dual) else phi[None, :])
        out = []
        for k in range(2):
            nk = n[k]
            nk_j = nk[g.nb]
            dmu = self.z[k] * (dphi - self.e_dot_c[:, None])
            avg = 0.5 * (1.0 + dexp(-dmu))
            nk_r = lift(nk)[None] if isinstance(nk, Dual) else nk[None, :]
            J = open_ * (-(d[k] / LEN[:, None]) * avg * (nk_j * dexp(dmu) - nk_r))
            out.append(nk - dsum(J, axis=0))
        return out

    def charge(self, phi, chi, n_elec):
        g = self.g
        chi_j = chi[g.nb]
        chi_r = lift(chi)[None] if isinstance(chi, Dual) else chi[None, :]
        phi_r = lift(phi)[None] if isinstance(phi, Dual) else phi[None, :]
        diff = chi_r - chi_j
        s = dsum((1.0 - chi_j) * (W[:, None] * g.exist) * (1.0 + diff * diff) * (phi[g.nb] - phi_r), axis=0)
        per = -self.eps * (chi * s)
        q = []
        for e in range(1, n_elec + 1):
            sel = self.label == e
            q.append(dsum(per[sel]))
        return q

    def run(self, psi, debye, D, chi, steps, trace=False):
        """Q_e after `steps` steps.  Any of psi (array), debye (float), D
        (pair), chi (array N) may be Dual: the result then carries the
        directional derivative."""
        dual = any(isinstance(a, Dual) for a in (psi, debye, D, chi))
        n_elec = int(self.label.max())
        rho_b = 1.0 / (8.0 * math.pi * self.bjerrum * (debye * debye))
        d = [D[0] / A0, D[1] / A0] if not isinstance(D, Dual) else [D[0] / A0, D[1] / A0]
        coef = self._link_coef(chi)
        lu = self._factor(val(chi), self._assemble(coef, chi, "v"))
        Md = self._assemble(coef, chi, "d") if isinstance(chi, Dual) else None
        n0 = rho_b * (1.0 - chi)
        n = [n0, n0]
        phi = self._solve(lu, Md, self._rhs(n, chi, psi), dual)
        qs = [self.charge(phi, chi, n_elec)] if trace else None
        for _ in range(steps):
            n = self._flux_step(n, phi, chi, d)
            phi = self._solve(lu, Md, self._rhs(n, chi, psi), dual)
            if trace:
                qs.append(self.charge(phi, chi, n_elec))
        q = self.charge(phi, chi, n_elec)
        return (q, qs) if trace else q, (n, phi)

    def tangent(self, psi, debye, D, chi, steps, dpsi=None, ddebye=0.0, dD=None, dchi=None):
        """(Q, dQ) along the direction (dpsi, ddebye, dD, dchi)."""
        M = int(self.label.max())
        dpsi = np.zeros(M) if dpsi is None else np.asarray(dpsi, dtype=np.float64)
        dD = np.zeros(2) if dD is None else np.asarray(dD, dtype=np.float64)
        dchi = np.zeros(self.g.N) if dchi is None else np.asarray(dchi, dtype=np.float64)
        q, _ = self.run(Dual(np.asarray(psi, dtype=np.float64), dpsi), Dual(float(debye), float(ddebye)),
                        Dual(np.asarray(D, dtype=np.float64), dD), Dual(np.asarray(chi, dtype=np.float64), dchi),
                        steps)
        return np.array([lift(x).v for x in q], dtype=np.float64), np.array([lift(x).d for x in q],
                                                                            dtype=np.float64)

    def forward(self, psi, debye, D, chi, steps):
        q, state = self.run(np.asarray(psi, dtype=np.float64), float(debye), np.asarray(D, dtype=np.float64),
                            np.asarray(chi, dtype=np.float64), steps)
        return np.array(q, dtype=np.float64), state


def from_ids(ids, soft_electrode=1):
    """Binary occupancy and labels from a node-id array (0 fluid, e >= 1
    electrode e); fluid nodes are labelled with the soft electrode."""
    ids = np.asarray(ids)
    chi = (ids != 0).astype(np.float64).reshape(-1)
    label = np.where(ids != 0, ids, soft_electrode).astype(np.int64)
    return chi, label
