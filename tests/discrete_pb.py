"""Steady state of a plate column from the equations of the method (test
helper, CPU, numpy).

On a 1 x 1 x (L+2) column with the solvent at rest and no applied field, the
link fluxes of Eq. LF2 vanish exactly when each species follows a Boltzmann
distribution n_k = A_k exp(-z_k phi) (Sec. "Lattice Boltzmann
Electrokinetics").  The steady state is then the discrete nonlinear
Poisson-Boltzmann problem

    lap(phi)(z) + 4 pi l_B sum_k z_k A_k exp(-z_k phi(z)) = 0,  z = 1..L,

with the stencil of Eq. DiscreteLaplacianModif reduced to the column (the
D3Q19 links of one side sum to the weight 1; the link to an electrode is
doubled) and the prefactors A_k fixed by the solute amounts (the method
conserves them: rho_k L from a uniform start).  Solved here by Newton's method
with the constraints eliminated.
"""
import math

import numpy as np


def plate_column_steady(L, psi1, psi2, bjerrum, rho_bulk, z=(1.0, -1.0), tol=1e-15, maxit=100):
    """phi (L fluid nodes) and n (len(z) x L) of the steady column."""
    z = np.asarray(z, dtype=float)
    rho = np.broadcast_to(np.asarray(rho_bulk, dtype=float), z.shape)
    c = 4.0 * math.pi * bjerrum
    # start from the Laplace profile through psi at the mid-planes
    zz = np.arange(1, L + 1, dtype=float)
    phi = psi1 + (psi2 - psi1) * (zz - 0.5) / L
    for _ in range(maxit):
        lap = np.empty(L)
        lap[1:-1] = phi[2:] - 2 * phi[1:-1] + phi[:-2]
        lap[0] = 2 * (psi1 - phi[0]) + (phi[1] - phi[0])
        lap[-1] = (phi[-2] - phi[-1]) + 2 * (psi2 - phi[-1])
        Jl = np.diag(np.full(L, -2.0)) + np.diag(np.ones(L - 1), 1) + np.diag(np.ones(L - 1), -1)
        Jl[0, 0] = Jl[-1, -1] = -3.0
        F = lap.copy()
        J = Jl.copy()
        for k in range(len(z)):
            e = np.exp(-z[k] * phi)
            S = e.sum()
            A = rho[k] * L / S
            F += c * z[k] * A * e
            # d(A e_i)/dphi_j = -z A e_i delta_ij + z A e_i e_j / S
            J += c * z[k] * (np.diag(-z[k] * A * e) + z[k] * A * np.outer(e, e) / S)
        dphi = np.linalg.solve(J, -F)
        phi = phi + dphi
        if np.abs(dphi).max() < tol:
            break
    n = np.stack([rho[k] * L * np.exp(-z[k] * phi) / np.exp(-z[k] * phi).sum() for k in range(len(z))])
    return phi, n
