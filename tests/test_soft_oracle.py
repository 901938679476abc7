"""Pins of the soft-occupancy oracle (oracle/soft.py) and of its dual-number
tangent, the reference for the GPU adjoint.

* At a binary occupancy the soft model is the method: its trajectory equals
  the C oracle's (solvent at rest) to the Poisson tolerance.
* The tangent equals central finite differences of the soft forward model
  for every parameter kind (voltage, Debye length, both diffusivities,
  occupancy of fluid, interface and buried nodes).
* Exact identities: a common shift of all electrode potentials changes
  nothing; at t = 0 the charge does not depend on the bulk concentration
  (the initial ions are neutral everywhere); the total induced charge is
  minus the (conserved, zero) ionic charge, so its derivative with respect
  to voltages and diffusivities vanishes.
"""
import math

import numpy as np
import pytest

from oracle import Oracle
from oracle.soft import SoftLBE, from_ids
from paper_1907_04732_gb300 import workloads as wl


def small_case():
    ids = wl.porous(10, 9, 12, 2, 1.5, 2.5, 5.0, seed=11)
    return ids, (1, 1, 0)


def test_soft_model_is_the_method_at_binary_occupancy():
    ids, per = small_case()
    chi, label = from_ids(ids)
    psi, debye, D = (0.0, 0.15), 3.0, (0.05, 0.08)
    bj = 1.44
    m = SoftLBE(ids.shape[::-1], per, label.reshape(ids.shape), bj, e_app=(1e-3, 0.0, 0.0))
    steps = 40
    q, (n, phi) = m.forward(psi, debye, D, chi, steps)
    rb = wl.bulk_density(debye, bj)
    o = Oracle(ids.shape[::-1], per, tau=1.0, bjerrum=bj, z=(1.0, -1.0), D=D, rho_bulk=(rb, rb),
               e_app=(1e-3, 0.0, 0.0), flow=False, tol=1e-14)
    o.set_geometry(ids, 2)
    o.set_voltage(psi)
    o.init()
    o.step(steps)
    np.testing.assert_allclose(q, o.charge(), rtol=1e-9, atol=1e-15)
    np.testing.assert_allclose(phi.reshape(ids.shape), o.phi(), rtol=0, atol=1e-11)
    np.testing.assert_allclose(np.stack(n).reshape((2,) + ids.shape), o.n(), rtol=0, atol=1e-12 * rb)


def central_fd(m, base, steps, which, idx=None, h=1e-4):
    def q_at(sign):
        psi, debye, D, chi = [np.array(a, dtype=np.float64) if np.ndim(a) else float(a) for a in base]
        if which == "psi":
            psi[idx] += sign * h
        elif which == "debye":
            debye += sign * h
        elif which == "D":
            D[idx] += sign * h
        else:
            chi[idx] += sign * h
        return m.forward(psi, debye, D, chi, steps)[0]
    return (q_at(+1) - q_at(-1)) / (2 * h)


def test_tangent_matches_central_differences():
    ids, per = small_case()
    chi, label = from_ids(ids)
    m = SoftLBE(ids.shape[::-1], per, label.reshape(ids.shape), 1.44, e_app=(1e-3, 0.0, 0.0))
    base = ((0.0, 0.15), 3.0, (0.05, 0.08), chi)
    steps = 25
    N = chi.size
    flat = ids.reshape(-1)
    # a fluid node next to the porous electrode, a solid interface node, a
    # fluid node far from any electrode
    nbr_solid = np.zeros(N, dtype=bool)
    for s in (-1, 1):
        for ax in range(3):
            nbr_solid |= (np.roll(ids, s, axis=ax) != 0).reshape(-1)
    near = int(np.flatnonzero((flat == 0) & nbr_solid)[3])
    iface = int(np.flatnonzero((flat == 1) & (np.roll(ids, -1, axis=0).reshape(-1) == 0))[2])
    far = int(np.flatnonzero((flat == 0) & ~nbr_solid)[0])
    cases = [("psi", 1, {"dpsi": [0.0, 1.0]}), ("debye", None, {"ddebye": 1.0}),
             ("D", 0, {"dD": [1.0, 0.0]}), ("D", 1, {"dD": [0.0, 1.0]})]
    for node in (near, iface, far):
        e = np.zeros(N)
        e[node] = 1.0
        cases.append(("chi", node, {"dchi": e}))
    for which, idx, kw in cases:
        q, dq = m.tangent(*base, steps, **kw)
        fd = central_fd(m, base, steps, which, idx)
        scale = np.abs(fd).max() + 1e-12
        assert np.abs(dq - fd).max() <= 1e-6 * scale + 1e-13, (which, idx, dq, fd)


def test_tangent_identities():
    ids, per = small_case()
    chi, label = from_ids(ids)
    m = SoftLBE(ids.shape[::-1], per, label.reshape(ids.shape), 1.44)
    base = ((0.05, 0.2), 3.0, (0.05, 0.05), chi)
    # common potential shift
    _, dq = m.tangent(*base, 15, dpsi=[1.0, 1.0])
    assert np.abs(dq).max() < 1e-12
    # t = 0: no dependence on the bulk concentration
    _, dq = m.tangent(*base, 0, ddebye=1.0)
    assert np.abs(dq).max() < 1e-13
    # total charge: d(Q1 + Q2) = 0 for voltages and diffusivities
    for kw in ({"dpsi": [0.0, 1.0]}, {"dD": [1.0, -0.5]}):
        q, dq = m.tangent(*base, 15, **kw)
        assert abs(q.sum()) < 1e-12 * np.abs(q).max() + 1e-14
        assert abs(dq.sum()) < 1e-9 * np.abs(dq).max() + 1e-14, (kw, dq)
