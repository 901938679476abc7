"""Hand-written adjoint of the LBE step with the solvent at rest (FP32
forward and backward, checkpointing) against the FP64 soft-occupancy
oracle's dual-number tangent, against central differences of the GPU
forward pass itself, and for independence of the checkpoint interval.

Tolerances: the forward pass is the FP32 form (potential within 1e-6 of
the voltage); the backward pass keeps the ion adjoint in FP32 and sums the
parameter gradients in FP64.  Gradients agree with the FP64 tangent to
2e-4 of the largest gradient of each kind (voltage, Debye length,
diffusivity, occupancy).
"""
import math

import numpy as np
import pytest

from paper_1907_04732_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 2e-4


def crop_case(nx=14, ny=12, nz=14, seed=11):
    ids = wl.porous(nx, ny, nz, 2, 1.5, 2.5, 6.0, seed=seed)
    w = wl.Workload("crop", ids, 2, (1, 1, 0), (0.0, 0.12), 1.44, 3.0, D=(0.05, 0.08),
                    e_app=(1e-3, 0.0, 0.0), flow=False)
    return w


def gpu_grad(lbe, w, steps, every, dq, soft=1):
    from paper_1907_04732_gb300 import adjoint
    spec = adjoint.ChargeSpec.from_workload(w, steps=steps, every=every)
    rho_b = w.rho_bulk[0]
    lat, _ = adjoint._lattice(spec, w.psi, w.debye, w.D)
    lat.set_geometry(w.ids, w.n_elec)
    lat.set_voltage(w.psi)
    q = lat.adjoint_forward(steps, every)
    g, dchi = lat.adjoint_backward(dq, soft)
    ddebye = g.drho_bulk * (-2.0 * rho_b / w.debye)
    return q, np.array(g.dpsi[:w.n_elec]), ddebye, np.array(g.dD[:2]), dchi, g, lat


def oracle_model(w):
    from oracle.soft import SoftLBE, from_ids
    chi, label = from_ids(w.ids)
    m = SoftLBE(w.shape, w.periodic, label.reshape(w.ids.shape), w.bjerrum, e_app=w.e_app)
    return m, chi


def test_adjoint_matches_oracle_tangent(lbe):
    w = crop_case()
    steps, every = 60, 16
    dq = np.array([1.0, 0.3])
    q, dpsi, ddebye, dD, dchi, g, _ = gpu_grad(lbe, w, steps, every, dq)
    m, chi = oracle_model(w)
    base = (w.psi, w.debye, w.D, chi)
    q_o, _ = m.forward(*base, steps)
    assert np.abs(q - q_o).max() <= 1e-5 * np.abs(q_o).max()

    def tan(**kw):
        return float(np.dot(dq, m.tangent(*base, steps, **kw)[1]))

    t_psi = np.array([tan(dpsi=[1.0, 0.0]), tan(dpsi=[0.0, 1.0])])
    assert np.abs(dpsi - t_psi).max() <= TOL * np.abs(t_psi).max(), (dpsi, t_psi)
    t_deb = tan(ddebye=1.0)
    assert abs(ddebye - t_deb) <= TOL * abs(t_deb), (ddebye, t_deb)
    t_D = np.array([tan(dD=[1.0, 0.0]), tan(dD=[0.0, 1.0])])
    assert np.abs(dD - t_D).max() <= TOL * np.abs(t_D).max(), (dD, t_D)
    # occupancy: a seeded dense direction and single nodes of each kind
    rng = np.random.Generator(np.random.PCG64(wl.SEED))
    v = rng.standard_normal(chi.size)
    t_v = tan(dchi=v)
    scale = np.abs(dchi).max() * np.sqrt(chi.size)
    assert abs(float(np.dot(dchi, v)) - t_v) <= TOL * scale, (np.dot(dchi, v), t_v)
    flat = w.ids.reshape(-1)
    near_solid = np.zeros(chi.size, dtype=bool)
    for s in (-1, 1):
        for ax in range(3):
            near_solid |= (np.roll(w.ids, s, axis=ax) != 0).reshape(-1)
    nodes = [int(np.flatnonzero((flat == 0) & near_solid)[5]),
             int(np.flatnonzero((flat == 1) & near_solid & (np.roll(w.ids, -1, 0).reshape(-1) == 0))[1]),
             int(np.flatnonzero((flat == 0) & ~near_solid)[7])]
    for r in nodes:
        e = np.zeros(chi.size)
        e[r] = 1.0
        t_r = tan(dchi=e)
        assert abs(dchi[r] - t_r) <= TOL * np.abs(dchi).max(), (r, dchi[r], t_r)
    assert g.recomputed_steps == steps - math.ceil(steps / every)


def test_adjoint_checkpoint_interval_does_not_matter(lbe):
    w = crop_case(12, 12, 12, seed=3)
    dq = np.array([0.0, 1.0])
    a = gpu_grad(lbe, w, 40, 7, dq)
    b = gpu_grad(lbe, w, 40, 40, dq)
    for x, y in zip(a[:5], b[:5]):
        np.testing.assert_array_equal(x, y)


def test_adjoint_vs_gpu_central_differences(lbe):
    w = crop_case(12, 12, 12, seed=5)
    steps = 40
    dq = np.array([1.0, 0.0])
    q, dpsi, ddebye, dD, dchi, g, _ = gpu_grad(lbe, w, steps, 10, dq)

    def q_at(**kw):
        return float(np.dot(dq, gpu_grad(lbe, w.with_(**kw), steps, 10, dq)[0]))

    h = 1e-3
    fd_psi = (q_at(psi=(0.0, w.psi[1] + h)) - q_at(psi=(0.0, w.psi[1] - h))) / (2 * h)
    assert abs(dpsi[1] - fd_psi) <= 1e-3 * abs(fd_psi)
    hD = 1e-3 * w.D[0]
    fd_D = (q_at(D=(w.D[0] + hD, w.D[1])) - q_at(D=(w.D[0] - hD, w.D[1]))) / (2 * hD)
    assert abs(dD[0] - fd_D) <= 2e-3 * abs(fd_D) + 1e-9


def test_autograd_function(lbe):
    import torch
    from paper_1907_04732_gb300 import adjoint
    w = crop_case(12, 12, 12, seed=5)
    spec = adjoint.ChargeSpec.from_workload(w, steps=30, every=8)
    psi = torch.tensor(w.psi, dtype=torch.float64, requires_grad=True)
    debye = torch.tensor(w.debye, dtype=torch.float64, requires_grad=True)
    D = torch.tensor(w.D, dtype=torch.float64, requires_grad=True)
    chi = torch.tensor((w.ids != 0).astype(np.float64).reshape(-1), requires_grad=True)
    q = adjoint.induced_charge(psi, debye, D, chi, spec)
    (0.7 * q[0] - q[1]).backward()
    ref = gpu_grad(lbe, w, 30, 8, np.array([0.7, -1.0]))
    np.testing.assert_allclose(psi.grad.numpy(), ref[1], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(float(debye.grad), ref[2], rtol=1e-12)
    np.testing.assert_allclose(D.grad.numpy(), ref[3], rtol=1e-12)
    np.testing.assert_allclose(chi.grad.numpy(), ref[4], rtol=1e-12, atol=1e-18)
    with pytest.raises(ValueError):
        adjoint.induced_charge(psi, debye, D, chi * 0.5, spec)


def test_adjoint_errors(lbe):
    w = crop_case(10, 10, 10, seed=2)
    g = lbe.Lattice.from_workload(w.with_(flow=True), precision=lbe.LBE_FP32)
    with pytest.raises(lbe.LBEError) as e:
        g.adjoint_forward(5, 2)
    assert e.value.code == lbe.LBE_ERR_STATE
    g = lbe.Lattice.from_workload(w, precision=lbe.LBE_FP32)
    with pytest.raises(lbe.LBEError) as e:
        g.adjoint_backward([1.0, 0.0])
    assert e.value.code == lbe.LBE_ERR_STATE
    g.adjoint_forward(6, 4)
    g.step(1)  # the state moved on: the forward pass is gone
    with pytest.raises(lbe.LBEError) as e:
        g.adjoint_backward([1.0, 0.0])
    assert e.value.code == lbe.LBE_ERR_STATE
    q = g.adjoint_forward(6, 4)
    g.adjoint_backward([1.0, 0.0])
    g.adjoint_backward([0.0, 1.0])  # the handle is left in the forward pass's final state
    np.testing.assert_array_equal(g.charge(), q)


def test_adjoint_porous_crop_2000_steps_vs_stored_tangent(lbe):
    """The 32x32x16 porous crop, 2000 FP32 steps with checkpoints every 100,
    against the FP64 oracle tangent stored by tests/golden/make_adjoint_golden.py."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "adjoint_porous_crop32x32x16.json")
    ref = json.load(open(path))
    w = wl.porous_crop()
    assert list(w.shape) == ref["shape"] and w.steps == ref["steps"] == 2000
    q, dpsi, ddebye, dD, dchi, g, _ = gpu_grad(lbe, w, w.steps, 100, np.array([1.0, 0.0]))
    dQ = {k: np.array(v)[0] for k, v in ref["dQ"].items()}
    np.testing.assert_allclose(q, ref["Q"], rtol=1e-5)
    assert abs(dpsi[1] - dQ["psi2"]) <= TOL * abs(dQ["psi2"])
    assert abs(dpsi[0] + dQ["psi2"]) <= TOL * abs(dQ["psi2"])  # a common shift changes nothing
    assert abs(ddebye - dQ["debye"]) <= TOL * abs(dQ["debye"])
    assert abs(dD[0] - dQ["D+"]) <= TOL * max(abs(dQ["D+"]), abs(dQ["D-"]))
    assert abs(dD[1] - dQ["D-"]) <= TOL * max(abs(dQ["D+"]), abs(dQ["D-"]))
    rng = np.random.Generator(np.random.PCG64(ref["chi_random_seed"]))
    v = rng.standard_normal(dchi.size)
    assert abs(float(np.dot(dchi, v)) - dQ["chi_random"]) <= TOL * np.abs(dchi).max() * np.sqrt(dchi.size)
    for key in ("chi_fluid_node", "chi_interface_node"):
        assert abs(dchi[ref[key]] - dQ[key]) <= TOL * np.abs(dchi).max(), key
    assert g.recomputed_steps == 2000 - 20


@pytest.mark.parametrize("slots", [2, 3, 5, 9])
def test_revolve_schedule_matches_uniform_checkpoints(lbe, slots):
    """Binomial ("revolve") checkpointing within a memory budget of `slots`
    checkpoints reproduces the uniform-checkpoint gradient bit for bit, with
    each forward step recomputed at most r times (r the smallest with
    C(s + r, s) >= T, s = slots - 2); two slots recompute from the start for
    every step."""
    w = crop_case()
    steps, dq = 60, np.array([1.0, 0.3])
    _, dpsi, ddebye, dD, dchi, g, lat = gpu_grad(lbe, w, steps, 7, dq)
    per_slot = w.nodes * (2 * 8 + 8 + 3 * 8)
    q2 = lat.adjoint_forward_budget(steps, slots * per_slot + per_slot // 2)
    g2, dchi2 = lat.adjoint_backward(dq, 1)
    np.testing.assert_array_equal(np.array(g2.dpsi[:2]), dpsi)
    np.testing.assert_array_equal(np.array(g2.dD[:2]), dD)
    assert g2.drho_bulk == g.drho_bulk
    np.testing.assert_array_equal(dchi2, dchi)
    s = slots - 2
    if s > 0:
        r = 0
        while math.comb(s + r, s) < steps:
            r += 1
        assert g2.recomputed_steps <= (r + 1) * steps
    else:
        assert g2.recomputed_steps <= steps * steps // 2
    print("revolve: %d slots, %d recomputed steps for %d steps" % (slots, g2.recomputed_steps, steps))
    with pytest.raises(lbe.LBEError) as e:
        lat.adjoint_forward_budget(steps, per_slot)  # one slot
    assert e.value.code == lbe.LBE_ERR_ARG
