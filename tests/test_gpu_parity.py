"""GPU (C-ABI) vs FP64 oracle, element by element, on seeded lattices.

The FP64 CUDA path and the oracle both solve the Poisson equation to a
Jacobi-scaled residual of 1e-14; the potentials then agree to that residual
times the inverse smallest eigenvalue of the Jacobi-scaled operator
(< 1e-10 relative to the voltage on these lattices), and every other field to
round-off propagated through a few steps.
"""
import math

import numpy as np
import pytest

from paper_1907_04732_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-14


def run_both(w, steps, lbe, flow=None, n_set=None, tol=TOL):
    from oracle import Oracle
    flow = w.flow if flow is None else flow
    o = Oracle(w.shape, w.periodic, tau=w.tau, bjerrum=w.bjerrum, z=w.z, D=w.D, rho_bulk=w.rho_bulk,
               e_app=w.e_app, flow=flow, tol=tol)
    o.set_geometry(w.ids, w.n_elec)
    o.set_voltage(w.psi)
    o.init()
    g = lbe.Lattice.from_workload(w, tol=tol, flow=flow)
    g.init()
    if n_set is not None:
        o.set_state(n=n_set)
        g.set_state(n=n_set)
    if steps:
        o.step(steps)
        g.step(steps)
    return o, g


# the oracle's population order (see oracle/lbe_oracle.c)
ORACLE_VELOCITIES = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
                     (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1),
                     (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]


def gpu_populations_in_oracle_order(g, lbe):
    f = g.populations()
    order = [lbe.VELOCITIES.index(c) for c in ORACLE_VELOCITIES]
    return f[order]


def compare(o, g, scale_phi, lbe):
    np.testing.assert_allclose(g.phi(), o.phi(), rtol=0, atol=1e-10 * scale_phi)
    n_o, n_g = o.n(), g.n()
    np.testing.assert_allclose(n_g, n_o, rtol=1e-10, atol=1e-12 * np.abs(n_o).max())
    q_o, q_g = o.charge(), g.charge()
    np.testing.assert_allclose(q_g, q_o, rtol=1e-8, atol=1e-12 * max(np.abs(q_o).max(), 1e-30))
    u_o, u_g = o.u(), g.u()
    np.testing.assert_allclose(u_g, u_o, rtol=0, atol=1e-9 * np.abs(u_o).max() + 1e-15)
    np.testing.assert_allclose(g.rho(), o.rho(), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(gpu_populations_in_oracle_order(g, lbe), o.populations(), rtol=0, atol=1e-12)


def test_init_laplace_plates(lbe):
    w = wl.plate_capacitor(3, 2, 20, psi=(0.1, 0.2))
    o, g = run_both(w, 0, lbe)
    compare(o, g, 0.1, lbe)
    L = 18
    eps = 1 / (4 * math.pi * w.bjerrum)
    np.testing.assert_allclose(g.charge(), [-eps * 0.1 / L * 6, eps * 0.1 / L * 6], rtol=1e-11)


@pytest.mark.parametrize("flow", [True, False])
def test_random_geometry_ragged(lbe, flow):
    ids = wl.random_blobs(21, 19, 17, 2, 0.2, seed=17)
    w = wl.Workload("blob", ids, 2, (1, 1, 1), (0.0, 0.25), 1.1, 2.5, e_app=(2e-3, -1e-3, 5e-4))
    o, g = run_both(w, 12, lbe, flow=flow)
    compare(o, g, 0.25, lbe)


def test_coax_slice(lbe):
    w = wl.coax_capacitor(30, 30, 3, r1=3.0, r2=12.0, debye=3.0, bjerrum=1.2)
    o, g = run_both(w, 8, lbe)
    compare(o, g, 0.1, lbe)


def test_plates_column_perturbed_with_flow(lbe):
    w = wl.plate_capacitor(1, 1, 26, debye=3.0, bjerrum=1.0, psi=(0.0, 0.1), e_app=(1e-3, 0.0, 0.0))
    rng = np.random.default_rng(3)
    n = np.stack([np.full(w.ids.shape, r) for r in w.rho_bulk]) * (1 + 0.05 * rng.normal(size=(2,) + w.ids.shape))
    n *= (w.ids == 0)
    o, g = run_both(w, 20, lbe, n_set=n)
    compare(o, g, 0.1, lbe)


def test_mass_conservation_and_gauss(lbe):
    ids = wl.random_blobs(24, 20, 18, 2, 0.15, seed=5)
    w = wl.Workload("blob", ids, 2, (1, 1, 1), (-0.1, 0.2), 1.3, 3.0, e_app=(1e-3, 1e-3, 0.0))
    g = lbe.Lattice.from_workload(w, tol=TOL)
    g.init()
    m0 = g.n().sum(axis=(1, 2, 3))
    g.step(25)
    n = g.n()
    np.testing.assert_allclose(n.sum(axis=(1, 2, 3)), m0, rtol=1e-13)
    q = g.charge()
    assert abs(q.sum() + (n[0] - n[1]).sum()) < 1e-12 * np.abs(q).max()


def test_determinism_and_checkpoint(lbe):
    ids = wl.random_blobs(16, 15, 14, 2, 0.2, seed=9)
    w = wl.Workload("blob", ids, 2, (1, 1, 1), (0.0, 0.2), 1.0, 2.0, e_app=(1e-3, 0.0, 0.0))
    a = lbe.Lattice.from_workload(w, tol=TOL)
    a.init()
    a.step(5)
    blob = a.save_state()
    a.step(5)
    b = lbe.Lattice.from_workload(w, tol=TOL)
    b.init()
    b.step(10)
    np.testing.assert_array_equal(a.phi(), b.phi())
    np.testing.assert_array_equal(a.n(), b.n())
    np.testing.assert_array_equal(a.charge(), b.charge())
    c = lbe.Lattice.from_workload(w, tol=TOL)
    c.load_state(blob)
    c.step(5)
    np.testing.assert_array_equal(c.populations(), a.populations())
    np.testing.assert_array_equal(c.n(), a.n())


def test_errors(lbe):
    p = lbe.params_for(wl.plate_capacitor(2, 2, 8))
    p.periodic[2] = 0
    lat = lbe.Lattice(p)
    bad = wl.plates(2, 2, 8)
    bad[0, 0, 0] = 0  # fluid on the non-periodic face
    with pytest.raises(lbe.LBEError) as e:
        lat.set_geometry(bad, 2)
    assert e.value.code == lbe.LBE_ERR_GEOMETRY
    with pytest.raises(lbe.LBEError) as e:
        lat.step(1)
    assert e.value.code == lbe.LBE_ERR_STATE
    p2 = lbe.params_for(wl.plate_capacitor(2, 2, 30), maxit=1)
    lat2 = lbe.Lattice(p2)
    lat2.set_geometry(wl.plates(2, 2, 30), 2)
    lat2.set_voltage((0.0, 0.1))
    with pytest.raises(lbe.LBEError) as e:
        lat2.init()
    assert e.value.code == lbe.LBE_ERR_NOCONVERGE


# Full-size lattices of the nanocapacitor workloads: they are translation
# invariant along their periodic directions, so the GPU run on the full
# lattice must equal the oracle on a one-node-wide column / slice.
@pytest.mark.parametrize("which", ["plates_4x4x64", "eof_64x64x256", "coax_128x128x4"])
def test_full_size_vs_reduced_oracle(lbe, which):
    from oracle import Oracle
    if which == "plates_4x4x64":
        full = wl.plate_capacitor()
        red = wl.plate_capacitor(1, 1, 64)
        steps = 40
    elif which == "eof_64x64x256":
        full = wl.eof_plates()
        red = wl.eof_plates(1, 1, 256)
        steps = 6
    else:
        full = wl.coax_capacitor()
        red = wl.coax_capacitor(128, 128, 1)
        steps = 4
    g = lbe.Lattice.from_workload(full, tol=TOL)
    g.init()
    g.step(steps)
    o = Oracle(red.shape, red.periodic, tau=red.tau, bjerrum=red.bjerrum, z=red.z, D=red.D,
               rho_bulk=red.rho_bulk, e_app=red.e_app, flow=red.flow, tol=TOL)
    o.set_geometry(red.ids, red.n_elec)
    o.set_voltage(red.psi)
    o.init()
    o.step(steps)
    scale = abs(full.psi[1] - full.psi[0])
    phi_g, phi_o = g.phi(), o.phi()
    n_g, n_o = g.n(), o.n()
    reps = (full.shape[2] // red.shape[2], full.shape[1] // red.shape[1], full.shape[0] // red.shape[0])
    np.testing.assert_allclose(phi_g, np.tile(phi_o, reps), rtol=0, atol=1e-9 * scale)
    np.testing.assert_allclose(n_g, np.tile(n_o, (1,) + reps), rtol=1e-9, atol=1e-12 * n_o.max())
    area = full.nodes // red.nodes
    np.testing.assert_allclose(g.charge(), o.charge() * area, rtol=1e-7)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_charge_map_sums_to_electrode_charges(lbe, precision):
    """The per-node charge map (LBE_FIELD_QNODE): nonzero only on electrode
    nodes with fluid neighbours; its sum over each electrode is Q_e, and
    over all electrodes minus the ionic charge (Gauss)."""
    ids = wl.porous(15, 14, 13, 3, 1.5, 2.5, 6.0, seed=21)  # electrodes do not touch
    w = wl.Workload("porous", ids, 2, (1, 1, 0), (0.0, 0.2), 1.0, 2.5, e_app=(1e-3, 0.0, 0.0))
    prec = lbe.LBE_FP64 if precision == "fp64" else lbe.LBE_FP32
    g = lbe.Lattice.from_workload(w, precision=prec, tol=1e-13)
    g.init()
    g.step(20)
    qmap, q = g.charge_map(), g.charge()
    assert np.all(qmap[ids == 0] == 0.0)
    for e in range(1, 3):
        assert abs(qmap[ids == e].sum() - q[e - 1]) <= 1e-12 * np.abs(q).max()
    n = g.n()
    ionic = (n[0] - n[1]).sum()
    assert abs(qmap.sum() + ionic) <= 1e-9 * np.abs(q).max()


def test_first_order_rule_matches_oracle(lbe):
    """The first-order boundary rule (LBE_RULE_NODE: plain Laplacian, solid
    nodes at their potential) against the oracle's same rule, element by
    element, with flow, field and two electrodes."""
    from oracle import Oracle
    ids = wl.random_blobs(21, 19, 17, 2, 0.2, seed=17)
    w = wl.Workload("blob", ids, 2, (1, 1, 1), (0.0, 0.25), 1.1, 2.5, e_app=(2e-3, -1e-3, 5e-4))
    o = Oracle(w.shape, w.periodic, tau=w.tau, bjerrum=w.bjerrum, z=w.z, D=w.D, rho_bulk=w.rho_bulk,
               e_app=w.e_app, flow=True, tol=TOL)
    o.set_geometry(w.ids, w.n_elec)
    o.set_voltage(w.psi)
    o.set_boundary_rule(1)
    o.init()
    g = lbe.Lattice.from_workload(w, tol=TOL, rule=lbe.LBE_RULE_NODE)
    g.init()
    o.step(12)
    g.step(12)
    compare(o, g, 0.25, lbe)
    # Gauss: the induced charges still balance the ionic charge exactly
    n = g.n()
    assert abs(g.charge().sum() + (n[0] - n[1]).sum()) < 1e-12 * np.abs(g.charge()).max()


def test_first_order_rule_needs_fp64(lbe):
    p = lbe.params_for(wl.plate_capacitor(2, 2, 8), precision=lbe.LBE_FP32, rule=lbe.LBE_RULE_NODE)
    with pytest.raises(lbe.LBEError) as e:
        lbe.Lattice(p)
    assert e.value.code == lbe.LBE_ERR_ARG


def test_fp32_in_place_populations_both_step_kinds(lbe):
    """The FP32 form streams its populations in place, alternating two kinds
    of step (the AA pattern); its populations field is what the next step's
    collision reads, in the layout of that step's kind.  After 1, 2, 3 and 4
    steps (both kinds, on a ragged periodic lattice with solid blobs, so
    that bounce-back links of both kinds are exercised) the field, the
    density and the velocity match the FP64 oracle to FP32 accuracy
    (populations to 2e-9, where a slot taken from the wrong layout would be
    off by a deviation between directions, asserted above 1e-7)."""
    from oracle import Oracle
    ids = wl.random_blobs(19, 17, 15, 2, 0.2, seed=29)
    w = wl.Workload("blob", ids, 2, (1, 1, 1), (0.0, 0.2), 1.0, 2.0, e_app=(2e-3, -1e-3, 5e-4))
    o = Oracle(w.shape, w.periodic, tau=w.tau, bjerrum=w.bjerrum, z=w.z, D=w.D, rho_bulk=w.rho_bulk,
               e_app=w.e_app, flow=True, tol=1e-14)
    o.set_geometry(w.ids, w.n_elec)
    o.set_voltage(w.psi)
    o.init()
    g = lbe.Lattice.from_workload(w, precision=lbe.LBE_FP32, tol=1e-12)
    g.init()
    dev_max = 0.0
    for _ in range(4):
        o.step(1)
        g.step(1)
        fo = o.populations()
        w_i = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)[:, None, None, None]
        dev_max = max(dev_max, float(np.abs(fo - w_i * (fo.sum(axis=0) > 0)).max()))
        np.testing.assert_allclose(gpu_populations_in_oracle_order(g, lbe), fo, rtol=0, atol=2e-9)
        np.testing.assert_allclose(g.rho(), o.rho(), rtol=0, atol=1e-8)
        u_o = o.u()
        # velocity 1e-5 of its largest value, with a floor for the first
        # steps' tiny velocities: the sum of 19 FP32 deviations of ~1e-4
        # resolves u to ~1e-11
        np.testing.assert_allclose(g.u(), u_o, rtol=0, atol=1e-5 * np.abs(u_o).max() + 1e-10)
    assert dev_max > 1e-7, dev_max  # the populations did move away from rest
    g.close()
