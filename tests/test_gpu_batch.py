"""Batched FP32 form (lbe_batch_*): many instances of uneven sizes in one
persistent launch per kernel and one graph launch per step.

Each instance is checked against the FP64 oracle with the FP32 form's
tolerances (potential 1e-6 of the voltage scale, induced charge 1e-5
relative), its solute is conserved exactly, and the full 256-instance sweep
is checked on sampled instances against the oracle run on the equivalent
reduced lattice (a plate capacitor's column, a coaxial capacitor's slice:
the fields are uniform along the periodic directions).
"""
import numpy as np
import pytest

from paper_1907_04732_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL_PHI, TOL_Q = 1e-6, 1e-5
MAXE = 4


def oracle_for(w, tol=1e-14):
    from oracle import Oracle
    o = Oracle(w.shape, w.periodic, tau=w.tau, bjerrum=w.bjerrum, z=w.z, D=w.D, rho_bulk=w.rho_bulk,
               e_app=w.e_app, flow=w.flow, tol=tol)
    o.set_geometry(w.ids, w.n_elec)
    o.set_voltage(w.psi)
    o.init()
    return o


def units(n, w):
    """Fixed-point solute amounts (units of rho_b 2^-40) of the fluid nodes."""
    rb = np.array(w.rho_bulk)[:, None, None, None]
    return np.rint((n - rb) / (rb * 2.0 ** -40)).astype(np.int64) * (w.ids == 0)


def small_mix(flow=True):
    blob2 = wl.random_blobs(13, 11, 9, 2, 0.2, seed=5)
    blob3 = wl.random_blobs(10, 12, 14, 3, 0.25, seed=6)
    return [
        wl.plate_capacitor(3, 3, 40, debye=4.0, bjerrum=1.44, psi=(0.0, 0.3), flow=flow),
        wl.coax_capacitor(20, 20, 3, r1=2.5, r2=8.0, debye=3.0, bjerrum=1.44, psi=(0.0, -0.2), flow=flow),
        wl.Workload("blob2", blob2, 2, (1, 1, 1), (0.1, -0.15), 1.0, 2.5, e_app=(1e-3, 0.0, -5e-4), flow=flow),
        wl.plate_capacitor(1, 1, 70, debye=10.0, bjerrum=1.44, psi=(0.0, 0.5), D=(0.1, 0.03), flow=flow),
        wl.Workload("blob3", blob3, 3, (1, 1, 1), (0.2, -0.1, 0.05), 0.9, 3.0, tau=0.8, flow=flow),
    ]


@pytest.mark.parametrize("flow", [True, False])
def test_batch_small_mix_vs_oracle(lbe, flow):
    ws = small_mix(flow)
    b = lbe.Batch(ws, tol=1e-12)
    b.init()
    units0 = [units(b.n_field(i), w).sum(axis=(1, 2, 3)) for i, w in enumerate(ws)]
    steps = 60
    b.step(steps)
    q = b.charge()
    st = b.stats()
    assert st.poisson_solves == steps and st.poisson_iters > 0
    for i, w in enumerate(ws):
        o = oracle_for(w)
        o.step(steps)
        scale = max(abs(v) for v in w.psi)
        phi_b, phi_o = b.phi(i), o.phi()
        assert np.abs(phi_b - phi_o).max() <= TOL_PHI * scale, (w.name, np.abs(phi_b - phi_o).max() / scale)
        qo = o.charge()
        assert np.all(np.abs(q[i, :w.n_elec] - qo) <= TOL_Q * np.abs(qo).max()), (w.name, q[i], qo)
        assert np.all(q[i, w.n_elec:] == 0.0)
        rb = w.rho_bulk[0]
        assert np.abs(b.n_field(i) - o.n()).max() <= 2e-6 * rb, w.name
        np.testing.assert_array_equal(units(b.n_field(i), w).sum(axis=(1, 2, 3)), units0[i])


def test_batch_matches_single_lattice_fp32(lbe):
    ws = small_mix(True)[:3]
    b = lbe.Batch(ws, tol=1e-12)
    b.init()
    b.step(25)
    q = b.charge()
    for i, w in enumerate(ws):
        g = lbe.Lattice.from_workload(w, precision=lbe.LBE_FP32, tol=1e-12)
        g.init()
        g.step(25)
        scale = max(abs(v) for v in w.psi)
        assert np.abs(b.phi(i) - g.phi()).max() <= TOL_PHI * scale
        qg = g.charge()
        assert np.all(np.abs(q[i, :w.n_elec] - qg) <= TOL_Q * np.abs(qg).max())


def test_batch_deterministic(lbe):
    ws = small_mix(True)
    runs = []
    for _ in range(2):
        b = lbe.Batch(ws, tol=1e-12)
        b.init()
        b.step(12)
        runs.append((b.charge(), [b.phi(i) for i in range(len(ws))], [b.n_field(i) for i in range(len(ws))]))
        b.close()
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    for a, c in zip(runs[0][1] + runs[0][2], runs[1][1] + runs[1][2]):
        np.testing.assert_array_equal(a, c)


def test_batch_errors_and_tuning(lbe):
    ws = small_mix(True)[:2]
    b = lbe.Batch(ws)
    with pytest.raises(lbe.LBEError) as e:
        b.step(1)
    assert e.value.code == lbe.LBE_ERR_STATE
    bad = np.zeros((5, 4, 4), dtype=np.uint8)  # fluid on the non-periodic z faces
    b2 = lbe.Batch([wl.plate_capacitor(4, 4, 5)])
    with pytest.raises(lbe.LBEError) as e:
        lbe.lbe_batch_set_geometry(b2.b, 0, bad.ctypes.data, 2)
    assert e.value.code == lbe.LBE_ERR_GEOMETRY
    b.init()
    with pytest.raises(lbe.LBEError) as e:
        lbe.lbe_batch_set_voltage(b.b, 0, [0.0, 0.1])
    assert e.value.code == lbe.LBE_ERR_STATE
    grid, ms = b.tuning()
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert grid in [k * sms for k in (1, 2, 3, 4, 6, 8)]
    assert all(t > 0 for t in ms)


def reduced(w):
    """The equivalent reduced lattice of a batch instance and the factor
    that scales its induced charge to the full instance."""
    nx, ny, nz = w.shape
    if w.name.endswith("plates_%dx%dx%d" % (nx, ny, nz)):
        return wl.plate_capacitor(1, 1, nz, debye=w.debye, bjerrum=w.bjerrum, psi=w.psi), nx * ny
    r = w.extra
    return wl.coax_capacitor(nx, ny, 1, r1=r["r1"], r2=r["r2"], debye=w.debye, bjerrum=w.bjerrum, psi=w.psi), nz


def test_batch_full_size_sampled_vs_oracle(lbe):
    ws = wl.batch_instances(256)
    b = lbe.Batch(ws, tol=1e-12)
    b.init()
    rng = np.random.Generator(np.random.PCG64(wl.SEED))
    big = int(np.argmax([w.nodes for w in ws]))
    sample = sorted({0, 1, big} | set(int(i) for i in rng.choice(256, 5, replace=False)))
    units0 = {i: units(b.n_field(i), ws[i]).sum(axis=(1, 2, 3)) for i in sample}
    steps = 20
    b.step(steps)
    q = b.charge()
    assert np.all(np.isfinite(q))
    for i in sample:
        w = ws[i]
        red, factor = reduced(w)
        o = oracle_for(red)
        o.step(steps)
        qo = o.charge() * factor
        assert np.all(np.abs(q[i, :2] - qo) <= TOL_Q * np.abs(qo).max()), (w.name, q[i, :2], qo)
        phi_b = b.phi(i)
        # a plate column broadcast over x, y; a coaxial slice repeated along z
        ref = np.broadcast_to(o.phi(), phi_b.shape)
        scale = max(abs(v) for v in w.psi)
        assert np.abs(phi_b - ref).max() <= TOL_PHI * scale, (w.name, np.abs(phi_b - ref).max() / scale)
        np.testing.assert_array_equal(units(b.n_field(i), w).sum(axis=(1, 2, 3)), units0[i])


def test_batch_polled_matches_graph_and_profile(lbe, monkeypatch):
    """The host-polled solve (LBE_POISSON_GRAPH=0, used to list kernels in a
    profiler) launches the same kernels in the same order as the graph: the
    results are bitwise equal.  The phase profiler reports every step."""
    ws = small_mix(True)
    out = []
    for polled in (False, True):
        if polled:
            monkeypatch.setenv("LBE_POISSON_GRAPH", "0")
        b = lbe.Batch(ws, tol=1e-12)
        monkeypatch.delenv("LBE_POISSON_GRAPH", raising=False)
        b.init()
        b.profile_begin()
        b.step(7)
        p = b.profile_end()
        assert p.sweep_launches == 7 and p.poisson_ms > 0 and p.sweep_ms > 0 and p.advect_ms > 0
        assert p.poisson_iters > 0
        assert (p.kernel_launches > 0) if polled else (p.kernel_launches == -1)
        b.step(3)  # unprofiled steps after profiling use the plain graphs
        out.append((b.charge(), [b.phi(i) for i in range(len(ws))]))
        b.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    for a, c in zip(out[0][1], out[1][1]):
        np.testing.assert_array_equal(a, c)
