"""FP32 form (FP32 deviations streamed in place, int64 fixed-point solute in
units of rho_b 2^-40, int64 fixed-point potential in units of 2^-48 refined
on an exact-Laplacian residual) against the FP64 oracle.

Tolerances (relative): potential 1e-6 of the voltage, induced charge 1e-5,
velocity 1e-5 of the largest velocity; total solute amount of each species
conserved exactly (integer fixed-point sums).
"""
import numpy as np
import pytest

from paper_1907_04732_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL_PHI, TOL_Q, TOL_U = 1e-6, 1e-5, 1e-5


def oracle_for(w, tol=1e-14):
    from oracle import Oracle
    o = Oracle(w.shape, w.periodic, tau=w.tau, bjerrum=w.bjerrum, z=w.z, D=w.D, rho_bulk=w.rho_bulk,
               e_app=w.e_app, flow=w.flow, tol=tol)
    o.set_geometry(w.ids, w.n_elec)
    o.set_voltage(w.psi)
    o.init()
    return o


def gpu_for(lbe, w, tol=1e-12):
    g = lbe.Lattice.from_workload(w, precision=lbe.LBE_FP32, tol=tol)
    g.init()
    return g


def fixed_point_units(n, w):
    """Recover the integer solute amounts (units of rho_b 2^-40)."""
    s = np.array(w.rho_bulk)[:, None, None, None] * 2.0 ** -40
    rb = np.array(w.rho_bulk)[:, None, None, None]
    return np.rint((n - rb) / s).astype(np.int64) * (w.ids == 0)


def check(o, g, w, scale_phi, tol_n=2e-6):
    phi_o, phi_g = o.phi(), g.phi()
    assert np.abs(phi_g - phi_o).max() <= TOL_PHI * scale_phi, np.abs(phi_g - phi_o).max() / scale_phi
    q_o, q_g = o.charge(), g.charge()
    assert np.all(np.abs(q_g - q_o) <= TOL_Q * np.abs(q_o).max()), (q_g, q_o)
    u_o, u_g = o.u(), g.u()
    umax = np.abs(u_o).max()
    assert np.abs(u_g - u_o).max() <= TOL_U * umax + 1e-12, (np.abs(u_g - u_o).max(), umax)
    n_o, n_g = o.n(), g.n()
    rb = np.array(w.rho_bulk)[:, None, None, None]
    assert np.abs(n_g - n_o).max() <= tol_n * rb.max(), np.abs(n_g - n_o).max() / rb.max()


@pytest.mark.parametrize("flow", [True, False])
def test_fp32_random_geometry(lbe, flow):
    ids = wl.random_blobs(21, 19, 17, 2, 0.2, seed=17)
    w = wl.Workload("blob", ids, 2, (1, 1, 1), (0.0, 0.25), 1.1, 2.5, e_app=(2e-3, -1e-3, 5e-4), flow=flow)
    o, g = oracle_for(w), gpu_for(lbe, w)
    q0 = fixed_point_units(g.n(), w).sum(axis=(1, 2, 3))
    o.step(30)
    g.step(30)
    check(o, g, w, 0.25)
    # exact conservation of the solute in fixed point
    np.testing.assert_array_equal(fixed_point_units(g.n(), w).sum(axis=(1, 2, 3)), q0)


def test_fp32_plate_charging_column(lbe):
    w = wl.plate_capacitor(1, 1, 64, psi=(0.1, 0.2))
    o, g = oracle_for(w), gpu_for(lbe, w)
    for _ in range(4):
        o.step(500)
        g.step(500)
        check(o, g, w, 0.1)


def test_fp32_full_coax_vs_oracle_slice(lbe):
    full = wl.coax_capacitor()
    red = wl.coax_capacitor(128, 128, 1)
    o, g = oracle_for(red), gpu_for(lbe, full)
    o.step(20)
    g.step(20)
    phi_g = g.phi()
    assert np.abs(phi_g - np.tile(o.phi(), (4, 1, 1))).max() <= TOL_PHI * 0.1
    q_o = o.charge() * 4
    assert np.all(np.abs(g.charge() - q_o) <= TOL_Q * np.abs(q_o).max())


def test_fp32_eof_column_flow(lbe):
    # charged state from the oracle, then the tangential field drives flow
    base = wl.plate_capacitor(1, 1, 42, debye=5.0, bjerrum=1.0, psi=(0.0, 0.05), D=(0.15, 0.15), flow=False)
    ob = oracle_for(base)
    ob.step(2000)
    w = base.with_(e_app=(2e-3, 0.0, 0.0), flow=True)
    o, g = oracle_for(w), gpu_for(lbe, w)
    o.set_state(n=ob.n(), phi=ob.phi())
    g.set_state(n=ob.n(), phi=ob.phi())
    o.step(600)
    g.step(600)
    check(o, g, w, 0.05)


def test_fp32_full_size_eof_vs_oracle_column(lbe):
    """The benchmarked lattice itself: 64x64x256 electro-osmosis (1,048,576
    nodes, so every finest-level solve kernel runs several planes per thread)
    against the oracle on its 1x1x256 column (the workload is translation
    invariant along x and y), 30 steps from the uncharged start, with exact
    fixed-point conservation over the whole lattice."""
    full, red = wl.eof_plates(), wl.eof_plates(1, 1, 256)
    o, g = oracle_for(red), gpu_for(lbe, full)
    q0 = fixed_point_units(g.n(), full).sum(axis=(1, 2, 3))
    reps = (1, 64, 64)
    scale = abs(full.psi[1] - full.psi[0])
    for _ in range(2):
        o.step(15)
        g.step(15)
        assert np.abs(g.phi() - np.tile(o.phi(), reps)).max() <= TOL_PHI * scale
        q_o = o.charge() * 4096
        assert np.all(np.abs(g.charge() - q_o) <= TOL_Q * np.abs(q_o).max()), (g.charge(), q_o)
        u_o = np.tile(o.u(), (1,) + reps)
        assert np.abs(g.u() - u_o).max() <= TOL_U * np.abs(u_o).max() + 1e-12
        rb = max(full.rho_bulk)
        assert np.abs(g.n() - np.tile(o.n(), (1,) + reps)).max() <= 2e-6 * rb
    np.testing.assert_array_equal(fixed_point_units(g.n(), full).sum(axis=(1, 2, 3)), q0)
    g.close()


def test_fp32_unsigned_population_offsets_vs_oracle_column(lbe):
    """A plate lattice of 115,343,360 nodes (256x256x1760): 19 N lies
    between 2^31 and 2^32, so the odd in-place sweeps index the populations
    with unsigned 32-bit offsets (the even ones with 64-bit offsets).  Four
    steps (both step kinds twice) against the oracle on the 1x1x1760 column,
    on sampled columns of the device fields, with exact fixed-point
    conservation over the whole lattice summed on the device."""
    import torch
    nx, ny, nz = 256, 256, 1760
    assert 2 ** 31 <= 19 * nx * ny * nz < 2 ** 32
    full, red = wl.eof_plates(nx, ny, nz), wl.eof_plates(1, 1, nz)
    o, g = oracle_for(red), gpu_for(lbe, full)
    fluid = torch.from_numpy(full.ids == 0).to("cuda")
    rb = torch.tensor(full.rho_bulk, dtype=torch.float64, device="cuda")[:, None, None, None]

    def total_units():
        n = g.field(lbe.FIELD_N, device=True)
        q = torch.round((n - rb) / (rb * 2.0 ** -40)).to(torch.int64) * fluid
        return q.sum(dim=(1, 2, 3)).cpu().numpy()

    q0 = total_units()
    o.step(4)
    g.step(4)
    cols = [(0, 0), (255, 255), (17, 200), (128, 64)]
    scale = abs(full.psi[1] - full.psi[0])
    phi = g.field(lbe.FIELD_PHI, device=True)
    u = g.field(lbe.FIELD_U, device=True)
    n = g.field(lbe.FIELD_N, device=True)
    u_o, n_o = o.u()[:, :, 0, 0], o.n()[:, :, 0, 0]
    for x, y in cols:
        assert np.abs(phi[:, y, x].cpu().numpy() - o.phi()[:, 0, 0]).max() <= TOL_PHI * scale
        assert np.abs(u[:, :, y, x].cpu().numpy() - u_o).max() <= TOL_U * np.abs(u_o).max() + 1e-12
        assert np.abs(n[:, :, y, x].cpu().numpy() - n_o).max() <= 2e-6 * max(full.rho_bulk)
    del phi, u, n
    q_o = o.charge() * (nx * ny)
    assert np.all(np.abs(g.charge() - q_o) <= TOL_Q * np.abs(q_o).max()), (g.charge(), q_o)
    np.testing.assert_array_equal(total_units(), q0)
    g.close()


@pytest.mark.parametrize("flow", [True, False])
def test_fp32_large_random_geometry(lbe, flow):
    """A random two-electrode lattice above 262,144 nodes (72x72x64 =
    331,776: the solve's kernels run several planes per thread, ragged in
    x, y and the last plane group) against the oracle element by element,
    tau = 0.8, a three-component field, 4 steps."""
    ids = wl.random_blobs(72, 72, 64, 2, 0.15, seed=29)
    w = wl.Workload("blob", ids, 2, (1, 1, 1), (0.0, 0.2), 1.44, 4.0, tau=0.8,
                    e_app=(1e-3, -5e-4, 2.5e-4), flow=flow)
    o, g = oracle_for(w), gpu_for(lbe, w)
    q0 = fixed_point_units(g.n(), w).sum(axis=(1, 2, 3))
    o.step(4)
    g.step(4)
    check(o, g, w, 0.2)
    np.testing.assert_array_equal(fixed_point_units(g.n(), w).sum(axis=(1, 2, 3)), q0)
    g.close()


def test_fp32_determinism_and_checkpoint(lbe):
    ids = wl.random_blobs(16, 15, 14, 2, 0.2, seed=9)
    w = wl.Workload("blob", ids, 2, (1, 1, 1), (0.0, 0.2), 1.0, 2.0, e_app=(1e-3, 0.0, 0.0))
    a = gpu_for(lbe, w)
    a.step(5)
    blob = a.save_state()
    a.step(5)
    b = gpu_for(lbe, w)
    b.step(10)
    np.testing.assert_array_equal(a.phi(), b.phi())
    np.testing.assert_array_equal(a.n(), b.n())
    np.testing.assert_array_equal(a.populations(), b.populations())
    c = lbe.Lattice.from_workload(w, precision=lbe.LBE_FP32, tol=1e-12)
    c.load_state(blob)
    c.step(5)
    np.testing.assert_array_equal(c.populations(), a.populations())
    np.testing.assert_array_equal(c.n(), a.n())
    np.testing.assert_array_equal(c.charge(), a.charge())


def test_set_voltage_unchanged_keeps_state(lbe):
    """Setting the potentials the electrodes already hold uploads them and
    leaves the trajectory bitwise unchanged; a new value re-solves at once."""
    ids = wl.random_blobs(14, 13, 12, 2, 0.2, seed=23)
    w = wl.Workload("blob", ids, 2, (1, 1, 1), (0.0, 0.15), 1.0, 2.5, e_app=(1e-3, 0.0, 0.0))
    a, b = gpu_for(lbe, w), gpu_for(lbe, w)
    for _ in range(6):
        a.set_voltage(w.psi)
        a.step(1)
        b.step(1)
    np.testing.assert_array_equal(a.phi(), b.phi())
    np.testing.assert_array_equal(a.n(), b.n())
    a.set_voltage((0.0, 0.2))
    assert np.abs(a.phi() - b.phi()).max() > 1e-3  # re-solved for the new voltage


def test_exact_coarsest_solve_matches_jacobi_sweeps(lbe, monkeypatch):
    """The exact coarsest-level solve (inverse formed at set-up) and the 32
    Jacobi sweeps it replaces are two preconditioners of the same CG: the
    converged potentials agree to the solve tolerance, and the exact one
    needs no more iterations."""
    w = wl.Workload("plates", wl.plates(32, 32, 96), 2, (1, 1, 0), (0.0, 0.2), 1.44, 8.0,
                    e_app=(1e-3, 0.0, 0.0))
    runs = []
    for direct in ("0", "1"):
        monkeypatch.setenv("LBE_MG_DIRECT", direct)
        g = gpu_for(lbe, w)
        g.step(10)
        runs.append((g.phi(), g.stats().poisson_iters))
        g.close()
    (p_jac, it_jac), (p_dir, it_dir) = runs
    assert np.abs(p_dir - p_jac).max() <= 1e-9, np.abs(p_dir - p_jac).max()
    assert it_dir <= it_jac, (it_dir, it_jac)


def test_periodic_box_without_electrodes(lbe):
    """A fully periodic lattice without electrodes has a singular coarsest
    operator: the set-up keeps the Jacobi sweeps there, and with a uniform
    salt the potential stays zero."""
    ids = np.zeros((16, 12, 10), dtype=np.uint8)
    w = wl.Workload("box", ids, 0, (1, 1, 1), (), 1.0, 4.0, e_app=(1e-3, 0.0, 0.0))
    g = gpu_for(lbe, w)
    g.step(5)
    assert np.all(np.isfinite(g.phi()))
    assert np.abs(g.phi()).max() <= 1e-12
    g.close()

