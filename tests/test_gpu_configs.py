"""The nanocapacitor workloads run to their stated protocol on the GPU.

* plates 4x4x64 (FP64 form): 20,000 steps from the uncharged start; the
  oracle's column after the same 20,000 steps; the steady capacitance from
  an exponential fit of Q(t) (as in Sec. "Charge and capacitance") against
  Eq. SLITcapaDH and the discrete Poisson-Boltzmann steady state; the final
  profiles against Eq. DHslitpotential.
* coaxial 128x128x4, FP32 form against the FP64 form: 20,000 steps; the
  charging curves agree at every sample; the steady potential against Eq.
  PSIcoxialDH and the capacitance against Eq. CYLcapaDH.
* electro-osmosis 64x64x256 (FP32 form): from the charged steady state (the
  discrete Poisson-Boltzmann solution, which is the oracle's steady state),
  E_x = 1e-3 switched on and 50,000 steps (reading c12); the oracle's column
  after 10,000 and 20,000 steps (the velocity within max(1e-5, T 2^-24) of
  its largest value after T steps: one FP32 rounding per population and
  step); the steady velocity against Eq. DHslitEOF.
"""
import math

import numpy as np
import pytest
from scipy.optimize import curve_fit

from paper_1907_04732_gb300 import workloads as wl
import analytic as an
from discrete_pb import plate_column_steady

pytestmark = pytest.mark.gpu


def _oracle(w, tol=1e-14):
    from oracle import Oracle
    o = Oracle(w.shape, w.periodic, tau=w.tau, bjerrum=w.bjerrum, z=w.z, D=w.D, rho_bulk=w.rho_bulk,
               e_app=w.e_app, flow=w.flow, tol=tol)
    o.set_geometry(w.ids, w.n_elec)
    o.set_voltage(w.psi)
    return o


def _fit_qinf(t, q):
    f = lambda t, qi, b, tau: qi - b * np.exp(-t / tau)
    p, _ = curve_fit(f, t, q, p0=(q[-1], q[-1] - q[0], (t[-1] - t[0]) / 3))
    return p[0], p[2]


def test_config_plates_4x4x64_protocol(lbe):
    w = wl.plate_capacitor()  # l_B = 4.8, lambda_D = 8, voltage 0.1, D = 0.05
    L, dV, lam = 62, 0.1, 8.0
    g = lbe.Lattice.from_workload(w, precision=lbe.LBE_FP64, tol=1e-13)
    g.init()
    t, q = [], []
    for k in range(200):
        g.step(100)
        t.append(100 * (k + 1))
        q.append(g.charge()[1] / 16.0)  # per unit area
    t, q = np.array(t, float), np.array(q)
    # the oracle's column after the same 20,000 steps
    col = wl.plate_capacitor(1, 1, 64)
    o = _oracle(col)
    o.init()
    o.step(20000)
    np.testing.assert_allclose(g.phi(), np.tile(o.phi(), (1, 4, 4)), rtol=0, atol=1e-9 * dV)
    np.testing.assert_allclose(g.n(), np.tile(o.n(), (1, 1, 4, 4)), rtol=1e-9)
    np.testing.assert_allclose(q[-1], o.charge()[1], rtol=1e-8)
    # steady capacitance: exponential fit over the last three quarters
    qinf, tau = _fit_qinf(t[50:], q[50:])
    eps = an.eps_of(w.bjerrum)
    qdh = an.dh_plate_charge_per_area(eps, 1.0 / lam, L, dV)
    phi_pb, _ = plate_column_steady(L, 0.1, 0.2, w.bjerrum, w.rho_bulk)
    q_pb = -eps * 2.0 * (phi_pb[-1] - 0.2)  # Eq. Qelec at the doubled links of electrode 2
    print("plates 4x4x64: Q(20000) %.6e  Q_inf fit %.6e  discrete PB %.6e  DH %.6e  tau %.0f"
          % (q[-1], qinf, q_pb, qdh, tau))
    assert abs(qinf - q_pb) <= 2e-3 * q_pb
    assert abs(qinf - qdh) <= 5e-3 * qdh
    assert 0.7 * L * lam / (2 * 0.05) < tau < 1.1 * L * lam / (2 * 0.05)  # charging time ~ L lambda/(2D)
    # profiles after 20,000 steps (four charging times) against Debye-Hueckel
    zc = np.arange(64) - 31.5
    dh = an.dh_plate_potential(zc[1:-1], L, 1.0 / lam, 0.1, 0.2)
    phi = g.phi()[1:-1, 0, 0]
    assert np.abs(phi - dh).max() <= 3e-3 * dV
    n = g.n()[:, 1:-1, 0, 0] / w.rho_bulk[0]
    assert np.abs(n[0] - 1 + (dh - 0.15)).max() <= 3e-3
    assert np.abs(n[1] - 1 - (dh - 0.15)).max() <= 3e-3


def test_config_coax_128x128x4_fp32_vs_fp64(lbe):
    w = wl.coax_capacitor()  # R1 10, R2 50, lambda_D 5, l_B 1.2, voltage 0.1
    runs = {}
    for prec in (lbe.LBE_FP64, lbe.LBE_FP32):
        g = lbe.Lattice.from_workload(w, precision=prec, tol=1e-12)  # populations on
        g.init()
        q = []
        for k in range(40):
            g.step(500)
            q.append(g.charge()[0])
        runs[prec] = (np.array(q), g.phi())
        g.close()
    q64, phi64 = runs[lbe.LBE_FP64]
    q32, phi32 = runs[lbe.LBE_FP32]
    assert np.all(np.abs(q32 - q64) <= 1e-5 * np.abs(q64).max()), np.abs(q32 - q64).max() / np.abs(q64).max()
    assert np.abs(phi32 - phi64).max() <= 1e-6 * 0.1
    # steady state: the charge no longer moves, and matches Debye-Hueckel
    assert abs(q64[-1] - q64[-2]) <= 2e-5 * abs(q64[-1])
    eps, kappa = an.eps_of(w.bjerrum), 1.0 / w.debye
    c = abs(q64[-1]) / (4 * 0.1)
    c_dh = an.coax_cdh_per_length(eps, 10.0, 50.0, kappa)
    ny, nx = w.ids.shape[1:]
    y, x = np.mgrid[0:ny, 0:nx]
    r = np.hypot(x - (nx - 1) / 2, y - (ny - 1) / 2)
    fl = w.ids[0] == 0
    th = an.coax_dh_potential(r[fl], 10.0, 50.0, kappa, 0.0, 0.1)
    err = np.abs(phi64[0][fl] - th) / 0.1
    rms = np.sqrt(np.mean(err ** 2))
    # the staircase walls lie up to half a lattice spacing from the circles
    # r = R1, R2, so near a wall the potential may be off by up to half a
    # spacing times the largest radial field of Eq. PSIcoxialDH (at r = R1)
    rr = np.linspace(10.0, 50.0, 4001)
    slope = np.abs(np.gradient(an.coax_dh_potential(rr, 10.0, 50.0, kappa, 0.0, 0.1), rr)).max() / 0.1
    far = err[(r[fl] >= 13.0) & (r[fl] <= 47.0)].max()
    print("coax 128x128x4: C/C_DH - 1 = %.4f, |phi - phi_DH|/dV: max %.4f (bound %.4f), rms %.4f, "
          "max 3+ from the walls %.4f" % (c / c_dh - 1, err.max(), 0.5 * slope, rms, far))
    assert abs(c / c_dh - 1) < 0.03
    assert err.max() <= 0.5 * slope
    assert rms < 0.02


def test_config_eof_64x64x256_protocol(lbe):
    full, col = wl.eof_plates(), wl.eof_plates(1, 1, 256)
    L, lam, dV, E = 254, 16.0, 0.2, 1e-3
    phi_pb, n_pb = plate_column_steady(L, 0.0, dV, full.bjerrum, full.rho_bulk)
    phi0 = np.concatenate([[0.0], phi_pb, [dV]])
    n0 = np.concatenate([np.zeros((2, 1)), n_pb, np.zeros((2, 1))], axis=1)
    g = lbe.Lattice.from_workload(full, precision=lbe.LBE_FP32, tol=1e-12)
    g.init()
    g.set_state(n=np.broadcast_to(n0[:, :, None, None], (2, 256, 64, 64)).copy(),
                phi=np.broadcast_to(phi0[:, None, None], (256, 64, 64)).copy())
    o = _oracle(col)
    o.init()
    o.set_state(n=n0[:, :, None, None].copy(), phi=phi0[:, None, None].copy())
    for t in (10000, 20000):  # the oracle's column at steps 10,000 and 20,000
        g.step(10000)
        o.step(10000)
        uo = o.u()
        ug = g.u()
        # the FP32 populations take one rounding each per step; in a slowly
        # varying flow these do not average out, and move u by up to about
        # 2^-24 |u| per step (measured: 1.0e-4 and 2.5e-4 of max |u| here)
        tol_u = max(1e-5, t * 2.0 ** -24)
        du = np.abs(ug - np.tile(uo, (1, 1, 64, 64))).max() / np.abs(uo).max()
        print("eof 64x64x256: step %d, max |u - u_oracle| / max |u| = %.2e (bound %.2e)" % (t, du, tol_u))
        assert du <= tol_u
        assert np.abs(g.phi() - np.tile(o.phi(), (1, 64, 64))).max() <= 1e-6 * dV
        qo = o.charge() * 4096
        assert np.all(np.abs(g.charge() - qo) <= 1e-5 * np.abs(qo).max())
    g.step(30000)
    # steady electro-osmotic flow against Eq. DHslitEOF (the antisymmetric
    # lowest mode decays in L^2/(4 pi^2 nu) = 9.8k steps: 0.6 % left)
    eps, eta = an.eps_of(full.bjerrum), 1.0 / 6.0
    zc = np.arange(256) - 127.5
    th = an.dh_plate_eof(zc[1:-1], L, 1.0 / lam, eps, eta, E, dV)
    uref = eps * E * dV / eta
    ux = g.u()[0, 1:-1, 0, 0]
    dev = np.abs(ux - th).max() / uref
    print("eof 64x64x256: max |u - u_DH| / u_ref = %.4f after 50,000 steps" % dev)
    assert dev < 0.015


def test_config_batch_capacitance_per_instance(lbe):
    """The batched sweep of seeded capacitors: the 24 instances of the
    256-instance generator with the shortest charging times (L lambda_D/2D
    <= ~310 steps: coaxial cells of sides 8-36) run to steady state in one
    batch (10 charging times); each instance's capacitance C = Q/dV, with
    its voltage, matches the plain FP64 single-lattice form run the same
    way (1e-5), and C stays within 3 % of the same instance at half the
    voltage (the linear regime of Eq. CYLcapaDH)."""
    ws = wl.batch_instances(256)
    taus = []
    for i, w in enumerate(ws):
        nx = w.shape[0]
        gap = (w.shape[2] - 2) if i % 2 == 0 else (nx / 2 - 2) - max(1.0, (nx / 2 - 2) / 5)
        taus.append((gap * w.debye / (2 * 0.05), i))
    pick = [i for _, i in sorted(taus)[:24]]
    steps = int(10 * sorted(taus)[23][0])
    sel = [ws[i].with_(flow=False) for i in pick]
    half = [w.with_(psi=(w.psi[0], 0.5 * w.psi[1])) for w in sel]
    b = lbe.Batch(sel + half, tol=1e-12)
    b.init()
    b.step(steps)
    q = b.charge()
    n = len(sel)
    c = np.array([abs(q[k, 1]) / abs(w.psi[1] - w.psi[0]) for k, w in enumerate(sel)])
    c_half = np.array([abs(q[n + k, 1]) / abs(w.psi[1] - w.psi[0]) for k, w in enumerate(half)])
    print("batch capacitance per instance (C, voltage):",
          [(round(float(ci), 4), round(w.psi[1], 3)) for ci, w in zip(c, sel)])
    assert np.all(np.abs(c_half / c - 1) < 0.03), np.abs(c_half / c - 1).max()
    for k in np.argsort([w.nodes for w in sel])[:3]:
        g = lbe.Lattice.from_workload(sel[k], precision=lbe.LBE_FP64, tol=1e-13)
        g.init()
        g.step(steps)
        qg = g.charge()
        g.close()
        np.testing.assert_allclose(q[k, :2], qg, rtol=1e-5)
