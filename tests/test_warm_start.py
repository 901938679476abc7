"""The warm start of each step's Poisson solve extrapolates the earlier
converged potentials in time (cubic in the library).  The converged
potential does not depend on the start, so the choice is about how close the
start lands: pinned here on the oracle's trajectory of the charging
electro-osmosis section (periodic 2 x 2 x 256 column of the 64 x 64 x 256
lattice, tolerance 1e-12), where each higher order lands closer."""
import numpy as np

from paper_1907_04732_gb300 import workloads as wl


def test_higher_order_start_lands_closer():
    from oracle import Oracle
    w = wl.eof_plates(nx=2, ny=2, nz=256)
    o = Oracle(w.shape, w.periodic, tau=w.tau, bjerrum=w.bjerrum, z=w.z, D=w.D, rho_bulk=w.rho_bulk,
               e_app=w.e_app, flow=w.flow, tol=1e-12)
    o.set_geometry(w.ids, w.n_elec)
    o.set_voltage(w.psi)
    o.init()
    phi = []
    for _ in range(30):
        o.step(1)
        phi.append(np.array(o.phi(), dtype=np.float64).ravel())
    p0, p1, p2, p3, p4 = phi[-1], phi[-2], phi[-3], phi[-4], phi[-5]
    err = {
        "linear": np.abs(p0 - (2 * p1 - p2)).max(),
        "quadratic": np.abs(p0 - (3 * p1 - 3 * p2 + p3)).max(),
        "cubic": np.abs(p0 - (4 * p1 - 6 * p2 + 4 * p3 - p4)).max(),
    }
    assert err["quadratic"] < err["linear"] / 10, err
    assert err["cubic"] < err["quadratic"] / 4, err
