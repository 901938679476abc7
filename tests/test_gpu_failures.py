"""Failure detection through the C ABI, with every failure made on the host.

A non-finite or out-of-range value is handed to the library through its
public calls (lbe_set_state, lbe_load_state, electrode potentials); the
library must report LBE_ERR_NONFINITE from the call that meets it, without
hanging (every device loop is bounded) and without a GPU fault.  Nothing here
faults, traps or hangs a GPU: NaN and infinity are ordinary IEEE values.
"""
import struct

import numpy as np
import pytest

from paper_1907_04732_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _lattice(lbe, precision, flow=True):
    ids = wl.random_blobs(14, 13, 12, 2, 0.2, seed=23)
    w = wl.Workload("blob", ids, 2, (1, 1, 1), (0.0, 0.15), 1.0, 2.5, e_app=(1e-3, 0.0, 0.0), flow=flow)
    prec = lbe.LBE_FP64 if precision == "fp64" else lbe.LBE_FP32
    g = lbe.Lattice.from_workload(w, precision=prec, tol=1e-12)
    g.init()
    g.step(2)
    return g, w


def _fluid_node(w):
    return np.argwhere(w.ids == 0)[len(np.argwhere(w.ids == 0)) // 2]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_nan_solute_is_reported(lbe, precision):
    """A NaN solute amount at one fluid node: the FP32 form rejects it while
    converting to fixed point (range flag); the FP64 form carries it into the
    Poisson residual, whose stopping test reports it."""
    g, w = _lattice(lbe, precision)
    n = g.n()
    n[(0,) + tuple(_fluid_node(w))] = np.nan
    with pytest.raises(lbe.LBEError) as e:
        g.set_state(n=n)
        g.step(1)
    assert e.value.code == lbe.LBE_ERR_NONFINITE, e.value
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_nan_potential_is_reported(lbe, precision):
    """A NaN potential at one fluid node.  The FP64 form takes it, and the
    next step's flux, force and Poisson residual meet it: lbe_step returns
    LBE_ERR_NONFINITE.  The FP32 form converts the potential to its fixed
    point at once and lbe_set_state itself returns LBE_ERR_NONFINITE."""
    g, w = _lattice(lbe, precision)
    phi = g.phi()
    phi[tuple(_fluid_node(w))] = np.nan
    with pytest.raises(lbe.LBEError) as e:
        g.set_state(phi=phi)
        g.step(1)
    assert e.value.code == lbe.LBE_ERR_NONFINITE, e.value
    g.close()


def test_potential_beyond_fixed_point_range(lbe):
    """The FP32 form holds |potential| < 100: a larger electrode potential is
    refused (LBE_ERR_ARG) and a larger node value handed to lbe_set_state
    raises the range flag (LBE_ERR_NONFINITE)."""
    g, w = _lattice(lbe, "fp32")
    with pytest.raises(lbe.LBEError) as e:
        g.set_voltage((0.0, 150.0))
    assert e.value.code == lbe.LBE_ERR_ARG, e.value
    phi = g.phi()
    phi[tuple(_fluid_node(w))] = 120.0
    with pytest.raises(lbe.LBEError) as e:
        g.set_state(phi=phi)
    assert e.value.code == lbe.LBE_ERR_NONFINITE, e.value
    g.close()


def test_out_of_range_solute_raises_range_flag(lbe):
    """An amount beyond the FP32 form's fixed-point range (about 3.6e6 times
    the bulk value) sets the range flag when it is converted."""
    g, w = _lattice(lbe, "fp32")
    n = g.n()
    n[(1,) + tuple(_fluid_node(w))] = 1e8 * w.rho_bulk[1]
    with pytest.raises(lbe.LBEError) as e:
        g.set_state(n=n)
    assert e.value.code == lbe.LBE_ERR_NONFINITE, e.value
    g.close()


def test_potential_spike_raises_flux_range_flag(lbe):
    """A finite potential spike of 60 kT/e at one fluid node makes its link
    fluxes (e^60 times the bulk) overflow the fixed-point unit: the sweep
    raises the range flag and lbe_step reports it."""
    g, w = _lattice(lbe, "fp32")
    phi = g.phi()
    phi[tuple(_fluid_node(w))] = 60.0
    g.set_state(phi=phi)
    with pytest.raises(lbe.LBEError) as e:
        g.step(1)
    assert e.value.code == lbe.LBE_ERR_NONFINITE, e.value
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_nan_population_in_loaded_state_is_reported(lbe, precision):
    """A checkpoint whose populations hold a NaN at one fluid node (written
    on the host into a saved blob): after lbe_load_state the next step
    reports LBE_ERR_NONFINITE (FP32: the sweep's density check; FP64: the
    velocity carries it into the solute and the Poisson residual)."""
    g, w = _lattice(lbe, precision)
    blob = bytearray(g.save_state())
    header = struct.calcsize("<QqiiIIii")  # magic, N, ns, flow, precision, history, step kind, pad
    N = w.nodes
    z, y, x = _fluid_node(w)
    r = x + w.shape[0] * (y + w.shape[1] * z)
    size = 4 if precision == "fp32" else 8
    off = header + (3 * N + r) * size  # population 3 of node r
    blob[off:off + size] = struct.pack("<f" if size == 4 else "<d", float("nan"))
    g.load_state(bytes(blob))
    with pytest.raises(lbe.LBEError) as e:
        g.step(2)
    assert e.value.code == lbe.LBE_ERR_NONFINITE, e.value
    g.close()


def test_batch_voltage_spike_raises_range_flag(lbe):
    """The batched form: an instance at 96 kT/e across a gap of 4 nodes (a
    finite, accepted potential, below the fixed-point potential's bound of
    100: 24 kT/e per link, link fluxes e^24 times the bulk) overflows the
    solute's fixed-point unit in the first sweep; lbe_batch_step reports
    LBE_ERR_NONFINITE, and the error names the range flag.  A potential of
    100 or more is refused when it is set."""
    big = wl.plate_capacitor(4, 4, 6, debye=4.0, bjerrum=1.44, psi=(0.0, 100.0))
    with pytest.raises(lbe.LBEError) as e:
        lbe.Batch([big], tol=1e-12)
    assert e.value.code == lbe.LBE_ERR_ARG, e.value
    ws = [wl.plate_capacitor(4, 4, 20, debye=4.0, bjerrum=1.44, psi=(0.0, 0.1)),
          wl.plate_capacitor(4, 4, 6, debye=4.0, bjerrum=1.44, psi=(0.0, 96.0))]
    b = lbe.Batch(ws, tol=1e-12)
    b.init()
    with pytest.raises(lbe.LBEError) as e:
        b.step(2)
    assert e.value.code == lbe.LBE_ERR_NONFINITE, e.value
    assert "range" in str(e.value)
    b.close()
