"""The allocation-free induced-charge entry point (lbe_induced_charge_static).

It exists for callers that cannot allocate device memory themselves being
called into (their memory comes from their own pool, or they are recording
work); it must give the same charges as lbe_induced_charge of a lattice, on
two calls in a row that share its static scratch array.  This file is
collected last, and passes alone or after the other tests.
"""
import numpy as np
import pytest

from paper_1907_04732_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _case(name):
    if name == "blob_23x18x15":
        ids = wl.random_blobs(23, 18, 15, 2, 0.2, seed=21)
        return wl.Workload("blob", ids, 2, (1, 1, 1), (-0.05, 0.3), 1.2, 2.5, e_app=(1e-3, 0.0, 0.0))
    # parallel plates, z not periodic (links leaving the box are skipped);
    # 331,776 nodes: more than the 1024 x 256 threads of the static grid, so
    # every block strides over several nodes
    return wl.Workload("plates", wl.plates(72, 72, 64), 2, (1, 1, 0), (0.0, 0.2), 1.44, 8.0,
                       e_app=(1e-3, 0.0, 0.0))


@pytest.mark.parametrize("case", ["blob_23x18x15", "plates_72x72x64"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_static_charge_matches_lattice_charge(lbe, precision, case):
    import torch
    w = _case(case)
    prec = lbe.LBE_FP32 if precision == "fp32" else lbe.LBE_FP64
    lat = lbe.Lattice.from_workload(w, precision=prec, tol=1e-13)
    lat.init()
    lat.step(8)
    q_ref = lat.charge()
    phi = lat.field(lbe.FIELD_PHI, device=True).contiguous()
    node_id = torch.from_numpy(np.ascontiguousarray(w.ids.reshape(-1))).to("cuda")
    outs = []
    for _ in range(2):
        q = torch.full((w.n_elec,), float("nan"), dtype=torch.float64, device="cuda")
        lbe.lbe_induced_charge_static(phi.data_ptr(), node_id.data_ptr(), w.shape, w.periodic, w.bjerrum,
                                      w.n_elec, q.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        outs.append(q.cpu().numpy())
    for q in outs:
        np.testing.assert_allclose(q, q_ref, rtol=1e-12, atol=1e-15 * np.abs(q_ref).max())
    np.testing.assert_array_equal(outs[0], outs[1])
    lat.close()


def test_static_charge_rejects_too_many_electrodes(lbe):
    import torch
    phi = torch.zeros(8, dtype=torch.float64, device="cuda")
    ids = torch.zeros(8, dtype=torch.uint8, device="cuda")
    q = torch.zeros(32, dtype=torch.float64, device="cuda")
    with pytest.raises(lbe.LBEError) as e:
        lbe.lbe_induced_charge_static(phi.data_ptr(), ids.data_ptr(), (2, 2, 2), (1, 1, 1), 1.0,
                                      lbe.LBE_MAX_ELECTRODES + 1, q.data_ptr())
    assert e.value.code == lbe.LBE_ERR_ARG
    assert b"n_electrodes" in lbe.load().lbe_last_error(None)
