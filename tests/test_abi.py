"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/lbe.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_1907_04732_gb300 import build as nvbuild
from paper_1907_04732_gb300 import lbe

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(lbe_\w+)\s*\(", text, flags=re.M))
        names |= set(re.findall(r"int\s+(lbe_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    nvbuild.build()
    return lbe.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 13, names
    for n in names:
        assert hasattr(lib, n), n
    assert set(lbe.EXPORTED) <= set(names)


def test_default_params_and_argument_checks(lib):
    p = lbe.lbe_default_params()
    assert (p.nx, p.ny, p.nz) == (1, 1, 1)
    assert p.tau == 1.0 and p.nspecies == 2 and list(p.z)[:2] == [1.0, -1.0]
    assert p.precision == lbe.LBE_FP64 and p.poisson_tol == 1e-13
    # invalid parameters are rejected before any CUDA call
    h = ctypes.c_void_p()
    for field, val in (("nx", 0), ("tau", 0.5), ("nspecies", 5), ("poisson_max_iter", 0)):
        q = lbe.lbe_default_params()
        setattr(q, field, val)
        assert lib.lbe_create(ctypes.byref(q), None, ctypes.byref(h)) == lbe.LBE_ERR_ARG
    q = lbe.lbe_default_params()
    q.z[0] = 0.5
    assert lib.lbe_create(ctypes.byref(q), None, ctypes.byref(h)) == lbe.LBE_ERR_ARG
    assert lib.lbe_step(None, 1) == lbe.LBE_ERR_ARG
    assert lib.lbe_last_error(None) == b"invalid handle"
    assert lib.lbe_destroy(None) == lbe.LBE_OK


def test_batch_argument_checks(lib):
    """lbe_batch_create rejects what the batched form does not cover before
    any CUDA call."""
    b = ctypes.c_void_p()

    def create(plist):
        arr = (lbe.lbe_params * len(plist))(*plist)
        return lib.lbe_batch_create(arr, len(plist), None, ctypes.byref(b))

    def fp32(**kw):
        q = lbe.lbe_default_params()
        q.precision = lbe.LBE_FP32
        q.nx, q.ny, q.nz = 4, 4, 8
        for k, v in kw.items():
            setattr(q, k, v)
        return q

    assert lib.lbe_batch_create(None, 1, None, ctypes.byref(b)) == lbe.LBE_ERR_ARG
    assert create([fp32(precision=lbe.LBE_FP64)]) == lbe.LBE_ERR_ARG
    assert create([fp32(nspecies=3)]) == lbe.LBE_ERR_ARG
    q = fp32()
    q.rho_bulk[1] = 2 * q.rho_bulk[0]  # not a symmetric 1:1 salt
    assert create([q]) == lbe.LBE_ERR_ARG
    assert create([fp32(), fp32(flow=0)]) == lbe.LBE_ERR_ARG
    assert create([fp32(), fp32(poisson_tol=1e-9)]) == lbe.LBE_ERR_ARG
    assert create([fp32(nz=0)]) == lbe.LBE_ERR_ARG
    assert lib.lbe_batch_step(None, 1) == lbe.LBE_ERR_ARG
    assert lib.lbe_batch_last_error(None) == b"invalid batch"
    assert lib.lbe_batch_destroy(None) == lbe.LBE_OK
