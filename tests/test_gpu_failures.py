"""Failure detection on the GPU, without faulting it: a bounded device wait
that runs out comes back as a status, and non-finite data are reported."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1607_01650_gb300 as dect  # noqa: E402


def test_bounded_wait_times_out_and_context_survives():
    L = dect.load()
    st = L.dect_selftest_bounded_wait(1000, dect._stream())
    assert st == 4  # DECT_ERR_TIMEOUT
    assert b"ran out" in L.dect_last_error()
    # the context is still usable
    x = torch.ones(1024, device="cuda")
    assert float(x.sum()) == 1024.0


def test_nonfinite_data_is_reported():
    g = synth.tiny_geometry(n=24, nv=12, nb=40)
    plan = dect.Plan(g)
    m = torch.rand((1, 2, g.nv, g.nb), device="cuda")
    m[0, 1, 3, 5] = float("nan")
    with pytest.raises(dect.DectError, match="non-finite"):
        dect.adm_tv(plan, m, dect.AdmParams(max_iter=5))
    # the healthy channel set still runs afterwards
    m2 = torch.rand((1, 2, g.nv, g.nb), device="cuda")
    x, reps = dect.adm_tv(plan, m2, dect.AdmParams(max_iter=5))
    assert torch.isfinite(x).all()


def test_invalid_arguments_raise():
    g = synth.tiny_geometry(n=16, nv=8, nb=24)
    plan = dect.Plan(g)
    with pytest.raises(dect.DectError):
        dect.project(plan, torch.zeros((1, 15, 15), device="cuda"))
    with pytest.raises(dect.DectError):
        dect.adm_tv(plan, torch.zeros((1, 2, g.nv, g.nb), device="cuda"), dect.AdmParams(rho=0.0))
    with pytest.raises(dect.DectError):
        dect.pls_decompose(torch.zeros((1, 2, 16, 16), device="cuda"),
                           dect.PlsParams(eta=((1.0, 2.0), (2.0, 4.0))))  # singular D
