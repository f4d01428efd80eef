"""Failure detection on the GPU without a fault: a bounded device wait that runs out.

lls_selftest_wait_timeout launches a cooperative kernel whose grid barrier (the barrier every
persistent kernel of the library uses) can never complete; each wait gives up after its time
limit, sets the device error word and returns. The host must read LLS_ERR_TIMEOUT, and the
context must still run a solve afterwards.
"""
import time

import torch
import pytest

from oracle import metrics
from paper_1912_05508_gb300 import lls, synth

pytestmark = pytest.mark.gpu

LLS_ERR_TIMEOUT = -5


def test_bounded_wait_reports_timeout_and_the_context_survives():
    ws = lls.workspace(256).zero_()
    s = torch.cuda.current_stream().cuda_stream
    t0 = time.perf_counter()
    st = lls.lls_selftest_wait_timeout(ws.data_ptr(), ws.numel(), s)
    dt = time.perf_counter() - t0
    assert st == LLS_ERR_TIMEOUT, lls.lls_status_string(st)
    assert 1.0 < dt < 10.0                   # the limit is about 2 s of device time
    assert lls.lls_status_string(st) == "device wait timed out"
    p = synth.svd_lls(1024, 128, "geometric", 1e3, seed=1)
    x, info = lls.solve(lls.colmajor(p.A), torch.from_numpy(p.b).cuda())
    assert info["status"] == 0
    assert metrics.eta_kw(p.A, p.b, x.cpu().numpy()) <= 1e-12


def test_selftest_rejects_a_small_workspace():
    ws = lls.workspace(256)
    assert lls.lls_selftest_wait_timeout(ws.data_ptr(), 128, torch.cuda.current_stream().cuda_stream) == -1
