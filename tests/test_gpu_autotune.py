"""The autotuner on the GPU: lls_autotune measures the implementation choices on the caller's
problem and records the fastest; later "auto" calls (panel_width 0) on that shape use it and
still solve the problem to the oracle's accuracy; the batched variant picks the CTAs per SM.
The JSON cache written on the way is a temporary file."""
import numpy as np
import pytest
import torch

from oracle import direct, metrics
from paper_1912_05508_gb300 import lls, synth, tuning

pytestmark = pytest.mark.gpu


@pytest.fixture
def cache(tmp_path, monkeypatch):
    path = str(tmp_path / "tuning.json")
    monkeypatch.setenv("LLS_TUNE_CACHE", path)
    lls.lls_tuning_clear()
    yield path
    lls.lls_tuning_clear()


def test_autotune_records_a_setting_that_auto_calls_use(cache):
    p = synth.svd_lls(8192, 384, "geometric", 1e3, seed=71)
    A = lls.colmajor(p.A)
    b = torch.from_numpy(p.b).cuda()
    best = lls.autotune(A, b, reps=2, cache_path=cache)
    assert best["panel_width"] in (8, 16, 32) and best["node_mode"] in (0, 1, 2)
    assert best["gemm_kernel"] in (0, 1, 2) and best["ms"] > 0
    o = lls.make_options()
    rec = lls.lls_tuning_get(0, 8192, 384, o)
    assert rec is not None and rec.as_dict()["panel_width"] == best["panel_width"]
    # the cache file holds it under this GPU's name
    name = torch.cuda.get_device_properties(0).name
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ent = tuning.entries_for_device(tuning.load(cache), name, sms)
    assert [(k, m, n) for k, m, n, _, _ in ent] == [(0, 8192, 384)]
    # an auto solve takes the recorded setting and reaches the FP64 target
    x, info = lls.solve(A, b)
    assert info["status"] == 0
    xs = direct.lls(p.A, p.b)
    assert metrics.forward_error(x.cpu().numpy(), xs) <= 10 * p.kappa * 1e-12
    # a fresh table restored from the file gives the same setting
    lls.lls_tuning_clear()
    lls._tuning_loaded.clear()
    assert lls.load_tuning_cache(0, cache) == 1
    assert lls.lls_tuning_get(0, 8192, 384, o).as_dict() == rec.as_dict()


@pytest.mark.parametrize("pw,node_mode,gemm_kernel", [(8, 0, 0), (32, 1, 1), (16, 2, 2), (16, 0, 2)])
def test_every_recorded_setting_solves_to_the_oracle(cache, pw, node_mode, gemm_kernel):
    # whatever the tuner picks, the solve is the same method: each setting reaches the target
    p = synth.svd_lls(6000, 320, "geometric", 1e3, seed=72)
    o = lls.make_options()
    assert lls.lls_tuning_set(0, 6000, 320, o, lls.lls_tuning(pw, node_mode, gemm_kernel, 0, 0, 1.0)) == 0
    x, info = lls.solve(lls.colmajor(p.A), torch.from_numpy(p.b).cuda())
    assert info["status"] == 0, info
    xs = direct.lls(p.A, p.b)
    assert metrics.forward_error(x.cpu().numpy(), xs) <= 10 * p.kappa * 1e-12


def test_autotune_batched(cache):
    As, bs, kap = synth.batched_problems_torch(96, seed=73, m_range=(256, 2048), n_range=(16, 128),
                                               kappa_exp=(1.0, 3.0))
    best = lls.autotune_batched(As, bs, reps=1, cache_path=cache)
    assert best["batched_ctas_per_sm"] >= 1 and best["ms"] > 0
    xs, infos = lls.solve_batched(As, bs, target="fp32")
    assert all(i["status"] == 0 for i in infos)
    for i in (0, 50, 95):
        xo = direct.lls(As[i].cpu().numpy(), bs[i].cpu().numpy())
        assert metrics.forward_error(xs[i].cpu().numpy(), xo) <= 1e-5
