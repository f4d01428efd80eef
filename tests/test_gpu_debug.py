"""The LLS_DEBUG build on the GPU (index checks on the kernels' global-memory accesses).

1. The checks change no arithmetic: a fixed set of seeded calls (a solve through the block
   kernels, fused nodes and persistent tensor-core products; a ragged BF16 QR with a
   direct-start LSQR solve; an uneven batch and its adjoint) gives bitwise equal results in the
   release and the debug build, and no check fires.
2. A planted index error is caught: with lls_debug_inject(1), the panel kernel's stores of Q
   compute row indices one panel height past the last row; every such store is rejected by its
   check (so the matrix is left as it was), the call returns LLS_ERR_BOUNDS and the site is
   named on stderr. Disarmed, the same call succeeds. No access leaves its buffer.
3. A wait that cannot complete is reported: with lls_debug_inject(2), the panel's grid barrier
   waits for one CTA more than the grid holds; every CTA gives up after the wait limit (about
   2 s), so qr_factor leaves NaN on R's diagonal and lls_solve returns LLS_ERR_TIMEOUT.
   Disarmed, both succeed. The GPU stays usable throughout.
Each build runs in a child process (tests/debug_child.py), since a process loads one build.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1912_05508_gb300 import build

pytestmark = pytest.mark.gpu

CHILD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "debug_child.py")


@pytest.fixture(scope="module")
def debug_lib():
    build.build()
    return build.build(debug=True)


def child(mode, out, debug, tmp_path):
    env = dict(os.environ, LLS_DEBUG="1" if debug else "0",
               LLS_TUNE_CACHE=str(tmp_path / "no_tuning.json"))
    return subprocess.run([sys.executable, CHILD, mode, str(out)], env=env, capture_output=True, text=True,
                          timeout=900)


def test_debug_build_matches_release_bitwise(debug_lib, tmp_path):
    rel, dbg = tmp_path / "rel.npz", tmp_path / "dbg.npz"
    r = child("run", rel, False, tmp_path)
    assert r.returncode == 0, r.stderr[-3000:]
    d = child("run", dbg, True, tmp_path)
    assert d.returncode == 0, d.stderr[-3000:]
    assert "[lls debug]" not in d.stderr, d.stderr[-3000:]
    a, b = np.load(rel), np.load(dbg)
    assert sorted(a.files) == sorted(b.files)
    for k in a.files:
        assert np.array_equal(a[k], b[k], equal_nan=True), k
    assert a["solve_iters"][1] == 0


@pytest.fixture(scope="module")
def injected(debug_lib, tmp_path_factory):
    d = tmp_path_factory.mktemp("inject")
    out = d / "inject.json"
    r = child("inject", out, True, d)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(out.read_text()), r.stderr


def test_planted_index_error_is_caught(injected):
    res, stderr = injected
    assert res["debug_build"] == 1
    assert res["arm"] == 0 and res["disarm"] == 0
    assert res["armed_status"] == -8          # LLS_ERR_BOUNDS
    assert res["q_untouched"]                 # every store was rejected
    assert "[lls debug] index check failed at panel_flat.cu:" in stderr
    assert res["disarmed_status"] == 0
    assert res["q_written"]


def test_withheld_barrier_arrival_is_reported(injected):
    res, _ = injected
    assert res["arm2"] == 0 and res["disarm2"] == 0
    assert res["armed_qr_diag_nan"]
    assert res["armed_solve_status"] == -5    # LLS_ERR_TIMEOUT
    assert res["disarmed_qr_diag_finite"]
    assert res["disarmed_solve_status"] == 0
    assert res["bad_mode"] == -1              # LLS_ERR_ARG
