"""Host-side checks of the C ABI: the library builds, loads and exports every entry point
declared in include/lls_gb300.h, and argument checks answer without a GPU."""
import ctypes as C
import os
import re

import pytest

from paper_1912_05508_gb300 import build, lls

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "lls_gb300.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    txt = re.sub(r"^\s*#.*$", "", txt, flags=re.M)
    names = []
    for stmt in txt.split(";"):
        if "(" not in stmt or "typedef" in stmt or "{" in stmt.split("(")[0]:
            continue
        head = stmt.split("(")[0].split()
        if len(head) >= 2:
            names.append(head[-1].lstrip("*"))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return lls.load()


def test_every_declared_symbol_is_exported(lib):
    names = header_functions()
    assert "qr_factor" in names and "lls_solve" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(lls.EXPORTS) <= set(names)


def test_defaults_and_status_strings(lib):
    o = lls.lls_default_options()
    assert (o.gemm_prec, o.target, o.max_iter, o.panel_width, o.krylov) == (0, 1, 200, 0, 0)
    assert lls.lls_status_string(0) == "ok"
    assert "singular" in lls.lls_status_string(-2)


def test_workspace_queries_and_argument_errors(lib):
    o = lls.make_options()
    assert lls.qr_factor_workspace_size(1000, 100, o) > 1000 * 100 * 6
    assert lls.qr_factor_workspace_size(10, 20, o) == 0          # m < n
    assert lls.lls_solve_workspace_size(1000, 100, o) > lls.qr_factor_workspace_size(1000, 100, o)
    bad = lls.make_options(panel_width=40)
    assert lls.qr_factor_workspace_size(100, 10, bad) == 0
    # argument errors are detected before any device work: null pointers, ld < m
    assert lls.qr_factor(100, 10, None, 100, None, 0, None, 10, None, 0, o, None) == -1
    assert lls.qr_factor(100, 10, 256, 50, None, 0, 256, 10, 256, 1 << 20, o, None) == -1
    info = lls.lls_info()
    assert lls.lls_solve(5, 10, 256, 5, 256, 256, None, 0, 256, 1 << 20, o, info, None) == -1
    # misaligned / too small workspace
    assert lls.qr_factor(100, 10, 256, 100, None, 0, 256, 10, 257, 1 << 30, o, None) == -4
    assert lls.qr_factor(100, 10, 256, 100, None, 0, 256, 10, 256, 1024, o, None) == -4


def test_host_solve_block_and_selftest_entry_points(lib):
    o = lls.make_options()
    # the host-operand solve needs the device solve's workspace plus copies of A, b and x
    m, n = 1000, 100
    assert lls.lls_solve_host_workspace_size(m, n, o) >= lls.lls_solve_workspace_size(m, n, o) + m * n * 4 + (m + n) * 8
    assert lls.lls_solve_host_workspace_size(10, 20, o) == 0
    info = lls.lls_info()
    assert lls.lls_solve_host(m, n, None, m, None, None, 256, 1 << 20, o, info, None) == -1
    assert lls.lls_solve_host(m, n, 256, m - 1, 256, 256, 256, 1 << 20, o, info, None) == -1
    # the lowest-node block: sizes and arguments
    assert lls.lls_panel_block_qr_workspace_size(4000, 16, 16) > 0
    assert lls.lls_panel_block_qr_workspace_size(20, 16, 16) == 0          # m < w1 + w2
    assert lls.lls_panel_block_qr(4000, 16, 16, 0, None, 4000, None, 4000, None, 32, 256, 1 << 20, None) == -1
    assert lls.lls_panel_block_qr(4000, 16, 16, 0, 256, 4000, 256, 4000, 256, 31, 256, 1 << 20, None) == -1
    assert lls.lls_panel_block_qr(4000, 16, 16, lls.PREC["fp32"], 256, 4000, 256, 4000, 256, 32, 256, 1 << 20,
                                  None) == -1
    # the wait self-test: workspace checks before any device work
    assert lls.lls_selftest_wait_timeout(None, 256, None) == -1
    assert lls.lls_selftest_wait_timeout(256, 128, None) == -1
    assert lls.lls_selftest_wait_timeout(257, 1024, None) == -1


def test_panel_leaf_option(lib):
    # the options struct carries the panel leaf (0 CGS2, 1 MGS of Alg. 4); other values are
    # argument errors, and the default is CGS2
    assert lls.lls_default_options().panel_leaf == 0
    assert lls.qr_factor_workspace_size(1000, 64, lls.make_options(panel_leaf="mgs")) > 0
    assert lls.qr_factor_workspace_size(1000, 64, lls.make_options(panel_leaf=2)) == 0
    assert lls.lls_solve_workspace_size(1000, 64, lls.make_options(panel_leaf=-1)) == 0


@pytest.mark.parametrize("n", [1, 40, 64, 65, 128, 700, 4096, 5000, 16384, 2 ** 31 - 1])
def test_upload_chunks_partition_the_columns(lib, n):
    # the host-operand solve uploads A in these chunks: contiguous, covering [0, n), the first
    # 64 columns wide and then doubling, so the factorization waits only for the first chunk
    s = lls.lls_upload_chunks(n)
    assert s[0] == 0 and s[-1] == n and all(a < b for a, b in zip(s, s[1:]))
    assert len(s) - 1 <= 32
    assert s[1] == min(64, n)
    for k in range(2, len(s) - 1):
        assert s[k] == 2 * s[k - 1]


def test_upload_chunks_argument_errors(lib):
    buf = (C.c_int * 64)()
    assert lib.lls_upload_chunks(0, buf, 64) == -1
    assert lib.lls_upload_chunks(4096, None, 64) == -1
    assert lib.lls_upload_chunks(4096, buf, 3) == -1          # 7 chunks need 8 entries


def test_x0_option(lib):
    # the starting point of the Krylov iteration: 0 zero (default), 1 the caller's x, 2 the
    # direct solve R^{-1} Q^T b; other values are argument errors, and the batched solver takes
    # the zero start only
    assert lls.lls_default_options().x0 == 0
    for mode in ("zero", "given", "direct"):
        assert lls.lls_solve_workspace_size(1000, 64, lls.make_options(x0=mode)) > 0
    assert lls.lls_solve_workspace_size(1000, 64, lls.make_options(x0=3)) == 0
    assert lls.lls_solve_workspace_size(1000, 64, lls.make_options(x0=-1)) == 0
    assert lls.lls_solve_batched_workspace_size(1, [256], [16], lls.make_options(x0=3)) == 0
    info = lls.lls_info()
    assert lls.lls_solve(1000, 64, 256, 1000, 256, 256, None, 0, 256, 1 << 30, lls.make_options(x0=5), info,
                         None) == -1


def test_tuning_table_set_get_clear(lib):
    # the library's table of tuned settings: keyed by kind, shape and the options that change
    # the arithmetic; invalid settings are rejected; clear forgets everything
    lls.lls_tuning_clear()
    o = lls.make_options(prec="fp16", target="fp64")
    assert lls.lls_tuning_get(0, 32768, 4096, o) is None
    t = lls.lls_tuning(8, 1, 1, 0, 0, 12.5)
    assert lls.lls_tuning_set(0, 32768, 4096, o, t) == 0
    got = lls.lls_tuning_get(0, 32768, 4096, o)
    assert got is not None and got.as_dict() == {"panel_width": 8, "node_mode": 1, "gemm_kernel": 1,
                                                 "batched_ctas_per_sm": 0, "krylov_ctas": 0, "ms": 12.5}
    # another precision or shape is another key
    assert lls.lls_tuning_get(0, 32768, 4096, lls.make_options(prec="bf16")) is None
    assert lls.lls_tuning_get(0, 32768, 2048, o) is None
    # the panel width does not take part in the key (it is what the setting chooses)
    assert lls.lls_tuning_get(0, 32768, 4096, lls.make_options(prec="fp16", panel_width=32)) is not None
    # invalid settings and kinds
    assert lls.lls_tuning_set(0, 100, 10, o, lls.lls_tuning(40, 0, 0, 0, 0, 1.0)) == -1
    assert lls.lls_tuning_set(0, 100, 10, o, lls.lls_tuning(16, 3, 0, 0, 0, 1.0)) == -1
    assert lls.lls_tuning_set(0, 100, 10, o, lls.lls_tuning(16, 0, 3, 0, 0, 1.0)) == -1
    assert lls.lls_tuning_set(0, 100, 10, o, lls.lls_tuning(16, 0, 0, 0, -1, 1.0)) == -1
    assert lls.lls_tuning_set(2, 100, 10, o, lls.lls_tuning(16, 0, 0, 0, 0, 1.0)) == -1
    assert lls.lls_tuning_set(0, 100, 10, lls.make_options(prec="fp8"), lls.lls_tuning(8, 0, 0, 0, 0, 1.0)) == -1
    assert lls.lls_tuning_set(1, 4096, 512, o, lls.lls_tuning(16, 0, 0, 2, 0, 9.0)) == 0
    assert lls.lls_tuning_get(1, 4096, 512, o).batched_ctas_per_sm == 2
    lls.lls_tuning_clear()
    assert lls.lls_tuning_get(0, 32768, 4096, o) is None and lls.lls_tuning_get(1, 4096, 512, o) is None


def test_auto_panel_width_workspace_covers_every_candidate(lib):
    # an "auto" call (panel_width 0) may run with any width a tuning picks: its workspace query
    # answers for the largest of them
    auto = lls.make_options(panel_width=0)
    for m, n in ((1000, 100), (32768, 4096), (5000, 7)):
        need = max(lls.lls_solve_workspace_size(m, n, lls.make_options(panel_width=w)) for w in (8, 16, 32))
        assert lls.lls_solve_workspace_size(m, n, auto) == need
        assert lls.lls_autotune_workspace_size(m, n, auto) == need
        assert lls.qr_factor_workspace_size(m, n, auto) == max(
            lls.qr_factor_workspace_size(m, n, lls.make_options(panel_width=w)) for w in (8, 16, 32))
