"""The LLS_DEBUG build without a GPU: it compiles for sm_103a, exports the release build's ABI
and reports itself as the debug build; the release build reports the opposite and refuses to
arm the planted index error (host-only calls, no device work)."""
import ctypes
import os
import subprocess
import sys

from paper_1912_05508_gb300 import build, lls

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_release_build_is_not_debug():
    lib = lls.load()
    assert lib.lls_debug_build() == 0
    assert lib.lls_debug_inject(1) == -6            # LLS_ERR_UNSUPPORTED
    assert lls.lls_status_string(-8) == "index check failed (debug build)"


def test_debug_build_compiles_and_exports_the_abi():
    path = build.build(debug=True)
    code = (
        "import ctypes, sys\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "from paper_1912_05508_gb300 import lls\n"
        f"lib = ctypes.CDLL({path!r})\n"
        "missing = [n for n in lls.EXPORTS if not hasattr(lib, n)]\n"
        "assert not missing, missing\n"
        "lib.lls_debug_build.restype = ctypes.c_int\n"
        "print(lib.lls_debug_build())\n"
    )
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "1"
