"""Python binding of the C ABI in include/lls_gb300.h (ctypes; argument marshalling only).

The raw functions keep the C names and take integer device pointers, sizes and a CUDA
stream handle. The torch helpers below them (``qr``, ``solve``) only allocate device
memory with torch and pass pointers; every arithmetic step runs in the library's kernels.
Loading fails loudly when the compiled library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "liblls_gb300.so")
# LLS_DEBUG=1 in the environment selects the index-checking build (build(debug=True))
LIB_DEBUG_PATH = os.path.join(PKG, "liblls_gb300_debug.so")

PREC = {"fp16": 0, "bf16": 1, "fp8": 2, "fp32": 3, "fp64": 4}
TARGET = {"fp32": 0, "fp64": 1}
KRYLOV = {"cgls": 0, "lsqr": 1}
PANEL_LEAF = {"cgs2": 0, "mgs": 1}
X0 = {"zero": 0, "given": 1, "direct": 2}
STATUS = {0: "LLS_OK", 1: "LLS_NOT_CONVERGED", -1: "LLS_ERR_ARG", -2: "LLS_ERR_SINGULAR",
          -3: "LLS_ERR_CUDA", -4: "LLS_ERR_WORKSPACE", -5: "LLS_ERR_TIMEOUT", -6: "LLS_ERR_UNSUPPORTED",
          -7: "LLS_ERR_TOO_LARGE", -8: "LLS_ERR_BOUNDS"}

EXPORTS = ("lls_default_options", "lls_status_string", "lls_kernel_launch_count",
           "qr_factor_workspace_size", "qr_factor", "lls_solve_workspace_size", "lls_solve",
           "lls_lowp_projection_workspace_size", "lls_lowp_projection", "lls_lowp_update",
           "lls_backward_workspace_size", "lls_backward",
           "lls_solve_batched_workspace_size", "lls_solve_batched",
           "lls_lowp_projection_noalloc", "lls_panel_qr_workspace_size", "lls_panel_qr",
           "lls_panel_block_qr_workspace_size", "lls_panel_block_qr",
           "lls_solve_host_workspace_size", "lls_solve_host", "lls_selftest_wait_timeout",
           "lls_upload_chunks",
           "lls_householder_workspace_size", "lls_householder_solve",
           "lls_autotune_workspace_size", "lls_autotune", "lls_autotune_batched", "lls_tuning_set",
           "lls_tuning_get", "lls_tuning_clear", "lls_debug_build", "lls_debug_inject")


class lls_options(C.Structure):
    _fields_ = [("gemm_prec", C.c_int), ("target", C.c_int), ("tol", C.c_double),
                ("max_iter", C.c_int), ("panel_width", C.c_int), ("krylov", C.c_int),
                ("leaf_rows", C.c_int), ("reorth", C.c_int), ("panel_leaf", C.c_int), ("x0", C.c_int)]


class lls_info(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("eta", C.c_double),
                ("fwd_est", C.c_double), ("res_norm", C.c_double), ("atr_norm", C.c_double),
                ("anorm_f", C.c_double), ("xnorm", C.c_double), ("qr_ms", C.c_float),
                ("krylov_ms", C.c_float), ("a_passes", C.c_int), ("m_passes", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class lls_tuning(C.Structure):
    _fields_ = [("panel_width", C.c_int), ("node_mode", C.c_int), ("gemm_kernel", C.c_int),
                ("batched_ctas_per_sm", C.c_int), ("krylov_ctas", C.c_int), ("ms", C.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class LLSError(RuntimeError):
    def __init__(self, status, where):
        super().__init__(f"{where}: {STATUS.get(status, status)}")
        self.status = status


_lib = None


def load(path: str | None = None):
    """Load the compiled library (built by paper_1912_05508_gb300.build); with LLS_DEBUG=1 in
    the environment, the index-checking debug build."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = LIB_DEBUG_PATH if os.environ.get("LLS_DEBUG", "0") not in ("", "0") else LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} missing (run __graft_entry__.build())")
    lib = C.CDLL(path)
    i, sz, vp, dp = C.c_int, C.c_size_t, C.c_void_p, C.c_double
    lib.lls_default_options.argtypes = [C.POINTER(lls_options)]
    lib.lls_default_options.restype = None
    lib.lls_status_string.argtypes = [i]
    lib.lls_status_string.restype = C.c_char_p
    lib.lls_kernel_launch_count.argtypes = []
    lib.lls_kernel_launch_count.restype = C.c_ulonglong
    lib.qr_factor_workspace_size.argtypes = [i, i, C.POINTER(lls_options)]
    lib.qr_factor_workspace_size.restype = sz
    lib.qr_factor.argtypes = [i, i, vp, i, vp, i, vp, i, vp, sz, C.POINTER(lls_options), vp]
    lib.qr_factor.restype = i
    lib.lls_solve_workspace_size.argtypes = [i, i, C.POINTER(lls_options)]
    lib.lls_solve_workspace_size.restype = sz
    lib.lls_solve.argtypes = [i, i, vp, i, vp, vp, vp, i, vp, sz, C.POINTER(lls_options),
                              C.POINTER(lls_info), vp]
    lib.lls_solve.restype = i
    lib.lls_solve_host_workspace_size.argtypes = [i, i, C.POINTER(lls_options)]
    lib.lls_solve_host_workspace_size.restype = sz
    lib.lls_solve_host.argtypes = [i, i, vp, i, vp, vp, vp, sz, C.POINTER(lls_options), C.POINTER(lls_info), vp]
    lib.lls_solve_host.restype = i
    lib.lls_selftest_wait_timeout.argtypes = [vp, sz, vp]
    lib.lls_selftest_wait_timeout.restype = i
    lib.lls_upload_chunks.argtypes = [i, C.POINTER(C.c_int), i]
    lib.lls_upload_chunks.restype = i
    lib.lls_lowp_projection_workspace_size.argtypes = [i, i, i]
    lib.lls_lowp_projection_workspace_size.restype = sz
    lib.lls_lowp_projection.argtypes = [i, i, i, i, vp, vp, i, vp, vp, i, vp, i, vp, vp, sz, vp]
    lib.lls_lowp_projection.restype = i
    lib.lls_lowp_projection_noalloc.argtypes = [i, i, i, i, vp, vp, i, vp, vp, i, vp, i, vp, vp]
    lib.lls_lowp_projection_noalloc.restype = i
    lib.lls_panel_qr_workspace_size.argtypes = [i, i]
    lib.lls_panel_qr_workspace_size.restype = sz
    lib.lls_panel_qr.argtypes = [i, i, i, vp, i, vp, i, vp, i, vp, sz, vp]
    lib.lls_panel_qr.restype = i
    lib.lls_panel_block_qr_workspace_size.argtypes = [i, i, i]
    lib.lls_panel_block_qr_workspace_size.restype = sz
    lib.lls_panel_block_qr.argtypes = [i, i, i, i, vp, i, vp, i, vp, i, vp, sz, vp]
    lib.lls_panel_block_qr.restype = i
    lib.lls_householder_workspace_size.argtypes = [i, i, i]
    lib.lls_householder_workspace_size.restype = sz
    lib.lls_householder_solve.argtypes = [i, i, i, vp, i, vp, vp, vp, sz, vp]
    lib.lls_householder_solve.restype = i
    lib.lls_lowp_update.argtypes = [i, i, i, i, vp, i, vp, i, vp, vp, i, vp, sz, vp]
    lib.lls_lowp_update.restype = i
    ip = C.POINTER(C.c_int)
    pp = C.POINTER(C.c_void_p)
    lib.lls_backward_workspace_size.argtypes = [i, ip, ip, C.POINTER(lls_options)]
    lib.lls_backward_workspace_size.restype = sz
    lib.lls_backward.argtypes = [i, ip, ip, pp, ip, pp, pp, pp, ip, pp, pp, ip, pp, vp, sz,
                                 C.POINTER(lls_options), vp]
    lib.lls_backward.restype = i
    lib.lls_solve_batched_workspace_size.argtypes = [i, ip, ip, C.POINTER(lls_options)]
    lib.lls_solve_batched_workspace_size.restype = sz
    lib.lls_solve_batched.argtypes = [i, ip, ip, pp, ip, pp, pp, pp, ip, vp, sz, C.POINTER(lls_options),
                                      C.POINTER(lls_info), vp]
    lib.lls_solve_batched.restype = i
    tp = C.POINTER(lls_tuning)
    lib.lls_autotune_workspace_size.argtypes = [i, i, C.POINTER(lls_options)]
    lib.lls_autotune_workspace_size.restype = sz
    lib.lls_autotune.argtypes = [i, i, vp, i, vp, vp, vp, sz, C.POINTER(lls_options), i, tp, vp]
    lib.lls_autotune.restype = i
    lib.lls_autotune_batched.argtypes = [i, ip, ip, pp, ip, pp, pp, vp, sz, C.POINTER(lls_options), i, tp, vp]
    lib.lls_autotune_batched.restype = i
    lib.lls_tuning_set.argtypes = [i, i, i, C.POINTER(lls_options), tp]
    lib.lls_tuning_set.restype = i
    lib.lls_tuning_get.argtypes = [i, i, i, C.POINTER(lls_options), tp]
    lib.lls_tuning_get.restype = i
    lib.lls_tuning_clear.argtypes = []
    lib.lls_tuning_clear.restype = None
    lib.lls_debug_build.argtypes = []
    lib.lls_debug_build.restype = i
    lib.lls_debug_inject.argtypes = [i]
    lib.lls_debug_inject.restype = i
    _lib = lib
    return lib


def default_options() -> lls_options:
    """The library's defaults (lls_default_options)."""
    o = lls_options()
    load().lls_default_options(C.byref(o))
    return o


def make_options(prec="fp16", target="fp64", tol=0.0, max_iter=200, panel_width=0,
                 krylov="cgls", leaf_rows=256, reorth=0, panel_leaf="cgs2", x0="zero") -> lls_options:
    o = lls_options()
    load().lls_default_options(C.byref(o))
    o.gemm_prec = PREC[prec] if isinstance(prec, str) else int(prec)
    o.target = TARGET[target] if isinstance(target, str) else int(target)
    o.tol = float(tol)
    o.max_iter = int(max_iter)
    o.panel_width = int(panel_width)
    o.krylov = KRYLOV[krylov] if isinstance(krylov, str) else int(krylov)
    o.leaf_rows = int(leaf_rows)
    o.reorth = int(reorth)
    o.panel_leaf = PANEL_LEAF[panel_leaf] if isinstance(panel_leaf, str) else int(panel_leaf)
    o.x0 = X0[x0] if isinstance(x0, str) else int(x0)
    return o


# ---- raw C entry points (same names as the C ABI) ------------------------------------------

def lls_default_options() -> lls_options:
    o = lls_options()
    load().lls_default_options(C.byref(o))
    return o


def lls_status_string(status: int) -> str:
    return load().lls_status_string(int(status)).decode()


def lls_kernel_launch_count() -> int:
    return int(load().lls_kernel_launch_count())


def qr_factor_workspace_size(m, n, opts=None) -> int:
    return load().qr_factor_workspace_size(m, n, C.byref(opts) if opts is not None else None)


def qr_factor(m, n, A, lda, Q, ldq, R, ldr, ws, ws_bytes, opts, stream) -> int:
    return load().qr_factor(m, n, A, lda, Q, ldq, R, ldr, ws, ws_bytes,
                            C.byref(opts) if opts is not None else None, stream)


def lls_solve_workspace_size(m, n, opts=None) -> int:
    return load().lls_solve_workspace_size(m, n, C.byref(opts) if opts is not None else None)


def lls_solve(m, n, A, lda, b, x, R_out, ldr, ws, ws_bytes, opts, info, stream) -> int:
    return load().lls_solve(m, n, A, lda, b, x, R_out, ldr, ws, ws_bytes,
                            C.byref(opts) if opts is not None else None,
                            C.byref(info) if info is not None else None, stream)


def lls_upload_chunks(n):
    """Column boundaries of lls_solve_host's upload chunks (a list starting at 0, ending at n)."""
    buf = (C.c_int * 64)()
    count = load().lls_upload_chunks(n, buf, 64)
    if count < 0:
        raise LLSError(count, "lls_upload_chunks")
    return list(buf[:count + 1])


def lls_selftest_wait_timeout(ws, ws_bytes, stream) -> int:
    return load().lls_selftest_wait_timeout(ws, ws_bytes, stream)


def lls_solve_host_workspace_size(m, n, opts=None) -> int:
    return load().lls_solve_host_workspace_size(m, n, C.byref(opts) if opts is not None else None)


def lls_solve_host(m, n, A, lda, b, x, ws, ws_bytes, opts, info, stream) -> int:
    return load().lls_solve_host(m, n, A, lda, b, x, ws, ws_bytes,
                                 C.byref(opts) if opts is not None else None,
                                 C.byref(info) if info is not None else None, stream)


def lls_lowp_projection_workspace_size(m, w1, w2) -> int:
    return load().lls_lowp_projection_workspace_size(m, w1, w2)


def lls_lowp_projection(m, w1, w2, prec, Q1l, A2l, ldh, e, R12, ldr, R12l, ldrl, f, ws, ws_bytes,
                        stream) -> int:
    return load().lls_lowp_projection(m, w1, w2, prec, Q1l, A2l, ldh, e, R12, ldr, R12l, ldrl, f,
                                      ws, ws_bytes, stream)


def lls_panel_qr_workspace_size(m, b) -> int:
    return load().lls_panel_qr_workspace_size(m, b)


def lls_panel_qr(m, b, prec, W, ldw, Wh, ldh, R, ldr, ws, ws_bytes, stream) -> int:
    return load().lls_panel_qr(m, b, prec, W, ldw, Wh, ldh, R, ldr, ws, ws_bytes, stream)


def lls_panel_block_qr_workspace_size(m, w1, w2) -> int:
    return load().lls_panel_block_qr_workspace_size(m, w1, w2)


def lls_panel_block_qr(m, w1, w2, prec, W, ldw, Wh, ldh, R, ldr, ws, ws_bytes, stream) -> int:
    return load().lls_panel_block_qr(m, w1, w2, prec, W, ldw, Wh, ldh, R, ldr, ws, ws_bytes, stream)


def lls_householder_workspace_size(m, n, prec) -> int:
    return load().lls_householder_workspace_size(m, n, prec)


def lls_householder_solve(m, n, prec, A, lda, b, x, ws, ws_bytes, stream) -> int:
    return load().lls_householder_solve(m, n, prec, A, lda, b, x, ws, ws_bytes, stream)


def householder_solve(A, b, prec="fp64", stream=None):
    """x of min ||A x - b|| by the plain Householder solver (FP64 or FP32 arithmetic)."""
    torch = _torch()
    _check_colmajor(A)
    m, n = A.shape
    nb = lls_householder_workspace_size(m, n, PREC[prec])
    if nb == 0:
        raise LLSError(-1, "lls_householder_workspace_size")
    ws = workspace(nb, A.device)
    x = torch.empty(n, dtype=torch.float64, device=A.device)
    s = stream if stream is not None else torch.cuda.current_stream(A.device).cuda_stream
    st = lls_householder_solve(m, n, PREC[prec], A.data_ptr(), A.stride(1), b.data_ptr(), x.data_ptr(),
                               ws.data_ptr(), ws.numel(), s)
    if st < 0:
        raise LLSError(st, "lls_householder_solve")
    return x


def lls_lowp_projection_noalloc(m, w1, w2, prec, Q1l, A2l, ldh, e, R12, ldr, R12l, ldrl, f, stream) -> int:
    """lls_lowp_projection with the library's fixed device scratch instead of a workspace."""
    return load().lls_lowp_projection_noalloc(m, w1, w2, prec, Q1l, A2l, ldh, e, R12, ldr, R12l, ldrl, f,
                                              stream)


def lls_lowp_update(m, w1, w2, prec, Q1l, ldh, R12l, ldrl, f, A2, lda, ws, ws_bytes, stream) -> int:
    return load().lls_lowp_update(m, w1, w2, prec, Q1l, ldh, R12l, ldrl, f, A2, lda, ws, ws_bytes,
                                  stream)


def _ints(v):
    return (C.c_int * len(v))(*[int(t) for t in v])


def _ptrs(v):
    return (C.c_void_p * len(v))(*[int(t) if t else None for t in v])


def lls_backward_workspace_size(batch, m, n, opts=None) -> int:
    return load().lls_backward_workspace_size(batch, _ints(m), _ints(n),
                                              C.byref(opts) if opts is not None else None)


def lls_backward(batch, m, n, A, lda, b, x, R, ldr, grad_x, grad_A, ldga, grad_b, ws, ws_bytes,
                 opts, stream) -> int:
    """m, n, lda, ldr, ldga: int sequences; A ... grad_b: sequences of device pointers."""
    return load().lls_backward(batch, _ints(m), _ints(n), _ptrs(A), _ints(lda), _ptrs(b), _ptrs(x),
                               _ptrs(R), _ints(ldr), _ptrs(grad_x), _ptrs(grad_A), _ints(ldga),
                               _ptrs(grad_b), ws, ws_bytes, C.byref(opts) if opts is not None else None,
                               stream)


def lls_solve_batched_workspace_size(batch, m, n, opts=None) -> int:
    return load().lls_solve_batched_workspace_size(batch, _ints(m), _ints(n),
                                                   C.byref(opts) if opts is not None else None)


def lls_solve_batched(batch, m, n, A, lda, b, x, R_out, ldr, ws, ws_bytes, opts, infos, stream) -> int:
    """m, n, lda, ldr: int sequences; A, b, x, R_out: sequences of device pointers (R_out may be
    None); infos: a ctypes array of lls_info or None."""
    return load().lls_solve_batched(batch, _ints(m), _ints(n), _ptrs(A), _ints(lda), _ptrs(b), _ptrs(x),
                                    _ptrs(R_out) if R_out is not None else None,
                                    _ints(ldr) if ldr is not None else None, ws, ws_bytes,
                                    C.byref(opts) if opts is not None else None, infos, stream)


def lls_autotune_workspace_size(m, n, opts=None) -> int:
    return load().lls_autotune_workspace_size(m, n, C.byref(opts) if opts is not None else None)


def lls_autotune(m, n, A, lda, b, x, ws, ws_bytes, opts, reps, best, stream) -> int:
    return load().lls_autotune(m, n, A, lda, b, x, ws, ws_bytes, C.byref(opts) if opts is not None else None,
                               reps, C.byref(best), stream)


def lls_autotune_batched(batch, m, n, A, lda, b, x, ws, ws_bytes, opts, reps, best, stream) -> int:
    return load().lls_autotune_batched(batch, _ints(m), _ints(n), _ptrs(A), _ints(lda), _ptrs(b), _ptrs(x), ws,
                                       ws_bytes, C.byref(opts) if opts is not None else None, reps,
                                       C.byref(best), stream)


def lls_tuning_set(kind, m, n, opts, tuning) -> int:
    return load().lls_tuning_set(kind, m, n, C.byref(opts) if opts is not None else None, C.byref(tuning))


def lls_tuning_get(kind, m, n, opts=None):
    """The recorded lls_tuning for the key, or None."""
    t = lls_tuning()
    r = load().lls_tuning_get(kind, m, n, C.byref(opts) if opts is not None else None, C.byref(t))
    return t if r == 1 else None


def lls_tuning_clear() -> None:
    load().lls_tuning_clear()


# ---- torch helpers (allocation and pointer passing only) -----------------------------------

def _torch():
    import torch
    return torch


def colmajor(A, dtype=None, device="cuda"):
    """Column-major copy of a 2-D array/tensor on the device: shape (m, n), strides (1, m)."""
    torch = _torch()
    t = torch.as_tensor(A)
    dtype = dtype or torch.float32
    out = torch.empty((t.shape[1], t.shape[0]), dtype=dtype, device=device).t()
    out.copy_(t.to(device=device, dtype=dtype))
    return out


def _check_colmajor(A):
    assert A.dim() == 2 and A.stride(0) == 1 and A.stride(1) >= A.shape[0], "A must be column-major"


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def workspace(nbytes: int, device="cuda"):
    torch = _torch()
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


# ---- tuned settings: the library's table, saved to and restored from the JSON cache ----------

_tuning_loaded = set()


def _device_ident(device):
    torch = _torch()
    props = torch.cuda.get_device_properties(device)
    return props.name, props.multi_processor_count


def _opt_ints(o):
    return {f: int(getattr(o, f)) for f in ("gemm_prec", "target", "krylov", "reorth", "panel_leaf")}


def load_tuning_cache(device=None, path=None):
    """Restore the settings saved for this GPU model into the library's table (once per device
    and process); returns the number restored."""
    from . import tuning
    torch = _torch()
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    idx = dev.index if dev.index is not None else torch.cuda.current_device()
    if (idx, path) in _tuning_loaded:
        return 0
    _tuning_loaded.add((idx, path))
    name, sms = _device_ident(idx)
    count = 0
    with torch.cuda.device(idx):
        for kind, m, n, opts, t in tuning.entries_for_device(tuning.load(path), name, sms):
            o = lls_default_options()
            for f, v in opts.items():
                setattr(o, f, v)
            rec = lls_tuning(int(t["panel_width"]), int(t["node_mode"]), int(t["gemm_kernel"]),
                             int(t["batched_ctas_per_sm"]), int(t.get("krylov_ctas", 0)), float(t["ms"]))
            if lls_tuning_set(kind, m, n, o, rec) == 0:
                count += 1
    return count


def _save_tuning(kind, m, n, o, best, device, path=None):
    from . import tuning
    name, sms = _device_ident(device)
    try:
        tuning.record(tuning.make_key(name, sms, kind, m, n, _opt_ints(o)), best.as_dict(), path)
    except OSError:
        pass      # a read-only cache location: the setting stays in the process's table


def autotune(A, b, prec="fp16", target="fp64", krylov="cgls", reorth=0, panel_leaf="cgs2", reps=2, stream=None,
             cache=True, cache_path=None):
    """Measure the implementation choices for this problem's shape (lls_autotune), record the
    fastest in the library's table and, with cache=True, in the JSON cache. Returns it as a dict."""
    torch = _torch()
    _check_colmajor(A)
    m, n = A.shape
    o = make_options(prec=prec, target=target, krylov=krylov, reorth=reorth, panel_leaf=panel_leaf)
    nb = lls_autotune_workspace_size(m, n, o)
    if nb == 0:
        raise LLSError(-1, "lls_autotune_workspace_size")
    ws = workspace(nb, A.device)
    bb = b.to(device=A.device, dtype=torch.float64).contiguous()
    x = torch.empty(n, dtype=torch.float64, device=A.device)
    best = lls_tuning()
    st = lls_autotune(m, n, A.data_ptr(), A.stride(1), bb.data_ptr(), x.data_ptr(), ws.data_ptr(), ws.numel(), o,
                      int(reps), best, _stream(stream))
    if st != 0:
        raise LLSError(st, "lls_autotune")
    if cache:
        _save_tuning(0, m, n, o, best, A.device, cache_path)
    return best.as_dict()


def autotune_batched(As, bs, prec="fp16", target="fp32", reps=2, stream=None, cache=True, cache_path=None):
    """lls_autotune_batched for a list of problems (column-major FP32 A_i, FP64 b_i)."""
    torch = _torch()
    batch = len(As)
    ms = [A.shape[0] for A in As]
    ns = [A.shape[1] for A in As]
    o = make_options(prec=prec, target=target, panel_width=16)
    nb = lls_solve_batched_workspace_size(batch, ms, ns, o)
    if nb == 0:
        raise LLSError(-6, "lls_solve_batched_workspace_size")
    dev = As[0].device
    ws = workspace(nb, dev)
    bs = [b.to(device=dev, dtype=torch.float64).contiguous() for b in bs]
    xs = [torch.empty(n_, dtype=torch.float64, device=dev) for n_ in ns]
    best = lls_tuning()
    st = lls_autotune_batched(batch, ms, ns, [A.data_ptr() for A in As], [A.stride(1) for A in As],
                              [b.data_ptr() for b in bs], [x.data_ptr() for x in xs], ws.data_ptr(), ws.numel(), o,
                              int(reps), best, _stream(stream))
    if st != 0:
        raise LLSError(st, "lls_autotune_batched")
    if cache:
        _save_tuning(1, batch, max(ns), o, best, dev, cache_path)
    return best.as_dict()


def qr(A, prec="fp16", panel_width=0, want_q=True, ws=None, stream=None, reorth=0, panel_leaf="cgs2"):
    """(Q, R) of a column-major FP32 device matrix A (m x n). Q is None when want_q is False.
    panel_width 0 uses the setting recorded for the shape (lls_autotune), if any."""
    torch = _torch()
    _check_colmajor(A)
    load_tuning_cache(A.device)
    m, n = A.shape
    o = make_options(prec=prec, panel_width=panel_width, reorth=reorth, panel_leaf=panel_leaf)
    nb = qr_factor_workspace_size(m, n, o)
    if nb == 0:
        raise LLSError(-1, "qr_factor_workspace_size")
    ws = ws if ws is not None and ws.numel() >= nb else workspace(nb, A.device)
    R = torch.empty((n, n), dtype=torch.float32, device=A.device).t()
    Q = torch.empty((n, m), dtype=torch.float32, device=A.device).t() if want_q else None
    st = qr_factor(m, n, A.data_ptr(), A.stride(1), Q.data_ptr() if want_q else None, m,
                   R.data_ptr(), n, ws.data_ptr(), ws.numel(), o, _stream(stream))
    if st != 0:
        raise LLSError(st, "qr_factor")
    return Q, R


def solve(A, b, prec="fp16", target="fp64", tol=0.0, max_iter=200, panel_width=0,
          krylov="cgls", want_r=False, ws=None, stream=None, check=True, reorth=0, panel_leaf="cgs2",
          x0=None):
    """x = argmin ||A x - b|| for column-major FP32 A (m x n) and FP64 b on the device.

    x0: None (start from zero), "direct" (start from R^{-1} Q^T b) or a vector (warm start).
    panel_width 0 uses the setting recorded for the shape (lls_autotune), if any.
    Returns (x, info_dict[, R]). Synchronizes the stream (to fill info)."""
    torch = _torch()
    _check_colmajor(A)
    load_tuning_cache(A.device)
    m, n = A.shape
    mode = "zero" if x0 is None else ("direct" if isinstance(x0, str) and x0 == "direct" else "given")
    o = make_options(prec=prec, target=target, tol=tol, max_iter=max_iter,
                     panel_width=panel_width, krylov=krylov, reorth=reorth, panel_leaf=panel_leaf, x0=mode)
    nb = lls_solve_workspace_size(m, n, o)
    if nb == 0:
        raise LLSError(-1, "lls_solve_workspace_size")
    ws = ws if ws is not None and ws.numel() >= nb else workspace(nb, A.device)
    b = b.to(device=A.device, dtype=torch.float64).contiguous()
    if mode == "given":
        x = torch.as_tensor(x0).to(device=A.device, dtype=torch.float64).clone().contiguous()
    else:
        x = torch.empty(n, dtype=torch.float64, device=A.device)
    R = torch.empty((n, n), dtype=torch.float32, device=A.device).t() if want_r else None
    info = lls_info()
    st = lls_solve(m, n, A.data_ptr(), A.stride(1), b.data_ptr(), x.data_ptr(),
                   R.data_ptr() if want_r else None, n, ws.data_ptr(), ws.numel(), o, info,
                   _stream(stream))
    if check and st < 0:
        raise LLSError(st, "lls_solve")
    d = info.as_dict()
    d["status_code"] = st
    return (x, d, R) if want_r else (x, d)


def backward(As, bs, xs, Rs, gxs, prec="fp16", target="fp64", max_iter=200, stream=None):
    """Adjoint for a list of problems: returns (grad_As, grad_bs) as column-major FP32 and FP64
    device tensors. As: column-major FP32 (m, n); bs, xs, gxs: FP64 vectors; Rs: (n, n) FP32."""
    torch = _torch()
    batch = len(As)
    ms = [A.shape[0] for A in As]
    ns = [A.shape[1] for A in As]
    o = make_options(prec=prec, target=target, max_iter=max_iter)
    nb = lls_backward_workspace_size(batch, ms, ns, o)
    if nb == 0:
        raise LLSError(-1, "lls_backward_workspace_size")
    dev = As[0].device
    ws = workspace(nb, dev)
    gAs = [torch.empty((n_, m_), dtype=torch.float32, device=dev).t() for m_, n_ in zip(ms, ns)]
    gbs = [torch.empty(m_, dtype=torch.float64, device=dev) for m_ in ms]
    bs = [b.to(device=dev, dtype=torch.float64).contiguous() for b in bs]
    xs = [x.to(device=dev, dtype=torch.float64).contiguous() for x in xs]
    gxs = [g.to(device=dev, dtype=torch.float64).contiguous() for g in gxs]
    for A in As:
        _check_colmajor(A)
    for R in Rs:
        _check_colmajor(R)
    st = lls_backward(batch, ms, ns, [A.data_ptr() for A in As], [A.stride(1) for A in As],
                      [b.data_ptr() for b in bs], [x.data_ptr() for x in xs],
                      [R.data_ptr() for R in Rs], [R.stride(1) for R in Rs],
                      [g.data_ptr() for g in gxs], [g.data_ptr() for g in gAs],
                      [g.stride(1) for g in gAs], [g.data_ptr() for g in gbs],
                      ws.data_ptr(), ws.numel(), o, _stream(stream))
    if st != 0:
        raise LLSError(st, "lls_backward")
    return gAs, gbs


class _LstsqFunction:
    """Namespace holder; the autograd Function is created lazily so importing this module
    does not import torch."""
    fn = None


def _make_function():
    torch = _torch()

    class LLSFunction(torch.autograd.Function):
        """x = argmin ||A x - b||_2 for A (m, n) or a batch (B, m, n); differentiable in A and b.

        Forward: lls_solve (RGSQRF + preconditioned CGLS), or lls_solve_batched for a batch (one
        persistent launch). Backward: lls_backward (the textbook adjoint, with
        z = (A^T A)^{-1} g from CG preconditioned by the forward R; a batch in one launch)."""

        @staticmethod
        def forward(ctx, A, b, opts):
            batched = A.dim() == 3
            As = list(A) if batched else [A]
            bs = list(b) if batched else [b]
            Acm = [colmajor(a.detach(), device=a.device) for a in As]
            if batched and len(As) > 1:
                # the whole batch in one persistent launch
                bopts = {k: v for k, v in opts.items() if k in ("prec", "target", "tol", "max_iter")}
                xs, infos, Rs = solve_batched(Acm, [bv.detach() for bv in bs], want_r=True,
                                              **{"target": "fp64", **bopts})
                for info in infos:
                    if info["status"] < 0:
                        raise LLSError(info["status"], "lls_solve_batched")
            else:
                xs, Rs = [], []
                for a_cm, bv in zip(Acm, bs):
                    x, info, R = solve(a_cm, bv.detach(), want_r=True, **opts)
                    if info["status_code"] < 0:
                        raise LLSError(info["status_code"], "lls_solve")
                    xs.append(x)
                    Rs.append(R)
            ctx.batched = batched
            ctx.opts = opts
            ctx.bdtype = b.dtype
            ctx.Adtype = A.dtype
            ctx.Acm, ctx.Rs = Acm, Rs
            ctx.save_for_backward(b, *xs)
            x = torch.stack(xs) if batched else xs[0]
            return x.to(b.dtype)

        @staticmethod
        def backward(ctx, gx):
            b = ctx.saved_tensors[0]
            xs = list(ctx.saved_tensors[1:])
            bs = list(b) if ctx.batched else [b]
            gxs = list(gx) if ctx.batched else [gx]
            gAs, gbs = backward(ctx.Acm, bs, xs, ctx.Rs, gxs, prec=ctx.opts.get("prec", "fp16"),
                                target=ctx.opts.get("target", "fp64"),
                                max_iter=ctx.opts.get("max_iter", 200))
            gA = torch.stack(gAs) if ctx.batched else gAs[0]
            gb = torch.stack(gbs) if ctx.batched else gbs[0]
            return gA.to(ctx.Adtype), gb.to(ctx.bdtype), None

    return LLSFunction


def lstsq(A, b, **opts):
    """Differentiable least-squares solve on the GPU (see LLSFunction)."""
    if _LstsqFunction.fn is None:
        _LstsqFunction.fn = _make_function()
    return _LstsqFunction.fn.apply(A, b, opts)


def solve_batched(As, bs, prec="fp16", target="fp32", tol=0.0, max_iter=200, want_r=False, ws=None,
                  stream=None, check=True):
    """Solve a list of independent problems in one persistent launch.

    As: column-major FP32 device matrices (m_i, n_i); bs: FP64 device vectors.
    Returns (xs, infos[, Rs]) with infos a list of dicts."""
    torch = _torch()
    batch = len(As)
    for A in As:
        _check_colmajor(A)
    load_tuning_cache(As[0].device)
    ms = [A.shape[0] for A in As]
    ns = [A.shape[1] for A in As]
    o = make_options(prec=prec, target=target, tol=tol, max_iter=max_iter, panel_width=0)
    nb = lls_solve_batched_workspace_size(batch, ms, ns, o)
    if nb == 0:
        raise LLSError(-6, "lls_solve_batched_workspace_size")
    dev = As[0].device
    ws = ws if ws is not None and ws.numel() >= nb else workspace(nb, dev)
    bs = [b.to(device=dev, dtype=torch.float64).contiguous() for b in bs]
    xs = [torch.empty(n_, dtype=torch.float64, device=dev) for n_ in ns]
    Rs = [torch.empty((n_, n_), dtype=torch.float32, device=dev).t() for n_ in ns] if want_r else None
    infos = (lls_info * batch)()
    st = lls_solve_batched(batch, ms, ns, [A.data_ptr() for A in As], [A.stride(1) for A in As],
                           [b.data_ptr() for b in bs], [x.data_ptr() for x in xs],
                           [R.data_ptr() for R in Rs] if want_r else None,
                           ns if want_r else None, ws.data_ptr(), ws.numel(), o, infos, _stream(stream))
    if check and st < 0:
        raise LLSError(st, "lls_solve_batched")
    out = [infos[i].as_dict() for i in range(batch)]
    return (xs, out, Rs) if want_r else (xs, out)
