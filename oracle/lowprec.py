"""Rounding operations applied to the inputs of the low-precision tensor-core products.

Test infrastructure only. The paper runs the two products of each recursion
step (Alg. 2, R12 = Q1^T A2 and A2 - Q1 R12) as FP16 TensorCore GEMMs with FP32
accumulation (Sec. 2.1, Sec. 3.1.2) and notes FP16's narrow range (Sec. 2.1).
It does not say how range is handled; the reading used here is an exact
power-of-two scale per column chosen from the column's largest magnitude,
which changes no significand bit, so unscaling the product is exact. The optional
FP8 (E4M3) products use the same kind of scale, on both operands.

All functions take FP64 arrays and return FP64 arrays holding values exactly
representable in the target format.
"""
from __future__ import annotations

import numpy as np

# Target of the scaled column maximum: [2^14, 2^15) for FP16 (largest finite 65504).
FP16_TARGET_EXP = 15      # max|x| * 2^e has frexp exponent 15, i.e. lies in [2^14, 2^15)
# FP8 E4M3 (largest finite 448 = 1.75 * 2^8): the scaled maximum lies in [2^7, 2^8).
FP8_TARGET_EXP = 8
FP8_MAX = 448.0
SCALE_EXP_LIMIT = 100     # |e| is clamped so 2^e stays a normal FP32 number


def round_fp16(x: np.ndarray) -> np.ndarray:
    """Round to IEEE binary16, round-to-nearest-even, overflow to inf (numpy's cast)."""
    return np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round to bfloat16 (8-bit significand), round-to-nearest-even.

    Done in two steps, as the GPU does it: the value is first an FP32 number
    (here: rounded to FP32), then its low 16 bits are rounded away with ties to
    even on the bit pattern.
    """
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    rounded = (u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)
    nan = np.isnan(f)
    out = (rounded << np.uint64(16)).astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def round_fp8_e4m3(x: np.ndarray) -> np.ndarray:
    """Round to FP8 E4M3 (4 exponent bits, bias 7, 3 significand bits), round-to-nearest-even,
    saturating to +-448 (the GPU conversion's satfinite mode).

    Normal numbers |x| >= 2^-6 have 3 fraction bits, so the spacing in [2^k, 2^(k+1)) is
    2^(k-3); below 2^-6 the subnormal spacing is 2^-9. x / spacing is exact (a power of two),
    and numpy's round is half-to-even."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    _, ex = np.frexp(a)                          # a = f * 2^ex, f in [0.5, 1): floor(log2 a) = ex - 1
    qexp = np.maximum(ex - 1, -6) - 3
    r = np.round(np.ldexp(a, -qexp))
    out = np.minimum(np.ldexp(r, qexp), FP8_MAX)
    out = np.copysign(out, x)
    out[np.isnan(x)] = np.nan
    return out


def round_to(prec: str, x: np.ndarray) -> np.ndarray:
    if prec == "fp16":
        return round_fp16(x)
    if prec == "fp8":
        return round_fp8_e4m3(x)
    if prec == "bf16":
        return round_bf16(x)
    if prec in ("fp32", "fp64"):
        return np.asarray(x, dtype=np.float64)
    raise ValueError(prec)


def column_scale_exponents(X: np.ndarray, prec: str) -> np.ndarray:
    """Per-column exponent e_j so that max_i |X_ij| * 2^e_j lies in [2^14, 2^15) (FP16) or
    [2^7, 2^8) (FP8 E4M3).

    BF16 has FP32's exponent range and FP32/FP64 need none, so e_j = 0 there.
    An all-zero column gets e_j = 0. e_j is clamped to [-100, 100].
    """
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[1]
    if prec not in ("fp16", "fp8"):
        return np.zeros(n, dtype=np.int64)
    target = FP16_TARGET_EXP if prec == "fp16" else FP8_TARGET_EXP
    mx = np.max(np.abs(X), axis=0) if X.shape[0] else np.zeros(n)
    _, ex = np.frexp(mx)                      # mx = f * 2^ex, f in [0.5, 1)
    e = (target - ex).astype(np.int64)
    e[mx == 0] = 0
    return np.clip(e, -SCALE_EXP_LIMIT, SCALE_EXP_LIMIT)


def scaled_round(X: np.ndarray, prec: str) -> tuple[np.ndarray, np.ndarray]:
    """(X_low, e): X_low = round(X * 2^e) column by column, e from column_scale_exponents."""
    e = column_scale_exponents(X, prec)
    return round_to(prec, np.ldexp(np.asarray(X, dtype=np.float64), e[None, :])), e
