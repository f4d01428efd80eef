"""The entrywise R predicate of the GPU parity tests sees a localized mistake that the
normwise predicate lets through (checked on the oracle's own factors, on the CPU)."""
import numpy as np

from oracle import rgsqrf
from paper_1912_05508_gb300 import synth
from parity import r_entry_err

U16 = 2.0 ** -11


def test_one_wrong_tile_is_seen_entrywise_not_normwise():
    A = synth.svd_lls(3000, 256, "geometric", 1e3, seed=8, noise=0.0).A
    _, Ro = rgsqrf.rgsqrf(A, 16, "fp16", leaf_rows=256)
    # one 16 x 16 tile of R12 off by 6 u16 of its columns' norms
    R = Ro.copy()
    cn = np.linalg.norm(Ro, axis=0)
    R[32:48, 160:176] += 6 * U16 * cn[None, 160:176]
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= 8 * U16      # the normwise bound passes
    assert r_entry_err(R, Ro) > 4 * U16                                 # the entrywise bound does not
    assert r_entry_err(Ro, Ro) == 0.0


def test_zero_column_counts_absolute_differences():
    Ro = np.triu(np.ones((4, 4)))
    Ro[:, 2] = 0.0
    R = Ro.copy()
    R[1, 2] = 1e-3
    assert r_entry_err(R, Ro) == 1e-3
