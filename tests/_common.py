"""Helpers shared by the GPU parity tests (comparison logic only, no method arithmetic)."""
import numpy as np


def csc_to_slots(colptr, rowidx, val, s):
    """CSC (numpy) -> (idx (m, s) with -1 padding, val (m, s), cnt (m,))."""
    colptr = np.asarray(colptr, np.int64)
    m = len(colptr) - 1
    cnt = np.diff(colptr).astype(np.int32)
    nnz = int(colptr[-1])
    idx = np.full((m, s), -1, np.int32)
    vals = np.zeros((m, s), np.float64)
    if nnz:
        col = np.repeat(np.arange(m), cnt)
        pos = np.arange(nnz) - np.repeat(colptr[:-1], cnt)
        idx[col, pos] = np.asarray(rowidx[:nnz])
        vals[col, pos] = np.asarray(val[:nnz], np.float64)
    return idx, vals, cnt


def compare_supports(idx_g, cnt_g, idx_o, cnt_o, gaps_o, tie_rel=1e-5):
    """Count signals whose supports differ, and those not explained by a near-tie
    (the oracle met a top-two relative gap below tie_rel at some step)."""
    same = np.all(idx_g == idx_o, axis=1) & (cnt_g == cnt_o)
    diff = ~same
    near_tie = np.min(gaps_o, axis=1) < tie_rel
    return int(diff.sum()), int((diff & ~near_tie).sum()), same


def assert_support_parity(idx_g, cnt_g, idx_o, cnt_o, gaps_o, frac=0.999, tie_rel=1e-5):
    """Supports identical on >= frac of the signals, and every mismatch explained
    by a near-tie of the top two correlations (relative gap < tie_rel)."""
    m = len(cnt_o)
    ndiff, nbad, same = compare_supports(idx_g, cnt_g, idx_o, cnt_o, gaps_o, tie_rel)
    assert m - ndiff >= frac * m, f"{ndiff} of {m} supports differ"
    assert nbad == 0, f"{nbad} of {m} supports differ without a near-tie"
    return same
