"""The reduction the many-right-hand-side step uses before its radix select, checked by brute force.

H_s keeps the s largest keys, ties to the lower index. For any set G of s entries (the current
support), the s-th largest key is at least the smallest key on G: those s keys are all at least
their own minimum. So H_s over all n keys equals H_s over G and the entries off G whose key is at
least that minimum. The kernel lists G and those entries and selects among them only. This test
compares the two selections on random keys with many exact ties (keys drawn from a few values),
random supports G, and the degenerate cases of a support holding the s smallest keys and of all
keys equal.
"""
import numpy as np


def top_s(keys: np.ndarray, idx: np.ndarray, s: int) -> np.ndarray:
    """The s largest of keys[idx], ties to the lower index; the chosen indices, ascending."""
    order = sorted(idx.tolist(), key=lambda j: (-int(keys[j]), j))
    return np.array(sorted(order[:s]), dtype=np.int64)


def reduced(keys: np.ndarray, support: np.ndarray, s: int) -> np.ndarray:
    kmin = keys[support].min()
    off = np.setdiff1d(np.arange(keys.size), support)
    cand = off[keys[off] >= kmin]
    return top_s(keys, np.concatenate([support, cand]), s)


def test_candidates_hold_the_selection():
    rng = np.random.Generator(np.random.PCG64(5))
    for trial in range(400):
        n = int(rng.integers(2, 300))
        s = int(rng.integers(1, n + 1))
        nvals = int(rng.integers(1, 12))                 # few distinct values: many exact ties
        keys = rng.integers(0, nvals, n).astype(np.uint32)
        support = rng.choice(n, s, replace=False)
        full = top_s(keys, np.arange(n), s)
        assert np.array_equal(reduced(keys, support, s), full), (trial, n, s)


def test_degenerate_supports():
    rng = np.random.Generator(np.random.PCG64(6))
    for n, s in ((50, 10), (64, 64), (7, 1)):
        keys = rng.permutation(n).astype(np.uint32)
        worst = np.argsort(keys, kind="stable")[:s]     # the support on the s smallest keys
        assert np.array_equal(reduced(keys, worst, s), top_s(keys, np.arange(n), s))
        same = np.full(n, 3, dtype=np.uint32)           # all keys equal: the s lowest indices
        sup = rng.choice(n, s, replace=False)
        assert np.array_equal(reduced(same, sup, s), np.arange(s))
