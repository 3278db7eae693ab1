"""Exact cardinalities over a window of slices, and detection error rates --
TEST INFRASTRUCTURE ONLY (and the accuracy leg of the benchmark).

The cardinality of a host in window W(t, k) is the number of distinct
opposite hosts it talked to in the slices of that window (Sec. 2.1); a super
point is a host whose cardinality is at least theta.  FPR and FNR follow the
definition of Sec. 5: with N true super points, N+ reported hosts that are
not super points and N- super points not reported, FPR = N+/N, FNR = N-/N,
and FTR = FPR + FNR."""
from __future__ import annotations

import numpy as np


def slice_keys(pairs: np.ndarray) -> np.ndarray:
    """The distinct (aip, bip) pairs of one slice, as sorted uint64 keys."""
    p = np.ascontiguousarray(pairs, dtype=np.uint32).reshape(-1, 2)
    return np.unique((p[:, 0].astype(np.uint64) << np.uint64(32)) | p[:, 1].astype(np.uint64))


def window_cardinalities(keys_per_slice) -> tuple[np.ndarray, np.ndarray]:
    """(hosts, cardinalities) over the union of the slices' distinct pairs."""
    allk = np.unique(np.concatenate(list(keys_per_slice))) if keys_per_slice else np.zeros(0, np.uint64)
    hosts, counts = np.unique((allk >> np.uint64(32)).astype(np.uint32), return_counts=True)
    return hosts, counts


def super_points(keys_per_slice, theta: int) -> set:
    hosts, counts = window_cardinalities(keys_per_slice)
    return set(hosts[counts >= theta].tolist())


def error_rates(reported: set, true_super: set) -> dict:
    """FPR, FNR and FTR of Sec. 5 for one window (None if there is no super
    point in it)."""
    n = len(true_super)
    n_plus = len(reported - true_super)
    n_minus = len(true_super - reported)
    if n == 0:
        return {"n": 0, "n_plus": n_plus, "n_minus": 0, "fpr": None, "fnr": None, "ftr": None}
    return {"n": n, "n_plus": n_plus, "n_minus": n_minus, "fpr": n_plus / n, "fnr": n_minus / n,
            "ftr": (n_plus + n_minus) / n}
