"""Pins of the exact window cardinalities (oracle/truth.py) against a plain
set-based count, and of the error rates against the definition of Sec. 5."""
import numpy as np

import synth
from oracle import truth


def test_window_cardinalities_match_sets():
    slices = [synth.random_pairs(4, t, 3000, n_hosts=50, n_bips=400) for t in range(6)]
    keys = [truth.slice_keys(p) for p in slices]
    for lo in range(3):
        hosts, counts = truth.window_cardinalities(keys[lo:lo + 3])
        seen = {}
        for p in slices[lo:lo + 3]:
            for a, b in p.tolist():
                seen.setdefault(a, set()).add(b)
        assert sorted(seen) == hosts.tolist()
        assert [len(seen[a]) for a in hosts.tolist()] == counts.tolist()
        assert truth.super_points(keys[lo:lo + 3], 30) == {a for a, s in seen.items() if len(s) >= 30}


def test_planted_hosts_have_their_constructed_cardinality():
    """tiny_b's planted hosts emit every member of their sets in every slice:
    their window cardinality is the set size, by construction."""
    w = synth.workload("tiny_b")
    keys = [truth.slice_keys(w.pairs(t)) for t in range(w.k)]
    hosts, counts = truth.window_cardinalities(keys)
    got = dict(zip(hosts.tolist(), counts.tolist()))
    for aip, size in zip(w.planted_aip.tolist(), w.planted_set.tolist()):
        assert got[aip] == size


def test_error_rates_definition():
    r = truth.error_rates({1, 2, 3, 9}, {1, 2, 5, 6})
    assert (r["n"], r["n_plus"], r["n_minus"]) == (4, 2, 2)
    assert r["fpr"] == 0.5 and r["fnr"] == 0.5 and r["ftr"] == 1.0
    assert truth.error_rates({1}, set())["fpr"] is None
