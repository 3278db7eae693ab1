"""Pins of the oracle's reversible hash RRH and of BH (Sec. 4.1), and of the
restore of Algorithm 4 (Sec. 4.2):

* p = 2^32 + 15 is prime (trial division), A^-1 is A's inverse mod p;
* f is the linear map x -> A*x mod p (f(1) = A, f(x+y) = f(x)+f(y) mod p),
  one-to-one, and its cycle walk only ever multiplies by further powers of A;
* the column-split example of Sec. 4.1 (golden fixture);
* recoverability: a tuple RRH(aip) restores exactly aip, for random and edge
  addresses, including the ones whose mangled value needed a cycle walk;
* Algorithm 4 on random super-ATV sets equals an independent brute force
  that checks every multiply-covered position (the consecutive-row check of
  the paper is equivalent when the windows are contiguous).
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
P = (1 << 32) + 15


def _is_prime(n):
    if n % 2 == 0:
        return n == 2
    for d in range(3, math.isqrt(n) + 1, 2):
        if n % d == 0:
            return False
    return True


def test_modulus_is_prime_and_just_above_2_32():
    assert _is_prime(P)
    assert not any(_is_prime(n) for n in range((1 << 32) + 1, P))


def _oracle(oracle_mod, seed=1, **kw):
    p = dict(k=4, theta=64, g=128, r=4, c=10, u=0, s=8, **synth.method_keys(seed))
    p.update(kw)
    return oracle_mod.Oracle.from_params(p)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_mangle_is_the_linear_map(oracle_mod, seed):
    o = _oracle(oracle_mod, seed)
    A = o.params.A
    assert o.inverse_A() == pow(A, -1, P)
    assert o.mangle(1) == A
    assert o.mangle(0) == 0
    rng = np.random.default_rng(seed)
    xs = rng.integers(0, 1 << 31, 3000, dtype=np.uint64).tolist()
    ys = rng.integers(0, 1 << 31, 3000, dtype=np.uint64).tolist()
    for x, y in zip(xs, ys):
        assert (o.mangle(x) + o.mangle(y) - o.mangle(x + y)) % P == 0
        assert (2 * o.mangle(x) - o.mangle(2 * x)) % P == 0


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_cycle_walk_cases(oracle_mod, seed):
    """The 15 residues in [2^32, p) are the only ones that need a walk; their
    preimages still map below 2^32, onto powers of A times aip, one-to-one."""
    o = _oracle(oracle_mod, seed)
    A = o.params.A
    Ai = pow(A, -1, P)
    walkers = [(Ai * v) % P for v in range(1 << 32, P)]
    walkers = [a for a in walkers if a < (1 << 32)]
    images = set()
    for aip in walkers:
        y = o.mangle(aip)
        assert y < (1 << 32)
        assert any(pow(A, j, P) * aip % P == y for j in range(2, 40))
        assert o.unmangle(y) == aip
        images.add(y)
    assert len(images) == len(walkers)


def test_mangle_one_to_one_sampled(oracle_mod):
    o = _oracle(oracle_mod, 7)
    xs = list(range(0, 1 << 16)) + list(range((1 << 32) - (1 << 14), 1 << 32))
    ys = [o.mangle(x) for x in xs]
    assert len(set(ys)) == len(xs)
    assert all(o.unmangle(y) == x for x, y in zip(xs[::97], ys[::97]))


def test_column_split_example(oracle_mod):
    ex = json.load(open(os.path.join(GOLDEN, "column_split_example.json")))
    r, s, u, c, W = ex["r"], ex["s"], ex["u"], ex["c"], ex["W"]
    assert W == 32 - u and c + s * (r - 1) >= W        # completeness holds
    o = _oracle(oracle_mod, 5, r=r, s=s, u=u, c=c)
    rng = np.random.default_rng(0)
    for aip in rng.integers(0, 1 << 32, 500, dtype=np.uint64).tolist():
        f = o.mangle(aip)
        L = f >> u
        bit = lambda pos: (L >> (W - 1 - pos)) & 1
        x, z = o.rrh(aip)
        assert z == f & ((1 << u) - 1)
        for row, ranges in ex["x_ranges"].items():
            want = []
            for lo, hi in ranges:
                want += [bit(pp) for pp in range(lo, hi + 1)]
            got = [(x[int(row)] >> (c - 1 - n)) & 1 for n in range(c)]
            assert got == want, (aip, row)
    cover = {i: {(s * i + n) % W for n in range(c)} for i in range(r)}
    assert sorted(cover[0] & cover[1]) == ex["duplicate_x0_x1"]
    assert sorted(cover[3] & cover[0]) == ex["duplicate_x3_x0"]
    assert (s * ex["wrap"]["x"] + ex["wrap"]["bit"]) % W == ex["wrap"]["lbs_position"]
    assert set().union(*cover.values()) == set(range(W))


def test_bh_range_and_uniformity(oracle_mod):
    for g in (128, 500, 512, 1024):
        o = _oracle(oracle_mod, 3, g=g)
        hs = np.array([o.bh(b) for b in range(40000)])
        assert hs.min() >= 0 and hs.max() < g
        counts = np.bincount(hs, minlength=g)
        exp = 40000 / g
        chi2 = ((counts - exp) ** 2 / exp).sum()
        # chi-square with g-1 dof: mean g-1, sd sqrt(2(g-1)); allow 6 sd
        assert chi2 < (g - 1) + 6 * math.sqrt(2 * (g - 1)), (g, chi2)


def _cnt_with_super(o, supers, value=None):
    cnt = np.zeros((o.r, o.E), dtype=np.uint32)
    for i, e in supers:
        cnt[i, e] = o.g if value is None else value
    return cnt


@pytest.mark.parametrize("cfg", [dict(c=10, u=0, s=8), dict(c=12, u=4, s=6), dict(c=14, u=4, s=5),
                                 dict(c=9, u=2, s=7), dict(c=8, u=0, s=8, r=5)])
def test_restore_recovers_single_host(oracle_mod, cfg):
    o = _oracle(oracle_mod, 11, **cfg)
    A = o.params.A
    Ai = pow(A, -1, P)
    walkers = [a for a in ((Ai * v) % P for v in range(1 << 32, P)) if a < (1 << 32)]
    rng = np.random.default_rng(4)
    aips = [0, 1, 2, (1 << 32) - 1, 0x80000000] + walkers[:3] + rng.integers(0, 1 << 32, 60, dtype=np.uint64).tolist()
    for aip in aips:
        x, z = o.rrh(aip)
        cnt = _cnt_with_super(o, [(i, (z << o.c) | x[i]) for i in range(o.r)])
        n, cand = o.restore(cnt, 16)
        assert n == 1 and cand.tolist() == [aip], (aip, n, cand)


def _brute_restore(o, cnt):
    """Independent Algorithm 4: every tuple, every position checked across
    every row covering it, LBS rebuilt bit by bit, f^-1 by Python integers."""
    W, c, s, r, u = 32 - o.u, o.c, o.s, o.r, o.u
    Ai = pow(o.params.A, -1, P)
    T = o.threshold()
    out = set()
    for j in range(1 << u):
        sa = [[x for x in range(1 << c) if cnt[i, (j << c) | x] >= T] for i in range(r)]
        for tup in itertools.product(*sa):
            bits = {}
            ok = True
            for i, xi in enumerate(tup):
                for n in range(c):
                    pos = (s * i + n) % W
                    b = (xi >> (c - 1 - n)) & 1
                    if bits.setdefault(pos, b) != b:
                        ok = False
            if not ok:
                continue
            L = 0
            for pos in range(W):
                L = (L << 1) | bits[pos]
            y = (L << u) | j
            x = Ai * y % P
            while x >= (1 << 32):
                x = Ai * x % P
            out.add(x)
    return out


@pytest.mark.parametrize("cfg,per_row,seed", [(dict(c=9, u=2, s=7), 6, 1), (dict(c=10, u=0, s=8), 7, 2),
                                              (dict(c=7, u=1, s=7, r=5), 5, 3), (dict(c=12, u=4, s=6), 5, 4)])
def test_restore_matches_brute_force(oracle_mod, cfg, per_row, seed):
    o = _oracle(oracle_mod, seed, **cfg)
    rng = np.random.default_rng(seed)
    supers = []
    frames = 1 << o.u
    # a few true hosts (all-super RRH tuples) plus random super ATVs per row-frame
    for aip in rng.integers(0, 1 << 32, 3, dtype=np.uint64).tolist():
        x, z = o.rrh(aip)
        supers += [(i, (z << o.c) | x[i]) for i in range(o.r)]
    for i in range(o.r):
        for j in range(min(frames, 4)):
            for x in rng.integers(0, 1 << o.c, per_row).tolist():
                supers.append((i, (j << o.c) | x))
    cnt = _cnt_with_super(o, supers, value=o.threshold())
    n, cand = o.restore(cnt, 1 << 16)
    assert n == len(cand) == len(set(cand.tolist()))
    assert set(cand.tolist()) == _brute_restore(o, cnt)
    # every candidate's own RRH tuple is all super (no false tuple survives)
    T = o.threshold()
    for aip in cand.tolist():
        x, z = o.rrh(aip)
        assert all(cnt[i, (z << o.c) | x[i]] >= T for i in range(o.r))


def test_restore_capacity_count(oracle_mod):
    o = _oracle(oracle_mod, 2, c=9, u=2, s=7)
    rng = np.random.default_rng(9)
    supers = [(i, int(e)) for i in range(o.r) for e in rng.integers(0, o.E, 40)]
    cnt = _cnt_with_super(o, supers)
    n_all, cand = o.restore(cnt, 1 << 20)
    assert n_all == len(cand)
    n_cap, first = o.restore(cnt, 5)
    assert n_cap == n_all and first.tolist() == cand[:5].tolist()
    n_stop, _ = o.restore(cnt, 5, limit_extra=0)
    assert n_stop == min(n_all, 6)
