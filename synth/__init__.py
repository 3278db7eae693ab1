"""Seeded synthetic inputs for the ASSE hot path.

This module is shared by the tests, the benchmark and the oracle-side checks,
and holds none of the method's arithmetic: it draws random numbers (a
counter-based SplitMix64 keyed by (seed, stream, index)), builds (aip, bip)
pair streams shaped like the paper's edge-router traffic, and derives the
random parameters the method consumes (the mangling multiplier A and the BH
keys).  Ground-truth cardinalities follow from construction (every host's
bips come from a set of known size made of distinct values), not from
counting.

Workloads (k = window slices, theta = threshold, r rows x 2^(c+u) ATVs x g ATs):

* ``tiny``   -- k=4, 16 slices of 65,536 pairs, 4,096 Zipf(1.1) hosts with bips
  uniform over 2^24, 3 planted hosts of 200/300/400 bips, theta=64,
  4 x 1,024 x 128.
* ``tiny_b`` -- as ``tiny`` but each background host draws from its own fixed
  set of U[1,16] bips (keeps the pool unsaturated so restore stays small).
* ``link``   -- k=10, 60 slices of 8 Mi pairs, 2^20 Zipf(1.1) hosts whose bip
  sets follow a power law P(d) ~ d^-2, 200 planted hosts with sets log-uniform
  in [1k, 200k] cycling over the window, theta=1024, 4 x 65,536 x 512.
* ``long``   -- k=60, 300 slices of 32 Mi*(1+0.4 sin(2 pi t/300)) pairs,
  2^22 Zipf(1.2) hosts, 1,000 planted hosts with sets log-uniform in
  [theta, 50 theta] live over random intervals, theta=4096, 4 x 262,144 x 1,024.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

M64 = (1 << 64) - 1
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele, Lea, Flood 2014) on a uint64 array."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _C1
        z = (z ^ (z >> np.uint64(27))) * _C2
        return z ^ (z >> np.uint64(31))


def key(seed: int, *stream: int) -> np.uint64:
    """Stream key: SplitMix64 chained over the seed and the stream labels."""
    z = splitmix64(np.uint64(seed & M64))
    for s in stream:
        z = splitmix64(z ^ np.uint64(s & M64))
    return np.uint64(z)


def rand_u64(k: np.uint64, idx: np.ndarray) -> np.ndarray:
    """Counter-based draw: the idx-th 64-bit value of stream k."""
    with np.errstate(over="ignore"):
        return splitmix64(np.asarray(idx, dtype=np.uint64) * _GOLDEN ^ np.uint64(k))


def rand_unit(k: np.uint64, idx: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits."""
    return (rand_u64(k, idx) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def mix32(x: np.ndarray) -> np.ndarray:
    """A bijection of uint32 (murmur3 finaliser), used to make distinct values."""
    x = np.asarray(x, dtype=np.uint32)
    with np.errstate(over="ignore"):
        x = x ^ (x >> np.uint32(16))
        x = x * np.uint32(0x85EBCA6B)
        x = x ^ (x >> np.uint32(13))
        x = x * np.uint32(0xC2B2AE35)
        x = x ^ (x >> np.uint32(16))
    return x


def method_keys(seed: int) -> dict:
    """The random parameters the method draws, from the seed: the mangling
    multiplier A in [2, 2^32) and the BH keys (odd multiplier, offset)."""
    r = rand_u64(key(seed, 0xA5A5), np.arange(3, dtype=np.uint64))
    A = 2 + int(r[0] % np.uint64((1 << 32) - 2))
    return {"A": A, "bh_a": int(r[1]) | 1, "bh_b": int(r[2])}


def column_split(E_log2: int, r: int = 4) -> tuple[int, int, int]:
    """(c, u, s) for 2^E_log2 ATVs per row: u = 4 frames bits when r*c covers
    the 32-u bits of LBS with c = E_log2 - 4, else u = 0; s is the smallest
    offset that makes the r windows cover LBS (c + s(r-1) >= 32-u)."""
    for u in (4, 0):
        c = E_log2 - u
        W = 32 - u
        if c >= 1 and r * c >= W and c <= W:
            s = max(1, -(-(W - c) // (r - 1))) if r > 1 else 1
            if s <= c and s * (r - 1) < W:
                return c, u, s
    raise ValueError("no column split covers LBS")


def zipf_cdf(n: int, alpha: float) -> np.ndarray:
    w = np.arange(1, n + 1, dtype=np.float64) ** (-alpha)
    c = np.cumsum(w)
    return c / c[-1]


@dataclass
class Workload:
    name: str
    k: int
    theta: int
    g: int
    r: int
    E_log2: int
    slices: int
    n_per_slice: int
    n_hosts: int
    zipf: float
    bip_mode: str            # "uniform24", "set16", "powerlaw"
    n_planted: int
    planted_lo: float
    planted_hi: float
    planted_live: str        # "always" or "interval"
    seed: int = 1
    diurnal: float = 0.0
    planted_sizes: list = field(default_factory=list)

    def __post_init__(self):
        self.c, self.u, self.s = column_split(self.E_log2, self.r)
        self.params = dict(k=self.k, theta=self.theta, g=self.g, r=self.r, c=self.c, u=self.u,
                           s=self.s, **method_keys(self.seed))
        self._cdf = None
        kp = key(self.seed, 0x9A, 1)
        idx = np.arange(self.n_planted, dtype=np.uint64)
        if self.planted_sizes:
            sizes = np.asarray(self.planted_sizes, dtype=np.int64)
        else:
            uu = rand_unit(kp, idx)
            sizes = np.exp(math.log(self.planted_lo) + uu * (math.log(self.planted_hi) - math.log(self.planted_lo)))
            sizes = np.maximum(1, np.round(sizes)).astype(np.int64)
        self.planted_set = sizes
        self.planted_aip = self.host_aip(np.arange(self.n_hosts, self.n_hosts + self.n_planted))
        if self.planted_live == "interval":
            st = rand_u64(key(self.seed, 0x9A, 2), idx) % np.uint64(self.slices)
            ln = self.k // 2 + rand_u64(key(self.seed, 0x9A, 3), idx) % np.uint64(3 * self.k - self.k // 2 + 1)
            self.planted_start = st.astype(np.int64)
            self.planted_len = ln.astype(np.int64)
        else:
            self.planted_start = np.zeros(self.n_planted, dtype=np.int64)
            self.planted_len = np.full(self.n_planted, 1 << 40, dtype=np.int64)

    # --- hosts and their bips
    def host_aip(self, rank) -> np.ndarray:
        """Distinct aip addresses: a bijection of the host rank."""
        return mix32((np.asarray(rank, dtype=np.uint64) + np.uint64(key(self.seed, 0xA1) & np.uint64(0xFFFFFFFF)))
                     .astype(np.uint32))

    def host_set_size(self, rank) -> np.ndarray:
        rank = np.asarray(rank, dtype=np.uint64)
        if self.bip_mode == "set16":
            return 1 + (rand_u64(key(self.seed, 0xD1), rank) % np.uint64(16)).astype(np.int64)
        if self.bip_mode == "powerlaw":
            # P(D >= d) = 1/d, i.e. P(D = d) ~ d^-2, capped at 2^20.
            v = rand_unit(key(self.seed, 0xD2), rank)
            d = np.floor(1.0 / np.maximum(1.0 - v, 1e-300))
            return np.minimum(d, float(1 << 20)).astype(np.int64)
        return np.zeros(rank.shape, dtype=np.int64)

    def host_bip(self, aip: np.ndarray, j: np.ndarray) -> np.ndarray:
        """Member j of a host's bip set; distinct over j < 2^32 for one host."""
        base = mix32(aip ^ np.uint32(0x5BD1E995))
        with np.errstate(over="ignore"):
            v = mix32((base.astype(np.uint64) + np.asarray(j, dtype=np.uint64)).astype(np.uint32))
        if self.bip_mode in ("set16", "uniform24"):
            v = v & np.uint32(0xFFFFFF)
        return v

    def slice_size(self, t: int) -> int:
        if self.diurnal:
            return int(round(self.n_per_slice * (1.0 + self.diurnal * math.sin(2 * math.pi * t / self.slices))))
        return self.n_per_slice

    def planted_per_slice(self) -> np.ndarray:
        if self.planted_live == "always" and self.bip_mode != "powerlaw":
            return self.planted_set.copy()           # every member in every slice
        return -(-self.planted_set // self.k)        # ceil(set/k): the set cycles over the window

    def planted_live_at(self, t: int) -> np.ndarray:
        return (t >= self.planted_start) & (t < self.planted_start + self.planted_len)

    # --- one slice of pairs
    def pairs(self, t: int, n: int | None = None) -> np.ndarray:
        """The (n, 2) uint32 (aip, bip) pairs of slice t, shuffled."""
        N = self.slice_size(t) if n is None else n
        per = self.planted_per_slice()
        live = self.planted_live_at(t)
        parts_a, parts_b = [], []
        for p in np.nonzero(live)[0]:
            m = int(per[p])
            q = np.arange(m, dtype=np.int64)
            j = (t * m + q) % int(self.planted_set[p])
            parts_a.append(np.full(m, self.planted_aip[p], dtype=np.uint32))
            parts_b.append(self.host_bip(np.full(m, self.planted_aip[p], dtype=np.uint32), j))
        n_pl = sum(len(a) for a in parts_a)
        n_bg = max(0, N - n_pl)
        if self._cdf is None:
            self._cdf = zipf_cdf(self.n_hosts, self.zipf)
        idx = np.arange(n_bg, dtype=np.uint64)
        rank = np.searchsorted(self._cdf, rand_unit(key(self.seed, 0xB0, t), idx), side="right")
        rank = np.minimum(rank, self.n_hosts - 1)
        aip = self.host_aip(rank)
        if self.bip_mode == "uniform24":
            bip = (rand_u64(key(self.seed, 0xB1, t), idx) >> np.uint64(40)).astype(np.uint32)
        else:
            d = self.host_set_size(rank)
            j = np.floor(rand_unit(key(self.seed, 0xB2, t), idx) * d).astype(np.int64)
            bip = self.host_bip(aip, j)
        A = np.concatenate(parts_a + [aip]) if parts_a else aip
        B = np.concatenate(parts_b + [bip]) if parts_b else bip
        order = np.argsort(rand_u64(key(self.seed, 0xB3, t), np.arange(A.shape[0], dtype=np.uint64)), kind="stable")
        out = np.empty((A.shape[0], 2), dtype=np.uint32)
        out[:, 0] = A[order]
        out[:, 1] = B[order]
        if n is not None and out.shape[0] > n:
            out = out[:n]
        return out


def workload(name: str, seed: int = 1) -> Workload:
    if name == "tiny":
        return Workload("tiny", k=4, theta=64, g=128, r=4, E_log2=10, slices=16, n_per_slice=65536,
                        n_hosts=4096, zipf=1.1, bip_mode="uniform24", n_planted=3, planted_lo=0,
                        planted_hi=0, planted_live="always", seed=seed, planted_sizes=[200, 300, 400])
    if name == "tiny_b":
        return Workload("tiny_b", k=4, theta=64, g=128, r=4, E_log2=10, slices=16, n_per_slice=65536,
                        n_hosts=4096, zipf=1.1, bip_mode="set16", n_planted=3, planted_lo=0,
                        planted_hi=0, planted_live="always", seed=seed, planted_sizes=[200, 300, 400])
    if name == "link":
        return Workload("link", k=10, theta=1024, g=512, r=4, E_log2=16, slices=60, n_per_slice=8 << 20,
                        n_hosts=1 << 20, zipf=1.1, bip_mode="powerlaw", n_planted=200, planted_lo=1000,
                        planted_hi=200000, planted_live="always", seed=seed)
    if name == "long":
        return Workload("long", k=60, theta=4096, g=1024, r=4, E_log2=18, slices=300, n_per_slice=32 << 20,
                        n_hosts=1 << 22, zipf=1.2, bip_mode="powerlaw", n_planted=1000, planted_lo=4096,
                        planted_hi=50 * 4096, planted_live="interval", seed=seed, diurnal=0.4)
    raise KeyError(name)


def _unit_sm(key: int, i) -> np.ndarray:
    """The draw the training-state generator of the CUDA library uses:
    SplitMix64(key ^ SplitMix64(i)), top 53 bits as a double in [0, 1)."""
    i = np.asarray(i, dtype=np.uint64)
    z = splitmix64(np.uint64(key) ^ splitmix64(i))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def training_state_draws(seed: int, index: int, k: int, g: int, n_max_log2: int, bg_max: float) -> dict:
    """The random inputs of synthetic training state `index` (the library's
    asse_synth_states draws the same numbers from the same counter-based
    generator): the host's cardinality n, log-uniform in [1, 2^n_max_log2];
    its split over the k slices by exponential shares, as the index ranges
    [ends[s], ends[s+1]) of its distinct bips mix32(base + j); and the
    background, which sets AT h in slice s with probability p (drawn in
    [0, bg_max] per state) independently: bg[s][h]."""
    key = int(splitmix64(np.uint64(seed & M64) ^ splitmix64(np.uint64((index + 0x51ED270B27) & M64))))
    lnmax = n_max_log2 * 0.6931471805599453
    card = max(1, int(math.floor(math.exp(float(_unit_sm(key, 1)) * lnmax))))
    pbg = float(np.float32(float(_unit_sm(key, 2)) * float(np.float32(bg_max))))
    w = [-math.log(float(_unit_sm(key, 16 + s)) + 1e-300) for s in range(k)]
    tot = 0.0
    for v in w:
        tot += v
    ends, cum = [0], 0.0
    for s in range(k):
        cum += w[s]
        ends.append(card if s + 1 == k else int(math.floor(card * cum / tot)))
    base = key >> 32
    bips = [mix32((np.arange(ends[s], ends[s + 1], dtype=np.uint64) + np.uint64(base)).astype(np.uint32))
            for s in range(k)]
    idx = (np.arange(k, dtype=np.uint64)[:, None] << np.uint64(32)) | np.arange(g, dtype=np.uint64)[None, :]
    bg = _unit_sm(key ^ 0xB5, idx) < pbg
    return {"card": card, "pbg": pbg, "ends": ends, "bips": bips, "bg": bg}


def candidate_state_draws(seed: int, index: int, k: int, g: int, r: int, n_max_log2: int, bg_max: float) -> dict:
    """The random inputs of synthetic candidate state `index` (the library's
    asse_synth_candidates draws the same numbers): the host's cardinality n
    and its split over the k slices as in training_state_draws, and for each
    of the r rows its own background probability p[i] in [0, bg_max] and the
    ATs it sets, bg[i][s][h]."""
    key = int(splitmix64(np.uint64(seed & M64) ^ splitmix64(np.uint64((index + 0x3C6EF372FE94F82B) & M64))))
    lnmax = n_max_log2 * 0.6931471805599453
    card = max(1, int(math.floor(math.exp(float(_unit_sm(key, 1)) * lnmax))))
    p = [float(np.float32(float(_unit_sm(key, 4 + i)) * float(np.float32(bg_max)))) for i in range(r)]
    w = [-math.log(float(_unit_sm(key, 16 + s)) + 1e-300) for s in range(k)]
    tot = 0.0
    for v in w:
        tot += v
    ends, cum = [0], 0.0
    for s in range(k):
        cum += w[s]
        ends.append(card if s + 1 == k else int(math.floor(card * cum / tot)))
    base = key >> 32
    bips = [mix32((np.arange(ends[s], ends[s + 1], dtype=np.uint64) + np.uint64(base)).astype(np.uint32))
            for s in range(k)]
    idx = (np.arange(k, dtype=np.uint64)[:, None] << np.uint64(32)) | np.arange(g, dtype=np.uint64)[None, :]
    bg = np.stack([_unit_sm(key ^ (0xB5 + 0x100 * (i + 1)), idx) < p[i] for i in range(r)])
    return {"card": card, "p": p, "ends": ends, "bips": bips, "bg": bg}


def random_pairs(seed: int, stream: int, n: int, n_hosts: int = 64, n_bips: int = 1 << 16) -> np.ndarray:
    """Small uniform test streams: n pairs over n_hosts aips and n_bips bips."""
    idx = np.arange(n, dtype=np.uint64)
    a = rand_u64(key(seed, 0xC0, stream), idx) % np.uint64(n_hosts)
    b = rand_u64(key(seed, 0xC1, stream), idx) % np.uint64(n_bips)
    out = np.empty((n, 2), dtype=np.uint32)
    out[:, 0] = mix32(a.astype(np.uint32) + np.uint32(seed))
    out[:, 1] = mix32(b.astype(np.uint32) ^ np.uint32(0xABCDEF))
    return out
