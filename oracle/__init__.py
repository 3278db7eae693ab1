"""CPU oracle of the ASSE hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, literal implementation (``asse_oracle.c``, one byte per AT,
double-precision estimates) of what the paper defines:

* Algorithm 1 (checkAT), Algorithm 2 (preserveAT) and the ATV block/ACT
  layout of Sec. 3;
* the reversible hash RRH (IP mangling f, frame Z, column split x_i) and the
  bip hash BH of Sec. 4.1, and Algorithm 3 (Scan IP pair);
* the super-ATV threshold and Algorithm 4 (restore) of Sec. 4.2;
* Algorithm 5 (NAT), the row-frame loads, UP and Eq. 4 of Sec. 4.3;
* the aging-counter (ACE) variant described in Sec. 2.3.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may import this package.  The CUDA library never does, and shares no code with
it.  Parity of every function here is pinned by the ``-m "not gpu"`` tests
(paper examples, closed forms, brute-force models); see ``tests/test_oracle_*``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "asse_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libasse_oracle.so")

P_MOD = (1 << 32) + 15


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc into oracle/_build (host code only)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        # -ffp-contract=off: no fused multiply-add, so Eq. 2/Eq. 4 round each
        # operation exactly as written on every host architecture.
        subprocess.check_call(["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_uint32), ("theta", ctypes.c_uint32), ("g", ctypes.c_uint32),
                ("r", ctypes.c_uint32), ("c", ctypes.c_uint32), ("u", ctypes.c_uint32),
                ("s", ctypes.c_uint32), ("A", ctypes.c_uint32), ("bh_a", ctypes.c_uint64),
                ("bh_b", ctypes.c_uint64), ("mode", ctypes.c_uint32), ("pad", ctypes.c_uint32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        u32, u64, i64, vp, dbl = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_double
        sig = {
            "oracle_create": (vp, [ctypes.POINTER(Params)]),
            "oracle_destroy": (None, [vp]),
            "oracle_check_at": (ctypes.c_int, [u32, u32, u32, u32]),
            "oracle_preserve_at": (u32, [u32, u32, u32]),
            "oracle_block": (u32, [vp, u32]),
            "oracle_act": (u32, [vp, u32]),
            "oracle_mangle": (u32, [vp, u32]),
            "oracle_unmangle": (u32, [vp, u32]),
            "oracle_inverse_A": (u64, [vp]),
            "oracle_rrh": (None, [vp, u32, vp, vp]),
            "oracle_bh": (u32, [vp, u32]),
            "oracle_at": (vp, [vp]),
            "oracle_slice": (u64, [vp]),
            "oracle_num_atv": (u32, [vp]),
            "oracle_ingest": (None, [vp, vp, u64]),
            "oracle_advance": (None, [vp]),
            "oracle_active": (ctypes.c_int, [vp, u32, u32, u32, u32]),
            "oracle_counts": (None, [vp, u32, vp]),
            "oracle_aat": (None, [vp, vp, vp]),
            "oracle_threshold": (u32, [vp]),
            "oracle_restore": (i64, [vp, vp, vp, i64, i64]),
            "oracle_nat": (u32, [vp, u32, u32]),
            "oracle_up": (dbl, [vp, vp, u32]),
            "oracle_eq4": (dbl, [u32, u32, dbl]),
            "oracle_eq2": (dbl, [u32, u32]),
            "oracle_estimate": (dbl, [vp, vp, u32, u32, vp]),
            "oracle_cores": (ctypes.c_int, []),
            "oracle_ingest_mt": (None, [vp, vp, u64, ctypes.c_int]),
            "oracle_advance_mt": (None, [vp, ctypes.c_int]),
            "oracle_counts_mt": (None, [vp, u32, vp, ctypes.c_int]),
            "oracle_restore_mt": (i64, [vp, vp, vp, i64, i64, ctypes.c_int]),
            "oracle_estimate_mt": (None, [vp, vp, vp, u64, u32, vp, vp, ctypes.c_int]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check_at(value: int, act: int, k: int, kp: int) -> bool:
    """Algorithm 1 on one AT."""
    return bool(lib().oracle_check_at(value, act, k, kp))


def preserve_at(value: int, act: int, k: int) -> int:
    """Algorithm 2 on one AT."""
    return int(lib().oracle_preserve_at(value, act, k))


def eq4(g: int, nat: int, up: float) -> float:
    """Eq. 4 (bias-corrected estimate) with the edge readings of the C code."""
    return float(lib().oracle_eq4(g, nat, up))


def eq2(g: int, cnt: int) -> float:
    """Eq. 2 (ATV estimate)."""
    return float(lib().oracle_eq2(g, cnt))


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def cores() -> int:
    """Host cores the multi-threaded oracle calls use by default."""
    return int(lib().oracle_cores())


class Oracle:
    """One ATV cube (Sec. 4) with its slice clock, on the host."""

    def __init__(self, *, k, theta, g, r, c, u, s, A, bh_a, bh_b, mode=0):
        self.params = Params(k, theta, g, r, c, u, s, A, bh_a, bh_b, mode, 0)
        self.k, self.theta, self.g, self.r, self.c, self.u, self.s = k, theta, g, r, c, u, s
        self.mode = mode
        self._st = lib().oracle_create(ctypes.byref(self.params))
        if not self._st:
            raise ValueError("oracle_create rejected the parameters")
        self.E = int(lib().oracle_num_atv(self._st))
        self.frames = 1 << u

    @classmethod
    def from_params(cls, p: dict, mode: int = 0) -> "Oracle":
        keys = ("k", "theta", "g", "r", "c", "u", "s", "A", "bh_a", "bh_b")
        return cls(**{key: int(p[key]) for key in keys}, mode=mode)

    def close(self):
        if self._st:
            lib().oracle_destroy(self._st)
            self._st = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- state
    @property
    def t(self) -> int:
        return int(lib().oracle_slice(self._st))

    def at(self) -> np.ndarray:
        """Copy of the AT values, shape [r][E][g], uint8."""
        n = self.r * self.E * self.g
        buf = (ctypes.c_uint8 * n).from_address(lib().oracle_at(self._st))
        return np.frombuffer(buf, dtype=np.uint8).reshape(self.r, self.E, self.g).copy()

    # -- hashes (Sec. 4.1)
    def mangle(self, aip: int) -> int:
        return int(lib().oracle_mangle(self._st, aip))

    def unmangle(self, y: int) -> int:
        return int(lib().oracle_unmangle(self._st, y))

    def inverse_A(self) -> int:
        return int(lib().oracle_inverse_A(self._st))

    def rrh(self, aip: int):
        x = np.zeros(32, dtype=np.uint32)
        z = np.zeros(1, dtype=np.uint32)
        lib().oracle_rrh(self._st, aip, _ptr(x), _ptr(z))
        return [int(v) for v in x[: self.r]], int(z[0])

    def bh(self, bip: int) -> int:
        return int(lib().oracle_bh(self._st, bip))

    def block(self, h: int) -> int:
        return int(lib().oracle_block(self._st, h))

    def act(self, h: int) -> int:
        return int(lib().oracle_act(self._st, h))

    # -- slice operations
    def ingest(self, pairs: np.ndarray, threads: int = 1):
        """Algorithm 3 over an (n, 2) uint32 array of (aip, bip) pairs; with
        threads != 1 the same arithmetic on that many threads (0: every
        core), split by (row, frame)."""
        pairs = np.ascontiguousarray(pairs, dtype=np.uint32).reshape(-1, 2)
        if threads == 1:
            lib().oracle_ingest(self._st, _ptr(pairs), pairs.shape[0])
        else:
            lib().oracle_ingest_mt(self._st, _ptr(pairs), pairs.shape[0], threads)

    def advance(self, threads: int = 1):
        """Close the open slice and open the next (refresh of Algorithm 2)."""
        if threads == 1:
            lib().oracle_advance(self._st)
        else:
            lib().oracle_advance_mt(self._st, threads)

    def active(self, row: int, est: int, h: int, kp: int) -> bool:
        return bool(lib().oracle_active(self._st, row, est, h, kp))

    def counts(self, kp: int, threads: int = 1) -> np.ndarray:
        """|ATV|^{k'} per ATV, shape [r][E]."""
        cnt = np.zeros((self.r, self.E), dtype=np.uint32)
        if threads == 1:
            lib().oracle_counts(self._st, kp, _ptr(cnt))
        else:
            lib().oracle_counts_mt(self._st, kp, _ptr(cnt), threads)
        return cnt

    def aat(self, cnt: np.ndarray) -> np.ndarray:
        """|AAT(k', i, j)| per row and frame, shape [r][2^u]."""
        cnt = np.ascontiguousarray(cnt, dtype=np.uint32)
        out = np.zeros((self.r, self.frames), dtype=np.uint64)
        lib().oracle_aat(self._st, _ptr(cnt), _ptr(out))
        return out

    def threshold(self) -> int:
        return int(lib().oracle_threshold(self._st))

    def super_atvs(self, cnt: np.ndarray):
        """SA(i, j): sorted column indices of the super ATVs of row i, frame j."""
        T = self.threshold()
        cols = 1 << self.c
        out = {}
        for i in range(self.r):
            for j in range(self.frames):
                seg = cnt[i, j * cols:(j + 1) * cols]
                out[(i, j)] = np.nonzero(seg >= T)[0].astype(np.uint32)
        return out

    def restore(self, cnt: np.ndarray, cap: int, limit_extra: int = -1):
        """Algorithm 4.  Returns (number of candidates, first min(n, cap) of them)."""
        cnt = np.ascontiguousarray(cnt, dtype=np.uint32)
        out = np.zeros(max(cap, 1), dtype=np.uint32)
        n = int(lib().oracle_restore(self._st, _ptr(cnt), _ptr(out), cap, limit_extra))
        return n, out[: min(n, cap)].copy()

    def nat(self, aip: int, kp: int) -> int:
        return int(lib().oracle_nat(self._st, aip, kp))

    def up(self, aat: np.ndarray, frame: int) -> float:
        aat = np.ascontiguousarray(aat, dtype=np.uint64)
        return float(lib().oracle_up(self._st, _ptr(aat), frame))

    def estimate(self, aat: np.ndarray, aip: int, kp: int):
        """(Eq. 4 estimate, NAT) of one host at the end of the open slice."""
        aat = np.ascontiguousarray(aat, dtype=np.uint64)
        nat = np.zeros(1, dtype=np.uint32)
        v = float(lib().oracle_estimate(self._st, _ptr(aat), aip, kp, _ptr(nat)))
        return v, int(nat[0])

    def restore_mt(self, cnt: np.ndarray, cap: int, frame_cap: int, threads: int = 0):
        """Algorithm 4 with the frames spread over threads (no stop rule;
        each frame keeps up to frame_cap candidates).  Returns (number of
        candidates, the first min(n, cap) in frame order)."""
        cnt = np.ascontiguousarray(cnt, dtype=np.uint32)
        out = np.zeros(max(cap, 1), dtype=np.uint32)
        n = int(lib().oracle_restore_mt(self._st, _ptr(cnt), _ptr(out), cap, frame_cap, threads))
        return n, out[: min(n, cap)].copy()

    def estimate_many(self, aat: np.ndarray, aips: np.ndarray, kp: int, threads: int = 0):
        """(Eq. 4 estimates, NAT) of many hosts, on threads."""
        aat = np.ascontiguousarray(aat, dtype=np.uint64)
        aips = np.ascontiguousarray(aips, dtype=np.uint32)
        est = np.zeros(aips.size, dtype=np.float64)
        nat = np.zeros(aips.size, dtype=np.uint32)
        lib().oracle_estimate_mt(self._st, _ptr(aat), _ptr(aips), aips.size, kp, _ptr(est), _ptr(nat), threads)
        return est, nat

    # -- the whole close of one slice (Sec. 4.2-4.3), before the refresh
    def close_report(self, kp: int, cap: int = 1 << 22, limit_extra: int = -1, threads: int = 1):
        """Counts, loads, candidates, NAT and Eq. 4 for the window ending at the
        open slice.  Returns a dict; 'report' holds (aip, est, nat) rows with
        est >= theta, sorted by aip.  Does not advance the slice.  threads !=
        1 runs the same steps on that many threads (0: every core); the
        restore then has no stop rule and keeps up to cap candidates per
        frame."""
        cnt = self.counts(kp, threads)
        aat = self.aat(cnt)
        rows = []
        if threads == 1:
            n, cand = self.restore(cnt, cap, limit_extra)
            if n <= cap:
                for aip in cand.tolist():
                    est, nat = self.estimate(aat, aip, kp)
                    rows.append((aip, est, nat))
        else:
            n, cand = self.restore_mt(cnt, cap, cap, threads)
            if n <= cap:
                est, nat = self.estimate_many(aat, cand, kp, threads)
                rows = [(int(a), float(e), int(m)) for a, e, m in zip(cand.tolist(), est.tolist(), nat.tolist())]
        rows.sort()
        report = [row for row in rows if row[1] >= self.theta]
        return {"counts": cnt, "aat": aat, "n_candidates": n, "candidates": rows, "report": report}
