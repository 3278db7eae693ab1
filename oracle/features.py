"""Feature rows of the learned estimators, from the oracle's unpacked state
-- TEST INFRASTRUCTURE ONLY.

The paper has no learned component (its estimates are Eq. 2 per ATV and
Eq. 4 per candidate, Sec. 3 and Sec. 4.3); these are the definitions of the
model inputs the CUDA library computes from its packed pool, written out
plainly on one-byte-per-AT state so the tests can compare them:

per ATV (80 values, the last 12 zero):
  [0]      |ATV|^{k'} / g: the active ATs of the window (Algorithm 1)
  [1 + a]  active ATs of age a, / g, for a < min(k', 64); the age of an AT is
           the number of slices since it was set
  [65]     P = |AAT(k', i, j)| / (g 2^c), the load of the ATV's row and frame
  [66]     UP of the frame (the product of P over the rows)
  [67]     the mean of P over the rows of the frame

Values are rounded to BF16 (the type the model reads)."""
from __future__ import annotations

import numpy as np

from .mlp import bf16

FEAT = 80


def ages(at: np.ndarray, act: np.ndarray, k: int, mode: int) -> tuple[np.ndarray, np.ndarray]:
    """(age, set) of every counter: for timestamps (mode 0 or 2) an AT with
    value v < 2k was set (act - v) mod 2k slices ago (Sec. 3: v is the ACT of
    its block in the slice that set it); for aging counters (mode 1) a value
    v > 0 was set k - v slices ago."""
    at = np.asarray(at, dtype=np.int64)
    if mode == 1:
        return k - at, at > 0
    return (np.asarray(act, dtype=np.int64) - at) % (2 * k), at != 2 * k


def atv_rows(at: np.ndarray, act: np.ndarray, k: int, kp: int, mode: int, load: np.ndarray,
             up: np.ndarray, mean: np.ndarray) -> np.ndarray:
    """Feature rows [n][80] of n ATVs with counter values at [n][g], the ACT
    of each AT index act [g], window kp, and the three load values of each
    ATV (arrays of n)."""
    n, g = at.shape
    age, was_set = ages(at, np.broadcast_to(act, at.shape), k, mode)
    active = was_set & (age < kp)           # Algorithm 1: set within the latest k' slices
    out = np.zeros((n, FEAT))
    out[:, 0] = active.sum(axis=1) / g
    for a in range(min(kp, 64)):
        out[:, 1 + a] = (active & (age == a)).sum(axis=1) / g
    out[:, 65] = load
    out[:, 66] = up
    out[:, 67] = mean
    return bf16(out)


def pool_rows(orc, kp: int) -> np.ndarray:
    """Feature rows [r*E][80] of every ATV of an oracle pool in ATV order
    (row-major: row i, then ATV index), for the window of the latest kp
    slices ending at the open slice."""
    at = orc.at()                                            # [r][E][g]
    act = np.array([orc.act(h) for h in range(orc.g)])
    aat = orc.aat(orc.counts(kp)).astype(np.float64) / (orc.g * (1 << orc.c))   # [r][frames]
    frame = np.arange(orc.E) >> orc.c
    rows = []
    for i in range(orc.r):
        rows.append(atv_rows(at[i], act, orc.k, kp, orc.mode, aat[i, frame], np.prod(aat, axis=0)[frame],
                             aat.mean(axis=0)[frame]))
    return np.concatenate(rows)


def candidate_rows(at_rows: np.ndarray, act: np.ndarray, k: int, kp: int, mode: int, loads: np.ndarray,
                   cnts: np.ndarray) -> np.ndarray:
    """Feature rows [n][80] of n candidate hosts, each given by the counter
    values of its r ATVs at_rows [n][r][g], the ACT of each AT index act [g],
    its frame's row loads loads [n][r] (P_i = |AAT(k', i, j)| / (g 2^c)) and
    its ATVs' active counts cnts [n][r]:

      [0]      NAT / g: the ATs active in all r ATVs (Algorithm 5)
      [1 + a]  ATs active in all r ATVs whose oldest timestamp (largest age
               over the rows) is a slices old, / g, for a < min(k', 64): the
               host sets all r ATs of a bip in the same slice, and another
               host can only make some of them younger
      [65]     UP of the frame: the product of P_i over the rows (Eq. 4)
      [66]     the smallest P_i, [67] the largest P_i
      [68 + i] |ATV_i|^{k'} / g for each row i (r <= 8)

    rounded to BF16."""
    n, r, g = at_rows.shape
    age, was_set = ages(at_rows, np.broadcast_to(act, at_rows.shape), k, mode)
    active = was_set & (age < kp)
    all_rows = active.all(axis=1)                        # [n][g]
    oldest = np.where(active, age, -1).max(axis=1)       # [n][g]
    out = np.zeros((n, FEAT))
    out[:, 0] = all_rows.sum(axis=1) / g
    for a in range(min(kp, 64)):
        out[:, 1 + a] = (all_rows & (oldest == a)).sum(axis=1) / g
    out[:, 65] = np.prod(loads, axis=1)
    out[:, 66] = loads.min(axis=1)
    out[:, 67] = loads.max(axis=1)
    out[:, 68:68 + r] = np.asarray(cnts, dtype=np.float64) / g
    return bf16(out)


def pool_candidate_rows(orc, aips, kp: int) -> np.ndarray:
    """candidate_rows of the hosts aips in an oracle pool, for the window of
    the latest kp slices ending at the open slice."""
    at = orc.at()
    act = np.array([orc.act(h) for h in range(orc.g)])
    cnt = orc.counts(kp)
    P = orc.aat(cnt).astype(np.float64) / (orc.g * (1 << orc.c))     # [r][frames]
    rows, loads, cnts = [], [], []
    for aip in np.asarray(aips, dtype=np.uint32).tolist():
        x, z = orc.rrh(int(aip))
        e = [(z << orc.c) | x[i] for i in range(orc.r)]
        rows.append(np.stack([at[i, e[i]] for i in range(orc.r)]))
        loads.append(P[:, z])
        cnts.append([cnt[i, e[i]] for i in range(orc.r)])
    if not rows:
        return np.zeros((0, FEAT))
    return candidate_rows(np.stack(rows), act, orc.k, kp, orc.mode, np.array(loads), np.array(cnts))
