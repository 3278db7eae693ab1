"""The serving loop (include/asse_serve.h): streams with different k, g and
pool sizes, batches of uneven size, run through captured CUDA graphs.

* every stream's reports through the server equal those of the plain pool
  path (asse_ingest + asse_close_slice, itself oracle-checked);
* run together, interleaved on the device, with a budget that admits only
  some streams at a time (the rest wait until memory frees up), every stream's
  reports are identical to its reports when it runs alone.
"""
import numpy as np
import pytest

import synth
from gpu_util import mixed_pairs, to_device

pytestmark = pytest.mark.gpu


def _streams():
    out = []
    specs = [(4, 128, 10), (10, 512, 12), (30, 256, 11), (6, 150, 12), (10, 128, 13), (20, 512, 10)]
    for i, (k, g, elog) in enumerate(specs):
        c, u, s = synth.column_split(elog, 4)
        p = dict(k=k, theta=max(16, g // 3), g=g, r=4, c=c, u=u, s=s, **synth.method_keys(100 + i))
        rng = np.random.default_rng(i)
        slices = []
        for t in range(2 * k + 2 if k <= 6 else 6):
            nb = int(rng.integers(1, 4))
            batches = [mixed_pairs(200 + i, 10 * t + b, int(rng.integers(1, 40000)), [g // 2, g, 3 * g])
                       for b in range(nb)]
            slices.append(batches)
        out.append((p, k, slices))
    return out


def _key(rep):
    return sorted((int(r["aip"]), int(r["nat"]), float(r["est"]), int(r["flags"])) for r in rep)


@pytest.fixture(scope="module")
def mods():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_01527_gb300 import asse, build
    build.build()
    return asse, torch


def _run_alone(asse, p, k, slices):
    srv = asse.Server(1 << 40)
    sid = srv.open(p, k, max_batch=40000)
    reps = []
    for batches in slices:
        for j, b in enumerate(batches):
            assert srv.submit(sid, b, close=(j == len(batches) - 1))   # pageable: copied before return
        res = None
        while res is None:
            res = srv.poll(sid)
        reps.append(_key(res[0]))
    srv.close(sid)
    srv.destroy()
    return reps


def test_server_equals_plain_pool_path(mods):
    asse, torch = mods
    for p, k, slices in _streams()[:3]:
        pool = asse.Pool(p)
        want = []
        for batches in slices:
            for b in batches:
                pool.ingest(to_device(b))
            pool.close_slice(k)
            want.append(_key(pool.report()))
        pool.close()
        assert _run_alone(asse, p, k, slices) == want


def test_mix_equals_alone_with_admission(mods):
    asse, torch = mods
    streams = _streams()
    alone = [_run_alone(asse, p, k, slices) for p, k, slices in streams]
    sizes = [asse.Server.stream_bytes(p, 40000) for p, _k, _s in streams]
    budget = sum(sorted(sizes)[-3:])                  # room for about three streams at a time
    srv = asse.Server(budget)
    waiting = list(range(len(streams)))
    running = {}                                       # stream index -> [sid, next slice, next batch, results]
    deferred, max_open = 0, 0
    while waiting or running:
        while waiting:
            i = waiting[0]
            sid = srv.open(streams[i][0], streams[i][1], max_batch=40000)
            if sid is None:
                deferred += 1
                break
            waiting.pop(0)
            running[i] = [sid, 0, 0, []]
        max_open = max(max_open, len(running))
        for i in list(running):                        # one batch of every open stream per round
            sid, t, b, res = running[i]
            slices = streams[i][2]
            if t < len(slices):
                batch = slices[t][b]
                last = b == len(slices[t]) - 1
                if srv.submit(sid, batch, close=last):
                    running[i][1:3] = [t + 1, 0] if last else [t, b + 1]
            r = srv.poll(sid)
            if r is not None:
                res.append(_key(r[0]))
            if len(res) == len(slices):
                srv.close(sid)
                del running[i]
                assert res == alone[i], f"stream {i} differs in the mix"
    assert deferred > 0 and max_open >= 2
    assert srv.bytes_in_use() == 0
    srv.destroy()
