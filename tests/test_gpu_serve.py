"""The serving loop (include/asse_serve.h): streams with different k, g and
pool sizes, batches of uneven size, run through captured CUDA graphs.

* every stream's reports through the server equal the oracle's close of the
  same batches (NAT exact, Eq. 4 within 1e-5 relative), and those of the
  plain pool path (asse_ingest + asse_close_slice);
* run together, interleaved on the device, with a budget that admits only
  some streams at a time (the rest wait until memory frees up), every stream's
  reports are identical to its reports when it runs alone, and equal the
  oracle's.
"""
import numpy as np
import pytest

import synth
from gpu_util import compare_lists, mixed_pairs, to_device

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
    import oracle
    from paper_1807_01527_gb300 import asse, build
    build.build()
    oracle.build()
    return asse, torch


def _oracle_reports(p, k, slices):
    """The oracle's report rows (aip, est, nat) of every slice of a stream."""
    import oracle
    orc = oracle.Oracle.from_params(p)
    out = []
    for batches in slices:
        for b in batches:
            orc.ingest(b)
        out.append(orc.close_report(k)["report"])
        orc.advance()
    return out


def _run_alone(asse, p, k, slices, raw=None):
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
        if raw is not None:
            raw.append(res[0].copy())
    srv.close(sid)
    srv.destroy()
    return reps


def test_server_equals_oracle_and_plain_pool_path(mods):
    asse, torch = mods
    for i, (p, k, slices) in enumerate(_streams()[:3]):
        pool = asse.Pool(p)
        want = []
        for batches in slices:
            for b in batches:
                pool.ingest(to_device(b))
            pool.close_slice(k)
            want.append(_key(pool.report()))
        pool.close()
        raw = []
        assert _run_alone(asse, p, k, slices, raw) == want
        for t, (got, rows) in enumerate(zip(raw, _oracle_reports(p, k, slices))):
            compare_lists(got, rows, p["theta"], "stream %d slice %d" % (i, t))


def test_mix_equals_alone_with_admission(mods):
    asse, torch = mods
    streams = _streams()
    raws = [[] for _ in streams]
    alone = [_run_alone(asse, p, k, slices, raws[i]) for i, (p, k, slices) in enumerate(streams)]
    for i, (p, k, slices) in enumerate(streams):
        for t, (got, rows) in enumerate(zip(raws[i], _oracle_reports(p, k, slices))):
            compare_lists(got, rows, p["theta"], "stream %d slice %d" % (i, t))
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


@pytest.mark.parametrize("counter", ["at", "hist"])
def test_learned_inference_in_close_graphs(mods, counter):
    """A model attached to a stream runs inside its captured close graphs
    (feature rows, tensor-core MLP, Eq. 2 fallback between the scan and the
    refresh): every close's learned estimates equal asse_estimate_learned on
    a plain pool fed the same batches, and the reports still equal the
    oracle's (the refresh now runs as its own kernel after the restore).
    With slice counts the feature rows come from the counts, C0 read from
    the device slice state as each graph replays."""
    asse, torch = mods
    k, g, elog = 10, 512, 12
    c, u, s = synth.column_split(elog, 4)
    p = dict(k=k, theta=g // 3, g=g, r=4, c=c, u=u, s=s, **synth.method_keys(77))
    rng = np.random.default_rng(3)
    slices = [[mixed_pairs(300, 10 * t + b, int(rng.integers(1000, 30000)), [g // 2, g, 3 * g, 9 * g])
               for b in range(int(rng.integers(1, 3)))] for t in range(2 * k + 3)]
    stream = torch.cuda.current_stream().cuda_stream
    model = asse.MLP(seed=3, stream=stream)
    rows = 4 << elog
    # the plain pool path: scan, learned estimate, restore, refresh
    pool = asse.Pool(p, stream=stream, counter=counter)
    # the model's outputs moved to straddle max_log_n, so that the model and
    # the fallback both serve some ATVs
    for b in slices[0]:
        pool.ingest(to_device(b))
    pool.scan(k)
    y0 = model.forward(pool.features()).cpu().numpy()
    prm = model.params()
    prm[-1] += np.float32(2.0 - np.median(y0))
    model.set_params(prm)
    max_log_n = 2.0
    pool.close()
    pool = asse.Pool(p, stream=stream, counter=counter)
    want_est, want_nfb = [], []
    for batches in slices:
        for b in batches:
            pool.ingest(to_device(b))
        pool.scan(k)
        est, nfb, _x = pool.estimate_learned(model, max_log_n)
        want_est.append(est.cpu().numpy())
        want_nfb.append(int(nfb.item()))
        pool.restore()
        pool.advance()
    pool.close()
    srv = asse.Server(1 << 40)
    sid = srv.open(p, k, max_batch=40000, counter=counter)
    srv.attach_model(sid, model, max_log_n)
    for t, (batches, rows_want) in enumerate(zip(slices, _oracle_reports(p, k, slices))):
        for j, b in enumerate(batches):
            assert srv.submit(sid, b, close=(j == len(batches) - 1))
        res = None
        while res is None:
            res = srv.poll(sid)
        compare_lists(res[0], rows_want, p["theta"], "slice %d" % t)
        est, nfb = srv.estimates(sid, rows)
        np.testing.assert_array_equal(est, want_est[t], err_msg="learned estimates, slice %d" % t)
        assert nfb == want_nfb[t]
    assert 0 < min(want_nfb) and max(want_nfb) < rows      # both the model and the fallback were used
    srv.close(sid)
    srv.destroy()


def test_close_with_closes_in_flight(mods):
    """A stream closed while closes of it are still queued (never polled)
    ends cleanly: its memory returns to the budget, and a stream opened in
    its place, fed the same batches, reports exactly what the oracle does."""
    asse, torch = mods
    p, k, slices = _streams()[1]
    size = asse.Server.stream_bytes(p, 40000)
    srv = asse.Server(size)                            # room for one stream only
    sid = srv.open(p, k, max_batch=40000)
    for batches in slices[:asse.SERVE_RING]:
        for j, b in enumerate(batches):
            assert srv.submit(sid, b, close=(j == len(batches) - 1))
    assert srv.open(p, k, max_batch=40000) is None     # the budget is taken
    srv.close(sid)                                     # four closes still queued
    assert srv.bytes_in_use() == 0
    sid = srv.open(p, k, max_batch=40000)
    assert sid is not None
    for t, (batches, rows) in enumerate(zip(slices, _oracle_reports(p, k, slices))):
        for j, b in enumerate(batches):
            assert srv.submit(sid, b, close=(j == len(batches) - 1))
        res = None
        while res is None:
            res = srv.poll(sid)
        compare_lists(res[0], rows, p["theta"], "slice %d" % t)
    srv.close(sid)
    assert srv.bytes_in_use() == 0
    srv.destroy()
