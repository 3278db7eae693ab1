"""ctypes binding of libasse.so (include/asse.h): argument marshalling only.

Every step of the hot path runs in the library's CUDA kernels; this module
passes pointers, sizes and the current torch CUDA stream, and turns status
codes into exceptions.  There is no fallback: if the library is not built,
``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libasse.so")

OK, EINVAL, ENOMEM, ECAPACITY, ECUDA, ESTATE, EAGAIN, ETIMEOUT = 0, 1, 2, 3, 4, 5, 6, 7
HOST, DEVICE = 0, 1
COUNTER_AT, COUNTER_ACE, COUNTER_AT_ALIGNED, COUNTER_AT_HIST = 0, 1, 2, 3
COUNTERS = {"at": COUNTER_AT, "ace": COUNTER_ACE, "aligned": COUNTER_AT_ALIGNED, "hist": COUNTER_AT_HIST}
KEY_TABLE = {"auto": 0, "on": 1, "off": 2}
SP_SATURATED, SP_REPORTED, SP_LEARNED = 1, 2, 4
SERVE_RING = 4   # ASSE_SERVE_RING of include/asse_serve.h: closes a stream may have in flight

u32, u64, i32, vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p


class Config(ctypes.Structure):
    _fields_ = [("k", u32), ("theta", u32), ("g", u32), ("r", u32), ("c", u32), ("u", u32), ("s", u32),
                ("A", u32), ("bh_a", u64), ("bh_b", u64), ("counter", u32), ("restore_cap", u32),
                ("max_batch", u64), ("key_table", u32), ("cluster", u32)]


class SuperPoint(ctypes.Structure):
    _fields_ = [("aip", u32), ("nat", u32), ("est", ctypes.c_float), ("flags", u32)]


class PoolInfo(ctypes.Structure):
    _fields_ = [("w", u32), ("fields", u32), ("words", u32), ("E", u32), ("threshold", u32), ("block", u32),
                ("k", u32), ("paired", u32), ("slice", u64), ("pool_words", u64), ("pool", vp)]


class SynthCfg(ctypes.Structure):
    _fields_ = [("k", u32), ("g", u32), ("r", u32), ("n_max_log2", u32), ("bg_max", ctypes.c_float),
                ("pad", u32), ("seed", u64), ("bh_a", u64), ("bh_b", u64)]


SP_DTYPE = np.dtype([("aip", "<u4"), ("nat", "<u4"), ("est", "<f4"), ("flags", "<u4")])
FEAT, HID = 80, 256
MLP_NPARAMS = HID * FEAT + HID + HID * HID + HID + HID + 1

# Every entry point of include/asse.h: name -> (restype, argtypes).
EXPORTS = {
    "asse_create": (i32, [ctypes.POINTER(Config), vp, ctypes.POINTER(vp)]),
    "asse_destroy": (None, [vp]),
    "asse_set_stream": (i32, [vp, vp]),
    "asse_ingest": (i32, [vp, vp, u64, i32]),
    "asse_close_slice": (i32, [vp, u32]),
    "asse_close_slice_multi": (i32, [vp, vp, u32]),
    "asse_select_window": (i32, [vp, u32]),
    "asse_scan": (i32, [vp, u32]),
    "asse_restore": (i32, [vp]),
    "asse_advance": (i32, [vp]),
    "asse_restore_static": (i32, [vp, u32, vp, vp, u64, vp]),
    "asse_estimate": (i32, [vp, vp, u64, vp, i32]),
    "asse_report": (i32, [vp, vp, u64, ctypes.POINTER(u64), i32]),
    "asse_candidates": (i32, [vp, vp, u64, ctypes.POINTER(u64), i32]),
    "asse_counts": (i32, [vp, vp, i32]),
    "asse_loads": (i32, [vp, vp]),
    "asse_info": (i32, [vp, ctypes.POINTER(PoolInfo)]),
    "asse_read_pool": (i32, [vp, vp, i32]),
    "asse_snapshot": (i32, [vp, vp, u64, ctypes.POINTER(u64)]),
    "asse_load": (i32, [vp, vp, u64]),
    "asse_probe_random_reads": (i32, [vp, u64, ctypes.POINTER(u64)]),
    "asse_probe_bounded_wait": (i32, [vp, u64, i32, ctypes.POINTER(u64)]),
    "asse_set_timing": (i32, [vp, i32]),
    "asse_close_timing": (i32, [vp, vp]),
    "asse_launches": (u64, [vp]),
    "asse_last_error": (ctypes.c_char_p, [vp]),
    "asse_strerror": (ctypes.c_char_p, [i32]),
    # include/asse_learn.h
    "asse_features": (i32, [vp, vp]),
    "asse_estimate_learned": (i32, [vp, vp, ctypes.c_float, vp, vp, vp]),
    "asse_synth_states": (i32, [ctypes.POINTER(SynthCfg), u64, u64, vp, vp, vp, vp]),
    "asse_candidate_features": (i32, [vp, vp, u64, vp]),
    "asse_report_learned": (i32, [vp, vp, ctypes.c_float, vp, u64, ctypes.POINTER(u64), i32]),
    "asse_synth_candidates": (i32, [ctypes.POINTER(SynthCfg), u64, u64, vp, vp, vp, vp]),
    "asse_mlp_create": (i32, [u64, vp, ctypes.POINTER(vp)]),
    "asse_mlp_destroy": (None, [vp]),
    "asse_mlp_set_stream": (i32, [vp, vp]),
    "asse_mlp_get_params": (i32, [vp, vp]),
    "asse_mlp_set_params": (i32, [vp, vp]),
    "asse_mlp_forward": (i32, [vp, vp, u64, vp]),
    "asse_mlp_backward": (i32, [vp, vp, vp, u64, vp]),
    "asse_mlp_get_grads": (i32, [vp, vp]),
    "asse_mlp_train_step": (i32, [vp, vp, vp, u64, ctypes.c_float, vp]),
    "asse_mlp_check": (i32, [vp]),
    "asse_mlp_set_loss": (i32, [vp, i32]),
    "asse_mlp_last_error": (ctypes.c_char_p, [vp]),
    # include/asse_serve.h
    "asse_server_create": (i32, [u64, ctypes.POINTER(vp)]),
    "asse_server_destroy": (None, [vp]),
    "asse_server_stream_bytes": (u64, [ctypes.POINTER(Config), u64]),
    "asse_server_bytes_in_use": (u64, [vp]),
    "asse_server_open": (i32, [vp, ctypes.POINTER(Config), u32, u64, ctypes.POINTER(u32)]),
    "asse_server_submit": (i32, [vp, u32, vp, u64, i32, i32]),
    "asse_server_poll": (i32, [vp, u32, vp, u64, ctypes.POINTER(u64), ctypes.POINTER(u64),
                               ctypes.POINTER(ctypes.c_float)]),
    "asse_server_sync": (i32, [vp]),
    "asse_server_close": (i32, [vp, u32]),
    "asse_server_attach_model": (i32, [vp, u32, vp, ctypes.c_float]),
    "asse_server_estimates": (i32, [vp, u32, vp, u64, i32, ctypes.POINTER(u32)]),
    "asse_server_pool": (vp, [vp, u32]),
    "asse_server_last_error": (ctypes.c_char_p, [vp]),
}

_lib = None


def lib():
    """Load libasse.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libasse.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class AsseError(RuntimeError):
    def __init__(self, status: int, message: str, n_needed: int | None = None):
        super().__init__("%s: %s" % (lib().asse_strerror(status).decode(), message))
        self.status = status
        self.n_needed = n_needed


def _current_stream() -> int:
    import torch
    return torch.cuda.current_stream().cuda_stream


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _pairs_arg(pairs):
    """(pointer, n, where, keepalive) of an (n, 2) 32-bit pair array."""
    if _is_torch(pairs):
        if pairs.element_size() != 4 or not pairs.is_contiguous():
            raise ValueError("pairs must be a contiguous 32-bit tensor")
        n = pairs.numel() // 2
        return pairs.data_ptr(), n, DEVICE if pairs.is_cuda else HOST, pairs
    a = np.ascontiguousarray(pairs, dtype=np.uint32).reshape(-1)
    return a.ctypes.data, a.size // 2, HOST, a


def make_config(params: dict, counter: str = "at", restore_cap: int = 0, max_batch: int = 0,
                key_table: str = "auto", cluster: int = 0) -> Config:
    return Config(int(params["k"]), int(params["theta"]), int(params["g"]), int(params["r"]), int(params["c"]),
                  int(params["u"]), int(params["s"]), int(params["A"]), int(params["bh_a"]), int(params["bh_b"]),
                  COUNTERS[counter], int(restore_cap), int(max_batch), KEY_TABLE[key_table], int(cluster))


class Server:
    """Multi-stream serving loop (include/asse_serve.h)."""

    def __init__(self, budget_bytes: int):
        self._h = vp()
        rc = lib().asse_server_create(int(budget_bytes), ctypes.byref(self._h))
        if rc != OK:
            raise AsseError(rc, "asse_server_create failed")
        self.rcap = {}
        self._bufs = {}

    def _err(self, rc):
        return AsseError(rc, lib().asse_server_last_error(self._h).decode())

    def destroy(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().asse_server_destroy(self._h)
            self._h = vp()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    @staticmethod
    def stream_bytes(params: dict, max_batch: int, counter: str = "at", restore_cap: int = 0) -> int:
        cfg = make_config(params, counter, restore_cap)
        return int(lib().asse_server_stream_bytes(ctypes.byref(cfg), max_batch))

    def bytes_in_use(self) -> int:
        return int(lib().asse_server_bytes_in_use(self._h))

    def open(self, params: dict, kp: int, max_batch: int, counter: str = "at", restore_cap: int = 0):
        """Stream id, or None if it does not fit the budget now."""
        cfg = make_config(params, counter, restore_cap)
        sid = u32(0)
        rc = lib().asse_server_open(self._h, ctypes.byref(cfg), kp, max_batch, ctypes.byref(sid))
        if rc == ENOMEM:
            return None
        if rc != OK:
            raise self._err(rc)
        self.rcap[sid.value] = (restore_cap or 4096)
        self._bufs[sid.value] = np.empty(self.rcap[sid.value], dtype=SP_DTYPE)   # poll's output, reused
        return sid.value

    def submit(self, sid: int, pairs, close: bool) -> bool:
        """False if the stream's report ring is full (poll first)."""
        if pairs is None:
            ptr, n, where = None, 0, DEVICE
        else:
            ptr, n, where, _keep = _pairs_arg(pairs)
        rc = lib().asse_server_submit(self._h, sid, vp(ptr), n, where, 1 if close else 0)
        if rc == EAGAIN:
            return False
        if rc != OK:
            raise self._err(rc)
        return True

    def poll(self, sid: int):
        """(report array, slice, latency ms) of the oldest finished close, or None."""
        cap = self.rcap[sid]
        buf = self._bufs[sid]
        n, sl, ms = u64(0), u64(0), ctypes.c_float(0)
        rc = lib().asse_server_poll(self._h, sid, vp(buf.ctypes.data), cap, ctypes.byref(n), ctypes.byref(sl),
                                    ctypes.byref(ms))
        if rc == EAGAIN:
            return None
        if rc != OK:
            raise self._err(rc)
        return buf[: n.value].copy(), int(sl.value), float(ms.value)

    def attach_model(self, sid: int, model, max_log_n: float):
        """Run learned per-ATV inference in every later close of stream sid."""
        rc = lib().asse_server_attach_model(self._h, sid, model._h, float(max_log_n))
        if rc != OK:
            raise self._err(rc)

    def estimates(self, sid: int, rows: int):
        """(learned estimates [rows] float32 numpy array of the last polled
        close of stream sid, number of Eq. 2 fallbacks)."""
        out = np.zeros(rows, dtype=np.float32)
        nfb = u32(0)
        rc = lib().asse_server_estimates(self._h, sid, vp(out.ctypes.data), rows, HOST, ctypes.byref(nfb))
        if rc != OK:
            raise self._err(rc)
        return out, int(nfb.value)

    def sync(self):
        rc = lib().asse_server_sync(self._h)
        if rc != OK:
            raise self._err(rc)

    def close(self, sid: int):
        rc = lib().asse_server_close(self._h, sid)
        if rc != OK:
            raise self._err(rc)


class Pool:
    """One ATV cube in device memory (include/asse.h)."""

    def __init__(self, params: dict, *, counter: str = "at", restore_cap: int = 0, max_batch: int = 0,
                 stream: int | None = None, key_table: str = "auto", cluster: int = 0):
        cfg = make_config(params, counter, restore_cap, max_batch, key_table, cluster)
        self.cfg = cfg
        self._h = vp()
        self._stream = _current_stream() if stream is None else stream
        rc = lib().asse_create(ctypes.byref(cfg), vp(self._stream), ctypes.byref(self._h))
        if rc != OK:
            raise AsseError(rc, lib().asse_last_error(None).decode())
        self.r, self.g, self.k = cfg.r, cfg.g, cfg.k
        self.frames = 1 << cfg.u
        self.cap = restore_cap or 4096
        self.out_cap = self.cap * self.frames
        self._info = self.info()

    # -- plumbing
    def _check(self, rc: int, n_needed=None):
        if rc != OK:
            raise AsseError(rc, lib().asse_last_error(self._h).decode(), n_needed)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().asse_destroy(self._h)
            self._h = vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream: int):
        self._stream = stream
        self._check(lib().asse_set_stream(self._h, vp(stream)))

    def set_timing(self, on: bool = True):
        """Record device events around the scan and restore of every close."""
        self._check(lib().asse_set_timing(self._h, 1 if on else 0))

    def close_timing(self):
        """(scan ms, restore ms) of the last close recorded with timing on."""
        ms = (ctypes.c_float * 2)()
        self._check(lib().asse_close_timing(self._h, ms))
        return float(ms[0]), float(ms[1])

    @property
    def launches(self) -> int:
        return int(lib().asse_launches(self._h))

    def info(self) -> dict:
        inf = PoolInfo()
        self._check(lib().asse_info(self._h, ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in PoolInfo._fields_}

    # -- slice lifecycle
    def ingest(self, pairs):
        ptr, n, where, _keep = _pairs_arg(pairs)
        self._check(lib().asse_ingest(self._h, vp(ptr), n, where))

    def close_slice(self, kp: int | None = None):
        self._check(lib().asse_close_slice(self._h, self.k if kp is None else kp))

    def close_slice_multi(self, kps):
        """Close the open slice for several windows k' in one scan pass;
        window 0 is selected for the readers afterwards."""
        arr = (ctypes.c_uint32 * len(kps))(*[int(k) for k in kps])
        self._check(lib().asse_close_slice_multi(self._h, arr, len(kps)))

    def select_window(self, i: int):
        """Make report / candidates / counts / loads return window i of the last close."""
        self._check(lib().asse_select_window(self._h, int(i)))

    def scan(self, kp: int | None = None):
        self._check(lib().asse_scan(self._h, self.k if kp is None else kp))

    def restore(self):
        self._check(lib().asse_restore(self._h))

    def advance(self):
        self._check(lib().asse_advance(self._h))

    # -- results
    def _list(self, fn, out=None):
        n = u64(0)
        if out is not None:       # device tensor of SuperPoint records
            rc = fn(self._h, vp(out.data_ptr()), out.numel() * out.element_size() // 16, ctypes.byref(n), DEVICE)
            self._check(rc, int(n.value))
            return int(n.value)
        buf = np.empty(self.out_cap, dtype=SP_DTYPE)
        rc = fn(self._h, vp(buf.ctypes.data), self.out_cap, ctypes.byref(n), HOST)
        self._check(rc, int(n.value))
        return buf[: int(n.value)]

    def report(self, out=None):
        """Reported super points of the last close (structured array)."""
        return self._list(lib().asse_report, out)

    def candidates(self, out=None):
        """Every restored candidate (CSIP) of the last close."""
        return self._list(lib().asse_candidates, out)

    def estimate(self, aips):
        """NAT and Eq. 4 of given hosts, between scan() and advance()."""
        if _is_torch(aips):
            import torch
            out = torch.zeros(aips.numel() * 4, dtype=torch.int32, device=aips.device)
            self._check(lib().asse_estimate(self._h, vp(aips.data_ptr()), aips.numel(), vp(out.data_ptr()),
                                            DEVICE))
            return out
        a = np.ascontiguousarray(aips, dtype=np.uint32)
        out = np.zeros(a.size, dtype=SP_DTYPE)
        self._check(lib().asse_estimate(self._h, vp(a.ctypes.data), a.size, vp(out.ctypes.data), HOST))
        return out

    def counts(self) -> np.ndarray:
        out = np.zeros((self.r, self._info["E"]), dtype=np.uint16)
        self._check(lib().asse_counts(self._h, vp(out.ctypes.data), HOST))
        return out

    def loads(self) -> np.ndarray:
        out = np.zeros((self.r, self.frames), dtype=np.uint64)
        self._check(lib().asse_loads(self._h, vp(out.ctypes.data)))
        return out

    def read_pool(self) -> np.ndarray:
        inf = self._info
        out = np.zeros(inf["pool_words"], dtype=np.uint32)
        self._check(lib().asse_read_pool(self._h, vp(out.ctypes.data), HOST))
        return out.reshape(self.r, inf["E"], inf["words"])

    def snapshot(self) -> bytes:
        n = u64(0)
        self._check(lib().asse_snapshot(self._h, None, 0, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        self._check(lib().asse_snapshot(self._h, buf, n.value, ctypes.byref(n)))
        return buf.raw

    def probe_random_reads(self, n_reads: int) -> int:
        """Enqueue >= n_reads random 4-byte reads of the pool's words on its
        stream (a measurement aid); returns the number issued."""
        n = u64(0)
        self._check(lib().asse_probe_random_reads(self._h, int(n_reads), ctypes.byref(n)))
        return int(n.value)

    def load(self, image: bytes):
        self._check(lib().asse_load(self._h, image, len(image)))

    def estimate_learned(self, model, max_log_n: float):
        """Per-ATV learned cardinality estimates [r*E] (torch float32 on the
        device) with the Eq. 2 fallback outside the model's training range,
        and the number of ATVs that fell back; between scan() and advance()."""
        import torch
        rows = self.r * self._info["E"]
        x = torch.empty((rows, FEAT), dtype=torch.bfloat16, device="cuda")
        est = torch.empty(rows, dtype=torch.float32, device="cuda")
        nfb = torch.zeros(1, dtype=torch.int32, device="cuda")
        self._check(lib().asse_estimate_learned(self._h, model._h, float(max_log_n), vp(x.data_ptr()),
                                                vp(est.data_ptr()), vp(nfb.data_ptr())))
        return est, nfb, x

    def candidate_features(self, aips):
        """Candidate feature rows [n][FEAT] (torch bfloat16 on the device) of
        the hosts aips (numpy or torch), between scan() and advance()."""
        import torch
        a = aips if _is_torch(aips) else torch.from_numpy(np.ascontiguousarray(aips, dtype=np.uint32).view(np.int32))
        a = a.cuda().contiguous()
        x = torch.empty((a.numel(), FEAT), dtype=torch.bfloat16, device="cuda")
        self._check(lib().asse_candidate_features(self._h, vp(a.data_ptr()), a.numel(), vp(x.data_ptr())))
        return x

    def report_learned(self, mlp: "MLP", max_log_n: float, out=None):
        """The report with the learned candidate estimate in place of Eq. 4
        (asse_report_learned), between scan() + restore() and advance():
        a structured array, or the count when out (a device tensor of
        SuperPoint records) is given."""
        fn = lambda h, o, cap, n, where: lib().asse_report_learned(h, mlp._h, ctypes.c_float(max_log_n), o, cap, n,
                                                                   where)
        return self._list(fn, out)

    def features(self):
        """Feature rows [r*E][FEAT] (torch bfloat16 on the device) of every
        ATV, between scan() and advance()."""
        import torch
        x = torch.empty((self.r * self._info["E"], FEAT), dtype=torch.bfloat16, device="cuda")
        self._check(lib().asse_features(self._h, vp(x.data_ptr())))
        return x


def probe_bounded_wait(limit_cycles: int, complete: bool) -> tuple[int, int]:
    """Run the library's bounded mbarrier wait once on the current torch
    stream (asse_probe_bounded_wait); returns (status, cycles waited), status
    OK if the barrier completed and ETIMEOUT if the wait gave up."""
    waited = u64(0)
    rc = lib().asse_probe_bounded_wait(vp(_current_stream()), int(limit_cycles), int(bool(complete)),
                                       ctypes.byref(waited))
    if rc not in (OK, ETIMEOUT):
        raise AsseError(rc, "bounded-wait probe failed")
    return rc, int(waited.value)


def synth_candidates(cfg: dict, first: int, n: int, stream: int | None = None):
    """Synthetic candidate states (include/asse_learn.h): (x [n][FEAT] bf16,
    ln n [n] fp32, Eq. 4 estimate [n] fp32), torch tensors on the device."""
    import torch
    c = SynthCfg(int(cfg["k"]), int(cfg["g"]), int(cfg["r"]), int(cfg.get("n_max_log2", 20)),
                 float(cfg.get("bg_max", 0.01)), 0, int(cfg["seed"]), int(cfg["bh_a"]), int(cfg["bh_b"]))
    x = torch.empty((n, FEAT), dtype=torch.bfloat16, device="cuda")
    ln = torch.empty(n, dtype=torch.float32, device="cuda")
    e4 = torch.empty(n, dtype=torch.float32, device="cuda")
    rc = lib().asse_synth_candidates(ctypes.byref(c), first, n, vp(x.data_ptr()), vp(ln.data_ptr()),
                                     vp(e4.data_ptr()), vp(_current_stream() if stream is None else stream))
    if rc != OK:
        raise AsseError(rc, "asse_synth_candidates failed")
    return x, ln, e4


def synth_states(cfg: dict, first: int, n: int, stream: int | None = None):
    """Synthetic training states (include/asse_learn.h): (x [n][FEAT] bf16,
    ln n [n] fp32, Eq. 2 estimate [n] fp32), torch tensors on the device."""
    import torch
    c = SynthCfg(int(cfg["k"]), int(cfg["g"]), int(cfg["r"]), int(cfg.get("n_max_log2", 20)),
                 float(cfg.get("bg_max", 0.01)), 0, int(cfg["seed"]), int(cfg["bh_a"]), int(cfg["bh_b"]))
    x = torch.empty((n, FEAT), dtype=torch.bfloat16, device="cuda")
    ln = torch.empty(n, dtype=torch.float32, device="cuda")
    lc = torch.empty(n, dtype=torch.float32, device="cuda")
    rc = lib().asse_synth_states(ctypes.byref(c), first, n, vp(x.data_ptr()), vp(ln.data_ptr()), vp(lc.data_ptr()),
                                 vp(_current_stream() if stream is None else stream))
    if rc != OK:
        raise AsseError(rc, "asse_synth_states failed")
    return x, ln, lc


class MLP:
    """The learned per-ATV estimator of include/asse_learn.h."""

    def __init__(self, seed: int = 1, stream: int | None = None):
        self._h = vp()
        rc = lib().asse_mlp_create(seed, vp(_current_stream() if stream is None else stream), ctypes.byref(self._h))
        if rc != OK:
            raise AsseError(rc, "asse_mlp_create failed")

    def _check(self, rc):
        if rc != OK:
            raise AsseError(rc, lib().asse_mlp_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().asse_mlp_destroy(self._h)
            self._h = vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        out = np.zeros(MLP_NPARAMS, dtype=np.float32)
        self._check(lib().asse_mlp_get_params(self._h, vp(out.ctypes.data)))
        return out

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == MLP_NPARAMS
        self._check(lib().asse_mlp_set_params(self._h, vp(p.ctypes.data)))

    def grads(self) -> np.ndarray:
        out = np.zeros(MLP_NPARAMS, dtype=np.float32)
        self._check(lib().asse_mlp_get_grads(self._h, vp(out.ctypes.data)))
        return out

    def forward(self, x, y=None):
        """Model outputs of the feature rows x ([n][FEAT] bfloat16 on the
        device), by the tensor-core inference kernel; stream-ordered."""
        import torch
        if y is None:
            y = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        self._check(lib().asse_mlp_forward(self._h, vp(x.data_ptr()), x.shape[0], vp(y.data_ptr())))
        return y

    def set_loss(self, kind: str):
        """'log_mse' (squared error of ln n, the default) or 'rel_mse'
        (squared relative error of the estimate)."""
        self._check(lib().asse_mlp_set_loss(self._h, {"log_mse": 0, "rel_mse": 1}[kind]))

    def check(self):
        """Synchronise; raises if a kernel of this model gave up a wait."""
        self._check(lib().asse_mlp_check(self._h))

    def backward(self, x, t):
        import torch
        loss = torch.zeros(1, dtype=torch.float32, device=x.device)
        self._check(lib().asse_mlp_backward(self._h, vp(x.data_ptr()), vp(t.data_ptr()), x.shape[0],
                                            vp(loss.data_ptr())))
        return loss

    def train_step(self, x, t, lr: float):
        import torch
        loss = torch.zeros(1, dtype=torch.float32, device=x.device)
        self._check(lib().asse_mlp_train_step(self._h, vp(x.data_ptr()), vp(t.data_ptr()), x.shape[0], lr,
                                              vp(loss.data_ptr())))
        return loss
