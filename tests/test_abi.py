"""CPU-side checks of the C ABI: libasse.so builds, loads without a GPU,
exports every entry point include/asse.h declares (and the binding knows
them all), and rejects invalid pool parameters before any CUDA call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1807_01527_gb300 import asse, build
    build.build()
    return asse.lib()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^ASSE_API\s+[\w\s\*]*?\b(asse_\w+)\s*\(", txt, flags=re.M))
    return names


def test_every_declared_symbol_is_exported(lib):
    from paper_1807_01527_gb300 import asse
    declared = _declared()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(asse.EXPORTS), declared ^ set(asse.EXPORTS)


def test_struct_sizes_match_header(lib):
    from paper_1807_01527_gb300 import asse
    assert ctypes.sizeof(asse.Config) == 8 * 4 + 2 * 8 + 2 * 4 + 8 + 2 * 4
    assert ctypes.sizeof(asse.SuperPoint) == 16 == asse.SP_DTYPE.itemsize


def _cfg(**kw):
    from paper_1807_01527_gb300 import asse
    base = dict(k=10, theta=1024, g=512, r=4, c=12, u=4, s=6, A=123456789, bh_a=0x9E3779B97F4A7C15, bh_b=7,
                counter=0, restore_cap=0, max_batch=0, key_table=0, cluster=0)
    base.update(kw)
    return asse.Config(*[base[f] for f, _ in asse.Config._fields_])


@pytest.mark.parametrize("bad,msg", [
    (dict(k=0), "k must"), (dict(k=128), "k must"), (dict(g=19, k=10), "g must"), (dict(g=5000), "g must"),
    (dict(r=1), "r must"), (dict(r=9), "r must"), (dict(c=17), "c <= 16"), (dict(u=9), "u <= 8"),
    (dict(s=0), "s <= c"), (dict(s=13), "s <= c"), (dict(s=3), "completeness"), (dict(A=1), "A must"),
    (dict(bh_a=2), "odd"), (dict(counter=4), "counter"), (dict(theta=0), "theta"),
    (dict(key_table=3), "key_table"), (dict(cluster=3), "cluster"), (dict(cluster=16), "cluster"),
    (dict(c=12, u=4, s=10), "s*(r-1) < 32-u"), (dict(k=100, g=4000), "512 words"),
])
def test_invalid_configs_rejected_without_gpu(lib, bad, msg):
    from paper_1807_01527_gb300 import asse
    h = ctypes.c_void_p()
    cfg = _cfg(**bad)
    rc = lib.asse_create(ctypes.byref(cfg), None, ctypes.byref(h))
    assert rc == asse.EINVAL
    assert not h.value
    assert msg in lib.asse_last_error(None).decode()


def test_null_arguments(lib):
    from paper_1807_01527_gb300 import asse
    assert lib.asse_create(None, None, ctypes.byref(ctypes.c_void_p())) == asse.EINVAL
    assert lib.asse_ingest(None, None, 5, 0) == asse.EINVAL
    assert lib.asse_close_slice(None, 1) == asse.EINVAL
    lib.asse_destroy(None)
    assert lib.asse_strerror(asse.ECAPACITY) == b"ASSE_ECAPACITY"
    assert lib.asse_strerror(asse.EAGAIN) == b"ASSE_EAGAIN"
    assert lib.asse_strerror(asse.ETIMEOUT) == b"ASSE_ETIMEOUT"
    assert lib.asse_report_learned(None, None, 1.0, None, 0, None, asse.HOST) == asse.EINVAL
    # the wait bound is checked before any CUDA call
    assert lib.asse_probe_bounded_wait(None, 0, 0, None) == asse.EINVAL
    assert lib.asse_probe_bounded_wait(None, (1 << 36) + 1, 0, None) == asse.EINVAL
