"""The C-ABI library builds, loads and exports every function that
include/vqhull.h declares; host-side argument checks (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "vqhull.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vq_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import paper_2510_09417_gb300 as v
    return v.load()


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    import paper_2510_09417_gb300 as v
    assert set(v.SYMBOLS) == set(names)


def test_status_strings(lib):
    import paper_2510_09417_gb300 as v
    for code in range(-9, 2):
        s = v.status_string(code)
        assert s and s != "unknown status"
    assert v.status_string(1234) == "unknown status"
    assert v.vq_version() >= 100


def test_host_side_argument_checks(lib):
    h = ctypes.c_int64(7)
    # n = 0 is a valid empty hull and touches no device
    assert lib.vq_hull2d(None, None, 0, None, ctypes.byref(h), None) == 0 and h.value == 0
    assert lib.vq_hull2d(None, None, -1, None, ctypes.byref(h), None) == -1
    assert lib.vq_hull2d(None, None, 5, None, ctypes.byref(h), None) == -1
    assert lib.vq_hull2d(1, 1, 5, 1, None, None) == -1
    assert lib.vq_hull2d(1, 1, 2 ** 31, 1, ctypes.byref(h), None) == -3
    assert lib.vq_hull2d_batched(1, 1, None, 1, 1, 1, None) == -1
    assert lib.vq_hull2d_batched(1, 1, 1, 0, 1, 1, None) == -1
    assert lib.vq_hull2d_host(None, None, 0, None, ctypes.byref(h), None) == 0


def test_config_validation(lib):
    import paper_2510_09417_gb300 as v
    cfg = v.vq_get_config()
    assert cfg.points_per_thread in (4, 8, 16)
    for bad in ({"points_per_thread": 5}, {"small_max": 1}, {"small_max": 4096},
                {"timeout_ns": 0}, {"k1_blocks_per_sm": -1}):
        c = v.vq_get_config()
        for k, val in bad.items():
            setattr(c, k, val)
        assert lib.vq_set_config(ctypes.byref(c)) == -1
    assert lib.vq_set_config(ctypes.byref(cfg)) == 0
    # the level-loop and pre-filter switches round-trip
    c = v.vq_get_config()
    c.host_loop, c.prefilter = 1, 0
    assert lib.vq_set_config(ctypes.byref(c)) == 0
    got = v.vq_get_config()
    assert (got.host_loop, got.prefilter) == (1, 0)
    assert lib.vq_set_config(ctypes.byref(cfg)) == 0
    assert (v.vq_get_config().host_loop, v.vq_get_config().prefilter) == (cfg.host_loop, cfg.prefilter)


def test_autotune_argument_checks(lib):
    import paper_2510_09417_gb300 as v
    c = v.vqhull.Config()
    ms = ctypes.c_double()
    assert lib.vq_autotune(1, 1, 0, 2, ctypes.byref(c), ctypes.byref(ms), None) == -1
    assert lib.vq_autotune(None, 1, 10, 2, ctypes.byref(c), ctypes.byref(ms), None) == -1
    assert lib.vq_autotune(1, 1, 10, 0, ctypes.byref(c), ctypes.byref(ms), None) == -1
    assert lib.vq_autotune(1, 1, 10, 17, ctypes.byref(c), ctypes.byref(ms), None) == -1
    assert lib.vq_autotune(1, 1, 2 ** 31, 2, ctypes.byref(c), ctypes.byref(ms), None) == -3


def test_server_rejects_bad_config(lib):
    import paper_2510_09417_gb300 as v
    out = ctypes.c_void_p()
    cfg = v.vqhull.ServerConfig(0, 1, 0)
    assert lib.vq_server_create(ctypes.byref(cfg), ctypes.byref(out)) == -1
    cfg = v.vqhull.ServerConfig(1 << 30, 0, 0)
    assert lib.vq_server_create(ctypes.byref(cfg), ctypes.byref(out)) == -1
    cfg = v.vqhull.ServerConfig(1 << 30, 4, 0, 17)   # more lanes than allowed
    assert lib.vq_server_create(ctypes.byref(cfg), ctypes.byref(out)) == -1
    cfg = v.vqhull.ServerConfig(1 << 30, 4, 0, -1)
    assert lib.vq_server_create(ctypes.byref(cfg), ctypes.byref(out)) == -1
