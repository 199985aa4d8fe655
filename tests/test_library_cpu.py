"""Host-side checks of the C-ABI library that need no GPU: it builds, loads,
exports every symbol include/bouquet.h declares, and rejects bad arguments
before touching the device."""

import ctypes
import os
import re

import pytest

import paper_2410_14056_gb300 as bq
from paper_2410_14056_gb300 import bouquet as binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    names = set()
    include = os.path.join(ROOT, "include")
    for fn in os.listdir(include):
        if fn.endswith(".h"):
            text = open(os.path.join(include, fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(bq_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return bq.load_library()


def test_exports_every_declared_symbol(lib):
    declared = header_functions()
    assert {"bq_graph_create", "bq_walk_batch", "bq_aesc_estimate", "bq_sync"} <= declared
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert set(binding.EXPORTS) <= declared | set()


def test_strerror_and_version(lib):
    assert lib.bq_strerror(0) == b"ok"
    assert lib.bq_strerror(bq.ENOEDGE) == b"vertex pair is not an edge"
    assert lib.bq_strerror(-99) == b"unknown status code"
    assert bq.version().startswith("bouquet-gb300")


def test_argument_errors_without_device(lib):
    out = ctypes.c_void_p()
    assert lib.bq_graph_create(3, None, None, 0, None, ctypes.byref(out)) == bq.EINVAL
    assert b"offsets" in lib.bq_last_error()
    assert lib.bq_graph_create(3, None, None, 0, None, None) == bq.EINVAL
    assert lib.bq_walk_batch(None, 0, None, 0, 1, 0, None, 0, None, None, None) == bq.EINVAL
    assert lib.bq_aesc_plan(None, None, 0, 0.1, 0.01, 0, None, None, None) == bq.EINVAL
    assert lib.bq_aesc_estimate_push(None, 0, None, 0, None, None, 1, 512, 0, None, None, None, None) == bq.EINVAL
    assert lib.bq_graph_destroy(None) == bq.OK


def test_server_argument_errors_without_device(lib):
    out = ctypes.c_void_p()
    assert lib.bq_server_create(None, 0, None, ctypes.byref(out)) == bq.EINVAL
    assert out.value is None
    assert lib.bq_server_create(None, 1, None, None) == bq.EINVAL
    rid = ctypes.c_uint64()
    assert lib.bq_server_submit(None, 0, None, 0, 0.1, 0, ctypes.byref(rid)) == bq.EINVAL
    assert lib.bq_server_wait(None, 1, 0.0, None, None, None) == bq.EINVAL
    assert lib.bq_server_stats_get(None, None) == bq.EINVAL
    assert lib.bq_server_destroy(None) == bq.OK


def test_tuning_roundtrip_and_validation(lib):
    old = bq.get_tuning()
    try:
        bq.set_tuning(walk_lanes=2, aggregate_visits=1, aesc_lanes=8)
        assert bq.get_tuning() == dict(old, walk_lanes=2, aggregate_visits=1, aesc_lanes=8)
        assert (old["relabel_hub8"], old["hub8_hubs"], old["hub8_count_bits"], old["shared_lanes"]) == (1, 0, 0, 2)
        assert (old["group_walks"], old["push_lanes"]) == (1, 2)
        for ok in (4, 8, 2):
            bq.set_tuning(push_lanes=ok)
            assert bq.get_tuning()["push_lanes"] == ok
        for bad in (dict(shared_lanes=3), dict(shared_lanes=0), dict(push_lanes=1), dict(push_lanes=0)):
            with pytest.raises(bq.BouquetError):
                bq.set_tuning(**bad)
        bq.set_tuning(relabel_hub8=0, hub8_hubs=28000, hub8_count_bits=31)
        assert bq.get_tuning()["hub8_hubs"] == 28000
        for bad in (dict(relabel_hub8=2), dict(hub8_hubs=28001), dict(hub8_count_bits=32)):
            with pytest.raises(bq.BouquetError):
                bq.set_tuning(**bad)
        with pytest.raises(ValueError):
            bq.set_tuning(no_such_knob=1)
        bq.set_tuning(relabel_hub8=1, hub8_hubs=0, hub8_count_bits=0)
        bq.set_tuning(hub_relabel=1)
        assert bq.get_tuning()["hub_relabel"] == 1
        with pytest.raises(bq.BouquetError):
            bq.set_tuning(hub_relabel=2)
        bq.set_tuning(hub_relabel=0)
        assert old["aesc_hub"] == 0  # off by default
        for ok in (1, 2, 4, 8):
            bq.set_tuning(hub_cluster=ok)
            assert bq.get_tuning()["hub_cluster"] == ok
        bq.set_tuning(hub_cluster=0)
        assert bq.get_tuning()["hub_cluster"] == 1  # 0 means one CTA
        for bad in (3, 16):
            with pytest.raises(bq.BouquetError):
                bq.set_tuning(hub_cluster=bad)
        bq.set_tuning(aesc_hub=1)
        assert bq.get_tuning()["aesc_hub"] == 1
        with pytest.raises(bq.BouquetError):
            bq.set_tuning(aesc_hub=2)
        with pytest.raises(bq.BouquetError):
            bq.set_tuning(layout=6)
        assert old["hub_slots"] == 8192
        for bad in (1, 1023, 13313, 1 << 14):
            with pytest.raises(bq.BouquetError):
                bq.set_tuning(hub_slots=bad)
        for ok in (0, 1024, 5000, 13312):
            bq.set_tuning(hub_slots=ok)
            assert bq.get_tuning()["hub_slots"] == ok
        with pytest.raises(bq.BouquetError) as ei:
            bq.set_tuning(walk_lanes=3)
        assert ei.value.code == bq.EINVAL
        with pytest.raises(bq.BouquetError):
            bq.set_tuning(aesc_lanes=1)
    finally:
        bq.set_tuning(**old)


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        binding.load_library(str(tmp_path / "libbouquet.so"))
