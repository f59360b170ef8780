"""The committed ncu records that bench.py reports (host logic, no GPU): the DROP traffic
record and the on-the-fly kernel's fractions are used only while the hash of the kernel
sources they were taken on matches, and the traffic only on the configuration it was
scaled to; every other line reports null."""
import json

import pytest


def _record(bench, name):
    return json.load(open(bench.os.path.join(bench.ROOT, "profiles", name)))


def _headline_config(bench):
    want = dict(_record(bench, "drop_block_traffic.json")["applies_to"])
    dtype = want.pop("dtype")
    return want, dtype


@pytest.fixture
def sources_as_recorded(monkeypatch):
    """The kernel sources hashed as the records say (whether or not they changed since)."""
    import bench
    monkeypatch.setattr(bench, "drop_kernel_hash",
                        lambda: _record(bench, "drop_block_traffic.json")["kernel_src_sha256"])
    monkeypatch.setattr(bench, "otf_kernel_hash",
                        lambda: _record(bench, "otf_drop_kernel_fractions.json")["kernel_src_sha256"])
    return bench


def test_traffic_record_applies_to_its_configuration_only(sources_as_recorded):
    bench = sources_as_recorded
    cfg, dtype = _headline_config(bench)
    got = bench.ncu_traffic_per_launch(cfg, dtype)
    assert got is not None and got > 0
    # the record is per launch of the full workload: above the algorithmic bytes of a
    # launch (entries x 8 B + rows x 16 B), never wildly so
    d = _record(bench, "drop_block_traffic.json")
    assert 1.0 < got / min(d["dram_bytes_per_captured_launch"]) < 1.5
    for key, other in [("workload", cfg["workload"] + "_first1000000rows"), ("storage", "delta16"),
                       ("drop_schedule", "plain"), ("voxel_tile", "1x1")]:
        assert bench.ncu_traffic_per_launch(dict(cfg, **{key: other}), dtype) is None, key
    assert bench.ncu_traffic_per_launch(cfg, "f64") is None


def test_records_are_dropped_when_the_kernel_source_changes(sources_as_recorded, monkeypatch):
    bench = sources_as_recorded
    cfg, dtype = _headline_config(bench)
    assert bench.ncu_traffic_per_launch(cfg, dtype) is not None
    assert bench.otf_profile_fractions() is not None
    monkeypatch.setattr(bench, "drop_kernel_hash", lambda: "0" * 64)
    monkeypatch.setattr(bench, "otf_kernel_hash", lambda: "0" * 64)
    assert bench.ncu_traffic_per_launch(cfg, dtype) is None
    assert bench.otf_profile_fractions() is None


@pytest.mark.parametrize("name", ["drop_block_traffic.json", "otf_drop_kernel_fractions.json"])
def test_records_name_their_source_hash(name):
    import bench
    h = _record(bench, name)["kernel_src_sha256"]
    assert len(h) == 64 and all(ch in "0123456789abcdef" for ch in h)
