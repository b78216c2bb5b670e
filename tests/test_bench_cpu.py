"""Host logic of bench.py (no GPU): the algorithmic byte count of the trace
roofline, the surrogate's tensor roofline, the hand-off schedule labels, and
that the committed DRAM-traffic capture still belongs to the current trace
sources and to the schedule the default benchmark runs."""
import argparse
import hashlib
import json
import os

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _args(**kw):
    a = dict(method="ddm", continue_cells=False, handoff_waves=1)
    a.update(kw)
    return argparse.Namespace(**a)


def test_trace_bytes_leave_out_carried_crossings():
    st = dict(ray_visits=1000, crossings=300, segments_ext=400, node_visits=5000, tri_tests=2000)
    base = 48 * 1000 + 48 * 300 + 32 * 400 + 64 * 5000 + 48 * 2000
    assert bench._trace_bytes(st) == base
    # a crossing the tracing thread carries on itself reads and writes no ray record
    assert bench._trace_bytes(dict(st, ray_continues=120)) == base - 120 * 96


def test_mlp_tensor_roofline():
    assert bench.MLP_TENSOR_FLOP_PER_ROW == 2 * (4 * 64 + 64 * 64 + 64 * 64)
    r = bench._mlp_tensor([dict(mlp_ms=2.0, mlp_rows=10 ** 8), dict(mlp_ms=2.0, mlp_rows=10 ** 8)])
    want = 2 * 10 ** 8 * bench.MLP_TENSOR_FLOP_PER_ROW / 4e-3 / 1e12
    assert r["achieved"] == pytest.approx(want, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-3)
    assert r["rows_per_step"] == 10 ** 8 and r["bound"] == "tensor"
    assert bench._mlp_tensor([dict(mlp_ms=0.0, mlp_rows=0)]) is None


def test_handoff_names():
    assert bench._handoff_name(_args(handoff_waves=0)) == "neighbour queue"
    assert bench._handoff_name(_args(continue_cells=True)) == "lane continues"
    assert bench._handoff_name(_args()) == "neighbour queue for 1 wave, then the thread carries the rest"
    assert bench._handoff_name(_args(handoff_waves=2)).startswith("neighbour queue for 2 waves")
    assert bench._handoff_name(_args(method="megakernel")) is None


def test_traffic_capture_matches_sources_and_default_schedule():
    with open(os.path.join(ROOT, "profiles", "trace_traffic.json")) as f:
        tt = json.load(f)
    ent = tt["ddm:hotel_room_512x512_16spp_d5_L41"]
    m = hashlib.sha256()
    for src in ent["sources"]:
        with open(os.path.join(ROOT, src), "rb") as f:
            m.update(f.read())
    assert m.hexdigest()[:16] == ent["source_sha256_16"], "trace sources changed since the traffic capture"
    default = bench._handoff_name(_args(handoff_waves=1))
    assert ent["ddm_handoff"] == default
    assert ent["dram_bytes_per_launch"] > 0
