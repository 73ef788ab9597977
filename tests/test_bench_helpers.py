"""Host logic of bench.py that decides what its JSON line reports:
the DRAM traffic of a kernel is reported only for the kernel source it was
captured on, the algorithmic FLOP count follows the model's sizes, and the CPU
description is non-empty."""
import os

import bench
from synth import configs as C


def test_traffic_is_reported_only_for_the_captured_source(monkeypatch):
    rel, sha = bench.NCU_TRAFFIC_SOURCE
    assert os.path.exists(os.path.join(bench.ROOT, rel))
    current = bench._source_sha(rel)
    want = bench.NCU_TRAFFIC_PER_ATOM["k_af_bwd"]
    if current == sha:
        assert bench.traffic_per_atom("k_af_bwd") == want
    # another source: no number
    monkeypatch.setattr(bench, "NCU_TRAFFIC_SOURCE", (rel, "0" * 16))
    assert bench.traffic_per_atom("k_af_bwd") is None
    monkeypatch.setattr(bench, "NCU_TRAFFIC_SOURCE", (rel, current))
    assert bench.traffic_per_atom("k_af_bwd") == want
    assert bench.traffic_per_atom("k_fit") is None      # never captured


def test_algorithmic_flops_follow_the_model():
    m = C.ATTN_MODEL
    fwd, fit, bwd = bench.af_flops_per_atom(m, 90)
    # embedding 2 n (e1 + e1 e2 + e2 m1) at n = 90
    emb = 2 * 90 * (32 + 32 * 64 + 64 * 128)
    assert fwd > emb and bwd > emb
    # fitting forward + input gradient: 2 x 2 (m1 m2 f1 + f1 f2 + f2 f3 + f3)
    assert fit == 4 * (128 * 16 * 240 + 240 * 240 + 240 * 240 + 240)
    # attention terms grow as n^2: doubling n more than doubles each part
    f2, _, b2 = bench.af_flops_per_atom(m, 180)
    assert f2 > 2 * fwd and b2 > 2 * bwd
    # no neighbours: the fitting alone (and the descriptor's constant term)
    f0, _, _ = bench.af_flops_per_atom(m, 0)
    assert f0 == 2 * 4 * 128 * 16


def test_cpu_model_is_described():
    assert isinstance(bench.cpu_model(), str) and bench.cpu_model()
