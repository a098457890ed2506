"""Host-side arithmetic of bench.py (no GPU): the attention pair count behind the
roofline's algorithmic exponentials, full and windowed, against the oracle's
window mask counted element by element."""
import numpy as np

import bench
import oracle
import synth


def test_attention_pairs_full():
    sizes = np.array([1, 17, 300, 0, 2500])
    assert bench.attention_pairs(sizes, 0) == float((sizes.astype(np.int64) ** 2).sum())


def test_attention_pairs_windowed_match_mask():
    for w in (1, 2, 4):
        sizes = np.array([1, 127, 128, 129, 700, 1300])
        expect = sum(int(oracle.window_mask(int(n), w).sum()) for n in sizes)
        assert bench.attention_pairs(sizes, w) == expect
    # a window reaching every block is full attention
    assert bench.attention_pairs(np.array([700]), 6) == 700 ** 2


def test_gemm_flops_per_element_d64_model():
    """About 2.7e5 GEMM flops per element for the d=64, FFN 256, 1 + 1 model (an
    estimate made independently from the layer sizes); one more encoder block adds
    its projections and FFN."""
    import bench
    f = bench.gemm_flops_per_element(synth.SMALL)
    assert abs(f - 2.7e5) / 2.7e5 < 0.03, f
    # one more encoder block adds 2 (3 d^2 + d^2 + 2 d F) flops
    import dataclasses
    deeper = dataclasses.replace(synth.SMALL, l_pid=2)
    assert bench.gemm_flops_per_element(deeper) - f == 2 * (4 * 64 * 64 + 2 * 64 * 256)


def test_gemm_chain_bytes_per_element_d64_model():
    """About 2.7 KB of algorithmic DRAM traffic per element for the d=64 1 + 1 model's
    four chain kernels (808 + 536 + 936 + 412 bytes from the tensors each one reads and
    writes); a block boundary adds O, the residual stream in and out and Q, K, V^T."""
    import bench
    assert bench.gemm_chain_bytes_per_element(64, 0) == 808 + 536 + 936 + 412
    assert bench.gemm_chain_bytes_per_element(64, 1) - bench.gemm_chain_bytes_per_element(64, 0) == \
        2 * 64 + 2 * 4 * 64 + 3 * 2 * 64


def test_reference_arm_json_line(capsys, monkeypatch):
    """`bench.py --impl reference`: one JSON line with the contract's keys (the oracle
    timed on the host cores, no host-device copies), printed by rank 0 only."""
    import argparse
    import json
    monkeypatch.setenv("RANK", "0")
    args = argparse.Namespace(gpus=1, steps=1, warmup=0, model="small")
    bench.run_reference(args)
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "events/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["dtype"] == "f64"
    assert d["steps"] == 1 and d["n_gpus"] == 1 and d["vs_baseline"] is None
    assert d["config"]["workload"].startswith(bench.WORKLOAD)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    monkeypatch.setenv("RANK", "1")
    bench.run_reference(args)
    assert capsys.readouterr().out.strip() == ""


def test_oracle_baseline_on_all_cores():
    """The CPU baseline: the oracle over a bounded sample of events on one worker
    process per host core, extrapolated to the batch by sum N^2, a one-core run of
    the next events, per-event latencies, and the host's core count and CPU model;
    the sampled outputs are the oracle's own."""
    import os
    cfg = synth.SMALL
    sizes = np.array([40, 90, 10, 70, 30, 55, 20, 65, 80, 15, 35, 45])
    x, cu = synth.gen_events(7, sizes)
    res, cb = bench.oracle_baseline(cfg, 0, x, cu, sizes, budget_s=0.0)
    assert cb["kind"] == "oracle" and cb["cores"] == (os.cpu_count() or 1) == cb["nproc"]
    assert cb["value"] > 0 and cb["one_core"]["value"] > 0 and cb["cpu_model"]
    assert 0 < cb["p50_ms_per_event"] <= cb["p99_ms_per_event"]
    # a zero budget still runs the first event; results come back in event order
    assert [r[0] for r in res] == list(range(len(res))) and len(res) >= 1
    W = synth.make_weights(cfg, 0)
    e, _, lo, reg, cls, sums = res[0]
    ref = oracle.forward(W, cfg, x[cu[e]:cu[e + 1]], [0, int(sizes[e])])
    assert np.array_equal(lo, ref.logits) and np.array_equal(cls, ref.cls)
