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


def test_reference_arm_json_line(capsys, monkeypatch):
    """`bench.py --impl reference`: one JSON line with the contract's keys (the oracle
    timed on the host cores, no host-device copies), printed by rank 0 only."""
    import argparse
    import json
    monkeypatch.setenv("RANK", "0")
    args = argparse.Namespace(gpus=1, steps=1, warmup=0)
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
