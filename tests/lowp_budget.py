"""Error budget of the 16-bit forward: which rounding costs the accuracy.

TEST INFRASTRUCTURE.  Runs the float64 emulation of `tests/lowp_emul.py` on the
64-event precision workload (N ~ U{1000..6000}, d = 64 model, Xavier weights of
seed 0) and prints, for one stage rounded at a time and for every stage but
one, the class-argmax agreement with the FP64 oracle, the RMS class-logit error
and the largest normwise column error of the decoded regressions.

Usage: python -m tests.lowp_budget [--fmt bf16] [--events 64] [--procs 8]
       [--set stage=fmt ...]   (the reference configuration: the GPU mode's
                                formats with these stages changed)
       [--blob model.blob]     (weights from a blob file of the d = 64 architecture,
                                e.g. a trained model, instead of the seeded ones)
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402
from tests.lowp_emul import STAGES, Emulation, gpu_formats  # noqa: E402


def _weights(blob):
    """The workload model's weights: seeded, or from a blob of the same architecture."""
    cfg, wseed, _, _ = synth.workload("prec64")
    if not blob:
        return cfg, synth.make_weights(cfg, wseed)
    bcfg, W = synth.unpack_blob(open(blob, "rb").read())
    assert bcfg == cfg, (bcfg, cfg)
    return cfg, W


def _calib(args):
    fmt, ev, blob = args
    cfg, W = _weights(blob)
    sizes = synth.sizes_lognormal(999, 32)
    x, cu = synth.gen_events(999, sizes)
    em = Emulation(W, cfg, fmt)
    em.record = {}
    em.forward(x, cu, events=[ev])
    return em.record


def calibrate(pool, n_events, blob=""):
    """Static E4M3 activation scales amax/448 from the FP16 emulation on the first
    n_events of the calibration events (seed 999), as the library calibrates."""
    recs = pool.map(_calib, [(gpu_formats("fp16"), e, blob) for e in range(n_events)])
    amax = {}
    for r in recs:
        for k, v in r.items():
            amax[k] = max(amax.get(k, 0.0), v)
    return {k: (v / 448.0 if v > 0 else 1.0) for k, v in amax.items()}


def _run(args):
    fmt, ev, scales, blob = args
    _, _, seed, sizes = synth.workload("prec64")
    cfg, W = _weights(blob)
    x, cu = synth.gen_events(seed, sizes)
    em = Emulation(W, cfg, fmt, scales)
    lo, raw, reg, cls, rows = em.forward(x, cu, events=[ev])
    return lo, reg, cls


def batch(pool, fmt, events, scales=None, blob=""):
    res = pool.map(_run, [(fmt, e, scales, blob) for e in events])
    return tuple(np.concatenate([r[i] for r in res]) for i in range(3))


def stats(out, ref):
    lo, reg, cls = out
    rlo, rreg, rcls = ref
    agree = float((cls == rcls).mean())
    lerr = float(np.sqrt(((lo - rlo) ** 2).mean()))
    col = np.sqrt(((reg - rreg) ** 2).sum(0)) / np.sqrt((rreg ** 2).sum(0))
    return agree, lerr, float(col.max()), REG_COLS[int(col.argmax())]


REG_COLS = ("pT", "eta", "sin", "cos", "E")


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--fmt", default="bf16")
    ap.add_argument("--events", type=int, default=64)
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--set", action="append", default=[], help="stage=fmt override (fmt 'none' = float64)")
    ap.add_argument("--only-config", action="store_true", help="just the reference configuration")
    ap.add_argument("--calib", type=int, default=8, help="calibration events for E4M3 scales")
    ap.add_argument("--stages", default="", help="comma-separated stages to ablate (default: all rounded)")
    ap.add_argument("--blob", default="", help="weights from this blob (the d = 64 architecture)")
    a = ap.parse_args(argv)
    base = gpu_formats(a.fmt)
    for kv in a.set:
        k, v = kv.split("=")
        assert k in STAGES, k
        base[k] = None if v == "none" else v
    events = list(range(a.events))
    ctx = mp.get_context("spawn")
    with ctx.Pool(a.procs) as pool:
        scales = calibrate(pool, a.calib, a.blob) if "e4m3" in base.values() else None
        ref = batch(pool, {}, events, blob=a.blob)
        n = len(ref[2])
        print(f"{a.fmt}: {a.events} events, {n} elements; overrides {a.set or 'none'}; "
              f"weights {a.blob or 'seeded'}")
        ag, le, ce, cn = stats(batch(pool, base, events, scales, a.blob), ref)
        print(f"{'configuration':28s} {'agree':>8s} {'flips':>6s} {'rms logit err':>14s} {'max col err':>12s}")
        print(f"{'all stages as configured':28s} {ag:8.5f} {round((1 - ag) * n):6d} {le:14.3e} {ce:12.3e} {cn}",
              flush=True)
        if a.only_config:
            return
        only = [t for t in a.stages.split(",") if t] or STAGES
        for s in only:
            if base.get(s) is None:
                continue
            f = dict(base)
            f[s] = None
            ag, le, ce, cn = stats(batch(pool, f, events, scales, a.blob), ref)
            print(f"{'all but ' + s:28s} {ag:8.5f} {round((1 - ag) * n):6d} {le:14.3e} {ce:12.3e} {cn}", flush=True)
        for s in only:
            if base.get(s) is None:
                continue
            ag, le, ce, cn = stats(batch(pool, {s: base[s]}, events, scales, a.blob), ref)
            print(f"{'only ' + s:28s} {ag:8.5f} {round((1 - ag) * n):6d} {le:14.3e} {ce:12.3e} {cn}", flush=True)


if __name__ == "__main__":
    main()
