"""Distil a student MLPF from the full model and measure gated inference.

Teacher: the full-size model (width 256, 8 heads of 32, FFN 1024, 3 + 3 blocks), either
(--teacher random) with random weights and its class head's last layer scaled so that
about 95 % of elements get a class probability >= 0.9 (random weights give flat class
scores), or (--teacher trained) trained first, with the same kernels and LAMB, on the
deterministic synthetic truth of synth.gen_pf_truth (target logits TRUTH_LOGIT on the
true class, 0 elsewhere; the truth's decoded regression targets), as the paper's full
model is a trained one; run in BF16 on the generic-width tensor-core path for the
training targets and the gated fallback (--teacher-precision), and in FP32 as the
reference the agreement is measured against.
Student (--student): d64 = width 64, 4 heads of 16, FFN 256, 1 + 1 blocks (the fused
tensor-core kernels), or cfg5 = width 128, 4 heads of 32, FFN 512, 2 + 2 blocks (the
distillation configuration; the generic-width tensor-core path), both run in BF16;
trained on the teacher's per-element outputs (class scores and the 5 regressions) of
synthetic events with N ~ U{1000..6000} elements, with the library's hand-written
forward/backward kernels (BF16 tensor-core GEMMs and attention by default,
--train-precision) and LAMB (learning rate 2e-3 -> 2e-4 on a cosine schedule, Sec. 5.3).
Evaluation: the 512-event workload run by the teacher alone, the student alone and
the student with per-event fallback to the teacher below a class confidence threshold.

    python -m paper_2601_17554_b300.distill [--train-events 20000] [--epochs 2]
        [--batch-events 32] [--student d64|cfg5] [--out student.blob] [--json result.json]
        [--teacher random|trained] [--teacher-steps 1500] [--teacher-blob t.blob]
        [--teacher-out t.blob]
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

TEACHER_SEED, STUDENT_SEED = 1, 0
# the distillation configuration's student: width 128, 4 heads of 32, FFN 512, 2 + 2 blocks
STUDENT_CFG5 = synth.ModelConfig(d=128, heads=4, ffn=512, l_pid=2, l_reg=2)
TRAIN_SEED, SCALE_SEED = 2000, 12345
TRUTH_LOGIT = 6.0   # target logit of the true class when the teacher is trained on the truth


def _gen_chunk(args):
    seed, sizes, first, truth = args
    x, cu = synth.gen_events(seed, sizes, first_event=first)
    if not truth:
        return x, cu
    return (x, cu) + synth.gen_pf_truth(x, cu)


def gen_parallel(seed, sizes, chunk, workers, truth=False):
    """Events in chunks of `chunk` (with their synthetic truth if `truth`), generated
    by a spawn process pool."""
    jobs = [(seed, sizes[i:i + chunk], i, truth) for i in range(0, len(sizes), chunk)]
    if workers <= 1:
        return [_gen_chunk(j) for j in jobs]
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_gen_chunk, jobs)


def softmax_max(logits):
    z = logits - logits.max(1, keepdims=True)
    return 1.0 / np.exp(z).sum(1)


def find_cls_scale(logits, target_frac=0.95, conf=0.9):
    """Smallest s (bisection) with frac(max softmax(s * logits) >= conf) >= target_frac."""
    lo, hi = 1.0, 4096.0
    for _ in range(60):
        mid = math.sqrt(lo * hi)
        if (softmax_max(mid * logits) >= conf).mean() >= target_frac:
            hi = mid
        else:
            lo = mid
    return hi


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--train-events", type=int, default=20000)
    ap.add_argument("--epochs", type=int, default=2)
    ap.add_argument("--batch-events", type=int, default=32)
    ap.add_argument("--threshold", type=float, default=0.9)
    ap.add_argument("--workers", type=int, default=min(16, os.cpu_count() or 1))
    ap.add_argument("--out", default="")
    ap.add_argument("--json", default="")
    ap.add_argument("--student", default="d64", choices=["d64", "cfg5"])
    ap.add_argument("--train-precision", default="bf16", choices=["fp32", "bf16", "fp16"],
                    help="trainer arithmetic: 16-bit tensor-core GEMMs and attention, or FP32")
    ap.add_argument("--teacher-precision", default="bf16", choices=["fp32", "bf16", "fp16"],
                    help="teacher forward for the training targets and the gated fallback "
                         "(agreement is always measured against the FP32 teacher)")
    ap.add_argument("--student-blob", default="",
                    help="evaluate this trained student (skip the training)")
    ap.add_argument("--teacher", default="random", choices=["random", "trained"],
                    help="random weights with a scaled class head, or trained on synth.gen_pf_truth")
    ap.add_argument("--teacher-steps", type=int, default=1500,
                    help="LAMB steps of the teacher's training (--teacher trained)")
    ap.add_argument("--teacher-blob", default="", help="a trained teacher to load (skips its training)")
    ap.add_argument("--teacher-out", default="", help="write the trained teacher here")
    args = ap.parse_args(argv)
    if args.student_blob:
        args.train_events = args.batch_events   # only the teacher's confidence scale is needed

    # generate the training set before any CUDA call (spawned workers)
    t0 = time.time()
    train_sizes = synth.sizes_uniform(TRAIN_SEED, args.train_events)
    chunks = gen_parallel(TRAIN_SEED, train_sizes, args.batch_events, args.workers,
                          truth=args.teacher == "trained")
    gen_s = time.time() - t0

    import torch
    from paper_2601_17554_b300 import Model, Trainer, _lib, forward_gated

    dev = torch.device("cuda", 0)
    res = {"train_events": args.train_events, "train_elements": int(train_sizes.sum()),
           "generation_s": gen_s}

    res["teacher_kind"] = args.teacher
    if args.teacher == "random":
        # teacher class-head scale (A15 reading): 95 % of elements at max softmax >= 0.9
        w1 = synth.make_weights(synth.FULL, TEACHER_SEED)
        probe = Model(synth.pack_blob(synth.FULL, w1))
        ps = synth.sizes_uniform(SCALE_SEED, 8)
        px, pcu = synth.gen_events(SCALE_SEED, ps)
        plog, _, _, _ = probe.forward(torch.from_numpy(px).to(dev), torch.from_numpy(pcu).to(dev),
                                      int(ps.max()), precision="fp32")
        scale = find_cls_scale(plog.cpu().numpy().astype(np.float64))
        probe.close()
        res["teacher_cls_scale"] = scale
        teacher = Model(synth.pack_blob(synth.FULL, synth.make_weights(synth.FULL, TEACHER_SEED, cls_scale=scale)))
    else:
        if args.teacher_blob:
            with open(args.teacher_blob, "rb") as f:
                tblob = f.read()
        else:
            tblob = train_teacher(args, chunks, dev, res)
            if args.teacher_out:
                with open(args.teacher_out, "wb") as f:
                    f.write(tblob)
        teacher = Model(tblob)
        chunks = [c[:2] for c in chunks]

    # teacher targets for every training batch (kept on the device)
    t0 = time.time()
    batches = []
    for x, cu in chunks:
        X = torch.from_numpy(x).to(dev)
        CU = torch.from_numpy(cu).to(dev)
        mn = int(np.diff(cu).max())
        tl, tr, _, _ = teacher.forward(X, CU, mn, precision=args.teacher_precision, want_cls=False,
                                       want_sums=False)
        batches.append((X, CU, mn, tl, tr))
    torch.cuda.synchronize()
    res["teacher_targets_s"] = time.time() - t0

    # training
    scfg = synth.SMALL if args.student == "d64" else STUDENT_CFG5
    sprec = "bf16"   # d64: the fused kernels; cfg5: the generic-width tensor-core path
    res["student"] = {"config": args.student, "d": scfg.d, "heads": scfg.heads, "ffn": scfg.ffn,
                      "l_pid": scfg.l_pid, "l_reg": scfg.l_reg, "precision": sprec,
                      "train_precision": args.train_precision}
    res["teacher_precision"] = args.teacher_precision
    init_blob = synth.pack_blob(scfg, synth.make_weights(scfg, STUDENT_SEED))
    if args.student_blob:
        batches = []
        args.epochs = 0
    trainer = Trainer(init_blob, precision=args.train_precision)
    total_steps = args.epochs * len(batches)
    rng = np.random.default_rng(0)
    losses = []
    step = 0
    t0 = time.time()
    for ep in range(args.epochs):
        for bi in rng.permutation(len(batches)):
            X, CU, mn, tl, tr = batches[bi]
            lr = 2e-4 + 0.5 * (2e-3 - 2e-4) * (1 + math.cos(math.pi * step / total_steps))
            want = step % 25 == 0 or step == total_steps - 1
            loss = trainer.step(X, CU, mn, tl, tr, lr, want_loss=want)
            if want:
                losses.append((step, loss))
            step += 1
    torch.cuda.synchronize()
    res["train_s"] = time.time() - t0
    res["train_steps"] = total_steps
    res["train_ms_per_step"] = 1e3 * res["train_s"] / max(1, total_steps)
    res["loss_curve"] = losses
    blob = trainer.export()
    trainer.close()
    if args.student_blob:
        with open(args.student_blob, "rb") as f:
            blob = f.read()
    if args.out:
        with open(args.out, "wb") as f:
            f.write(blob)

    # evaluation on the 512-event workload
    cfg, _, iseed, sizes = synth.workload("batch512")
    x, cu = synth.gen_events(iseed, sizes)
    X, CU, mn = torch.from_numpy(x).to(dev), torch.from_numpy(cu).to(dev), int(sizes.max())
    ev = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        a, b = ev()
        a.record()
        for _ in range(reps):
            out = fn()
        b.record()
        torch.cuda.synchronize()
        return out, a.elapsed_time(b) / reps

    tout, t32_ms = timed(lambda: teacher.forward(X, CU, mn, precision="fp32"), reps=1)
    t_cls = tout[2].cpu().numpy()
    t_reg = tout[1].cpu().numpy()
    # the teacher as the gated path runs it (its own agreement with the FP32 teacher)
    tlp, t_ms = timed(lambda: teacher.forward(X, CU, mn, precision=args.teacher_precision), reps=1)
    res["teacher_lowp_agreement"] = float((tlp[2].cpu().numpy() == t_cls).mean())
    res["teacher_fp32_ms"] = t32_ms
    if args.teacher == "trained":
        tr_cls, _ = synth.gen_pf_truth(x, cu)
        res["teacher_truth_accuracy"] = float((t_cls == tr_cls).mean())
        conf_t = softmax_max(tout[0].cpu().numpy().astype(np.float64))
        res["teacher_confidence_fraction"] = {f">={c}": float((conf_t >= c).mean()) for c in (0.9, 0.99)}

    def evaluate(name, blob_):
        student = Model(blob_)
        sout, s_ms = timed(lambda: student.forward(X, CU, mn, precision=sprec))
        s_cls = sout[2].cpu().numpy()
        s_reg = sout[1].cpu().numpy()
        r = {"student_agreement": float((s_cls == t_cls).mean()),
             "student_reg_rel_err_vs_teacher": [
                 float(v) for v in np.sqrt(((s_reg - t_reg) ** 2).sum(0) / (t_reg ** 2).sum(0))],
             "student_ms": s_ms, "gated": {}}
        # per-event confidence statistics: can an event-level gate separate the events
        # the student gets wrong?
        conf_el = softmax_max(sout[0].cpu().numpy().astype(np.float64))
        ev_mean = np.array([conf_el[cu[e]:cu[e + 1]].mean() for e in range(len(sizes))])
        ev_min = np.array([conf_el[cu[e]:cu[e + 1]].min() for e in range(len(sizes))])
        ev_agree = np.array([(s_cls[cu[e]:cu[e + 1]] == t_cls[cu[e]:cu[e + 1]]).mean() for e in range(len(sizes))])
        pct = [0, 10, 50, 90, 100]
        r["event_confidence"] = {
            "mean_conf_percentiles": {str(q): float(np.percentile(ev_mean, q)) for q in pct},
            "min_conf_percentiles": {str(q): float(np.percentile(ev_min, q)) for q in pct},
            "event_agreement_percentiles": {str(q): float(np.percentile(ev_agree, q)) for q in pct},
            "corr_mean_conf_vs_agreement": float(np.corrcoef(ev_mean, ev_agree)[0, 1]),
            "element_agreement_by_conf": {
                f">={c}": float((s_cls[conf_el >= c] == t_cls[conf_el >= c]).mean()) if (conf_el >= c).any() else None
                for c in (0.5, 0.9, 0.99)},
            "element_fraction_by_conf": {f">={c}": float((conf_el >= c).mean()) for c in (0.5, 0.9, 0.99)}}
        # event confidence: mean (mode 0) or minimum (mode 1) of the per-element max softmax
        for mode, mname in ((0, "mean"), (1, "min")):
            student.set_option(_lib.OPT_GATE_CONFIDENCE, mode)
            # fixed thresholds and the 10th-90th percentiles of this mode's event confidence
            evc = ev_mean if mode == 0 else ev_min
            pct_thr = {round(float(np.percentile(evc, q)), 5) for q in (10, 25, 50, 75, 90)}
            for thr in sorted({args.threshold, 0.5, 0.7, 0.95, 0.97, 0.98, 0.99, 0.995, 0.999} | pct_thr):
                gout, g_ms = timed(lambda: forward_gated(student, teacher, thr, X, CU, mn,
                                                         student_precision=sprec,
                                                         teacher_precision=args.teacher_precision), reps=1)
                g_cls = gout[2].cpu().numpy()
                g_reg = gout[1].cpu().numpy()
                rel = np.sqrt(((g_reg - t_reg) ** 2).sum(0) / (t_reg ** 2).sum(0))
                r["gated"][f"{mname}@{thr}"] = {
                    "agreement": float((g_cls == t_cls).mean()), "fallback_events": int(gout[5]),
                    "fallback_rate": gout[5] / len(sizes), "ms": g_ms, "speedup_vs_teacher": t_ms / g_ms,
                    "reg_rel_err_vs_teacher": [float(v) for v in rel]}
        res[name] = r
        student.close()

    res["teacher_ms"] = t_ms
    evaluate("trained", blob)
    evaluate("untrained", init_blob)
    line = json.dumps(res)
    print(line, flush=True)
    if args.json:
        with open(args.json, "w") as f:
            f.write(line + "\n")


def train_teacher(args, chunks, dev, res):
    """The full model trained on the synthetic truth with the library's kernels and LAMB
    (lr 2e-3 -> 2e-4 cosine over --teacher-steps, batches in a random order, epoch after
    epoch); returns its weight blob."""
    import torch
    from paper_2601_17554_b300 import Trainer
    init = synth.pack_blob(synth.FULL, synth.make_weights(synth.FULL, TEACHER_SEED))
    tr = Trainer(init, precision=args.train_precision)
    data = []
    for x, cu, cls, reg in chunks:
        lg = np.zeros((len(cls), synth.N_CLS), np.float32)
        lg[np.arange(len(cls)), cls] = TRUTH_LOGIT
        data.append((torch.from_numpy(x).to(dev), torch.from_numpy(cu).to(dev), int(np.diff(cu).max()),
                     torch.from_numpy(lg).to(dev), torch.from_numpy(reg).to(dev)))
    rng = np.random.default_rng(1)
    order = []
    while len(order) < args.teacher_steps:
        order.extend(rng.permutation(len(data)).tolist())
    losses = []
    torch.cuda.synchronize()
    t0 = time.time()
    for step in range(args.teacher_steps):
        X, CU, mn, tl, trg = data[order[step]]
        lr = 2e-4 + 0.5 * (2e-3 - 2e-4) * (1 + math.cos(math.pi * step / args.teacher_steps))
        want = step % 25 == 0 or step == args.teacher_steps - 1
        loss = tr.step(X, CU, mn, tl, trg, lr, want_loss=want)
        if want:
            losses.append((step, loss))
    torch.cuda.synchronize()
    res["teacher_training"] = {"steps": args.teacher_steps, "train_s": time.time() - t0,
                               "ms_per_step": 1e3 * (time.time() - t0) / max(1, args.teacher_steps),
                               "truth_logit": TRUTH_LOGIT, "loss_curve": losses,
                               "precision": args.train_precision}
    blob = tr.export()
    tr.close()
    del data
    return blob


if __name__ == "__main__":
    main()
