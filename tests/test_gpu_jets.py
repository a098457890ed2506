"""Anti-kt jets on the GPU (mlpf_cluster_jets) against the FP64 oracle.

Events of at most 12,288 elements run on the shared-memory kernel, larger ones on
the global-memory kernel (same algorithm and tie rules).  Inputs: seeded synthetic
reconstructed particles (synth.gen_targets: classes by
element type, pT, eta, phi and E near the element's own), the same arrays for
both sides.  What is unique is compared exactly: the partition of the particles
into jets (constituent sets) and the jet count; the jets' 4-vectors (FP32 sums on
the GPU) within 1e-4 relative.  The GPU decides merges in FP32 and the oracle in
FP64, so a near-tie (two distances equal to FP32 precision) may be taken in the
other order; where that changes a jet, the jet is not matched.  Unmatched jets are
checked too: the GPU's and the oracle's unmatched jets hold the same particles and
the same summed 4-vector (the difference is a local reordering, no particle lost or
double counted), and at least 99.5 % of the particles sit in matched jets.
"""
import numpy as np
import pytest

import synth
from oracle import jets as J

pytestmark = pytest.mark.gpu


def run_jets(model, reg, cls, cu, R):
    import torch
    r = torch.from_numpy(np.ascontiguousarray(reg, np.float32)).cuda()
    c = torch.from_numpy(np.ascontiguousarray(cls, np.int32)).cuda()
    u = torch.from_numpy(np.ascontiguousarray(cu, np.int32)).cuda()
    jets, nj, jof = model.cluster_jets(r, c, u, R)
    torch.cuda.synchronize()
    return jets.cpu().numpy(), nj.cpu().numpy(), jof.cpu().numpy()


@pytest.fixture(scope="module")
def model():
    from tests.util import make_model
    m, _ = make_model(synth.SMALL, 0)
    yield m
    m.close()


def partition(jof):
    return {frozenset(np.nonzero(jof == t)[0].tolist()) for t in range(int(jof.max()) + 1)} if len(jof) and jof.max() >= 0 else set()


def compare_event(gj, gnj, gjof, cls, reg, R, ref=None):
    """(particles, particles in matched jets) of one event, checking matched jets' 4-vectors;
    ref: the oracle's (jets, jet index per element), computed here if None."""
    oj, ojof = J.event_jets(cls, reg, R) if ref is None else ref
    assert gjof.shape == ojof.shape
    assert ((gjof < 0) == (ojof < 0)).all()          # the same particles
    n_part = int((ojof >= 0).sum())
    assert gnj >= 1 or n_part == 0
    gp = {frozenset(np.nonzero(gjof == t)[0].tolist()): t for t in range(gnj)}
    matched, hit = 0, set()
    un_o, un_o_p4 = set(), np.zeros(4)
    for t in range(len(oj)):
        s = frozenset(np.nonzero(ojof == t)[0].tolist())
        if s in gp:
            matched += len(s)
            hit.add(gp[s])
            np.testing.assert_allclose(gj[gp[s]], oj[t], rtol=1e-4, atol=1e-4 * np.abs(oj[t]).max())
        else:
            un_o |= s
            un_o_p4 += oj[t]
    # the unmatched jets of both sides: the same particles, the same total 4-vector
    un_g = set(np.nonzero(np.isin(gjof, [t for t in range(gnj) if t not in hit]))[0].tolist())
    assert un_g == un_o
    un_g_p4 = gj[[t for t in range(gnj) if t not in hit]].astype(np.float64).sum(0) if gnj else np.zeros(4)
    scale = max(np.abs(oj).sum(), 1.0) if len(oj) else 1.0
    np.testing.assert_allclose(un_g_p4, un_o_p4, rtol=0, atol=1e-5 * scale)
    return n_part, matched


@pytest.mark.parametrize("R", [0.4, 0.8])
def test_jets_match_oracle(model, R):
    sizes = [1, 2, 17, 150, 400, 0, 700, 64]
    x, cu = synth.gen_events(41, sizes)
    cls, reg = synth.gen_targets(42, x, cu)
    gj, gnj, gjof = run_jets(model, reg, cls, cu, R)
    tot = mat = 0
    for e in range(len(sizes)):
        sl = slice(cu[e], cu[e + 1])
        n, m = compare_event(gj[cu[e]:cu[e + 1]], int(gnj[e]), gjof[sl], cls[sl], reg[sl], R)
        tot, mat = tot + n, mat + m
    assert sizes[5] == 0 and gnj[5] == 0
    assert mat >= 0.995 * tot, (mat, tot)


def test_many_small_events(model):
    """5,000 events of 0-7 elements: more events than the launch-order sort takes (4,096),
    so the CTAs run in event order; every event matches the oracle."""
    rng = np.random.default_rng(49)
    sizes = rng.integers(0, 8, 5000)
    x, cu = synth.gen_events(50, sizes)
    cls, reg = synth.gen_targets(51, x, cu)
    gj, gnj, gjof = run_jets(model, reg, cls, cu, 0.4)
    tot = mat = 0
    for e in range(len(sizes)):
        sl = slice(cu[e], cu[e + 1])
        n, m = compare_event(gj[cu[e]:cu[e + 1]], int(gnj[e]), gjof[sl], cls[sl], reg[sl], 0.4)
        tot, mat = tot + n, mat + m
    assert tot > 10000 and mat >= 0.995 * tot, (mat, tot)


def test_non_finite_values_stay_contained(model):
    """An event whose regressions hold NaN and infinite values (pT, eta, sin, cos) between
    two finite events: the call succeeds, its jet indices are -1 or a jet of the event, and
    the finite events still match the oracle."""
    sizes = [300, 200, 250]
    x, cu = synth.gen_events(52, sizes)
    cls, reg = synth.gen_targets(53, x, cu)
    reg, cls = reg.copy(), cls.copy()
    rows = np.arange(cu[1], cu[2])
    reg[rows[0:10], 1] = np.nan          # eta
    reg[rows[10:20], 1] = np.inf
    reg[rows[20:30], 0] = np.inf         # pT
    reg[rows[30:40], 2] = np.nan         # sin phi
    reg[rows[40:50], 3] = -np.inf        # cos phi
    cls[rows[:50]] = 1
    gj, gnj, gjof = run_jets(model, reg, cls, cu, 0.4)
    sl = slice(cu[1], cu[2])
    assert 0 <= gnj[1] <= sizes[1]
    assert ((gjof[sl] >= -1) & (gjof[sl] < gnj[1])).all()
    for e in (0, 2):
        sl = slice(cu[e], cu[e + 1])
        n, m = compare_event(gj[cu[e]:cu[e + 1]], int(gnj[e]), gjof[sl], cls[sl], reg[sl], 0.4)
        assert m >= 0.995 * n


def test_closed_forms(model):
    # event 0: two particles within R -> one jet, their sum; event 1: two beyond R ->
    # two jets, the harder first; event 2: a class-0 element and a pT = 0 element only
    reg = np.array([[5.0, 0.1, 0.0, 1.0, 1.0], [2.0, 0.3, np.sin(0.2), np.cos(0.2), 1.0],
                    [2.0, 0.1, 0.0, 1.0, 1.0], [5.0, 0.5, np.sin(0.2), np.cos(0.2), 1.0],
                    [3.0, 0.0, 0.0, 1.0, 1.0], [0.0, 0.0, 0.0, 1.0, 1.0]], np.float32)
    cls = np.array([1, 2, 1, 3, 0, 4], np.int32)
    cu = np.array([0, 2, 4, 6], np.int32)
    gj, gnj, gjof = run_jets(model, reg, cls, cu, 0.4)
    assert gnj.tolist() == [1, 2, 0]
    assert gjof.tolist() == [0, 0, 1, 0, -1, -1]
    _, v = J.particles(cls[:4], reg[:4])
    np.testing.assert_allclose(gj[0], v[0] + v[1], rtol=2e-6)
    np.testing.assert_allclose(gj[2], v[3], rtol=2e-6)
    np.testing.assert_allclose(gj[3], v[2], rtol=2e-6)


def test_bad_arguments_rejected(model):
    from paper_2601_17554_b300 import _lib
    L = model.L
    assert L.mlpf_cluster_jets(model.h, None, None, None, 1, 0, 0.4, None, None, None, None) == _lib.MLPF_E_INVALID
    assert L.mlpf_cluster_jets(model.h, None, None, None, 0, 0, 0.0, None, None, None, None) == _lib.MLPF_E_INVALID
    assert L.mlpf_cluster_jets(model.h, None, None, None, 0, 0, 0.4, None, None, None, None) == _lib.MLPF_OK


def test_full_batch_conserves_momentum(model):
    """The 512-event workload through the BF16 forward, then jets: every event's
    jets add up to its particles (FP32 sums), and the timing is printed."""
    import torch
    cfg, wseed, iseed, sizes = synth.workload("batch512")
    x, cu = synth.gen_events(iseed, sizes)
    from tests.util import make_model
    fm, _ = make_model(cfg, wseed)
    xt, ct = torch.from_numpy(x).cuda(), torch.from_numpy(cu).cuda()
    lo, rg, cl, su = fm.forward(xt, ct, int(sizes.max()), precision="bf16")
    fm.sync()
    model.cluster_jets(rg, cl, ct, 0.4)   # warm-up (scratch allocation)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    jets, nj, _ = model.cluster_jets(rg, cl, ct, 0.4)
    t1.record()
    torch.cuda.synchronize()
    print(f"anti-kt R=0.4 on 512 events ({len(x)} elements): {t0.elapsed_time(t1):.2f} ms, "
          f"{int(nj.sum())} jets")
    # the largest event alone: the floor of the batch time (one CTA per event)
    big = int(np.argmax(sizes))
    s0, s1 = int(cu[big]), int(cu[big + 1])
    ub = torch.tensor([0, s1 - s0], dtype=torch.int32, device="cuda")
    rb, cb = rg[s0:s1].contiguous(), cl[s0:s1].contiguous()
    model.cluster_jets(rb, cb, ub, 0.4)
    torch.cuda.synchronize()
    t0.record()
    _, njb, _ = model.cluster_jets(rb, cb, ub, 0.4)
    t1.record()
    torch.cuda.synchronize()
    print(f"anti-kt R=0.4 on its largest event alone ({s1 - s0} elements, "
          f"{int((cb != 0).sum())} with a class): {t0.elapsed_time(t1):.2f} ms")
    assert int(njb[0]) == int(nj[big])
    jets, nj = jets.cpu().numpy().astype(np.float64), nj.cpu().numpy()
    reg, cls = rg.cpu().numpy(), cl.cpu().numpy()
    for e in range(0, len(sizes), 37):
        sl = slice(cu[e], cu[e + 1])
        _, v = J.particles(cls[sl], reg[sl])
        tot = jets[cu[e]:cu[e] + nj[e]].sum(0)
        np.testing.assert_allclose(tot, v.sum(0), rtol=1e-3, atol=1e-3 * np.abs(v).sum())
    fm.close()


def test_large_event_matches_oracle_golden(model):
    """One event of 7,500 elements (5,201 particles) against the FP64 oracle's jets,
    stored in tests/golden/antikt_large_r04.json by tests/golden/make_antikt_large.py
    (the oracle's plain O(N^3) clustering takes about 20 minutes on it)."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "antikt_large_r04.json")
    g = json.load(open(path))
    x, cu = synth.gen_events(g["seed_events"], [g["size"]])
    cls, reg = synth.gen_targets(g["seed_targets"], x, cu)
    gj, gnj, gjof = run_jets(model, reg, cls, cu, g["R"])
    oj, ojof = np.asarray(g["jets"], np.float64).reshape(-1, 4), np.asarray(g["jet_of"], np.int64)
    n, m = compare_event(gj, int(gnj[0]), gjof, cls, reg, g["R"], ref=(oj, ojof))
    assert n == g["n_particles"]
    assert m >= 0.995 * n, (m, n)


def test_event_above_shared_memory_capacity(model):
    """An event of 13,000 elements (beyond the 12,288 that the shared-memory kernel
    holds) runs on the global-memory kernel in the same call as small events: every
    particle is in exactly one jet and each event's jets add up to its particles; the
    small events match the oracle."""
    sizes = [13000, 150, 700]
    x, cu = synth.gen_events(47, sizes)
    cls, reg = synth.gen_targets(48, x, cu)
    gj, gnj, gjof = run_jets(model, reg, cls, cu, 0.4)
    sl = slice(cu[0], cu[1])
    rows, v = J.particles(cls[sl], reg[sl])
    assert ((gjof[sl] >= 0) == np.isin(np.arange(sizes[0]), rows)).all()
    assert set(np.unique(gjof[sl][gjof[sl] >= 0]).tolist()) == set(range(int(gnj[0])))
    tot = gj[cu[0]:cu[0] + gnj[0]].astype(np.float64).sum(0)
    np.testing.assert_allclose(tot, v.sum(0), rtol=1e-3, atol=1e-3 * np.abs(v).sum())
    for e in (1, 2):
        sl = slice(cu[e], cu[e + 1])
        n, m = compare_event(gj[cu[e]:cu[e + 1]], int(gnj[e]), gjof[sl], cls[sl], reg[sl], 0.4)
        assert m >= 0.995 * n
