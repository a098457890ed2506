"""The deterministic synthetic truth used to train the full model as a teacher.

Pinned on a hand-built event whose classes and targets follow from the rule by
hand, plus its invariants: each event's classes depend on that event only, and the
element order within an event does not matter.
"""
import numpy as np

import synth


def _elem(typ, logpt, loge, eta, phi, f13=0.0):
    x = np.zeros(42, np.float32)
    x[typ] = 1.0
    x[8], x[9], x[10] = logpt, loge, eta
    x[11], x[12] = np.sin(phi), np.cos(phi)
    x[13] = f13
    return x


def test_hand_event():
    # ECAL log E: 0.0, 1.0, -1.2 (mean -0.0667): the third is below mean - 0.5
    # HCAL log E: 2.0, 0.0 (mean 1.0): the second (0.0 <= 0.5) is below mean - 0.5
    ev = [_elem(0, 0.3, 0.0, 0.5, 0.1, f13=2.0),   # track, muon match -> muon
          _elem(0, -0.2, 0.0, -1.0, 2.0, f13=1.0),  # track -> charged hadron
          _elem(5, 1.0, 0.0, 0.2, -1.0),            # GSF -> electron
          _elem(6, 0.0, 0.0, 0.0, 0.0),             # brem -> none
          _elem(1, 0.0, 0.0, 1.0, 0.5),             # ECAL -> photon
          _elem(1, 0.0, 1.0, 0.0, 0.5),             # ECAL -> photon
          _elem(1, 0.0, -1.2, 0.0, 0.5),            # ECAL -> none
          _elem(2, 0.0, 2.0, 2.0, 0.5),             # HCAL -> neutral hadron
          _elem(2, 0.0, 0.0, 0.0, 0.5),             # HCAL -> none
          _elem(3, 0.0, 0.0, 4.0, 0.5),             # HF-EM -> photon
          _elem(4, 0.0, 0.0, -4.0, 0.5),            # HF-HAD -> neutral hadron
          _elem(7, 0.0, 0.0, 0.0, 0.5)]             # supercluster -> photon
    x = np.stack(ev)
    cu = np.array([0, len(ev)], np.int32)
    cls, reg = synth.gen_pf_truth(x, cu)
    assert cls.tolist() == [5, 1, 4, 0, 3, 3, 0, 2, 0, 3, 2, 3]
    # track: pT = exp(log pT), E = pT cosh(eta); ECAL at eta 1: E = exp(0), pT = 1 / cosh(1)
    np.testing.assert_allclose(reg[0], [np.exp(0.3), 0.5, np.sin(0.1), np.cos(0.1), np.exp(0.3) * np.cosh(0.5)],
                               rtol=1e-6)
    np.testing.assert_allclose(reg[4], [1.0 / np.cosh(1.0), 1.0, np.sin(0.5), np.cos(0.5), 1.0], rtol=1e-6)
    np.testing.assert_allclose(reg[7, [0, 4]], [np.exp(2.0) / np.cosh(2.0), np.exp(2.0)], rtol=1e-6)


def test_events_independent_and_order_free():
    x, cu = synth.gen_events(7, [300, 0, 41, 800])
    cls, reg = synth.gen_pf_truth(x, cu)
    for e in range(4):
        a, b = cu[e], cu[e + 1]
        c1, r1 = synth.gen_pf_truth(x[a:b], np.array([0, b - a], np.int32))
        assert (c1 == cls[a:b]).all()
        np.testing.assert_array_equal(r1, reg[a:b])
        perm = np.random.default_rng(e).permutation(b - a)
        c2, _ = synth.gen_pf_truth(x[a:b][perm], np.array([0, b - a], np.int32))
        assert (c2 == cls[a:b][perm]).all()
    # every class occurs in a realistic event
    assert set(np.unique(cls[cu[3]:cu[4]])) == {0, 1, 2, 3, 4, 5}
