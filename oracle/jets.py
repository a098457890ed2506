"""Anti-kt jets of an event's reconstructed particles -- test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs may import this
module; the library never does.

The paper clusters jets from the PF or MLPF candidates of each event with the
anti-kt algorithm, distance parameter R = 0.4 (AK4) or 0.8 (AK8) (Sec. 3.3, Sec.
6.2); its PUPPI pileup weights need vertex information that the synthetic events
do not have, so none are applied.  The algorithm (Cacciari, Salam, Soyez, "The
anti-k_t jet clustering algorithm", JHEP 04 (2008) 063), written out plainly:

  particles   every element with class != 0, pT > 0 and (sin phi, cos phi) != 0,
              taken as massless: px = pT c / r, py = pT s / r with r = sqrt(s^2 + c^2),
              pz = pT sinh(eta), E = pT cosh(eta).
  distances   d_ij = min(pT_i^-2, pT_j^-2) dR_ij^2 / R^2 between entries i != j and
              d_iB = pT_i^-2 to the beam; dR^2 = (y_i - y_j)^2 + dphi^2 with the
              rapidity y = ln((E + pz) / (E - pz)) / 2, phi = atan2(py, px) and dphi
              wrapped into [0, pi].
  step        take the smallest of all d_ij and d_iB: a d_ij replaces i and j by
              their 4-vector sum (E scheme); a d_iB makes i a jet and removes it.
              Repeat until no entry is left.

Jets are returned in the order they leave the list.  Every distance is computed in
float64 from the entries' current 4-vectors; there is no nearest-neighbour bookkeeping
(the GPU kernel's is a reordering of the same minimum).
"""
from __future__ import annotations

import numpy as np

F64 = np.float64


def particles(cls, reg):
    """Rows and massless 4-vectors (px, py, pz, E) of the event's particles."""
    cls = np.asarray(cls)
    reg = np.asarray(reg, F64)
    pt, eta, s, c = reg[:, 0], reg[:, 1], reg[:, 2], reg[:, 3]
    r = np.sqrt(s * s + c * c)
    rows = np.nonzero((cls != 0) & (pt > 0) & (r > 0))[0]
    pt, eta, s, c, r = pt[rows], eta[rows], s[rows], c[rows], r[rows]
    p4 = np.stack([pt * c / r, pt * s / r, pt * np.sinh(eta), pt * np.cosh(eta)], axis=1)
    return rows, p4


def kinematics(p4):
    """(pT^-2, y, phi) of 4-vectors [n, 4]."""
    px, py, pz, e = p4[:, 0], p4[:, 1], p4[:, 2], p4[:, 3]
    pt2 = px * px + py * py
    y = 0.5 * np.log((e + pz) / (e - pz))
    phi = np.arctan2(py, px)
    return 1.0 / pt2, y, phi


def antikt(p4, R):
    """Anti-kt with the E scheme: (jets [m, 4], jet index of every input entry)."""
    p4 = np.asarray(p4, F64)
    n = len(p4)
    vec = p4.copy()
    active = list(range(n))
    members = {i: [i] for i in range(n)}
    jets, jet_of = [], np.full(n, -1, np.int64)
    while active:
        a = np.asarray(active)
        pinv, y, phi = kinematics(vec[a])
        dy = y[:, None] - y[None, :]
        dphi = np.abs(phi[:, None] - phi[None, :])
        dphi = np.where(dphi > np.pi, 2.0 * np.pi - dphi, dphi)
        dij = np.minimum(pinv[:, None], pinv[None, :]) * (dy * dy + dphi * dphi) / (R * R)
        np.fill_diagonal(dij, np.inf)
        ij = np.unravel_index(np.argmin(dij), dij.shape)
        ib = int(np.argmin(pinv))
        if pinv[ib] <= dij[ij]:
            i = int(a[ib])
            for m in members.pop(i):
                jet_of[m] = len(jets)
            jets.append(vec[i].copy())
            active.remove(i)
        else:
            i, j = int(a[ij[0]]), int(a[ij[1]])
            k, l = min(i, j), max(i, j)
            vec[k] = vec[k] + vec[l]
            members[k] += members.pop(l)
            active.remove(l)
    return np.asarray(jets, F64).reshape(-1, 4), jet_of


def event_jets(cls, reg, R=0.4):
    """Jets of one event from its decoded outputs: (jets [m, 4], jet index per
    element of the event, -1 for elements that are not particles)."""
    rows, p4 = particles(cls, reg)
    jets, jof = antikt(p4, R)
    out = np.full(len(cls), -1, np.int64)
    out[rows] = jof
    return jets, out
