"""Pins of the anti-kt oracle (oracle/jets.py) against what the algorithm's
definition fixes (Cacciari, Salam, Soyez, JHEP 04 (2008) 063): closed forms on
one and two particles, the wrap of phi, the perfect cone around an isolated hard
particle, 4-momentum conservation and independence of the input order."""
import numpy as np

from oracle import jets as J


def p4(pt, eta, phi):
    pt, eta, phi = (np.atleast_1d(np.asarray(v, np.float64)) for v in (pt, eta, phi))
    return np.stack([pt * np.cos(phi), pt * np.sin(phi), pt * np.sinh(eta), pt * np.cosh(eta)], 1)


def test_single_particle_is_one_jet():
    v = p4(3.0, 0.7, 1.1)
    jets, jof = J.antikt(v, 0.4)
    np.testing.assert_allclose(jets, v, rtol=1e-15)
    assert jof.tolist() == [0]


def test_two_particles_within_R_merge_into_their_sum():
    v = p4([5.0, 2.0], [0.1, 0.3], [0.0, 0.2])     # dR = 0.283 < 0.4
    jets, jof = J.antikt(v, 0.4)
    assert len(jets) == 1 and jof.tolist() == [0, 0]
    np.testing.assert_allclose(jets[0], v.sum(0), rtol=1e-14)


def test_two_particles_beyond_R_stay_apart_harder_first():
    v = p4([2.0, 5.0], [0.1, 0.5], [0.0, 0.2])     # dR = 0.447 > 0.4
    jets, jof = J.antikt(v, 0.4)
    # d_iB = pT^-2: the harder particle leaves the list first
    np.testing.assert_allclose(jets, v[[1, 0]], rtol=1e-15)
    assert jof.tolist() == [1, 0]


def test_phi_wraps_at_pi():
    v = p4([4.0, 3.0], [0.0, 0.0], [np.pi - 0.05, -np.pi + 0.05])   # dR = 0.1 across the seam
    jets, _ = J.antikt(v, 0.4)
    assert len(jets) == 1


def test_rapidity_not_azimuth_alone():
    v = p4([4.0, 3.0], [0.0, 0.5], [0.0, 0.0])     # same phi, dy = 0.5 > 0.4
    assert len(J.antikt(v, 0.4)[0]) == 2
    assert len(J.antikt(v, 0.8)[0]) == 1


def test_isolated_hard_particle_makes_a_perfect_cone():
    """Anti-kt's defining property: soft particles are absorbed by a hard one
    within R of it before they cluster among themselves, and none beyond R."""
    rng = np.random.default_rng(5)
    n = 60
    eta = rng.uniform(-1.2, 1.2, n)
    phi = rng.uniform(-1.2, 1.2, n)
    dr = np.hypot(eta, phi)
    keep = (dr < 0.32) | (dr > 0.48)                 # away from the cone edge
    eta, phi, dr = eta[keep], phi[keep], dr[keep]
    v = np.concatenate([p4(200.0, 0.0, 0.0), p4(np.full(len(eta), 0.5), eta, phi)])
    jets, jof = J.antikt(v, 0.4)
    inside = np.concatenate([[True], dr < 0.4])
    assert (jof[inside] == jof[0]).all()
    assert (jof[~inside] != jof[0]).all()
    assert jof[0] == 0                                # the hard jet leaves first


def test_four_momentum_conserved_and_order_independent():
    rng = np.random.default_rng(7)
    n = 80
    v = p4(np.exp(rng.normal(0, 1, n)), rng.uniform(-2.5, 2.5, n), rng.uniform(-np.pi, np.pi, n))
    jets, jof = J.antikt(v, 0.4)
    np.testing.assert_allclose(jets.sum(0), v.sum(0), rtol=1e-12)
    assert (jof >= 0).all() and set(jof.tolist()) == set(range(len(jets)))
    # each jet is the sum of its constituents
    for t in range(len(jets)):
        np.testing.assert_allclose(jets[t], v[jof == t].sum(0), rtol=1e-12)
    perm = rng.permutation(n)
    jets2, jof2 = J.antikt(v[perm], 0.4)
    part = lambda jo: sorted(tuple(sorted(np.nonzero(jo == t)[0].tolist())) for t in range(jo.max() + 1))
    inv = np.argsort(perm)   # jof2[inv[i]] is the jet of input i
    assert part(jof) == part(jof2[inv])


def test_particles_from_outputs():
    cls = np.array([0, 1, 3, 2, 5])
    reg = np.array([[1.0, 0.0, 0.0, 1.0, 1.0],
                    [2.0, 0.5, 0.0, 2.0, 1.0],      # (s, c) = (0, 2): normalised to phi = 0
                    [3.0, -1.0, 1.0, 0.0, 1.0],
                    [0.0, 0.0, 0.0, 1.0, 1.0],      # pT = 0: not a particle
                    [1.5, 0.2, 0.0, 0.0, 1.0]])     # (s, c) = (0, 0): not a particle
    rows, v = J.particles(cls, reg)
    assert rows.tolist() == [1, 2]
    np.testing.assert_allclose(v[0], [2.0, 0.0, 2.0 * np.sinh(0.5), 2.0 * np.cosh(0.5)], rtol=1e-15)
    np.testing.assert_allclose(v[1], [0.0, 3.0, 3.0 * np.sinh(-1.0), 3.0 * np.cosh(-1.0)], atol=1e-15)
    # massless: E = |p|
    np.testing.assert_allclose(v[:, 3], np.linalg.norm(v[:, :3], axis=1), rtol=1e-14)
