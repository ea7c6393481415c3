"""Pins of the oracle's self-collision test (robot spheres of non-adjacent frames against
each other): clearances against brute-force pairwise distances of independently computed
sphere centres, the frame-pair mask, and the first self-colliding waypoint of a motion."""
import numpy as np

from paper_2505_06791_gb300 import synth as S
from tests import indep


def brute_self_clearance(rb, q, pairs):
    c = indep.sphere_centres(rb.joints, rb.ee, rb.spheres, q)
    f = rb.spheres[:, 0].astype(int)
    r = rb.spheres[:, 4]
    d = np.linalg.norm(c[:, None, :] - c[None, :, :], axis=2) - (r[:, None] + r[None, :])
    use = pairs[f[:, None], f[None, :]].astype(bool) & (f[:, None] != f[None, :])
    use &= np.triu(np.ones_like(use), 1).astype(bool)
    return d[use].min() if use.any() else np.inf


def test_self_clearance_matches_brute_force(oracle_mod):
    rb = S.make_arm7(1)
    pairs = S.self_pairs_gap(rb, 2)
    orc = oracle_mod.Oracle(rb, S.Scene(), S.no_constraint(), self_pairs=pairs)
    plain = oracle_mod.Oracle(rb, S.Scene(), S.no_constraint())
    for q in S.uniform_configs(rb, 40, 120):
        got = orc.config_clearance(q)
        assert abs(got - brute_self_clearance(rb, q, pairs)) < 1e-12
        assert plain.config_clearance(q) == np.inf  # no obstacles, no self test


def test_mask_selects_frame_pairs(oracle_mod):
    """A wider gap tests fewer pairs (clearance can only grow); an empty mask tests none."""
    rb = S.make_arm7(1)
    o2 = oracle_mod.Oracle(rb, S.Scene(), S.no_constraint(), self_pairs=S.self_pairs_gap(rb, 2))
    o4 = oracle_mod.Oracle(rb, S.Scene(), S.no_constraint(), self_pairs=S.self_pairs_gap(rb, 4))
    none = oracle_mod.Oracle(rb, S.Scene(), S.no_constraint(),
                             self_pairs=np.zeros((rb.dof + 1, rb.dof + 1), np.uint8))
    for q in S.uniform_configs(rb, 30, 121):
        assert o4.config_clearance(q) >= o2.config_clearance(q)
        assert none.config_clearance(q) == np.inf


def test_first_self_colliding_waypoint(oracle_mod):
    """Validation reports the first waypoint whose clearance (self pairs included) is
    negative, and the motion's margin is the smallest clearance on the way to it."""
    rb = S.make_arm7(1)
    pairs = S.self_pairs_gap(rb, 2)
    orc = oracle_mod.Oracle(rb, S.Scene(), S.no_constraint(), self_pairs=pairs)
    q0 = S.uniform_configs(rb, 64, 122)
    q1 = S.uniform_configs(rb, 64, 123)
    r = orc.validate(q0, q1, 32)
    hits = 0
    for m in range(64):
        xi = oracle_mod.interpolate(S.f32(q0[m]), S.f32(q1[m]), 32)
        cl = np.array([brute_self_clearance(rb, x, pairs) for x in xi])
        neg = np.nonzero(cl < 0)[0]
        if len(neg):
            hits += 1
            assert r["status"][m] == 2 and r["first_fail"][m] == neg[0]
        else:
            assert r["status"][m] == 0
    assert hits >= 5
