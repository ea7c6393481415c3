"""Pins of the oracle's Philox4x32-10 (published known answers) and properties of its
RRT-Connect planner (Sec. II-III)."""
import os

import numpy as np

from paper_2505_06791_gb300 import synth as S
from tests import indep

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def kat_vectors():
    for line in open(GOLDEN):
        f = line.split()
        if len(f) == 12 and f[0] == "philox4x32":
            yield ([int(x, 16) for x in f[2:6]], [int(x, 16) for x in f[6:8]],
                   [int(x, 16) for x in f[8:12]])


def test_philox_known_answers(oracle_mod):
    n = 0
    for ctr, key, out in kat_vectors():
        assert oracle_mod.philox4x32_10(ctr, key) == out
        n += 1
    assert n == 3


def test_philox_uniforms_are_sane(oracle_mod):
    u = []
    for i in range(4000):
        u += [(x >> 8) / 16777216.0 for x in oracle_mod.philox4x32_10([i, 7, 0, 0], [1, 0])]
    u = np.array(u)
    assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1 / 12) < 0.005
    assert u.min() >= 0.0 and u.max() < 1.0


def test_planner_paths_are_valid(oracle_mod):
    rb = S.make_arm7(1)
    sc = S.make_scene(7, n_sph=6)
    c = S.roll_pitch()
    orc = oracle_mod.Oracle(rb, sc, c)
    starts = []
    for q in S.uniform_configs(rb, 40, 71):
        ok, qp, _, _ = orc.project_config(q, max_iters=60)
        if ok and orc.config_clearance(qp) > 1e-3:
            starts.append(qp)
    starts = S.f32(np.array(starts))
    s, g = starts[:3], starts[3:6]
    out = orc.plan(s, g, range_=0.3, W=32, max_rounds=300, n_workers=8, seed=5)
    solved = 0
    for p in range(3):
        L = out["path_len"][p]
        if L <= 0:
            continue
        solved += 1
        path = out["path"][p, :L]
        assert np.abs(path[0] - s[p]).max() < 1e-12 and np.abs(path[-1] - g[p]).max() < 1e-12
        for q in path:
            assert np.abs(indep.task_error(rb.joints, rb.ee, q, 1)).max() < c.tol_task
            assert orc.config_clearance(q) > 0
        steps = np.linalg.norm(np.diff(path, axis=0), axis=1)
        assert steps.max() <= 0.3 + 1e-3
    assert solved >= 2
    again = orc.plan(s, g, range_=0.3, W=32, max_rounds=300, n_workers=8, seed=5, n_threads=3)
    assert np.array_equal(again["path_len"], out["path_len"])
    assert np.array_equal(again["path"], out["path"])
    # problem p alone, drawing with its batch index (R19), is problem p of the batch; with
    # index 0 instead it is another search
    for p in range(3):
        alone = orc.plan(s[p:p + 1], g[p:p + 1], range_=0.3, W=32, max_rounds=300, n_workers=8,
                         seed=5, first_problem=p)
        for k in ("path_len", "rounds", "waypoints"):
            assert alone[k][0] == out[k][p], (p, k)
        assert np.array_equal(alone["path"][0], out["path"][p])
    # the naive baseline's planner: every motion projected waypoint by waypoint (R27); its
    # path nodes are valid too (on the manifold, collision-free, one steering range apart)
    seq = orc.plan(s, g, range_=0.3, W=32, max_rounds=300, n_workers=8, seed=5, sequential=True)
    assert (seq["path_len"] > 0).sum() >= 2
    for p in range(3):
        L = seq["path_len"][p]
        if L <= 0:
            continue
        path = seq["path"][p, :L]
        assert np.abs(path[0] - s[p]).max() < 1e-12 and np.abs(path[-1] - g[p]).max() < 1e-12
        for q in path:
            assert np.abs(indep.task_error(rb.joints, rb.ee, q, 1)).max() < c.tol_task
            assert orc.config_clearance(q) > 0
        steps = np.linalg.norm(np.diff(path, axis=0), axis=1)
        assert steps.max() <= 0.3 + 1e-3
    moved = orc.plan(s[1:2], g[1:2], range_=0.3, W=32, max_rounds=300, n_workers=8, seed=5)
    assert not (moved["rounds"][0] == out["rounds"][1] and
                np.array_equal(moved["path"][0], out["path"][1]))


def test_free_space_connect_is_a_straight_greedy_chain(oracle_mod):
    """RRT-Connect in empty space without a constraint (Sec. II): the first extension adds
    one node within `range` of its root, then CONNECT walks straight at the other root in
    steps of exactly `range` (every step strictly closer, nothing rejects it) until it lands
    on it, and the closing hop ends the problem. The round count is one per node of the
    winning chain plus the hop, and the path is that chain with both roots."""
    rb = S.make_arm7(1)
    c = S.no_constraint()
    orc = oracle_mod.Oracle(rb, S.Scene(), c)
    s, g = S.uniform_configs(rb, 6, 91), S.uniform_configs(rb, 6, 92)
    rng_ = 0.3
    out = orc.plan(s, g, range_=rng_, W=16, max_rounds=100, n_workers=8, seed=3)
    reach = 10 * c.tau_floor
    for p in range(6):
        L = int(out["path_len"][p])
        assert L > 0
        path = out["path"][p, :L]
        assert np.array_equal(path[0], s[p].astype(np.float64))
        assert np.array_equal(path[-1], g[p].astype(np.float64))
        assert out["rounds"][p] == L - 1
        # the node that landed on the other root duplicates it (within the hop reach)
        gaps = np.abs(np.diff(path, axis=0)).max(axis=1)
        hops = np.flatnonzero(gaps <= reach)
        assert len(hops) == 1 and hops[0] in (0, L - 2)
        chain = np.delete(path, hops[0] + (1 if hops[0] == 0 else 0), axis=0)
        if hops[0] == 0:  # grown from the goal tree: walk it from the goal side
            chain = chain[::-1]
        steps = np.diff(chain, axis=0)
        length = np.linalg.norm(steps, axis=1)
        assert length[0] <= rng_ + 1e-9  # the extension toward the sample
        walk, left = steps[1:], length[1:]
        assert np.allclose(left[:-1], rng_, atol=1e-9) and left[-1] <= rng_ + 1e-9
        # straight at the other root
        u = (chain[-1] - chain[1]) / np.linalg.norm(chain[-1] - chain[1])
        assert np.allclose(walk / left[:, None], u[None, :], atol=1e-9)
