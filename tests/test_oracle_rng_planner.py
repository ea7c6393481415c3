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
