"""Pins of the oracle's line and fixed-orientation task constraints (the paper's other
constraint variants, Sec. V-B): task errors against scipy's Euler angles and the closed-form
end-effector position, task Jacobians against finite differences, the yaw wrap, and
Alg. 1 at W = 2 against an independent damped Gauss-Newton."""
import math

import numpy as np
import pytest

from paper_2505_06791_gb300 import synth as S
from tests import indep
from tests.test_oracle_projection import gauss_newton_reference

CASES = {
    3: lambda: S.line(0.1, 0.6),
    4: lambda: S.orient_plane(0.5, 0.6),
    5: lambda: S.orient_line(-0.4, 0.1, 0.6),
}


def ref_error(rb, c, q):
    return indep.task_error(rb.joints, rb.ee, q, c.type, c.target, c.line_y, c.yaw)


@pytest.mark.parametrize("ctype", [3, 4, 5])
def test_task_error_matches_independent_reference(oracle_mod, ctype):
    rb, c = S.make_arm7(1), CASES[ctype]()
    orc = oracle_mod.Oracle(rb, constraint=c)
    rows = {3: 2, 4: 4, 5: 5}[ctype]
    for qi in S.uniform_configs(rb, 30, 40 + ctype):
        e, J = orc.task(qi)
        assert e.shape == (rows,) and J.shape == (rows, 7)
        ref = ref_error(rb, c, qi)
        d = np.abs(e - ref)
        if ctype >= 4:  # yaw rows equal up to the representation of a wrap at +-pi
            d[2] = min(d[2], abs(d[2] - 2 * math.pi))
        assert d.max() < 1e-12, (e, ref)


def test_yaw_error_is_wrapped(oracle_mod):
    """The yaw row is psi - yaw in (-pi, pi]: a target one turn away gives the same error."""
    rb = S.make_arm7(1)
    q = S.uniform_configs(rb, 10, 50)
    a = oracle_mod.Oracle(rb, constraint=S.orient_plane(0.3, 0.6))
    b = oracle_mod.Oracle(rb, constraint=S.orient_plane(0.3 + 2 * math.pi, 0.6))
    for qi in q:
        ea, _ = a.task(qi)
        eb, _ = b.task(qi)
        assert -math.pi < ea[2] <= math.pi
        assert abs(ea[2] - eb[2]) < 1e-12


@pytest.mark.parametrize("arm", ["arm7", "arm8"])
@pytest.mark.parametrize("ctype", [3, 4, 5])
def test_task_jacobian_finite_differences(oracle_mod, ctype, arm):
    """Task Jacobians against central differences, also on the 8-DOF arm whose prismatic
    torso adds a column with linear velocity only."""
    rb = S.make_arm7(1) if arm == "arm7" else S.make_arm8(1)
    c = CASES[ctype]()
    orc = oracle_mod.Oracle(rb, constraint=c)
    checked = 0
    for qi in S.uniform_configs(rb, 30, 60 + ctype):
        e, J = orc.task(qi)
        if ctype >= 4:
            # away from the roll branch cut, the yaw wrap and pitch = +-pi/2
            if abs(abs(e[0]) - math.pi) < 0.3 or abs(abs(e[2]) - math.pi) < 0.3 or \
                    abs(e[1]) > 1.3:
                continue
        Jfd = indep.fd_jacobian(lambda q: ref_error(rb, c, q), qi)
        assert J.shape == (Jfd.shape[0], rb.dof)
        assert np.abs(J - Jfd).max() < 1e-7, np.abs(J - Jfd).max()
        checked += 1
    assert checked >= 8


@pytest.mark.parametrize("ctype", [3, 4, 5])
def test_two_waypoints_reduce_to_damped_gauss_newton(oracle_mod, ctype):
    """W = 2 with the smoothing term inactive: Alg. 1 is damped Gauss-Newton on waypoint 1
    (the reference takes scipy's angles, a finite-difference Jacobian and numpy lstsq).
    One iteration: the same damped step to 1e-6. Run to convergence: the same acceptance
    iteration, and both points on the manifold (with four or five task rows the damped
    steps drift along the null space, which the reference's finite-difference Jacobian
    perturbs by ~1e-4 rad over tens of iterations)."""
    rb, c = S.make_arm7(1), CASES[ctype]()
    c.c_sm = 1e9
    c.max_iters = 40
    orc = oracle_mod.Oracle(rb, constraint=c)
    c1 = CASES[ctype]()
    c1.c_sm, c1.max_iters = 1e9, 1
    one = oracle_mod.Oracle(rb, constraint=c1)
    q0 = S.uniform_configs(rb, 16, 70 + ctype)
    q1 = S.nearby_configs(rb, q0, 0.2, 80 + ctype)
    compared = 0
    for a, b in zip(q0, q1):
        xi = oracle_mod.interpolate(a, b, 2)
        r1 = one.project_motion(xi, tau=1e9)
        ok1, _, qs = gauss_newton_reference(rb, c1, xi[1], 1)
        if not ok1:
            assert np.abs(r1["xi"][1] - qs).max() < 1e-6
        r = orc.project_motion(xi, tau=1e9)
        ok, it, q = gauss_newton_reference(rb, c, xi[1], c.max_iters)
        if not ok:
            continue
        assert r["ok"] and r["iters"] == it
        assert np.abs(ref_error(rb, c, r["xi"][1])).max() < c.tol_task
        assert np.abs(ref_error(rb, c, q)).max() < c.tol_task
        assert np.array_equal(r["xi"][0], xi[0])
        compared += 1
    assert compared >= 6


@pytest.mark.parametrize("ctype", [3, 4, 5])
def test_projected_configurations_satisfy_the_constraint(oracle_mod, ctype):
    """Single-configuration projections that succeed lie on the manifold: the position rows
    put the end effector on the plane or line, the orientation rows give roll = pitch = 0
    and the target yaw, all checked with the independent forward kinematics."""
    rb, c = S.make_arm7(1), CASES[ctype]()
    orc = oracle_mod.Oracle(rb, constraint=c)
    ok_count = 0
    for q in S.uniform_configs(rb, 40, 90 + ctype):
        ok, qp, _, _ = orc.project_config(q, max_iters=80)
        if not ok:
            continue
        F = indep.fk_frames(rb.joints, rb.ee, qp)[-1]
        assert abs(F[2, 3] - c.target) < c.tol_task
        if ctype in (3, 5):
            assert abs(F[1, 3] - c.line_y) < c.tol_task
        if ctype >= 4:
            assert np.abs(F[:3, 2] - np.array([0.0, 0.0, 1.0])).max() < 2 * c.tol_task
            assert abs(math.atan2(F[1, 0], F[0, 0]) - c.yaw) < 2 * c.tol_task
        ok_count += 1
    assert ok_count >= 5
