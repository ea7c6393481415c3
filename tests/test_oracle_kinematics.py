"""Pins of the oracle's kinematics and task functions (GetTaskError / GetTaskJacobian,
Alg. 1) against closed forms, scipy rotation primitives, the product-of-exponentials form
and finite differences."""
import math

import numpy as np
import pytest

from paper_2505_06791_gb300 import synth as S
from tests import indep


def planar2(l1, l2):
    joints = np.array([[0, 0.0, l1, 0.0, 0.0, -3.0, 3.0],
                       [0, 0.0, l2, 0.0, 0.0, -3.0, 3.0]])
    return S.Robot(joints, np.zeros(3), np.array([[2, 0.0, 0.0, 0.0, 0.05]]))


def test_fk_planar_two_link_closed_form(oracle_mod):
    rb = planar2(0.7, 0.4)
    orc = oracle_mod.Oracle(rb)
    rng = np.random.default_rng(0)
    for _ in range(20):
        q = rng.uniform(-3, 3, 2)
        F = orc.fk(q)[-1]
        x = 0.7 * math.cos(q[0]) + 0.4 * math.cos(q[0] + q[1])
        y = 0.7 * math.sin(q[0]) + 0.4 * math.sin(q[0] + q[1])
        assert abs(F[0, 3] - x) < 1e-15 and abs(F[1, 3] - y) < 1e-15 and abs(F[2, 3]) < 1e-15
        th = q[0] + q[1]
        R = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0],
                      [0, 0, 1]])
        assert np.abs(F[:3, :3] - R).max() < 1e-15


@pytest.mark.parametrize("arm", ["arm7", "arm8", "arm6"])
def test_fk_matches_scipy_chain_and_poe(oracle_mod, arm):
    rb = getattr(S, "make_" + arm)(3)
    orc = oracle_mod.Oracle(rb)
    q = S.uniform_configs(rb, 10, 5)
    for qi in q:
        F = orc.fk(qi)
        G = indep.fk_frames(rb.joints, rb.ee, qi)
        assert np.abs(F - G).max() < 1e-13
        P = indep.fk_poe(rb.joints, rb.ee, qi)
        assert np.abs(F[-1] - P).max() < 1e-11
        for T in F:
            R = T[:3, :3]
            assert np.abs(R.T @ R - np.eye(3)).max() < 1e-14
            assert abs(np.linalg.det(R) - 1) < 1e-14


def test_joint_origin_distances_are_invariant(oracle_mod):
    rb = S.make_arm7(4)
    orc = oracle_mod.Oracle(rb)
    q = S.uniform_configs(rb, 6, 6)
    ref = None
    for qi in q:
        F = orc.fk(qi)
        dist = [np.linalg.norm(F[k + 1][:3, 3] - F[k][:3, 3]) for k in range(7)]
        if ref is None:
            ref = dist
        assert np.allclose(dist, ref, atol=1e-14)
        assert np.allclose(dist, np.hypot(rb.joints[:, 1], rb.joints[:, 2]), atol=1e-14)


@pytest.mark.parametrize("arm", ["arm7", "arm8"])
def test_geometric_jacobian_finite_differences(oracle_mod, arm):
    rb = getattr(S, "make_" + arm)(2)
    orc = oracle_mod.Oracle(rb)
    for qi in S.uniform_configs(rb, 5, 9):
        J = orc.jacobian(qi)
        Jv = indep.fd_jacobian(lambda q: indep.fk_frames(rb.joints, rb.ee, q)[-1][:3, 3], qi)
        assert np.abs(J[:3] - Jv).max() < 1e-8
        # angular part: dR/dq_k R^T is the skew matrix of column k of J_w
        h = 1e-6
        R0 = indep.fk_frames(rb.joints, rb.ee, qi)[-1][:3, :3]
        for k in range(rb.dof):
            dq = np.zeros(rb.dof)
            dq[k] = h
            Rp = indep.fk_frames(rb.joints, rb.ee, qi + dq)[-1][:3, :3]
            Rm = indep.fk_frames(rb.joints, rb.ee, qi - dq)[-1][:3, :3]
            Wk = (Rp - Rm) / (2 * h) @ R0.T
            w = np.array([Wk[2, 1], Wk[0, 2], Wk[1, 0]])
            assert np.abs(J[3:, k] - w).max() < 1e-8


def test_roll_pitch_error_matches_scipy_euler(oracle_mod):
    rb = S.make_arm7(1)
    orc = oracle_mod.Oracle(rb, constraint=S.roll_pitch())
    for qi in S.uniform_configs(rb, 20, 10):
        e, J = orc.task(qi)
        assert e.shape == (2,) and J.shape == (2, 7)
        ref = indep.task_error(rb.joints, rb.ee, qi, 1)
        assert np.abs(e - ref).max() < 1e-12


@pytest.mark.parametrize("ctype", [1, 2])
def test_task_jacobian_finite_differences(oracle_mod, ctype):
    rb = S.make_arm8(1) if ctype == 2 else S.make_arm7(1)
    c = S.roll_pitch() if ctype == 1 else S.z_plane(0.9)
    orc = oracle_mod.Oracle(rb, constraint=c)
    rng = np.random.default_rng(1)
    checked = 0
    for qi in S.uniform_configs(rb, 20, 11):
        e, J = orc.task(qi)
        if ctype == 1 and abs(abs(e[0]) - math.pi) < 0.3:
            continue  # roll branch cut: the error is not differentiable there
        f = lambda q: indep.task_error(rb.joints, rb.ee, q, ctype, c.target)  # noqa: E731
        Jfd = indep.fd_jacobian(f, qi)
        assert np.abs(J - Jfd).max() < 1e-7
        checked += 1
    assert checked >= 10
    del rng


def test_z_plane_error(oracle_mod):
    rb = S.make_arm8(1)
    orc = oracle_mod.Oracle(rb, constraint=S.z_plane(0.9))
    for qi in S.uniform_configs(rb, 5, 12):
        e, _ = orc.task(qi)
        z = indep.fk_frames(rb.joints, rb.ee, qi)[-1][2, 3]
        assert abs(e[0] - (z - 0.9)) < 1e-13


def test_sphere_centres_match_independent_fk(oracle_mod):
    rb = S.make_arm7(7)
    orc = oracle_mod.Oracle(rb)
    for qi in S.uniform_configs(rb, 4, 13):
        c = orc.sphere_centres(qi)
        ref = indep.sphere_centres(rb.joints, rb.ee, rb.spheres, qi)
        assert np.abs(c - ref).max() < 1e-13


def test_damped_step_against_numpy_pinv_and_lstsq(oracle_mod):
    rng = np.random.default_rng(3)
    for m in (1, 2, 3, 5):
        for _ in range(5):
            J = rng.normal(size=(m, 7))
            e = rng.normal(size=m)
            # lambda -> 0 on a full-rank J: the Moore-Penrose pseudoinverse (SVD)
            g0 = oracle_mod.Oracle.damped_step(J, e, 1e-12)
            assert np.abs(g0 - np.linalg.pinv(J) @ e).max() < 1e-9
            # lambda > 0: the minimiser of ||J g - e||^2 + lambda^2 ||g||^2
            lam = 0.3
            g = oracle_mod.Oracle.damped_step(J, e, lam)
            A = np.vstack([J, lam * np.eye(7)])
            b = np.concatenate([e, np.zeros(7)])
            ref = np.linalg.lstsq(A, b, rcond=None)[0]
            assert np.abs(g - ref).max() < 1e-12


def test_damped_step_identities(oracle_mod):
    """J J^+_lambda = I - lambda^2 (J J^T + lambda^2 I)^-1 (the damped pseudoinverse's
    residual map) for every row count a constraint uses (1, 2, 4, 5), and on a rank-deficient
    J (two equal rows) the damped step stays finite, lies in the row space of J and tends to
    the minimum-norm least-squares step of numpy's SVD pseudoinverse as lambda -> 0."""
    rng = np.random.default_rng(5)
    for m in (1, 2, 4, 5):
        J = rng.normal(size=(m, 7))
        lam = 0.2
        Ginv = np.linalg.inv(J @ J.T + lam ** 2 * np.eye(m))
        for _ in range(4):
            e = rng.normal(size=m)
            g = oracle_mod.Oracle.damped_step(J, e, lam)
            assert np.abs(J @ g - (e - lam ** 2 * Ginv @ e)).max() < 1e-12
    J = rng.normal(size=(4, 7))
    J[3] = J[1]
    e = rng.normal(size=4)
    P = np.linalg.pinv(J)
    row_space = P @ J  # projector onto the row space
    for lam in (1e-2, 1e-4):
        g = oracle_mod.Oracle.damped_step(J, e, lam)
        assert np.all(np.isfinite(g))
        # J J^T + lambda^2 I has condition ~1/lambda^2 here: rounding grows with it
        assert np.abs(row_space @ g - g).max() < 1e-14 / lam ** 2
        assert np.abs(g - P @ e).max() < 50 * lam ** 2 * np.abs(P @ e).max() + 1e-9


def test_prismatic_torso_translates_the_arm(oracle_mod):
    """The 8-DOF arm's first joint slides along the base z axis: changing only it by delta
    moves every later frame by delta along world z and rotates none of them (the prismatic
    form of the DH factor adds q to d)."""
    rb = S.make_arm8(3)
    orc = oracle_mod.Oracle(rb)
    for qi in S.uniform_configs(rb, 5, 17):
        q2 = qi.copy()
        delta = 0.4 - qi[0] if qi[0] < 0.2 else -qi[0]
        q2[0] = qi[0] + delta
        F, G = orc.fk(qi), orc.fk(q2)
        for k in range(1, len(F)):
            assert np.abs(G[k][:3, :3] - F[k][:3, :3]).max() < 1e-14
            assert np.abs(G[k][:3, 3] - F[k][:3, 3] - [0.0, 0.0, delta]).max() < 1e-14
