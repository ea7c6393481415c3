"""Pins of the oracle's Algorithm 1 (ParallelProject, Sec. III-A) and of the single-
configuration projection, against an independent damped Gauss-Newton, invariants the
algorithm guarantees, and special cases."""
import numpy as np
import pytest

from paper_2505_06791_gb300 import synth as S
from tests import indep


def on_manifold(orc, rb, n, seed, max_iters=60):
    qs = S.uniform_configs(rb, 4 * n, seed)
    out = []
    for q in qs:
        ok, qp, _, _ = orc.project_config(q, max_iters=max_iters)
        if ok:
            out.append(qp)
        if len(out) == n:
            break
    return S.f32(np.array(out))


def gauss_newton_reference(rb, c, q, max_iters):
    """Damped Gauss-Newton written from library pieces: scipy Euler angles for E_task, a
    finite-difference Jacobian, and numpy lstsq for the damped least-squares step."""
    f = lambda x: indep.task_error(rb.joints, rb.ee, x, c.type, c.target,  # noqa: E731
                                   getattr(c, "line_y", 0.0), getattr(c, "yaw", 0.0))
    q = np.array(q, np.float64)
    for it in range(1, max_iters + 1):
        e = f(q)
        if np.abs(e).max() < c.tol_task:
            return True, it, q
        J = indep.fd_jacobian(f, q, 1e-7)
        A = np.vstack([J, c.lam * np.eye(rb.dof)])
        b = np.concatenate([e, np.zeros(rb.dof)])
        g = np.linalg.lstsq(A, b, rcond=None)[0]
        q = np.clip(q - c.alpha * g, rb.lo, rb.hi)
    return False, max_iters, q


@pytest.mark.parametrize("ctype", [1, 2])
def test_two_waypoints_reduce_to_damped_gauss_newton(oracle_mod, ctype):
    """W = 2 with the smoothing term inactive: Alg. 1 is damped Gauss-Newton on waypoint 1,
    accepted at the first iteration whose current point meets the tolerance."""
    rb = S.make_arm7(1) if ctype == 1 else S.make_arm8(1)
    c = S.roll_pitch() if ctype == 1 else S.z_plane(0.9)
    c.c_sm = 1e9  # tau far above any step: E_sm = 0
    orc = oracle_mod.Oracle(rb, constraint=c)
    q0 = S.uniform_configs(rb, 12, 21)
    q1 = S.nearby_configs(rb, q0, 0.2, 22)
    compared = 0
    for a, b in zip(q0, q1):
        xi = oracle_mod.interpolate(a, b, 2)
        r = orc.project_motion(xi, tau=1e9)
        ok, it, q = gauss_newton_reference(rb, c, xi[1], c.max_iters)
        if ctype == 1 and not ok:
            continue
        assert r["ok"] == ok and r["iters"] == it
        assert np.abs(r["xi"][1] - q).max() < 1e-6
        assert np.array_equal(r["xi"][0], xi[0])
        compared += 1
    assert compared >= 8


@pytest.mark.parametrize("ctype", [1, 2])
def test_base_yaw_motion_is_returned_unchanged(oracle_mod, ctype):
    """Joint 1 turns about the world z axis: roll, pitch and EE height are invariant under
    it, so a base-yaw motion from an on-manifold start is accepted at iteration 1 as is."""
    rb = S.make_arm7(2) if ctype == 1 else S.make_arm8(2)
    c = S.roll_pitch() if ctype == 1 else S.z_plane(0.9)
    orc = oracle_mod.Oracle(rb, constraint=c)
    j1 = 0 if ctype == 1 else 1
    for q0 in on_manifold(orc, rb, 5, 23):
        q1 = q0.copy()
        q1[j1] = np.clip(q1[j1] + 0.4, -2.8, 2.8)
        xi = oracle_mod.interpolate(q0, q1, 32)
        r = orc.project_motion(xi, tau=oracle_mod.tau_step(c, q0, q1, 32))
        assert r["ok"] and r["iters"] == 1
        assert np.array_equal(r["xi"], xi)


def test_projection_invariants_on_random_motions(oracle_mod):
    rb = S.make_arm7(1)
    c = S.roll_pitch()
    orc = oracle_mod.Oracle(rb, constraint=c)
    q0 = on_manifold(orc, rb, 24, 31)
    q1 = np.concatenate([S.nearby_configs(rb, q0[:12], 0.3, 32), S.uniform_configs(rb, 12, 33)])
    n_ok = 0
    for a, b in zip(q0, q1):
        xi = oracle_mod.interpolate(a, b, 32)
        tau = oracle_mod.tau_step(c, a, b, 32)
        r = orc.project_motion(xi, tau, trace=True)
        out = r["xi"]
        assert np.array_equal(out[0], xi[0])                       # q0 fixed
        assert np.all(np.diff(r["prog_trace"]) >= 0)               # prog never decreases
        assert np.all(out >= rb.lo) and np.all(out <= rb.hi)       # within limits
        if r["ok"]:
            n_ok += 1
            for i in range(1, 32):
                e = indep.task_error(rb.joints, rb.ee, out[i], 1)
                assert np.abs(e).max() < c.tol_task
                assert np.max(np.abs(out[i] - out[i - 1])) - tau < c.tol_sm
            assert r["prog_trace"][-1] == 31 and r["first_fail"] == -1
        else:
            assert r["iters"] == c.max_iters
            assert r["first_fail"] == r["prog_trace"][-1] + 1
    assert n_ok >= 10


def test_acceptance_is_a_contiguous_prefix(oracle_mod):
    """A waypoint pushed off the manifold blocks acceptance of everything after it in the
    first iteration, even though the later waypoints are valid."""
    rb = S.make_arm7(2)
    c = S.roll_pitch()
    orc = oracle_mod.Oracle(rb, constraint=c)
    q0 = on_manifold(orc, rb, 1, 41)[0]
    q1 = q0.copy()
    q1[0] = q0[0] + 0.3
    xi = oracle_mod.interpolate(q0, q1, 16)
    xi[5, 3] += 0.02  # off the manifold
    tau = 1.0
    r = orc.project_motion(xi, tau, trace=True)
    assert r["prog_trace"][0] == 4
    assert r["ok"] and r["iters"] >= 2
    # waypoints 1..4 were accepted in iteration 1 and never moved again
    assert np.array_equal(r["xi"][:5], xi[:5])


def test_single_config_projection_converges_to_manifold(oracle_mod):
    rb = S.make_arm7(1)
    c = S.roll_pitch()
    orc = oracle_mod.Oracle(rb, constraint=c)
    n_ok = 0
    for q in S.uniform_configs(rb, 30, 51):
        ok, qp, it, res = orc.project_config(q, max_iters=60)
        if ok:
            n_ok += 1
            e = indep.task_error(rb.joints, rb.ee, qp, 1)
            assert np.abs(e).max() < c.tol_task and abs(np.abs(e).max() - res) < 1e-15
    assert n_ok >= 25


def test_sequential_projection_produces_continuous_segment(oracle_mod):
    rb = S.make_arm7(1)
    c = S.roll_pitch()
    orc = oracle_mod.Oracle(rb, constraint=c)
    q0 = on_manifold(orc, rb, 6, 61)
    q1 = S.nearby_configs(rb, q0, 0.3, 62)
    n_ok = 0
    for a, b in zip(q0, q1):
        xi = oracle_mod.interpolate(a, b, 32)
        tau = oracle_mod.tau_step(c, a, b, 32)
        ok, out, ff, tot = orc.project_motion_sequential(xi, tau)
        if ok:
            n_ok += 1
            assert ff == -1
            for i in range(1, 32):
                assert np.abs(indep.task_error(rb.joints, rb.ee, out[i], 1)).max() < c.tol_task
                assert np.max(np.abs(out[i] - out[i - 1])) - tau < c.tol_sm
    assert n_ok >= 3


@pytest.mark.parametrize("ctype", [1, 2])
def test_sequential_projection_composes_single_projections(oracle_mod, ctype):
    """The naive baseline's projection is a chain of single-configuration projections:
    waypoint i is the damped Gauss-Newton projection (the independent reference) of its
    interpolated point moved by waypoint i-1's correction, its step count adds to the total,
    and with W = 2 the whole motion is the projection of its end point. Both constraints
    the GPU's sequential form takes (roll-pitch, z-plane)."""
    rb = S.make_arm7(1)
    c = S.roll_pitch() if ctype == 1 else S.z_plane(0.6)
    orc = oracle_mod.Oracle(rb, constraint=c)
    q0 = on_manifold(orc, rb, 6, 63)
    q1 = S.nearby_configs(rb, q0, 0.3, 64)
    checked = 0
    for a, b in zip(q0, q1):
        xi = oracle_mod.interpolate(a, b, 8)
        tau = oracle_mod.tau_step(c, a, b, 8)
        ok, out, ff, tot = orc.project_motion_sequential(xi, tau)
        last = 8 if ok else ff + 1
        steps = 0
        for i in range(1, last):
            start = np.clip(xi[i] + (out[i - 1] - xi[i - 1]), rb.lo, rb.hi)
            pok, qp, it, _ = orc.project_config(start, max_iters=c.max_iters)
            assert np.array_equal(qp, out[i]), i
            ref_ok, ref_it, ref_q = gauss_newton_reference(rb, c, start, c.max_iters + 1)
            if pok:
                assert ref_ok and ref_it - 1 == it
                assert np.abs(ref_q - qp).max() < 1e-6
            steps += it
        assert steps == tot
        checked += 1
        ok2, out2, ff2, tot2 = orc.project_motion_sequential(oracle_mod.interpolate(a, b, 2),
                                                             oracle_mod.tau_step(c, a, b, 2))
        pok, qp, it, _ = orc.project_config(np.asarray(b, np.float64), max_iters=c.max_iters)
        assert np.array_equal(out2[1], qp) and tot2 == it
    assert checked == 6


@pytest.mark.parametrize("ctype", [1, 2, 5])
def test_first_iteration_combines_task_and_smoothing_terms(oracle_mod, ctype):
    """One iteration of Alg. 1 on an uneven segment, the smoothing hinge active on some
    joints and not on others: every waypoint after the accepted prefix moves by
    -alpha (J^+ E_task + d * max(0, |d| - tau)) with d its difference to the previous
    waypoint (the task step from the independent damped least squares), then clamped to the
    limits; the prefix stays as it was."""
    rb = S.make_arm7(1)
    c = {1: S.roll_pitch(), 2: S.z_plane(0.6), 5: S.orient_line(-0.4, 0.1, 0.6)}[ctype]
    c.max_iters = 1
    orc = oracle_mod.Oracle(rb, constraint=c)
    q0s = on_manifold(orc, rb, 6, 121)
    rng = np.random.default_rng(122)
    t = np.array([0.0, 0.05, 0.1, 0.4, 0.45, 0.7, 1.0])
    tau = 0.03
    active = inactive = 0
    for q0 in q0s:
        delta = rng.normal(size=rb.dof)
        delta *= 0.6 / np.linalg.norm(delta)
        xi = np.clip(q0[None, :] + t[:, None] * delta[None, :], rb.lo, rb.hi)
        r = orc.project_motion(xi, tau=tau, trace=True)
        assert not r["ok"] and r["iters"] == 1
        prog = int(r["prog_trace"][0])
        assert np.array_equal(r["xi"][: prog + 1], xi[: prog + 1])
        assert r["first_fail"] == prog + 1
        f = lambda x: indep.task_error(rb.joints, rb.ee, x, c.type, c.target,  # noqa: E731
                                       c.line_y, c.yaw)
        for i in range(prog + 1, len(t)):
            J = indep.fd_jacobian(f, xi[i], 1e-7)
            A = np.vstack([J, c.lam * np.eye(rb.dof)])
            b = np.concatenate([f(xi[i]), np.zeros(rb.dof)])
            g_task = np.linalg.lstsq(A, b, rcond=None)[0]
            d = xi[i] - xi[i - 1]
            hinge = np.maximum(0.0, np.abs(d) - tau)
            want = np.clip(xi[i] - c.alpha * (g_task + d * hinge), rb.lo, rb.hi)
            assert np.abs(r["xi"][i] - want).max() < 1e-6, (i, r["xi"][i] - want)
            active += int((hinge > 0).sum())
            inactive += int((hinge == 0).sum())
    assert active >= 20 and inactive >= 20
