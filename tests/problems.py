"""Seeded planning problems for tests: per-problem mixed scenes (synth) and start/goal pairs
drawn uniformly, projected onto the manifold and kept when collision-free, both decided by
the oracle. Inputs only: the same arrays go to the CUDA path and to the oracle."""
import numpy as np

from paper_2505_06791_gb300 import synth as S


def planning_problems(oracle_mod, robot, constraint, n, seed, counts=(100, 60, 40),
                      clearance=1e-3, self_pairs=None):
    scenes, starts, goals = [], [], []
    p = 0
    attempt = 0
    while p < n:
        sc = S.make_planning_scene(seed + 7919 * attempt + p, *counts)
        orc = oracle_mod.Oracle(robot, sc, constraint, self_pairs=self_pairs)
        found = []
        for q in S.uniform_configs(robot, 60, seed + 104729 * attempt + p):
            if constraint.type != 0:
                ok, q, _, _ = orc.project_config(q, max_iters=60)
                if not ok:
                    continue
            if orc.config_clearance(q) > clearance:
                found.append(q)
            if len(found) == 2:
                break
        if len(found) < 2:
            attempt += 1
            continue
        scenes.append(sc)
        starts.append(found[0])
        goals.append(found[1])
        p += 1
    return scenes, S.f32(np.array(starts)), S.f32(np.array(goals))


def check_paths(oracle_mod, robot, constraint, scenes, start, goal, out, W, range_,
                problems=None, slack=2e-6, contact=1e-5, self_pairs=None):
    """Re-validates every returned path with the oracle (with `self_pairs`, the robot's named
    frame pairs count as obstacles too); returns (#checked, list of issues)."""
    to_np = lambda x: x.detach().cpu().numpy() if hasattr(x, "detach") else np.asarray(x)  # noqa
    L = to_np(out["path_len"])
    path = to_np(out["path"])
    edges = to_np(out["path_edges"])
    issues, checked = [], 0
    tau = max(constraint.c_sm * range_ / (W - 1), constraint.tau_floor)
    for p in (range(len(L)) if problems is None else problems):
        n = int(L[p])
        if n <= 0:
            continue
        checked += 1
        orc = oracle_mod.Oracle(robot, scenes[p], constraint, self_pairs=self_pairs)
        P = path[p, :n].astype(np.float64)
        if not (np.array_equal(path[p, 0], start[p].astype(np.float32)) and
                np.array_equal(path[p, n - 1], goal[p].astype(np.float32))):
            issues.append((p, "endpoints"))
        for j in range(n - 1):
            E = edges[p, j].astype(np.float64)
            if np.abs(E[0] - P[j]).max() > 1e-6 or np.abs(E[-1] - P[j + 1]).max() > 1e-6:
                issues.append((p, j, "edge does not join its nodes"))
                continue
            t, s_, c = orc.check_segment(E, tau)
            if constraint.type != 0 and t >= constraint.tol_task + slack:
                issues.append((p, j, "off manifold", t))
            if s_ >= constraint.tol_sm + slack:
                issues.append((p, j, "discontinuous", s_))
            if c <= -contact:
                issues.append((p, j, "collision", c))
    return checked, issues


def batch_start_goal(oracle_mod, robots, constraints, problems, scenes, seed, clearance=1e-3):
    """Start and goal [n][8] for a batch: per problem, uniform configurations of its robot,
    projected under its constraint and kept when collision-free in its scene (oracle)."""
    n = len(problems)
    start = np.zeros((n, 8))
    goal = np.zeros((n, 8))
    for p, (r, c, sc, W) in enumerate(problems):
        rb, cons = robots[r], constraints[c]
        orc = oracle_mod.Oracle(rb, scenes[sc], cons)
        found, k = [], 0
        while len(found) < 2:
            for q in S.uniform_configs(rb, 40, seed + 7919 * p + 104729 * k):
                if cons.type != 0:
                    ok, q, _, _ = orc.project_config(q, max_iters=60)
                    if not ok:
                        continue
                if orc.config_clearance(q) > clearance:
                    found.append(q)
                if len(found) == 2:
                    break
            k += 1
            if k > 50:
                raise RuntimeError(f"no free start/goal for problem {p}")
        start[p, :rb.dof] = found[0]
        goal[p, :rb.dof] = found[1]
    return S.f32(start), S.f32(goal)


def check_batch_paths(oracle_mod, robots, constraints, problems, scenes, start, goal, out,
                      range_, slack=2e-6, contact=1e-5, sample=None):
    """Oracle re-validation of batch paths ([n][max_path][8] nodes, [n][max_path-1][Wmax][8]
    edges); `sample` restricts it to those problem indices."""
    to_np = lambda x: x.detach().cpu().numpy() if hasattr(x, "detach") else np.asarray(x)  # noqa
    L = to_np(out["path_len"])
    path = to_np(out["path"])
    edges = to_np(out["path_edges"]) if out.get("path_edges") is not None else None
    issues, checked = [], 0
    for p, (r, c, sc, W) in enumerate(problems):
        if sample is not None and p not in sample:
            continue
        n = int(L[p])
        if n <= 0:
            continue
        checked += 1
        rb, cons = robots[r], constraints[c]
        dof = rb.dof
        tau = max(cons.c_sm * range_ / (W - 1), cons.tau_floor)
        orc = oracle_mod.Oracle(rb, scenes[sc], cons)
        P = path[p, :n, :dof].astype(np.float64)
        if not (np.array_equal(path[p, 0, :dof], start[p, :dof].astype(np.float32)) and
                np.array_equal(path[p, n - 1, :dof], goal[p, :dof].astype(np.float32))):
            issues.append((p, "endpoints"))
        if edges is None:
            continue
        for j in range(n - 1):
            E = edges[p, j, :W, :dof].astype(np.float64)
            if np.abs(E[0] - P[j]).max() > 1e-6 or np.abs(E[-1] - P[j + 1]).max() > 1e-6:
                issues.append((p, j, "edge does not join its nodes"))
                continue
            t, s_, cl = orc.check_segment(E, tau)
            if cons.type != 0 and t >= cons.tol_task + slack:
                issues.append((p, j, "off manifold", t))
            if s_ >= cons.tol_sm + slack:
                issues.append((p, j, "discontinuous", s_))
            if cl <= -contact:
                issues.append((p, j, "collision", cl))
    return checked, issues


def assert_same_plans(a, b, keys=("path_len", "path", "rounds", "waypoints"), dofs=None,
                      Ws=None):
    """Two planner outputs (dicts of numpy arrays) agree: per-problem fields exactly, and
    the path rows (and path_edges motions) that path_len says were written, over problem
    p's dofs[p] joints and Ws[p] waypoints when given; rows beyond path_len and padding are
    not part of the result."""
    L = np.asarray(a["path_len"])
    for k in keys:
        if k in ("path", "path_edges"):
            if a.get(k) is None:
                continue
            for p in range(len(L)):
                n = int(L[p]) if L[p] > 0 else 0
                d = a[k].shape[-1] if dofs is None else int(dofs[p])
                if k == "path":
                    x, y = a[k][p, :n, :d], b[k][p, :n, :d]
                else:
                    w = a[k].shape[2] if Ws is None else int(Ws[p])
                    x, y = a[k][p, :max(n - 1, 0), :w, :d], b[k][p, :max(n - 1, 0), :w, :d]
                assert np.array_equal(x, y), (k, p)
        else:
            assert np.array_equal(a[k], b[k]), k
