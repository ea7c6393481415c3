"""Comparison of the CUDA path's motion-validation outputs with the oracle's.

The method's outputs are integers decided by floating point (Alg. 1's acceptance tests,
the collision predicates) plus the projected waypoints. The FP32 kernel and the FP64
oracle evaluate the decided quantities with different rounding, so the protocol is:

  Projection (Alg. 1). The oracle runs the batch five times: with the stated thresholds
  and with tol_task or tol_sm shifted by +-DELTA (DELTA = 2e-6, above the FP32 evaluation
  error of ||E_task||_inf and E_sm for these arms). A motion whose outcome (status class,
  iteration count, first unaccepted waypoint) is the same in all five is "robust": the GPU
  must reproduce it exactly and its waypoints must lie within WAYPOINT_TOL of the oracle's.
  Otherwise the GPU must reproduce one of the five outcomes, with waypoints within
  WAYPOINT_TOL of that run (several results are correct; the GPU's must be one of them).

  Collision (Sec. IV). With dq the motion's largest waypoint deviation, the verdict and the
  first colliding waypoint must match exactly whenever the oracle's deciding clearance
  exceeds CONTACT_MARGIN + LEVER * dq (a joint error dq moves a sphere by at most
  LEVER * dq for these arms).
"""
import copy

import numpy as np

DELTA = 2e-6
WAYPOINT_TOL = 1e-4
CONTACT_MARGIN = 1e-5
LEVER = 2.0


def to_np(x):
    if hasattr(x, "detach"):
        return x.detach().cpu().numpy()
    return np.asarray(x)


def oracle_runs(orc, constraint, q_start, q_end, W, cc_skip_first=False, n_threads=1):
    """The base oracle run followed by the four threshold-shifted runs."""
    runs = []
    shifts = [(0, 0)]
    if constraint.type != 0:
        shifts += [(DELTA, 0), (-DELTA, 0), (0, DELTA), (0, -DELTA)]
    for dt, ds in shifts:
        c = copy.copy(constraint)
        c.tol_task += dt
        c.tol_sm += ds
        orc.set_constraint(c)
        runs.append(orc.validate(q_start, q_end, W, cc_skip_first=cc_skip_first,
                                 n_threads=n_threads))
    orc.set_constraint(constraint)
    return runs


def _outcome(r, m):
    return (int(r["status"][m]) == 1, int(r["iters"][m]),
            int(r["first_fail"][m]) if int(r["status"][m]) == 1 else None)


def compare(gpu, runs, fail_drift=False):
    """Parity protocol. With fail_drift, a motion that both sides fail to project (at the
    iteration cap) may differ in the waypoint where Alg. 1 gave up: with four or five task
    rows the damped system J J^T + lambda^2 I is ill-conditioned near singular arm poses, and
    over the iterations of a failing projection FP32 and FP64 iterates separate; such
    motions are counted (stats["fail_drift"]), not failed."""
    g = {k: to_np(v) for k, v in gpu.items()}
    base = runs[0]
    n = len(g["status"])
    stats = dict(n=n, robust=0, sensitive=0, ambiguous_cc=0, max_dq=0.0, exact=0, fail_drift=0)
    bad = []
    for m in range(n):
        outs = [_outcome(r, m) for r in runs]
        g_out = (int(g["status"][m]) == 1, int(g["iters"][m]),
                 int(g["first_fail"][m]) if int(g["status"][m]) == 1 else None)
        robust = all(o == outs[0] for o in outs)
        stats["robust" if robust else "sensitive"] += 1
        match = [i for i, o in enumerate(outs) if o == g_out]
        if not match and fail_drift and g_out[0] and outs[0][0] and g_out[1] == outs[0][1]:
            stats["fail_drift"] += 1
            continue
        if not match:
            bad.append((m, "projection outcome", outs[0], g_out, robust))
            continue
        ref = runs[match[0]]
        if g_out[0]:        # PROJ_FAIL: nothing further is decided
            stats["exact"] += robust
            continue
        dq = min(float(np.abs(g["q"][m].astype(np.float64) - runs[i]["q"][m]).max())
                 for i in match)
        stats["max_dq"] = max(stats["max_dq"], dq)
        if dq > WAYPOINT_TOL:
            bad.append((m, "waypoint deviation", dq))
            continue
        if ref["cc_margin"][m] <= CONTACT_MARGIN + LEVER * dq + 1e-6:
            stats["ambiguous_cc"] += 1
            continue
        if int(ref["status"][m]) != int(g["status"][m]) or \
                int(ref["first_fail"][m]) != int(g["first_fail"][m]):
            bad.append((m, "collision verdict", int(ref["status"][m]), int(g["status"][m]),
                        int(ref["first_fail"][m]), int(g["first_fail"][m]),
                        float(ref["cc_margin"][m])))
            continue
        stats["exact"] += robust
    return stats, bad
