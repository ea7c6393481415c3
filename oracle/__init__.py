"""ctypes loader for the FP64 CPU oracle (oracle/cprrtc_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the benchmark's
CPU legs (the cpu_baseline figure and the reference arm), never by the library. It shares
no code with the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cprrtc_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

VALID, PROJ_FAIL, COLLISION = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-ffp-contract=off keeps rounding identical on x86 and
    Arm). Returns the library path."""
    if not force and os.path.exists(_LIB_PATH) and \
            os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                               os.path.getmtime(_SRC[:-1] + "h")):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
                           "-o", tmp, _SRC, "-lm", "-lpthread"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Robot(C.Structure):
    _fields_ = [("dof", C.c_int), ("joints", C.POINTER(C.c_double)),
                ("ee", C.POINTER(C.c_double)), ("n_spheres", C.c_int),
                ("spheres", C.POINTER(C.c_double)), ("self_pairs", C.POINTER(C.c_ubyte))]


class _Scene(C.Structure):
    _fields_ = [("n_sph", C.c_int), ("sph", C.POINTER(C.c_double)),
                ("n_box", C.c_int), ("box", C.POINTER(C.c_double)),
                ("n_cap", C.c_int), ("cap", C.POINTER(C.c_double))]


class _Constraint(C.Structure):
    _fields_ = [("type", C.c_int), ("target", C.c_double), ("tol_task", C.c_double),
                ("c_sm", C.c_double), ("tau_floor", C.c_double), ("tol_sm", C.c_double),
                ("alpha", C.c_double), ("lam", C.c_double), ("max_iters", C.c_int),
                ("line_y", C.c_double), ("yaw", C.c_double)]


class _PlanParams(C.Structure):
    _fields_ = [("range", C.c_double), ("W", C.c_int), ("max_rounds", C.c_int),
                ("n_workers", C.c_int), ("max_nodes", C.c_int), ("max_connect", C.c_int),
                ("seed", C.c_uint32), ("first_problem", C.c_uint32), ("sequential", C.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _lib.orc_project_motion.restype = C.c_int
            _lib.orc_project_config.restype = C.c_int
            _lib.orc_project_motion_sequential.restype = C.c_int
            _lib.orc_task.restype = C.c_int
            _lib.orc_validate.restype = C.c_int
            _lib.orc_plan.restype = C.c_int
            _lib.orc_mlp_param_count.restype = C.c_long
            _lib.orc_mlp_loss_grad.restype = C.c_double
            for f in ("orc_clear_sphere", "orc_clear_box", "orc_clear_capsule",
                      "orc_config_clearance"):
                getattr(_lib, f).restype = C.c_double
    return _lib


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class Oracle:
    """Holds one robot, scene and constraint (numpy float64 copies) for oracle calls."""

    def __init__(self, robot, scene=None, constraint=None, self_pairs=None):
        """self_pairs: optional [(dof+1)][(dof+1)] 0/1 matrix of frame pairs whose spheres are
        tested against each other (self-collision)."""
        self._keep = []
        j, ee, sp = _d(robot.joints), _d(robot.ee), _d(robot.spheres)
        self._keep += [j, ee, sp]
        self.dof = robot.dof
        if self_pairs is None:
            sp_ptr = None
        else:
            pm = np.ascontiguousarray(np.asarray(self_pairs) != 0, np.uint8)
            assert pm.shape == (robot.dof + 1, robot.dof + 1)
            self._keep.append(pm)
            sp_ptr = pm.ctypes.data_as(C.POINTER(C.c_ubyte))
        self.rb = _Robot(robot.dof, _p(j), _p(ee), len(sp), _p(sp), sp_ptr)
        self.set_scene(scene)
        self.set_constraint(constraint)

    def set_scene(self, scene):
        if scene is None:
            arrs = [np.zeros((0, 4)), np.zeros((0, 15)), np.zeros((0, 7))]
        else:
            arrs = [_d(scene.sph).reshape(-1, 4), _d(scene.box).reshape(-1, 15),
                    _d(scene.cap).reshape(-1, 7)]
        arrs = [a if a.size else np.zeros((1, a.shape[1])) for a in arrs]
        self._scene_keep = arrs
        n = [0, 0, 0] if scene is None else [len(scene.sph), len(scene.box), len(scene.cap)]
        self.sc = _Scene(n[0], _p(arrs[0]), n[1], _p(arrs[1]), n[2], _p(arrs[2]))

    def set_constraint(self, c):
        if c is None:
            self.c = _Constraint(0, 0.0, 1e-4, 2.0, 1e-3, 1e-4, 1.0, 1e-3, 20, 0.0, 0.0)
        else:
            self.c = _Constraint(c.type, c.target, c.tol_task, c.c_sm, c.tau_floor, c.tol_sm,
                                 c.alpha, c.lam, c.max_iters, getattr(c, "line_y", 0.0),
                                 getattr(c, "yaw", 0.0))

    # ---- kinematics ----
    def fk(self, q) -> np.ndarray:
        q = _d(q)
        out = np.zeros((self.dof + 2, 4, 4))
        lib().orc_fk(C.byref(self.rb), _p(q), _p(out))
        return out

    def jacobian(self, q) -> np.ndarray:
        q = _d(q)
        out = np.zeros((6, self.dof))
        lib().orc_jacobian(C.byref(self.rb), _p(q), _p(out))
        return out

    def sphere_centres(self, q) -> np.ndarray:
        q = _d(q)
        out = np.zeros((self.rb.n_spheres, 3))
        lib().orc_sphere_centres(C.byref(self.rb), _p(q), _p(out))
        return out

    def task(self, q):
        q = _d(q)
        e = np.zeros(6)
        J = np.zeros((6, self.dof))
        m = lib().orc_task(C.byref(self.rb), C.byref(self.c), _p(q), _p(e), _p(J))
        return e[:m].copy(), J.reshape(-1)[: m * self.dof].reshape(m, self.dof).copy()

    @staticmethod
    def damped_step(J, e, lam) -> np.ndarray:
        J, e = _d(J), _d(e)
        m, n = J.shape
        g = np.zeros(n)
        lib().orc_damped_step(_p(J), _p(e), m, n, C.c_double(lam), _p(g))
        return g

    # ---- Algorithm 1 ----
    def project_motion(self, xi_init, tau, trace=False):
        xi_init = _d(xi_init)
        W = xi_init.shape[0]
        out = np.zeros_like(xi_init)
        it, ff = C.c_int(), C.c_int()
        res, mg = C.c_double(), C.c_double()
        tr = np.zeros(max(self.c.max_iters, 1), dtype=np.int32)
        ok = lib().orc_project_motion(C.byref(self.rb), C.byref(self.c), _p(xi_init), W,
                                      C.c_double(tau), _p(out), C.byref(it), C.byref(ff),
                                      C.byref(res), C.byref(mg),
                                      tr.ctypes.data_as(C.POINTER(C.c_int)))
        r = dict(ok=bool(ok), xi=out, iters=it.value, first_fail=ff.value, resid=res.value,
                 margin=mg.value)
        if trace:
            r["prog_trace"] = tr[: it.value].copy()
        return r

    def project_config(self, q, max_iters=None):
        q = _d(q)
        out = np.zeros_like(q)
        it, res = C.c_int(), C.c_double()
        mi = self.c.max_iters if max_iters is None else max_iters
        ok = lib().orc_project_config(C.byref(self.rb), C.byref(self.c), _p(q), mi, _p(out),
                                      C.byref(it), C.byref(res))
        return bool(ok), out, it.value, res.value

    def project_configs(self, q, max_iters=None, n_threads=1):
        """orc_project_config over a batch [n][dof] (FP32 inputs), threaded."""
        qs = np.ascontiguousarray(q, dtype=np.float32)
        n = qs.shape[0]
        out = np.zeros((n, self.dof))
        ok = np.zeros(n, dtype=np.int32)
        res = np.zeros(n)
        mi = self.c.max_iters if max_iters is None else max_iters
        lib().orc_project_configs(C.byref(self.rb), C.byref(self.c),
                                  qs.ctypes.data_as(C.POINTER(C.c_float)), n, mi, n_threads,
                                  _p(out), ok.ctypes.data_as(C.POINTER(C.c_int)), _p(res))
        return ok.astype(bool), out, res

    def project_motion_sequential(self, xi_init, tau):
        xi_init = _d(xi_init)
        out = np.zeros_like(xi_init)
        ff, tot = C.c_int(), C.c_int()
        ok = lib().orc_project_motion_sequential(C.byref(self.rb), C.byref(self.c),
                                                 _p(xi_init), xi_init.shape[0],
                                                 C.c_double(tau), _p(out), C.byref(ff),
                                                 C.byref(tot))
        return bool(ok), out, ff.value, tot.value

    # ---- collision ----
    @staticmethod
    def clear_sphere(p, r, o):
        return lib().orc_clear_sphere(_p(_d(p)), C.c_double(r), _p(_d(o)))

    @staticmethod
    def clear_box(p, r, b):
        return lib().orc_clear_box(_p(_d(p)), C.c_double(r), _p(_d(b)))

    @staticmethod
    def clear_capsule(p, r, cp):
        return lib().orc_clear_capsule(_p(_d(p)), C.c_double(r), _p(_d(cp)))

    def config_clearance(self, q):
        return lib().orc_config_clearance(C.byref(self.rb), C.byref(self.sc), _p(_d(q)))

    # ---- validation ----
    def validate(self, q_start, q_end, W, cc_skip_first=False, n_threads=1):
        qs = np.ascontiguousarray(q_start, dtype=np.float32)
        qe = np.ascontiguousarray(q_end, dtype=np.float32)
        n = qs.shape[0]
        out_q = np.zeros((n, W, self.dof))
        ints = [np.zeros(n, dtype=np.int32) for _ in range(3)]
        dbl = [np.zeros(n) for _ in range(3)]
        ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int))  # noqa: E731
        fp = lambda a: a.ctypes.data_as(C.POINTER(C.c_float))  # noqa: E731
        rc = lib().orc_validate(C.byref(self.rb), C.byref(self.sc), C.byref(self.c), fp(qs),
                                fp(qe), n, W, int(cc_skip_first), n_threads, _p(out_q),
                                ip(ints[0]), ip(ints[1]), ip(ints[2]), _p(dbl[0]), _p(dbl[1]),
                                _p(dbl[2]))
        if rc != 0:
            raise ValueError("orc_validate rejected its arguments")
        return dict(q=out_q, status=ints[0], first_fail=ints[1], iters=ints[2], resid=dbl[0],
                    proj_margin=dbl[1], cc_margin=dbl[2])

    def check_segment(self, xi, tau):
        """(max task error, max step excess over tau, min clearance) of a given segment."""
        xi = _d(xi)
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        lib().orc_check_segment(C.byref(self.rb), C.byref(self.sc), C.byref(self.c), _p(xi),
                                xi.shape[0], C.c_double(tau), C.byref(a), C.byref(b), C.byref(c))
        return a.value, b.value, c.value

    # ---- planner ----
    def plan(self, start, goal, range_=0.3, W=32, max_rounds=200, n_workers=8,
             max_nodes=4096, max_connect=64, seed=1, max_path=512, n_threads=1,
             first_problem=0, sequential=False):
        """Plans each problem; problem p draws its samples with Philox problem index
        first_problem + p (R19), so one problem of a batch can be planned alone. With
        sequential, motions are projected by the naive baseline's sequential projection
        (R27) instead of Alg. 1."""
        s = np.ascontiguousarray(start, dtype=np.float32)
        g = np.ascontiguousarray(goal, dtype=np.float32)
        n = s.shape[0]
        pp = _PlanParams(range_, W, max_rounds, n_workers, max_nodes, max_connect, seed,
                         first_problem, int(bool(sequential)))
        path_len = np.zeros(n, dtype=np.int32)
        path = np.zeros((n, max_path, self.dof))
        rounds = np.zeros(n, dtype=np.int32)
        wp = np.zeros(n, dtype=np.int64)
        lib().orc_plan(C.byref(self.rb), C.byref(self.sc), C.byref(self.c),
                       s.ctypes.data_as(C.POINTER(C.c_float)),
                       g.ctypes.data_as(C.POINTER(C.c_float)), n, C.byref(pp), max_path,
                       n_threads, path_len.ctypes.data_as(C.POINTER(C.c_int)), _p(path),
                       rounds.ctypes.data_as(C.POINTER(C.c_int)),
                       wp.ctypes.data_as(C.POINTER(C.c_longlong)))
        return dict(path_len=path_len, path=path, rounds=rounds, waypoints=wp)


def mlp_param_count(dof: int, H: int = 256) -> int:
    return int(lib().orc_mlp_param_count(dof, H))


def mlp_forward(params, q, dof: int, H: int = 256):
    """FP64 corrections f(q) [rows][dof] of the warm-start network (compact layout)."""
    p, q = _d(params), _d(q)
    out = np.zeros((q.shape[0], dof))
    lib().orc_mlp_forward(dof, H, _p(p), _p(q), q.shape[0], _p(out))
    return out


def mlp_loss_grad(params, q, t, dof: int, H: int = 256, n_threads: int = 1, grad=True):
    """(loss, gradient) of (1/rows) sum 0.5 |f(q) - (t - q)|^2, FP64."""
    p, q, t = _d(params), _d(q), _d(t)
    g = np.zeros(p.size) if grad else None
    loss = lib().orc_mlp_loss_grad(dof, H, _p(p), _p(q), _p(t), q.shape[0], n_threads,
                                   _p(g) if grad else None)
    return float(loss), g


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def tau_step(c, q0, q1, W):
    """Step threshold of a motion (same reading as the oracle's validate)."""
    span = float(np.max(np.abs(np.asarray(q1, np.float64) - np.asarray(q0, np.float64))))
    return max(c.c_sm * span / (W - 1), c.tau_floor)


def interpolate(q0, q1, W) -> np.ndarray:
    q0, q1 = np.asarray(q0, np.float64), np.asarray(q1, np.float64)
    t = np.arange(W, dtype=np.float64)[:, None] / (W - 1)
    return q0[None, :] + t * (q1 - q0)[None, :]
