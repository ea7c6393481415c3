"""Thin ctypes binding of libcprrtc.so (include/cprrtc.h): argument marshalling only.

Every function of the C ABI is exposed under its own name; `Context` wraps a context
handle. Arrays may be numpy arrays (host memory) or CUDA torch tensors (device memory);
all computation happens in the library's CUDA kernels. If the library is missing this
module raises on first use: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import synth

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libcprrtc.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "cprrtc.h")

OK = 0
E_INVALID_ARG, E_NOT_CONFIGURED, E_CUDA, E_OOM, E_CAPACITY, E_TIMEOUT, E_UNSUPPORTED = \
    -1, -2, -3, -4, -5, -6, -7
MOTION_VALID, MOTION_PROJ_FAIL, MOTION_COLLISION = 0, 1, 2
MLP_BF16, MLP_FP32 = 0, 1
MAX_DOF, MAX_W, MAX_SPHERES = 8, 64, 256

JOINT_DT = np.dtype([("type", "<i4"), ("d", "<f8"), ("a", "<f8"), ("alpha", "<f8"),
                     ("theta0", "<f8"), ("lo", "<f8"), ("hi", "<f8")], align=True)
SPHERE_DT = np.dtype([("frame", "<i4"), ("x", "<f8"), ("y", "<f8"), ("z", "<f8"),
                      ("r", "<f8")], align=True)
OBS_SPHERE_DT = np.dtype([("x", "<f8"), ("y", "<f8"), ("z", "<f8"), ("r", "<f8")], align=True)
OBS_BOX_DT = np.dtype([("c", "<f8", 3), ("h", "<f8", 3), ("R", "<f8", 9)], align=True)
OBS_CAPSULE_DT = np.dtype([("p0", "<f8", 3), ("p1", "<f8", 3), ("r", "<f8")], align=True)


class cprrtc_constraint(C.Structure):
    _fields_ = [("type", C.c_int), ("target", C.c_double), ("tol_task", C.c_double),
                ("c_sm", C.c_double), ("tau_floor", C.c_double), ("tol_sm", C.c_double),
                ("alpha", C.c_double), ("lambda_", C.c_double), ("max_iters", C.c_int),
                ("line_y", C.c_double), ("yaw", C.c_double)]


class cprrtc_plan_params(C.Structure):
    _fields_ = [("range", C.c_double), ("W", C.c_int), ("max_rounds", C.c_int),
                ("workers", C.c_int), ("max_nodes", C.c_int), ("max_connect", C.c_int),
                ("max_path", C.c_int), ("seed", C.c_uint32), ("use_scene_batch", C.c_int),
                ("time_budget_ms", C.c_double)]


class cprrtc_robot_desc(C.Structure):
    _fields_ = [("joints", C.c_void_p), ("dof", C.c_int), ("spheres", C.c_void_p),
                ("n_spheres", C.c_int), ("ee", C.c_double * 3)]


class cprrtc_problem(C.Structure):
    _fields_ = [("robot", C.c_int), ("constraint", C.c_int), ("scene", C.c_int), ("W", C.c_int)]


BATCH_CLASSES = 6


class cprrtc_tuning(C.Structure):
    _fields_ = [("ctas_per_sm", C.c_int * BATCH_CLASSES),
                ("stage_obstacles", C.c_int * BATCH_CLASSES),
                ("warps_per_motion", C.c_int * BATCH_CLASSES),
                ("pair_problems", C.c_int * BATCH_CLASSES)]

    def as_dict(self):
        return {"ctas_per_sm": list(self.ctas_per_sm),
                "stage_obstacles": list(self.stage_obstacles),
                "warps_per_motion": list(self.warps_per_motion),
                "pair_problems": list(self.pair_problems)}


def default_tuning(warps_per_motion: int = 1, pair_problems: int = 0) -> "cprrtc_tuning":
    """The library's launch shapes when no tuning is given or tuned: as many CTAs per SM as
    fit, obstacles staged when they fit, `warps_per_motion` warps per motion (1; 2: every
    class on warp pairs) and `pair_problems` of each class's heaviest problems on warp pairs
    (0)."""
    t = cprrtc_tuning()
    for c in range(BATCH_CLASSES):
        t.ctas_per_sm[c] = 0
        t.stage_obstacles[c] = 1
        t.warps_per_motion[c] = warps_per_motion
        t.pair_problems[c] = pair_problems
    return t


class CprrtcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"cprrtc error {code}: {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()

_SIGS = {
    "cprrtc_create": [C.POINTER(C.c_void_p), C.c_int, C.c_void_p],
    "cprrtc_destroy": [C.c_void_p],
    "cprrtc_set_stream": [C.c_void_p, C.c_void_p],
    "cprrtc_last_error": [C.c_void_p],
    "cprrtc_set_robot": [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p],
    "cprrtc_set_obstacles": [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p,
                             C.c_int],
    "cprrtc_set_constraint": [C.c_void_p, C.POINTER(cprrtc_constraint)],
    "cprrtc_validate": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p,
                        C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "cprrtc_project_configs": [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p,
                               C.c_void_p, C.c_void_p],
    "cprrtc_set_scene_batch": [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.c_void_p, C.c_void_p, C.c_void_p],
    "cprrtc_plan": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                    C.POINTER(cprrtc_plan_params), C.c_void_p, C.c_void_p, C.c_void_p,
                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "cprrtc_plan_static": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                           C.POINTER(cprrtc_plan_params), C.c_void_p, C.c_void_p, C.c_void_p,
                           C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "cprrtc_set_robot_table": [C.c_void_p, C.c_void_p, C.c_int],
    "cprrtc_set_constraint_table": [C.c_void_p, C.c_void_p, C.c_int],
    "cprrtc_plan_batch": [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                          C.POINTER(cprrtc_plan_params), C.c_void_p, C.c_void_p, C.c_void_p,
                          C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "cprrtc_autotune_batch": [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                              C.POINTER(cprrtc_plan_params), C.c_int, C.c_void_p],
    "cprrtc_batch_capture": [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                             C.POINTER(cprrtc_plan_params), C.c_void_p, C.c_void_p, C.c_void_p,
                             C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "cprrtc_batch_replay": [C.c_void_p],
    "cprrtc_batch_spans": [C.c_void_p, C.c_void_p, C.c_int],
    "cprrtc_philox": [C.c_void_p, C.c_uint32, C.c_uint32, C.c_void_p, C.c_int, C.c_void_p],
    "cprrtc_set_cc_mode": [C.c_void_p, C.c_int, C.c_double],
    "cprrtc_cc_stats": [C.c_void_p, C.POINTER(C.c_double), C.c_void_p, C.c_int],
    "cprrtc_mlp_param_count": [C.c_int],
    "cprrtc_mlp_init": [C.c_void_p, C.c_uint64],
    "cprrtc_mlp_set_precision": [C.c_void_p, C.c_int],
    "cprrtc_set_wait_limit": [C.c_void_p, C.c_double],
    "cprrtc_set_plan_warm_start": [C.c_void_p, C.c_int],
    "cprrtc_set_plan_slicing": [C.c_void_p, C.c_int, C.c_int],
    "cprrtc_set_table_self_collision": [C.c_void_p, C.c_int, C.c_void_p, C.c_int],
    "cprrtc_batch_adopt_network": [C.c_void_p, C.c_int, C.c_int],
    "cprrtc_mlp_set_params": [C.c_void_p, C.c_void_p, C.c_int64],
    "cprrtc_mlp_get_params": [C.c_void_p, C.c_void_p, C.c_int64],
    "cprrtc_mlp_save": [C.c_void_p, C.c_char_p],
    "cprrtc_mlp_load": [C.c_void_p, C.c_char_p],
    "cprrtc_mlp_grad": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p],
    "cprrtc_mlp_train": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                         C.c_float, C.c_uint64, C.c_void_p],
    "cprrtc_mlp_infer": [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p],
    "cprrtc_validate_ws": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                           C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                           C.c_void_p],
    "cprrtc_set_timing": [C.c_void_p, C.c_int],
    "cprrtc_work_counters": [C.c_void_p, C.c_void_p, C.c_int],
    "cprrtc_kernel_time": [C.c_void_p, C.c_char_p, C.POINTER(C.c_double),
                           C.POINTER(C.c_longlong)],
    "cprrtc_reset_timing": [C.c_void_p],
    "cprrtc_measure_fp32_peak": [C.c_void_p, C.c_void_p],
    "cprrtc_set_early_exit": [C.c_void_p, C.c_int],
    "cprrtc_set_projection": [C.c_void_p, C.c_int],
    "cprrtc_set_self_collision": [C.c_void_p, C.c_void_p, C.c_int],
}


def header_symbols() -> list:
    """Function names declared in include/cprrtc.h."""
    import re
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|int64_t|const char\*)\s+(cprrtc_\w+)\s*\(", text,
                                 re.M)))


def lib():
    """Loads libcprrtc.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: build it with "
                                  "paper_2505_06791_gb300.build.build()")
            L = C.CDLL(LIB_PATH)
            for name, args in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = {"cprrtc_last_error": C.c_char_p,
                              "cprrtc_mlp_param_count": C.c_int64}.get(name, C.c_int)
            _lib = L
    return _lib


def _need(x, dtype, what="array"):
    """x (numpy array or torch tensor, or None) must hold `dtype` elements ('float32', 'int32',
    'uint8', 'int64'): the library reads the bytes as that type, so a float64 array would be
    misread, not converted."""
    if x is None:
        return x
    name = str(x.dtype).replace("torch.", "")
    if name != dtype:
        raise TypeError(f"{what} must be {dtype}, got {name}")
    return x


def _ptr(x):
    """Address of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported array type {type(x)}")


def _is_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and x.is_cuda


def joints_array(robot) -> np.ndarray:
    a = np.zeros(robot.dof, JOINT_DT)
    j = np.asarray(robot.joints, np.float64)
    a["type"] = j[:, 0].astype(np.int32)
    for i, f in enumerate(["d", "a", "alpha", "theta0", "lo", "hi"]):
        a[f] = j[:, i + 1]
    return a


def spheres_array(robot) -> np.ndarray:
    s = np.asarray(robot.spheres, np.float64)
    a = np.zeros(len(s), SPHERE_DT)
    a["frame"] = s[:, 0].astype(np.int32)
    a["x"], a["y"], a["z"], a["r"] = s[:, 1], s[:, 2], s[:, 3], s[:, 4]
    return a


def scene_arrays(scene):
    sph = np.zeros(len(scene.sph), OBS_SPHERE_DT)
    if len(scene.sph):
        s = np.asarray(scene.sph, np.float64)
        sph["x"], sph["y"], sph["z"], sph["r"] = s[:, 0], s[:, 1], s[:, 2], s[:, 3]
    box = np.zeros(len(scene.box), OBS_BOX_DT)
    if len(scene.box):
        b = np.asarray(scene.box, np.float64)
        box["c"], box["h"], box["R"] = b[:, 0:3], b[:, 3:6], b[:, 6:15]
    cap = np.zeros(len(scene.cap), OBS_CAPSULE_DT)
    if len(scene.cap):
        c = np.asarray(scene.cap, np.float64)
        cap["p0"], cap["p1"], cap["r"] = c[:, 0:3], c[:, 3:6], c[:, 6]
    return sph, box, cap


def constraint_struct(c) -> cprrtc_constraint:
    return cprrtc_constraint(c.type, c.target, c.tol_task, c.c_sm, c.tau_floor, c.tol_sm,
                             c.alpha, c.lam, c.max_iters, getattr(c, "line_y", 0.0),
                             getattr(c, "yaw", 0.0))


class Context:
    """One library context (device, stream, robot, obstacles, constraint)."""

    def __init__(self, device: int = 0, stream=None):
        self._L = lib()
        h = C.c_void_p()
        rc = self._L.cprrtc_create(C.byref(h), device, stream)
        if rc != OK:
            raise CprrtcError(rc, "cprrtc_create failed")
        self.h = h
        self.dof = None

    def _check(self, rc):
        if rc != OK:
            raise CprrtcError(rc, self._L.cprrtc_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            self._L.cprrtc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t integer or None."""
        raw = getattr(stream, "cuda_stream", stream)
        self._check(self._L.cprrtc_set_stream(self.h, raw))

    def set_robot(self, robot):
        j = joints_array(robot)
        s = spheres_array(robot)
        ee = np.ascontiguousarray(robot.ee, np.float64)
        self._check(self._L.cprrtc_set_robot(self.h, j.ctypes.data, robot.dof, s.ctypes.data,
                                             len(s), ee.ctypes.data))
        self.dof = robot.dof

    def set_obstacles(self, scene):
        sph, box, cap = scene_arrays(scene)
        self._check(self._L.cprrtc_set_obstacles(
            self.h, sph.ctypes.data if len(sph) else None, len(sph),
            box.ctypes.data if len(box) else None, len(box),
            cap.ctypes.data if len(cap) else None, len(cap)))

    def set_constraint(self, c):
        cs = constraint_struct(c)
        self._check(self._L.cprrtc_set_constraint(self.h, C.byref(cs)))

    def set_timing(self, on: bool):
        self._check(self._L.cprrtc_set_timing(self.h, int(on)))

    def kernel_time(self, name: str):
        ms, n = C.c_double(), C.c_longlong()
        self._check(self._L.cprrtc_kernel_time(self.h, name.encode(), C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def work_counters(self, reset: bool = False) -> np.ndarray:
        """[Alg. 1 updates, collision-check chains, world transforms, sphere tests, box tests,
        capsule tests, warm-started extend motions tried, accepted] since the last reset."""
        out = np.zeros(8, np.int64)
        self._check(self._L.cprrtc_work_counters(self.h, out.ctypes.data, int(reset)))
        return out

    def batch_adopt_network(self, robot: int, constraint: int):
        """The context's network for the uneven batch's problems of (robot, constraint)."""
        self._check(self._L.cprrtc_batch_adopt_network(self.h, int(robot), int(constraint)))

    def set_table_self_collision(self, robot: int, frame_pairs=None):
        """Self-collision frame pairs of a robot of the batch's robot table (None: none)."""
        if frame_pairs is None:
            self._check(self._L.cprrtc_set_table_self_collision(self.h, int(robot), None, 0))
            return
        pm = np.ascontiguousarray(np.asarray(frame_pairs) != 0, np.uint8)
        self._check(self._L.cprrtc_set_table_self_collision(self.h, int(robot), pm.ctypes.data, pm.size))

    def set_self_collision(self, frame_pairs=None):
        """Self-collision test of cprrtc_validate and the planner: frame_pairs
        [(dof+1)][(dof+1)] 0/1 (None: off)."""
        if frame_pairs is None:
            self._check(self._L.cprrtc_set_self_collision(self.h, None, 0))
            return
        pm = np.ascontiguousarray(np.asarray(frame_pairs) != 0, np.uint8)
        self._check(self._L.cprrtc_set_self_collision(self.h, pm.ctypes.data, pm.size))

    def set_projection(self, sequential: bool):
        """Alg. 1 (default) or the naive baseline's sequential projection."""
        self._check(self._L.cprrtc_set_projection(self.h, int(bool(sequential))))

    def set_early_exit(self, enabled: bool):
        """Ablation switch of the early termination of collision checking (default on)."""
        self._check(self._L.cprrtc_set_early_exit(self.h, int(bool(enabled))))

    def measure_fp32_peak(self) -> float:
        """FP32 FMA throughput of this context's GPU in TFLOP/s (measured on the device)."""
        t = C.c_double()
        self._check(self._L.cprrtc_measure_fp32_peak(self.h, C.byref(t)))
        return t.value

    def reset_timing(self):
        self._check(self._L.cprrtc_reset_timing(self.h))

    def alloc_validate_outputs(self, n, W, like):
        """Output buffers matching `like` (CUDA tensor -> CUDA tensors, else numpy)."""
        dof = self.dof or int(like.shape[1])
        if _is_cuda(like):
            import torch
            dev = like.device
            return dict(q=torch.empty((n, W, dof), dtype=torch.float32, device=dev),
                        status=torch.empty(n, dtype=torch.uint8, device=dev),
                        first_fail=torch.empty(n, dtype=torch.int32, device=dev),
                        iters=torch.empty(n, dtype=torch.uint8, device=dev),
                        resid=torch.empty(n, dtype=torch.float32, device=dev))
        return dict(q=np.empty((n, W, dof), np.float32), status=np.empty(n, np.uint8),
                    first_fail=np.empty(n, np.int32), iters=np.empty(n, np.uint8),
                    resid=np.empty(n, np.float32))

    def validate(self, q_start, q_end, W: int, out=None, with_q: bool = True):
        """cprrtc_validate on n motions. Returns the output dict."""
        n = int(q_start.shape[0])
        if out is None:
            out = self.alloc_validate_outputs(n, W, q_start)
        self._check(cprrtc_validate(self.h, q_start, q_end, n, W,
                                    out["q"] if with_q else None, out["status"],
                                    out["first_fail"], out["iters"], out["resid"]))
        return out

    def validate_ws(self, q_start, q_end, W: int, refine_iters: int = 5, out=None,
                    with_q: bool = True):
        """cprrtc_validate_ws: validation with the learned warm start (adds out["warm"])."""
        n = int(q_start.shape[0])
        if out is None:
            out = self.alloc_validate_outputs(n, W, q_start)
        if "warm" not in out:
            if _is_cuda(q_start):
                import torch
                out["warm"] = torch.empty(n, dtype=torch.uint8, device=q_start.device)
            else:
                out["warm"] = np.empty(n, np.uint8)
        self._check(cprrtc_validate_ws(self.h, q_start, q_end, n, W, refine_iters,
                                       out["q"] if with_q else None, out["status"],
                                       out["first_fail"], out["iters"], out["resid"],
                                       out["warm"]))
        return out

    # -- collision checking in GEMM form --
    CC_EXACT, CC_GEMM_TF32, CC_GEMM_BF16 = 0, 1, 2

    def set_cc_mode(self, mode: int, guard: float = 0.005):
        self._check(self._L.cprrtc_set_cc_mode(self.h, int(mode), float(guard)))

    def cc_stats(self, reset: bool = False):
        """(error bound E in m^2, pairs rechecked exactly) of the GEMM-form check."""
        b = C.c_double()
        cnt = np.zeros(2, np.int64)
        self._check(self._L.cprrtc_cc_stats(self.h, C.byref(b), cnt.ctypes.data, int(reset)))
        return b.value, int(cnt[0])

    # -- learned warm start --
    def mlp_param_count(self, dof=None) -> int:
        return int(self._L.cprrtc_mlp_param_count(int(dof or self.dof)))

    def mlp_init(self, seed: int = 0):
        self._check(self._L.cprrtc_mlp_init(self.h, int(seed)))

    def set_plan_warm_start(self, refine_iters: int):
        """Planner's learned form: extend motions warm-started by the network (0: off)."""
        self._check(self._L.cprrtc_set_plan_warm_start(self.h, int(refine_iters)))

    def set_plan_slicing(self, first_slice: int, slice_rounds: int = 50):
        """cprrtc_set_plan_slicing: first_slice 0 plans each problem on one CTA in one stretch."""
        self._check(self._L.cprrtc_set_plan_slicing(self.h, int(first_slice), int(slice_rounds)))

    def set_wait_limit(self, seconds: float):
        """Limit of the tensor-core kernels' bounded waits (0: the default, 1 s)."""
        self._check(self._L.cprrtc_set_wait_limit(self.h, float(seconds)))

    def mlp_set_precision(self, fp32: bool):
        """FP32 checking mode (True) or the BF16 tensor-core arithmetic (False)."""
        self._check(self._L.cprrtc_mlp_set_precision(self.h, MLP_FP32 if fp32 else MLP_BF16))

    def mlp_set_params(self, params):
        p = np.ascontiguousarray(params, np.float32)
        self._check(self._L.cprrtc_mlp_set_params(self.h, p.ctypes.data, p.size))

    def mlp_get_params(self) -> np.ndarray:
        p = np.empty(self.mlp_param_count(), np.float32)
        self._check(self._L.cprrtc_mlp_get_params(self.h, p.ctypes.data, p.size))
        return p

    def mlp_save(self, path: str):
        self._check(self._L.cprrtc_mlp_save(self.h, os.fsencode(path)))

    def mlp_load(self, path: str):
        self._check(self._L.cprrtc_mlp_load(self.h, os.fsencode(path)))

    def mlp_grad(self, q, t):
        """(loss, gradient in the compact parameter layout) for pairs (q, t)."""
        g = np.empty(self.mlp_param_count(), np.float32)
        loss = np.zeros(1, np.float32)
        self._check(cprrtc_mlp_grad(self.h, q, t, int(q.shape[0]), g, loss))
        return float(loss[0]), g

    def mlp_train(self, q, t, batch: int, epochs: int, lr: float, seed: int = 0):
        """Minibatch Adam; returns the mean batch loss of each epoch."""
        losses = np.zeros(max(epochs, 1), np.float32)
        self._check(cprrtc_mlp_train(self.h, q, t, int(q.shape[0]), batch, epochs, lr, seed,
                                     losses))
        return losses[:epochs]

    def mlp_infer(self, q, out=None):
        if out is None:
            if _is_cuda(q):
                import torch
                out = torch.empty_like(q)
            else:
                out = np.empty_like(np.asarray(q, np.float32))
        self._check(cprrtc_mlp_infer(self.h, q, int(q.shape[0]), out))
        return out

    def set_scene_batch(self, scenes):
        """One obstacle set per planning problem (problem p uses scenes[p])."""
        parts = [scene_arrays(sc) for sc in scenes]
        arrs, offs = [], []
        for t, dt in enumerate((OBS_SPHERE_DT, OBS_BOX_DT, OBS_CAPSULE_DT)):
            counts = [len(pt[t]) for pt in parts]
            offs.append(np.concatenate([[0], np.cumsum(counts)]).astype(np.int32))
            a = np.concatenate([pt[t] for pt in parts]) if sum(counts) else np.zeros(1, dt)
            arrs.append(np.ascontiguousarray(a))
        self._check(self._L.cprrtc_set_scene_batch(
            self.h, len(scenes), arrs[0].ctypes.data, offs[0].ctypes.data, arrs[1].ctypes.data,
            offs[1].ctypes.data, arrs[2].ctypes.data, offs[2].ctypes.data))

    @staticmethod
    def plan_params(range_=0.3, W=32, max_rounds=200, workers=8, max_nodes=2048,
                    max_connect=32, max_path=512, seed=1, use_scene_batch=True, time_budget_ms=0.0):
        return cprrtc_plan_params(range_, W, max_rounds, workers, max_nodes, max_connect,
                                  max_path, seed, int(use_scene_batch), float(time_budget_ms))

    def alloc_plan_outputs(self, n, params, like, edges=True):
        dof, W, mp = self.dof, params.W, params.max_path
        if _is_cuda(like):
            import torch
            d = like.device
            out = dict(path_len=torch.empty(n, dtype=torch.int32, device=d),
                       path=torch.empty((n, mp, dof), dtype=torch.float32, device=d),
                       rounds=torch.empty(n, dtype=torch.int32, device=d),
                       waypoints=torch.empty(n, dtype=torch.int64, device=d),
                       plan_ms=torch.empty(n, dtype=torch.float32, device=d),
                       work=torch.empty((n, 2), dtype=torch.int64, device=d))
            out["path_edges"] = torch.empty((n, mp - 1, W, dof), dtype=torch.float32,
                                            device=d) if edges else None
            return out
        out = dict(path_len=np.empty(n, np.int32), path=np.empty((n, mp, dof), np.float32),
                   rounds=np.empty(n, np.int32), waypoints=np.empty(n, np.int64),
                   plan_ms=np.empty(n, np.float32), work=np.empty((n, 2), np.int64))
        out["path_edges"] = np.empty((n, mp - 1, W, dof), np.float32) if edges else None
        return out

    def plan(self, start, goal, params, out=None, edges=True):
        """cprrtc_plan on n problems; returns the output dict."""
        n = int(start.shape[0])
        if out is None:
            out = self.alloc_plan_outputs(n, params, start, edges)
        self._check(cprrtc_plan(self.h, start, goal, n, params, out["path_len"], out["path"],
                                out.get("path_edges"), out.get("rounds"), out.get("waypoints"),
                                out.get("plan_ms"), out.get("work")))
        return out

    # ---- batches of uneven problems ----
    def set_robot_table(self, robots):
        descs = (cprrtc_robot_desc * len(robots))()
        keep = []
        for i, rb in enumerate(robots):
            j, sp = joints_array(rb), spheres_array(rb)
            keep += [j, sp]
            descs[i].joints = j.ctypes.data
            descs[i].dof = rb.dof
            descs[i].spheres = sp.ctypes.data
            descs[i].n_spheres = len(sp)
            for k in range(3):
                descs[i].ee[k] = float(rb.ee[k])
        self._check(self._L.cprrtc_set_robot_table(self.h, C.addressof(descs), len(robots)))
        self.batch_dofs = [rb.dof for rb in robots]

    def set_constraint_table(self, constraints):
        arr = (cprrtc_constraint * len(constraints))(*[constraint_struct(c) for c in constraints])
        self._check(self._L.cprrtc_set_constraint_table(self.h, C.addressof(arr),
                                                        len(constraints)))

    @staticmethod
    def problems_array(problems):
        """problems: iterable of (robot, constraint, scene, W)."""
        problems = list(problems)
        arr = (cprrtc_problem * max(1, len(problems)))()
        for i, (r, c, sc, W) in enumerate(problems):
            arr[i].robot, arr[i].constraint, arr[i].scene, arr[i].W = r, c, sc, W
        return arr

    def alloc_batch_outputs(self, n, params, max_W, like, edges=False):
        mp = params.max_path
        if _is_cuda(like):
            import torch
            d = like.device
            out = dict(path_len=torch.empty(n, dtype=torch.int32, device=d),
                       path=torch.empty((n, mp, 8), dtype=torch.float32, device=d),
                       rounds=torch.empty(n, dtype=torch.int32, device=d),
                       waypoints=torch.empty(n, dtype=torch.int64, device=d),
                       plan_ms=torch.empty(n, dtype=torch.float32, device=d),
                       work=torch.empty((n, 2), dtype=torch.int64, device=d))
            out["path_edges"] = torch.empty((n, mp - 1, max_W, 8), dtype=torch.float32,
                                            device=d) if edges else None
            return out
        out = dict(path_len=np.empty(n, np.int32), path=np.empty((n, mp, 8), np.float32),
                   rounds=np.empty(n, np.int32), waypoints=np.empty(n, np.int64),
                   plan_ms=np.empty(n, np.float32), work=np.empty((n, 2), np.int64))
        out["path_edges"] = np.empty((n, mp - 1, max_W, 8), np.float32) if edges else None
        return out

    def plan_batch(self, problems, start, goal, params, tuning=None, out=None, edges=False):
        """problems: list of (robot, constraint, scene, W); start, goal: [n][8]."""
        probs = self.problems_array(problems)
        n = len(list(problems))
        max_W = max(p[3] for p in problems)
        if out is None:
            out = self.alloc_batch_outputs(n, params, max_W, start, edges)
        self._check(cprrtc_plan_batch(self.h, probs, n, start, goal, params, tuning,
                                      out["path_len"], out["path"], out.get("path_edges"),
                                      out.get("rounds"), out.get("waypoints"),
                                      out.get("plan_ms"), out.get("work")))
        return out

    def autotune_batch(self, problems, start, goal, params, trial_rounds=20):
        probs = self.problems_array(problems)
        t = cprrtc_tuning()
        self._check(cprrtc_autotune_batch(self.h, probs, len(list(problems)), start, goal, params,
                                          trial_rounds, t))
        return t

    def batch_capture(self, problems, start, goal, params, out, tuning=None):
        probs = self.problems_array(problems)
        self._check(cprrtc_batch_capture(self.h, probs, len(list(problems)), start, goal, params,
                                         tuning, out["path_len"], out["path"],
                                         out.get("path_edges"), out.get("rounds"),
                                         out.get("waypoints"), out.get("plan_ms"),
                                         out.get("work")))

    def batch_replay(self):
        self._check(cprrtc_batch_replay(self.h))

    def batch_spans(self, n: int):
        """[n][2] int64: each problem's start and end (GPU global-timer ns) in the last batch
        run on this context."""
        span = np.zeros((n, 2), np.int64)
        self._check(cprrtc_batch_spans(self.h, span, n))
        return span

    def philox(self, key0, key1, counters):
        c = np.ascontiguousarray(counters, dtype=np.uint32)
        out = np.empty_like(c)
        self._check(cprrtc_philox(self.h, key0, key1, c, len(c), out))
        return out

    def project_configs(self, q_in, max_iters: int, out=None):
        n = int(q_in.shape[0])
        if out is None:
            if _is_cuda(q_in):
                import torch
                out = dict(q=torch.empty_like(q_in),
                           ok=torch.empty(n, dtype=torch.uint8, device=q_in.device),
                           resid=torch.empty(n, dtype=torch.float32, device=q_in.device))
            else:
                out = dict(q=np.empty_like(np.asarray(q_in, np.float32)),
                           ok=np.empty(n, np.uint8), resid=np.empty(n, np.float32))
        self._check(cprrtc_project_configs(self.h, q_in, n, max_iters, out["q"], out["ok"],
                                           out["resid"]))
        return out


# ---- functions under the C names (pointer marshalling only) ----

def _plan_io(start, goal, path_len, path, path_edges, rounds, waypoints, plan_ms, work):
    for x, t, w in ((start, "float32", "start"), (goal, "float32", "goal"),
                    (path_len, "int32", "path_len"), (path, "float32", "path"),
                    (path_edges, "float32", "path_edges"), (rounds, "int32", "rounds"),
                    (waypoints, "int64", "waypoints"), (plan_ms, "float32", "plan_ms"),
                    (work, "int64", "work")):
        _need(x, t, w)


def cprrtc_plan(h, start, goal, n, params, path_len, path, path_edges, rounds, waypoints,
                plan_ms, work):
    _plan_io(start, goal, path_len, path, path_edges, rounds, waypoints, plan_ms, work)
    return lib().cprrtc_plan(h, _ptr(start), _ptr(goal), n, C.byref(params), _ptr(path_len),
                             _ptr(path), _ptr(path_edges), _ptr(rounds), _ptr(waypoints),
                             _ptr(plan_ms), _ptr(work))


def cprrtc_plan_static(h, start, goal, n, params, path_len, path, path_edges, rounds,
                       waypoints, plan_ms, work):
    _plan_io(start, goal, path_len, path, path_edges, rounds, waypoints, plan_ms, work)
    return lib().cprrtc_plan_static(h, _ptr(start), _ptr(goal), n, C.byref(params),
                                    _ptr(path_len), _ptr(path), _ptr(path_edges), _ptr(rounds),
                                    _ptr(waypoints), _ptr(plan_ms), _ptr(work))


def cprrtc_plan_batch(h, problems, n, start, goal, params, tuning, path_len, path, path_edges,
                      rounds, waypoints, plan_ms, work):
    _plan_io(start, goal, path_len, path, path_edges, rounds, waypoints, plan_ms, work)
    return lib().cprrtc_plan_batch(h, C.addressof(problems), n, _ptr(start), _ptr(goal),
                                   C.byref(params), C.addressof(tuning) if tuning else None,
                                   _ptr(path_len), _ptr(path), _ptr(path_edges), _ptr(rounds),
                                   _ptr(waypoints), _ptr(plan_ms), _ptr(work))


def cprrtc_autotune_batch(h, problems, n, start, goal, params, trial_rounds, out):
    _need(start, "float32", "start")
    _need(goal, "float32", "goal")
    return lib().cprrtc_autotune_batch(h, C.addressof(problems), n, _ptr(start), _ptr(goal),
                                       C.byref(params), trial_rounds,
                                       C.addressof(out) if out is not None else None)


def cprrtc_batch_capture(h, problems, n, start, goal, params, tuning, path_len, path, path_edges,
                         rounds, waypoints, plan_ms, work):
    _plan_io(start, goal, path_len, path, path_edges, rounds, waypoints, plan_ms, work)
    return lib().cprrtc_batch_capture(h, C.addressof(problems), n, _ptr(start), _ptr(goal),
                                      C.byref(params), C.addressof(tuning) if tuning else None,
                                      _ptr(path_len), _ptr(path), _ptr(path_edges), _ptr(rounds),
                                      _ptr(waypoints), _ptr(plan_ms), _ptr(work))


def cprrtc_batch_replay(h):
    return lib().cprrtc_batch_replay(h)


def cprrtc_batch_spans(h, span, n):
    _need(span, "int64", "span")
    return lib().cprrtc_batch_spans(h, _ptr(span), n)


def cprrtc_philox(h, key0, key1, counters, n, out):
    return lib().cprrtc_philox(h, key0, key1, _ptr(counters), n, _ptr(out))


def _validate_io(q_start, q_end, out_q, status, first_fail, iters, resid, warm_used=None):
    for x, t, w in ((q_start, "float32", "q_start"), (q_end, "float32", "q_end"),
                    (out_q, "float32", "out_q"), (status, "uint8", "status"),
                    (first_fail, "int32", "first_fail"), (iters, "uint8", "iters"),
                    (resid, "float32", "resid"), (warm_used, "uint8", "warm_used")):
        _need(x, t, w)


def cprrtc_validate(h, q_start, q_end, n, W, out_q, status, first_fail, iters, resid):
    _validate_io(q_start, q_end, out_q, status, first_fail, iters, resid)
    return lib().cprrtc_validate(h, _ptr(q_start), _ptr(q_end), n, W, _ptr(out_q),
                                 _ptr(status), _ptr(first_fail), _ptr(iters), _ptr(resid))


def cprrtc_validate_ws(h, q_start, q_end, n, W, refine_iters, out_q, status, first_fail, iters,
                       resid, warm_used):
    _validate_io(q_start, q_end, out_q, status, first_fail, iters, resid, warm_used)
    return lib().cprrtc_validate_ws(h, _ptr(q_start), _ptr(q_end), n, W, refine_iters,
                                    _ptr(out_q), _ptr(status), _ptr(first_fail), _ptr(iters),
                                    _ptr(resid), _ptr(warm_used))


def cprrtc_mlp_grad(h, q, t, rows, grads, loss):
    for x, w in ((q, "q"), (t, "t"), (grads, "grads"), (loss, "loss")):
        _need(x, "float32", w)
    return lib().cprrtc_mlp_grad(h, _ptr(q), _ptr(t), rows, _ptr(grads), _ptr(loss))


def cprrtc_mlp_train(h, q, t, n, batch, epochs, lr, seed, loss_per_epoch):
    for x, w in ((q, "q"), (t, "t"), (loss_per_epoch, "loss_per_epoch")):
        _need(x, "float32", w)
    return lib().cprrtc_mlp_train(h, _ptr(q), _ptr(t), n, batch, epochs, lr, seed,
                                  _ptr(loss_per_epoch))


def cprrtc_mlp_infer(h, q, rows, q_out):
    _need(q, "float32", "q")
    _need(q_out, "float32", "q_out")
    return lib().cprrtc_mlp_infer(h, _ptr(q), rows, _ptr(q_out))


def cprrtc_project_configs(h, q_in, n, max_iters, q_out, ok, resid):
    for x, t, w in ((q_in, "float32", "q_in"), (q_out, "float32", "q_out"), (ok, "uint8", "ok"),
                    (resid, "float32", "resid")):
        _need(x, t, w)
    return lib().cprrtc_project_configs(h, _ptr(q_in), n, max_iters, _ptr(q_out), _ptr(ok),
                                        _ptr(resid))


__all__ = ["Context", "CprrtcError", "lib", "header_symbols", "synth", "cprrtc_validate",
           "cprrtc_project_configs", "cprrtc_plan", "cprrtc_plan_static", "cprrtc_philox",
           "cprrtc_plan_batch", "cprrtc_autotune_batch", "cprrtc_batch_capture",
           "cprrtc_batch_replay", "cprrtc_batch_spans", "cprrtc_validate_ws", "cprrtc_mlp_grad", "cprrtc_mlp_train",
           "cprrtc_mlp_infer"]
