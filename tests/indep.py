"""Test-side kinematics written independently of the oracle, from scipy rotation primitives.

Used only to pin the oracle: a DH chain composed from scipy's elementary rotations, the
product-of-exponentials form, and Euler angles from scipy.
"""
import numpy as np
from scipy.linalg import expm
from scipy.spatial.transform import Rotation as Rot


def _rot(axis, ang):
    T = np.eye(4)
    T[:3, :3] = Rot.from_euler(axis, ang).as_matrix()
    return T


def _trans(x=0.0, y=0.0, z=0.0):
    T = np.eye(4)
    T[:3, 3] = [x, y, z]
    return T


def fk_frames(joints, ee, q):
    """Frames 0..dof and the EE, each Rz(theta) Tz(d) Tx(a) Rx(alpha) from scipy pieces."""
    T = np.eye(4)
    out = [T.copy()]
    for k, (typ, d, a, alpha, th0, lo, hi) in enumerate(joints):
        theta = th0 + (q[k] if int(typ) == 0 else 0.0)
        dd = d + (q[k] if int(typ) == 1 else 0.0)
        T = T @ _rot("z", theta) @ _trans(z=dd) @ _trans(x=a) @ _rot("x", alpha)
        out.append(T.copy())
    out.append(T @ _trans(*ee))
    return np.array(out)


def _hat(w):
    return np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])


def fk_poe(joints, ee, q):
    """EE pose by the product of exponentials with screw axes read at q = 0."""
    home = fk_frames(joints, ee, np.zeros(len(joints)))
    T = np.eye(4)
    for k, jt in enumerate(joints):
        z = home[k][:3, 2]
        p = home[k][:3, 3]
        S = np.zeros((4, 4))
        if int(jt[0]) == 0:
            S[:3, :3] = _hat(z)
            S[:3, 3] = -np.cross(z, p)
        else:
            S[:3, 3] = z
        T = T @ expm(S * q[k])
    return T @ home[-1]


def roll_pitch(R):
    yaw, pitch, roll = Rot.from_matrix(R).as_euler("ZYX")
    return np.array([roll, pitch])


def task_error(joints, ee, q, ctype, target=0.0, line_y=0.0, yaw=0.0):
    """The task errors of every constraint type from scipy's Euler angles: roll-pitch,
    z-plane, line {y = line_y, z = target}, and the fixed orientation (roll, pitch, yaw
    wrapped into (-pi, pi]) with the plane or the line."""
    F = fk_frames(joints, ee, q)[-1]
    if ctype == 1:
        return roll_pitch(F[:3, :3])
    if ctype == 2:
        return np.array([F[2, 3] - target])
    if ctype == 3:
        return np.array([F[1, 3] - line_y, F[2, 3] - target])
    if ctype in (4, 5):
        yaw_, _, _ = Rot.from_matrix(F[:3, :3]).as_euler("ZYX")
        dy = (yaw_ - yaw + np.pi) % (2 * np.pi) - np.pi
        if dy <= -np.pi:
            dy += 2 * np.pi
        pos = [F[2, 3] - target] if ctype == 4 else [F[1, 3] - line_y, F[2, 3] - target]
        return np.concatenate([roll_pitch(F[:3, :3]), [dy], pos])
    return np.zeros(0)


def fd_jacobian(f, q, h=1e-6):
    q = np.asarray(q, np.float64)
    f0 = np.asarray(f(q))
    J = np.zeros((f0.size, q.size))
    for k in range(q.size):
        dq = np.zeros_like(q)
        dq[k] = h
        J[:, k] = (np.asarray(f(q + dq)) - np.asarray(f(q - dq))) / (2 * h)
    return J


def sphere_centres(joints, ee, spheres, q):
    F = fk_frames(joints, ee, q)
    out = []
    for f, x, y, z, r in spheres:
        T = F[int(f)]
        out.append(T[:3, :3] @ np.array([x, y, z]) + T[:3, 3])
    return np.array(out)
