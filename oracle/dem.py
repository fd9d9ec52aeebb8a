"""Rigid-body update of the oracle (test infrastructure only), float64.

Sec. 2.3.1: m a = m g + sum F^c + F^e and d(I omega)/dt = sum T^c + T^e.
Reading A22 (the scheme is not given): semi-implicit Euler per substep of
length dt = 1 / n_sub, Euler's equations in the body frame, and the
orientation advanced by the exponential map of the body-frame angular
velocity; FP64.  Reading A14: the LBM carries no hydrostatic pressure, so the
buoyancy -rho0 V g is added explicitly: gravity force (m - rho0 V) g.
"""
import numpy as np

from .metaball import quat_to_matrix


def quat_mul(a, b):
    aw, ax, ay, az = a
    bw, bx, by, bz = b
    return np.array([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw])


def quat_exp_half(theta):
    """Unit quaternion of the rotation vector theta: (cos |t|/2, sin(|t|/2) t/|t|)."""
    t = float(np.sqrt(theta @ theta))
    if t == 0.0:
        return np.array([1.0, 0.0, 0.0, 0.0])
    s = np.sin(0.5 * t) / t
    return np.array([np.cos(0.5 * t), s * theta[0], s * theta[1], s * theta[2]])


def integrate(state, F, T, gravity, rho0=1.0, dt=1.0):
    """Advance one particle by one substep.

    state: dict with pos, quat (w,x,y,z), vel, omega (world frame), mass,
    volume, inertia (3x3, body frame, about the centroid).  F, T: total
    external force and torque (world frame, hydrodynamic + contact).
    Returns the new state dict.
    """
    m = state["mass"]
    Ib = np.asarray(state["inertia"], dtype=np.float64)
    g = np.asarray(gravity, dtype=np.float64)
    v = np.asarray(state["vel"], dtype=np.float64) + dt * (np.asarray(F) + (m - rho0 * state["volume"]) * g) / m
    R = quat_to_matrix(state["quat"])
    wb = R.T @ np.asarray(state["omega"], dtype=np.float64)
    Tb = R.T @ np.asarray(T, dtype=np.float64)
    wb = wb + dt * np.linalg.solve(Ib, Tb - np.cross(wb, Ib @ wb))
    qn = quat_mul(np.asarray(state["quat"], dtype=np.float64) /
                  np.linalg.norm(state["quat"]), quat_exp_half(wb * dt))
    qn = qn / np.linalg.norm(qn)
    w_world = quat_to_matrix(qn) @ wb
    x = np.asarray(state["pos"], dtype=np.float64) + dt * v
    out = dict(state)
    out.update(pos=x, quat=qn, vel=v, omega=w_world)
    return out
