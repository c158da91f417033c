"""GPE in the rotating frame: the time-dependent trap, the energy E_{beta,omega} and the
lab-frame reconstruction (the oracle's side of Sec. 5.2 of Besse & Xing, arXiv:1603.05110).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it; it shares no code with
the CUDA library.

Sec. 5.2.1, eq. (GPE), (x1Ax), (GPE_Trans), (u1u): the rotation term omega L_z of the GPE
disappears in the coordinates (x~, y~) = A(t)^T (x, y), A(t) = [[cos wt, sin wt],
[-sin wt, cos wt]]; the trap becomes the time-dependent V_t(t, x~) = V(A(t) x~), and
u(t, x, y) = u~(t, A(t)^T (x, y)).  Everything here is written in the sign of eq. (Sch),
    i u_t + lap Lap u + V u + kappa |u|^2 u = 0,
so the GPE trap V = (gx^2 x^2 + gy^2 y^2)/2 enters as V_sch = -V (with lap = 1/2,
kappa = -beta).

Parity status: pinned by ``tests/test_oracle_gpe.py`` (closed forms of the rotated trap,
the angular momentum of vortex states, Q1 interpolation identities).
"""
import math

import numpy as np

from . import fem


def rotation(t, omega):
    """A(t) of eq. (x1Ax)."""
    c, s = math.cos(omega * t), math.sin(omega * t)
    return np.array([[c, s], [-s, c]])


def trap_potential(prob, t, gx, gy, omega):
    """V_t(t, x~) = V(A(t) x~) of eq. (u1u) at the nodes of ``prob``, in the sign of eq. (Sch):
    -(gx^2 x^2 + gy^2 y^2)/2 with (x, y) = A(t) (x~, y~)."""
    Xt, Yt = prob.grid()
    A = rotation(t, omega)
    x = A[0, 0] * Xt + A[0, 1] * Yt
    y = A[1, 0] * Xt + A[1, 1] * Yt
    return -0.5 * (gx * gx * x * x + gy * gy * y * y)


def step_potential(prob, n, gx, gy, omega, V_static=None):
    """W_n = (V_n + V_{n-1})/2 of eq. (CNS) for step n (t_n = n dt), plus an optional static
    part; the potential the n-th step solves with (eq. Sch sign, before division by lap)."""
    W = 0.5 * (trap_potential(prob, n * prob.dt, gx, gy, omega)
               + trap_potential(prob, (n - 1) * prob.dt, gx, gy, omega))
    return W if V_static is None else W + V_static


def _central(u, h, axis):
    """Central differences along ``axis``, one-sided (first order) at the two ends."""
    d = np.zeros_like(u)
    n = u.shape[axis]
    if n < 2:
        return d
    sl = [slice(None)] * u.ndim

    def at(i):
        s2 = list(sl)
        s2[axis] = i
        return tuple(s2)
    d[at(slice(1, n - 1))] = (u[at(slice(2, n))] - u[at(slice(0, n - 2))]) / (2.0 * h)
    d[at(0)] = (u[at(1)] - u[at(0)]) / h
    d[at(n - 1)] = (u[at(n - 1)] - u[at(n - 2)]) / h
    return d


def angular_momentum(prob, u):
    """<u, L_z u> with L_z = -i (x d_y - y d_x) (Sec. 5.2.1): nodal (trapezoid) quadrature and
    central differences, real part (L_z is symmetric; the boundary terms of a box are dropped).
    u has shape (ny+1, nx+1), x fastest; (x, y) are the node coordinates."""
    X, Y = prob.grid()
    ux = _central(u, prob.hx, axis=1)
    uy = _central(u, prob.hy, axis=0)
    w = fem.lumped_weights(prob.nx, prob.ny, prob.hx, prob.hy)
    Lu = -1j * (X * uy - Y * ux)
    return float(np.real(np.sum(w * np.conj(u) * Lu)))


def energy_lab(prob, u, V, omega, region=None):
    """The energy of eq. (GPE) as the Hamiltonian of the equation, in the sign of eq. (Sch):
        E = lap u^H S u - sum_i w_i V_i |u_i|^2 - (kappa/2) sum_i w_i |u_i|^4 - omega <u, L_z u>,
    for the GPE (lap = 1/2, V = -V_trap, kappa = -beta):
        E = int 1/2 |grad u|^2 + V_trap |u|^2 + beta/2 |u|^4 - omega u* L_z u.
    The printed E_{beta,omega} (Sec. 5.2.2) puts 1/2 in front of every term, which does not agree
    with the printed mu = E + beta/4 int |u|^4 nor with the equation; the Hamiltonian, whose
    variation is the equation and for which mu = E + beta/2 int |u|^4, is the reading taken.
    V: nodal potential (eq. Sch sign) of the instant the energy refers to."""
    from .nls import mono_region
    reg = region or mono_region(prob)
    uu = u.ravel()
    w = reg.w
    e = prob.lap * np.real(np.vdot(uu, reg.S @ uu))
    e -= np.sum(w * np.asarray(V).ravel() * np.abs(uu) ** 2)
    e -= 0.5 * prob.kappa * np.sum(w * np.abs(uu) ** 4)
    return float(e - omega * angular_momentum(prob, u))


def valid_zone(prob):
    """The square of Sec. 5.2.1 (after eq. u1u) that every rotated copy A(t) Omega covers."""
    r = math.sqrt(2.0)
    return prob.xl / r, prob.xr / r, prob.yb / r, prob.yu / r


def q1_interpolate(prob, u, xq, yq):
    """The Q1 (bilinear) interpolant of the nodal field u at the points (xq, yq) inside Omega."""
    fx = (np.asarray(xq) - prob.xl) / prob.hx
    fy = (np.asarray(yq) - prob.yb) / prob.hy
    ix = np.clip(np.floor(fx).astype(int), 0, prob.nx - 1)
    iy = np.clip(np.floor(fy).astype(int), 0, prob.ny - 1)
    sx = fx - ix
    sy = fy - iy
    return ((1 - sx) * (1 - sy) * u[iy, ix] + sx * (1 - sy) * u[iy, ix + 1]
            + (1 - sx) * sy * u[iy + 1, ix] + sx * sy * u[iy + 1, ix + 1])


def lab_frame(prob, u, t, omega, nx_out, ny_out):
    """u(t, x, y) = u~(t, A(t)^T (x, y)) (eq. u1u) on a uniform grid of (nx_out+1) x (ny_out+1)
    points over the valid zone, x fastest, by Q1 interpolation of the rotating-frame field u~."""
    x0, x1, y0, y1 = valid_zone(prob)
    x = x0 + (x1 - x0) * np.arange(nx_out + 1) / nx_out
    y = y0 + (y1 - y0) * np.arange(ny_out + 1) / ny_out
    X, Y = np.meshgrid(x, y, indexing="xy")
    A = rotation(t, omega)
    xt = A[0, 0] * X + A[1, 0] * Y          # A^T (x, y)
    yt = A[0, 1] * X + A[1, 1] * Y
    return q1_interpolate(prob, u, xt, yt)
