"""Pins of the oracle's rotating-frame GPE helpers (Sec. 5.2.1, eq. x1Ax, GPE_Trans, u1u; no GPU).

* the time-dependent trap: equal to the lab trap at t = 0, independent of t for an isotropic
  trap, and with the roles of gx, gy exchanged after a quarter turn (closed forms);
* the angular momentum <u, L_z u> of the vortex states (x + i y)^m e^{-r^2/2}, which are
  eigenfunctions of L_z = -i d_theta with eigenvalue m: the ratio to the mass tends to m at
  second order in the mesh size; real states carry none;
* the energy of eq. (GPE): its rotation term is -omega <u, L_z u>, and without rotation it is lap
  times the NLS energy already pinned (mass/energy invariants of the midpoint scheme);
* the lab-frame reconstruction: Q1 interpolation reproduces bilinear functions exactly, so a
  bilinear rotating-frame field comes back exactly at t = 0 and after quarter and half turns;
  a smooth field comes back within the interpolation error O(h^2).
"""
import math

import numpy as np
import pytest

from oracle import gpe, nls


def box(n, L=6.0, **kw):
    d = dict(xl=-L, xr=L, yb=-L, yu=L, nx=n, ny=n, dt=0.01, lap=0.5, kappa=-10.0)
    d.update(kw)
    return nls.Problem(**d)


def test_trap_at_t0_is_the_lab_trap():
    prob = box(8)
    X, Y = prob.grid()
    np.testing.assert_allclose(gpe.trap_potential(prob, 0.0, 1.3, 0.7, 0.4), -0.5 * (1.69 * X ** 2 + 0.49 * Y ** 2))


def test_isotropic_trap_does_not_depend_on_time():
    prob = box(8)
    v0 = gpe.trap_potential(prob, 0.0, 1.1, 1.1, 0.9)
    for t in (0.3, 1.7, 5.0):
        np.testing.assert_allclose(gpe.trap_potential(prob, t, 1.1, 1.1, 0.9), v0, rtol=1e-14, atol=1e-13)


def test_quarter_turn_exchanges_the_trap_axes():
    prob = box(8)
    X, Y = prob.grid()
    omega = 0.8
    t = 0.5 * math.pi / omega
    np.testing.assert_allclose(gpe.trap_potential(prob, t, 1.3, 0.7, omega), -0.5 * (1.69 * Y ** 2 + 0.49 * X ** 2),
                               atol=1e-12)


def test_step_potential_is_the_midpoint_average():
    prob = box(8)
    n = 7
    want = 0.5 * (gpe.trap_potential(prob, n * prob.dt, 1.3, 0.7, 2.0) + gpe.trap_potential(prob, (n - 1) * prob.dt, 1.3, 0.7, 2.0))
    np.testing.assert_allclose(gpe.step_potential(prob, n, 1.3, 0.7, 2.0), want)


def vortex(prob, m):
    X, Y = prob.grid()
    return (X + 1j * Y) ** m * np.exp(-(X ** 2 + Y ** 2) / 2.0) if m >= 0 else \
        (X - 1j * Y) ** (-m) * np.exp(-(X ** 2 + Y ** 2) / 2.0)


@pytest.mark.parametrize("m", [1, 2, -1])
def test_vortex_states_carry_angular_momentum_m(m):
    errs = []
    for n in (32, 64, 128):
        prob = box(n)
        u = vortex(prob, m)
        ratio = gpe.angular_momentum(prob, u) / nls.mass(nls.Problem(**{**prob.__dict__, "lap": 1.0}), u)
        errs.append(abs(ratio - m))
    assert errs[-1] < 2e-3 * abs(m)
    for i in range(2):
        assert 1.8 < math.log2(errs[i] / errs[i + 1]) < 2.3, errs


def test_real_states_carry_no_angular_momentum():
    prob = box(20)
    X, Y = prob.grid()
    u = np.exp(-(X - 0.3) ** 2 - 2 * Y ** 2) * (1 + 0.2 * X * Y)
    assert abs(gpe.angular_momentum(prob, u)) < 1e-14


def test_energy_rotation_term_and_its_nls_part():
    prob = box(24, kappa=-7.0, lap=0.5)
    X, Y = prob.grid()
    u = vortex(prob, 1) + 0.3 * np.exp(-(X - 1) ** 2 - Y ** 2)
    V = gpe.trap_potential(prob, 0.0, 1.0, 1.2, 0.0)
    prob.V = V
    e0 = gpe.energy_lab(prob, u, V, 0.0)
    e1 = gpe.energy_lab(prob, u, V, 0.4)
    assert abs((e1 - e0) + 0.4 * gpe.angular_momentum(prob, u)) < 1e-12 * abs(e0)
    # without rotation: lap times the (pinned) NLS-form energy of the scaled equation
    assert abs(e0 - prob.lap * nls.energy(prob, u)) < 1e-12 * abs(e0)


def test_energy_of_the_gpe_in_its_own_terms():
    """int 1/2 |grad u|^2 + V_trap |u|^2 + beta/2 |u|^4 for a Gaussian, against its closed form
    (mesh error O(h^2) at h = 12/256)."""
    beta = 3.0
    prob = box(256, kappa=-beta, lap=0.5)
    X, Y = prob.grid()
    u = np.exp(-(X ** 2 + Y ** 2) / 2.0)
    Vsch = gpe.trap_potential(prob, 0.0, 1.0, 1.0, 0.0)           # V_trap = r^2/2
    e = gpe.energy_lab(prob, u, Vsch, 0.0)
    # |grad u|^2 = r^2 e^{-r^2}: int = pi;  V_trap|u|^2 = r^2/2 e^{-r^2}: pi/2;  |u|^4 = e^{-2r^2}: pi/2
    exact = 0.5 * math.pi + 0.5 * math.pi + 0.5 * beta * 0.5 * math.pi
    assert abs(e - exact) < 2e-3 * exact


def test_q1_interpolation_reproduces_bilinear_functions():
    prob = box(7, L=3.0)
    X, Y = prob.grid()
    f = lambda x, y: 0.3 - 1.2 * x + 0.7 * y + 0.25 * x * y       # noqa: E731
    rng = np.random.default_rng(4)
    xq, yq = rng.uniform(-3, 3, 50), rng.uniform(-3, 3, 50)
    np.testing.assert_allclose(gpe.q1_interpolate(prob, f(X, Y), xq, yq), f(xq, yq), atol=1e-13)


@pytest.mark.parametrize("turn", [0.0, 0.25, 0.5])
def test_lab_frame_is_exact_for_bilinear_fields(turn):
    """u~ bilinear in (x~, y~): its Q1 interpolant is itself, so u(x, y) = u~(A(t)^T (x, y)) holds
    to round-off at every point of the valid zone (t = 0: the identity; a quarter turn:
    u~(-y, x); a half turn: u~(-x, -y))."""
    omega = 0.5
    t = turn * 2.0 * math.pi / omega
    prob = box(12)
    X, Y = prob.grid()
    f = lambda x, y: (0.3 + 0.1j) - 1.2 * x + 0.7j * y + 0.25 * x * y       # noqa: E731
    out = gpe.lab_frame(prob, f(X, Y), t, omega, 9, 7)
    x0, x1, y0, y1 = gpe.valid_zone(prob)
    XS, YS = np.meshgrid(np.linspace(x0, x1, 10), np.linspace(y0, y1, 8), indexing="xy")
    c, s = math.cos(omega * t), math.sin(omega * t)
    np.testing.assert_allclose(out, f(c * XS - s * YS, s * XS + c * YS), atol=1e-12)
    if turn == 0.25:
        np.testing.assert_allclose(out, f(-YS, XS), atol=1e-12)


def test_lab_frame_quarter_turn_of_a_smooth_field():
    omega = 0.5
    t = 0.5 * math.pi / omega             # A(t) = [[0, 1], [-1, 0]]: u(x, y) = u~(-y, x)
    errs = []
    for n in (32, 64, 128):
        prob = box(n)
        X, Y = prob.grid()
        ut = np.exp(-((X - 1.0) ** 2 + 0.5 * Y ** 2)) * np.exp(0.5j * X)
        out = gpe.lab_frame(prob, ut, t, omega, 20, 20)
        x0, x1, y0, y1 = gpe.valid_zone(prob)
        XS, YS = np.meshgrid(np.linspace(x0, x1, 21), np.linspace(y0, y1, 21), indexing="xy")
        xt, yt = -YS, XS
        want = np.exp(-((xt - 1.0) ** 2 + 0.5 * yt ** 2)) * np.exp(0.5j * xt)
        errs.append(np.max(np.abs(out - want)))
    assert errs[-1] < 5e-3, errs
    assert all(errs[i + 1] < errs[i] / 2.5 for i in range(2)), errs
