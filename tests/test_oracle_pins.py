"""Pins of the FP64 oracle against what the mathematics fixes (no GPU).

* brute force / library: the oracle's sparse LU path agrees with dense numpy solves, and its
  GMRES with numpy.linalg.solve;
* textbook special case: y-independent data reduce the 2D scheme to the 1D P1 midpoint
  scheme, solved here by the Thomas algorithm;
* invariants: mass conservation (closed Neumann BC, real potential), the exact Robin mass
  balance, energy conservation of the linear scheme;
* manufactured solution: second-order convergence to an exact plane wave;
* closed form: the Pade sum of eq. (TCS) approximates the square root;
* algebra: converged Schwarz = monodomain (Robin and S_pade, classical and preconditioned),
  the free problem converges in one preconditioned update (Prop. 3.1 / eq. algo_pd),
  equal strips have equal L_h blocks, and any interface guess reaches the same step.
"""
import math

import numpy as np
import pytest

from oracle import nls


def small_problem(nx=16, ny=12, tc="robin", bc="same", kappa=1.0, with_V=True, m=4, p=2.0, dt=0.05):
    prob = nls.Problem(xl=-4.0, xr=4.0, yb=-3.0, yu=3.0, nx=nx, ny=ny, dt=dt, kappa=kappa,
                       tc=tc, p=p, m=m, bc=bc)
    X, Y = prob.grid()
    if with_V:
        prob.V = 2.0 * np.exp(-(X ** 2 + Y ** 2) / 4.0)
    u0 = np.exp(-(X ** 2 + Y ** 2)) * np.exp(2j * X)
    return prob, u0


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# ---------------------------------------------------------------------------- brute force
def test_sparse_solve_matches_dense_numpy():
    prob, u0 = small_problem(nx=5, ny=4, kappa=0.0)
    reg = nls.mono_region(prob)
    A = reg.robin_matrix(np.zeros(reg.n)).toarray()
    b = reg.rhs(u0.ravel(), None, None)
    v_dense = np.linalg.solve(A, b)
    _, v, _ = nls.mono_step(prob, u0)
    assert rel(v.ravel(), v_dense) < 1e-13


def test_gmres_matches_direct_solve():
    rng = np.random.default_rng(7)
    n = 60
    A = np.eye(n) + 0.3 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, its = nls.gmres(lambda z: A @ z, b, tol=1e-13, restart=10)
    assert rel(x, np.linalg.solve(A, b)) < 1e-11
    assert its > 10          # restarted at least once


# ------------------------------------------------------------------ textbook special case
def thomas(a, b, c, d):
    """Tridiagonal solve: a sub-, b main, c super-diagonal."""
    n = len(b)
    cp = np.zeros(n, complex)
    dp = np.zeros(n, complex)
    cp[0] = c[0] / b[0]
    dp[0] = d[0] / b[0]
    for i in range(1, n):
        den = b[i] - a[i] * cp[i - 1]
        cp[i] = c[i] / den if i < n - 1 else 0.0
        dp[i] = (d[i] - a[i] * dp[i - 1]) / den
    x = np.zeros(n, complex)
    x[-1] = dp[-1]
    for i in range(n - 2, -1, -1):
        x[i] = dp[i] - cp[i] * x[i + 1]
    return x


def midpoint_1d(x, h, dt, V, kappa, p, u_prev, tol=1e-14):
    """1D P1 midpoint step with Robin -ip at both ends (the same scheme in one dimension)."""
    n = len(x)
    alpha = 2.0 / dt
    w = np.full(n, h)
    w[0] = w[-1] = h / 2
    mdiag = np.full(n, 4 * h / 6)
    mdiag[0] = mdiag[-1] = 2 * h / 6
    kdiag = np.full(n, 2 / h)
    kdiag[0] = kdiag[-1] = 1 / h
    moff = np.full(n, h / 6)
    koff = np.full(n, -1 / h)
    rhs = 1j * alpha * (mdiag * u_prev)
    rhs[1:] += 1j * alpha * moff[1:] * u_prev[:-1]
    rhs[:-1] += 1j * alpha * moff[:-1] * u_prev[1:]
    v = u_prev.astype(complex)
    for _ in range(200):
        main = 1j * alpha * mdiag - kdiag + w * V + w * kappa * np.abs(v) ** 2
        main[0] += 1j * p
        main[-1] += 1j * p
        off = 1j * alpha * moff - koff
        new = thomas(off, main, off, rhs)
        done = np.linalg.norm(new - v) <= tol * np.linalg.norm(new)
        v = new
        if done:
            break
    return 2 * v - u_prev


def test_y_independent_data_reduce_to_1d_scheme():
    prob = nls.Problem(xl=-5.0, xr=5.0, yb=0.0, yu=2.0, nx=40, ny=6, dt=0.02, kappa=1.5, p=3.0)
    X, Y = prob.grid()
    prob.V = 1.0 + np.cos(X)
    u0 = np.exp(-X ** 2) * np.exp(1j * X)
    u2 = u0.copy()
    x1 = X[0]
    u1 = u0[0].copy()
    for _ in range(3):
        u2, _, _ = nls.mono_step(prob, u2)
        u1 = midpoint_1d(x1, prob.hx, prob.dt, prob.V[0], prob.kappa, prob.p, u1)
    for iy in range(prob.ny + 1):
        assert rel(u2[iy], u1) < 1e-12


# ------------------------------------------------------------------------------ invariants
def test_mass_conserved_with_closed_neumann_boundary():
    prob, u0 = small_problem(bc="neumann", kappa=-2.0)
    m0 = nls.mass(prob, u0)
    u = u0
    for _ in range(5):
        u, _, _ = nls.mono_step(prob, u)
        assert abs(nls.mass(prob, u) / m0 - 1.0) < 1e-13


def test_robin_mass_balance_is_exact():
    """Im(v^H (i alpha M - S + D + i p M^G) v) gives m_n - m_{n-1} = -(4p/alpha) v^H M^G v."""
    prob, u0 = small_problem(kappa=1.0)
    reg = nls.mono_region(prob)
    u_prev = u0
    for _ in range(3):
        u, v, _ = nls.mono_step(prob, u_prev, region=reg)
        vv = v.ravel()
        mg_term = sum(np.real(np.vdot(reg.Q[s] @ vv, reg.mg @ (reg.Q[s] @ vv))) for s in "lr")
        lhs = nls.mass(prob, u, reg) - nls.mass(prob, u_prev, reg)
        rhs = -(4 * prob.p / prob.alpha) * mg_term
        assert abs(lhs - rhs) < 1e-13 * nls.mass(prob, u_prev, reg)
        assert lhs < 0
        u_prev = u


def test_energy_conserved_linear_closed():
    prob, u0 = small_problem(bc="neumann", kappa=0.0)
    e0 = nls.energy(prob, u0)
    u = u0
    for _ in range(5):
        u, _, _ = nls.mono_step(prob, u)
        assert abs(nls.energy(prob, u) - e0) < 1e-12 * abs(e0)


def test_nonlinear_energy_is_only_a_drift_diagnostic():
    prob, u0 = small_problem(bc="neumann", kappa=2.0)
    u, _, _ = nls.mono_step(prob, u0)
    e0, e1 = nls.energy(prob, u0), nls.energy(prob, u)
    assert abs(e1 - e0) < 1e-2 * abs(e0)


# ------------------------------------------------------------------ manufactured solution
def plane_wave_error(nx, ny, nt, T=0.5, p=2.0, V0=0.5):
    k, ky = 1.0, 1.0
    omega = k * k + ky * ky - V0
    prob = nls.Problem(xl=0.0, xr=2 * math.pi, yb=0.0, yu=math.pi, nx=nx, ny=ny, dt=T / nt,
                       kappa=0.0, p=p)
    X, Y = prob.grid()
    prob.V = np.full_like(X, V0)

    def exact(t):
        return np.cos(ky * Y) * np.exp(1j * (k * X - omega * t))

    reg = nls.mono_region(prob)
    u = exact(0.0)
    for n in range(1, nt + 1):
        tm = (n - 0.5) * prob.dt
        ue = exact(tm)
        l = -1j * (k + p) * ue[:, 0]          # d_n u + S u at x = xl, n = -e_x
        r = 1j * (k - p) * ue[:, -1]          # d_n u + S u at x = xr, n = +e_x
        u, _, _ = nls.mono_step(prob, u, l=l, r=r, region=reg)
    return rel(u, exact(T))


def test_manufactured_plane_wave_second_order():
    errs = [plane_wave_error(16 * 2 ** i, 8 * 2 ** i, 4 * 2 ** i) for i in range(3)]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[-1] < 5e-3
    for o in orders:
        assert 1.85 < o < 2.2, (errs, orders)


# ----------------------------------------------------------------------------- closed form
@pytest.mark.parametrize("dt", [0.01, 0.001])
def test_pade_sum_approximates_sqrt(dt):
    """sum_s a_s - sum_s a_s d_s/(z+d_s) -> sqrt(z) for z = 2i/dt - lambda (eq. TCS).

    The m-point rule is accurate once the largest pole d_m ~ (4m/pi)^2 exceeds |z|, which is
    why small time steps need a large order m (Sec. 5.2.2)."""
    lam = np.linspace(0.0, 1e3, 400)
    z = 2j / dt - lam
    errs = []
    for m in (4, 16, 64, 256):
        a, d = nls.pade_coefficients(m)
        approx = (a[None, :] * z[:, None] / (z[:, None] + d[None, :])).sum(axis=1)
        assert np.allclose(approx, a.sum() - (a * d / (z[:, None] + d)).sum(axis=1))
        errs.append(np.max(np.abs(approx - np.sqrt(z)) / np.abs(np.sqrt(z))))
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1))
    assert errs[-1] < 1e-5


# -------------------------------------------------------------------------------- Schwarz
@pytest.mark.parametrize("tc", ["robin", "pade"])
@pytest.mark.parametrize("N", [2, 4])
@pytest.mark.parametrize("algorithm", ["classical", "preconditioned"])
def test_converged_schwarz_equals_monodomain(tc, N, algorithm):
    prob, u0 = small_problem(tc=tc, m=3)
    u_mono, _, _ = nls.mono_step(prob, u0)
    tol = 1e-12
    u, _, info = nls.schwarz_step(prob, N, u0, algorithm=algorithm, tol=tol)
    assert rel(u, u_mono) < 1e3 * tol
    if algorithm == "preconditioned":
        assert info.iterations < 40


def test_free_problem_converges_in_one_preconditioned_update():
    """V = 0, f = 0: R(g) = L_h g + d, so g^1 = (I - L_h)^{-1} d is the fixed point."""
    prob, u0 = small_problem(nx=18, kappa=0.0, with_V=False)
    u_mono, _, _ = nls.mono_step(prob, u0)
    u, _, info = nls.schwarz_step(prob, 3, u0, algorithm="preconditioned", tol=1e-11,
                                  gmres_tol=1e-14)
    assert info.iterations == 2
    assert rel(u, u_mono) < 1e-10


def test_equal_strips_have_equal_blocks_and_blocks_match_R():
    prob, u0 = small_problem(nx=20, kappa=0.0, with_V=False)
    st = nls.Strips(prob, 5)
    b1, b2 = st.strip_blocks(1), st.strip_blocks(2)
    for x1, x2 in zip(b1, b2):
        np.testing.assert_allclose(x1, x2, atol=1e-13)
    # L_h g = R(g) - R(0) for the free problem (linearity, Sec. 3)
    Lh = st.build_Lh()
    rng = np.random.default_rng(3)
    g = rng.standard_normal(st.zero_g().shape) + 1j * rng.standard_normal(st.zero_g().shape)
    R0, _, _ = st.apply_R(st.zero_g(), u0)
    Rg, _, _ = st.apply_R(g, u0)
    np.testing.assert_allclose(st.apply_Lh(Lh, g), Rg - R0, atol=1e-11)


def test_any_initial_guess_reaches_the_same_step():
    prob, u0 = small_problem()
    st = nls.Strips(prob, 2)
    rng = np.random.default_rng(11)
    g_rand = rng.standard_normal(st.zero_g().shape) + 1j * rng.standard_normal(st.zero_g().shape)
    ua, _, _ = nls.schwarz_step(prob, 2, u0, tol=1e-12, strips=st)
    ub, _, ib = nls.schwarz_step(prob, 2, u0, g0=g_rand, tol=1e-12, strips=st)
    assert rel(ua, ub) < 1e-10


def cosine_basis(ny):
    j = np.arange(ny + 1)
    Z = np.cos(np.pi * np.outer(j, j) / ny)
    D = np.ones(ny + 1)
    D[0] = D[-1] = 0.5
    sig = np.diag((Z.T * D) @ Z)
    return Z, np.diag(1.0 / sig) @ Z.T @ np.diag(D)


@pytest.mark.parametrize("bc", ["same", "neumann"])
def test_lh_blocks_are_diagonal_in_the_cosine_basis(bc):
    """Uniform Q1 mesh with Neumann data in y: My and Ky share the eigenvectors cos(pi j k/ny)
    (w.r.t. D = diag(1/2,1,..,1,1/2)), so every block of L_h built by unit solves is diagonal
    in that basis.  This is what the exact modal P solve relies on."""
    prob, _ = small_problem(nx=20, ny=10, kappa=0.0, with_V=False, bc=bc)
    st = nls.Strips(prob, 4)
    Z, Zi = cosine_basis(prob.ny)
    np.testing.assert_allclose(Zi @ Z, np.eye(prob.ny + 1), atol=1e-14)
    for j in (0, 1, 3):
        for X in st.strip_blocks(j):
            Xh = Zi @ X @ Z
            assert np.max(np.abs(Xh - np.diag(np.diag(Xh)))) < 1e-13


def test_relaxed_fixed_point_has_the_same_limit_and_converges_where_plain_diverges():
    """Strong defocusing nonlinearity (GPE, beta = 900, dt = 0.002): the plain fixed point of
    eq. (localpbrobin) diverges; relaxed by 0.6 it converges, to a v that satisfies the
    discrete nonlinear system (checked by its residual), and for a mild nonlinearity both
    reach the same v."""
    prob = nls.Problem(xl=-4.0, xr=4.0, yb=-4.0, yu=4.0, nx=16, ny=33, dt=0.002, kappa=-900.0, lap=0.5, p=45.0)
    X, Y = prob.grid()
    prob.V = -0.5 * (X ** 2 + Y ** 2)
    u0 = np.pi ** -0.5 * np.exp(-(X ** 2 + Y ** 2) / 2)
    with pytest.raises(RuntimeError):
        nls.mono_step(prob, u0, relax=1.0)
    u1, v, _ = nls.mono_step(prob, u0, relax=0.6)
    reg = nls.mono_region(prob)
    vv = v.ravel()
    res = reg.robin_matrix(vv) @ vv - reg.rhs(u0.ravel(), None, None)
    assert np.linalg.norm(res) < 1e-11 * np.linalg.norm(reg.rhs(u0.ravel(), None, None))
    mild = nls.Problem(xl=-4.0, xr=4.0, yb=-4.0, yu=4.0, nx=16, ny=33, dt=0.002, kappa=-100.0, lap=0.5, p=45.0, V=prob.V)
    a, _, _ = nls.mono_step(mild, u0, relax=1.0)
    b, _, _ = nls.mono_step(mild, u0, relax=0.6)
    assert rel(b, a) < 1e-12
