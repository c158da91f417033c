"""Pins of the oracle's S_pade coupling, its nonlinear energy and its cosine-mode P^{-1} (no GPU).

* S_pade (eq. TCS, TCS_phi, NproblemSPNL, TCSdist): eliminating the auxiliary unknowns phi_s from
  the oracle's block matrix must leave, on every cosine mode c_k of an edge, the Pade sum
  i (sum a_s - sum a_s d_s / (z_k + d_s)) M^Gamma c_k, z_k = i alpha - lambda_k, with lambda_k the
  closed-form eigenvalue of the 1D P1 stiffness against the mass along y; and the outgoing
  operator S v of eq. (TCSdist) must be -i times the same sum on each mode of the trace.
* energy (reading D13): with the correct coefficient kappa/2 of the quartic term the discrete
  energy of the midpoint scheme (eq. CNS) drifts by O(dt^2) over a fixed time; any other
  coefficient leaves an O(1) drift.
* the exact P^{-1} on the cosine modes equals the paper's construction (L_h from unit solves,
  Sec. 4.2, solved by GMRES).
"""
import math
import os

import numpy as np
import pytest

from oracle import fem, nls
from tests.helpers import printed_p_table


def cosine_modes(ny):
    j = np.arange(ny + 1)
    return np.cos(np.pi * np.outer(j, j) / ny)          # column k = c_k


def lam_closed_form(ny, hy):
    th = np.pi * np.arange(ny + 1) / ny
    return (6.0 / hy ** 2) * (1.0 - np.cos(th)) / (2.0 + np.cos(th))


def test_cosine_modes_are_generalised_eigenvectors_of_the_edge_matrices():
    ny, hy = 11, 0.37
    mg, sg = fem.assemble_p1(ny, hy)
    Z = cosine_modes(ny)
    lam = lam_closed_form(ny, hy)
    for k in range(ny + 1):
        np.testing.assert_allclose(sg @ Z[:, k], lam[k] * (mg @ Z[:, k]), atol=1e-12 * (1 + lam[k]))


def pade_strip(m=4, theta=math.pi / 4, ny=10, ncx=6, dt=0.02):
    prob = nls.Problem(xl=0.0, xr=3.0, yb=-1.0, yu=1.5, nx=ncx, ny=ny, dt=dt, kappa=0.0, tc="pade", m=m,
                       theta=theta)
    return prob, nls.Region(prob, 0, ncx, left="tc", right="tc")


@pytest.mark.parametrize("m,theta", [(4, math.pi / 4), (7, 0.3)])
def test_pade_schur_complement_is_the_pade_sum_on_each_cosine_mode(m, theta):
    prob, reg = pade_strip(m=m, theta=theta)
    n = reg.n
    K = reg.pade_matrix(np.zeros(n)).toarray()
    Azz, Azf, Afz, Aff = K[:n, :n], K[:n, n:], K[n:, :n], K[n:, n:]
    schur = Azz - Azf @ np.linalg.solve(Aff, Afz)
    E = schur - reg.A.toarray()            # what the transmission edges add to the strip rows
    a, d = nls.pade_coefficients(m, theta)
    lam = lam_closed_form(prob.ny, prob.hy)
    z = 1j * prob.alpha - lam
    rho = a.sum() - (a[None, :] * d[None, :] / (z[:, None] + d[None, :])).sum(axis=1)
    Z = cosine_modes(prob.ny)
    Ql, Qr = reg.Q["l"].toarray(), reg.Q["r"].toarray()
    inner = E - Ql.T @ (Ql @ E @ Ql.T) @ Ql - Qr.T @ (Qr @ E @ Qr.T) @ Qr
    assert np.max(np.abs(inner)) < 1e-10 * np.max(np.abs(E))      # edges only, no cross terms
    for Q in (Ql, Qr):
        Ee = Q @ E @ Q.T
        for k in range(prob.ny + 1):
            want = 1j * rho[k] * (reg.mg @ Z[:, k])
            np.testing.assert_allclose(Ee @ Z[:, k], want, atol=1e-10 * np.abs(want).max())


def test_pade_outgoing_trace_is_minus_i_times_the_pade_sum_on_each_mode():
    prob, reg = pade_strip(m=5)
    rng = np.random.default_rng(8)
    ne = prob.ny + 1
    h = rng.standard_normal(reg.n) + 1j * rng.standard_normal(reg.n)
    l = rng.standard_normal(ne) + 1j * rng.standard_normal(ne)
    r = rng.standard_normal(ne) + 1j * rng.standard_normal(ne)
    v, phi, _ = reg.solve(h, l, r)
    a, d = nls.pade_coefficients(prob.m, prob.theta)
    z = 1j * prob.alpha - lam_closed_form(prob.ny, prob.hy)
    rho = a.sum() - (a[None, :] * d[None, :] / (z[:, None] + d[None, :])).sum(axis=1)
    Z = cosine_modes(prob.ny)
    for side in "lr":
        vt = np.linalg.solve(Z, reg.Q[side] @ v)                # trace on the modes
        St = np.linalg.solve(Z, reg.trace_S(v, phi, side))
        np.testing.assert_allclose(St, -1j * rho * vt, atol=1e-10 * np.abs(St).max())


def test_robin_outgoing_trace_is_minus_ip():
    prob = nls.Problem(xl=0.0, xr=3.0, yb=-1.0, yu=1.5, nx=6, ny=10, dt=0.02, kappa=0.0, p=3.5)
    reg = nls.Region(prob, 0, 6)
    rng = np.random.default_rng(9)
    v = rng.standard_normal(reg.n) + 1j * rng.standard_normal(reg.n)
    np.testing.assert_array_equal(reg.trace_S(v, {}, "l"), -3.5j * (reg.Q["l"] @ v))


# ------------------------------------------------------------------------------ energy
def energy_drift(dt, T=0.4):
    prob = nls.Problem(xl=-4.0, xr=4.0, yb=-3.0, yu=3.0, nx=16, ny=12, dt=dt, kappa=2.0, bc="neumann")
    X, Y = prob.grid()
    prob.V = 2.0 * np.exp(-(X ** 2 + Y ** 2) / 4.0)
    u = np.exp(-(X ** 2 + Y ** 2)) * np.exp(2j * X)
    reg = nls.mono_region(prob)
    e0 = nls.energy(prob, u, reg)
    drift = 0.0
    for _ in range(int(round(T / dt))):
        u, _, _ = nls.mono_step(prob, u, region=reg)
        drift = max(drift, abs(nls.energy(prob, u, reg) - e0))
    return drift / abs(e0)


def test_nonlinear_energy_drift_is_second_order_in_dt():
    """The midpoint scheme conserves the NLS energy only up to O(dt^2) (the quartic term is not a
    quadratic invariant); the drift over a fixed time must fall by ~4 per halving of dt."""
    drifts = [energy_drift(0.4 / 2 ** i) for i in range(2, 6)]
    orders = [math.log2(drifts[i] / drifts[i + 1]) for i in range(3)]
    assert drifts[-1] < 2e-4, drifts
    assert all(1.6 < o < 2.4 for o in orders), (drifts, orders)


# ------------------------------------------------------------------------ P^{-1} on modes
def cos_basis(ny):
    Z = cosine_modes(ny)
    D = np.ones(ny + 1)
    D[0] = D[-1] = 0.5
    sig = np.diag((Z.T * D) @ Z)
    return Z, np.diag(1.0 / sig) @ Z.T @ np.diag(D)


@pytest.mark.parametrize("tc,bc", [("robin", "same"), ("robin", "neumann"), ("pade", "same")])
def test_modal_entries_equal_the_unit_solve_blocks(tc, bc):
    prob = nls.Problem(xl=-4.0, xr=4.0, yb=-3.0, yu=3.0, nx=20, ny=9, dt=0.05, kappa=0.0, tc=tc, m=3, p=2.5, bc=bc)
    st = nls.Strips(prob, 4)
    Z, Zi = cos_basis(prob.ny)
    xm = st.modal_blocks()
    for j in range(4):
        X = st.strip_blocks(j)
        reg = st.regions[j]
        for a in range(4):
            if (a in (0, 2) and reg.kind["l"] != "tc") or (a in (1, 3) and reg.kind["r"] != "tc"):
                continue
            np.testing.assert_allclose(xm[j][a], np.diag(Zi @ X[a] @ Z), atol=1e-12)


def test_modal_P_solve_equals_gmres_on_the_assembled_blocks():
    prob = nls.Problem(xl=-4.0, xr=4.0, yb=-3.0, yu=3.0, nx=20, ny=9, dt=0.05, kappa=0.0, p=2.5)
    st = nls.Strips(prob, 5)
    Lh = st.build_Lh()
    xm = st.modal_blocks()
    rng = np.random.default_rng(12)
    y = rng.standard_normal(st.zero_g().shape) + 1j * rng.standard_normal(st.zero_g().shape)
    x = st.modal_P_solve(xm, y)
    np.testing.assert_allclose(x - st.apply_Lh(Lh, x), y, atol=1e-12)
    xg, _ = nls.gmres(lambda v: v - st.apply_Lh(Lh, v.reshape(y.shape)).ravel(), y.ravel(), tol=1e-14)
    np.testing.assert_allclose(x.ravel(), xg, atol=1e-11)


def test_preconditioned_step_with_the_modal_solve_equals_the_gmres_step():
    prob = nls.Problem(xl=-4.0, xr=4.0, yb=-3.0, yu=3.0, nx=16, ny=12, dt=0.05, kappa=1.0, p=2.0)
    X, Y = prob.grid()
    prob.V = 2.0 * np.exp(-(X ** 2 + Y ** 2) / 4.0)
    u0 = np.exp(-(X ** 2 + Y ** 2)) * np.exp(2j * X)
    ua, _, ia = nls.schwarz_step(prob, 4, u0, algorithm="preconditioned", tol=1e-12)
    ub, _, ib = nls.schwarz_step(prob, 4, u0, algorithm="preconditioned", tol=1e-12, psolve="modal")
    assert np.linalg.norm(ua - ub) < 1e-11 * np.linalg.norm(ua)
    assert abs(ia.iterations - ib.iterations) <= 1


def test_strip_pool_gives_the_serial_result():
    prob = nls.Problem(xl=-4.0, xr=4.0, yb=-3.0, yu=3.0, nx=12, ny=7, dt=0.05, kappa=1.0, p=2.0)
    X, Y = prob.grid()
    u0 = np.exp(-(X ** 2 + Y ** 2)) * np.exp(2j * X)
    ua, _, _ = nls.schwarz_step(prob, 3, u0, tol=1e-12)
    with nls.strip_pool(prob, 3, 2) as pool:
        ub, _, _ = nls.schwarz_step(prob, 3, u0, tol=1e-12, strips=nls.Strips(prob, 3, pool=pool))
    np.testing.assert_array_equal(ua, ub)


# -------------------------------------------------- the paper's iteration counts (opt-in)
TABLE = printed_p_table()          # tests/golden: the printed table
P9_CLASSICAL_N2 = dict(zip(TABLE["p"], TABLE["cls"][2]))


def test_printed_table_fixture_is_the_printed_table():
    """The stored copy of Table Influence_p_NL_2_32: p = 5..50, the preconditioned count 6 at
    every p and N, the classical counts U-shaped with their minimum at p = 15 for both N."""
    assert TABLE["p"] == list(range(5, 51, 5))
    for N in (2, 32):
        assert TABLE["pd"][N] == [6] * 10
        cls = TABLE["cls"][N]
        assert int(np.argmin(cls)) == 2 and cls[0] == 57 and cls[-1] == 73
        assert all(a > b for a, b in zip(cls[:2], cls[1:3])) and all(a < b for a, b in zip(cls[2:], cls[3:]))


def p9_problem(p):
    """Sec. 5.1: (-16,16) x (-8,8), dx = 1/128, dy = 1/8 (4096 x 128 cells), V = 0, f = |u|^2,
    u0 = exp(-x^2 - y^2 - 0.5 i x), dt = 0.01, Robin p on the interfaces and the physical edges."""
    prob = nls.Problem(xl=-16.0, xr=16.0, yb=-8.0, yu=8.0, nx=4096, ny=128, dt=0.01, kappa=1.0, p=float(p))
    X, Y = prob.grid()
    return prob, np.exp(-X ** 2 - Y ** 2 - 0.5j * X)


@pytest.mark.slow
@pytest.mark.skipif(os.environ.get("ORACLE_SLOW") != "1", reason="opt-in: ORACLE_SLOW=1 (about an hour)")
@pytest.mark.parametrize("p", [10, 15, 20])
def test_paper_iteration_counts_for_robin_p_classical_two_strips(p):
    """Table Influence_p_NL_2_32, zero guess, N = 2, classical: the first step needs the printed
    count of iterations to reach ||g^{k+1} - g^k|| < 1e-10, within 3 (the paper does not state
    its norm's scaling nor its quadrature, so this is a soft pin)."""
    prob, u0 = p9_problem(p)
    with nls.strip_pool(prob, 2, 2) as pool:
        _, _, info = nls.schwarz_step(prob, 2, u0, tol=1e-10, absolute=True,
                                      strips=nls.Strips(prob, 2, pool=pool))
    # k Schwarz iterations produce g^1..g^k; the test on ||R(g^k) - g^k|| = ||g^{k+1} - g^k||
    assert abs(info.iterations - P9_CLASSICAL_N2[p]) <= 3, info.iterations
