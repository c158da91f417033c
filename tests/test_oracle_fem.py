"""Pins of the oracle's Q1 assembly (Sec. 2.2) against closed forms from the textbook.

The oracle assembles M and S cell by cell with a 2x2 Gauss rule; here the same matrices are
written as Kronecker products of the 1D P1 matrices (h/6)[1 4 1] and (1/h)[-1 2 -1], whose
tensor-product structure is a property of the Q1 space, not of the oracle's code.
"""
import numpy as np
import pytest

from oracle import fem


def p1_closed_form(n, h):
    m = np.zeros((n + 1, n + 1))
    k = np.zeros((n + 1, n + 1))
    for i in range(n + 1):
        m[i, i] = 4 * h / 6 if 0 < i < n else 2 * h / 6
        k[i, i] = 2 / h if 0 < i < n else 1 / h
        if i + 1 <= n:
            m[i, i + 1] = m[i + 1, i] = h / 6
            k[i, i + 1] = k[i + 1, i] = -1 / h
    return m, k


@pytest.mark.parametrize("ncx,ncy,hx,hy", [(1, 1, 1.0, 1.0), (3, 2, 0.5, 0.25), (6, 5, 0.1, 0.3)])
def test_q1_assembly_equals_kronecker(ncx, ncy, hx, hy):
    M, S = fem.assemble_q1(ncx, ncy, hx, hy)
    mx, kx = p1_closed_form(ncx, hx)
    my, ky = p1_closed_form(ncy, hy)
    # node index iy*(ncx+1)+ix  <=>  kron(y-matrix, x-matrix)
    np.testing.assert_allclose(M.toarray(), np.kron(my, mx), atol=1e-15)
    np.testing.assert_allclose(S.toarray(), np.kron(my, kx) + np.kron(ky, mx), atol=1e-13)


def test_interior_nine_point_stencils():
    """Textbook Q1 stencils on a square mesh: M = h^2/36 [1 4 1; 4 16 4; 1 4 1],
    S = 1/3 [-1 -1 -1; -1 8 -1; -1 -1 -1]."""
    h = 0.2
    M, S = fem.assemble_q1(4, 4, h, h)
    c = 2 * 5 + 2
    rowm = M.toarray()[c].reshape(5, 5)[1:4, 1:4]
    rows = S.toarray()[c].reshape(5, 5)[1:4, 1:4]
    np.testing.assert_allclose(rowm, h * h / 36 * np.array([[1, 4, 1], [4, 16, 4], [1, 4, 1]]), atol=1e-16)
    np.testing.assert_allclose(rows, np.array([[-1, -1, -1], [-1, 8, -1], [-1, -1, -1]]) / 3, atol=1e-14)


def test_mass_row_sums_are_lumped_weights_and_S_kills_constants():
    M, S = fem.assemble_q1(5, 3, 0.3, 0.7)
    w = fem.lumped_weights(5, 3, 0.3, 0.7).ravel()
    np.testing.assert_allclose(M @ np.ones(M.shape[0]), w, rtol=1e-14)
    np.testing.assert_allclose(S @ np.ones(S.shape[0]), 0.0, atol=1e-13)
    assert abs(w.sum() - 5 * 0.3 * 3 * 0.7) < 1e-13


def test_edge_matrices():
    m, k = fem.assemble_p1(7, 0.25)
    mc, kc = p1_closed_form(7, 0.25)
    np.testing.assert_allclose(m, mc, atol=1e-15)
    np.testing.assert_allclose(k, kc, atol=1e-13)
    # int_0^L x^2 dx with the P1 interpolant of x is exact for the consistent mass (x^T M x)
    x = 0.25 * np.arange(8)
    assert abs(x @ m @ x - (7 * 0.25) ** 3 / 3) < 1e-12
