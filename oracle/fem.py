"""Q1 finite elements on a uniform rectangular mesh (the oracle's space discretisation).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package: only the
tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` use it.

The matrices follow Sec. 2.2 of Besse & Xing (arXiv:1603.05110), "Preliminaries related to
space discretization": the standard Q1 element on a uniform mesh with cells of size
(dx, dy), the mass matrix M, the stiffness matrix S, the generalised mass matrices M_W and
M_f, and the boundary mass / stiffness matrices M^Gamma, S^Gamma on the vertical edges
x = a and x = b.

Everything here is *assembled element by element* from the bilinear basis functions with a
2x2 Gauss rule (exact for the Q1 mass and stiffness integrands).  The generalised mass
matrices for a nodal field (potential W, nonlinearity f) are not specified by the paper;
this code uses nodal (trapezoidal) quadrature, i.e. the diagonal matrix diag(w * W) with the
lumped weights w (reading D3 of the design notes: it keeps the matrices real symmetric and
additive across strips).

Node numbering of a region of ncx x ncy cells: node (iy, ix) has index iy*(ncx+1) + ix
(x fastest), matching arrays of shape (ncy+1, ncx+1).
"""
import numpy as np
import scipy.sparse as sp

_GAUSS_PTS = (0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0))   # on [0, 1]
_GAUSS_WTS = (0.5, 0.5)

# local node order of one cell: (dx, dy) offsets
_LOCAL = ((0, 0), (1, 0), (0, 1), (1, 1))


def _q1_basis(a, xi, eta):
    dx, dy = _LOCAL[a]
    bx = xi if dx else 1.0 - xi
    by = eta if dy else 1.0 - eta
    dbx = 1.0 if dx else -1.0
    dby = 1.0 if dy else -1.0
    return bx * by, dbx * by, bx * dby          # value, d/dxi, d/deta


def q1_element_matrices(hx, hy):
    """4x4 element mass and stiffness matrices of one hx-by-hy cell (2x2 Gauss rule)."""
    me = np.zeros((4, 4))
    ke = np.zeros((4, 4))
    for gx, wx in zip(_GAUSS_PTS, _GAUSS_WTS):
        for gy, wy in zip(_GAUSS_PTS, _GAUSS_WTS):
            jac = hx * hy * wx * wy
            vals = [_q1_basis(a, gx, gy) for a in range(4)]
            for a in range(4):
                na, dxa, dya = vals[a]
                for b in range(4):
                    nb, dxb, dyb = vals[b]
                    me[a, b] += na * nb * jac
                    ke[a, b] += (dxa * dxb / hx**2 + dya * dyb / hy**2) * jac
    return me, ke


def p1_edge_matrices(h):
    """2x2 element mass and stiffness of a 1D P1 segment of length h (2-point Gauss)."""
    me = np.zeros((2, 2))
    ke = np.zeros((2, 2))
    for g, wg in zip(_GAUSS_PTS, _GAUSS_WTS):
        n = (1.0 - g, g)
        dn = (-1.0 / h, 1.0 / h)
        for a in range(2):
            for b in range(2):
                me[a, b] += n[a] * n[b] * h * wg
                ke[a, b] += dn[a] * dn[b] * h * wg
    return me, ke


def assemble_q1(ncx, ncy, hx, hy):
    """Global M and S (scipy CSR) of a region of ncx x ncy cells, by element assembly."""
    me, ke = q1_element_matrices(hx, hy)
    nxn = ncx + 1
    cx, cy = np.meshgrid(np.arange(ncx), np.arange(ncy), indexing="xy")
    cx = cx.ravel()
    cy = cy.ravel()
    glob = np.stack([(cy + dy) * nxn + (cx + dx) for dx, dy in _LOCAL], axis=1)   # (ncell, 4)
    rows = np.repeat(glob, 4, axis=1).ravel()
    cols = np.tile(glob, (1, 4)).ravel()
    n = (ncy + 1) * nxn
    m = sp.coo_matrix((np.tile(me.ravel(), len(cx)), (rows, cols)), shape=(n, n)).tocsr()
    s = sp.coo_matrix((np.tile(ke.ravel(), len(cx)), (rows, cols)), shape=(n, n)).tocsr()
    return m, s


def assemble_p1(nc, h):
    """1D P1 mass and stiffness (dense) along an edge of nc segments, by element assembly."""
    me, ke = p1_edge_matrices(h)
    m = np.zeros((nc + 1, nc + 1))
    k = np.zeros((nc + 1, nc + 1))
    for e in range(nc):
        idx = [e, e + 1]
        m[np.ix_(idx, idx)] += me
        k[np.ix_(idx, idx)] += ke
    return m, k


def lumped_weights_1d(nc, h):
    """Trapezoidal (nodal quadrature) weights of a 1D uniform mesh: h inside, h/2 at the ends."""
    w = np.full(nc + 1, h)
    w[0] = w[-1] = 0.5 * h
    return w


def lumped_weights(ncx, ncy, hx, hy):
    """Nodal quadrature weights of a region, shape (ncy+1, ncx+1)."""
    return np.outer(lumped_weights_1d(ncy, hy), lumped_weights_1d(ncx, hx))


def edge_embedding(ncx, ncy, side):
    """Restriction Q (sparse, (ncy+1) x nnodes) onto the vertical edge x=a ('l') or x=b ('r')."""
    nxn = ncx + 1
    ix = 0 if side == "l" else ncx
    rows = np.arange(ncy + 1)
    cols = rows * nxn + ix
    return sp.csr_matrix((np.ones(ncy + 1), (rows, cols)), shape=(ncy + 1, (ncy + 1) * nxn))
