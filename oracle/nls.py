"""FP64 CPU oracle of the optimized Schwarz method for the 2D NLS / GPE (Besse & Xing).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this module: only the
tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` use it.  It shares no code with the CUDA library.

What it computes, in the paper's notation (sections and equation labels of arXiv:1603.05110):

* Sec. 2.1, eq. (Sch) and (CNS): the Duran--Sanz-Serna midpoint scheme.  One time step solves
  the stationary problem  L_x v = (2i/dt) u_{n-1}  for v = (u_n + u_{n-1})/2 and commits
  u_n = 2 v - u_{n-1}.  The GPE (eq. GPE_Trans) has 1/2 in front of the Laplacian; dividing
  the equation by that coefficient ``lap`` gives the same form with alpha = 2/(lap*dt),
  W = V/lap and f = (kappa/lap)|u|^2 (reading D6).  V and kappa are given in the sign of
  eq. (Sch):  i u_t + lap*Lap u + V u + kappa |u|^2 u = 0.
* Sec. 2.2, eq. (NproblemRobinNL): a strip (or the whole domain) with Robin data,
  (A + i p M^Gamma + M_f(zeta^{q-1})) zeta^q = (2i/dt) M h - M^Gamma Q^T (l; r),
  A = alpha M - S + M_W, solved by the fixed point of eq. (localpbrobin) with zeta^0 = h.
* Sec. 2.2, eq. (localpbS2p) and (NproblemSPNL): the S_pade^m transmission condition with
  auxiliary unknowns phi_s on each vertical edge; the coupled (zeta, phi_1..phi_m) system is
  assembled as printed and solved by sparse LU.  The nonlinear term is semi-implicit in the
  zeta rows and lagged in the phi rows (reading D12); the fixed point is the same.
* Sec. 2.1, eq. (fluxlr) and Sec. 2.3, eq. (AlgoGraph), (algo_d): the classical algorithm
  g^{k+1} = R(g^k) on the interface vector g = (r_1, l_2, r_2, ..., l_N).
* Sec. 3, eq. (algo_pd), (Lmpi): the preconditioned algorithm
  g^{k+1} = g^k - P^{-1}(g^k - R(g^k)), P = I - L_h, with L_h the linear part of R for the
  free equation (V = 0, f = 0).  L_h is built column by column from strip solves on unit
  data (Sec. 4.2), never from the printed X formulas (reading D9); P x = y is solved by
  restarted GMRES (Sec. 4.2).
* Sec. 5, the stopping test on the interface residual; here relative,
  ||R(g) - g|| / ||R(g)|| (reading D11); the absolute value is returned too.

Linear solves use SuperLU (scipy.sparse.linalg.splu), a library primitive.  No blocking,
fusion or reordering beyond the paper's algorithms is done here.
"""
import math
from dataclasses import dataclass, field, replace

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem


# ----------------------------------------------------------------------------------------
# problem statement
# ----------------------------------------------------------------------------------------
@dataclass
class Problem:
    """Omega = (xl, xr) x (yb, yu) cut into nx x ny cells; eq. (Sch) with BC (BC)."""
    xl: float
    xr: float
    yb: float
    yu: float
    nx: int
    ny: int
    dt: float
    V: np.ndarray = None          # nodal real potential, shape (ny+1, nx+1), eq. (Sch) sign
    kappa: float = 0.0            # f(u) = kappa |u|^2, eq. (Sch) sign
    lap: float = 1.0              # coefficient of the Laplacian (1 NLS, 1/2 GPE)
    tc: str = "robin"             # transmission condition: 'robin' (TCSRobin) or 'pade' (TCS)
    p: float = 1.0                # Robin parameter, eq. (TCSRobin)
    m: int = 4                    # Pade order, eq. (TCS)
    theta: float = math.pi / 4    # branch-cut rotation of the Pade approximation
    bc: str = "same"              # physical x-edges: 'same' operator as the interfaces, or 'neumann'

    def __post_init__(self):
        if self.V is None:
            self.V = np.zeros((self.ny + 1, self.nx + 1))
        self.V = np.asarray(self.V, dtype=np.float64)
        assert self.V.shape == (self.ny + 1, self.nx + 1)

    @property
    def hx(self):
        return (self.xr - self.xl) / self.nx

    @property
    def hy(self):
        return (self.yu - self.yb) / self.ny

    @property
    def alpha(self):
        """2/dt of eq. (CNS) after dividing the equation by ``lap``."""
        return 2.0 / (self.lap * self.dt)

    @property
    def kap(self):
        return self.kappa / self.lap

    def grid(self):
        x = self.xl + self.hx * np.arange(self.nx + 1)
        y = self.yb + self.hy * np.arange(self.ny + 1)
        return np.meshgrid(x, y, indexing="xy")

    def free(self):
        """The free equation of Sec. 3 (V = 0, f = 0) on the same geometry."""
        return replace(self, V=np.zeros_like(self.V), kappa=0.0)


def pade_coefficients(m, theta=math.pi / 4):
    """a_s^m and d_s^m of eq. (TCS), s = 1..m (reading D8: the sums start at s = 1)."""
    s = np.arange(1, m + 1)
    ang = (2 * s - 1) * math.pi / (4 * m)
    a = np.exp(0.5j * theta) / (m * np.cos(ang) ** 2)
    d = np.exp(1j * theta) * np.tan(ang) ** 2
    return a, d


# ----------------------------------------------------------------------------------------
# one rectangular region (a strip Omega_j, or Omega itself)
# ----------------------------------------------------------------------------------------
class Region:
    """Discrete operators of eq. (eqdist) on cells ix0 .. ix0+ncx-1 of ``prob``.

    ``left`` / ``right`` say what sits on each vertical edge: 'tc' (transmission operator
    S-bar with data l or r) or 'neumann' (homogeneous Neumann, no data).
    """

    def __init__(self, prob, ix0, ncx, left="tc", right="tc"):
        self.prob = prob
        self.ix0, self.ncx = ix0, ncx
        self.ny = prob.ny
        self.kind = {"l": left, "r": right}
        hx, hy = prob.hx, prob.hy
        self.shape = (prob.ny + 1, ncx + 1)
        self.n = self.shape[0] * self.shape[1]
        self.M, self.S = fem.assemble_q1(ncx, prob.ny, hx, hy)
        self.w = fem.lumped_weights(ncx, prob.ny, hx, hy).ravel()
        self.W = (prob.V[:, ix0:ix0 + ncx + 1] / prob.lap).ravel()
        self.mg, self.sg = fem.assemble_p1(prob.ny, hy)           # M^Gamma, S^Gamma along an edge
        self.wg = fem.lumped_weights_1d(prob.ny, hy)
        self.Q = {s: fem.edge_embedding(ncx, prob.ny, s) for s in "lr"}
        alpha = prob.alpha
        # A = (2i/dt) M - S + M_W  (eq. NproblemRobinNL, in the scaled form)
        self.A = (1j * alpha) * self.M - self.S + sp.diags(self.w * self.W)
        self.edge_W = {s: self.Q[s] @ self.W for s in "lr"}
        if prob.tc == "pade":
            self.a, self.d = pade_coefficients(prob.m, prob.theta)

    # -- data ------------------------------------------------------------------------
    def restrict(self, u_global):
        return u_global[:, self.ix0:self.ix0 + self.ncx + 1].ravel()

    def rhs(self, h, l, r):
        """(2i/dt) M h - M^Gamma Q^T (l; r): right side of eq. (NproblemRobinNL)."""
        b = (1j * self.prob.alpha) * (self.M @ h)
        for s, data in (("l", l), ("r", r)):
            if data is not None and self.kind[s] == "tc":
                b = b - self.Q[s].T @ (self.mg @ data)
        return b

    # -- Robin, eq. (NproblemRobinNL) --------------------------------------------------
    def robin_matrix(self, zeta):
        p = self.prob.p
        A = self.A + sp.diags(self.w * self.prob.kap * np.abs(zeta) ** 2)
        for s in "lr":
            if self.kind[s] == "tc":
                A = A + (1j * p) * (self.Q[s].T @ sp.csr_matrix(self.mg) @ self.Q[s])
        return A.tocsc()

    # -- S_pade, eq. (NproblemSPNL) -----------------------------------------------------
    def pade_edges(self):
        return [s for s in "lr" if self.kind[s] == "tc"]

    def pade_matrix(self, zeta):
        """The block matrix of eq. (NproblemSPNL), zeta rows semi-implicit in f (D12).

        Unknown order: zeta, then for each transmission edge e in (l, r) the blocks
        phi_{e,1} .. phi_{e,m}.
        """
        prob = self.prob
        m, a, d = prob.m, self.a, self.d
        edges = self.pade_edges()
        ne = self.ny + 1
        mg = sp.csr_matrix(self.mg)
        blocks = [[None] * (1 + m * len(edges)) for _ in range(1 + m * len(edges))]
        A = self.A + sp.diags(self.w * prob.kap * np.abs(zeta) ** 2)
        for e in edges:
            A = A + (1j * a.sum()) * (self.Q[e].T @ mg @ self.Q[e])
        blocks[0][0] = A
        for ie, e in enumerate(edges):
            D0 = (1j * prob.alpha) * mg - sp.csr_matrix(self.sg) + sp.diags(self.wg * self.edge_W[e])
            for s in range(m):
                k = 1 + ie * m + s
                blocks[0][k] = (-1j * a[s] * d[s]) * (self.Q[e].T @ mg)          # B_s
                blocks[k][0] = -(mg @ self.Q[e])                                   # C
                blocks[k][k] = D0 + d[s] * mg                                      # D_s
        for i in range(len(blocks)):
            for j in range(len(blocks)):
                if blocks[i][j] is None and i == j:
                    blocks[i][j] = sp.csr_matrix((ne, ne))
        return sp.bmat(blocks, format="csc")

    def pade_rhs(self, b, zeta_prev, phi_prev):
        """Right side of eq. (NproblemSPNL) with the phi rows lagged in f (D12)."""
        prob = self.prob
        edges = self.pade_edges()
        parts = [b]
        for e in edges:
            fe = self.wg * prob.kap * np.abs(self.Q[e] @ zeta_prev) ** 2
            for s in range(prob.m):
                parts.append(-fe * phi_prev[e][s])
        return np.concatenate(parts)

    def trace_S(self, v, phi, side):
        """S v on one edge, eq. (TCSdist)."""
        prob = self.prob
        vt = self.Q[side] @ v
        if prob.tc == "robin":
            return -1j * prob.p * vt
        out = -1j * self.a.sum() * vt
        for s in range(prob.m):
            out = out + 1j * self.a[s] * self.d[s] * phi[side][s]
        return out

    # -- nonlinear solve of the local problem ---------------------------------------------
    def solve(self, h, l, r, tol=1e-13, maxit=400, relax=1.0):
        """Fixed point of eq. (localpbrobin) / (localpbS2p), zeta^0 = h, phi^0 = 0.

        Stops when ||F(zeta^{q-1}) - zeta^{q-1}|| <= tol ||F(zeta^{q-1})||, F one solve of the
        fixed point.  ``relax`` < 1 takes zeta^q = relax F(zeta^{q-1}) + (1 - relax) zeta^{q-1}
        (same fixed point; the plain iteration diverges for strong nonlinearity, the paper is
        silent on safeguards).  Returns (v, phi, iterations); phi maps an edge to its list of m
        traces (empty for Robin).
        """
        prob = self.prob
        b = self.rhs(h, l, r)
        zeta = h.astype(np.complex128).copy()
        ne = self.ny + 1
        phi = {e: [np.zeros(ne, complex) for _ in range(prob.m)] for e in self.pade_edges()} \
            if prob.tc == "pade" else {}
        linear = prob.kap == 0.0
        for q in range(1, maxit + 1):
            if prob.tc == "robin":
                new = spla.splu(self.robin_matrix(zeta)).solve(b)
                new_phi = phi
            else:
                sol = spla.splu(self.pade_matrix(zeta)).solve(self.pade_rhs(b, zeta, phi))
                new = sol[:self.n]
                new_phi = {}
                for ie, e in enumerate(self.pade_edges()):
                    off = self.n + ie * prob.m * ne
                    new_phi[e] = [sol[off + s * ne: off + (s + 1) * ne] for s in range(prob.m)]
            step = np.linalg.norm(new - zeta)
            done = linear or step <= tol * np.linalg.norm(new)
            if done or relax == 1.0:
                zeta, phi = new, new_phi
            else:
                zeta = relax * new + (1.0 - relax) * zeta
                phi = {e: [relax * a + (1.0 - relax) * b for a, b in zip(new_phi[e], phi[e])] for e in new_phi}
            if done:
                return zeta, phi, q
        raise RuntimeError("fixed point did not converge")


# ----------------------------------------------------------------------------------------
# monodomain step (the limit every Schwarz iteration must reach)
# ----------------------------------------------------------------------------------------
def physical_kind(prob):
    return "tc" if prob.bc == "same" else "neumann"


def mono_region(prob):
    k = physical_kind(prob)
    return Region(prob, 0, prob.nx, left=k, right=k)


def mono_step(prob, u_prev, tol=1e-13, l=None, r=None, region=None, relax=1.0):
    """One step of eq. (CNS) on the whole of Omega.  ``l``/``r`` are optional physical
    Robin data on x = xl / x = xr (eq. eqdist); they default to the homogeneous BC (BC)."""
    reg = region or mono_region(prob)
    h = u_prev.ravel().astype(np.complex128)
    v, _, q = reg.solve(h, l, r, tol=tol, relax=relax)
    v = v.reshape(reg.shape)
    return 2.0 * v - u_prev, v, q


# ----------------------------------------------------------------------------------------
# Schwarz algorithms
# ----------------------------------------------------------------------------------------
class Strips:
    """Omega cut into N equal x-strips (Sec. 2.1, Fig. figsub3).

    ``pool`` (optional, from ``strip_pool``): the strip solves of one Schwarz iteration are
    independent (one MPI rank per strip in Sec. 4), so they may run in worker processes; the
    arithmetic is the same either way."""

    def __init__(self, prob, N, pool=None):
        assert prob.nx % N == 0, "strips must be equal"
        self.prob, self.N = prob, N
        self.pool = pool
        self.c = prob.nx // N
        pk = physical_kind(prob)
        self.regions = [Region(prob, j * self.c, self.c,
                               left=pk if j == 0 else "tc",
                               right=pk if j == N - 1 else "tc") for j in range(N)]
        self.ne = prob.ny + 1

    def zero_g(self):
        return np.zeros((2 * (self.N - 1), self.ne), complex)

    def data(self, g, j):
        """(l_j, r_j) of strip j from g = (r_1, l_2, r_2, ..., l_N); l_1 = r_N = 0."""
        l = g[2 * (j - 1) + 1] if j > 0 else np.zeros(self.ne, complex)
        r = g[2 * j] if j < self.N - 1 else np.zeros(self.ne, complex)
        return l, r

    def apply_R(self, g, u_prev, tol_fp=1e-13, relax=1.0):
        """R(g) of eq. (algo_d): solve every strip, then the flux update of eq. (fluxlr)."""
        Rg = np.zeros_like(g)
        vs, fp_its = [], []
        tasks = [(j, *self.data(g, j), reg.restrict(u_prev), tol_fp, relax) for j, reg in enumerate(self.regions)]
        if self.pool is not None:
            sols = self.pool.map(_pool_solve, tasks)
        else:
            sols = [reg.solve(h, l, r, tol=t, relax=rx) for reg, (_, l, r, h, t, rx) in zip(self.regions, tasks)]
        for j, reg in enumerate(self.regions):
            l, r = self.data(g, j)
            v, phi, q = sols[j]
            vs.append(v)
            fp_its.append(q)
            if j > 0:        # new r_{j-1} = -l_j + 2 S v_j(a_j)
                Rg[2 * (j - 1)] = -l + 2.0 * reg.trace_S(v, phi, "l")
            if j < self.N - 1:   # new l_{j+1} = -r_j + 2 S v_j(b_j)
                Rg[2 * j + 1] = -r + 2.0 * reg.trace_S(v, phi, "r")
        return Rg, vs, fp_its

    def assemble(self, vs):
        """Global nodal field from strip fields; interface columns from the left strip."""
        p = self.prob
        out = np.zeros((p.ny + 1, p.nx + 1), complex)
        for j in reversed(range(self.N)):
            out[:, j * self.c: (j + 1) * self.c + 1] = vs[j].reshape(p.ny + 1, self.c + 1)
        return out

    # -- L_h of eq. (Lmpi) ---------------------------------------------------------------
    def strip_blocks(self, j):
        """X^{j,1..4} of strip j for the free equation (Props 3.1 / 3.2), built from
        2(Ny+1) solves on unit data (Sec. 4.2): out_left = X1 l + X2 r (the new r_{j-1}),
        out_right = X3 l + X4 r (the new l_{j+1})."""
        free = self.prob.free()
        base = self.regions[j]
        reg = Region(free, base.ix0, base.ncx, left=base.kind["l"], right=base.kind["r"])
        ne = self.ne
        X = [np.zeros((ne, ne), complex) for _ in range(4)]
        h0 = np.zeros(reg.n, complex)
        z = np.zeros(ne, complex)
        for s in range(ne):
            e = np.zeros(ne, complex)
            e[s] = 1.0
            if reg.kind["l"] == "tc":
                v, phi, _ = reg.solve(h0, e, z)
                X[0][:, s] = -e + 2.0 * reg.trace_S(v, phi, "l")
                X[2][:, s] = 2.0 * reg.trace_S(v, phi, "r")
            if reg.kind["r"] == "tc":
                v, phi, _ = reg.solve(h0, z, e)
                X[1][:, s] = 2.0 * reg.trace_S(v, phi, "l")
                X[3][:, s] = -e + 2.0 * reg.trace_S(v, phi, "r")
        return X

    def build_Lh(self):
        """Blocks of L_h per strip; equal strips share their blocks (Prop 3.1)."""
        cache, blocks = {}, []
        for j, reg in enumerate(self.regions):
            key = (reg.kind["l"], reg.kind["r"])
            if key not in cache:
                cache[key] = self.strip_blocks(j)
            blocks.append(cache[key])
        return blocks

    # -- exact P^{-1} in the cosine basis ---------------------------------------------------
    def modal_blocks(self):
        """Per strip, the entries x1..x4 of its L_h blocks on the cosine modes c_k(iy) =
        cos(k pi iy / ny), k = 0..ny (each block X^{j,a} is diagonal in that basis: the 1D
        P1 matrices along y with Neumann ends satisfy K_y c_k = lambda_k M_y c_k).

        On mode k the free strip problem (V = 0, f = 0) of eq. (NproblemRobinNL) becomes the
        1D problem in x  (i alpha M_x - K_x - lambda_k M_x + i rho_k E) a = -e_edge  for a unit
        datum on one edge, with rho_k = p (Robin) or, after eliminating phi_s of eq. (TCS_phi)
        (D_s phi_s = M^Gamma zeta on the edge, diagonal on the modes too),
        rho_k = sum_s a_s - sum_s a_s d_s / (z_k + d_s), z_k = i alpha - lambda_k (S_pade).
        The outgoing traces of eq. (fluxlr) are -datum + 2 S v with S v = -i rho_k a(edge).
        Returns a list over strips of arrays (4, ny+1)."""
        prob = self.prob
        ny, c = prob.ny, self.c
        hy = prob.hy
        k = np.arange(ny + 1)
        th = np.pi * k / ny if ny > 0 else np.zeros(1)
        lam = (6.0 / hy ** 2) * (1.0 - np.cos(th)) / (2.0 + np.cos(th))
        mx, kx = fem.assemble_p1(c, prob.hx)
        if prob.tc == "robin":
            rho = np.full(ny + 1, complex(prob.p))
        else:
            a, d = pade_coefficients(prob.m, prob.theta)
            z = 1j * prob.alpha - lam
            rho = a.sum() - (a[None, :] * d[None, :] / (z[:, None] + d[None, :])).sum(axis=1)
        cache, out = {}, []
        for reg in self.regions:
            key = (reg.kind["l"], reg.kind["r"])
            if key not in cache:
                X = np.zeros((4, ny + 1), complex)
                # the ny+1 mode problems as one batch of dense (c+1) x (c+1) solves
                B = (1j * prob.alpha * mx - kx)[None, :, :] - lam[:, None, None] * mx[None, :, :]
                if key[0] == "tc":
                    B[:, 0, 0] += 1j * rho
                if key[1] == "tc":
                    B[:, c, c] += 1j * rho
                if key[0] == "tc":
                    e = np.zeros((ny + 1, c + 1, 1), complex)
                    e[:, 0, 0] = -1.0
                    al = np.linalg.solve(B, e)[:, :, 0]
                    X[0] = -1.0 - 2j * rho * al[:, 0]
                    X[2] = -2j * rho * al[:, c]
                if key[1] == "tc":
                    e = np.zeros((ny + 1, c + 1, 1), complex)
                    e[:, c, 0] = -1.0
                    ar = np.linalg.solve(B, e)[:, :, 0]
                    X[1] = -2j * rho * ar[:, 0]
                    X[3] = -1.0 - 2j * rho * ar[:, c]
                cache[key] = X
            out.append(cache[key])
        return out

    def modal_P_solve(self, xm, y):
        """x with (I - L_h) x = y, exactly: cosine transform of every trace, one dense
        2(N-1) x 2(N-1) solve per mode with the entries of ``modal_blocks``, back-transform."""
        ny, N = self.prob.ny, self.N
        n = 2 * (N - 1)
        if n == 0:
            return y.copy()
        jj = np.arange(ny + 1)
        Z = np.cos(np.pi * np.outer(jj, jj) / ny) if ny > 0 else np.ones((1, 1))
        D = np.ones(ny + 1)
        D[0] = D[-1] = 0.5
        sig = np.diag((Z.T * D) @ Z)
        yh = (y * D[None, :]) @ Z / sig[None, :]          # coefficients, (n, ny+1)
        Pk = np.zeros((ny + 1, n, n), complex)
        Pk[:, np.arange(n), np.arange(n)] = 1.0
        for j in range(N):
            X = xm[j]
            il = 2 * (j - 1) + 1 if j > 0 else None       # l_j
            ir = 2 * j if j < N - 1 else None              # r_j
            if j > 0:                                      # rows of the new r_{j-1}
                if il is not None:
                    Pk[:, 2 * (j - 1), il] -= X[0]
                if ir is not None:
                    Pk[:, 2 * (j - 1), ir] -= X[1]
            if j < N - 1:                                  # rows of the new l_{j+1}
                if il is not None:
                    Pk[:, 2 * j + 1, il] -= X[2]
                if ir is not None:
                    Pk[:, 2 * j + 1, ir] -= X[3]
        xh = np.linalg.solve(Pk, yh.T[:, :, None])[:, :, 0]    # (ny+1, n)
        return xh.T @ Z.T

    def apply_Lh(self, blocks, x):
        y = np.zeros_like(x)
        for j in range(self.N):
            l, r = self.data(x, j)
            X1, X2, X3, X4 = blocks[j]
            if j > 0:
                y[2 * (j - 1)] += X1 @ l + X2 @ r
            if j < self.N - 1:
                y[2 * j + 1] += X3 @ l + X4 @ r
        return y


def gmres(matvec, b, tol=1e-13, restart=30, maxit=2000):
    """Restarted GMRES (modified Gram-Schmidt Arnoldi, least squares by numpy.linalg.lstsq)."""
    x = np.zeros_like(b)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return x, 0
    its = 0
    while its < maxit:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        if beta <= tol * nb:
            break
        Vb = [r / beta]
        H = np.zeros((restart + 1, restart), complex)
        for k in range(restart):
            w = matvec(Vb[k])
            for i in range(k + 1):
                H[i, k] = np.vdot(Vb[i], w)
                w = w - H[i, k] * Vb[i]
            H[k + 1, k] = np.linalg.norm(w)
            its += 1
            e1 = np.zeros(k + 2, complex)
            e1[0] = beta
            y, *_ = np.linalg.lstsq(H[:k + 2, :k + 1], e1, rcond=None)
            res = np.linalg.norm(H[:k + 2, :k + 1] @ y - e1)
            if H[k + 1, k] != 0.0:
                Vb.append(w / H[k + 1, k])
            if res <= tol * nb or H[k + 1, k] == 0.0 or its >= maxit:
                break
        x = x + np.stack(Vb[:len(y)], axis=1) @ y
    return x, its


@dataclass
class StepInfo:
    iterations: int = 0
    history: list = field(default_factory=list)       # relative interface residuals
    history_abs: list = field(default_factory=list)   # absolute ||R(g) - g||
    fixed_point_its: list = field(default_factory=list)
    gmres_its: list = field(default_factory=list)
    g: np.ndarray = None                              # R(g) at the last iteration
    converged: bool = True


def schwarz_step(prob, N, u_prev, g0=None, algorithm="classical", tol=1e-10, max_iter=2000,
                 strips=None, Lh=None, tol_fp=1e-13, gmres_tol=1e-13, absolute=False, relax=1.0,
                 psolve="gmres", modal=None, strict=True):
    """One time step by the classical (eq. algo_d) or preconditioned (eq. algo_pd) algorithm.

    Stops at the first k with ||R(g^k) - g^k|| <= tol * ||R(g^k)|| (or <= tol if
    ``absolute``) and returns u_n built from v^k (the strip solutions for g^k).  The
    preconditioned update solves P x = y by GMRES on the L_h blocks (``psolve='gmres'``,
    Sec. 4.2) or exactly in the cosine basis (``psolve='modal'``, the same P).  With
    ``strict=False`` a run that reaches ``max_iter`` returns what it has (info.converged False)
    instead of raising.
    """
    st = strips or Strips(prob, N)
    g = st.zero_g() if g0 is None else np.array(g0, dtype=complex)
    if algorithm == "preconditioned" and psolve == "modal" and modal is None:
        modal = st.modal_blocks()
    if algorithm == "preconditioned" and psolve != "modal" and Lh is None:
        Lh = st.build_Lh()
    info = StepInfo()
    for k in range(max_iter):
        Rg, vs, fp = st.apply_R(g, u_prev, tol_fp=tol_fp, relax=relax)
        diff = np.linalg.norm(Rg - g)
        nrm = np.linalg.norm(Rg)
        rel = diff / nrm if nrm > 0 else diff
        info.history.append(rel)
        info.history_abs.append(diff)
        info.fixed_point_its.append(fp)
        info.iterations = k + 1
        if (diff if absolute else rel) <= tol:
            break
        if algorithm == "classical":
            g = Rg
        elif psolve == "modal":
            g = g - st.modal_P_solve(modal, g - Rg)
        else:
            y = (g - Rg).ravel()
            x, its = gmres(lambda z: z - st.apply_Lh(Lh, z.reshape(g.shape)).ravel(), y,
                           tol=gmres_tol)
            info.gmres_its.append(its)
            g = g - x.reshape(g.shape)
    else:
        if strict:
            raise RuntimeError("Schwarz iteration did not converge")
        info.converged = False
    info.g = Rg
    v = st.assemble(vs)
    return 2.0 * v - u_prev, v, info


# ----------------------------------------------------------------------------------------
# worker processes for the strip solves (one per strip at a time, as one MPI rank per strip)
# ----------------------------------------------------------------------------------------
_WORKER = {}


def _pool_init(prob, N):
    _WORKER["prob"], _WORKER["N"], _WORKER["regions"] = prob, N, {}


def _pool_solve(task):
    j, l, r, h, tol, relax = task
    regs = _WORKER["regions"]
    if j not in regs:
        prob, N = _WORKER["prob"], _WORKER["N"]
        c = prob.nx // N
        pk = physical_kind(prob)
        regs[j] = Region(prob, j * c, c, left=pk if j == 0 else "tc", right=pk if j == N - 1 else "tc")
    return regs[j].solve(h, l, r, tol=tol, relax=relax)


def strip_pool(prob, N, processes):
    """A process pool (spawn start method) whose workers solve strips of ``prob``; each worker
    runs its numerical libraries on one thread, so the pool uses ``processes`` cores."""
    import multiprocessing as mp
    import os
    saved = {k: os.environ.get(k) for k in _THREAD_VARS}
    for k in _THREAD_VARS:
        os.environ[k] = "1"
    try:
        return mp.get_context("spawn").Pool(processes, initializer=_pool_init, initargs=(prob, N))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


# ----------------------------------------------------------------------------------------
# diagnostics
# ----------------------------------------------------------------------------------------
def mass(prob, u, region=None):
    """Discrete mass u^H M u (quadratic invariant of the midpoint scheme, eq. CNS)."""
    reg = region or mono_region(prob)
    uu = u.ravel()
    return float(np.real(np.vdot(uu, reg.M @ uu)))


def energy(prob, u, region=None):
    """Discrete energy u^H S u - u^H M_W u - (kappa/2) sum_i w_i |u_i|^4 of the scaled
    equation (reading D13).  Exactly conserved by eq. (CNS) for kappa = 0 and closed BCs."""
    reg = region or mono_region(prob)
    uu = u.ravel()
    e = np.real(np.vdot(uu, reg.S @ uu)) - np.sum(reg.w * reg.W * np.abs(uu) ** 2)
    e -= 0.5 * prob.kap * np.sum(reg.w * np.abs(uu) ** 4)
    return float(e)
