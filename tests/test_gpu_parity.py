"""Parity of the CUDA path (through the C-ABI) with the FP64 CPU oracle.

Tolerances: the plain FP64 path must agree with the oracle to 1e-11 relative L2 per step;
both sides iterate to interface residuals <= 1e-12 (so neither stops one iteration away from
the other) and strip nonlinear residuals <= 1e-13.  The FP32-inner path keeps its residuals
in FP64, so it reaches the same discrete solution; it is held to 1e-10 here and to the 1e-6
contract bound in the workload-size tests.  The double-word residual carries ~48 bits
(unit round-off 2^-48 ~ 3.6e-15 per operation, a few operations deep); a strip solve uses it
down to a relative residual of 1e-12 and finishes with the FP64 residual, so the same 1e-10
holds.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import nls  # noqa: E402
from paper_1603_05110_gb300 import binding, workloads as wl  # noqa: E402
from tests.helpers import gpu_params, oracle_problem, rel  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_05110_gb300 import build
    build.build()
    binding.load()


def run_gpu(w, steps, **kw):
    u0 = w.u0()
    out = np.zeros_like(u0)
    hist = []
    with binding.Solver(gpu_params(w, **kw), u0, w.V()) as s:
        for _ in range(steps):
            st = s.step(1, out)
            hist.append((out.copy(), st))
    return hist


def run_oracle(w, steps, algorithm="classical", bc="same", tol=TOL, tc="robin", m=4, relax=1.0):
    prob = oracle_problem(w, bc=bc, tc=tc, m=m)
    st = nls.Strips(prob, w.n_strips)
    Lh = st.build_Lh() if algorithm == "preconditioned" else None
    u = w.u0()
    g = None
    out = []
    for _ in range(steps):
        u, _, info = nls.schwarz_step(prob, w.n_strips, u, g0=g, algorithm=algorithm, tol=tol, strips=st, Lh=Lh,
                                      relax=relax)
        g = info.g
        out.append((u.copy(), info))
    return out


MIXED = [binding.FP32_INNER, binding.FP32_DW]


def prec(precision):
    """Solver settings of one arithmetic mode."""
    return dict(precision=precision)


SMALL = wl.scaled(wl.NLS_SMALL, 48, 37, n_strips=3, xl=-6.0, xr=6.0, yb=-5.0, yu=5.0, dt=0.02)
WELL = wl.scaled(wl.NLS_WELL, 40, 45, n_strips=4, xl=-8.0, xr=8.0, yb=-8.0, yu=8.0, dt=0.02, p=3.0)


@pytest.mark.parametrize("precision", [binding.FP64] + MIXED)
def test_classical_robin_matches_oracle(precision):
    ref = run_oracle(SMALL, 3)
    got = run_gpu(SMALL, 3, tol=TOL, **prec(precision))
    bound = 1e-11 if precision == binding.FP64 else 1e-10
    for (ug, st), (uo, info) in zip(got, ref):
        assert rel(ug, uo) < bound


def test_picard_operator_and_jacobian_diagonal_reach_the_same_step():
    """The strip correction operator (fixed point of eq. localpbrobin, or the Jacobian
    diagonal) changes the path only: the converged step is the oracle's either way."""
    ref = run_oracle(SMALL, 2)
    for picard in (0, 1):
        got = run_gpu(SMALL, 2, tol=TOL, nl_picard=picard)
        for (ug, _), (uo, _) in zip(got, ref):
            assert rel(ug, uo) < 1e-11


def test_schwarz_iteration_counts_match_oracle_away_from_roundoff():
    """At tol 1e-8 the interface residual histories agree, so the iteration counts do."""
    ref = run_oracle(SMALL, 2, tol=1e-8)
    got = run_gpu(SMALL, 2, tol=1e-8)
    for (_, st), (_, info) in zip(got, ref):
        assert abs(st["last_schwarz_iterations"] - info.iterations) <= 1


@pytest.mark.parametrize("psolve", [binding.PSOLVE_MODAL, binding.PSOLVE_GMRES])
@pytest.mark.parametrize("precision", [binding.FP64] + MIXED)
def test_preconditioned_robin_matches_oracle(precision, psolve):
    ref = run_oracle(WELL, 2, algorithm="preconditioned")
    got = run_gpu(WELL, 2, tol=TOL, algorithm=binding.PRECONDITIONED, gmres_tol=1e-12, psolve=psolve,
                  **prec(precision))
    bound = 1e-11 if precision == binding.FP64 else 1e-10
    for (ug, st), (uo, info) in zip(got, ref):
        assert rel(ug, uo) < bound
        assert st["last_schwarz_iterations"] <= info.iterations + 5


@pytest.mark.parametrize("precision", [binding.FP64] + MIXED)
def test_adaptive_strip_tolerance_reaches_the_same_step(precision):
    """nl_adapt: loose strip solves in early preconditioned iterations, same converged step."""
    ref = run_oracle(WELL, 2, algorithm="preconditioned")
    got = run_gpu(WELL, 2, tol=TOL, algorithm=binding.PRECONDITIONED, nl_adapt=0.01, **prec(precision))
    for (ug, st), (uo, info) in zip(got, ref):
        assert rel(ug, uo) < 1e-10


def test_lh_blocks_match_oracle():
    w = WELL
    prob = oracle_problem(w)
    st = nls.Strips(prob, w.n_strips)
    X = st.strip_blocks(1)
    with binding.Solver(gpu_params(w, algorithm=binding.PRECONDITIONED, nl_tol=1e-14, psolve=binding.PSOLVE_GMRES),
                        w.u0(), w.V()) as s:
        B = s.blocks(1)
    for k in range(4):
        assert np.max(np.abs(B[k] - X[k])) < 1e-11 * max(1.0, np.max(np.abs(X[k])))


@pytest.mark.parametrize("bc", ["same", "neumann"])
def test_modal_diagonal_matches_oracle_blocks(bc):
    """The GPU's per-mode entries x1..x4 equal the diagonal of the oracle's L_h blocks (built by
    unit solves) in the cosine basis."""
    w = WELL
    prob = oracle_problem(w, bc=bc)
    st = nls.Strips(prob, w.n_strips)
    ny = w.ny
    j = np.arange(ny + 1)
    Z = np.cos(np.pi * np.outer(j, j) / ny)
    D = np.ones(ny + 1)
    D[0] = D[-1] = 0.5
    Zi = np.diag(1.0 / np.diag((Z.T * D) @ Z)) @ Z.T @ np.diag(D)
    kw = dict(algorithm=binding.PRECONDITIONED, psolve=binding.PSOLVE_MODAL,
              bc=binding.BC_NEUMANN if bc == "neumann" else binding.BC_SAME)
    with binding.Solver(gpu_params(w, **kw), w.u0(), w.V()) as s:
        for strip in (0, 1, w.n_strips - 1):
            xm = s.modal(strip)
            X = st.strip_blocks(strip)
            reg = st.regions[strip]
            for a in range(4):
                if (a in (0, 2) and reg.kind["l"] != "tc") or (a in (1, 3) and reg.kind["r"] != "tc"):
                    continue
                np.testing.assert_allclose(xm[a], np.diag(Zi @ X[a] @ Z), atol=1e-11)


@pytest.mark.parametrize("precision", [binding.FP64, binding.FP32_INNER])
def test_free_problem_converges_in_one_exact_preconditioned_update(precision):
    """V = 0, f = 0: R is affine with linear part L_h, so g^1 = g^0 - P^{-1}(g^0 - R g^0) is the
    fixed point when P^{-1} is exact (the modal solve): the second residual is at round-off."""
    w = wl.scaled(WELL, 40, 45, n_strips=5, potential="zero", kappa=0.0)
    got = run_gpu(w, 1, tol=1e-10, precision=precision, algorithm=binding.PRECONDITIONED,
                  psolve=binding.PSOLVE_MODAL)
    # the FP32 form applies the cosine transforms in FP32 (P^{-1} exact to ~1e-6)
    assert got[0][1]["last_schwarz_iterations"] == (2 if precision == binding.FP64 else 3)


@pytest.mark.parametrize("precision", [binding.FP64] + MIXED)
@pytest.mark.parametrize("algorithm", ["classical", "preconditioned"])
def test_pade_transmission_matches_oracle(precision, algorithm):
    """S_pade^m (eq. TCS) with its auxiliary unknowns phi_s (eq. TCS_phi), m = 4, theta = pi/4."""
    w = SMALL
    ref = run_oracle(w, 2, algorithm=algorithm, tc="pade", m=4)
    got = run_gpu(w, 2, tol=TOL, precision=precision, tc=binding.TC_PADE, pade_m=4,
                  algorithm=binding.PRECONDITIONED if algorithm == "preconditioned" else binding.CLASSICAL)
    bound = 1e-11 if precision == binding.FP64 else 1e-10
    for (ug, st), (uo, info) in zip(got, ref):
        assert rel(ug, uo) < bound
        assert abs(st["last_schwarz_iterations"] - info.iterations) <= 3


def test_pade_modal_diagonal_matches_oracle_blocks():
    w = wl.scaled(WELL, 24, 20, n_strips=4)
    prob = oracle_problem(w, tc="pade", m=3)
    st = nls.Strips(prob, w.n_strips)
    ny = w.ny
    j = np.arange(ny + 1)
    Z = np.cos(np.pi * np.outer(j, j) / ny)
    D = np.ones(ny + 1)
    D[0] = D[-1] = 0.5
    Zi = np.diag(1.0 / np.diag((Z.T * D) @ Z)) @ Z.T @ np.diag(D)
    X = st.strip_blocks(1)
    with binding.Solver(gpu_params(w, algorithm=binding.PRECONDITIONED, tc=binding.TC_PADE, pade_m=3), w.u0(), w.V()) as s:
        xm = s.modal(1)
    for a in range(4):
        np.testing.assert_allclose(xm[a], np.diag(Zi @ X[a] @ Z), atol=1e-11)


@pytest.mark.parametrize("form", ["classical", "preconditioned_adapt"])
def test_single_strip_is_the_monodomain_solve(form):
    """One strip has no interface: the step is the monodomain solve, also with the
    preconditioned algorithm and nl_adapt set (the inexact early solves need an interface)."""
    w = wl.scaled(SMALL, 20, 33, n_strips=1)
    prob = oracle_problem(w)
    u1, _, _ = nls.mono_step(prob, w.u0())
    kw = {} if form == "classical" else dict(algorithm=binding.PRECONDITIONED, nl_adapt=0.01)
    got = run_gpu(w, 1, tol=TOL, **kw)
    assert rel(got[0][0], u1) < 1e-11
    assert got[0][1]["schwarz_iterations"] == 1


@pytest.mark.parametrize("precision", [binding.FP64, binding.FP32_DW])
def test_one_cell_strips_and_ragged_rows(precision):
    w = wl.scaled(SMALL, 6, 1, n_strips=6, yb=0.0, yu=0.5)       # c = 1, ny = 1
    ref = run_oracle(w, 2)
    got = run_gpu(w, 2, tol=TOL, **prec(precision))
    for (ug, _), (uo, _) in zip(got, ref):
        assert rel(ug, uo) < (1e-11 if precision == binding.FP64 else 1e-10)


def test_double_word_residual_on_a_strongly_nonlinear_trap():
    """GPE in a harmonic trap, beta = 500 (the cubic term outweighs the stencil) with a far
    field below 1e-31, where the low word of a double-word value leaves FP32's normal range:
    the double-word residual reaches the oracle's step."""
    w = wl.Workload("gpe_far", -18.0, 18.0, -18.0, 18.0, 36, 30, 6, 0.002, 2, lap=0.5, kappa=-500.0, p=45.0,
                    potential="trap", datum="ground_noise", seed=1603)
    assert np.abs(w.u0()[:, :7]).max() < 1e-31       # the first strip (x in [-18, -12])
    ref = run_oracle(w, 2, algorithm="preconditioned", relax=0.6)
    got = run_gpu(w, 2, tol=TOL, algorithm=binding.PRECONDITIONED, **prec(binding.FP32_DW))
    for (ug, _), (uo, _) in zip(got, ref):
        assert rel(ug, uo) < 1e-10


@pytest.mark.parametrize("precision", [binding.FP64, binding.FP32_DW])
def test_neumann_mass_is_conserved_and_matches_oracle(precision):
    w = wl.scaled(SMALL, 36, 29, n_strips=3)
    ref = run_oracle(w, 3, bc="neumann")
    got = run_gpu(w, 3, tol=TOL, bc=binding.BC_NEUMANN, **prec(precision))
    prob = oracle_problem(w, bc="neumann")
    m0 = nls.mass(prob, w.u0())
    fp64 = precision == binding.FP64
    for (ug, st), (uo, _) in zip(got, ref):
        assert rel(ug, uo) < (1e-11 if fp64 else 1e-10)
        assert abs(st["mass"] / m0 - 1.0) < (1e-12 if fp64 else 1e-11)


def test_random_interface_guess_reaches_the_same_step():
    w = SMALL
    rng = np.random.default_rng(5)
    u0 = w.u0()
    n = 2 * (w.n_strips - 1)
    g_rand = rng.standard_normal((n, w.ny + 1)) + 1j * rng.standard_normal((n, w.ny + 1))
    va = np.zeros_like(u0)
    vb = np.zeros_like(u0)
    with binding.Solver(gpu_params(w, tol=1e-11), u0, w.V()) as s:
        s.solve_interface(None, None, va)
        s.solve_interface(np.ascontiguousarray(g_rand), None, vb)
    assert rel(vb, va) < 1e-10


def test_checkpoint_resume_is_bitwise():
    w = SMALL
    u0 = w.u0()
    full = np.zeros_like(u0)
    with binding.Solver(gpu_params(w, tol=TOL), u0, w.V()) as s:
        s.step(4, full)
    part = np.zeros_like(u0)
    g = np.zeros((2 * (w.n_strips - 1), w.ny + 1), np.complex128)
    with binding.Solver(gpu_params(w, tol=TOL), u0, w.V()) as s:
        s.step(2)
        n = s.get_state(part, g)
    with binding.Solver(gpu_params(w, tol=TOL), u0, w.V()) as s2:
        s2.set_state(part, g, n)
        out = np.zeros_like(u0)
        s2.step(2, out)
    assert np.array_equal(out, full)


def test_device_pointers_and_stream():
    w = SMALL
    dev = torch.device("cuda:0")
    u0 = torch.from_numpy(w.u0()).to(dev)
    V = torch.from_numpy(w.V()).to(dev)
    out = torch.empty_like(u0)
    stream = torch.cuda.Stream()
    with binding.Solver(gpu_params(w, tol=TOL), u0, V, stream=stream) as s:
        s.step(2, out)
    host = run_gpu(w, 2, tol=TOL)[-1][0]
    assert np.array_equal(out.cpu().numpy(), host)


def test_nonfinite_input_is_reported_not_committed():
    w = SMALL
    u0 = w.u0()
    u0[5, 7] = np.nan
    with binding.Solver(gpu_params(w), u0, w.V()) as s:
        with pytest.raises(binding.DDNLSError) as e:
            s.step(1)
        assert e.value.code == 5
        assert s.get_state() == 0


def test_iteration_cap_reports_enoconv():
    w = SMALL
    with binding.Solver(gpu_params(w, max_schwarz=2, tol=1e-14), w.u0(), w.V()) as s:
        with pytest.raises(binding.DDNLSError) as e:
            s.step(1)
        assert e.value.code == 4


def test_batched_uneven_instances_match_oracle():
    """Instances of different meshes, strip counts and nonlinearities stepped in one batch."""
    shapes = [(24, 20, 3, -120.0), (30, 17, 5, -400.0), (16, 33, 2, -900.0), (40, 41, 4, -250.0)]
    ws = [wl.Workload(f"b{i}", -4.0, 4.0, -4.0, 4.0, nx, ny, N, 0.002, 2, lap=0.5, kappa=k, p=45.0,
                      potential="trap", datum="ground_noise", seed=1603 + i)
          for i, (nx, ny, N, k) in enumerate(shapes)]
    prms = [gpu_params(w, tol=TOL) for w in ws]
    with binding.Batch(prms, [w.u0() for w in ws], [w.V() for w in ws]) as b:
        for step in range(2):
            st = b.step(1)
            for i, w in enumerate(ws):
                assert st[i]["steps"] == 1 and st[i]["schwarz_iterations"] > 0
        got = [b.get_u(i) for i in range(len(ws))]
        bs, nblk = b.tuning()
        assert bs in (128, 256) and nblk >= sum(w.n_strips for w in ws)
    for i, w in enumerate(ws):
        # beta = 900 at dt = 0.002: the plain fixed point diverges; both sides relax it
        ref = run_oracle(w, 2, relax=0.6)
        assert rel(got[i], ref[-1][0]) < 1e-11


@pytest.mark.parametrize("precision", [binding.FP64, binding.FP32_DW])
def test_batched_preconditioned_and_classical_instances_match_oracle(precision):
    """A batch mixing preconditioned instances (eq. algo_pd, modal P^-1 per instance, nl_adapt)
    with classical ones, in FP64 and in FP32 with the double-word residual (its fields carry the
    strip states between launches): every instance reaches the oracle's steps.  FP64 at interface
    tolerance 1e-12 agrees to 1e-11; the double-word form at 1e-10 (strip tolerance 1e-12) to 1e-8."""
    shapes = [(24, 20, 3, -120.0, "preconditioned"), (30, 17, 5, -400.0, "preconditioned"),
              (16, 33, 2, -250.0, "classical"), (40, 41, 4, -250.0, "preconditioned")]
    ws = [wl.Workload(f"bp{i}", -4.0, 4.0, -4.0, 4.0, nx, ny, N, 0.002, 2, lap=0.5, kappa=k, p=45.0,
                      potential="trap", datum="ground_noise", seed=1700 + i)
          for i, (nx, ny, N, k, _) in enumerate(shapes)]
    dw = precision == binding.FP32_DW
    tol = 1e-10 if dw else TOL
    prms = [gpu_params(w, tol=tol, nl_tol=1e-12 if dw else 1e-14, precision=precision, nl_adapt=0.01,
                       algorithm=binding.PRECONDITIONED if sh[4] == "preconditioned" else binding.CLASSICAL,
                       psolve=binding.PSOLVE_MODAL)
            for w, sh in zip(ws, shapes)]
    with binding.Batch(prms, [w.u0() for w in ws], [w.V() for w in ws]) as b:
        its = []
        for step in range(2):
            st = b.step(1)
            its.append([st[i]["last_schwarz_iterations"] for i in range(len(ws))])
        got = [b.get_u(i) for i in range(len(ws))]
    for i, (w, sh) in enumerate(zip(ws, shapes)):
        ref = run_oracle(w, 2, algorithm=sh[4], tol=tol)
        assert rel(got[i], ref[-1][0]) < (1e-8 if dw else 1e-11), (i, rel(got[i], ref[-1][0]))
        # the same Schwarz iteration counts as the oracle's, within the inexact early solves
        for step in range(2):
            assert abs(its[step][i] - ref[step][1].iterations) <= 2, (i, step, its, ref[step][1].iterations)


@pytest.mark.parametrize("case", ["well", "gpe_far", "pade_well"])
def test_double_word_state_carried_between_launches(case):
    """Strip tolerances of 1e-12 and above: the double-word fields carry the strip state from
    one Schwarz launch to the next (only the edge columns go back to FP64 in between, and the
    whole field at the end of the step).  Interface tolerance 1e-10, so the step agrees with
    the oracle's (solved to 1e-12) to 1e-8."""
    tc = {}
    if case == "well":
        w, relax = WELL, 1.0
    elif case == "pade_well":
        # S_pade: the edge nodes' phi coupling and the phi rows enter the double-word residual
        w, relax = WELL, 1.0
        tc = dict(tc="pade", m=4)
    else:
        w = wl.Workload("gpe_far", -18.0, 18.0, -18.0, 18.0, 36, 30, 6, 0.002, 2, lap=0.5, kappa=-500.0, p=45.0,
                        potential="trap", datum="ground_noise", seed=1603)
        relax = 0.6
    ref = run_oracle(w, 2, algorithm="preconditioned", relax=relax, **tc)
    extra = dict(tc=binding.TC_PADE, pade_m=4) if tc else {}
    got = run_gpu(w, 2, tol=1e-10, nl_tol=1e-12, algorithm=binding.PRECONDITIONED, precision=binding.FP32_DW, **extra)
    for (ug, _), (uo, _) in zip(got, ref):
        assert rel(ug, uo) < 1e-8


def test_fp32_inner_solves_survive_a_long_gpe_trajectory():
    """GPE trap, beta = 300, 256^2 cells, 8 strips: around step 105 the FP32 single-reduction
    COCG of one strip stalls (its alpha recurrence loses accuracy); the strip must fall back to the
    two-reduction loop and the run must track the plain FP64 one."""
    dt = 0.002
    w = wl.Workload("gpe_long", -12.0, 12.0, -12.0, 12.0, 256, 256, 8, dt, 110, lap=0.5, kappa=-300.0,
                    p=float(np.sqrt(4 / dt)), potential="trap", datum="ground_noise", seed=1603)
    outs = {}
    for precision in (binding.FP64, binding.FP32_DW):
        u0 = w.u0()
        out = np.zeros_like(u0)
        with binding.Solver(gpu_params(w, tol=1e-8, nl_tol=1e-11, max_schwarz=400, precision=precision), u0,
                            w.V()) as s:
            st = s.step(110, out)
        assert st["steps"] == 110
        outs[precision] = out
    assert rel(outs[binding.FP32_DW], outs[binding.FP64]) < 1e-6


@pytest.mark.parametrize("precision", MIXED)
@pytest.mark.parametrize("algorithm", ["classical", "preconditioned"])
def test_cluster_and_cooperative_layouts_reach_the_oracle_step(precision, algorithm):
    """FP32 Robin strips are solved one strip per thread-block cluster when they fit on chip
    (solver_layout 2, also the default) or by the cooperative launch (solver_layout 1); both reach
    the oracle's step."""
    w = WELL if algorithm == "preconditioned" else SMALL
    ref = run_oracle(w, 2, algorithm=algorithm)
    alg = binding.PRECONDITIONED if algorithm == "preconditioned" else binding.CLASSICAL
    for layout in (1, 2):
        got = run_gpu(w, 2, tol=TOL, algorithm=alg, precision=precision, solver_layout=layout)
        for (ug, _), (uo, _) in zip(got, ref):
            assert rel(ug, uo) < 1e-10, (layout, rel(ug, uo))


def test_cluster_layout_on_strips_wider_than_a_cta_slab():
    """A strip of 25 x 161 nodes: 11 rows per CTA of the cluster, ragged last CTA, and strips of
    256+ nodes take the on-chip single-reduction COCG."""
    w = wl.scaled(wl.NLS_WELL, 96, 160, n_strips=4, xl=-8.0, xr=8.0, yb=-9.0, yu=9.0, dt=0.02, p=3.0)
    ref = run_oracle(w, 2, algorithm="preconditioned")
    got = run_gpu(w, 2, tol=TOL, algorithm=binding.PRECONDITIONED, precision=binding.FP32_DW, solver_layout=2)
    for (ug, _), (uo, _) in zip(got, ref):
        assert rel(ug, uo) < 1e-10


def test_strips_too_large_for_a_cluster_fall_back_to_the_cooperative_layout():
    """A strip of 101 x 481 nodes needs 31 rows x 101 columns = 3131 nodes per CTA of a 16-CTA
    cluster at most 4608 (fits); one of 201 x 481 nodes (6231 per CTA) does not, so the default
    layout falls back to the cooperative launch and reproduces solver_layout 1 bit for bit."""
    w = wl.scaled(wl.NLS_WELL, 400, 480, n_strips=2, xl=-8.0, xr=8.0, yb=-9.0, yu=9.0, dt=0.02, p=3.0)
    a = run_gpu(w, 1, tol=1e-10, nl_tol=1e-12, algorithm=binding.PRECONDITIONED, precision=binding.FP32_DW,
                solver_layout=0)
    b = run_gpu(w, 1, tol=1e-10, nl_tol=1e-12, algorithm=binding.PRECONDITIONED, precision=binding.FP32_DW,
                solver_layout=1)
    assert np.array_equal(a[0][0], b[0][0])
    assert a[0][1]["last_schwarz_iterations"] == b[0][1]["last_schwarz_iterations"]
