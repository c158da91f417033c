"""The GPE in the rotating frame on the GPU (Sec. 5.2.1, eq. x1Ax, GPE_Trans, u1u) against the oracle.

* anisotropic rotating trap: every step solves with W_n = (V_n + V_{n-1})/2 of the rotated trap;
  the steps, <u, L_z u> and the energy of eq. (GPE) match the oracle's;
* an isotropic trap given as a rotating trap reproduces the static potential bit for bit;
* the lab-frame field on the valid zone matches the oracle's Q1 interpolation;
* the partially constructed I - L_h (only the lowest cosine modes solved) reaches the same step;
* the mass and the energy reported by the library match the oracle's formulas.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import gpe, nls  # noqa: E402
from paper_1603_05110_gb300 import binding, workloads as wl  # noqa: E402
from tests.helpers import gpu_params, oracle_problem, rel  # noqa: E402

pytestmark = pytest.mark.gpu

GX, GY, OMEGA = 1.0, 1.5, 0.7


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_05110_gb300 import build
    build.build()
    binding.load()


def trap_workload():
    return wl.Workload("rot", -6.0, 6.0, -6.0, 6.0, 48, 45, 3, 0.02, 3, lap=0.5, kappa=-8.0, p=10.0,
                       potential="zero", datum="ground_noise", seed=1603)


def oracle_rotating(w, steps, bc="same"):
    """Steps of the oracle with the step potential of the rotating trap (eq. Sch sign)."""
    base = oracle_problem(w, bc=bc)
    u = w.u0()
    g = None
    out = []
    for n in range(1, steps + 1):
        prob = nls.Problem(**{**base.__dict__, "V": gpe.step_potential(base, n, GX, GY, OMEGA)})
        u, _, info = nls.schwarz_step(prob, w.n_strips, u, g0=g, tol=1e-12)
        g = info.g
        out.append(u.copy())
    return base, out


@pytest.mark.parametrize("precision", [binding.FP64, binding.FP32_DW])
def test_anisotropic_rotating_trap_matches_oracle(precision):
    w = trap_workload()
    base, ref = oracle_rotating(w, 3)
    prm = gpu_params(w, tol=1e-12, precision=precision, trap_gx=GX, trap_gy=GY, omega_rot=OMEGA)
    u0 = w.u0()
    out = np.zeros_like(u0)
    with binding.Solver(prm, u0, None) as s:
        for n in range(1, 4):
            st = s.step(1, out)
            assert rel(out, ref[n - 1]) < (1e-11 if precision == binding.FP64 else 1e-10)
            t = n * w.dt
            V = gpe.trap_potential(base, t, GX, GY, OMEGA)
            lz = gpe.angular_momentum(base, out)
            e = gpe.energy_lab(nls.Problem(**{**base.__dict__, "V": V}), out, V, OMEGA)
            assert abs(st["lz"] - lz) < 1e-11 * max(1.0, abs(lz))
            assert abs(st["energy_lab"] - e) < 1e-11 * abs(e)
        lab = s.lab_frame(30, 24)
    want = gpe.lab_frame(base, out, 3 * w.dt, OMEGA, 30, 24)
    assert np.max(np.abs(lab - want)) < 1e-13 * np.max(np.abs(want))


def test_isotropic_rotating_trap_is_the_static_potential():
    w = trap_workload()
    base = oracle_problem(w)
    V = gpe.trap_potential(base, 0.0, 1.2, 1.2, 0.0)
    u0 = w.u0()
    a = np.zeros_like(u0)
    b = np.zeros_like(u0)
    with binding.Solver(gpu_params(w, tol=1e-12), u0, V) as s:
        s.step(2, a)
    with binding.Solver(gpu_params(w, tol=1e-12, trap_gx=1.2, trap_gy=1.2, omega_rot=0.9), u0, None) as s:
        st = s.step(2, b)
    assert rel(b, a) < 1e-13
    # an isotropic trap carries the rotation only in the energy: -omega <u, L_z u>
    assert abs(st["energy_lab"] - (0.5 * st["energy"] - 0.9 * st["lz"])) < 1e-13 * abs(st["energy_lab"])


def test_lab_frame_of_the_initial_state():
    w = trap_workload()
    base = oracle_problem(w)
    u0 = w.u0()
    with binding.Solver(gpu_params(w, omega_rot=OMEGA), u0, None) as s:
        lab = s.lab_frame(17, 11)
        dev = torch.empty(12, 18, dtype=torch.complex128, device="cuda:0")
        s.lab_frame(17, 11, dev)
    want = gpe.lab_frame(base, u0, 0.0, OMEGA, 17, 11)
    assert np.max(np.abs(lab - want)) < 1e-13
    assert np.array_equal(dev.cpu().numpy(), lab)


def test_partial_modal_preconditioner_reaches_the_same_step():
    w = wl.scaled(wl.NLS_WELL, 40, 45, n_strips=4, xl=-8.0, xr=8.0, yb=-8.0, yu=8.0, dt=0.02, p=3.0)
    prob = oracle_problem(w)
    ref, _, _ = nls.schwarz_step(prob, w.n_strips, w.u0(), algorithm="preconditioned", tol=1e-12, psolve="modal")
    its = {}
    for modes in (0, 8, 1):
        out = np.zeros_like(w.u0())
        with binding.Solver(gpu_params(w, tol=1e-12, algorithm=binding.PRECONDITIONED, psolve_modes=modes),
                            w.u0(), w.V()) as s:
            st = s.step(1, out)
        assert rel(out, ref) < 1e-11
        its[modes] = st["last_schwarz_iterations"]
    assert its[0] <= its[8] <= its[1]


@pytest.mark.parametrize("precision", [binding.FP64, binding.FP32_DW])
def test_reported_mass_and_energy_match_the_oracle(precision):
    w = wl.scaled(wl.NLS_SMALL, 36, 29, n_strips=3, xl=-6.0, xr=6.0, yb=-5.0, yu=5.0, dt=0.02)
    prob = oracle_problem(w, bc="neumann")
    out = np.zeros_like(w.u0())
    with binding.Solver(gpu_params(w, tol=1e-12, bc=binding.BC_NEUMANN, precision=precision), w.u0(), w.V()) as s:
        for _ in range(3):
            st = s.step(1, out)
            assert abs(st["mass"] - nls.mass(prob, out)) < 1e-13 * nls.mass(prob, out)
            e = nls.energy(prob, out)
            assert abs(st["energy"] - e) < 1e-12 * abs(e)
            assert abs(st["lz"] - gpe.angular_momentum(prob, out)) < 1e-12 * max(1.0, nls.mass(prob, out))
