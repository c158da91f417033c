"""The oracle's pins catch plausible mistakes: each case plants one mistake (a flipped sign, a
dropped factor or weight, a wrong index or side, a transposed operand, a missing correction) in a
scratch copy of oracle/ on the CPU and runs one pin against that copy, which must fail.  A
control run of the same pins on an unchanged copy must pass, so the failures come from the
planted mistakes.  Nothing here touches the CUDA path."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PIN = "tests/test_oracle_pins.py::"
PADE = "tests/test_oracle_pade_energy.py::"
GPE = "tests/test_oracle_gpe.py::"

# name: (oracle file, [(text, planted text)], pin that must fail)
MUTATIONS = {
    # S_pade coupling of eq. (NproblemSPNL) / (TCSdist): sign of the phi terms
    "pade_phi_coupling_sign": (
        "nls.py",
        [("blocks[0][k] = (-1j * a[s] * d[s]) * (self.Q[e].T @ mg)",
          "blocks[0][k] = (1j * a[s] * d[s]) * (self.Q[e].T @ mg)"),
         ("out = out + 1j * self.a[s] * self.d[s] * phi[side][s]",
          "out = out - 1j * self.a[s] * self.d[s] * phi[side][s]")],
        PADE + "test_pade_outgoing_trace_is_minus_i_times_the_pade_sum_on_each_mode"),
    # Padé angles phi_s = (2s-1) pi / (4m) of eq. (TCS)
    "pade_angle_index": (
        "nls.py", [("ang = (2 * s - 1) * math.pi / (4 * m)", "ang = (2 * s) * math.pi / (4 * m)")],
        PIN + "test_pade_sum_approximates_sqrt"),
    # energy: kappa/2 in front of the quartic term
    "energy_quartic_coefficient": (
        "nls.py", [("e -= 0.5 * prob.kap * np.sum(reg.w * np.abs(uu) ** 4)",
                    "e -= 0.25 * prob.kap * np.sum(reg.w * np.abs(uu) ** 4)")],
        GPE + "test_energy_rotation_term_and_its_nls_part"),
    # flux update of eq. (fluxlr): sign of the incoming datum
    "flux_incoming_sign": (
        "nls.py", [('Rg[2 * (j - 1)] = -l + 2.0 * reg.trace_S(v, phi, "l")',
                    'Rg[2 * (j - 1)] = l + 2.0 * reg.trace_S(v, phi, "l")')],
        PIN + "test_equal_strips_have_equal_blocks_and_blocks_match_R"),
    # flux update: trace taken on the wrong edge
    "flux_trace_side": (
        "nls.py", [('Rg[2 * j + 1] = -r + 2.0 * reg.trace_S(v, phi, "r")',
                    'Rg[2 * j + 1] = -r + 2.0 * reg.trace_S(v, phi, "l")')],
        PIN + "test_equal_strips_have_equal_blocks_and_blocks_match_R"),
    # Robin term i p M^Gamma of eq. (NproblemRobinNL)
    "robin_sign": (
        "nls.py", [("A = A + (1j * p) * (self.Q[s].T @ sp.csr_matrix(self.mg) @ self.Q[s])",
                    "A = A + (-1j * p) * (self.Q[s].T @ sp.csr_matrix(self.mg) @ self.Q[s])")],
        PIN + "test_robin_mass_balance_is_exact"),
    # right side (2i/dt) M h: the factor of the midpoint scheme
    "rhs_time_factor": (
        "nls.py", [("b = (1j * self.prob.alpha) * (self.M @ h)", "b = (0.5j * self.prob.alpha) * (self.M @ h)")],
        PIN + "test_mass_conserved_with_closed_neumann_boundary"),
    # right side: sign of the interface data
    "rhs_data_sign": (
        "nls.py", [("b = b - self.Q[s].T @ (self.mg @ data)", "b = b + self.Q[s].T @ (self.mg @ data)")],
        PIN + "test_manufactured_plane_wave_second_order"),
    # nonlinear term without its quadrature weight (reading D3)
    "nonlinear_weight_dropped": (
        "nls.py", [("A = self.A + sp.diags(self.w * self.prob.kap * np.abs(zeta) ** 2)",
                    "A = self.A + sp.diags(self.prob.kap * np.abs(zeta) ** 2)")],
        PIN + "test_y_independent_data_reduce_to_1d_scheme"),
    # eigenvalues of the cosine modes
    "modal_eigenvalue_factor": (
        "nls.py", [("lam = (6.0 / hy ** 2) * (1.0 - np.cos(th)) / (2.0 + np.cos(th))",
                    "lam = (3.0 / hy ** 2) * (1.0 - np.cos(th)) / (2.0 + np.cos(th))")],
        PADE + "test_modal_entries_equal_the_unit_solve_blocks"),
    # L_h product of eq. (Lmpi): blocks applied to the wrong datum
    "lh_blocks_swapped": (
        "nls.py", [("y[2 * j + 1] += X3 @ l + X4 @ r", "y[2 * j + 1] += X4 @ l + X3 @ r")],
        PADE + "test_modal_P_solve_equals_gmres_on_the_assembled_blocks"),
    # Q1 stiffness: hx where hy belongs
    "stiffness_spacing_index": (
        "fem.py", [("ke[a, b] += (dxa * dxb / hx**2 + dya * dyb / hy**2) * jac",
                    "ke[a, b] += (dxa * dxb / hx**2 + dya * dyb / hx**2) * jac")],
        "tests/test_oracle_fem.py::test_q1_assembly_equals_kronecker"),
    # rotation A(t) of eq. (x1Ax) turned the other way
    "rotation_direction": (
        "gpe.py", [("return np.array([[c, s], [-s, c]])", "return np.array([[c, -s], [s, c]])")],
        GPE + "test_lab_frame_quarter_turn_of_a_smooth_field"),
    # L_z = -i (x d_y - y d_x): sign of the second term
    "angular_momentum_sign": (
        "gpe.py", [("Lu = -1j * (X * uy - Y * ux)", "Lu = -1j * (X * uy + Y * ux)")],
        GPE + "test_vortex_states_carry_angular_momentum_m"),
    # CNN: convolution instead of correlation (kernel flipped)
    "cnn_kernel_flipped": (
        "cnn.py", [('y += np.einsum("oc,chw->ohw", w[:, :, kh, kw], xp[:, kh:kh + H, kw:kw + W])',
                    'y += np.einsum("oc,chw->ohw", w[:, :, 2 - kh, 2 - kw], xp[:, kh:kh + H, kw:kw + W])')],
        "tests/test_oracle_cnn.py::test_conv_matches_scipy_correlate2d"),
    # Adam without the second-moment bias correction
    "adam_bias_correction_dropped": (
        "cnn.py", [("vh = v / (1.0 - b2 ** t)", "vh = v")],
        "tests/test_oracle_cnn.py::test_adam_steps_with_a_constant_gradient"),
}


def scratch_copy(dst):
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"),
                    ignore=shutil.ignore_patterns("__pycache__"))
    shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(dst, "tests"),
                    ignore=shutil.ignore_patterns("__pycache__", "golden"))
    golden = os.path.join(ROOT, "tests", "golden")
    if os.path.isdir(golden):
        shutil.copytree(golden, os.path.join(dst, "tests", "golden"))


def run_pins(cwd, pins):
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "not gpu", *pins]
    return subprocess.run(cmd, cwd=cwd, capture_output=True, text=True, timeout=600)


def test_the_pins_pass_on_an_unchanged_copy(tmp_path):
    scratch_copy(str(tmp_path))
    pins = sorted({m[2] for m in MUTATIONS.values()})
    r = run_pins(str(tmp_path), pins)
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_a_planted_mistake_fails_its_pin(tmp_path, name):
    fname, edits, pin = MUTATIONS[name]
    scratch_copy(str(tmp_path))
    path = os.path.join(str(tmp_path), "oracle", fname)
    src = open(path).read()
    for old, new in edits:
        assert src.count(old) == 1, f"{name}: the text to change is not in oracle/{fname} once"
        src = src.replace(old, new)
    with open(path, "w") as f:
        f.write(src)
    r = run_pins(str(tmp_path), [pin])
    assert r.returncode == 1, f"{name}: {pin} did not fail\n" + r.stdout[-2000:]
