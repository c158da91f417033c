// Host-side check of a dd_nls_params before any device work: sizes that the kernels' 32-bit
// strip indexing covers, every enum field one of its values, every real field finite and in
// its range.  Returns nullptr when the parameters are acceptable, else a message.
#pragma once
#include <cmath>

#include "../../include/dd_nls.h"
#include "kernels.h"

namespace ddnls {

inline const char* params_problem(const dd_nls_params& p) {
    if (p.nx < 1 || p.ny < 1 || p.n_strips < 1 || p.nx % p.n_strips != 0)
        return "need nx, ny >= 1 and nx a multiple of n_strips";
    const long long c = p.nx / p.n_strips, nyn = (long long)p.ny + 1;
    if (nyn > (1 << 20) || c + 1 > (1 << 20) || (c + 1) * nyn > (1LL << 30)) return "strip too large";
    const double reals[] = {p.xl, p.xr, p.yb, p.yu, p.dt, p.lap, p.kappa, p.p, p.pade_theta, p.tol, p.nl_tol,
                            p.inner_tol, p.gmres_tol, p.nl_relax, p.nl_adapt, p.omega_rot, p.trap_gx, p.trap_gy,
                            p.wait_limit_ms};
    for (double v : reals)
        if (!std::isfinite(v)) return "every real parameter must be finite";
    if (!(p.xr > p.xl) || !(p.yu > p.yb) || !(p.dt > 0) || !(p.lap > 0)) return "need xr > xl, yu > yb, dt > 0, lap > 0";
    if (p.tc != DD_NLS_TC_ROBIN && p.tc != DD_NLS_TC_PADE) return "unknown transmission condition";
    if (p.tc == DD_NLS_TC_ROBIN && !(p.p > 0.0)) return "Robin p must be > 0";
    if (p.tc == DD_NLS_TC_PADE && (p.pade_m < 1 || p.pade_m > kMaxPade)) return "Pade order m must be in 1..96";
    if (p.bc != DD_NLS_BC_SAME && p.bc != DD_NLS_BC_NEUMANN) return "unknown physical-edge condition bc";
    if (p.algorithm != DD_NLS_CLASSICAL && p.algorithm != DD_NLS_PRECONDITIONED) return "unknown algorithm";
    if (p.precision != DD_NLS_FP64 && p.precision != DD_NLS_FP32_INNER && p.precision != DD_NLS_FP32_DW)
        return "unknown precision";
    if (p.guess != DD_NLS_GUESS_ZERO && p.guess != DD_NLS_GUESS_PREVIOUS) return "unknown guess";
    if (p.psolve != DD_NLS_PSOLVE_GMRES && p.psolve != DD_NLS_PSOLVE_MODAL) return "unknown psolve";
    if (p.tol < 0 || p.nl_tol < 0 || p.inner_tol < 0 || p.gmres_tol < 0) return "tolerances must be >= 0";
    if (p.nl_adapt < 0 || p.trap_gx < 0 || p.trap_gy < 0 || p.wait_limit_ms < 0)
        return "need nl_adapt, trap_gx, trap_gy, wait_limit_ms >= 0";
    if (p.psolve_modes < 0 || p.solver_layout < 0 || p.solver_layout > 2) return "need psolve_modes >= 0, solver_layout 0, 1 or 2";
    return nullptr;
}

}  // namespace ddnls
