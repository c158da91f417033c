// Host runtime and C-ABI of dd_nls (see include/dd_nls.h).
//
// One handle owns the device state of one problem: u_{n-1} and the strip fields in the
// strip layout of common.cuh, the interface vectors, the inner Krylov vectors of the batched
// strip solver, and (preconditioned algorithm) the L_h blocks and the GMRES basis.  A time
// step (eq. CNS) is: right side (2i/dt) M u_{n-1}; Schwarz iterations, each one persistent
// launch of the strip solver followed by the flux update of eq. (fluxlr) and the interface
// residual; for eq. (algo_pd) a GMRES solve of (I - L_h) x = g - R(g); then the commit
// u_n = 2v - u_{n-1} and the diagnostics.  The host reads a few scalars per Schwarz
// iteration to decide convergence.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dd_nls.h"
#include "common.cuh"
#include "kernels.h"
#include "host_pinned.h"
#include "params_check.h"

using namespace ddnls;
using cplx = std::complex<double>;

// Text of the last error of a call without a handle (a failed create, the no-allocation step),
// one buffer per host thread: threads that drive different GPUs do not share it.
static thread_local char g_create_error[512];

namespace ddnls {
void set_handle_free_error(const char* msg) { std::snprintf(g_create_error, sizeof g_create_error, "%s", msg); }
}  // namespace ddnls

struct dd_nls {
    dd_nls_params P{};
    Geom G{};
    cudaStream_t s = nullptr;
    bool fp32 = false;
    long long nfield = 0;   // elements of one strip field (all strips)
    long long nI = 0;       // elements of one interface vector (padded)
    int maxb = 1;           // co-resident blocks of the strip solver
    int chunks = 1;         // 256-node chunks of one strip (most blocks a strip can use)
    int* d_blk = nullptr;   // [maxb] block -> strip, then [maxb+1] strip -> first block
    int* h_blk = nullptr;   // pinned mirror
    double* bnorm0 = nullptr;   // [N] per-strip ||(2i/dt) M h||
    long long* pcyc = nullptr;  // [maxb][8] phase cycles of the strip solver
    PinnedVec<long long> h_pcyc;   // pinned: copies into it stay asynchronous
    std::vector<double> wts;    // scheduling weights
    // device state
    double2 *u = nullptr, *zeta = nullptr, *rhs0 = nullptr, *gA = nullptr, *gB = nullptr, *gconv = nullptr;
    double* Wn = nullptr;
    // rotating trap (time-dependent potential): the static part V/lap and the potential at t_n
    bool trap = false;
    double* Ws = nullptr;
    double* Wt = nullptr;
    int test_skip = 0;          // test hook: block + 1 that skips its first barrier arrival, once
    unsigned cl_smem = 0;       // cluster mode: dynamic shared memory per CTA (0: cooperative blocks)
    void *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *cT = nullptr;
    void *w1 = nullptr, *s0 = nullptr, *s1 = nullptr, *dv = nullptr;
    bool dw = false;        // double-word residual (FP32 inner, Robin)
    bool dw_res = false;    // the double-word fields hold the strip state of this step
    float4 *zdw = nullptr, *ddw = nullptr, *bdw = nullptr;
    float2* wdw = nullptr;
    double* bint2 = nullptr;
    double* part = nullptr;
    unsigned* bar = nullptr;
    int* status = nullptr;
    int* nl_its = nullptr;
    long long* kry = nullptr;
    double* nl_res = nullptr;
    int* err = nullptr;
    double* red = nullptr;           // small device results
    double2* stage = nullptr;        // nodal IO staging (global layout)
    // preconditioner
    int ntypes = 0;
    double2* X64 = nullptr;
    float2* X32 = nullptr;
    int* btype = nullptr;
    std::vector<int> btype_h;
    double2 *V = nullptr, *w = nullptr, *tmp = nullptr, *hdev = nullptr, *xs = nullptr;
    double2* cpart = nullptr;   // cosine-transform partial sums (modal P solve)
    double* scratch = nullptr;
    // S_pade^m (eq. TCS): coefficients and auxiliary unknowns
    int pade_m = 0;
    double2 pade_a[kMaxPade], pade_d[kMaxPade];
    double2 *pa_dev = nullptr, *pd_dev = nullptr, *phi = nullptr;
    void *xf = nullptr, *rf = nullptr, *zf = nullptr, *pf = nullptr, *qf = nullptr, *cTf = nullptr;
    // modal P solve
    double *Cf = nullptr, *Ci = nullptr;
    float *Cf32 = nullptr, *Ci32 = nullptr;
    double2 *xm = nullptr, *fac = nullptr;
    float2* fac32 = nullptr;    // FP32 copy of the per-mode factors (FP32 forms)
    int* tkind = nullptr;
    // host mirrors
    double* hred = nullptr;          // pinned
    PinnedVec<int> h_status, h_nl;  // pinned per-strip results (read after the one wait per launch)
    std::vector<int> cl_order;      // cluster order last copied to d_blk (empty: none)
    PinnedVec<long long> h_kry;
    int step = 0;
    bool have_prev = false;
    std::string error;
    bool prof = false;
    long long launch_base = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr, ev3 = nullptr;
    dd_nls_profile profile{};
    double setup_ms = 0.0;
};

#define CK(call)                                                                           \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) return fail(h, DD_NLS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

static int fail(dd_nls* h, int code, const std::string& msg) {
    if (h) h->error = msg; else set_handle_free_error(msg.c_str());
    return code;
}

extern "C" void dd_nls_default_params(dd_nls_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->xl = -1; p->xr = 1; p->yb = -1; p->yu = 1;
    p->nx = 32; p->ny = 32; p->n_strips = 2;
    p->dt = 0.01; p->lap = 1.0; p->kappa = 1.0;
    p->tc = DD_NLS_TC_ROBIN; p->p = 1.0; p->pade_m = 4; p->pade_theta = M_PI / 4;
    p->bc = DD_NLS_BC_SAME;
    p->algorithm = DD_NLS_CLASSICAL;
    p->precision = DD_NLS_FP64;
    p->guess = DD_NLS_GUESS_PREVIOUS;
    p->tol = 1e-10; p->tol_absolute = 0; p->max_schwarz = 500;
    p->nl_tol = 1e-13; p->max_nl = 300;
    p->inner_tol = 1e-6; p->max_inner = 2000;
    p->gmres_tol = 1e-10; p->gmres_restart = 30; p->gmres_max = 300;
    p->psolve = DD_NLS_PSOLVE_MODAL;
    p->nl_relax = 1.0;
    p->nl_adapt = 0.0;
    p->omega_rot = 0.0;
    p->trap_gx = p->trap_gy = 0.0;
    p->psolve_modes = 0;
    p->wait_limit_ms = 0.0;
    p->solver_layout = 0;
}

// Test hook: DD_NLS_TEST_FAIL_ALLOC=k makes the k-th device allocation of the next create fail
// (as cudaMalloc would when the device is full), so that the clean-up path can be tested.
static thread_local long long g_alloc_count = 0, g_alloc_fail_at = 0;

template <typename T> static cudaError_t dalloc(T** ptr, size_t n) {
    if (g_alloc_fail_at > 0 && ++g_alloc_count == g_alloc_fail_at) { *ptr = nullptr; return cudaErrorMemoryAllocation; }
    cudaError_t e = cudaMalloc((void**)ptr, std::max<size_t>(n, 1) * sizeof(T));
    if (e == cudaSuccess) e = cudaMemset(*ptr, 0, std::max<size_t>(n, 1) * sizeof(T));
    return e;
}

static void release(dd_nls* h) {
    void* ptrs[] = {h->u, h->zeta, h->rhs0, h->gA, h->gB, h->gconv, h->Wn, h->Ws, h->Wt, h->x, h->r, h->z, h->p, h->q, h->cT,
                    h->w1, h->s0, h->s1, h->dv, h->zdw, h->ddw, h->bdw, h->wdw, h->bint2,
                    h->part, h->bar, h->status, h->nl_its, h->kry, h->nl_res, h->err, h->red, h->stage,
                    h->X64, h->X32, h->btype, h->V, h->w, h->tmp, h->hdev, h->xs, h->scratch, h->cpart,
                    h->Cf, h->Ci, h->Cf32, h->Ci32, h->xm, h->fac, h->fac32, h->tkind,
                    h->pa_dev, h->pd_dev, h->phi, h->xf, h->rf, h->zf, h->pf, h->qf, h->cTf};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (h->hred) cudaFreeHost(h->hred);
    if (h->h_blk) cudaFreeHost(h->h_blk);
    if (h->d_blk) cudaFree(h->d_blk);
    if (h->bnorm0) cudaFree(h->bnorm0);
    if (h->pcyc) cudaFree(h->pcyc);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->ev2) cudaEventDestroy(h->ev2);
    if (h->ev3) cudaEventDestroy(h->ev3);
}

// Device time of a section of stream work, added to *acc when profiling is on.
struct ProfScope {
    dd_nls* h;
    double* acc;
    ProfScope(dd_nls* hh, double* a) : h(hh), acc(a) {
        if (h->prof) cudaEventRecord(h->ev2, h->s);
    }
    ~ProfScope() {
        if (!h->prof) return;
        cudaEventRecord(h->ev3, h->s);
        cudaEventSynchronize(h->ev3);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev2, h->ev3) == cudaSuccess) *acc += ms;
    }
};

// ------------------------------------------------------------------------ IO
static bool known_ptr_kind(int k) { return k == DD_NLS_PTR_HOST || k == DD_NLS_PTR_DEVICE; }
static int upload_nodal(dd_nls* h, const double* src, int ptr_kind, double2* strips) {
    const size_t bytes = (size_t)(h->G.nx + 1) * h->G.nyn * sizeof(double2);
    CK(cudaMemcpyAsync(h->stage, src, bytes, ptr_kind == DD_NLS_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->s));
    CK(launch_scatter_u(h->G, h->stage, strips, h->s));
    return DD_NLS_OK;
}
static int download_nodal(dd_nls* h, const double2* strips, double* dst, int ptr_kind) {
    const size_t bytes = (size_t)(h->G.nx + 1) * h->G.nyn * sizeof(double2);
    CK(launch_gather_u(h->G, strips, h->stage, h->s));
    CK(cudaMemcpyAsync(dst, h->stage, bytes, ptr_kind == DD_NLS_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->s));
    return DD_NLS_OK;
}
// interface vectors cross the ABI unpadded: 2(N-1) traces of nyn nodes
static int upload_g(dd_nls* h, const double* src, int ptr_kind, double2* dst) {
    const int ntr = 2 * (h->G.N - 1);
    if (ntr == 0) return DD_NLS_OK;
    CK(cudaMemcpy2DAsync(dst, h->G.P * sizeof(double2), src, h->G.nyn * sizeof(double2), h->G.nyn * sizeof(double2), ntr,
                         ptr_kind == DD_NLS_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->s));
    return DD_NLS_OK;
}
static int download_g(dd_nls* h, const double2* src, double* dst, int ptr_kind) {
    const int ntr = 2 * (h->G.N - 1);
    if (ntr == 0) return DD_NLS_OK;
    CK(cudaMemcpy2DAsync(dst, h->G.nyn * sizeof(double2), src, h->G.P * sizeof(double2), h->G.nyn * sizeof(double2), ntr,
                         ptr_kind == DD_NLS_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->s));
    return DD_NLS_OK;
}

// --------------------------------------------------------------- strip solves
// Blocks per strip for the next launch: at least one each, the rest of the co-resident
// blocks in proportion to the weights, at most `cap` per strip.  Fills the pinned table
// (block -> strip, then strip -> first block), copies it to the device, returns the total.
static int schedule(dd_nls* h, const std::vector<double>& w, int nstrips, int cap, StripSolveArgs& a) {
    double W = 0.0;
    for (int j = 0; j < nstrips; ++j) W += w[j];
    const int spare = std::max(0, h->maxb - nstrips);
    int* bs = h->h_blk;                       // block -> strip
    int* st = h->h_blk + h->maxb;             // strip -> first block
    int total = 0;
    for (int j = 0; j < nstrips; ++j) {
        int n = 1 + (W > 0.0 ? (int)std::floor(spare * (w[j] / W)) : spare / nstrips);
        n = std::max(1, std::min(n, cap));
        st[j] = total;
        for (int k = 0; k < n; ++k) bs[total + k] = j;
        total += n;
    }
    st[nstrips] = total;
    cudaMemcpyAsync(h->d_blk, h->h_blk, sizeof(int) * (h->maxb + nstrips + 1), cudaMemcpyHostToDevice, h->s);
    h->cl_order.clear();                      // the device table no longer holds a cluster order
    a.blk_strip = h->d_blk;
    a.blk_start = h->d_blk + h->maxb;
    return total;
}

// Enqueue one strip-solver launch and the copies of its per-strip results (no host wait).
// Cluster mode: one cluster per strip, heaviest strips first (the hardware starts clusters in
// launch order, so strips that need corrections are not left for a second wave).
static int schedule_clusters(dd_nls* h, const std::vector<double>& w, int nstrips, StripSolveArgs& a) {
    std::vector<int> order(nstrips);
    for (int j = 0; j < nstrips; ++j) order[j] = j;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return w[x] > w[y]; });
    // the copy is skipped when the device already holds this order (the usual case from one
    // Schwarz iteration to the next)
    if (order != h->cl_order) {
        for (int j = 0; j < nstrips; ++j) h->h_blk[j] = order[j];
        cudaMemcpyAsync(h->d_blk, h->h_blk, sizeof(int) * nstrips, cudaMemcpyHostToDevice, h->s);
        h->cl_order = order;
    }
    a.blk_strip = h->d_blk;
    a.blk_start = nullptr;
    a.cluster = 1;
    a.cluster_smem = h->cl_smem;
    return nstrips;
}

// blocks a launch of nblocks (strips in cluster mode) actually runs
static int physical_blocks(const StripSolveArgs& a, int nblocks) { return a.cluster ? nblocks * kClusterCTAs : nblocks; }

static int strip_solve_enqueue(dd_nls* h, StripSolveArgs& a, int nstrips, int nblocks) {
    CK(cudaMemsetAsync(h->bar, 0, sizeof(unsigned) * nstrips, h->s));
    CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->s));
    a.pcyc = h->prof ? h->pcyc : nullptr;
    a.test_skip_arrival = h->test_skip <= physical_blocks(a, nblocks) ? h->test_skip : 0;
    h->test_skip = 0;
    if (h->prof) CK(cudaEventRecord(h->ev0, h->s));
    CK(launch_strip_solve(a, nblocks, h->fp32, h->s));
    if (h->prof)
        CK(cudaMemcpyAsync(h->h_pcyc.data(), h->pcyc, sizeof(long long) * 8 * physical_blocks(a, nblocks),
                           cudaMemcpyDeviceToHost, h->s));
    if (h->prof) CK(cudaEventRecord(h->ev1, h->s));
    CK(cudaMemcpyAsync(h->h_status.data(), h->status, sizeof(int) * nstrips, cudaMemcpyDeviceToHost, h->s));
    CK(cudaMemcpyAsync(h->h_nl.data(), h->nl_its, sizeof(int) * nstrips, cudaMemcpyDeviceToHost, h->s));
    CK(cudaMemcpyAsync(h->h_kry.data(), h->kry, sizeof(long long) * nstrips, cudaMemcpyDeviceToHost, h->s));
    CK(cudaMemcpyAsync(h->hred + 8, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->s));
    return DD_NLS_OK;
}

// Wait for the stream, then account for and check the launch enqueued last.
static int strip_solve_finish(dd_nls* h, const StripSolveArgs& a, int nstrips, int nblocks, dd_nls_stats* st,
                              bool count) {
    CK(cudaStreamSynchronize(h->s));
    long long nl = 0, kr = 0;
    double bytes = 0.0, flops = 0.0;
    const double nodes = (double)h->G.nxs * h->G.nyn;
    const double s2 = h->fp32 ? 8.0 : 16.0, s1 = h->fp32 ? 4.0 : 8.0;
    // per node: residual phase (r, c and D^-1 only, when the single-reduction loop follows), one Krylov
    // iteration (two passes, or the fused pass of the single-reduction loop), its w_0 = A z_0
    // pass, the epilogue
    const bool sr = h->fp32 && h->pade_m == 0;
    const double bR = 40 + s1 + (sr ? 2 : 5) * s2, bK = sr ? 11 * s2 + s1 : 12 * s2 + 2 * s1;
    // double-word residual: the epilogue updates zeta and the accumulated correction in
    // double-word form; once per launch a set-up pass (zeta, rhs0, W in; four double-word
    // fields out) and the FP64 write-back (correction and zeta in, zeta out)
    // (dw_mode 1: set-up only, edge columns written back; dw_mode 2: edge columns only)
    const bool dw = h->dw;
    const int dm = dw ? a.dw_mode : 0;
    const double bW = sr ? 6 * s2 + s1 : 0.0, bE = !dw ? 32 + s2 : (dm == 0 ? 64 + s2 : 32 + s2);
    const double bL = !dw ? 0.0 : (dm == 0 ? 96 + 48 : (dm == 1 ? 80 : 0.0));
    for (int j = 0; j < nstrips; ++j) {
        nl += h->h_nl[j];
        kr += h->h_kry[j];
        bytes += nodes * (bL + (h->h_nl[j] + 1) * bR + h->h_kry[j] * bK + h->h_nl[j] * (bW + bE));
        flops += nodes * ((h->h_nl[j] + 1) * 110.0 + h->h_kry[j] * 150.0);
    }
    if (h->prof) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
        h->profile.strip_solve_ms += ms;
        h->profile.strip_solve_launches += 1;
        h->profile.strip_solve_bytes += bytes;
        h->profile.strip_solve_flops += flops;
        const int nb = physical_blocks(a, nblocks);
        for (int k = 0; k < 5; ++k) {
            double sum = 0.0;
            for (int b = 0; b < nb; ++b) sum += (double)h->h_pcyc[(size_t)b * 8 + k];
            h->profile.phase_cycles[k] += sum / nb;
        }
    }
    if (st && count) {
        st->nl_iterations += nl;
        st->krylov_iterations += kr;
    }
    int errw = 0;
    std::memcpy(&errw, h->hred + 8, sizeof(int));
    if (errw) return fail(h, errw, "strip solver: device barrier timed out");
    for (int j = 0; j < nstrips; ++j)
        if (h->h_status[j]) {
            char buf[160];
            std::snprintf(buf, sizeof buf, "strip solver: strip %d status %d after %d nonlinear / %lld Krylov iterations",
                          j, h->h_status[j], h->h_nl[j], h->h_kry[j]);
            return fail(h, h->h_status[j], buf);
        }
    return DD_NLS_OK;
}

static StripSolveArgs base_args(dd_nls* h) {
    StripSolveArgs a{};
    a.g = h->G;
    a.mode = 0;
    a.bnorm0 = h->bnorm0;
    a.zeta = h->zeta;
    a.rhs0 = h->rhs0;
    a.Wn = h->Wn;
    a.x = h->x; a.r = h->r; a.z = h->z; a.p = h->p; a.q = h->q; a.cT = h->cT;
    a.w1 = h->w1; a.s0 = h->s0; a.s1 = h->s1; a.dv = h->dv;
    a.zdw = h->zdw; a.ddw = h->ddw; a.bdw = h->bdw; a.wdw = h->wdw; a.bint2 = h->bint2;
    a.nl_tol = h->P.nl_tol;
    a.inner_tol = h->P.inner_tol;
    a.inner_floor = 0.1 * h->P.nl_tol;
    a.bscale = h->red + 8;
    a.nl_floor_frac = 0.01 * h->P.nl_tol / std::sqrt((double)h->G.N);
    a.max_nl = h->P.max_nl;
    a.max_inner = h->P.max_inner;
    a.nl_relax = h->P.nl_relax;
    a.nl_picard = h->P.nl_picard;
    a.part = h->part;
    a.bar = h->bar;
    a.status = h->status;
    a.nl_its = h->nl_its;
    a.kry_its = h->kry;
    a.nl_res = h->nl_res;
    a.err = h->err;
    a.wait_ns = (unsigned long long)(h->P.wait_limit_ms > 0.0 ? h->P.wait_limit_ms * 1e6 : 2e9);
    a.pcyc = nullptr;
    a.pade_m = h->pade_m;
    a.phi = h->phi;
    a.xf = h->xf; a.rf = h->rf; a.zf = h->zf; a.pf = h->pf; a.qf = h->qf; a.cTf = h->cTf;
    for (int s2 = 0; s2 < h->pade_m; ++s2) { a.pade_a[s2] = h->pade_a[s2]; a.pade_d[s2] = h->pade_d[s2]; }
    // edge coefficient: i p (Robin) or i sum_s a_s (S_pade)
    double rre = 0.0, rim = h->G.p;
    if (h->pade_m) {
        double sre = 0.0, sim = 0.0;
        for (int s2 = 0; s2 < h->pade_m; ++s2) { sre += h->pade_a[s2].x; sim += h->pade_a[s2].y; }
        rre = -sim;
        rim = sre;
    }
    fill_fp32_constants(a, rre, rim, h->G.hy);
    return a;
}

// ----------------------------------------------------------------- L_h setup
// Columns of L_h from free strip solves with unit data (Sec. 4.2): for every strip type
// (edge kinds), 2(ny+1) independent solves batched as virtual strips of one launch.
// Strip types (edge kinds: transmission or Neumann on each side).  Equal strips of one type
// share their L_h blocks (Props 3.1/3.2).
static int strip_types(dd_nls* h, std::vector<std::pair<int, int>>& types) {
    const Geom& G = h->G;
    types.clear();
    h->btype_h.assign(G.N, 0);
    for (int j = 0; j < G.N; ++j) {
        const int l = (j > 0 || G.bc_same) ? 1 : 0, r = (j < G.N - 1 || G.bc_same) ? 1 : 0;
        auto key = std::make_pair(l, r);
        auto it = std::find(types.begin(), types.end(), key);
        if (it == types.end()) { types.push_back(key); h->btype_h[j] = (int)types.size() - 1; }
        else h->btype_h[j] = (int)(it - types.begin());
    }
    h->ntypes = (int)types.size();
    CK(dalloc(&h->btype, G.N));
    CK(cudaMemcpy(h->btype, h->btype_h.data(), sizeof(int) * G.N, cudaMemcpyHostToDevice));
    return DD_NLS_OK;
}

// Diagonal of L_h in the cosine basis and the per-mode block-Thomas factors of P (modal.cu).
static int build_modal(dd_nls* h) {
    const Geom& G = h->G;
    std::vector<std::pair<int, int>> types;
    int rc = strip_types(h, types);
    if (rc) return rc;
    const long long nn = (long long)G.nyn * G.nyn;
    std::vector<int> tk(2 * h->ntypes);
    for (int t = 0; t < h->ntypes; ++t) { tk[2 * t] = types[t].first; tk[2 * t + 1] = types[t].second; }
    CK(dalloc(&h->tkind, tk.size()));
    CK(cudaMemcpy(h->tkind, tk.data(), sizeof(int) * tk.size(), cudaMemcpyHostToDevice));
    CK(dalloc(&h->Cf, nn));
    CK(dalloc(&h->Ci, nn));
    if (h->fp32) { CK(dalloc(&h->Cf32, nn)); CK(dalloc(&h->Ci32, nn)); }
    CK(dalloc(&h->xm, (size_t)h->ntypes * 4 * G.nyn));
    CK(dalloc(&h->fac, (size_t)9 * std::max(1, G.N - 1) * G.nyn));
    CK(dalloc(&h->tmp, (size_t)h->nI));
    CK(dalloc(&h->xs, (size_t)h->nI));
    CK(dalloc(&h->cpart, (size_t)8 * h->nI));
    double2* work = nullptr;
    CK(cudaMalloc(&work, sizeof(double2) * (size_t)h->ntypes * G.nyn * 2 * G.nxs));
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    cudaEventRecord(t0, h->s);
    cudaError_t e = launch_modal_setup(G, h->ntypes, h->tkind, h->btype, h->Cf, h->Ci, h->Cf32, h->Ci32, h->xm, h->fac,
                                       work, h->s, h->pade_m, h->pa_dev, h->pd_dev);
    if (e == cudaSuccess && h->fp32) {
        const size_t nf = (size_t)9 * std::max(1, G.N - 1) * G.nyn;
        e = cudaMalloc(&h->fac32, nf * sizeof(float2));
        if (e == cudaSuccess) e = launch_to_float((const double*)h->fac, (float*)h->fac32, 2 * (long long)nf, h->s);
    }
    cudaEventRecord(t1, h->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    h->setup_ms = ms;
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaFree(work);
    if (e != cudaSuccess) return fail(h, DD_NLS_ECUDA, std::string("modal set-up: ") + cudaGetErrorString(e));
    return DD_NLS_OK;
}

static int build_Lh(dd_nls* h) {
    const Geom& G = h->G;
    const int nyn = G.nyn;
    const long long bs = (long long)nyn * nyn;
    std::vector<std::pair<int, int>> types;
    int rc0 = strip_types(h, types);
    if (rc0) return rc0;
    CK(dalloc(&h->X64, (size_t)h->ntypes * 4 * bs));

    // virtual-strip buffers
    const int maxb = strip_solve_max_blocks(h->fp32);
    const long long per_strip = (long long)G.nxs * G.P;
    const double bytes_per_strip = (double)per_strip * (16 + 9 * (h->fp32 ? 8 : 16) + (h->fp32 ? 4 : 8));
    int chunk = std::max(1, std::min(maxb, (int)std::min(2.0 * nyn, 6e9 / bytes_per_strip)));
    StripSolveArgs a = base_args(h);
    double2* vz = nullptr;
    void *vx = nullptr, *vr = nullptr, *vzz = nullptr, *vp = nullptr, *vq = nullptr, *vc = nullptr;
    void *vw1 = nullptr, *vs0 = nullptr, *vs1 = nullptr, *vdv = nullptr;
    unsigned* vbar = nullptr;
    int *vstat = nullptr, *vnl = nullptr;
    long long* vkry = nullptr;
    double *vres = nullptr, *vpart = nullptr;
    const size_t s2 = h->fp32 ? sizeof(float2) : sizeof(double2), s1 = h->fp32 ? sizeof(float) : sizeof(double);
    int rc = DD_NLS_OK;
    auto cleanup = [&]() {
        void* ptrs[] = {vz, vx, vr, vzz, vp, vq, vc, vw1, vs0, vs1, vdv, vbar, vstat, vnl, vkry, vres, vpart};
        for (void* p : ptrs)
            if (p) cudaFree(p);
    };
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaMalloc(&vz, chunk * per_strip * sizeof(double2));
    e = e ? e : cudaMalloc(&vx, chunk * per_strip * s2);
    e = e ? e : cudaMalloc(&vr, chunk * per_strip * s2);
    e = e ? e : cudaMalloc(&vzz, chunk * per_strip * s2);
    e = e ? e : cudaMalloc(&vp, chunk * per_strip * s2);
    e = e ? e : cudaMalloc(&vq, chunk * per_strip * s2);
    e = e ? e : cudaMalloc(&vc, chunk * per_strip * s1);
    e = e ? e : cudaMalloc(&vw1, chunk * per_strip * s2);
    e = e ? e : cudaMalloc(&vs0, chunk * per_strip * s2);
    e = e ? e : cudaMalloc(&vs1, chunk * per_strip * s2);
    e = e ? e : cudaMalloc(&vdv, chunk * per_strip * s2);
    e = e ? e : cudaMalloc(&vbar, chunk * sizeof(unsigned));
    e = e ? e : cudaMalloc(&vstat, chunk * sizeof(int));
    e = e ? e : cudaMalloc(&vnl, chunk * sizeof(int));
    e = e ? e : cudaMalloc(&vkry, chunk * sizeof(long long));
    e = e ? e : cudaMalloc(&vres, chunk * sizeof(double));
    e = e ? e : cudaMalloc(&vpart, (size_t)4 * maxb * 4 * sizeof(double));
    if (e != cudaSuccess) { cleanup(); return fail(h, DD_NLS_ENOMEM, std::string("L_h setup buffers: ") + cudaGetErrorString(e)); }
    std::vector<int> hs(chunk), hn(chunk);
    std::vector<long long> hk(chunk);

    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    cudaEventRecord(t0, h->s);
    for (int t = 0; t < h->ntypes && rc == DD_NLS_OK; ++t) {
        const int u0 = types[t].first ? 0 : nyn, u1 = types[t].second ? 2 * nyn : nyn;
        for (int ub = u0; ub < u1 && rc == DD_NLS_OK; ub += chunk) {
            const int nv = std::min(chunk, u1 - ub);
            std::vector<double> wu(nv, 1.0);
            const int nblk = schedule(h, wu, nv, h->chunks, a);
            a.bnorm0 = nullptr;
            a.mode = 1;
            a.unit_base = ub;
            a.unit_ltc = types[t].first;
            a.unit_rtc = types[t].second;
            a.zeta = vz; a.rhs0 = nullptr; a.Wn = nullptr; a.gtr = nullptr; a.bscale = nullptr;
            a.x = vx; a.r = vr; a.z = vzz; a.p = vp; a.q = vq; a.cT = vc;
            a.w1 = vw1; a.s0 = vs0; a.s1 = vs1; a.dv = vdv;
            a.zdw = a.ddw = a.bdw = nullptr; a.wdw = nullptr;     // unit-datum solves: FP64 residual
            a.bar = vbar; a.status = vstat; a.nl_its = vnl; a.kry_its = vkry; a.nl_res = vres; a.part = vpart;
            e = cudaMemsetAsync(vz, 0, nv * per_strip * sizeof(double2), h->s);
            if (!e) e = cudaMemsetAsync(vbar, 0, nv * sizeof(unsigned), h->s);
            if (!e) e = cudaMemsetAsync(h->err, 0, sizeof(int), h->s);
            if (!e) e = launch_strip_solve(a, nblk, h->fp32, h->s);
            if (!e) e = launch_extract_blocks(G, vz, nv, ub, h->X64 + (long long)t * 4 * bs, h->s);
            if (!e) e = cudaMemcpyAsync(hs.data(), vstat, nv * sizeof(int), cudaMemcpyDeviceToHost, h->s);
            if (!e) e = cudaStreamSynchronize(h->s);
            if (e) { rc = fail(h, DD_NLS_ECUDA, std::string("L_h setup: ") + cudaGetErrorString(e)); break; }
            for (int v = 0; v < nv; ++v)
                if (hs[v]) { rc = fail(h, hs[v], "L_h setup: free strip solve failed"); break; }
        }
    }
    cudaEventRecord(t1, h->s);
    cudaEventSynchronize(t1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    h->setup_ms = ms;
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cleanup();
    if (rc) return rc;
    if (h->fp32) {
        CK(dalloc(&h->X32, (size_t)h->ntypes * 4 * bs));
        CK(launch_convert_blocks(h->X64, h->X32, (long long)h->ntypes * 4 * bs, h->s));
        CK(cudaStreamSynchronize(h->s));
    }
    // GMRES workspace
    const int m = std::max(1, h->P.gmres_restart);
    CK(dalloc(&h->V, (size_t)(m + 1) * h->nI));
    CK(dalloc(&h->w, (size_t)h->nI));
    CK(dalloc(&h->tmp, (size_t)h->nI));
    CK(dalloc(&h->xs, (size_t)h->nI));
    CK(dalloc(&h->hdev, (size_t)(m + 1)));
    CK(dalloc(&h->scratch, (size_t)(m + 2) * 256 * 2));
    return DD_NLS_OK;
}

// y = (I - L_h) x
static int apply_P(dd_nls* h, const double2* x, double2* y) {
    CK(launch_apply_P(h->G, h->fp32 ? (const void*)h->X32 : (const void*)h->X64, h->fp32, h->btype, x, y, nullptr, h->s));
    return DD_NLS_OK;
}

// Solve (I - L_h) x = b by restarted GMRES(m) (Sec. 4.2).  Krylov vectors and products live
// on the device; the (m+1) x m Hessenberg least-squares problem is updated on the host with
// Givens rotations from the few scalars read back per iteration.
static int gmres(dd_nls* h, const double2* b, double2* x, long long* its_out) {
    const long long n = h->nI;
    const int m = std::max(1, h->P.gmres_restart);
    double* hn = h->hred;                                   // pinned scratch
    CK(cudaMemsetAsync(x, 0, n * sizeof(double2), h->s));
    CK(launch_nrm2(b, n, h->red, h->scratch, h->s));
    CK(cudaMemcpyAsync(hn, h->red, sizeof(double), cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    const double bnorm = hn[0];
    long long its = 0;
    if (!(bnorm > 0.0)) { *its_out = 0; return std::isfinite(bnorm) ? DD_NLS_OK : fail(h, DD_NLS_ENONFINITE, "GMRES: non-finite right side"); }
    std::vector<cplx> H((m + 1) * m), cs(m), sn(m), gv(m + 1), hcol(m + 1);
    bool first = true;
    while (its < h->P.gmres_max) {
        // r = b - P x
        if (first) { CK(launch_copy(h->w, b, n, h->s)); }
        else { int rc = apply_P(h, x, h->tmp); if (rc) return rc; CK(launch_sub(h->w, b, h->tmp, n, h->s)); }
        CK(launch_nrm2(h->w, n, h->red, h->scratch, h->s));
        CK(cudaMemcpyAsync(hn, h->red, sizeof(double), cudaMemcpyDeviceToHost, h->s));
        CK(cudaStreamSynchronize(h->s));
        const double beta = hn[0];
        if (beta <= h->P.gmres_tol * bnorm) break;
        CK(launch_scale(h->V, h->w, h->red, n, h->s));
        std::fill(gv.begin(), gv.end(), cplx(0));
        gv[0] = beta;
        int k = 0;
        bool done = false;
        for (; k < m && its < h->P.gmres_max; ++k) {
            double2* vk = h->V + (long long)k * n;
            { int rc = apply_P(h, vk, h->w); if (rc) return rc; }
            // classical Gram-Schmidt, twice
            CK(launch_dots(h->V, n, k + 1, h->w, n, h->hdev, h->scratch, h->s));
            CK(launch_axpy_multi(h->V, n, k + 1, h->hdev, h->w, n, h->s));
            CK(cudaMemcpyAsync(hn, h->hdev, sizeof(double2) * (k + 1), cudaMemcpyDeviceToHost, h->s));
            CK(cudaStreamSynchronize(h->s));
            for (int i = 0; i <= k; ++i) hcol[i] = cplx(hn[2 * i], hn[2 * i + 1]);
            CK(launch_dots(h->V, n, k + 1, h->w, n, h->hdev, h->scratch, h->s));
            CK(launch_axpy_multi(h->V, n, k + 1, h->hdev, h->w, n, h->s));
            CK(launch_nrm2(h->w, n, h->red, h->scratch, h->s));
            CK(cudaMemcpyAsync(hn, h->hdev, sizeof(double2) * (k + 1), cudaMemcpyDeviceToHost, h->s));
            CK(cudaMemcpyAsync(hn + 2 * (m + 1), h->red, sizeof(double), cudaMemcpyDeviceToHost, h->s));
            CK(cudaStreamSynchronize(h->s));
            for (int i = 0; i <= k; ++i) hcol[i] += cplx(hn[2 * i], hn[2 * i + 1]);
            const double hk1 = hn[2 * (m + 1)];
            if (hk1 > 0.0) CK(launch_scale(h->V + (long long)(k + 1) * n, h->w, h->red, n, h->s));
            ++its;
            // Givens rotations on the new column
            for (int i = 0; i < k; ++i) {
                const cplx t = std::conj(cs[i]) * hcol[i] + std::conj(sn[i]) * hcol[i + 1];
                hcol[i + 1] = -sn[i] * hcol[i] + cs[i] * hcol[i + 1];
                hcol[i] = t;
            }
            const double a = std::abs(hcol[k]);
            const double rr = std::hypot(a, hk1);
            if (rr == 0.0) { cs[k] = 1; sn[k] = 0; }
            else {
                cs[k] = hcol[k] / rr;
                sn[k] = cplx(hk1 / rr, 0.0);
            }
            hcol[k] = rr;
            for (int i = 0; i <= k; ++i) H[i * m + k] = hcol[i];
            gv[k + 1] = -sn[k] * gv[k];
            gv[k] = std::conj(cs[k]) * gv[k];
            if (!std::isfinite(std::abs(gv[k + 1]))) return fail(h, DD_NLS_ENONFINITE, "GMRES: non-finite iterate");
            if (std::abs(gv[k + 1]) <= h->P.gmres_tol * bnorm || hk1 == 0.0) { ++k; done = true; break; }
        }
        // y = H^{-1} g, x += V y
        std::vector<cplx> y(k);
        for (int i = k - 1; i >= 0; --i) {
            cplx s = gv[i];
            for (int l = i + 1; l < k; ++l) s -= H[i * m + l] * y[l];
            y[i] = s / H[i * m + i];
        }
        std::vector<double> ny(2 * k);
        for (int i = 0; i < k; ++i) { ny[2 * i] = -y[i].real(); ny[2 * i + 1] = -y[i].imag(); }
        CK(cudaMemcpyAsync(h->hdev, ny.data(), sizeof(double2) * k, cudaMemcpyHostToDevice, h->s));
        CK(launch_axpy_multi(h->V, n, k, h->hdev, x, n, h->s));
        CK(cudaStreamSynchronize(h->s));
        first = false;
        if (done) break;
    }
    *its_out = its;
    return DD_NLS_OK;
}

// ------------------------------------------------------------- Schwarz step
// Runs the iteration of the current step from the interface vector in h->gA.
// On success h->zeta holds v and h->gconv the converged R(g).
// Trap at the rotating-frame nodes: w0 trap(t0) + w1 trap(t1) added to the static V/lap.
static TrapArgs trap_args(const dd_nls* h, double t0, double w0, double t1, double w1) {
    TrapArgs t{};
    t.gx2 = h->P.trap_gx * h->P.trap_gx;
    t.gy2 = h->P.trap_gy * h->P.trap_gy;
    t.inv_lap = 1.0 / h->P.lap;
    t.c0 = std::cos(h->P.omega_rot * t0); t.s0 = std::sin(h->P.omega_rot * t0); t.w0 = w0;
    t.c1 = std::cos(h->P.omega_rot * t1); t.s1 = std::sin(h->P.omega_rot * t1); t.w1 = w1;
    return t;
}

static int schwarz(dd_nls* h, dd_nls_stats* st) {
    const Geom& G = h->G;
    if (h->trap) {         // W_n = (V(t_n) + V(t_{n-1}))/2 of eq. (CNS) for the step being solved
        ProfScope ps(h, &h->profile.other_ms);
        const double tn = (h->step + 1) * h->P.dt, tp = h->step * h->P.dt;
        CK(launch_trap_potential(G, h->Ws, h->Wn, trap_args(h, tp, 0.5, tn, 0.5), h->s));
    }
    {
        ProfScope ps(h, &h->profile.other_ms);
        int nb = 1;
        CK(launch_rhs0(G, h->u, h->rhs0, h->part, &nb, h->s));
        CK(launch_finalize(h->part, nb, 1, h->red + 8, h->s));
        CK(launch_sqrt(h->red + 8, h->s));
        CK(cudaMemcpyAsync(h->zeta, h->u, h->nfield * sizeof(double2), cudaMemcpyDeviceToDevice, h->s));   // zeta^0 = h
        h->dw_res = false;
        if (h->pade_m)        // phi^0 = 0 (eq. localpbS2p)
            CK(cudaMemsetAsync(h->phi, 0, sizeof(double2) * (size_t)G.N * 2 * h->pade_m * G.P, h->s));
        CK(launch_strip_norms(G, h->rhs0, h->bnorm0, h->part, 16 * h->maxb, h->s));
        CK(cudaMemcpyAsync(h->hred + 16, h->bnorm0, sizeof(double) * G.N, cudaMemcpyDeviceToHost, h->s));
        CK(cudaStreamSynchronize(h->s));
    }
    // First launch of the step: weight strips by their share of the right side (a strip that
    // holds nothing of the solution converges at once); later launches: by the work the
    // previous launch of this step did.  Nothing carries over from earlier steps, so a
    // restored checkpoint reproduces the same schedule and bitwise the same results.
    double bmax = 0.0;
    for (int j = 0; j < G.N; ++j) bmax = std::max(bmax, h->hred[16 + j]);
    h->wts.assign(G.N, 1.0);
    for (int j = 0; j < G.N; ++j) h->wts[j] = 1.0 + (bmax > 0.0 ? 15.0 * std::sqrt(h->hred[16 + j] / bmax) : 0.0);
    StripSolveArgs a = base_args(h);
    double2* g = h->gA;
    double2* gn = h->gB;
    double rel_prev = 1.0;
    // nl_adapt > 0 with the preconditioned algorithm: inexact strip solves while the interface
    // residual is large (nl_adapt x the last relative residual, at most 1e-6, down to nl_tol);
    // same fixed point, cheaper early iterations.  The classical algorithm contracts too slowly
    // (0.98-0.99 per iteration) to absorb that perturbation.  An iteration that does not cut the
    // interface residual by 4x ends the inexact solves for the rest of the step (strongly
    // nonlinear strips can stall the preconditioned iteration at the inexact solves' level).
    // A single strip has no interface: its one solve is the step, at nl_tol.
    bool adapt = G.N > 1 && h->P.algorithm == DD_NLS_PRECONDITIONED && h->P.nl_adapt > 0.0;
    for (int k = 0; k < h->P.max_schwarz; ++k) {
        a.gtr = g;
        const double tol_k = adapt ? std::max(h->P.nl_tol, std::min(1e-6, h->P.nl_adapt * rel_prev)) : h->P.nl_tol;
        a.nl_tol = tol_k;
        a.inner_floor = 0.1 * tol_k;
        a.nl_floor_frac = 0.01 * tol_k / std::sqrt((double)G.N);
        // double-word residual: while the strip tolerance stays at or above its resolution the
        // double-word fields carry the strip state from launch to launch; a tighter launch
        // first returns the state to zeta (FP64) and finishes in FP64
        a.dw_mode = 0;
        if (h->dw) {
            if (tol_k >= kDWFinish) {
                a.dw_mode = h->dw_res ? 2 : 1;
            } else if (h->dw_res) {
                CK(launch_dw_to_zeta(G, h->zdw, h->zeta, h->s));
                h->dw_res = false;
            }
        }
        const int nblk = h->cl_smem ? schedule_clusters(h, h->wts, G.N, a) : schedule(h, h->wts, G.N, h->chunks, a);
        // the trace exchange is enqueued behind the strip solve, so one host wait covers both
        int rc = strip_solve_enqueue(h, a, G.N, nblk);
        if (rc) return rc;
        int nb = 1;
        if (G.N > 1) {
            ProfScope ps(h, &h->profile.interface_ms);
            CK(launch_traces(G, h->zeta, g, gn, h->part, &nb, h->s, h->pade_m, h->phi, h->pa_dev, h->pd_dev));
            CK(launch_finalize(h->part, nb, 2, h->red, h->s));
            CK(cudaMemcpyAsync(h->hred, h->red, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->s));
        } else {
            h->hred[0] = h->hred[1] = 0.0;
        }
        rc = strip_solve_finish(h, a, G.N, nblk, st, true);
        if (rc) return rc;
        if (a.dw_mode) h->dw_res = true;
        for (int j = 0; j < G.N; ++j) h->wts[j] = 1.0 + (double)h->h_kry[j] + 4.0 * (h->h_nl[j] + 1);
        const double diff = std::sqrt(h->hred[0]), nrm = std::sqrt(h->hred[1]);
        const double rel = nrm > 0.0 ? diff / nrm : diff;
        if (st) {
            st->schwarz_iterations += 1;
            st->last_schwarz_iterations = k + 1;
            st->residual = rel;
            st->residual_abs = diff;
        }
        if (!std::isfinite(diff) || !std::isfinite(nrm)) return fail(h, DD_NLS_ENONFINITE, "interface residual is not finite");
        const bool stalled = adapt && k > 0 && rel > 0.25 * rel_prev;
        rel_prev = rel;
        // converged only once the strip solves behind R(g) were at full accuracy
        if ((h->P.tol_absolute ? diff : rel) <= h->P.tol && (!adapt || tol_k <= std::max(h->P.nl_tol, h->P.nl_adapt * h->P.tol))) {
            if (h->dw_res) {
                CK(launch_dw_to_zeta(G, h->zdw, h->zeta, h->s));
                h->dw_res = false;
            }
            if (G.N > 1) CK(cudaMemcpyAsync(h->gconv, gn, h->nI * sizeof(double2), cudaMemcpyDeviceToDevice, h->s));
            h->gA = g;
            h->gB = gn;
            return DD_NLS_OK;
        }
        if (h->P.algorithm == DD_NLS_CLASSICAL) {
            std::swap(g, gn);                     // g^{k+1} = R(g^k)
        } else {
            // g^{k+1} = g^k - P^{-1} (g^k - R(g^k))  (eq. algo_pd)
            ProfScope ps(h, &h->profile.interface_ms);
            if (h->P.psolve == DD_NLS_PSOLVE_MODAL) {
                CK(launch_modal_update(G, h->fp32, h->Cf, h->Ci, h->Cf32, h->Ci32, h->fac, h->fac32, g, gn, gn, h->tmp,
                                       h->cpart, h->P.psolve_modes, h->s));
            } else {
                CK(launch_sub(h->tmp, g, gn, h->nI, h->s));
                CK(launch_copy(gn, h->tmp, h->nI, h->s));          // gn := y
                long long its = 0;
                rc = gmres(h, gn, h->xs, &its);
                if (rc) return rc;
                if (st) st->gmres_iterations += its;
                CK(launch_sub(gn, g, h->xs, h->nI, h->s));
            }
            std::swap(g, gn);
        }
        if (stalled) adapt = false;
    }
    h->gA = g;
    h->gB = gn;
    if (h->dw_res) {
        CK(launch_dw_to_zeta(G, h->zdw, h->zeta, h->s));
        h->dw_res = false;
    }
    return fail(h, DD_NLS_ENOCONV, "Schwarz iteration reached max_schwarz");
}

static int load_guess(dd_nls* h, const double* g0, int ptr_kind) {
    if (h->G.N < 2) return DD_NLS_OK;
    if (g0) return upload_g(h, g0, ptr_kind, h->gA);
    if (h->P.guess == DD_NLS_GUESS_PREVIOUS && h->have_prev)
        CK(cudaMemcpyAsync(h->gA, h->gconv, h->nI * sizeof(double2), cudaMemcpyDeviceToDevice, h->s));
    else
        CK(cudaMemsetAsync(h->gA, 0, h->nI * sizeof(double2), h->s));
    return DD_NLS_OK;
}

// Mass, energy (potential at t_n), <u, L_z u> and the energy of eq. (GPE) of the current u_n.
static int diagnostics(dd_nls* h, dd_nls_stats* st) {
    ProfScope ps(h, &h->profile.other_ms);
    int nb = 1;
    const double* W = h->Wn;
    if (h->trap) {
        const double tn = h->step * h->P.dt;
        CK(launch_trap_potential(h->G, h->Ws, h->Wt, trap_args(h, tn, 1.0, tn, 0.0), h->s));
        W = h->Wt;
    }
    CK(launch_diagnostics(h->G, h->u, W, h->part, &nb, h->s));
    CK(launch_lz(h->G, h->u, h->part, nb, 2, h->s));
    CK(launch_finalize(h->part, nb, 3, h->red, h->s));
    CK(cudaMemcpyAsync(h->hred, h->red, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    if (st) {
        st->mass = h->hred[0];
        st->energy = h->hred[1];
        st->lz = h->hred[2];
        st->energy_lab = h->P.lap * h->hred[1] - h->P.omega_rot * h->hred[2];
    }
    return DD_NLS_OK;
}

// ------------------------------------------------------------------- C-ABI
extern "C" int dd_nls_create(const dd_nls_params* p, const double* V, const double* u0, int ptr_kind, void* stream,
                             dd_nls** out) {
    set_handle_free_error("");
    {
        const char* fa = std::getenv("DD_NLS_TEST_FAIL_ALLOC");
        g_alloc_count = 0;
        g_alloc_fail_at = fa ? std::atoll(fa) : 0;
    }
    if (!p || !u0 || !out) return fail(nullptr, DD_NLS_EINVAL, "dd_nls_create: NULL params, u0 or out");
    *out = nullptr;
    if (const char* why = params_problem(*p)) return fail(nullptr, DD_NLS_EINVAL, std::string("dd_nls_create: ") + why);
    if (p->tc == DD_NLS_TC_PADE && p->algorithm == DD_NLS_PRECONDITIONED && p->psolve == DD_NLS_PSOLVE_GMRES)
        return fail(nullptr, DD_NLS_EINVAL, "dd_nls_create: S_pade with the preconditioned algorithm uses the modal P solve");
    if (ptr_kind != DD_NLS_PTR_HOST && ptr_kind != DD_NLS_PTR_DEVICE)
        return fail(nullptr, DD_NLS_EINVAL, "dd_nls_create: unknown ptr_kind");
    const long long c = p->nx / p->n_strips;
    const long long nyn = (long long)p->ny + 1;

    dd_nls* h = new dd_nls();
    h->P = *p;
    if (h->P.max_schwarz < 1) h->P.max_schwarz = 1;
    if (h->P.gmres_restart < 1) h->P.gmres_restart = 30;
    h->s = (cudaStream_t)stream;
    h->fp32 = p->precision != DD_NLS_FP64;
    h->dw = p->precision == DD_NLS_FP32_DW;
    Geom& G = h->G;
    G.N = p->n_strips;
    G.nxs = (int)c + 1;
    G.nyn = (int)nyn;
    G.P = (int)((nyn + 31) / 32 * 32);
    G.hx = (p->xr - p->xl) / p->nx;
    G.hy = (p->yu - p->yb) / p->ny;
    G.alpha = 2.0 / (p->lap * p->dt);
    G.kap = p->kappa / p->lap;
    G.p = p->p;
    G.bc_same = p->bc == DD_NLS_BC_SAME;
    G.nx = p->nx;
    G.xl = p->xl;
    G.yb = p->yb;
    G.fill_coefficients();
    h->nfield = (long long)G.N * G.nxs * G.P;
    h->trap = p->trap_gx > 0.0 || p->trap_gy > 0.0;
    h->nI = std::max<long long>(1, (long long)2 * (G.N - 1) * G.P);

    auto bad = [&](int code) {
        std::string m = h->error;
        release(h);
        delete h;
        set_handle_free_error(m.c_str());
        g_alloc_fail_at = 0;
        return code;
    };
#define CKC(call)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) {                                                                    \
            h->error = std::string(#call) + ": " + cudaGetErrorString(e_);                         \
            return bad(e_ == cudaErrorMemoryAllocation ? DD_NLS_ENOMEM : DD_NLS_ECUDA);             \
        }                                                                                           \
    } while (0)
    const size_t s2 = h->fp32 ? sizeof(float2) : sizeof(double2), s1 = h->fp32 ? sizeof(float) : sizeof(double);
    CKC(dalloc(&h->u, h->nfield));
    CKC(dalloc(&h->zeta, h->nfield));
    CKC(dalloc(&h->rhs0, h->nfield));
    CKC(dalloc(&h->Wn, h->nfield));
    if (h->trap) {
        CKC(dalloc(&h->Ws, h->nfield));
        CKC(dalloc(&h->Wt, h->nfield));
    }
    CKC(dalloc(&h->gA, h->nI));
    CKC(dalloc(&h->gB, h->nI));
    CKC(dalloc(&h->gconv, h->nI));
    CKC(dalloc((char**)&h->x, h->nfield * s2));
    CKC(dalloc((char**)&h->r, h->nfield * s2));
    CKC(dalloc((char**)&h->z, h->nfield * s2));
    CKC(dalloc((char**)&h->p, h->nfield * s2));
    CKC(dalloc((char**)&h->q, h->nfield * s2));
    CKC(dalloc((char**)&h->cT, h->nfield * s1));
    CKC(dalloc((char**)&h->w1, h->nfield * s2));
    CKC(dalloc((char**)&h->s0, h->nfield * s2));
    CKC(dalloc((char**)&h->s1, h->nfield * s2));
    CKC(dalloc((char**)&h->dv, h->nfield * s2));
    if (h->dw) {
        CKC(dalloc(&h->zdw, h->nfield));
        CKC(dalloc(&h->ddw, h->nfield));
        CKC(dalloc(&h->bdw, h->nfield));
        CKC(dalloc(&h->wdw, h->nfield));
        CKC(dalloc(&h->bint2, G.N));
    }
    CKC(dalloc(&h->stage, (size_t)(p->nx + 1) * nyn));
    CKC(dalloc(&h->bar, G.N));
    CKC(dalloc(&h->status, G.N));
    CKC(dalloc(&h->nl_its, G.N));
    CKC(dalloc(&h->kry, G.N));
    CKC(dalloc(&h->nl_res, G.N));
    CKC(dalloc(&h->err, 1));
    CKC(dalloc(&h->red, 64));
    CKC(cudaMallocHost((void**)&h->hred, (size_t)(256 + p->n_strips) * sizeof(double)));
    CKC(cudaEventCreate(&h->ev0));
    CKC(cudaEventCreate(&h->ev1));
    CKC(cudaEventCreate(&h->ev2));
    CKC(cudaEventCreate(&h->ev3));
    if (!h->h_status.resize(G.N) || !h->h_nl.resize(G.N) || !h->h_kry.resize(G.N)) {
        h->error = "dd_nls_create: pinned host memory for the per-strip results";
        return bad(DD_NLS_ENOMEM);
    }

    // launch shape of the strip solver: all blocks co-resident, blocks split among strips per launch
    const int maxb = strip_solve_max_blocks(h->fp32);
    if (maxb < G.N) { h->error = "dd_nls_create: more strips than co-resident blocks of the strip solver"; return bad(DD_NLS_EINVAL); }
    h->maxb = maxb;
    h->chunks = (int)((G.nxs * (long long)G.nyn + 255) / 256);
    // cluster mode: FP32 Robin strips whose slab of one CTA fits on chip
    if (h->fp32 && p->tc == DD_NLS_TC_ROBIN && p->solver_layout != 1) {
        const unsigned sm = strip_cluster_smem(G.nxs, G.nyn);
        if (sm && strip_cluster_capacity(h->dw, sm) >= 1) h->cl_smem = sm;
    }
    const int maxphys = std::max(maxb, G.N * kClusterCTAs);
    CKC(dalloc(&h->part, (size_t)4 * maxb * 4));
    CKC(dalloc(&h->d_blk, (size_t)2 * maxb + 2));
    CKC(cudaMallocHost((void**)&h->h_blk, sizeof(int) * (2 * maxb + 2)));
    CKC(dalloc(&h->bnorm0, G.N));
    CKC(dalloc(&h->pcyc, (size_t)8 * maxphys));
    if (p->tc == DD_NLS_TC_PADE) {
        // a_s = e^{i theta/2} / (m cos^2 phi_s), d_s = e^{i theta} tan^2 phi_s, phi_s = (2s-1) pi/(4m),
        // s = 1..m (eq. TCS; the sums start at s = 1)
        const int m = p->pade_m;
        h->pade_m = m;
        for (int k = 1; k <= m; ++k) {
            const double ph = (2.0 * k - 1.0) * M_PI / (4.0 * m);
            const double ca = 1.0 / (m * std::cos(ph) * std::cos(ph)), tn = std::tan(ph) * std::tan(ph);
            h->pade_a[k - 1] = make_double2(ca * std::cos(0.5 * p->pade_theta), ca * std::sin(0.5 * p->pade_theta));
            h->pade_d[k - 1] = make_double2(tn * std::cos(p->pade_theta), tn * std::sin(p->pade_theta));
        }
        CKC(dalloc(&h->pa_dev, m));
        CKC(dalloc(&h->pd_dev, m));
        CKC(cudaMemcpy(h->pa_dev, h->pade_a, sizeof(double2) * m, cudaMemcpyHostToDevice));
        CKC(cudaMemcpy(h->pd_dev, h->pade_d, sizeof(double2) * m, cudaMemcpyHostToDevice));
        const size_t nf = (size_t)G.N * 2 * m * G.P;
        CKC(dalloc(&h->phi, nf));
        CKC(dalloc((char**)&h->xf, nf * s2));
        CKC(dalloc((char**)&h->rf, nf * s2));
        CKC(dalloc((char**)&h->zf, nf * s2));
        CKC(dalloc((char**)&h->pf, nf * s2));
        CKC(dalloc((char**)&h->qf, nf * s2));
        CKC(dalloc((char**)&h->cTf, (size_t)G.N * 2 * G.P * s1));
    }
    if (!h->h_pcyc.assign((size_t)8 * maxphys, 0)) {
        h->error = "dd_nls_create: pinned host memory for the phase profile";
        return bad(DD_NLS_ENOMEM);
    }

    if (upload_nodal(h, u0, ptr_kind, h->u)) return bad(DD_NLS_ECUDA);
    if (V) {
        const size_t bytes = (size_t)(p->nx + 1) * nyn * sizeof(double);
        CKC(cudaMemcpyAsync(h->stage, V, bytes, ptr_kind == DD_NLS_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->s));
        CKC(launch_scatter_real(G, (const double*)h->stage, 1.0 / p->lap, h->Wn, h->s));
    }
    if (h->trap) CKC(cudaMemcpyAsync(h->Ws, h->Wn, h->nfield * sizeof(double), cudaMemcpyDeviceToDevice, h->s));
    CKC(cudaStreamSynchronize(h->s));
    if (p->algorithm == DD_NLS_PRECONDITIONED && G.N > 1) {
        if (p->psolve != DD_NLS_PSOLVE_GMRES && p->psolve != DD_NLS_PSOLVE_MODAL) {
            h->error = "dd_nls_create: unknown psolve";
            return bad(DD_NLS_EINVAL);
        }
        int rc = p->psolve == DD_NLS_PSOLVE_MODAL ? build_modal(h) : build_Lh(h);
        if (rc) return bad(rc);
    }
    {
        const char* sk = std::getenv("DD_NLS_TEST_SKIP_ARRIVAL");
        h->test_skip = sk ? std::max(0, std::atoi(sk)) : 0;
    }
    g_alloc_fail_at = 0;
    *out = h;
    return DD_NLS_OK;
#undef CKC
}

extern "C" int dd_nls_step(dd_nls* h, int nsteps, double* u_out, int ptr_kind, dd_nls_stats* st) {
    if (!h) return fail(nullptr, DD_NLS_EINVAL, "dd_nls_step: NULL handle");
    if (!known_ptr_kind(ptr_kind)) return fail(h, DD_NLS_EINVAL, "dd_nls_step: unknown ptr_kind");
    if (nsteps < 0) return fail(h, DD_NLS_EINVAL, "dd_nls_step: nsteps < 0");
    if (st) { std::memset(st, 0, sizeof(*st)); st->setup_ms = h->setup_ms; }
    for (int n = 0; n < nsteps; ++n) {
        int rc = load_guess(h, nullptr, ptr_kind);
        if (rc) return rc;
        rc = schwarz(h, st);
        if (rc) return rc;
        {
            ProfScope ps(h, &h->profile.other_ms);
            CK(launch_commit(h->G, h->zeta, h->u, h->s));
        }
        h->have_prev = true;
        h->step += 1;
        if (st) st->steps += 1;
    }
    if (st) {
        int rc = diagnostics(h, st);
        if (rc) return rc;
    }
    if (u_out) {
        int rc = download_nodal(h, h->u, u_out, ptr_kind);
        if (rc) return rc;
    }
    CK(cudaStreamSynchronize(h->s));
    return DD_NLS_OK;
}

extern "C" int dd_nls_step_guess(dd_nls* h, const double* g0, double* u_out, int ptr_kind, dd_nls_stats* st) {
    if (!h) return fail(nullptr, DD_NLS_EINVAL, "dd_nls_step_guess: NULL handle");
    if (!known_ptr_kind(ptr_kind)) return fail(h, DD_NLS_EINVAL, "dd_nls_step_guess: unknown ptr_kind");
    if (!g0) return fail(h, DD_NLS_EINVAL, "dd_nls_step_guess: NULL guess");
    if (st) { std::memset(st, 0, sizeof(*st)); st->setup_ms = h->setup_ms; }
    int rc = load_guess(h, g0, ptr_kind);
    if (rc) return rc;
    rc = schwarz(h, st);
    if (rc) return rc;
    {
        ProfScope ps(h, &h->profile.other_ms);
        CK(launch_commit(h->G, h->zeta, h->u, h->s));
    }
    h->have_prev = true;
    h->step += 1;
    if (st) { st->steps = 1; rc = diagnostics(h, st); if (rc) return rc; }
    if (u_out) { rc = download_nodal(h, h->u, u_out, ptr_kind); if (rc) return rc; }
    CK(cudaStreamSynchronize(h->s));
    return DD_NLS_OK;
}

extern "C" int dd_nls_solve_interface(dd_nls* h, const double* g0, double* g_out, double* v_out, int ptr_kind,
                                      dd_nls_stats* st) {
    if (!h) return fail(nullptr, DD_NLS_EINVAL, "dd_nls_solve_interface: NULL handle");
    if (!known_ptr_kind(ptr_kind)) return fail(h, DD_NLS_EINVAL, "dd_nls_solve_interface: unknown ptr_kind");
    if (st) { std::memset(st, 0, sizeof(*st)); st->setup_ms = h->setup_ms; }
    int rc = load_guess(h, g0, ptr_kind);
    if (rc) return rc;
    rc = schwarz(h, st);
    if (rc) return rc;
    if (g_out) { rc = download_g(h, h->gconv, g_out, ptr_kind); if (rc) return rc; }
    if (v_out) { rc = download_nodal(h, h->zeta, v_out, ptr_kind); if (rc) return rc; }
    CK(cudaStreamSynchronize(h->s));
    return DD_NLS_OK;
}

extern "C" int dd_nls_get_state(dd_nls* h, double* u, double* g, int* step, int ptr_kind) {
    if (!h) return fail(nullptr, DD_NLS_EINVAL, "dd_nls_get_state: NULL handle");
    if (!known_ptr_kind(ptr_kind)) return fail(h, DD_NLS_EINVAL, "dd_nls_get_state: unknown ptr_kind");
    if (u) { int rc = download_nodal(h, h->u, u, ptr_kind); if (rc) return rc; }
    if (g) { int rc = download_g(h, h->gconv, g, ptr_kind); if (rc) return rc; }
    if (step) *step = h->step;
    CK(cudaStreamSynchronize(h->s));
    return DD_NLS_OK;
}

extern "C" int dd_nls_set_state(dd_nls* h, const double* u, const double* g, int step, int ptr_kind) {
    if (!h) return fail(nullptr, DD_NLS_EINVAL, "dd_nls_set_state: NULL handle");
    if (!known_ptr_kind(ptr_kind)) return fail(h, DD_NLS_EINVAL, "dd_nls_set_state: unknown ptr_kind");
    if (u) { int rc = upload_nodal(h, u, ptr_kind, h->u); if (rc) return rc; }
    if (g) { int rc = upload_g(h, g, ptr_kind, h->gconv); if (rc) return rc; h->have_prev = true; }
    h->step = step;
    CK(cudaStreamSynchronize(h->s));
    return DD_NLS_OK;
}

extern "C" int dd_nls_get_blocks(dd_nls* h, int strip, double* x, int ptr_kind) {
    if (!h) return fail(nullptr, DD_NLS_EINVAL, "dd_nls_get_blocks: NULL handle");
    if (!known_ptr_kind(ptr_kind)) return fail(h, DD_NLS_EINVAL, "dd_nls_get_blocks: unknown ptr_kind");
    if (!h->X64 || strip < 0 || strip >= h->G.N || !x) return fail(h, DD_NLS_EINVAL, "dd_nls_get_blocks: no L_h or bad strip");
    const long long bs = (long long)h->G.nyn * h->G.nyn;
    CK(cudaMemcpyAsync(x, h->X64 + (long long)h->btype_h[strip] * 4 * bs, 4 * bs * sizeof(double2),
                       ptr_kind == DD_NLS_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    return DD_NLS_OK;
}

extern "C" int dd_nls_get_modal(dd_nls* h, int strip, double* x, int ptr_kind) {
    if (!h) return fail(nullptr, DD_NLS_EINVAL, "dd_nls_get_modal: NULL handle");
    if (!known_ptr_kind(ptr_kind)) return fail(h, DD_NLS_EINVAL, "dd_nls_get_modal: unknown ptr_kind");
    if (!h->xm || strip < 0 || strip >= h->G.N || !x) return fail(h, DD_NLS_EINVAL, "dd_nls_get_modal: no modal P or bad strip");
    CK(cudaMemcpyAsync(x, h->xm + (long long)h->btype_h[strip] * 4 * h->G.nyn, 4 * h->G.nyn * sizeof(double2),
                       ptr_kind == DD_NLS_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    return DD_NLS_OK;
}

extern "C" int dd_nls_lab_frame(dd_nls* h, int nx_out, int ny_out, double* out, int ptr_kind) {
    if (!h) return fail(nullptr, DD_NLS_EINVAL, "dd_nls_lab_frame: NULL handle");
    if (nx_out < 1 || ny_out < 1 || nx_out >= (1 << 30) || ny_out >= (1 << 30) || !out || !known_ptr_kind(ptr_kind))
        return fail(h, DD_NLS_EINVAL, "dd_nls_lab_frame: need 1 <= nx_out, ny_out < 2^30, an output and a known ptr_kind");
    const double t = h->step * h->P.dt, r = std::sqrt(2.0);
    const double c = std::cos(h->P.omega_rot * t), s = std::sin(h->P.omega_rot * t);
    const size_t n = (size_t)(nx_out + 1) * (ny_out + 1);
    double2* dst = (double2*)out;
    double2* tmp = nullptr;
    if (ptr_kind == DD_NLS_PTR_HOST) {
        cudaError_t e = cudaMalloc(&tmp, n * sizeof(double2));
        if (e != cudaSuccess) return fail(h, DD_NLS_ENOMEM, std::string("dd_nls_lab_frame: ") + cudaGetErrorString(e));
        dst = tmp;
    }
    cudaError_t e = launch_lab_frame(h->G, h->u, nx_out, ny_out, h->P.xl / r, h->P.xr / r, h->P.yb / r, h->P.yu / r,
                                     c, s, dst, h->s);
    if (e == cudaSuccess && tmp) e = cudaMemcpyAsync(out, tmp, n * sizeof(double2), cudaMemcpyDeviceToHost, h->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return fail(h, DD_NLS_ECUDA, std::string("dd_nls_lab_frame: ") + cudaGetErrorString(e));
    return DD_NLS_OK;
}

extern "C" int dd_nls_set_profiling(dd_nls* h, int on) {
    if (!h) return fail(nullptr, DD_NLS_EINVAL, "dd_nls_set_profiling: NULL handle");
    h->prof = on != 0;
    std::memset(&h->profile, 0, sizeof(h->profile));
    h->launch_base = kernel_launch_count();
    return DD_NLS_OK;
}

extern "C" int dd_nls_get_profile(dd_nls* h, dd_nls_profile* prof) {
    if (!h || !prof) return fail(h, DD_NLS_EINVAL, "dd_nls_get_profile: NULL argument");
    *prof = h->profile;
    prof->kernel_launches = h->prof ? kernel_launch_count() - h->launch_base : 0;
    return DD_NLS_OK;
}

extern "C" void dd_nls_destroy(dd_nls* h) {
    if (!h) return;
    if (h->s) cudaStreamSynchronize(h->s);
    release(h);
    delete h;
}

extern "C" const char* dd_nls_last_error(const dd_nls* h) {
    return h ? h->error.c_str() : g_create_error;
}
