// Batched instances: many independent problems (uneven meshes and strip counts) stepped
// together.  Every Schwarz iteration solves the strips of all instances that have not
// converged yet in ONE persistent launch of the strip solver (per-strip geometry from a
// descriptor table), then one launch of the batched flux update (eq. fluxlr) computes every
// instance's new interface vector and residual (one block per instance).  Each instance stops
// at its own tolerance; the blocks of the launch are split among the remaining strips by
// their expected work.  An autotuner picks the solver's block size (tile of nodes per block
// pass) and the number of co-resident blocks once per batch shape by timing the candidates on
// the first Schwarz iteration.
//
// Scope: Robin transmission (eq. TCSRobin); per instance the classical algorithm (eq. algo_d) or
// the preconditioned one (eq. algo_pd) with the exact P^-1 on cosine modes (Sec. 4.2; one set of
// modal factors per instance); one precision for the whole batch (FP64, FP32 inner with the
// FP64 residual, or FP32 inner with the double-word residual, whose fields then carry every
// strip's state from launch to launch within a step).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/dd_nls.h"
#include "common.cuh"
#include "kernels.h"
#include "host_pinned.h"
#include "params_check.h"

using namespace ddnls;

namespace ddnls {

// Flux update and interface residual of every active instance: block b = instance b.
// g_cur / g_new: interface vectors of all instances at offsets goff[b] (+ the other half of
// the ping-pong buffer); res[b] = (||gnew - g||^2, ||gnew||^2).
__global__ void batch_traces_kernel(const Geom* __restrict__ geoms, const long long* __restrict__ foff,
                                    const long long* __restrict__ goff, const int* __restrict__ cur,
                                    const int* __restrict__ active, long long half, const double2* __restrict__ zeta,
                                    double2* __restrict__ gbuf, double* __restrict__ res) {
    __shared__ double sm[64];
    const int b = blockIdx.x;
    if (!active[b]) return;
    const Geom g = geoms[b];
    const int c = g.nxs - 1;
    const double2* zb = zeta + foff[b];
    const double2* gc = gbuf + goff[b] + (cur[b] ? half : 0);
    double2* gn = gbuf + goff[b] + (cur[b] ? 0 : half);
    const long long total = (long long)(g.N - 1) * g.nyn;
    double v[2] = {0.0, 0.0};
    for (long long t = threadIdx.x; t < total; t += blockDim.x) {
        const int iy = (int)(t % g.nyn);
        const int i = (int)(t / g.nyn);
        const double2 zl = zb[(long long)((i + 1) * g.nxs + 0) * g.P + iy];
        const double2 zr = zb[(long long)(i * g.nxs + c) * g.P + iy];
        const double2 gr = gc[(long long)(2 * i) * g.P + iy];
        const double2 gl = gc[(long long)(2 * i + 1) * g.P + iy];
        const double2 nr = make_double2(-gl.x + 2.0 * g.p * zl.y, -gl.y - 2.0 * g.p * zl.x);
        const double2 nl = make_double2(-gr.x + 2.0 * g.p * zr.y, -gr.y - 2.0 * g.p * zr.x);
        gn[(long long)(2 * i) * g.P + iy] = nr;
        gn[(long long)(2 * i + 1) * g.P + iy] = nl;
        v[0] += (nr.x - gr.x) * (nr.x - gr.x) + (nr.y - gr.y) * (nr.y - gr.y)
              + (nl.x - gl.x) * (nl.x - gl.x) + (nl.y - gl.y) * (nl.y - gl.y);
        v[1] += nr.x * nr.x + nr.y * nr.y + nl.x * nl.x + nl.y * nl.y;
    }
    block_sum<2>(v, sm);
    if (threadIdx.x == 0) { res[2 * b] = v[0]; res[2 * b + 1] = v[1]; }
}

}  // namespace ddnls

struct TuneKey {
    int n, strips, fp32;
    long long nodes;
    bool operator<(const TuneKey& o) const {
        return std::tie(n, strips, fp32, nodes) < std::tie(o.n, o.strips, o.fp32, o.nodes);
    }
};
static std::map<TuneKey, std::pair<int, int>> g_tuned;     // shape -> (block size, blocks)
static std::mutex g_tune_mu;

struct dd_nls_batch {
    int n = 0;
    std::vector<dd_nls_params> P;
    std::vector<Geom> G;
    std::vector<StripInfo> sinfo;
    std::vector<int> strip_first;   // first strip of each instance in the launch numbering
    std::vector<long long> foff, goff;
    int nstrips = 0;
    long long nfield = 0, nI = 0;
    bool fp32 = false;
    cudaStream_t s = nullptr;
    Geom* d_geoms = nullptr;
    StripInfo* d_sinfo = nullptr;
    long long *d_foff = nullptr, *d_goff = nullptr;
    int *d_cur = nullptr, *d_active = nullptr;
    double2 *u = nullptr, *zeta = nullptr, *rhs0 = nullptr, *gbuf = nullptr;
    double* Wn = nullptr;
    void *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *cT = nullptr;
    void *w1 = nullptr, *s0 = nullptr, *s1 = nullptr, *dv = nullptr;
    double *part = nullptr, *bscale = nullptr, *bnorm0 = nullptr, *res = nullptr, *nl_res = nullptr;
    double* d_tol = nullptr;        // per-strip nonlinear tolerance of the next launch
    double* h_tol = nullptr;        // pinned mirror
    std::vector<double> rel_prev;   // last relative interface residual per instance
    unsigned* bar = nullptr;
    int *status = nullptr, *nl_its = nullptr, *err = nullptr, *d_blk = nullptr;
    long long* kry = nullptr;
    // pinned host mirrors
    int* h_blk = nullptr;
    int* h_cur = nullptr;
    int* h_active = nullptr;
    double* h_res = nullptr;
    double* h_bn = nullptr;
    PinnedVec<int> h_status, h_nl;  // pinned: copies into them stay asynchronous
    PinnedVec<long long> h_kry;
    std::vector<int> cur;           // ping-pong half holding each instance's current g
    std::vector<int> conv_half;     // half holding the converged R(g) of the last step
    std::vector<char> have_prev;
    int maxb = 1;                   // co-resident blocks for the chosen block size
    int bs = 256;                   // block size chosen by the autotuner
    int blocks = 1;                 // blocks per launch chosen by the autotuner
    bool tuned = false;
    bool prof = false;
    bool dw = false;                // double-word residual (FP32 inner)
    // exact P^-1 of a preconditioned instance (modal.cu): strip types, cosine transforms, the
    // per-mode block-Thomas factors, scratch
    struct Modal {
        int ntypes = 0;
        int *btype = nullptr, *tkind = nullptr;
        double *Cf = nullptr, *Ci = nullptr;
        float *Cf32 = nullptr, *Ci32 = nullptr;
        double2 *xm = nullptr, *fac = nullptr, *tmp = nullptr, *xs = nullptr, *cpart = nullptr;
        float2* fac32 = nullptr;
    };
    std::vector<Modal> modal;
    std::vector<double> tolk;       // strip tolerance of each instance in the next launch
    float4 *zdw = nullptr, *bdw = nullptr;   // double-word state and right side
    float2* wdw = nullptr;                   // w W in double words
    double* bint2 = nullptr;                 // ||b||^2 off the edges per strip
    double2* stage = nullptr;       // nodal staging buffer of the largest instance (host IO)
    long long launch_base = 0;
    dd_nls_profile profile{};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::string error;
};

static int bfail(dd_nls_batch* b, int code, const std::string& msg) {
    if (b) b->error = msg;
    else set_handle_free_error(msg.c_str());
    return code;
}
#define BCK(call)                                                                           \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) return bfail(b, e_ == cudaErrorMemoryAllocation ? DD_NLS_ENOMEM : DD_NLS_ECUDA, \
                                            std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <typename T> static cudaError_t zalloc(T** ptr, size_t n) {
    cudaError_t e = cudaMalloc((void**)ptr, std::max<size_t>(n, 1) * sizeof(T));
    if (e == cudaSuccess) e = cudaMemset(*ptr, 0, std::max<size_t>(n, 1) * sizeof(T));
    return e;
}

static void batch_release(dd_nls_batch* b) {
    void* dev[] = {b->d_geoms, b->d_sinfo, b->d_foff, b->d_goff, b->d_cur, b->d_active, b->u, b->zeta, b->rhs0,
                   b->gbuf, b->Wn, b->x, b->r, b->z, b->p, b->q, b->cT, b->w1, b->s0, b->s1, b->dv, b->part,
                   b->bscale, b->bnorm0, b->res,
                   b->nl_res, b->bar, b->status, b->nl_its, b->err, b->d_blk, b->kry, b->d_tol, b->stage};
    for (void* p : dev)
        if (p) cudaFree(p);
    for (auto& m : b->modal) {
        void* md[] = {m.btype, m.tkind, m.Cf, m.Ci, m.Cf32, m.Ci32, m.xm, m.fac, m.tmp, m.xs, m.cpart, m.fac32};
        for (void* p : md)
            if (p) cudaFree(p);
    }
    void* dwp[] = {b->zdw, b->bdw, b->wdw, b->bint2};
    for (void* p : dwp)
        if (p) cudaFree(p);
    void* host[] = {b->h_blk, b->h_cur, b->h_active, b->h_res, b->h_bn, b->h_tol};
    for (void* p : host)
        if (p) cudaFreeHost(p);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
}

// Blocks for the strips in `strips` (ascending) in proportion to the weights (at least one
// each), `total` blocks at most.  Other strips get no block.
static int batch_schedule(dd_nls_batch* b, const std::vector<double>& w, const std::vector<int>& strips, int total) {
    double W = 0.0;
    for (int j : strips) W += w[j];
    const int ns = (int)strips.size();
    const int spare = std::max(0, total - ns);
    int* bs = b->h_blk;                       // block -> strip
    int* st = b->h_blk + b->maxb;             // strip -> first block (all strips)
    int nb = 0;
    int k = 0;
    for (int j = 0; j < b->nstrips; ++j) {
        st[j] = nb;
        if (k < ns && strips[k] == j) {
            const Geom& g = b->G[b->sinfo[j].inst];
            const int cap = (int)(((long long)g.nxs * g.nyn + b->bs - 1) / b->bs);
            int c = 1 + (W > 0.0 ? (int)std::floor(spare * (w[j] / W)) : 0);
            c = std::max(1, std::min(c, cap));
            for (int t = 0; t < c; ++t) bs[nb + t] = j;
            nb += c;
            ++k;
        }
    }
    st[b->nstrips] = nb;
    return nb;
}

// The active strips in waves of at most `total` strips (one cooperative launch per wave).
static std::vector<std::vector<int>> batch_waves(dd_nls_batch* b, int total) {
    std::vector<int> act;
    for (int i = 0; i < b->n; ++i)
        if (b->h_active[i])
            for (int j = b->strip_first[i]; j < b->strip_first[i + 1]; ++j) act.push_back(j);
    std::vector<std::vector<int>> waves;
    const int nw = std::max(1, (int)((act.size() + total - 1) / std::max(1, total)));
    const size_t per = (act.size() + nw - 1) / nw;
    for (size_t k = 0; k < act.size(); k += per)
        waves.emplace_back(act.begin() + k, act.begin() + std::min(act.size(), k + per));
    return waves;
}

static StripSolveArgs batch_args(dd_nls_batch* b) {
    StripSolveArgs a{};
    a.g = b->G[0];
    fill_fp32_constants(a, 0.0, a.g.p, a.g.hy);   // Robin only; per-instance p comes from geoms
    a.geoms = b->d_geoms;
    a.sinfo = b->d_sinfo;
    a.blk_strip = b->d_blk;
    a.blk_start = b->d_blk + b->maxb;
    a.bnorm0 = b->bnorm0;
    a.mode = 0;
    a.zeta = b->zeta;
    a.rhs0 = b->rhs0;
    a.Wn = b->Wn;
    a.gtr = b->gbuf;
    a.x = b->x; a.r = b->r; a.z = b->z; a.p = b->p; a.q = b->q; a.cT = b->cT;
    a.w1 = b->w1; a.s0 = b->s0; a.s1 = b->s1; a.dv = b->dv;
    a.nl_tol = b->P[0].nl_tol;
    a.nl_tol_strip = b->d_tol;
    a.inner_tol = b->P[0].inner_tol;
    a.inner_floor = 0.1 * b->P[0].nl_tol;
    a.bscale = b->bscale;
    a.nl_floor_frac = 0.01 * b->P[0].nl_tol / 4.0;
    a.max_nl = b->P[0].max_nl;
    a.max_inner = b->P[0].max_inner;
    a.nl_relax = b->P[0].nl_relax;
    a.nl_picard = b->P[0].nl_picard;
    a.part = b->part;
    a.bar = b->bar;
    a.status = b->status;
    a.nl_its = b->nl_its;
    a.kry_its = b->kry;
    a.nl_res = b->nl_res;
    a.err = b->err;
    if (b->dw) {
        // modes 1 (first launch of a step: state and right side from zeta and rhs0) and 2 (the
        // double-word fields already hold this step's state); set per launch by the caller
        a.zdw = b->zdw;
        a.bdw = b->bdw;
        a.wdw = b->wdw;
        a.ddw = nullptr;
        a.bint2 = b->bint2;
        a.dw_mode = 1;
    }
    return a;
}

// One launch over the scheduled strips; the descriptor table points each strip at the current
// half of its instance's interface vector.
static int batch_solve(dd_nls_batch* b, StripSolveArgs& a, int nblk, float* ms_out) {
    const long long half = b->nI;
    for (int j = 0; j < b->nstrips; ++j) {
        const int i = b->sinfo[j].inst;
        StripInfo s = b->sinfo[j];
        s.goff = b->goff[i] + (b->cur[i] ? half : 0);
        b->sinfo[j] = s;
    }
    BCK(cudaMemcpyAsync(b->d_sinfo, b->sinfo.data(), sizeof(StripInfo) * b->nstrips, cudaMemcpyHostToDevice, b->s));
    BCK(cudaMemcpyAsync(b->d_blk, b->h_blk, sizeof(int) * (b->maxb + b->nstrips + 1), cudaMemcpyHostToDevice, b->s));
    for (int j = 0; j < b->nstrips; ++j) b->h_tol[j] = b->tolk[b->sinfo[j].inst];
    BCK(cudaMemcpyAsync(b->d_tol, b->h_tol, sizeof(double) * b->nstrips, cudaMemcpyHostToDevice, b->s));
    BCK(cudaMemsetAsync(b->bar, 0, sizeof(unsigned) * b->nstrips, b->s));
    BCK(cudaMemsetAsync(b->err, 0, sizeof(int), b->s));
    BCK(cudaEventRecord(b->ev0, b->s));
    BCK(launch_strip_solve(a, nblk, b->fp32, b->s, b->bs));
    BCK(cudaEventRecord(b->ev1, b->s));
    BCK(cudaMemcpyAsync(b->h_status.data(), b->status, sizeof(int) * b->nstrips, cudaMemcpyDeviceToHost, b->s));
    BCK(cudaMemcpyAsync(b->h_nl.data(), b->nl_its, sizeof(int) * b->nstrips, cudaMemcpyDeviceToHost, b->s));
    BCK(cudaMemcpyAsync(b->h_kry.data(), b->kry, sizeof(long long) * b->nstrips, cudaMemcpyDeviceToHost, b->s));
    int errw = 0;
    BCK(cudaMemcpyAsync(b->h_cur + b->n, b->err, sizeof(int), cudaMemcpyDeviceToHost, b->s));
    BCK(cudaStreamSynchronize(b->s));
    float ms = 0.f;
    BCK(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
    if (ms_out) *ms_out = ms;
    errw = b->h_cur[b->n];
    if (errw) return bfail(b, errw, "batched strip solver: device barrier timed out");
    return DD_NLS_OK;
}

// Pick (block size, blocks per launch) for this batch shape: time one Schwarz iteration of the
// first step with each candidate, from the same starting state.
static int autotune(dd_nls_batch* b, std::vector<double>& w) {
    TuneKey key{b->n, b->nstrips, b->dw ? 2 : (b->fp32 ? 1 : 0), b->nfield};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            b->bs = it->second.first;
            b->blocks = std::min(it->second.second, strip_solve_max_blocks_bs(b->fp32, b->bs));
            b->tuned = true;
            return DD_NLS_OK;
        }
    }
    struct Cand { int bs; double occ; };
    const Cand cands[] = {{256, 1.0}, {256, 0.5}, {128, 1.0}, {128, 0.5}};
    double best = 1e300;
    int best_bs = 256, best_blocks = 1;
    const int maxb_all = std::max(strip_solve_max_blocks_bs(b->fp32, 128), strip_solve_max_blocks_bs(b->fp32, 256));
    for (const Cand& c : cands) {
        const int mb = strip_solve_max_blocks_bs(b->fp32, c.bs);
        const int blocks = std::max(1, (int)(mb * c.occ));
        if (blocks > mb || blocks > maxb_all) continue;
        if (b->dw && c.bs != 256) continue;      // the double-word kernel is built for 256 threads
        b->bs = c.bs;
        BCK(cudaMemcpyAsync(b->zeta, b->u, sizeof(double2) * b->nfield, cudaMemcpyDeviceToDevice, b->s));
        float ms = 0.f;
        for (const auto& wave : batch_waves(b, blocks)) {
            const int nblk = batch_schedule(b, w, wave, blocks);
            StripSolveArgs a = batch_args(b);
            float t = 0.f;
            int rc = batch_solve(b, a, nblk, &t);
            if (rc) return rc;
            ms += t;
        }
        if (ms < best) { best = ms; best_bs = c.bs; best_blocks = blocks; }
    }
    b->bs = best_bs;
    b->blocks = best_blocks;
    b->tuned = true;
    BCK(cudaMemcpyAsync(b->zeta, b->u, sizeof(double2) * b->nfield, cudaMemcpyDeviceToDevice, b->s));
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = {best_bs, best_blocks};
    return DD_NLS_OK;
}

// The exact P^-1 of instance i (eq. algo_pd, Sec. 4.2): strip types by edge kinds (equal strips
// share their L_h blocks), the diagonal of L_h in the cosine basis and the per-mode factors.
static int batch_modal_build(dd_nls_batch* b, int i) {
    const Geom& G = b->G[i];
    dd_nls_batch::Modal& m = b->modal[i];
    std::vector<std::pair<int, int>> types;
    std::vector<int> bt(G.N);
    for (int j = 0; j < G.N; ++j) {
        const auto key = std::make_pair((j > 0 || G.bc_same) ? 1 : 0, (j < G.N - 1 || G.bc_same) ? 1 : 0);
        auto it = std::find(types.begin(), types.end(), key);
        if (it == types.end()) { types.push_back(key); bt[j] = (int)types.size() - 1; }
        else bt[j] = (int)(it - types.begin());
    }
    m.ntypes = (int)types.size();
    std::vector<int> tk(2 * m.ntypes);
    for (int t = 0; t < m.ntypes; ++t) { tk[2 * t] = types[t].first; tk[2 * t + 1] = types[t].second; }
    const long long nn = (long long)G.nyn * G.nyn, nIi = 2LL * (G.N - 1) * G.P;
    const size_t nf = (size_t)9 * std::max(1, G.N - 1) * G.nyn;
    BCK(zalloc(&m.btype, G.N));
    BCK(zalloc(&m.tkind, tk.size()));
    BCK(cudaMemcpy(m.btype, bt.data(), sizeof(int) * G.N, cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(m.tkind, tk.data(), sizeof(int) * tk.size(), cudaMemcpyHostToDevice));
    BCK(zalloc(&m.Cf, nn));
    BCK(zalloc(&m.Ci, nn));
    if (b->fp32) { BCK(zalloc(&m.Cf32, nn)); BCK(zalloc(&m.Ci32, nn)); }
    BCK(zalloc(&m.xm, (size_t)m.ntypes * 4 * G.nyn));
    BCK(zalloc(&m.fac, nf));
    BCK(zalloc(&m.tmp, nIi));
    BCK(zalloc(&m.xs, nIi));
    BCK(zalloc(&m.cpart, 8 * nIi));
    double2* work = nullptr;
    BCK(cudaMalloc(&work, sizeof(double2) * (size_t)m.ntypes * G.nyn * 2 * G.nxs));
    cudaError_t e = launch_modal_setup(G, m.ntypes, m.tkind, m.btype, m.Cf, m.Ci, m.Cf32, m.Ci32, m.xm, m.fac, work, b->s);
    if (e == cudaSuccess && b->fp32) {
        e = cudaMalloc(&m.fac32, nf * sizeof(float2));
        if (e == cudaSuccess) e = launch_to_float((const double*)m.fac, (float*)m.fac32, 2 * (long long)nf, b->s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->s);
    cudaFree(work);
    if (e != cudaSuccess) return bfail(b, DD_NLS_ECUDA, std::string("batched modal set-up: ") + cudaGetErrorString(e));
    return DD_NLS_OK;
}

extern "C" int dd_nls_batch_create(int n, const dd_nls_params* params, const double* const* V,
                                   const double* const* u0, int ptr_kind, void* stream, dd_nls_batch** out) {
    dd_nls_batch* b = nullptr;
    if (n < 1 || !params || !u0 || !out) return bfail(nullptr, DD_NLS_EINVAL, "dd_nls_batch_create: bad arguments");
    *out = nullptr;
    const int prec = params[0].precision;
    for (int i = 0; i < n; ++i) {
        const dd_nls_params& p = params[i];
        if (!u0[i]) return bfail(nullptr, DD_NLS_EINVAL, "dd_nls_batch_create: NULL u0 of an instance");
        if (const char* why = params_problem(p))
            return bfail(nullptr, DD_NLS_EINVAL, std::string("dd_nls_batch_create: instance ") + std::to_string(i) + ": " + why);
        if (p.tc != DD_NLS_TC_ROBIN || !(p.p > 0))
            return bfail(nullptr, DD_NLS_EINVAL, "dd_nls_batch_create: batches take Robin transmission with p > 0");
        if (p.algorithm != DD_NLS_CLASSICAL && (p.algorithm != DD_NLS_PRECONDITIONED || p.psolve != DD_NLS_PSOLVE_MODAL))
            return bfail(nullptr, DD_NLS_EINVAL,
                         "dd_nls_batch_create: the classical algorithm, or the preconditioned one with the modal P solve");
        if (p.precision != prec || (prec != DD_NLS_FP64 && prec != DD_NLS_FP32_INNER && prec != DD_NLS_FP32_DW))
            return bfail(nullptr, DD_NLS_EINVAL, "dd_nls_batch_create: one precision for the whole batch");
        if (prec == DD_NLS_FP32_DW && !(p.nl_tol >= kDWFinish))
            return bfail(nullptr, DD_NLS_EINVAL, "dd_nls_batch_create: the double-word residual needs nl_tol >= 1e-12");
        if (p.trap_gx > 0.0 || p.trap_gy > 0.0)
            return bfail(nullptr, DD_NLS_EINVAL, "dd_nls_batch_create: batches take a static V (trap_gx = trap_gy = 0)");
        const dd_nls_params& q = params[0];       // one strip-solver launch serves every instance
        if (p.inner_tol != q.inner_tol || p.max_nl != q.max_nl || p.max_inner != q.max_inner ||
            p.nl_relax != q.nl_relax || p.nl_picard != q.nl_picard)
            return bfail(nullptr, DD_NLS_EINVAL,
                         "dd_nls_batch_create: inner_tol, max_nl, max_inner, nl_relax and nl_picard must agree across instances");
    }
    if (ptr_kind != DD_NLS_PTR_HOST && ptr_kind != DD_NLS_PTR_DEVICE)
        return bfail(nullptr, DD_NLS_EINVAL, "dd_nls_batch_create: unknown ptr_kind");
    b = new dd_nls_batch();
    auto bad = [&](int code) { std::string m = b->error; batch_release(b); delete b; set_handle_free_error(m.c_str()); return code; };
#define BCKC(call)                                                                          \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            b->error = std::string(#call) + ": " + cudaGetErrorString(e_);                 \
            return bad(e_ == cudaErrorMemoryAllocation ? DD_NLS_ENOMEM : DD_NLS_ECUDA);     \
        }                                                                                   \
    } while (0)
    b->n = n;
    b->s = (cudaStream_t)stream;
    b->fp32 = prec != DD_NLS_FP64;
    b->dw = prec == DD_NLS_FP32_DW;
    b->P.assign(params, params + n);
    b->G.resize(n);
    b->foff.resize(n);
    b->goff.resize(n);
    b->strip_first.assign(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        const dd_nls_params& p = params[i];
        Geom& G = b->G[i];
        G.N = p.n_strips;
        G.nxs = p.nx / p.n_strips + 1;
        G.nyn = p.ny + 1;
        G.P = (G.nyn + 31) / 32 * 32;
        G.hx = (p.xr - p.xl) / p.nx;
        G.hy = (p.yu - p.yb) / p.ny;
        G.alpha = 2.0 / (p.lap * p.dt);
        G.kap = p.kappa / p.lap;
        G.p = p.p;
        G.bc_same = p.bc == DD_NLS_BC_SAME;
        G.nx = p.nx;
        G.fill_coefficients();
        b->foff[i] = b->nfield;
        b->goff[i] = b->nI;
        b->strip_first[i] = b->nstrips;
        for (int j = 0; j < G.N; ++j)
            b->sinfo.push_back(StripInfo{i, j, b->nfield + (long long)j * G.sstride(), b->nI});
        b->nstrips += G.N;
        b->nfield += (long long)G.N * G.sstride();
        b->nI += (long long)2 * (G.N - 1) * G.P;
    }
    b->strip_first[n] = b->nstrips;
    b->nI = std::max<long long>(b->nI, 1);
    const int maxb = std::max(strip_solve_max_blocks_bs(b->fp32, 128), strip_solve_max_blocks_bs(b->fp32, 256));
    b->maxb = maxb;
    b->blocks = strip_solve_max_blocks(b->fp32);
    const size_t s2 = b->fp32 ? sizeof(float2) : sizeof(double2), s1 = b->fp32 ? sizeof(float) : sizeof(double);
    BCKC(zalloc(&b->u, b->nfield));
    BCKC(zalloc(&b->zeta, b->nfield));
    BCKC(zalloc(&b->rhs0, b->nfield));
    BCKC(zalloc(&b->Wn, b->nfield));
    BCKC(zalloc((char**)&b->x, b->nfield * s2));
    BCKC(zalloc((char**)&b->r, b->nfield * s2));
    BCKC(zalloc((char**)&b->z, b->nfield * s2));
    BCKC(zalloc((char**)&b->p, b->nfield * s2));
    BCKC(zalloc((char**)&b->q, b->nfield * s2));
    BCKC(zalloc((char**)&b->cT, b->nfield * s1));
    BCKC(zalloc((char**)&b->w1, b->nfield * s2));
    BCKC(zalloc((char**)&b->s0, b->nfield * s2));
    BCKC(zalloc((char**)&b->s1, b->nfield * s2));
    BCKC(zalloc((char**)&b->dv, b->nfield * s2));
    BCKC(zalloc(&b->gbuf, 2 * b->nI));
    BCKC(zalloc(&b->part, (size_t)16 * maxb + 2048));
    BCKC(zalloc(&b->bscale, n));
    BCKC(zalloc(&b->bnorm0, b->nstrips));
    BCKC(zalloc(&b->res, 2 * n));
    BCKC(zalloc(&b->nl_res, b->nstrips));
    BCKC(zalloc(&b->bar, b->nstrips));
    BCKC(zalloc(&b->status, b->nstrips));
    BCKC(zalloc(&b->nl_its, b->nstrips));
    BCKC(zalloc(&b->kry, b->nstrips));
    BCKC(zalloc(&b->err, 1));
    BCKC(zalloc(&b->d_blk, (size_t)maxb + b->nstrips + 2));
    BCKC(zalloc(&b->d_geoms, n));
    BCKC(zalloc(&b->d_sinfo, b->nstrips));
    BCKC(zalloc(&b->d_foff, n));
    BCKC(zalloc(&b->d_goff, n));
    BCKC(zalloc(&b->d_cur, n));
    BCKC(zalloc(&b->d_active, n));
    BCKC(zalloc(&b->d_tol, b->nstrips));
    b->tolk.assign(n, 0.0);
    for (int i = 0; i < n; ++i) b->tolk[i] = params[i].nl_tol;
    if (b->dw) {
        BCKC(zalloc(&b->zdw, b->nfield));
        BCKC(zalloc(&b->bdw, b->nfield));
        BCKC(zalloc(&b->wdw, b->nfield));
        BCKC(zalloc(&b->bint2, b->nstrips));
    }
    BCKC(cudaMallocHost((void**)&b->h_tol, sizeof(double) * b->nstrips));
    b->rel_prev.assign(n, 1.0);
    BCKC(cudaMallocHost((void**)&b->h_blk, sizeof(int) * (maxb + b->nstrips + 2)));
    BCKC(cudaMallocHost((void**)&b->h_cur, sizeof(int) * (n + 1)));
    BCKC(cudaMallocHost((void**)&b->h_active, sizeof(int) * n));
    BCKC(cudaMallocHost((void**)&b->h_res, sizeof(double) * 2 * n));
    BCKC(cudaMallocHost((void**)&b->h_bn, sizeof(double) * b->nstrips));
    BCKC(cudaEventCreate(&b->ev0));
    BCKC(cudaEventCreate(&b->ev1));
    if (!b->h_status.resize(b->nstrips) || !b->h_nl.resize(b->nstrips) || !b->h_kry.resize(b->nstrips)) {
        b->error = "dd_nls_batch_create: pinned host memory for the per-strip results";
        return bad(DD_NLS_ENOMEM);
    }
    b->cur.assign(n, 0);
    b->conv_half.assign(n, 0);
    b->have_prev.assign(n, 0);
    BCKC(cudaMemcpy(b->d_geoms, b->G.data(), sizeof(Geom) * n, cudaMemcpyHostToDevice));
    BCKC(cudaMemcpy(b->d_sinfo, b->sinfo.data(), sizeof(StripInfo) * b->nstrips, cudaMemcpyHostToDevice));
    BCKC(cudaMemcpy(b->d_foff, b->foff.data(), sizeof(long long) * n, cudaMemcpyHostToDevice));
    BCKC(cudaMemcpy(b->d_goff, b->goff.data(), sizeof(long long) * n, cudaMemcpyHostToDevice));
    // inputs: one staging buffer of the largest nodal field, per instance scatter
    size_t maxnodes = 0;
    for (int i = 0; i < n; ++i) maxnodes = std::max(maxnodes, (size_t)(params[i].nx + 1) * (params[i].ny + 1));
    BCKC(cudaMalloc(&b->stage, sizeof(double2) * maxnodes));
    double2* stage = b->stage;
    const cudaMemcpyKind kind = ptr_kind == DD_NLS_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        const size_t nodes = (size_t)(params[i].nx + 1) * (params[i].ny + 1);
        e = cudaMemcpyAsync(stage, u0[i], sizeof(double2) * nodes, kind, b->s);
        if (!e) e = launch_scatter_u(b->G[i], stage, b->u + b->foff[i], b->s);
        if (!e && V && V[i]) {
            e = cudaMemcpyAsync(stage, V[i], sizeof(double) * nodes, kind, b->s);
            if (!e) e = launch_scatter_real(b->G[i], (const double*)stage, 1.0 / params[i].lap, b->Wn + b->foff[i], b->s);
        }
        if (!e) e = cudaStreamSynchronize(b->s);
    }
    BCKC(e);
    b->modal.resize(n);
    for (int i = 0; i < n; ++i)
        if (params[i].algorithm == DD_NLS_PRECONDITIONED && b->G[i].N > 1) {
            const int rc = batch_modal_build(b, i);
            if (rc) return bad(rc);
        }
    *out = b;
    return DD_NLS_OK;
#undef BCKC
}

extern "C" int dd_nls_batch_step(dd_nls_batch* b, int nsteps, dd_nls_stats* stats) {
    if (!b) return bfail(nullptr, DD_NLS_EINVAL, "dd_nls_batch_step: NULL handle");
    if (nsteps < 0) return bfail(b, DD_NLS_EINVAL, "dd_nls_batch_step: nsteps < 0");
    if (stats) {
        std::memset(stats, 0, sizeof(dd_nls_stats) * b->n);
    }
    const long long half = b->nI;
    for (int step = 0; step < nsteps; ++step) {
        // right sides, per-strip scales, warm starts, guesses
        for (int i = 0; i < b->n; ++i) {
            const Geom& G = b->G[i];
            int nb = 1;
            BCK(launch_rhs0(G, b->u + b->foff[i], b->rhs0 + b->foff[i], b->part, &nb, b->s));
            BCK(launch_finalize(b->part, nb, 1, b->bscale + i, b->s));
            BCK(launch_sqrt(b->bscale + i, b->s));
            BCK(launch_strip_norms(G, b->rhs0 + b->foff[i], b->bnorm0 + b->strip_first[i], b->part, 16 * b->maxb + 2048, b->s));
            const bool prev = b->P[i].guess == DD_NLS_GUESS_PREVIOUS && b->have_prev[i];
            const size_t gb = sizeof(double2) * (size_t)2 * (G.N - 1) * G.P;
            if (prev) b->cur[i] = b->conv_half[i];
            else {
                b->cur[i] = 0;
                if (gb) BCK(cudaMemsetAsync(b->gbuf + b->goff[i], 0, gb, b->s));
            }
            b->h_active[i] = 1;
            b->rel_prev[i] = 1.0;
        }
        // inexact strip solves per instance until an iteration fails to cut its interface
        // residual by 4x (as in dd_nls_step)
        std::vector<char> adapt_on(b->n);
        for (int i = 0; i < b->n; ++i)
            adapt_on[i] = b->P[i].algorithm == DD_NLS_PRECONDITIONED && b->P[i].nl_adapt > 0.0 && b->G[i].N > 1;
        auto adapt_of = [&](int i) { return adapt_on[i] != 0; };
        BCK(cudaMemcpyAsync(b->zeta, b->u, sizeof(double2) * b->nfield, cudaMemcpyDeviceToDevice, b->s));
        BCK(cudaMemcpyAsync(b->h_bn, b->bnorm0, sizeof(double) * b->nstrips, cudaMemcpyDeviceToHost, b->s));
        BCK(cudaStreamSynchronize(b->s));
        std::vector<double> w(b->nstrips, 1.0);
        for (int i = 0; i < b->n; ++i) {
            double bmax = 0.0;
            for (int j = b->strip_first[i]; j < b->strip_first[i + 1]; ++j) bmax = std::max(bmax, b->h_bn[j]);
            for (int j = b->strip_first[i]; j < b->strip_first[i + 1]; ++j)
                w[j] = 1.0 + (bmax > 0.0 ? 15.0 * std::sqrt(b->h_bn[j] / bmax) : 0.0);
        }
        if (!b->tuned) { int rc = autotune(b, w); if (rc) return rc; }
        int max_it = 1;
        for (int i = 0; i < b->n; ++i) max_it = std::max(max_it, b->P[i].max_schwarz);
        int nact = b->n;
        std::vector<int> its(b->n, 0);
        for (int k = 0; k < max_it && nact > 0; ++k) {
            // strip tolerance per instance: nl_tol, or for a preconditioned instance with
            // nl_adapt > 0 the inexact solves of the single-instance path (nl_adapt x the last
            // relative interface residual, at most 1e-6, down to nl_tol)
            for (int i = 0; i < b->n; ++i)
                b->tolk[i] = adapt_of(i) ? std::max(b->P[i].nl_tol, std::min(1e-6, b->P[i].nl_adapt * b->rel_prev[i]))
                                         : b->P[i].nl_tol;
            for (const auto& wave : batch_waves(b, b->blocks)) {
                const int nblk = batch_schedule(b, w, wave, b->blocks);
                StripSolveArgs a = batch_args(b);
                if (b->dw) a.dw_mode = k == 0 ? 1 : 2;
                float ms = 0.f;
                int rc = batch_solve(b, a, nblk, &ms);
                if (rc) return rc;
                if (b->prof) { b->profile.strip_solve_ms += ms; b->profile.strip_solve_launches += 1; }
                for (int j : wave) {
                    const int i = b->sinfo[j].inst;
                    if (b->h_status[j]) {
                        char msg[160];
                        std::snprintf(msg, sizeof msg, "instance %d strip %d: status %d", i, b->sinfo[j].jloc, b->h_status[j]);
                        return bfail(b, b->h_status[j], msg);
                    }
                    if (stats) { stats[i].nl_iterations += b->h_nl[j]; stats[i].krylov_iterations += b->h_kry[j]; }
                    w[j] = 1.0 + (double)b->h_kry[j] + 4.0 * (b->h_nl[j] + 1);
                }
            }
            // flux update and residual of every active instance
            for (int i = 0; i < b->n; ++i) b->h_cur[i] = b->cur[i];
            BCK(cudaMemcpyAsync(b->d_cur, b->h_cur, sizeof(int) * b->n, cudaMemcpyHostToDevice, b->s));
            BCK(cudaMemcpyAsync(b->d_active, b->h_active, sizeof(int) * b->n, cudaMemcpyHostToDevice, b->s));
            count_launches(1);
            batch_traces_kernel<<<b->n, 256, 0, b->s>>>(b->d_geoms, b->d_foff, b->d_goff, b->d_cur, b->d_active, half,
                                                       b->zeta, b->gbuf, b->res);
            BCK(cudaGetLastError());
            BCK(cudaMemcpyAsync(b->h_res, b->res, sizeof(double) * 2 * b->n, cudaMemcpyDeviceToHost, b->s));
            BCK(cudaStreamSynchronize(b->s));
            for (int i = 0; i < b->n; ++i) {
                if (!b->h_active[i]) continue;
                its[i] = k + 1;
                const double diff = b->G[i].N > 1 ? std::sqrt(b->h_res[2 * i]) : 0.0;
                const double nrm = b->G[i].N > 1 ? std::sqrt(b->h_res[2 * i + 1]) : 0.0;
                const double rel = nrm > 0.0 ? diff / nrm : diff;
                if (!std::isfinite(diff) || !std::isfinite(nrm)) return bfail(b, DD_NLS_ENONFINITE, "non-finite interface residual");
                if (stats) { stats[i].residual = rel; stats[i].residual_abs = diff; stats[i].schwarz_iterations += 1;
                             stats[i].last_schwarz_iterations = k + 1; }
                const int old = b->cur[i];
                b->cur[i] ^= 1;                       // the new R(g) is the next g (classical)
                const bool stalled = adapt_of(i) && k > 0 && rel > 0.25 * b->rel_prev[i];
                b->rel_prev[i] = rel;
                const bool full = !adapt_of(i) || b->tolk[i] <= std::max(b->P[i].nl_tol, b->P[i].nl_adapt * b->P[i].tol);
                if (stalled) adapt_on[i] = 0;
                if (((b->P[i].tol_absolute ? diff : rel) <= b->P[i].tol && full) || b->G[i].N == 1) {
                    // zeta holds v for g^k; R(g^k) (now current) is the next step's guess
                    b->conv_half[i] = b->cur[i];
                    b->h_active[i] = 0;
                    --nact;
                    if (b->dw) BCK(launch_dw_to_zeta(b->G[i], b->zdw + b->foff[i], b->zeta + b->foff[i], b->s));
                } else if (b->P[i].algorithm == DD_NLS_PRECONDITIONED) {
                    // g^{k+1} = g^k - P^{-1} (g^k - R(g^k))  (eq. algo_pd), into the half of R(g^k)
                    const Geom& G = b->G[i];
                    dd_nls_batch::Modal& m = b->modal[i];
                    double2* gk = b->gbuf + b->goff[i] + (old ? half : 0);
                    double2* gr = b->gbuf + b->goff[i] + (old ? 0 : half);
                    BCK(launch_modal_update(G, b->fp32, m.Cf, m.Ci, m.Cf32, m.Ci32, m.fac, m.fac32, gk, gr, gr, m.tmp,
                                            m.cpart, b->P[i].psolve_modes, b->s));
                }
            }
        }
        if (nact > 0) return bfail(b, DD_NLS_ENOCONV, "a batched instance reached max_schwarz");
        for (int i = 0; i < b->n; ++i) {
            BCK(launch_commit(b->G[i], b->zeta + b->foff[i], b->u + b->foff[i], b->s));
            b->have_prev[i] = 1;
            if (stats) stats[i].steps += 1;
        }
        BCK(cudaStreamSynchronize(b->s));
    }
    return DD_NLS_OK;
}

extern "C" int dd_nls_batch_get_u(dd_nls_batch* b, int i, double* u, int ptr_kind) {
    if (!b || i < 0 || i >= b->n || !u || (ptr_kind != DD_NLS_PTR_HOST && ptr_kind != DD_NLS_PTR_DEVICE))
        return bfail(b, DD_NLS_EINVAL, "dd_nls_batch_get_u: bad arguments");
    const size_t nodes = (size_t)(b->P[i].nx + 1) * (b->P[i].ny + 1);
    if (ptr_kind == DD_NLS_PTR_DEVICE) {
        BCK(launch_gather_u(b->G[i], b->u + b->foff[i], (double2*)u, b->s));
    } else {
        BCK(launch_gather_u(b->G[i], b->u + b->foff[i], b->stage, b->s));
        BCK(cudaMemcpyAsync(u, b->stage, sizeof(double2) * nodes, cudaMemcpyDeviceToHost, b->s));
    }
    BCK(cudaStreamSynchronize(b->s));
    return DD_NLS_OK;
}

extern "C" int dd_nls_batch_set_u(dd_nls_batch* b, int i, const double* u, int ptr_kind) {
    if (!b || i < 0 || i >= b->n || !u || (ptr_kind != DD_NLS_PTR_HOST && ptr_kind != DD_NLS_PTR_DEVICE))
        return bfail(b, DD_NLS_EINVAL, "dd_nls_batch_set_u: bad arguments");
    const size_t nodes = (size_t)(b->P[i].nx + 1) * (b->P[i].ny + 1);
    if (ptr_kind == DD_NLS_PTR_DEVICE) {
        BCK(launch_scatter_u(b->G[i], (const double2*)u, b->u + b->foff[i], b->s));
    } else {
        BCK(cudaMemcpyAsync(b->stage, u, sizeof(double2) * nodes, cudaMemcpyHostToDevice, b->s));
        BCK(launch_scatter_u(b->G[i], b->stage, b->u + b->foff[i], b->s));
    }
    BCK(cudaStreamSynchronize(b->s));
    return DD_NLS_OK;
}

extern "C" int dd_nls_batch_tuning(dd_nls_batch* b, int* block_size, int* blocks) {
    if (!b) return bfail(nullptr, DD_NLS_EINVAL, "dd_nls_batch_tuning: NULL handle");
    if (block_size) *block_size = b->tuned ? b->bs : 0;
    if (blocks) *blocks = b->tuned ? b->blocks : 0;
    return DD_NLS_OK;
}

extern "C" int dd_nls_batch_set_profiling(dd_nls_batch* b, int on) {
    if (!b) return bfail(nullptr, DD_NLS_EINVAL, "dd_nls_batch_set_profiling: NULL handle");
    b->prof = on != 0;
    std::memset(&b->profile, 0, sizeof(b->profile));
    b->launch_base = kernel_launch_count();
    return DD_NLS_OK;
}

extern "C" int dd_nls_batch_get_profile(dd_nls_batch* b, dd_nls_profile* prof) {
    if (!b || !prof) return bfail(b, DD_NLS_EINVAL, "dd_nls_batch_get_profile: NULL argument");
    *prof = b->profile;
    prof->kernel_launches = b->prof ? kernel_launch_count() - b->launch_base : 0;
    return DD_NLS_OK;
}

extern "C" const char* dd_nls_batch_last_error(const dd_nls_batch* b) {
    return b ? b->error.c_str() : dd_nls_last_error(nullptr);
}

extern "C" void dd_nls_batch_destroy(dd_nls_batch* b) {
    if (!b) return;
    if (b->s) cudaStreamSynchronize(b->s);
    batch_release(b);
    delete b;
}
