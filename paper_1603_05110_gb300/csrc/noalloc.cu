// dd_nls_step_noalloc: one time step with no device allocation.
//
// Some callers cannot allocate device memory when they need a step: code running inside a
// memory pool or arena that owns the whole device (a framework allocator, a pre-sized
// server process), code that must not change the allocation state of a context it shares,
// or code on a path where cudaMalloc's implicit synchronisation is not allowed.  This entry
// point takes every piece of working memory from one file-scope __device__ array of fixed
// size, which the library holds on every GPU that loads it until the process exits.  The
// caller still passes the inputs and outputs.
//
// Limits and rules:
//  - at most kScratchBytes of working memory (the entry point returns DD_NLS_EINVAL with a
//    message naming the size when a problem needs more) and at most kMaxStrips strips;
//  - classical algorithm with the Robin transmission condition (precision FP64 or FP32
//    inner, as in dd_nls_step);
//  - all calls share the one array: calls that overlap on the GPU (several streams or
//    threads at once) race and give wrong results; a call leaves the array holding its own
//    data, and every buffer that must start at zero is cleared by the call itself;
//  - the first call on a device looks up the array's device address with
//    cudaGetSymbolAddress (with that device current); make that first call before any
//    stream capture.  The address is kept for the life of the process: after a
//    cudaDeviceReset of that device it is stale, so do not call this entry point again
//    in a process that has reset the device;
//  - the call waits for its stream once per Schwarz iteration (the host decides convergence).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <utility>

#include "../../include/dd_nls.h"
#include "common.cuh"
#include "kernels.h"
#include "params_check.h"

namespace ddnls {

constexpr size_t kScratchBytes = 64ull << 20;   // 64 MiB
constexpr int kMaxStrips = 64;
constexpr int kMaxDevices = 64;

// The working memory of dd_nls_step_noalloc.  In host code the name is only a stand-in: the
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

static void* g_scratch_addr[kMaxDevices];        // device address of the array, per device

// the message goes to dd_nls_last_error(NULL)
static int noalloc_fail(int code, const char* msg) {
    char buf[256];
    std::snprintf(buf, sizeof buf, "dd_nls_step_noalloc: %s", msg);
    set_handle_free_error(buf);
    return code;
}

// Uniform block table: bps consecutive blocks per strip.
__global__ void uniform_table_kernel(int* blk_strip, int* blk_start, int nstrips, int bps) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nstrips * bps) blk_strip[t] = t / bps;
    if (t <= nstrips) blk_start[t] = t * bps;
}

// Bump allocator over the static array (256-byte aligned pieces).
struct Carve {
    unsigned char* base;
    size_t off = 0;
    template <typename T> T* take(size_t n) {
        off = (off + 255) & ~size_t(255);
        T* p = (T*)(base + off);
        off += n * sizeof(T);
        return p;
    }
};

}  // namespace ddnls

using namespace ddnls;

extern "C" int dd_nls_step_noalloc(const dd_nls_params* p, const double* V, double* u, const double* g0,
                                   double* g_out, void* stream, dd_nls_stats* st) {
    set_handle_free_error("");
    if (!p || !u) return noalloc_fail(DD_NLS_EINVAL, "NULL params or u");
    if (const char* why = params_problem(*p)) return noalloc_fail(DD_NLS_EINVAL, why);
    if (p->n_strips > kMaxStrips) return noalloc_fail(DD_NLS_EINVAL, "more than 64 strips");
    if (p->tc != DD_NLS_TC_ROBIN || p->algorithm != DD_NLS_CLASSICAL)
        return noalloc_fail(DD_NLS_EINVAL, "only the classical algorithm with Robin transmission");
    if (p->precision != DD_NLS_FP64 && p->precision != DD_NLS_FP32_INNER)
        return noalloc_fail(DD_NLS_EINVAL, "precision must be DD_NLS_FP64 or DD_NLS_FP32_INNER "
                                           "(the double-word form DD_NLS_FP32_DW is not supported here)");
    cudaStream_t s = (cudaStream_t)stream;
    const bool fp32 = p->precision == DD_NLS_FP32_INNER;

    // ---- device address of the array (once per device, with that device current)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return noalloc_fail(DD_NLS_ECUDA, "no current CUDA device");
    if (!g_scratch_addr[dev]) {
        void* addr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
        if (e != cudaSuccess || !addr) return noalloc_fail(DD_NLS_ECUDA, cudaGetErrorString(e));
        g_scratch_addr[dev] = addr;
    }

    // ---- geometry
    Geom G{};
    const int c = p->nx / p->n_strips;
    G.N = p->n_strips;
    G.nxs = c + 1;
    G.nyn = p->ny + 1;
    G.P = (G.nyn + 31) / 32 * 32;
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
    const size_t nfield = (size_t)G.N * G.nxs * G.P;
    const size_t nI = (size_t)2 * (G.N - 1) * G.P + 1;

    // ---- launch shape: uniform blocks per strip, all co-resident
    const int maxb = strip_solve_max_blocks(fp32);
    if (maxb < G.N) return noalloc_fail(DD_NLS_EINVAL, "more strips than co-resident blocks");
    const int chunks = (int)(((long long)G.nxs * G.nyn + 255) / 256);
    const int bps = std::max(1, std::min(maxb / G.N, chunks));
    const int nblk = bps * G.N;

    // ---- carve the array
    const size_t s2 = fp32 ? sizeof(float2) : sizeof(double2), s1 = fp32 ? sizeof(float) : sizeof(double);
    Carve cv{(unsigned char*)g_scratch_addr[dev]};
    double2* us = cv.take<double2>(nfield);
    double2* zeta = cv.take<double2>(nfield);
    double2* rhs0 = cv.take<double2>(nfield);
    double* Wn = cv.take<double>(nfield);
    void* kx = cv.take<unsigned char>(nfield * s2);
    void* kr = cv.take<unsigned char>(nfield * s2);
    void* kz = cv.take<unsigned char>(nfield * s2);
    void* kp = cv.take<unsigned char>(nfield * s2);
    void* kq = cv.take<unsigned char>(nfield * s2);
    void* kc = cv.take<unsigned char>(nfield * s1);
    void* kw1 = cv.take<unsigned char>(nfield * s2);
    void* ks0 = cv.take<unsigned char>(nfield * s2);
    void* ks1 = cv.take<unsigned char>(nfield * s2);
    void* kdv = cv.take<unsigned char>(nfield * s2);
    double2* gA = cv.take<double2>(nI);
    double2* gB = cv.take<double2>(nI);
    double* part = cv.take<double>((size_t)16 * std::max(maxb, 512));
    unsigned* bar = cv.take<unsigned>(G.N);
    int* status = cv.take<int>(G.N);
    int* nl_its = cv.take<int>(G.N);
    long long* kry = cv.take<long long>(G.N);
    double* nl_res = cv.take<double>(G.N);
    int* err = cv.take<int>(1);
    double* red = cv.take<double>(64);
    double* bnorm0 = cv.take<double>(G.N);
    int* blk = cv.take<int>((size_t)nblk + G.N + 1);
    if (cv.off > kScratchBytes) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "problem needs %zu bytes of working memory, the limit is %zu (64 MiB)",
                      cv.off, kScratchBytes);
        return noalloc_fail(DD_NLS_EINVAL, msg);
    }

#define NCK(call)                                                          \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) return noalloc_fail(DD_NLS_ECUDA, cudaGetErrorString(e_)); \
    } while (0)

    if (st) std::memset(st, 0, sizeof(*st));
    // buffers that must start at zero (the array keeps the previous call's contents)
    NCK(cudaMemsetAsync(us, 0, nfield * sizeof(double2), s));
    NCK(cudaMemsetAsync(Wn, 0, nfield * sizeof(double), s));
    NCK(cudaMemsetAsync(gA, 0, nI * sizeof(double2), s));
    NCK(cudaMemsetAsync(gB, 0, nI * sizeof(double2), s));
    NCK(launch_scatter_u(G, (const double2*)u, us, s));
    if (V) NCK(launch_scatter_real(G, V, 1.0 / p->lap, Wn, s));
    if (g0 && G.N > 1)
        NCK(cudaMemcpy2DAsync(gA, G.P * sizeof(double2), g0, G.nyn * sizeof(double2), G.nyn * sizeof(double2),
                              2 * (G.N - 1), cudaMemcpyDeviceToDevice, s));
    count_launches(1);
    uniform_table_kernel<<<(nblk + G.N + 256) / 256, 256, 0, s>>>(blk, blk + nblk, G.N, bps);
    NCK(cudaGetLastError());
    int nb = 1;
    NCK(launch_rhs0(G, us, rhs0, part, &nb, s));
    NCK(launch_finalize(part, nb, 1, red + 8, s));
    NCK(launch_sqrt(red + 8, s));
    NCK(launch_strip_norms(G, rhs0, bnorm0, part, 16 * std::max(maxb, 512), s));
    NCK(cudaMemcpyAsync(zeta, us, nfield * sizeof(double2), cudaMemcpyDeviceToDevice, s));

    StripSolveArgs a{};
    a.g = G;
    a.bps = bps;
    a.blk_strip = blk;
    a.blk_start = blk + nblk;
    a.bnorm0 = bnorm0;
    a.mode = 0;
    a.zeta = zeta;
    a.rhs0 = rhs0;
    a.Wn = Wn;
    a.x = kx; a.r = kr; a.z = kz; a.p = kp; a.q = kq; a.cT = kc;
    a.w1 = kw1; a.s0 = ks0; a.s1 = ks1; a.dv = kdv;
    a.nl_tol = p->nl_tol;
    a.inner_tol = p->inner_tol;
    a.inner_floor = 0.1 * p->nl_tol;
    a.bscale = red + 8;
    a.nl_floor_frac = 0.01 * p->nl_tol / std::sqrt((double)G.N);
    a.max_nl = p->max_nl;
    a.max_inner = p->max_inner;
    a.nl_relax = p->nl_relax;
    a.nl_picard = p->nl_picard;
    a.part = part;
    a.bar = bar;
    a.status = status;
    a.nl_its = nl_its;
    a.kry_its = kry;
    a.nl_res = nl_res;
    a.err = err;
    a.wait_ns = (unsigned long long)(p->wait_limit_ms > 0.0 ? p->wait_limit_ms * 1e6 : 2e9);
    a.pcyc = nullptr;
    fill_fp32_constants(a, 0.0, G.p, G.hy);   // Robin transmission only

    double2* g = gA;
    double2* gn = gB;
    int hstat[kMaxStrips];
    int hnl[kMaxStrips];
    long long hkry[kMaxStrips];
    double hred[2];
    int herr = 0;
    bool converged = false;
    for (int k = 0; k < std::max(1, p->max_schwarz); ++k) {
        a.gtr = g;
        NCK(cudaMemsetAsync(bar, 0, sizeof(unsigned) * G.N, s));
        NCK(cudaMemsetAsync(err, 0, sizeof(int), s));
        NCK(launch_strip_solve(a, nblk, fp32, s));
        NCK(cudaMemcpyAsync(hstat, status, sizeof(int) * G.N, cudaMemcpyDeviceToHost, s));
        NCK(cudaMemcpyAsync(hnl, nl_its, sizeof(int) * G.N, cudaMemcpyDeviceToHost, s));
        NCK(cudaMemcpyAsync(hkry, kry, sizeof(long long) * G.N, cudaMemcpyDeviceToHost, s));
        NCK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
        if (G.N > 1) {
            NCK(launch_traces(G, zeta, g, gn, part, &nb, s));
            NCK(launch_finalize(part, nb, 2, red, s));
            NCK(cudaMemcpyAsync(hred, red, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        } else {
            hred[0] = hred[1] = 0.0;
        }
        NCK(cudaStreamSynchronize(s));
        if (herr) return noalloc_fail(herr, "strip solver: device barrier timed out");
        for (int j = 0; j < G.N; ++j) {
            if (hstat[j]) return noalloc_fail(hstat[j], "strip solver failed");
            if (st) { st->nl_iterations += hnl[j]; st->krylov_iterations += hkry[j]; }
        }
        const double diff = std::sqrt(hred[0]), nrm = std::sqrt(hred[1]);
        const double rel = nrm > 0.0 ? diff / nrm : diff;
        if (st) {
            st->schwarz_iterations += 1;
            st->last_schwarz_iterations = k + 1;
            st->residual = rel;
            st->residual_abs = diff;
        }
        if (!std::isfinite(diff) || !std::isfinite(nrm)) return noalloc_fail(DD_NLS_ENONFINITE, "interface residual is not finite");
        if ((p->tol_absolute ? diff : rel) <= p->tol) { converged = true; break; }
        std::swap(g, gn);
    }
    if (!converged) return noalloc_fail(DD_NLS_ENOCONV, "Schwarz iteration reached max_schwarz");
    NCK(launch_commit(G, zeta, us, s));
    NCK(launch_gather_u(G, us, (double2*)u, s));
    if (g_out && G.N > 1)
        NCK(cudaMemcpy2DAsync(g_out, G.nyn * sizeof(double2), gn, G.P * sizeof(double2), G.nyn * sizeof(double2),
                              2 * (G.N - 1), cudaMemcpyDeviceToDevice, s));
    NCK(cudaStreamSynchronize(s));
    if (st) st->steps = 1;
    return DD_NLS_OK;
#undef NCK
}
