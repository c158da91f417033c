// Auxiliary kernels of the time step: layout conversion, the step right side, the flux
// update of eq. (fluxlr), the commit of eq. (CNS), diagnostics, L_h (eq. Lmpi) extraction and
// products, and the vector operations of the interface GMRES.
#include "common.cuh"
#include "kernels.h"

#include <algorithm>

namespace ddnls {

static inline int nblocks(long long n, int bs) { return (int)((n + bs - 1) / bs); }

// ------------------------------------------------------------------ layout conversion
__global__ void scatter_u_kernel(Geom g, const double2* __restrict__ glob, double2* __restrict__ out) {
    const long long total = (long long)g.N * g.nxs * g.nyn;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        int j, ix, iy;
        split_strip_node(t, g.nxs, g.nyn, j, ix, iy);
        const int ixg = j * (g.nxs - 1) + ix;
        out[(long long)(j * g.nxs + ix) * g.P + iy] = glob[(long long)iy * (g.nx + 1) + ixg];
    }
}
__global__ void scatter_real_kernel(Geom g, const double* __restrict__ glob, double scale, double* __restrict__ out) {
    const long long total = (long long)g.N * g.nxs * g.nyn;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        int j, ix, iy;
        split_strip_node(t, g.nxs, g.nyn, j, ix, iy);
        const int ixg = j * (g.nxs - 1) + ix;
        out[(long long)(j * g.nxs + ix) * g.P + iy] = scale * glob[(long long)iy * (g.nx + 1) + ixg];
    }
}
// interface columns are taken from the left strip
__global__ void gather_u_kernel(Geom g, const double2* __restrict__ in, double2* __restrict__ glob) {
    const int c = g.nxs - 1;
    const long long total = (long long)(g.nx + 1) * g.nyn;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int ixg = (int)(t % (g.nx + 1));
        const int iy = (int)(t / (g.nx + 1));
        const int j = ixg == 0 ? 0 : (ixg - 1) / c;
        const int ix = ixg - j * c;
        glob[t] = in[(long long)(j * g.nxs + ix) * g.P + iy];
    }
}

cudaError_t launch_scatter_u(const Geom& g, const double2* glob, double2* strips, cudaStream_t s) {
    count_launches(1);
    scatter_u_kernel<<<1024, 256, 0, s>>>(g, glob, strips);
    return cudaGetLastError();
}
cudaError_t launch_scatter_real(const Geom& g, const double* glob, double scale, double* strips, cudaStream_t s) {
    count_launches(1);
    scatter_real_kernel<<<1024, 256, 0, s>>>(g, glob, scale, strips);
    return cudaGetLastError();
}
cudaError_t launch_gather_u(const Geom& g, const double2* strips, double2* glob, cudaStream_t s) {
    count_launches(1);
    gather_u_kernel<<<1024, 256, 0, s>>>(g, strips, glob);
    return cudaGetLastError();
}

// ------------------------------------------------------------- step right side
// Both per-step FP64 stencils below walk runs of kRX x-nodes at one row: on the uniform mesh the
// 1D mass and stiffness rows are exact multiples of [1 d 1] (d = 4 inside, 2 at an end; times
// h/6) and [-1 e -1] (e = 2 / 1; times 1/h), so the y sums of each column are formed once per
// column and shared by the run's nodes (about half the FP64 operations of the 9-point loop).
constexpr int kRX = 4;
__device__ __forceinline__ void run_item(long long t, const Geom& g, int& j, int& x0, int& x1, int& iy) {
    const int nseg = (g.nxs + kRX - 1) / kRX;
    int seg;
    split_strip_node(t, nseg, g.nyn, j, seg, iy);
    x0 = seg * kRX;
    x1 = min(x0 + kRX, g.nxs);
}
// y sums of column col at row iy: tm = [1 dy 1] u, tk = [-1 ey -1] u; zc = u(iy)
__device__ __forceinline__ void col_sums(const double2* col, int iy, int ny, double2& tm, double2& tk, double2& zc) {
    zc = col[0];
    const bool lo = iy > 0, hi = iy < ny;
    const double2 am = lo ? col[-1] : make_double2(0.0, 0.0), ap = hi ? col[1] : make_double2(0.0, 0.0);
    const double d = (lo && hi) ? 4.0 : 2.0, e = (lo && hi) ? 2.0 : 1.0;
    const double sx = am.x + ap.x, sy = am.y + ap.y;
    tm = make_double2(fma(d, zc.x, sx), fma(d, zc.y, sy));
    tk = make_double2(fma(e, zc.x, -sx), fma(e, zc.y, -sy));
}

// rhs0 = (2i/dt) M h on every strip (eq. NproblemRobinNL), M = Mx (x) My of the strip.
__global__ void rhs0_kernel(Geom g, const double2* __restrict__ h, double2* __restrict__ rhs, double* __restrict__ part) {
    __shared__ double sm[64];
    const int c = g.nxs - 1, ny = g.nyn - 1;
    const double cm = g.hx * g.hy / 36.0;
    double nv[1] = {0.0};
    const long long total = (long long)g.N * ((g.nxs + kRX - 1) / kRX) * g.nyn;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        int j, x0, x1, iy;
        run_item(t, g, j, x0, x1, iy);
        const double2* base = h + (long long)j * g.sstride() + iy;
        double2 tmm = make_double2(0.0, 0.0), tm0, tk, zc;
        if (x0 > 0) col_sums(base + (long long)(x0 - 1) * g.P, iy, ny, tmm, tk, zc);
        col_sums(base + (long long)x0 * g.P, iy, ny, tm0, tk, zc);
        for (int ix = x0; ix < x1; ++ix) {
            double2 tmp = make_double2(0.0, 0.0);
            if (ix < c) col_sums(base + (long long)(ix + 1) * g.P, iy, ny, tmp, tk, zc);
            const double dx = (ix > 0 && ix < c) ? 4.0 : 2.0;
            const double2 acc = make_double2(cm * fma(dx, tm0.x, tmm.x + tmp.x), cm * fma(dx, tm0.y, tmm.y + tmp.y));
            const long long idx = (long long)j * g.sstride() + (long long)ix * g.P + iy;
            rhs[idx] = make_double2(-g.alpha * acc.y, g.alpha * acc.x);
            nv[0] += g.alpha * g.alpha * (acc.x * acc.x + acc.y * acc.y);
            tmm = tm0;
            tm0 = tmp;
        }
    }
    block_sum<1>(nv, sm);
    if (threadIdx.x == 0) part[blockIdx.x * 4] = nv[0];
}
cudaError_t launch_rhs0(const Geom& g, const double2* h, double2* rhs0, double* part, int* nblk_out, cudaStream_t s) {
    count_launches(1);
    rhs0_kernel<<<512, 256, 0, s>>>(g, h, rhs0, part);
    *nblk_out = 512;
    return cudaGetLastError();
}

// ||rhs0|| per strip: B blocks per strip write partial sums to part (fixed slices of the strip's
// nodes), one thread per strip adds its B partials in order.  part holds N*B doubles.
__global__ void strip_norm_parts_kernel(Geom g, const double2* __restrict__ rhs0, int B, double* __restrict__ part) {
    __shared__ double sm[64];
    const int j = blockIdx.x / B, kb = blockIdx.x - j * B;
    const double2* b = rhs0 + (long long)j * g.sstride();
    const int Ns = g.nxs * g.nyn;
    double v[1] = {0.0};
    for (int n = kb * blockDim.x + threadIdx.x; n < Ns; n += B * blockDim.x) {
        const int ix = n / g.nyn, iy = n - ix * g.nyn;
        const double2 a = b[(long long)ix * g.P + iy];
        v[0] += a.x * a.x + a.y * a.y;
    }
    block_sum<1>(v, sm);
    if (threadIdx.x == 0) part[blockIdx.x] = v[0];
}
__global__ void strip_norm_sum_kernel(int N, int B, const double* __restrict__ part, double* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    double acc = 0.0;
    for (int k = 0; k < B; ++k) acc += part[(long long)j * B + k];
    out[j] = sqrt(acc);
}
cudaError_t launch_strip_norms(const Geom& g, const double2* rhs0, double* out, double* part, int part_cap,
                               cudaStream_t s) {
    // as many blocks per strip as the scratch allows, at most 32 (one block per strip before:
    // 16 blocks for the whole 1024^2 field)
    const int B = std::max(1, std::min(32, part_cap / std::max(1, g.N)));
    count_launches(2);
    strip_norm_parts_kernel<<<g.N * B, 256, 0, s>>>(g, rhs0, B, part);
    strip_norm_sum_kernel<<<(g.N + 127) / 128, 128, 0, s>>>(g.N, B, part, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ flux update
// eq. (fluxlr):  new r_i = -l_{i+1} + 2 S v_{i+1}(a_{i+1}),  new l_{i+1} = -r_i + 2 S v_i(b_i),
// with S of eq. (TCSdist): Robin  S v = -i p v;  S_pade  S v = -i sum_s a_s v + i sum_s a_s d_s phi_s
// (phi_s of the strip the trace belongs to, on that edge).
// Partial sums per block: ||gnew - g||^2, ||gnew||^2.
__device__ __forceinline__ double2 two_S(const Geom& g, double2 v, int pade_m, const double2* phi_e, long long P,
                                         int iy, const double2* pa, const double2* pd) {
    if (pade_m == 0) return make_double2(2.0 * g.p * v.y, -2.0 * g.p * v.x);
    double2 sa = make_double2(0, 0), acc = make_double2(0, 0);
    for (int s = 0; s < pade_m; ++s) {
        sa = cadd(sa, pa[s]);
        acc = cadd(acc, cmul(cmul(pa[s], pd[s]), phi_e[(long long)s * P + iy]));
    }
    // -i sa v + i acc
    const double2 t = csub(acc, cmul(sa, v));
    return make_double2(-2.0 * t.y, 2.0 * t.x);
}
__global__ void traces_kernel(Geom g, const double2* __restrict__ zeta, const double2* __restrict__ gtr,
                              double2* __restrict__ gnew, double* __restrict__ part, int pade_m,
                              const double2* __restrict__ phi, const double2* __restrict__ pa,
                              const double2* __restrict__ pd) {
    __shared__ double sm[64];
    const int c = g.nxs - 1;
    const long long total = (long long)(g.N - 1) * g.nyn;
    double v[2] = {0.0, 0.0};
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int iy = (int)(t % g.nyn);
        const int i = (int)(t / g.nyn);
        const double2 zl = zeta[(long long)((i + 1) * g.nxs + 0) * g.P + iy];     // strip i+1, x = a_{i+1}
        const double2 zr = zeta[(long long)(i * g.nxs + c) * g.P + iy];           // strip i,   x = b_i
        const double2 gr = gtr[(long long)(2 * i) * g.P + iy];
        const double2 gl = gtr[(long long)(2 * i + 1) * g.P + iy];
        const double2* phl = pade_m ? phi + ((long long)(i + 1) * 2 + 0) * pade_m * g.P : nullptr;   // strip i+1, left edge
        const double2* phr = pade_m ? phi + ((long long)i * 2 + 1) * pade_m * g.P : nullptr;         // strip i, right edge
        const double2 sl = two_S(g, zl, pade_m, phl, g.P, iy, pa, pd);
        const double2 sr = two_S(g, zr, pade_m, phr, g.P, iy, pa, pd);
        const double2 nr = make_double2(-gl.x + sl.x, -gl.y + sl.y);
        const double2 nl = make_double2(-gr.x + sr.x, -gr.y + sr.y);
        gnew[(long long)(2 * i) * g.P + iy] = nr;
        gnew[(long long)(2 * i + 1) * g.P + iy] = nl;
        v[0] += (nr.x - gr.x) * (nr.x - gr.x) + (nr.y - gr.y) * (nr.y - gr.y)
              + (nl.x - gl.x) * (nl.x - gl.x) + (nl.y - gl.y) * (nl.y - gl.y);
        v[1] += nr.x * nr.x + nr.y * nr.y + nl.x * nl.x + nl.y * nl.y;
    }
    block_sum<2>(v, sm);
    if (threadIdx.x == 0) { part[blockIdx.x * 4 + 0] = v[0]; part[blockIdx.x * 4 + 1] = v[1]; }
}
cudaError_t launch_traces(const Geom& g, const double2* zeta, const double2* gtr, double2* gnew, double* part,
                          int* nblk_out, cudaStream_t s, int pade_m, const double2* phi, const double2* pa,
                          const double2* pd) {
    const long long total = (long long)(g.N - 1) * g.nyn;
    int nb = nblocks(total, 256);
    if (nb > 512) nb = 512;
    if (nb < 1) nb = 1;
    count_launches(1);
    traces_kernel<<<nb, 256, 0, s>>>(g, zeta, gtr, gnew, part, pade_m, phi, pa, pd);
    *nblk_out = nb;
    return cudaGetLastError();
}

__global__ void finalize_kernel(const double* __restrict__ part, int nblk, int nv, double* __restrict__ out) {
    __shared__ double sm[64];
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
        for (int k = 0; k < nv; ++k) v[k] += part[b * 4 + k];
    block_sum<4>(v, sm);
    if (threadIdx.x == 0)
        for (int k = 0; k < nv; ++k) out[k] = v[k];
}
cudaError_t launch_finalize(const double* part, int nblk, int nv, double* out, cudaStream_t s) {
    count_launches(1);
    finalize_kernel<<<1, 256, 0, s>>>(part, nblk, nv, out);
    return cudaGetLastError();
}

__global__ void sqrt_kernel(double* v) { v[0] = sqrt(v[0]); }
cudaError_t launch_sqrt(double* v, cudaStream_t s) {
    count_launches(1);
    sqrt_kernel<<<1, 1, 0, s>>>(v);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------- commit
// u_n = 2 v - u_{n-1} (eq. CNS); the duplicated interface column of strip j >= 1 takes the
// left strip's v so that both copies stay equal.
__global__ void commit_kernel(Geom g, const double2* __restrict__ zeta, double2* __restrict__ u) {
    const int c = g.nxs - 1;
    const long long total = (long long)g.N * g.nxs * g.nyn;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        int j, ix, iy;
        split_strip_node(t, g.nxs, g.nyn, j, ix, iy);
        const long long idx = (long long)(j * g.nxs + ix) * g.P + iy;
        const long long src = (ix == 0 && j > 0) ? (long long)((j - 1) * g.nxs + c) * g.P + iy : idx;
        const double2 v = zeta[src];
        const double2 uo = u[idx];
        u[idx] = make_double2(2.0 * v.x - uo.x, 2.0 * v.y - uo.y);
    }
}
cudaError_t launch_commit(const Geom& g, const double2* zeta, double2* u, cudaStream_t s) {
    count_launches(1);
    commit_kernel<<<1024, 256, 0, s>>>(g, zeta, u);
    return cudaGetLastError();
}

// ----------------------------------------------------------------- diagnostics
// Per strip (assembly is additive over strips): u^H M u, u^H S u - sum w W |u|^2
// - (kap/2) sum w |u|^4.  Partial sums per block: (mass, energy).
__global__ void diagnostics_kernel(Geom g, const double2* __restrict__ u, const double* __restrict__ Wn,
                                   double* __restrict__ part) {
    __shared__ double sm[64];
    const int c = g.nxs - 1, ny = g.nyn - 1;
    const double cm = g.hx * g.hy / 36.0, ck = g.hy / (6.0 * g.hx), cl = g.hx / (6.0 * g.hy);
    const long long total = (long long)g.N * ((g.nxs + kRX - 1) / kRX) * g.nyn;
    double v[2] = {0.0, 0.0};
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        int j, x0, x1, iy;
        run_item(t, g, j, x0, x1, iy);
        const long long sb = (long long)j * g.sstride() + iy;
        const double2* base = u + sb;
        const double wy = wq(iy, ny, g.hy);
        double2 tmm = make_double2(0.0, 0.0), tkm = tmm, tm0, tk0, z0, zd;
        if (x0 > 0) col_sums(base + (long long)(x0 - 1) * g.P, iy, ny, tmm, tkm, zd);
        col_sums(base + (long long)x0 * g.P, iy, ny, tm0, tk0, z0);
        for (int ix = x0; ix < x1; ++ix) {
            double2 tmp = make_double2(0.0, 0.0), tkp = tmp, zp = tmp;
            if (ix < c) col_sums(base + (long long)(ix + 1) * g.P, iy, ny, tmp, tkp, zp);
            const bool in = ix > 0 && ix < c;
            const double dx = in ? 4.0 : 2.0, ex = in ? 2.0 : 1.0;
            // M u = cm [1 dx 1] tm;  S u = ck [-1 ex -1] tm + cl [1 dx 1] tk
            const double2 Mu = make_double2(cm * fma(dx, tm0.x, tmm.x + tmp.x), cm * fma(dx, tm0.y, tmm.y + tmp.y));
            const double2 Su = make_double2(ck * fma(ex, tm0.x, -(tmm.x + tmp.x)) + cl * fma(dx, tk0.x, tkm.x + tkp.x),
                                            ck * fma(ex, tm0.y, -(tmm.y + tmp.y)) + cl * fma(dx, tk0.y, tkm.y + tkp.y));
            const double a2 = z0.x * z0.x + z0.y * z0.y;
            const double w = wq(ix, c, g.hx) * wy;
            const double W = Wn ? Wn[sb + (long long)ix * g.P] : 0.0;
            v[0] += z0.x * Mu.x + z0.y * Mu.y;
            v[1] += z0.x * Su.x + z0.y * Su.y - w * W * a2 - 0.5 * g.kap * w * a2 * a2;
            tmm = tm0; tkm = tk0;
            tm0 = tmp; tk0 = tkp; z0 = zp;
        }
    }
    block_sum<2>(v, sm);
    if (threadIdx.x == 0) { part[blockIdx.x * 4 + 0] = v[0]; part[blockIdx.x * 4 + 1] = v[1]; }
}
cudaError_t launch_diagnostics(const Geom& g, const double2* u, const double* Wn, double* part, int* nblk_out,
                               cudaStream_t s) {
    count_launches(1);
    diagnostics_kernel<<<512, 256, 0, s>>>(g, u, Wn, part);
    *nblk_out = 512;
    return cudaGetLastError();
}

// ----------------------------------------------------------------------- L_h
// Virtual strip v solved the free strip problem with the unit datum e_pos on its left
// (side 0) or right (side 1) edge.  Its outgoing traces (eq. fluxlr / AlgoGraph)
//   out_left  = -l + 2 S v(a),  out_right = -r + 2 S v(b)
// are column pos of X1, X3 (unit l) or X2, X4 (unit r) (Props 3.1 / 3.2, Sec. 4.2).
// X: 4 row-major nyn x nyn blocks.
__global__ void extract_blocks_kernel(Geom g, const double2* __restrict__ zeta, int nvirt, int unit_base,
                                      double2* __restrict__ X) {
    const int c = g.nxs - 1, nyn = g.nyn;
    const long long total = (long long)nvirt * nyn;
    const long long bs = (long long)nyn * nyn;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int iy = (int)(t % nyn);
        const int v = (int)(t / nyn);
        const int u = unit_base + v;
        const int side = u / nyn, pos = u - side * nyn;
        const double2 zl = zeta[(long long)(v * g.nxs + 0) * g.P + iy];
        const double2 zr = zeta[(long long)(v * g.nxs + c) * g.P + iy];
        double2 ol = make_double2(2.0 * g.p * zl.y, -2.0 * g.p * zl.x);   // 2 S v = -2ip v
        double2 orr = make_double2(2.0 * g.p * zr.y, -2.0 * g.p * zr.x);
        if (iy == pos) {
            if (side == 0) ol.x -= 1.0; else orr.x -= 1.0;
        }
        const long long e = (long long)iy * nyn + pos;
        if (side == 0) { X[0 * bs + e] = ol; X[2 * bs + e] = orr; }
        else { X[1 * bs + e] = ol; X[3 * bs + e] = orr; }
    }
}
cudaError_t launch_extract_blocks(const Geom& g, const double2* zeta, int nvirt, int unit_base, double2* X,
                                  cudaStream_t s) {
    count_launches(1);
    extract_blocks_kernel<<<nblocks((long long)nvirt * g.nyn, 256) < 4096 ? nblocks((long long)nvirt * g.nyn, 256) : 4096, 256, 0, s>>>(
        g, zeta, nvirt, unit_base, X);
    return cudaGetLastError();
}

__global__ void convert_kernel(const double2* __restrict__ X, float2* __restrict__ Xf, long long n) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        Xf[t] = make_float2((float)X[t].x, (float)X[t].y);
}
cudaError_t launch_convert_blocks(const double2* X, float2* Xf, long long n, cudaStream_t s) {
    count_launches(1);
    convert_kernel<<<2048, 256, 0, s>>>(X, Xf, n);
    return cudaGetLastError();
}

// y = x - L_h x.  Output trace o is fed by exactly one strip:
//   o = 2(j-1) (new r_{j-1}):  X1 l_j + X2 r_j,     o = 2j+1 (new l_{j+1}): X3 l_j + X4 r_j,
// with l_j = x[2(j-1)+1] (j > 0) and r_j = x[2j] (j < N-1).  One warp per output node.
template <typename TX> struct Acc;
template <> struct Acc<float2> { using t = float; };
template <> struct Acc<double2> { using t = double; };

template <typename TX>
__global__ void apply_P_kernel(Geom g, const TX* __restrict__ X, const int* __restrict__ btype,
                               const double2* __restrict__ x, double2* __restrict__ y) {
    using A = typename Acc<TX>::t;    // accumulate in the precision of the blocks
    const int nyn = g.nyn, P = g.P;
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long total = (long long)2 * (g.N - 1) * nyn;
    const long long bs = (long long)nyn * nyn;
    for (long long t = warp; t < total; t += nwarps) {
        const int row = (int)(t % nyn);
        const int o = (int)(t / nyn);
        int j, ka, kb;
        if ((o & 1) == 0) { j = o / 2 + 1; ka = 0; kb = 1; }    // new r_{j-1}
        else { j = (o - 1) / 2; ka = 2; kb = 3; }               // new l_{j+1}
        const TX* Xs = X + (long long)btype[j] * 4 * bs;
        const double2* in_l = j > 0 ? x + (long long)(2 * (j - 1) + 1) * P : nullptr;
        const double2* in_r = j < g.N - 1 ? x + (long long)(2 * j) * P : nullptr;
        A sr = 0, si = 0;
        const TX* ra = Xs + ka * bs + (long long)row * nyn;
        const TX* rb = Xs + kb * bs + (long long)row * nyn;
        for (int col = lane; col < nyn; col += 32) {
            if (in_l) {
                const TX a = ra[col];
                const double2 v = in_l[col];
                const A vx = (A)v.x, vy = (A)v.y;
                sr += a.x * vx - a.y * vy;
                si += a.x * vy + a.y * vx;
            }
            if (in_r) {
                const TX b = rb[col];
                const double2 v = in_r[col];
                const A vx = (A)v.x, vy = (A)v.y;
                sr += b.x * vx - b.y * vy;
                si += b.x * vy + b.y * vx;
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            sr += __shfl_xor_sync(0xffffffffu, sr, off);
            si += __shfl_xor_sync(0xffffffffu, si, off);
        }
        if (lane == 0) {
            const long long e = (long long)o * P + row;
            y[e] = make_double2(x[e].x - (double)sr, x[e].y - (double)si);
        }
    }
}
cudaError_t launch_apply_P(const Geom& g, const void* X, bool fp32, const int* btype_dev, const double2* x,
                           double2* y, double2* work, cudaStream_t s) {
    (void)work;
    const long long total = (long long)2 * (g.N - 1) * g.nyn;
    int nb = nblocks(total * 32, 256);
    if (nb > 8192) nb = 8192;
    count_launches(1);
    if (fp32)
        apply_P_kernel<float2><<<nb, 256, 0, s>>>(g, (const float2*)X, btype_dev, x, y);
    else
        apply_P_kernel<double2><<<nb, 256, 0, s>>>(g, (const double2*)X, btype_dev, x, y);
    return cudaGetLastError();
}

// ----------------------------------------------------------------- GMRES vectors
// out[i] = V_i^H w for i < k (V_i at V + i*ld), two-pass fixed-order reduction.
__global__ void dots_partial_kernel(const double2* __restrict__ V, long long ld, const double2* __restrict__ w,
                                    long long n, double* __restrict__ scratch) {
    __shared__ double sm[64];
    const int i = blockIdx.y;
    const double2* vi = V + (long long)i * ld;
    double v[2] = {0.0, 0.0};
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const double2 a = vi[t], b = w[t];
        v[0] += a.x * b.x + a.y * b.y;
        v[1] += a.x * b.y - a.y * b.x;
    }
    block_sum<2>(v, sm);
    if (threadIdx.x == 0) {
        scratch[((long long)i * gridDim.x + blockIdx.x) * 2 + 0] = v[0];
        scratch[((long long)i * gridDim.x + blockIdx.x) * 2 + 1] = v[1];
    }
}
__global__ void dots_final_kernel(const double* __restrict__ scratch, int nb, double2* __restrict__ out) {
    __shared__ double sm[64];
    const int i = blockIdx.x;
    double v[2] = {0.0, 0.0};
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        v[0] += scratch[((long long)i * nb + b) * 2 + 0];
        v[1] += scratch[((long long)i * nb + b) * 2 + 1];
    }
    block_sum<2>(v, sm);
    if (threadIdx.x == 0) out[i] = make_double2(v[0], v[1]);
}
cudaError_t launch_dots(const double2* V, long long ld, int k, const double2* w, long long n, double2* out,
                        double* scratch, cudaStream_t s) {
    int nb = nblocks(n, 256);
    if (nb > 128) nb = 128;
    count_launches(1);
    dots_partial_kernel<<<dim3(nb, k), 256, 0, s>>>(V, ld, w, n, scratch);
    count_launches(1);
    dots_final_kernel<<<k, 128, 0, s>>>(scratch, nb, out);
    return cudaGetLastError();
}

// w -= sum_i h_i V_i  (h complex, i < k)
__global__ void axpy_multi_kernel(const double2* __restrict__ V, long long ld, int k, const double2* __restrict__ h,
                                  double2* __restrict__ w, long long n) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        double2 acc = w[t];
        for (int i = 0; i < k; ++i) {
            const double2 a = V[(long long)i * ld + t], c = h[i];
            acc.x -= c.x * a.x - c.y * a.y;
            acc.y -= c.x * a.y + c.y * a.x;
        }
        w[t] = acc;
    }
}
cudaError_t launch_axpy_multi(const double2* V, long long ld, int k, const double2* h, double2* w, long long n,
                              cudaStream_t s) {
    int nb = nblocks(n, 256);
    if (nb > 2048) nb = 2048;
    count_launches(1);
    axpy_multi_kernel<<<nb, 256, 0, s>>>(V, ld, k, h, w, n);
    return cudaGetLastError();
}

__global__ void nrm2_partial_kernel(const double2* __restrict__ w, long long n, double* __restrict__ scratch) {
    __shared__ double sm[64];
    double v[1] = {0.0};
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const double2 a = w[t];
        v[0] += a.x * a.x + a.y * a.y;
    }
    block_sum<1>(v, sm);
    if (threadIdx.x == 0) scratch[blockIdx.x] = v[0];
}
__global__ void nrm2_final_kernel(const double* __restrict__ scratch, int nb, double* __restrict__ out) {
    __shared__ double sm[64];
    double v[1] = {0.0};
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v[0] += scratch[b];
    block_sum<1>(v, sm);
    if (threadIdx.x == 0) out[0] = sqrt(v[0]);
}
cudaError_t launch_nrm2(const double2* w, long long n, double* out, double* scratch, cudaStream_t s) {
    int nb = nblocks(n, 256);
    if (nb > 128) nb = 128;
    count_launches(1);
    nrm2_partial_kernel<<<nb, 256, 0, s>>>(w, n, scratch);
    count_launches(1);
    nrm2_final_kernel<<<1, 128, 0, s>>>(scratch, nb, out);
    return cudaGetLastError();
}

__global__ void scale_kernel(double2* __restrict__ y, const double2* __restrict__ x, const double* __restrict__ nrm, long long n) {
    const double s = nrm[0] > 0.0 ? 1.0 / nrm[0] : 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        y[t] = make_double2(x[t].x * s, x[t].y * s);
}
cudaError_t launch_scale(double2* y, const double2* x, const double* inv_from, long long n, cudaStream_t s) {
    int nb = nblocks(n, 256);
    if (nb > 2048) nb = 2048;
    count_launches(1);
    scale_kernel<<<nb, 256, 0, s>>>(y, x, inv_from, n);
    return cudaGetLastError();
}
__global__ void sub_kernel(double2* __restrict__ y, const double2* __restrict__ a, const double2* __restrict__ b, long long n) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        y[t] = make_double2(a[t].x - b[t].x, a[t].y - b[t].y);
}
cudaError_t launch_sub(double2* y, const double2* a, const double2* b, long long n, cudaStream_t s) {
    int nb = nblocks(n, 256);
    if (nb > 2048) nb = 2048;
    count_launches(1);
    sub_kernel<<<nb, 256, 0, s>>>(y, a, b, n);
    return cudaGetLastError();
}
cudaError_t launch_copy(double2* y, const double2* x, long long n, cudaStream_t s) {
    return cudaMemcpyAsync(y, x, n * sizeof(double2), cudaMemcpyDeviceToDevice, s);
}

}  // namespace ddnls
