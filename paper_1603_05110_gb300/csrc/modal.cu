// Exact P^{-1} of eq. (algo_pd) in the cosine basis.
//
// L_h (eq. Lmpi) is the interface map of the free equation (V = 0, f = 0, Props 3.1/3.2).
// On a strip of the uniform Q1 mesh with homogeneous Neumann data on y = yb, yu the free strip
// operator is Bx (x) My - Mx (x) Ky with Bx = (2i/dt) Mx - Kx + i p E_x.  The 1D matrices
// My = (h/6)(4D + T), Ky = (1/h)(2D - T), D = diag(1/2, 1, .., 1, 1/2), share the generalised
// eigenvectors z_k(j) = cos(pi j k / ny):  My z_k = mu_k D z_k,  Ky z_k = lambda_k D z_k,
//     mu_k = (h/6)(4 + 2 cos th_k),  lambda_k = (2 - 2 cos th_k)/h,  th_k = pi k / ny.
// A datum l = z_k on the left edge therefore produces v = -w (x) z_k with
//     (mu_k Bx - lambda_k Mx) w = mu_k e_0
// (a tridiagonal solve across the strip), so each block X^{j,a} of L_h is diagonal in the z_k
// basis with entries x1 = -1 + 2ip w_l(0), x2 = 2ip w_r(0), x3 = 2ip w_l(c), x4 = -1 + 2ip w_r(c)
// (Robin, 2 S v = -2ip v).  P = I - L_h splits into ny+1 independent systems of size 2(N-1),
// block tridiagonal in 2x2 blocks (one block per interface), factored once at set-up.
// Applying P^{-1}: cosine transform of every trace, per-mode block-Thomas sweeps, inverse
// transform.  This is the same P as the paper's, solved exactly instead of by GMRES.
#include "common.cuh"
#include "kernels.h"

#include <algorithm>

namespace ddnls {

// C_fwd[k][j] = D_j cos(pi j k/ny) / sigma_k,  C_inv[j][k] = cos(pi j k/ny)
// (sigma_k = sum_j D_j cos^2 = ny/2, or ny for k = 0, ny).  Arguments reduced mod 2 ny.
__global__ void cosine_matrices_kernel(int ny, double* __restrict__ Cf, double* __restrict__ Ci) {
    const int n = ny + 1;
    const long long total = (long long)n * n;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(t / n), c = (int)(t % n);
        const long long m = ((long long)r * c) % (2LL * ny);
        const double cs = ny > 0 ? cospi((double)m / (double)ny) : 1.0;
        // Cf: row k = r, column j = c
        const double Dj = (c == 0 || c == ny) ? 0.5 : 1.0;
        const double sig = ny == 0 ? 1.0 : ((r == 0 || r == ny) ? (double)ny : 0.5 * ny);
        Cf[t] = Dj * cs / sig;
        Ci[t] = cs;     // Ci: row j = r, column k = c (symmetric in r, c)
    }
}

__global__ void to_float_kernel(const double* __restrict__ a, float* __restrict__ b, long long n) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        b[t] = (float)a[t];
}

// Per strip type (ltc, rtc) and mode k: x1..x4 of the diagonal blocks.  S_k is the transmission
// operator on mode k: -i p (Robin), or -i sum a_s + i sum a_s d_s mu_k / dh_s with
// dh_s = i alpha mu_k - lambda_k + d_s mu_k, since the auxiliary equation (eq. TCS_phi) of the
// free problem, D_s phi_s = M^G v, is diagonal on the modes too (S_pade).
__global__ void modal_eigs_kernel(Geom g, int ntypes, const int* __restrict__ tkind, double2* __restrict__ xm,
                                  double2* __restrict__ work, int pade_m, const double2* __restrict__ pa,
                                  const double2* __restrict__ pd) {
    const int n = g.nyn, ny = n - 1, c = g.nxs - 1, m = c + 1;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntypes * n) return;
    const int type = t / n, k = t - type * n;
    const int ltc = tkind[2 * type], rtc = tkind[2 * type + 1];
    const double th = ny > 0 ? (double)k / ny : 0.0;
    const double ck = cospi(th);
    const double mu = g.hy / 6.0 * (4.0 + 2.0 * ck);
    const double la = (2.0 - 2.0 * ck) / g.hy;
    double2 Sk = make_double2(0.0, -g.p);
    if (pade_m > 0) {
        double2 sa = make_double2(0, 0), acc = make_double2(0, 0);
        for (int s = 0; s < pade_m; ++s) {
            sa = cadd(sa, pa[s]);
            const double2 dh = make_double2(-la + pd[s].x * mu, g.alpha * mu + pd[s].y * mu);
            acc = cadd(acc, cmul(cmul(pa[s], pd[s]), cmul(make_double2(mu, 0.0), cinv(dh))));
        }
        const double2 t = csub(acc, sa);          // -sa + acc, times i
        Sk = make_double2(-t.y, t.x);
    }
    const double2 rk = make_double2(-Sk.x, -Sk.y);   // edge coefficient rho_k = -S_k
    // T = mu Bx - la Mx, tridiagonal; Bx = i alpha Mx - Kx + i p E
    double2* cp = work + (long long)t * 2 * m;   // Thomas scratch (c', d')
    double2* dp = cp + m;
    double2 out[4];
    for (int side = 0; side < 2; ++side) {
        const int active = side == 0 ? ltc : rtc;
        if (!active) { out[side] = out[side + 2] = make_double2(0, 0); continue; }   // side 0: x1, x3; side 1: x2, x4
        for (int i = 0; i < m; ++i) {
            const bool lo = i > 0, hi = i < c;
            const double mii = (lo && hi) ? g.mxi : g.mxe, kii = (lo && hi) ? g.kxi : g.kxe;
            double pre = 0.0, pim = 0.0;
            if (i == 0 && ltc) { pre += rk.x; pim += rk.y; }
            if (i == c && rtc) { pre += rk.x; pim += rk.y; }
            const double2 diag = make_double2(-mu * kii - la * mii + mu * pre, mu * (g.alpha * mii + pim));
            const double2 off = make_double2(-mu * g.kxo - la * g.mxo, mu * g.alpha * g.mxo);
            const double2 rhs = make_double2((side == 0 && i == 0) || (side == 1 && i == c) ? mu : 0.0, 0.0);
            if (i == 0) {
                const double2 inv = cinv(diag);
                cp[0] = hi ? cmul(off, inv) : make_double2(0, 0);
                dp[0] = cmul(rhs, inv);
            } else {
                const double2 den = csub(diag, cmul(off, cp[i - 1]));
                const double2 inv = cinv(den);
                cp[i] = hi ? cmul(off, inv) : make_double2(0, 0);
                dp[i] = cmul(csub(rhs, cmul(off, dp[i - 1])), inv);
            }
        }
        // back substitution, only w(0) and w(c) are needed but the sweep is sequential
        double2 wnext = dp[m - 1];
        const double2 wc = wnext;
        for (int i = m - 2; i >= 0; --i) wnext = csub(dp[i], cmul(cp[i], wnext));
        const double2 w0 = wnext;
        // -2 S_k w (the datum enters the right side with a minus sign)
        const double2 a0 = cmul(make_double2(-2.0 * Sk.x, -2.0 * Sk.y), w0);
        const double2 ac = cmul(make_double2(-2.0 * Sk.x, -2.0 * Sk.y), wc);
        if (side == 0) { out[0] = make_double2(a0.x - 1.0, a0.y); out[2] = ac; }   // x1, x3
        else { out[1] = a0; out[3] = make_double2(ac.x - 1.0, ac.y); }             // x2, x4
    }
    // layout xm[type][a][k]
    for (int a = 0; a < 4; ++a) xm[((long long)type * 4 + a) * n + k] = out[a];
}

__device__ __forceinline__ void inv2(const double2 (&A)[4], double2 (&B)[4]) {
    // [a b; c d]^-1 = [d -b; -c a] / (ad - bc)
    const double2 det = csub(cmul(A[0], A[3]), cmul(A[1], A[2]));
    const double2 id = cinv(det);
    B[0] = cmul(A[3], id);
    B[1] = cmul(make_double2(-A[1].x, -A[1].y), id);
    B[2] = cmul(make_double2(-A[2].x, -A[2].y), id);
    B[3] = cmul(A[0], id);
}
__device__ __forceinline__ void mul2(const double2 (&A)[4], const double2 (&B)[4], double2 (&C)[4]) {
    C[0] = cadd(cmul(A[0], B[0]), cmul(A[1], B[2]));
    C[1] = cadd(cmul(A[0], B[1]), cmul(A[1], B[3]));
    C[2] = cadd(cmul(A[2], B[0]), cmul(A[3], B[2]));
    C[3] = cadd(cmul(A[2], B[1]), cmul(A[3], B[3]));
}

// Block-Thomas factors per mode k.  Unknown block i (interface i) = (new r_i, new l_{i+1}):
//   D_i  = [1, -x1(t_{i+1}); -x4(t_i), 1],  Lo_i = [0, 0; 0, -x3(t_i)],  Up_i = [-x2(t_{i+1}), 0; 0, 0]
// S_0 = D_0, S_i = D_i - Lo_i S_{i-1}^{-1} Up_{i-1}.  Stored per (i, entry, k):
//   e 0..3: S_i^{-1};  e 4..7: G_i = Lo_i S_{i-1}^{-1};  e 8: Up_i(0,0).
__global__ void modal_factor_kernel(Geom g, const int* __restrict__ btype, const double2* __restrict__ xm,
                                    double2* __restrict__ fac) {
    const int n = g.nyn, NI = g.N - 1;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    auto X = [&](int strip, int a) { return xm[((long long)btype[strip] * 4 + a) * n + k]; };
    auto F = [&](int i, int e) -> double2& { return fac[((long long)i * 9 + e) * n + k]; };
    double2 Sprev_inv[4];
    double2 up_prev = make_double2(0, 0);
    for (int i = 0; i < NI; ++i) {
        double2 D[4];
        D[0] = make_double2(1, 0);
        D[1] = make_double2(-X(i + 1, 0).x, -X(i + 1, 0).y);
        D[2] = make_double2(-X(i, 3).x, -X(i, 3).y);
        D[3] = make_double2(1, 0);
        double2 G[4] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
        if (i > 0) {
            // Lo_i = [0 0; 0 lo], lo = -x3(t_i);  G = Lo S^{-1}: only row 1 nonzero
            const double2 lo = make_double2(-X(i, 2).x, -X(i, 2).y);
            G[2] = cmul(lo, Sprev_inv[2]);
            G[3] = cmul(lo, Sprev_inv[3]);
            // S_i = D_i - G Up_{i-1},  Up_{i-1} = [up 0; 0 0]
            D[2] = csub(D[2], cmul(G[2], up_prev));
        }
        double2 Si[4];
        inv2(D, Si);
        for (int e = 0; e < 4; ++e) { F(i, e) = Si[e]; F(i, 4 + e) = G[e]; }
        const double2 up = (i + 1 < NI) ? make_double2(-X(i + 1, 1).x, -X(i + 1, 1).y) : make_double2(0, 0);
        F(i, 8) = up;
        for (int e = 0; e < 4; ++e) Sprev_inv[e] = Si[e];
        up_prev = up;
    }
}

// y (modal coefficients of the right side, interface layout [2(N-1)][P]) -> x in place.
// Sweeps in the precision of the factors: FP64, or FP32 in the FP32 forms (whose cosine
// transforms around this solve are FP32 already).
// Modes k >= kmax (kmax > 0) are left as they are: P = I there (the partially constructed
// I - L_h of the paper's conclusion, on the low modes only).
template <typename T2>
__global__ void modal_solve_kernel(Geom g, const T2* __restrict__ fac, double2* __restrict__ y, int kmax) {
    const int n = g.nyn, NI = g.N - 1, P = g.P;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n || (kmax > 0 && k >= kmax)) return;
    auto F = [&](int i, int e) { return fac[((long long)i * 9 + e) * n + k]; };
    // forward: Yt_i = Y_i - G_i Yt_{i-1}
    auto ld = [&](long long q) { const double2 v = y[q]; return mk<T2>(v.x, v.y); };
    auto st = [&](long long q, T2 v) { y[q] = make_double2((double)v.x, (double)v.y); };
    T2 p0 = mk<T2>(0, 0), p1 = mk<T2>(0, 0);
    for (int i = 0; i < NI; ++i) {
        T2 a = ld((long long)(2 * i) * P + k), b = ld((long long)(2 * i + 1) * P + k);
        if (i > 0) {
            a = csub(a, cadd(cmul(F(i, 4), p0), cmul(F(i, 5), p1)));
            b = csub(b, cadd(cmul(F(i, 6), p0), cmul(F(i, 7), p1)));
        }
        st((long long)(2 * i) * P + k, a);
        st((long long)(2 * i + 1) * P + k, b);
        p0 = a;
        p1 = b;
    }
    // backward: U_i = S_i^{-1} (Yt_i - Up_i U_{i+1}),  Up_i U_{i+1} = (up * U_{i+1}[0], 0)
    T2 n0 = mk<T2>(0, 0);
    for (int i = NI - 1; i >= 0; --i) {
        T2 a = ld((long long)(2 * i) * P + k), b = ld((long long)(2 * i + 1) * P + k);
        a = csub(a, cmul(F(i, 8), n0));
        const T2 u0 = cadd(cmul(F(i, 0), a), cmul(F(i, 1), b));
        const T2 u1 = cadd(cmul(F(i, 2), a), cmul(F(i, 3), b));
        st((long long)(2 * i) * P + k, u0);
        st((long long)(2 * i + 1) * P + k, u1);
        n0 = u0;
    }
}

// The same solve with each mode's right side and factors first staged in shared memory: one
// warp of 32 modes per block, every load of the mode issued before the first step of its sweep
// (the sweeps are chains of 2(N-1) dependent steps; loading inside them exposes one memory
// latency per step).  Each thread reads only its own column of the staged arrays.
constexpr int kCosSlices = 8;
template <typename T2>
__global__ void modal_solve_staged_kernel(Geom g, const T2* __restrict__ fac, double2* __restrict__ y, int kmax) {
    extern __shared__ __align__(16) unsigned char s_modal[];
    const int n = g.nyn, NI = g.N - 1, P = g.P, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const int k0 = blockIdx.x * 32;
    T2* Fs = (T2*)s_modal;                       // [NI * 9][32]
    T2* Ys = Fs + (size_t)NI * 9 * 32;           // [2 NI][32]
    const T2 zero = mk<T2>(0, 0);
    // staging by all warps of the block (more loads in flight); warp 0 then runs the sweeps
    {
        const int kk = k0 + lane;
        const bool in = kk < n;
#pragma unroll 4
        for (int q = wid; q < NI * 9; q += nw) Fs[q * 32 + lane] = in ? fac[(long long)q * n + kk] : zero;
#pragma unroll 4
        for (int q = wid; q < 2 * NI; q += nw) {
            const double2 v = in ? y[(long long)q * P + kk] : make_double2(0.0, 0.0);
            Ys[q * 32 + lane] = mk<T2>(v.x, v.y);
        }
    }
    __syncthreads();
    const int k = k0 + lane;
    const bool on = wid == 0 && k < n && !(kmax > 0 && k >= kmax);
    if (!on) return;
    auto F = [&](int i, int e) { return Fs[(i * 9 + e) * 32 + lane]; };
    auto Y = [&](int q) -> T2& { return Ys[q * 32 + lane]; };
    // forward: Yt_i = Y_i - G_i Yt_{i-1}
    T2 p0 = zero, p1 = zero;
    for (int i = 0; i < NI; ++i) {
        T2 a = Y(2 * i), b = Y(2 * i + 1);
        if (i > 0) {
            a = csub(a, cadd(cmul(F(i, 4), p0), cmul(F(i, 5), p1)));
            b = csub(b, cadd(cmul(F(i, 6), p0), cmul(F(i, 7), p1)));
        }
        Y(2 * i) = a;
        Y(2 * i + 1) = b;
        p0 = a;
        p1 = b;
    }
    // backward: U_i = S_i^{-1} (Yt_i - Up_i U_{i+1})
    T2 n0 = zero;
    for (int i = NI - 1; i >= 0; --i) {
        T2 a = Y(2 * i), b = Y(2 * i + 1);
        a = csub(a, cmul(F(i, 8), n0));
        const T2 u0 = cadd(cmul(F(i, 0), a), cmul(F(i, 1), b));
        const T2 u1 = cadd(cmul(F(i, 2), a), cmul(F(i, 3), b));
        Y(2 * i) = u0;
        Y(2 * i + 1) = u1;
        n0 = u0;
    }
#pragma unroll 8
    for (int q = 0; q < 2 * NI; ++q) {
        const T2 v = Y(q);
        y[(long long)q * P + k] = make_double2((double)v.x, (double)v.y);
    }
}

// part[kz][o][r] = sum over c in slice kz of C[r][c] in[o][c], for the ntr traces of an interface
// vector (pitch P); in2 (nullable): the transform of in - in2.  Tiles of 32 rows x 8 traces per
// block, C and the trace tile staged in shared memory; the column range is split into kCosSlices
// slices (grid z) so that a 1025-point transform of 30 traces spreads over ~1000 blocks.
template <typename T>
__global__ void __launch_bounds__(256) cosine_partial_kernel(int n, int ntr, int P, int klen, const T* __restrict__ C,
                                                             const double2* __restrict__ in,
                                                             const double2* __restrict__ in2,
                                                             typename C2<T>::t* __restrict__ part) {
    using T2 = typename C2<T>::t;
    __shared__ T Cs[32][33];
    __shared__ T2 Is[8][32];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int r0 = blockIdx.x * 32, o0 = blockIdx.y * 8;
    const int r = r0 + tx, o = o0 + ty;
    const int kb = blockIdx.z * klen, ke = min(n, kb + klen);
    T ar = 0, ai = 0;
    for (int c0 = kb; c0 < ke; c0 += 32) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int rr = r0 + ty * 4 + q, cc = c0 + tx;
            Cs[ty * 4 + q][tx] = (rr < n && cc < ke) ? C[(long long)rr * n + cc] : (T)0;
        }
        {
            const int cc = c0 + tx;
            double2 v = make_double2(0, 0);
            if (o < ntr && cc < ke) {
                v = in[(long long)o * P + cc];
                if (in2) {
                    const double2 w = in2[(long long)o * P + cc];
                    v.x -= w.x;
                    v.y -= w.y;
                }
            }
            Is[ty][tx] = mk<T2>(v.x, v.y);
        }
        __syncthreads();
#pragma unroll 8
        for (int cc = 0; cc < 32; ++cc) {
            const T cv = Cs[tx][cc];
            const T2 iv = Is[ty][cc];
            ar += cv * iv.x;
            ai += cv * iv.y;
        }
        __syncthreads();
    }
    if (r < n && o < ntr) {
        T2 v;
        v.x = ar;
        v.y = ai;
        part[((long long)blockIdx.z * ntr + o) * P + r] = v;
    }
}

// out[o][r] = the slices' partial sums, added in slice order; from (nullable): out = from - sum
template <typename T2>
__global__ void cosine_reduce_kernel(int n, int ntr, int P, const T2* __restrict__ part, const double2* __restrict__ from,
                                     double2* __restrict__ out) {
    const long long total = (long long)ntr * n;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int o = (int)(t / n), r = (int)(t - (long long)o * n);
        T2 acc = part[(long long)o * P + r];
#pragma unroll
        for (int kz = 1; kz < kCosSlices; ++kz) {
            const T2 v = part[((long long)kz * ntr + o) * P + r];
            acc.x += v.x;
            acc.y += v.y;
        }
        double2 v = make_double2((double)acc.x, (double)acc.y);
        if (from) {
            const double2 f = from[(long long)o * P + r];
            v = make_double2(f.x - v.x, f.y - v.y);
        }
        out[(long long)o * P + r] = v;
    }
}

// the partial sums of the transform of in (- in2)
template <typename T>
static cudaError_t cosine_partial(int n, int ntr, int P, const T* C, const double2* in, const double2* in2, void* part,
                                  cudaStream_t s) {
    using T2 = typename C2<T>::t;
    const int klen = ((n + kCosSlices - 1) / kCosSlices + 31) / 32 * 32;
    dim3 grid((n + 31) / 32, (ntr + 7) / 8, kCosSlices);
    count_launches(1);
    cosine_partial_kernel<T><<<grid, 256, 0, s>>>(n, ntr, P, klen, C, in, in2, (T2*)part);
    return cudaGetLastError();
}
template <typename T>
static cudaError_t cosine_reduce(int n, int ntr, int P, const void* part, const double2* from, double2* out,
                                 cudaStream_t s) {
    using T2 = typename C2<T>::t;
    const long long total = (long long)ntr * n;
    const int nb = (int)std::min<long long>((total + 255) / 256, 152LL * 8);
    count_launches(1);
    cosine_reduce_kernel<T2><<<nb, 256, 0, s>>>(n, ntr, P, (const T2*)part, from, out);
    return cudaGetLastError();
}

// The per-mode solve on y in place: one warp per block (the per-mode sweeps are chains, spread
// over as many SMs as possible), staged in shared memory when the mode's data fit.
static cudaError_t modal_solve(const Geom& g, bool f32, const double2* fac, const float2* fac32, double2* y, int kmax,
                               cudaStream_t s) {
    count_launches(1);
    const int NI = g.N - 1;
    const size_t smem = (size_t)11 * NI * 32 * (f32 ? sizeof(float2) : sizeof(double2));
    bool staged = smem <= 220 * 1024;
    if (staged) {
        const void* kfn = f32 ? (const void*)modal_solve_staged_kernel<float2> : (const void*)modal_solve_staged_kernel<double2>;
        if (cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(smem, 1)) != cudaSuccess) {
            cudaGetLastError();
            staged = false;
        }
    }
    if (staged) {
        if (f32) modal_solve_staged_kernel<float2><<<(g.nyn + 31) / 32, 128, smem, s>>>(g, fac32, y, kmax);
        else modal_solve_staged_kernel<double2><<<(g.nyn + 31) / 32, 128, smem, s>>>(g, fac, y, kmax);
    } else if (f32) {
        modal_solve_kernel<float2><<<(g.nyn + 31) / 32, 32, 0, s>>>(g, fac32, y, kmax);
    } else {
        modal_solve_kernel<double2><<<(g.nyn + 31) / 32, 32, 0, s>>>(g, fac, y, kmax);
    }
    return cudaGetLastError();
}

cudaError_t launch_to_float(const double* a, float* b, long long n, cudaStream_t s) {
    count_launches(1);
    to_float_kernel<<<2048, 256, 0, s>>>(a, b, n);
    return cudaGetLastError();
}

cudaError_t launch_modal_setup(const Geom& g, int ntypes, const int* tkind_dev, const int* btype_dev,
                               double* Cf, double* Ci, float* Cf32, float* Ci32, double2* xm, double2* fac,
                               double2* work, cudaStream_t s, int pade_m, const double2* pa, const double2* pd) {
    const long long nn = (long long)g.nyn * g.nyn;
    count_launches(1);
    cosine_matrices_kernel<<<2048, 256, 0, s>>>(g.nyn - 1, Cf, Ci);
    if (Cf32) {
        count_launches(2);
        to_float_kernel<<<2048, 256, 0, s>>>(Cf, Cf32, nn);
        to_float_kernel<<<2048, 256, 0, s>>>(Ci, Ci32, nn);
    }
    const int nt = ntypes * g.nyn;
    count_launches(2);
    modal_eigs_kernel<<<(nt + 127) / 128, 128, 0, s>>>(g, ntypes, tkind_dev, xm, work, pade_m, pa, pd);
    modal_factor_kernel<<<(g.nyn + 127) / 128, 128, 0, s>>>(g, btype_dev, xm, fac);
    return cudaGetLastError();
}


// g_new = g_k - P^{-1} (g_k - R(g_k))  (eq. algo_pd) in five launches: the forward transform
// forms y = g_k - R(g_k) as it reads, and the inverse transform's reduction subtracts from g_k.
// g_new may be rg; tmp (the modal coefficients) may alias rg too.
cudaError_t launch_modal_update(const Geom& g, bool fp32, const double* Cf, const double* Ci, const float* Cf32,
                                const float* Ci32, const double2* fac, const float2* fac32, const double2* gk,
                                const double2* rg, double2* gnew, double2* tmp, void* cpart, int kmax, cudaStream_t s) {
    const int ntr = 2 * (g.N - 1), n = g.nyn, P = g.P;
    cudaError_t e = fp32 ? cosine_partial<float>(n, ntr, P, Cf32, gk, rg, cpart, s)
                         : cosine_partial<double>(n, ntr, P, Cf, gk, rg, cpart, s);
    if (e == cudaSuccess)
        e = fp32 ? cosine_reduce<float>(n, ntr, P, cpart, nullptr, tmp, s) : cosine_reduce<double>(n, ntr, P, cpart, nullptr, tmp, s);
    if (e == cudaSuccess) e = modal_solve(g, fp32 && fac32, fac, fac32, tmp, kmax, s);
    if (e == cudaSuccess)
        e = fp32 ? cosine_partial<float>(n, ntr, P, Ci32, tmp, nullptr, cpart, s)
                 : cosine_partial<double>(n, ntr, P, Ci, tmp, nullptr, cpart, s);
    if (e == cudaSuccess)
        e = fp32 ? cosine_reduce<float>(n, ntr, P, cpart, gk, gnew, s) : cosine_reduce<double>(n, ntr, P, cpart, gk, gnew, s);
    return e;
}

}  // namespace ddnls
