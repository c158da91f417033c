// Internal device helpers shared by the dd_nls kernels: complex arithmetic on float2 /
// double2, the strip geometry, 1D Q1 coefficients, a bounded inter-block barrier and
// deterministic block reductions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dd_nls.h"
#include "dw.cuh"

namespace ddnls {

// ------------------------------------------------------------------ complex helpers
template <typename T> struct C2;
template <> struct C2<float> { using t = float2; };
template <> struct C2<double> { using t = double2; };

template <typename T2> __host__ __device__ __forceinline__ T2 mk(double re, double im) {
    T2 r; r.x = re; r.y = im; return r;
}
template <typename T2> __device__ __forceinline__ T2 cadd(T2 a, T2 b) { a.x += b.x; a.y += b.y; return a; }
template <typename T2> __device__ __forceinline__ T2 csub(T2 a, T2 b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename T2, typename T> __device__ __forceinline__ T2 cscale(T2 a, T s) { a.x *= s; a.y *= s; return a; }
template <typename T2> __device__ __forceinline__ T2 cmul(T2 a, T2 b) {
    T2 r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// a + s*b for complex s
template <typename T2> __device__ __forceinline__ T2 cfma(T2 s, T2 b, T2 a) {
    a.x = fma(s.x, b.x, fma(-s.y, b.y, a.x));
    a.y = fma(s.x, b.y, fma(s.y, b.x, a.y));
    return a;
}
__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp(double x) { return __drcp_rn(x); }
template <typename T2> __device__ __forceinline__ T2 cinv(T2 a) {
    const auto r = rcp(a.x * a.x + a.y * a.y);
    T2 o; o.x = a.x * r; o.y = -a.y * r; return o;
}
__device__ __forceinline__ double2 cd(float2 a) { return make_double2(a.x, a.y); }
__device__ __forceinline__ double2 cd(double2 a) { return a; }
template <typename T2> __device__ __forceinline__ T2 cfrom(double2 a);
template <> __device__ __forceinline__ float2 cfrom<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }
template <> __device__ __forceinline__ double2 cfrom<double2>(double2 a) { return a; }

// -------------------------------------------------------------------- geometry
// Strip field layout: strip j, column ix in [0, nxs), row iy in [0, nyn) at
// (j*nxs + ix)*P + iy: y is the fastest index, so an interface trace is contiguous.
struct Geom {
    int N;        // strips
    int nxs;      // nodes per strip in x (cells per strip + 1)
    int nyn;      // nodes in y
    int P;        // row pitch in elements (>= nyn, multiple of 32)
    double hx, hy;
    double alpha; // 2/(lap*dt), eq. (CNS) after division by lap
    double kap;   // kappa/lap
    double p;     // Robin parameter
    int bc_same;  // physical x-edges carry S-bar (1) or Neumann (0)
    int nx;       // cells in x over all strips
    double xl, yb;   // lower-left corner of Omega (node coordinates x = xl + ixg hx, y = yb + iy hy)
    // 1D P1 coefficients (filled on the host so kernels never divide):
    // mass off-diagonal h/6, diagonal 4h/6 inside and 2h/6 at the ends; stiffness
    // off-diagonal -1/h, diagonal 2/h inside and 1/h at the ends; trapezoid weight h.
    double mxo, mxi, mxe, kxo, kxi, kxe;
    double myo, myi, mye, kyo, kyi, kye;
    // FP32 copies for the FP32 kernels, rounded once here: a conversion from FP64 in a kernel
    // runs on the FP64 pipe (~1/64 of the FP32 rate on GB300), and the compiler may repeat
    // such conversions inside loops instead of keeping their results in registers
    float cf[12];            // mxo mxi mxe kxo kxi kxe myo myi mye kyo kyi kye
    float alpha_f, p_f;
    // the double-word residual's constants (hi, lo pairs) for Robin transmission: -hy/(6hx),
    // alpha hx hy/36, -hx/(6hy), p hy/6, hx hy kappa, hx hy
    float dwk[12];
    // after hx, hy, alpha, kap and p are set
    __host__ void fill_coefficients() {
        mxo = hx / 6.0; mxi = 4.0 * hx / 6.0; mxe = 2.0 * hx / 6.0;
        kxo = -1.0 / hx; kxi = 2.0 / hx; kxe = 1.0 / hx;
        myo = hy / 6.0; myi = 4.0 * hy / 6.0; mye = 2.0 * hy / 6.0;
        kyo = -1.0 / hy; kyi = 2.0 / hy; kye = 1.0 / hy;
        const double d[12] = {mxo, mxi, mxe, kxo, kxi, kxe, myo, myi, mye, kyo, kyi, kye};
        for (int i = 0; i < 12; ++i) cf[i] = (float)d[i];
        alpha_f = (float)alpha;
        p_f = (float)p;
        const double k[6] = {-hy / (6.0 * hx), alpha * hx * hy / 36.0, -hx / (6.0 * hy), p * hy / 6.0, hx * hy * kap, hx * hy};
        for (int i = 0; i < 6; ++i) {
            dwk[2 * i] = (float)k[i];
            dwk[2 * i + 1] = (float)(k[i] - (double)dwk[2 * i]);
        }
    }
    __host__ __device__ long long sstride() const { return (long long)nxs * P; }
    __host__ __device__ int c() const { return nxs - 1; }
};

// 1D P1 coefficients of a uniform mesh with nodes 0..n: mass (h/6)[1 4 1] with h/3 at the
// ends, stiffness (1/h)[-1 2 -1] with 1/h at the ends (Sec. 2.2, Q1 = P1 x P1).
template <typename T> struct Coef1 {
    T m[3];   // M(i, i-1), M(i, i), M(i, i+1) (zero outside the mesh)
    T k[3];
};
// The six constants of one direction, converted once to the working precision.
template <typename T> struct Coef1Consts {
    T mo, mi, me, ko, ki, ke;
};
template <typename T> __device__ __forceinline__ Coef1Consts<T> consts_x(const Geom& g);
template <typename T> __device__ __forceinline__ Coef1Consts<T> consts_y(const Geom& g);
template <> __device__ __forceinline__ Coef1Consts<double> consts_x<double>(const Geom& g) {
    return {g.mxo, g.mxi, g.mxe, g.kxo, g.kxi, g.kxe};
}
template <> __device__ __forceinline__ Coef1Consts<double> consts_y<double>(const Geom& g) {
    return {g.myo, g.myi, g.mye, g.kyo, g.kyi, g.kye};
}
template <> __device__ __forceinline__ Coef1Consts<float> consts_x<float>(const Geom& g) {
    return {g.cf[0], g.cf[1], g.cf[2], g.cf[3], g.cf[4], g.cf[5]};
}
template <> __device__ __forceinline__ Coef1Consts<float> consts_y<float>(const Geom& g) {
    return {g.cf[6], g.cf[7], g.cf[8], g.cf[9], g.cf[10], g.cf[11]};
}
// alpha = 2/(lap dt) and the Robin p in the working precision (no conversion in the kernel)
template <typename T> __device__ __forceinline__ T alpha_t(const Geom& g);
template <> __device__ __forceinline__ double alpha_t<double>(const Geom& g) { return g.alpha; }
template <> __device__ __forceinline__ float alpha_t<float>(const Geom& g) { return g.alpha_f; }
template <typename T> __device__ __forceinline__ T p_t(const Geom& g);
template <> __device__ __forceinline__ double p_t<double>(const Geom& g) { return g.p; }
template <> __device__ __forceinline__ float p_t<float>(const Geom& g) { return g.p_f; }
template <typename T> __device__ __forceinline__ Coef1<T> coef1(int i, int n, const Coef1Consts<T>& k) {
    Coef1<T> c;
    const bool lo = (i > 0), hi = (i < n);
    c.m[0] = lo ? k.mo : (T)0;
    c.m[2] = hi ? k.mo : (T)0;
    c.m[1] = (lo && hi) ? k.mi : k.me;
    c.k[0] = lo ? k.ko : (T)0;
    c.k[2] = hi ? k.ko : (T)0;
    c.k[1] = (lo && hi) ? k.ki : k.ke;
    return c;
}
// trapezoidal (nodal quadrature) weight of node i of a 1D mesh 0..n
__device__ __forceinline__ double wq(int i, int n, double h) { return (i == 0 || i == n) ? 0.5 * h : h; }

// Strip j's vertical edges: transmission operator (interfaces, and the physical edges when
// bc_same) and whether a datum (l or r) enters the right side (interfaces only).
__device__ __forceinline__ bool left_tc(const Geom& g, int j) { return j > 0 || g.bc_same; }
__device__ __forceinline__ bool right_tc(const Geom& g, int j) { return j < g.N - 1 || g.bc_same; }

// flat node index n -> (ix, iy) with a float reciprocal and an exact fix-up
__device__ __forceinline__ void split_node(int n, int nyn, float inv_nyn, int& ix, int& iy) {
    ix = __float2int_rz((float)n * inv_nyn);
    iy = n - ix * nyn;
    if (iy < 0) { ix -= 1; iy += nyn; }
    else if (iy >= nyn) { ix += 1; iy -= nyn; }
}

// Node t of the strip-field enumeration t = (j nxs + ix) nyn + iy -> (j, ix, iy), with 32-bit
// divisions while t fits (64-bit ones cost several times more instructions).
__device__ __forceinline__ void split_strip_node(long long t, int nxs, int nyn, int& j, int& ix, int& iy) {
    if (t < 0x7fffffffLL) {
        const unsigned u = (unsigned)t, col = u / (unsigned)nyn, jj = col / (unsigned)nxs;
        iy = (int)(u - col * (unsigned)nyn);
        j = (int)jj;
        ix = (int)(col - jj * (unsigned)nxs);
    } else {
        const long long col = t / nyn;
        iy = (int)(t - col * nyn);
        j = (int)(col / nxs);
        ix = (int)(col - (long long)j * nxs);
    }
}

// ------------------------------------------------------------------- reductions
// Sum NV doubles over the block in a fixed order; the result is valid in thread 0.
template <int NV> __device__ __forceinline__ void block_sum(double (&v)[NV], double* smem) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) smem[wid * NV + k] = v[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = lane < nw ? smem[lane * NV + k] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            v[k] = s;
        }
    }
    __syncthreads();
}

// Block sum of NV values held in precision T: warp shuffles in T, the per-warp results are
// summed in double by warp 0 (fixed order); valid in thread 0.  Keeps FP64 instructions out of
// the per-thread path of FP32 kernels.
template <typename T, int NV> __device__ __forceinline__ void block_sum_t(T (&v)[NV], double (&out)[NV], double* smem) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) smem[wid * NV + k] = (double)v[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = lane < nw ? smem[lane * NV + k] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            out[k] = s;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Barrier among the nblk co-resident blocks that share *ctr.  The counter only grows:
// the k-th barrier of a launch waits for k*nblk arrivals.  The wait is bounded by limit_ns of
// wall time (globaltimer); on time-out it records DD_NLS_ETIMEOUT in *err and returns false,
// and every caller leaves its loop.  A block also stops waiting as soon as another block has
// recorded the time-out.  arrive = false (a test of the time-out path only) waits without
// adding this block's arrival.
__device__ __forceinline__ bool group_barrier(unsigned* ctr, unsigned target, int* err, int* s_flag,
                                              unsigned long long limit_ns, bool arrive = true) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (arrive) atomicAdd(ctr, 1u);
        int ok = 1;
        if (ld_acquire(ctr) < target) {
            const unsigned long long t0 = globaltimer();
            unsigned spins = 0;
            while (ld_acquire(ctr) < target) {
                __nanosleep(64);
                if ((++spins & 255u) == 0) {
                    if (*(volatile int*)err == DD_NLS_ETIMEOUT) { ok = 0; break; }
                    if (globaltimer() - t0 > limit_ns) {
                        atomicExch(err, DD_NLS_ETIMEOUT);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        if (ok && *(volatile int*)err == DD_NLS_ETIMEOUT) ok = 0;
        __threadfence();
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

// ---------------------------------------------------------- thread-block clusters
// A strip solved by one cluster: its CTAs exchange partial sums and halo rows through
// distributed shared memory (DSMEM) instead of global memory.
constexpr int kClusterCTAs = 16;   // CTAs per cluster (non-portable size, opted in at launch)

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
// the shared::cluster address of the same variable in CTA `rank` of the cluster
__device__ __forceinline__ unsigned mapa(unsigned a, unsigned rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_cluster(unsigned a, double v) {
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}
__device__ __forceinline__ void st_release_cluster(unsigned a, unsigned v) {
    asm volatile("st.release.cluster.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_cluster(unsigned a) {
    unsigned v;
    asm volatile("ld.acquire.cluster.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ float2 ld_cluster_f2(unsigned a) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void fence_cluster() { asm volatile("fence.acq_rel.cluster;" ::: "memory"); }
// all threads of all CTAs of the cluster (hardware barrier; every CTA must reach it)
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Exchange slots of one CTA: the partial sums every CTA of the cluster pushes, by epoch parity.
struct ClusterSlots {
    double v[2][kClusterCTAs][6];
    unsigned flag[2][kClusterCTAs];
};

// Strip-wide sum over the cluster's CTAs of NV values held by thread 0 (v): lanes q < ncta of
// warp 0 push the values into slot [parity][this rank] of CTA q and then release the epoch flag;
// each CTA waits (bounded by limit_ns) until all ncta flags of the epoch have arrived and sums
// the slots over a lane tree of fixed shape, so every CTA gets the same sums.  The push follows a fence at cluster
// scope, so everything this CTA wrote before the call (shared or global memory) is visible to
// the other CTAs once they return.  Results in out[] of every thread (after a __syncthreads).
// Returns false on time-out (DD_NLS_ETIMEOUT recorded in *err).  push = false (a test hook)
// leaves this CTA's values and flags out, so that every CTA's wait runs out.
template <int NV>
__device__ __forceinline__ bool cluster_allreduce(ClusterSlots& sl, const double (&v)[NV], double (&out)[NV],
                                                  unsigned epoch, int ncta, int* err, unsigned long long limit_ns,
                                                  double* s_out, int* s_flag, bool push = true) {
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const unsigned me = cluster_rank(), par = epoch & 1u;
        double val[NV > 0 ? NV : 1];
#pragma unroll
        for (int k = 0; k < NV; ++k) val[k] = __shfl_sync(0xffffffffu, v[k], 0);
        if (lane < ncta && push) {
            fence_cluster();
            const unsigned dst = mapa(smem_addr(&sl.v[par][me][0]), (unsigned)lane);
#pragma unroll
            for (int k = 0; k < NV; ++k) st_cluster(dst + 8u * k, val[k]);
            st_release_cluster(mapa(smem_addr(&sl.flag[par][me]), (unsigned)lane), epoch);
        }
        int ok = 1;
        if (lane < ncta) {
            const unsigned fa = mapa(smem_addr(&sl.flag[par][lane]), me);
            if (ld_acquire_cluster(fa) != epoch) {
                const unsigned long long t0 = globaltimer();
                unsigned spins = 0;
                while (ld_acquire_cluster(fa) != epoch) {
                    if ((++spins & 63u) == 0) {
                        if (*(volatile int*)err == DD_NLS_ETIMEOUT) { ok = 0; break; }
                        if (globaltimer() - t0 > limit_ns) {
                            atomicExch(err, DD_NLS_ETIMEOUT);
                            ok = 0;
                            break;
                        }
                    }
                }
            }
        }
        ok = __all_sync(0xffffffffu, ok);
        // lane q holds CTA q's values (read after its own acquire of flag q); a tree of fixed
        // shape over the lanes gives every CTA the same sums
        double acc[NV > 0 ? NV : 1];
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] = (ok && lane < ncta) ? sl.v[par][lane][k] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < NV; ++k) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < NV; ++k) s_out[k] = acc[k];
            *s_flag = ok;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = s_out[k];
    const bool ok = *s_flag != 0;
    __syncthreads();
    return ok;
}

// The same exchange for double-word values (pairs of FP32 numbers, ~48 bits): the sums over the
// cluster are formed with the accurate double-word addition over a fixed lane tree, so every CTA gets the
// same result without any FP64 instruction (GB300 runs FP64 at ~1/64 of the FP32 rate, and these
// exchanges sit on the critical path of every Krylov iteration).  v valid in thread 0; out in
// every thread.
struct __align__(16) ClusterSlotsDW {
    float v[2][kClusterCTAs][12];
    unsigned flag[2][kClusterCTAs];
};
template <int NV>
__device__ __forceinline__ bool cluster_allreduce_dw(ClusterSlotsDW& sl, const dw (&v)[NV], dw (&out)[NV],
                                                     unsigned epoch, int ncta, int* err, unsigned long long limit_ns,
                                                     float* s_out, int* s_flag) {
    static_assert(NV <= 6, "six double words per slot");
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const unsigned me = cluster_rank(), par = epoch & 1u;
        float vh[NV], vl[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            vh[k] = __shfl_sync(0xffffffffu, v[k].h, 0);
            vl[k] = __shfl_sync(0xffffffffu, v[k].l, 0);
        }
        if (lane < ncta) {
            fence_cluster();
            const unsigned dst = mapa(smem_addr(&sl.v[par][me][0]), (unsigned)lane);
#pragma unroll
            for (int k = 0; k < NV; ++k)
                asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(dst + 8u * k), "f"(vh[k]), "f"(vl[k]) : "memory");
            st_release_cluster(mapa(smem_addr(&sl.flag[par][me]), (unsigned)lane), epoch);
        }
        int ok = 1;
        if (lane < ncta) {
            const unsigned fa = mapa(smem_addr(&sl.flag[par][lane]), me);
            if (ld_acquire_cluster(fa) != epoch) {
                const unsigned long long t0 = globaltimer();
                unsigned spins = 0;
                while (ld_acquire_cluster(fa) != epoch) {
                    if ((++spins & 63u) == 0) {
                        if (*(volatile int*)err == DD_NLS_ETIMEOUT) { ok = 0; break; }
                        if (globaltimer() - t0 > limit_ns) {
                            atomicExch(err, DD_NLS_ETIMEOUT);
                            ok = 0;
                            break;
                        }
                    }
                }
            }
        }
        ok = __all_sync(0xffffffffu, ok);
        // lane q holds CTA q's values (read after its own acquire of flag q); a tree of fixed
        // shape over the lanes, in double words, gives every CTA the same sums
        dw acc[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k)
            acc[k] = (ok && lane < ncta) ? dw{sl.v[par][lane][2 * k], sl.v[par][lane][2 * k + 1]} : dw{0.f, 0.f};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                const dw t = {__shfl_down_sync(0xffffffffu, acc[k].h, o), __shfl_down_sync(0xffffffffu, acc[k].l, o)};
                acc[k] = dw_add(acc[k], t);
            }
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < NV; ++k) { s_out[2 * k] = acc[k].h; s_out[2 * k + 1] = acc[k].l; }
            *s_flag = ok;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = {s_out[2 * k], s_out[2 * k + 1]};
    const bool ok = *s_flag != 0;
    __syncthreads();
    return ok;
}

// Block sum of NV FP32 values: warp shuffles in FP32, then the warps' partials added in
// double words by warp 0 (fixed order); valid in thread 0.  smem: 16 * NV floats at least.
template <int NV>
__device__ __forceinline__ void block_sum_dw(float (&v)[NV], dw (&out)[NV], float* smem) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) smem[wid * NV + k] = v[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            dw s = {lane < nw ? smem[lane * NV + k] : 0.f, 0.f};
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const dw t = {__shfl_down_sync(0xffffffffu, s.h, o), __shfl_down_sync(0xffffffffu, s.l, o)};
                s = dw_add(s, t);
            }
            out[k] = s;
        }
    }
    __syncthreads();
}

// Sum slot values written by the nblk blocks of a group (fixed order); result broadcast.
// The same sums (same order, same result) formed by warp 0 alone, every lane of which gets
// them; the caller derives its scalars on one thread and broadcasts what the block needs.
template <int NV> __device__ __forceinline__ void group_sum_w0(const double* part, int nblk, double (&out)[NV]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = 0.0;
    for (int b0 = 0; b0 < nblk; b0 += 32) {
        const int b = b0 + lane;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = b < nblk ? __ldcg(part + (size_t)b * 4 + k) : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            out[k] += s;
        }
    }
}

template <int NV> __device__ __forceinline__ void group_sum(const double* part, int nblk, double (&out)[NV], double* smem) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        double acc[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] = 0.0;
        for (int b0 = 0; b0 < nblk; b0 += 32) {
            const int b = b0 + lane;
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                double s = b < nblk ? __ldcg(part + (size_t)b * 4 + k) : 0.0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                acc[k] += s;
            }
        }
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < NV; ++k) smem[k] = acc[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = smem[k];
    __syncthreads();
}

}  // namespace ddnls
