// Batched strip solver: every strip problem of one Schwarz iteration in one persistent
// (cooperative) launch.
//
// Each strip j solves the nonlinear local problem of eq. (localpbrobin) in the matrix form
// of eq. (NproblemRobinNL):
//     (A + i p M^Gamma + M_f(zeta)) zeta = (2i/dt) M h - M^Gamma Q^T (l; r),
//     A = (2i/dt) M - S + M_W,   M_f(zeta) = diag(w kappa |zeta|^2)   (nodal quadrature),
// by the fixed point of eq. (localpbrobin) written in defect-correction form: with
// c = w (W + kappa |zeta|^2) frozen at the current iterate,
//     res = b - A(c) zeta   (FP64, matrix-free 9-point Q1 stencil),
//     A(c) delta = res      (Jacobi-preconditioned COCG in precision T),
//     zeta += delta,
// until ||res|| <= max(nl_tol ||b||, floor) (floor: 1% of nl_tol times the whole step's right
// side per strip, so strips that hold almost nothing of the solution stop early).  The inner system is solved
// for res / s with s the previous residual norm, so FP32 never sees values below its range
// (far-field strips can hold values near 1e-111).  With an exact inner solve one correction is
// exactly one
// step zeta^q = A(c(zeta^{q-1}))^{-1} b of eq. (localpbrobin); the limit is the same fixed
// point.  A(c) is complex symmetric, so COCG (CG with the unconjugated bilinear form)
// applies.
//
// Work split: blocks [j*bps, (j+1)*bps) own strip j; they meet only at per-strip barriers
// (bounded spin, status word on time-out), so strips converge independently.  Every block
// derives the same scalars from the same fixed-order reductions, so all blocks of a strip
// take the same branches.
#include "common.cuh"
#include "dw.cuh"
#include "kernels.h"

#include <algorithm>
#include <atomic>
#include <type_traits>

namespace ddnls {

static std::atomic<long long> g_launches{0};
long long kernel_launch_count() { return g_launches.load(); }
void count_launches(int n) { g_launches += n; }

// y = A(c) v at one node: the 9-point Q1 stencil of Bx (x) My - Mx (x) Ky + diag(c), with
// Bx = -Kx + i alpha Mx + rho E_x, E_x the transmission edges of the strip and rho the edge
// coefficient: i p for Robin (eq. NproblemRobinNL), i sum a_s for S_pade (eq. NproblemSPNL).
template <typename T, typename T2>
__device__ __forceinline__ T2 apply_op(const T2* v, long long idx, int ix, int iy,
                                       int c, int ny, int P, const Coef1<T>& cx, const Coef1<T>& cy,
                                       T alpha, T rho_re, T rho_im, T cdiag) {
    T2 acc = mk<T2>(0.0, 0.0);
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
        if (ix + dx < 0 || ix + dx > c) continue;
        const T2* col = v + idx + (long long)dx * P;
        const T2 a0 = col[0];
        const T2 am = iy > 0 ? col[-1] : mk<T2>(0.0, 0.0);
        const T2 ap = iy < ny ? col[1] : mk<T2>(0.0, 0.0);
        T2 tM, tK;
        tM.x = cy.m[0] * am.x + cy.m[1] * a0.x + cy.m[2] * ap.x;
        tM.y = cy.m[0] * am.y + cy.m[1] * a0.y + cy.m[2] * ap.y;
        tK.x = cy.k[0] * am.x + cy.k[1] * a0.x + cy.k[2] * ap.x;
        tK.y = cy.k[0] * am.y + cy.k[1] * a0.y + cy.k[2] * ap.y;
        const T mx = cx.m[dx + 1];
        const T bre = -cx.k[dx + 1] + (dx == 0 ? rho_re : (T)0);
        const T bim = alpha * mx + (dx == 0 ? rho_im : (T)0);
        acc.x += bre * tM.x - bim * tM.y - mx * tK.x;
        acc.y += bre * tM.y + bim * tM.x - mx * tK.y;
    }
    const T2 vc = v[idx];
    acc.x += cdiag * vc.x;
    acc.y += cdiag * vc.y;
    return acc;
}

// The 9-point stencil of A(c) at a node off the strip's edges and off the y-boundary (uniform
// mesh): four complex weights, W(dx, dy) = Bx(dx) My(dy) - Mx(dx) Ky(dy) with Bx = -Kx + i alpha Mx,
// for the corners (ac), the x-neighbours (bx), the y-neighbours (ay) and the centre (bc, plus c).
// The same operator as apply_op there, in about a third of its arithmetic.
template <typename T2> struct Interior9 {
    T2 ac, bx, ay, bc;
};
template <typename T, typename T2>
__device__ __forceinline__ Interior9<T2> interior9(const Coef1Consts<T>& kx, const Coef1Consts<T>& ky, T alpha) {
    Interior9<T2> w;
    w.ac.x = -kx.ko * ky.mo - kx.mo * ky.ko;
    w.ac.y = alpha * kx.mo * ky.mo;
    w.bx.x = -kx.ko * ky.mi - kx.mo * ky.ki;
    w.bx.y = alpha * kx.mo * ky.mi;
    w.ay.x = -kx.ki * ky.mo - kx.mi * ky.ko;
    w.ay.y = alpha * kx.mi * ky.mo;
    w.bc.x = -kx.ki * ky.mi - kx.mi * ky.ki;
    w.bc.y = alpha * kx.mi * ky.mi;
    return w;
}
template <typename T, typename T2>
__device__ __forceinline__ T2 apply_interior(const T2* v, int idx, int P, const Interior9<T2>& w, T cdiag) {
    const T2* l = v + idx - P;
    const T2* m = v + idx;
    const T2* r = v + idx + P;
    const T2 c0 = m[0];
    T2 sc, sx, sy;
    sc.x = (l[-1].x + l[1].x) + (r[-1].x + r[1].x);
    sc.y = (l[-1].y + l[1].y) + (r[-1].y + r[1].y);
    sx.x = l[0].x + r[0].x;
    sx.y = l[0].y + r[0].y;
    sy.x = m[-1].x + m[1].x;
    sy.y = m[-1].y + m[1].y;
    const T bcx = w.bc.x + cdiag;
    T2 acc;
    acc.x = w.ac.x * sc.x - w.ac.y * sc.y + w.bx.x * sx.x - w.bx.y * sx.y + w.ay.x * sy.x - w.ay.y * sy.y +
            bcx * c0.x - w.bc.y * c0.y;
    acc.y = w.ac.x * sc.y + w.ac.y * sc.x + w.bx.x * sx.y + w.bx.y * sx.x + w.ay.x * sy.y + w.ay.y * sy.x +
            bcx * c0.y + w.bc.y * c0.x;
    return acc;
}

// z_{k+1} = D^{-1}(r_k - alpha (w_k + beta s_{k-1})) at node k (single-reduction COCG)
template <typename T2>
__device__ __forceinline__ T2 znext(const T2* rr, const T2* ww, const T2* ss, const T2* dvv, long long k, T2 al, T2 be) {
    const T2 sv = cfma(be, ss[k], ww[k]);
    T2 t = rr[k];
    t.x -= al.x * sv.x - al.y * sv.y;
    t.y -= al.x * sv.y + al.y * sv.x;
    return cmul(dvv[k], t);
}
// r_{k+1} = r_k - alpha (w_k + beta s_{k-1}) and s_k = w_k + beta s_{k-1}, from values (the same
// arithmetic as znext, so a neighbour's rebuilt z_{k+1} = D^-1 r_{k+1} matches the owner's)
template <typename T2>
__device__ __forceinline__ T2 rnext_v(T2 r, T2 w, T2 s, T2 al, T2 be, T2& sv) {
    sv = cfma(be, s, w);
    r.x -= al.x * sv.x - al.y * sv.y;
    r.y -= al.x * sv.y + al.y * sv.x;
    return r;
}

// w = A(c) z with z formed on the fly at the 9 stencil nodes (same arithmetic as apply_op)
template <typename T, typename T2>
__device__ __forceinline__ T2 apply_op_znext(const T2* rr, const T2* ww, const T2* ss, const T2* dvv, long long idx,
                                             int ix, int iy, int c, int ny, int P, const Coef1<T>& cx,
                                             const Coef1<T>& cy, T alpha, T rho_re, T rho_im, T cdiag, T2 al, T2 be,
                                             T2& zown) {
    T2 acc = mk<T2>(0.0, 0.0);
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
        if (ix + dx < 0 || ix + dx > c) continue;
        const long long k0 = idx + (long long)dx * P;
        const T2 a0 = znext(rr, ww, ss, dvv, k0, al, be);
        if (dx == 0) zown = a0;
        const T2 am = iy > 0 ? znext(rr, ww, ss, dvv, k0 - 1, al, be) : mk<T2>(0.0, 0.0);
        const T2 ap = iy < ny ? znext(rr, ww, ss, dvv, k0 + 1, al, be) : mk<T2>(0.0, 0.0);
        T2 tM, tK;
        tM.x = cy.m[0] * am.x + cy.m[1] * a0.x + cy.m[2] * ap.x;
        tM.y = cy.m[0] * am.y + cy.m[1] * a0.y + cy.m[2] * ap.y;
        tK.x = cy.k[0] * am.x + cy.k[1] * a0.x + cy.k[2] * ap.x;
        tK.y = cy.k[0] * am.y + cy.k[1] * a0.y + cy.k[2] * ap.y;
        const T mx = cx.m[dx + 1];
        const T bre = -cx.k[dx + 1] + (dx == 0 ? rho_re : (T)0);
        const T bim = alpha * mx + (dx == 0 ? rho_im : (T)0);
        acc.x += bre * tM.x - bim * tM.y - mx * tK.x;
        acc.y += bre * tM.y + bim * tM.x - mx * tK.y;
    }
    acc.x += cdiag * zown.x;
    acc.y += cdiag * zown.y;
    return acc;
}

template <typename T>
__device__ __forceinline__ typename C2<T>::t diag_inv(const Coef1<T>& cx, const Coef1<T>& cy, T alpha, T rho_re,
                                                      T rho_im, T cdiag) {
    using T2 = typename C2<T>::t;
    T2 d;
    d.x = (-cx.k[1] + rho_re) * cy.m[1] - cx.m[1] * cy.k[1] + cdiag;
    d.y = (alpha * cx.m[1] + rho_im) * cy.m[1];
    return cinv(d);
}

// (M^Gamma v)(iy) along an edge column (consistent 1D mass in y)
template <typename T, typename T2>
__device__ __forceinline__ T2 edge_mass(const T2* v, int iy, int ny, const Coef1<T>& cy) {
    const T2 a0 = v[iy];
    const T2 am = iy > 0 ? v[iy - 1] : mk<T2>(0.0, 0.0);
    const T2 ap = iy < ny ? v[iy + 1] : mk<T2>(0.0, 0.0);
    T2 t;
    t.x = cy.m[0] * am.x + cy.m[1] * a0.x + cy.m[2] * ap.x;
    t.y = cy.m[0] * am.y + cy.m[1] * a0.y + cy.m[2] * ap.y;
    return t;
}

// The auxiliary row of phi_s on one edge, eq. (NproblemSPNL) rows (C, D_s), scaled by
// sigma_s = i a_s d_s so that the coupled system is complex symmetric (sigma_s C = B_s^T):
//   sigma_s [ -(M^G zeta_e) + ((i alpha + d_s) M^G - S^G + diag(c_phi)) phi_s ]
template <typename T, typename T2>
__device__ __forceinline__ T2 phi_row_v(T2 zm, T2 z0, T2 zp, const T2* ph, int iy, int ny, const Coef1<T>& cy,
                                        T2 gam, T2 sig, T cphi) {
    T2 mz;
    mz.x = cy.m[0] * zm.x + cy.m[1] * z0.x + cy.m[2] * zp.x;
    mz.y = cy.m[0] * zm.y + cy.m[1] * z0.y + cy.m[2] * zp.y;
    const T2 a0 = ph[iy];
    const T2 am = iy > 0 ? ph[iy - 1] : mk<T2>(0.0, 0.0);
    const T2 ap = iy < ny ? ph[iy + 1] : mk<T2>(0.0, 0.0);
    T2 tM, tK;
    tM.x = cy.m[0] * am.x + cy.m[1] * a0.x + cy.m[2] * ap.x;
    tM.y = cy.m[0] * am.y + cy.m[1] * a0.y + cy.m[2] * ap.y;
    tK.x = cy.k[0] * am.x + cy.k[1] * a0.x + cy.k[2] * ap.x;
    tK.y = cy.k[0] * am.y + cy.k[1] * a0.y + cy.k[2] * ap.y;
    T2 j = cmul(gam, tM);
    j.x += -tK.x + cphi * a0.x - mz.x;
    j.y += -tK.y + cphi * a0.y - mz.y;
    return cmul(sig, j);
}
// the same row with the edge column of zeta read from memory (ze: the column, rows 0..ny)
template <typename T, typename T2>
__device__ __forceinline__ T2 phi_row(const T2* ze, const T2* ph, int iy, int ny, const Coef1<T>& cy, T2 gam,
                                      T2 sig, T cphi) {
    const T2 zm = iy > 0 ? ze[iy - 1] : mk<T2>(0.0, 0.0);
    const T2 zp = iy < ny ? ze[iy + 1] : mk<T2>(0.0, 0.0);
    return phi_row_v<T, T2>(zm, ze[iy], zp, ph, iy, ny, cy, gam, sig, cphi);
}
template <typename T, typename T2>
__device__ __forceinline__ T2 phi_diag_inv(const Coef1<T>& cy, T2 gam, T2 sig, T cphi) {
    T2 d = cmul(gam, mk<T2>(cy.m[1], 0.0));
    d.x += -cy.k[1] + cphi;
    return cinv(cmul(sig, d));
}

// Nodes per thread of the on-chip Krylov state in cluster mode (x and r in registers).
constexpr int kOnChipNPT = 9;

// CLU: one strip per thread-block cluster of kClusterCTAs CTAs (launched with cluster dimensions,
// no cooperative launch).  The CTAs of a strip exchange partial sums through distributed shared
// memory instead of global-memory barriers, and the single-reduction COCG keeps the strip's
// Krylov state on chip: each CTA owns a slab of rows [y0, y1) across the strip's whole width,
// with x and r in registers, z (with one halo row on each side), w, p, s, D^-1 and c in shared
// memory; the halo rows of z_{k+1} are rebuilt from the neighbours' exported rows of r_k, w_k and
// s_{k-1}, read through DSMEM, and their D^-1 (fixed during a solve, read once), so one cluster
// exchange per iteration suffices.
template <typename T, bool PADE, int BS, bool DW = false, bool CLU = false>
__global__ void __launch_bounds__(BS, CLU ? 1 : 512 / BS)
strip_solve_kernel(StripSolveArgs a) {
    using T2 = typename C2<T>::t;
    __shared__ double s_red[64];
    __shared__ int s_flag;
    __shared__ typename std::conditional<CLU, ClusterSlots, char>::type s_cl;
    __shared__ typename std::conditional<CLU, ClusterSlotsDW, char>::type s_cld;
    __shared__ double s_out[8];
    extern __shared__ __align__(16) unsigned char s_dyn[];
    static_assert(!CLU || (sizeof(T) == 4 && !PADE), "cluster mode is built for the FP32 Robin solver");
    // Krylov scalars: the FP64 recurrences run on thread 0 only (FP64 issues at ~1/64 of the
    // FP32 rate here; eight warps repeating them cost more than the vector work) and reach the
    // block through shared memory: s_ctl = {0 go on | 1 stop, x accepted | 2 error, status},
    // s_sc = alpha, beta in the inner precision
    __shared__ int s_ctl[2];
    __shared__ T s_sc[4];
    __shared__ float s_kr[24];    // thread 0's state of the on-chip recurrences (cluster mode)
    __shared__ int s_kri;

    // strip of the launch (virtual strip in setup mode); cluster mode: cluster c solves strip
    // blk_strip[c] and its CTAs are the strip's blocks
    const int j = CLU ? a.blk_strip[blockIdx.x / kClusterCTAs] : a.blk_strip[blockIdx.x];
    const int b0 = CLU ? 0 : a.blk_start[j];
    const int bps = CLU ? kClusterCTAs : a.blk_start[j + 1] - b0; // blocks of this strip (weighted by the host)
    const int rank = CLU ? (int)cluster_rank() : (int)blockIdx.x - b0;
    if constexpr (CLU) {
        // exchange slots start empty; no CTA pushes before every CTA has cleared its own
        for (int t = threadIdx.x; t < 2 * kClusterCTAs; t += blockDim.x) {
            (&s_cl.flag[0][0])[t] = 0u;
            (&s_cld.flag[0][0])[t] = 0u;
        }
        cluster_sync_all();
    }
    // geometry: the launch's, or the instance's when instances are batched
    // batched instances (per-instance geometry) take the cooperative Robin kernels only; the
    // others read the geometry from the kernel parameters
    constexpr bool kBatchable = !CLU && !PADE;
    const StripInfo si = (kBatchable && a.sinfo) ? a.sinfo[j] : StripInfo{0, j, (long long)j * a.g.sstride(), 0};
    const Geom g = (kBatchable && a.geoms) ? a.geoms[si.inst] : a.g;
    const int jl = si.jloc;                  // strip index inside its instance
    const int nyn = g.nyn, ny = nyn - 1, c = g.nxs - 1, P = g.P;
    const int Ns = g.nxs * nyn;
    const int m = PADE ? a.pade_m : 0;
    const int Nall = Ns + 2 * m * nyn;       // strip nodes, then phi_{e,s} nodes
    const float inv_nyn = 1.0f / (float)nyn;
    // residual phase work items: runs of RX x-nodes per row, then the phi nodes
    constexpr int RX = 4;
    const int NR = ((g.nxs + RX - 1) / RX) * nyn;
    const int NRall = NR + 2 * m * nyn;
    // The nodes (or work items) of this block.  Robin strips: the strip's total split evenly over
    // its blocks in contiguous ranges (loads stay coalesced; whole blockDim-node chunks dealt
    // round robin left up to 40% more work on some blocks).  S_pade strips: chunks dealt round
    // robin, which mixes the costlier edge nodes and the phi rows (stored after the nodes) over
    // all blocks; contiguous ranges put all of them on a few blocks.
    auto it_first = [&](int total) {
        return PADE ? rank * (int)blockDim.x + (int)threadIdx.x : (int)(((long long)total * rank) / bps) + (int)threadIdx.x;
    };
    auto it_end = [&](int total) { return PADE ? total : (int)(((long long)total * (rank + 1)) / bps); };
    const int it_step = PADE ? bps * (int)blockDim.x : (int)blockDim.x;
    const long long sbase = si.off;

    // edges of this strip
    bool ltc, rtc, ldata, rdata;
    int unit_side = -1, unit_pos = -1;
    if (a.mode == 0) {
        ltc = left_tc(g, jl);
        rtc = right_tc(g, jl);
        ldata = jl > 0;
        rdata = jl < g.N - 1;
    } else {      // L_h construction: unit datum on one edge of a free strip
        ltc = a.unit_ltc;
        rtc = a.unit_rtc;
        ldata = rdata = false;
        const int u = a.unit_base + j;
        unit_side = u / nyn;
        unit_pos = u - unit_side * nyn;
    }
    const double2* gl = ldata ? a.gtr + si.goff + (size_t)(2 * (jl - 1) + 1) * P : nullptr;
    const double2* gr = rdata ? a.gtr + si.goff + (size_t)(2 * jl) * P : nullptr;

    double2* zeta = a.zeta + sbase;
    const double2* __restrict__ rhs0 = a.rhs0 ? a.rhs0 + sbase : nullptr;
    const double* __restrict__ Wn = a.Wn ? a.Wn + sbase : nullptr;
    T2* x = (T2*)a.x + sbase;
    T2* r = (T2*)a.r + sbase;
    T2* z = (T2*)a.z + sbase;
    T2* p = (T2*)a.p + sbase;
    T2* q = (T2*)a.q + sbase;
    T* cT = (T*)a.cT + sbase;
    // single-reduction COCG (Robin, FP32 inner solve): r and w ping-pong (r|z, q|w1), s
    // ping-pong, D^-1.  In FP64 the 9-point rebuild of z costs more FP64-pipe time than the
    // second barrier saves, so the FP64 instance keeps the two-reduction loop.
    // Below a few hundred unknowns COCG exhausts the Krylov space before FP32 reaches the
    // target, and the single-reduction recurrence for alpha (delta - beta gamma/alpha) then
    // loses accuracy (FP32 model runs: a few failures in 10^4 random right sides on 4-node
    // strips, none on 12..544-node strips); such strips take the two-reduction loop.
    constexpr bool SR = !PADE && sizeof(T) == 4;
    constexpr int kSRMinNodes = 256;
    // A strip whose single-reduction solve stalls (32 steps without a 1% gain) or breaks down
    // takes the two-reduction loop for the rest of the launch (seen in FP32 on a GPE trap strip
    // after ~100 steps, where the recurrence for alpha had lost its accuracy).
    bool use_sr = SR && Ns >= kSRMinNodes;
    T2* rbuf[2] = {r, z};
    T2* wbuf[2] = {q, SR ? (T2*)a.w1 + sbase : nullptr};
    T2* sbuf[2] = {SR ? (T2*)a.s0 + sbase : nullptr, SR ? (T2*)a.s1 + sbase : nullptr};
    T2* dv = SR ? (T2*)a.dv + sbase : nullptr;
    // double-word residual: the nonlinear residual on the FP32 pipe in ~48-bit arithmetic
    // instead of FP64 (GB300's FP64 rate is ~1/64 of FP32); zeta itself stays FP64 and
    // receives the accumulated correction once, at the end of the launch
    static_assert(!DW || sizeof(T) == 4, "the double-word residual is built for the FP32 inner solvers");
    float4* zdw = DW ? a.zdw + sbase : nullptr;
    float4* ddw = (DW && a.ddw) ? a.ddw + sbase : nullptr;   // dw_mode 0 only
    float4* bdw = DW ? a.bdw + sbase : nullptr;
    const float2* wdw = DW ? a.wdw + sbase : nullptr;
    // auxiliary unknowns: phi_{e,s}(iy) at ((j*2 + e)*m + s)*P + iy
    const long long fbase = (long long)j * 2 * m * P;
    double2* phi = PADE ? a.phi + fbase : nullptr;
    T2* xf = PADE ? (T2*)a.xf + fbase : nullptr;
    T2* rf = PADE ? (T2*)a.rf + fbase : nullptr;
    T2* zf = PADE ? (T2*)a.zf + fbase : nullptr;
    T2* pf = PADE ? (T2*)a.pf + fbase : nullptr;
    T2* qf = PADE ? (T2*)a.qf + fbase : nullptr;
    T* cTf = PADE ? (T*)a.cTf + (long long)j * 2 * P : nullptr;

    unsigned* bar = a.bar + j;
    unsigned epoch = 0;
    // bounded waits (a.wait_ns, 0: two seconds); the test hook makes block test_skip_arrival - 1
    // skip its arrival at its first barrier, so that the wait runs out
    const unsigned long long wait_ns = a.wait_ns ? a.wait_ns : 2000000000ull;
    bool skip_arrival = a.test_skip_arrival == (int)blockIdx.x + 1;
    auto gbar = [&](unsigned target) {
        const bool ok = group_barrier(bar, target, a.err, &s_flag, wait_ns, !skip_arrival);
        skip_arrival = false;
        return ok;
    };
    const int NB = gridDim.x;
    double* part_base = a.part;
    auto slot_ptr = [&](unsigned e) { return part_base + ((size_t)(e & 3u) * NB + blockIdx.x) * 4; };
    auto group_ptr = [&](unsigned e) { return part_base + ((size_t)(e & 3u) * NB + (size_t)b0) * 4; };
    unsigned cepoch = 0;     // cluster exchange epoch
    // strip-wide sum of 4 values held by thread 0 (block sums), broadcast to every thread; also
    // a barrier of the strip's blocks
    auto strip_sum4 = [&](const double (&v)[4], double (&out)[4]) -> bool {
        if constexpr (CLU) {
            const bool ok = cluster_allreduce<4>(s_cl, v, out, ++cepoch, bps, a.err, wait_ns, s_out, &s_flag, !skip_arrival);
            skip_arrival = false;
            return ok;
        } else {
            if (threadIdx.x == 0) {
                double* sp = slot_ptr(epoch + 1);
                sp[0] = v[0]; sp[1] = v[1]; sp[2] = v[2]; sp[3] = v[3];
            }
            ++epoch;
            if (!gbar(epoch * bps)) return false;
            group_sum<4>(group_ptr(epoch), bps, out, s_red);
            return true;
        }
    };
    auto strip_barrier = [&]() -> bool {
        if constexpr (CLU) {
            const double z1[1] = {0.0};
            double o1[1];
            const bool ok = cluster_allreduce<1>(s_cl, z1, o1, ++cepoch, bps, a.err, wait_ns, s_out, &s_flag, !skip_arrival);
            skip_arrival = false;
            return ok;
        } else {
            ++epoch;
            return gbar(epoch * bps);
        }
    };

    // edge coefficient rho: i p (Robin) or i sum_s a_s (S_pade)
    double rho_re = 0.0, rho_im = g.p;
    if (PADE) {
        double sre = 0.0, sim = 0.0;
        for (int s2 = 0; s2 < m; ++s2) { sre += a.pade_a[s2].x; sim += a.pade_a[s2].y; }
        rho_re = -sim;
        rho_im = sre;
    }
    const Coef1Consts<double> KXd = consts_x<double>(g), KYd = consts_y<double>(g);
    const Coef1Consts<T> KXt = consts_x<T>(g), KYt = consts_y<T>(g);
    const T alphaT = alpha_t<T>(g);
    const double kap = a.mode == 0 ? g.kap : 0.0;
    // correction operator: the complex-linear part of the Jacobian of kappa|z|^2 z (2 kappa|z|^2),
    // or the frozen operator of the fixed point (kappa|z|^2)
    const double cfac = a.nl_picard ? 1.0 : 2.0;

    int status = 0, nl_it = 0;
    long long kry = 0;
    // thread 0's scalars of the nonlinear control live in shared memory: as registers they would
    // be live (and spilled) in every thread across the Krylov loops
    __shared__ double s_t0[12];
    double& nres = s_t0[0];
    double& bnorm = s_t0[1];
    double& nl_tol = s_t0[2];
    double& inner_floor = s_t0[3];
    double& floor_abs = s_t0[4];
    double& rnorm0 = s_t0[5];
    double& omega = s_t0[6];       // relaxation (below)
    double& rprev = s_t0[7];
    double& rho_r = s_t0[8];       // rho = r^T z and the inner target: they drive the recurrences
    double& rho_i = s_t0[9];
    double& target = s_t0[10];
    // optional phase timing (thread 0, SM clock cycles): R, A, B, epilogue compute; waits
    long long cyc[5] = {0, 0, 0, 0, 0};
    long long tmark = clock64();
    auto lap = [&](int slot) {
        const long long t = clock64();
        cyc[slot] += t - tmark;
        tmark = t;
    };

    // edge coefficient at column ix (zero inside the strip and on Neumann edges)
    auto rho_at = [&](int ix, double& re, double& im) {
        re = im = 0.0;
        if ((ix == 0 && ltc) || (ix == c && rtc)) { re = rho_re; im = rho_im; }
    };
    // the edge coefficient in the working precision, rounded on the host (Robin: i p of the strip's
    // instance; S_pade: i sum a_s)
    T rho_reT = (T)0, rho_imT = p_t<T>(g);
    if constexpr (sizeof(T) == 4 && PADE) { rho_reT = a.rho_f[0]; rho_imT = a.rho_f[1]; }
    else if constexpr (PADE) { rho_reT = (T)rho_re; rho_imT = (T)rho_im; }
    auto rho_atT = [&](int ix, T& re, T& im) {
        re = im = (T)0;
        if ((ix == 0 && ltc) || (ix == c && rtc)) { re = rho_reT; im = rho_imT; }
    };
    // edge index (0 left, 1 right) of a transmission-edge column, else -1
    auto tc_edge = [&](int ix) -> int { return (ix == 0 && ltc) ? 0 : ((ix == c && rtc) ? 1 : -1); };
    // datum of the Robin data term on an edge node (l on ix=0, r on ix=c)
    auto edge_term = [&](int ix, int iy, const Coef1<double>& cy) -> double2 {
        double2 t = make_double2(0.0, 0.0);
        if (ix == 0 && ldata) {
            const double2 lm = iy > 0 ? gl[iy - 1] : make_double2(0, 0), l0 = gl[iy], lp = iy < ny ? gl[iy + 1] : make_double2(0, 0);
            t.x += cy.m[0] * lm.x + cy.m[1] * l0.x + cy.m[2] * lp.x;
            t.y += cy.m[0] * lm.y + cy.m[1] * l0.y + cy.m[2] * lp.y;
        }
        if (ix == c && rdata) {
            const double2 rm = iy > 0 ? gr[iy - 1] : make_double2(0, 0), r0 = gr[iy], rp = iy < ny ? gr[iy + 1] : make_double2(0, 0);
            t.x += cy.m[0] * rm.x + cy.m[1] * r0.x + cy.m[2] * rp.x;
            t.y += cy.m[0] * rm.y + cy.m[1] * r0.y + cy.m[2] * rp.y;
        }
        if (unit_side >= 0 && ((unit_side == 0 && ix == 0) || (unit_side == 1 && ix == c))) {
            const int d = unit_pos - iy;
            if (d >= -1 && d <= 1) t.x += cy.m[d + 1];
        }
        return t;
    };
    // phi node n >= Ns -> edge e, order s, row iy
    auto split_phi = [&](int n, int& e, int& s2, int& iy) {
        const int qq = n - Ns;
        e = qq / (m * nyn);
        const int rem = qq - e * m * nyn;
        s2 = rem / nyn;
        iy = rem - s2 * nyn;
    };
    auto gam_of = [&](int s2) { return make_double2(a.pade_d[s2].x, g.alpha + a.pade_d[s2].y); };   // i alpha + d_s
    auto sig_of = [&](int s2) { return cmul(make_double2(0.0, 1.0), cmul(a.pade_a[s2], a.pade_d[s2])); };  // i a_s d_s
    // the same coefficients in the inner precision, formed once per launch (an FP64 product and
    // conversion per phi node and Krylov iteration would occupy the FP64 pipe)
    __shared__ T2 s_pgam[PADE ? kMaxPade : 1], s_psig[PADE ? kMaxPade : 1];
    if constexpr (PADE) {
        for (int s2 = threadIdx.x; s2 < m; s2 += blockDim.x) {
            s_pgam[s2] = cfrom<T2>(gam_of(s2));
            s_psig[s2] = cfrom<T2>(sig_of(s2));
        }
        __syncthreads();
    }

    // scale of the first correction: the strip's ||(2i/dt) M h|| (FP32 must not see ~1e-111),
    // but at least 1e-6 of the whole problem's: a far-field strip (h ~ 1e-32) whose residual
    // is set by interface data far above its own h would otherwise overflow FP32
    //
    // The scalar control of the nonlinear iteration (norms, tolerances, scales, relaxation) runs
    // on thread 0 in FP64 and reaches the block through shared memory: FP64 issues at ~1/64 of
    // the FP32 rate here, and sixteen warps repeating divisions and square roots would occupy
    // the FP64 pipe for longer than the vector work of a light strip.
    __shared__ double s_nld[2];   // inv_s, the correction's scale sc
    __shared__ float s_nlf[4];    // inv_s in FP32 (clamped), sf2 (on-chip rescale), sc as a double word
    __shared__ int s_nli[2];      // decision, status
    // relaxation of the fixed point: zeta += omega delta, i.e. zeta^q = omega F(zeta^{q-1}) +
    // (1 - omega) zeta^{q-1} (same limit); omega shrinks when a correction does not cut the
    // residual by 10% (the plain iteration diverges for strong nonlinearity)
    if (threadIdx.x == 0) {
        nres = bnorm = rnorm0 = rprev = rho_r = rho_i = target = 0.0;
        const double bscale_inst = a.bscale ? ((volatile const double*)a.bscale)[si.inst] : 0.0;
        const double s_first = fmax(a.bnorm0 ? a.bnorm0[j] : 0.0, 1e-6 * bscale_inst);
        nl_tol = a.nl_tol_strip ? a.nl_tol_strip[j] : a.nl_tol;
        const double nl_floor_frac = a.nl_tol_strip ? a.nl_floor_frac * nl_tol / a.nl_tol : a.nl_floor_frac;
        inner_floor = a.nl_tol_strip ? 0.1 * nl_tol : a.inner_floor;
        floor_abs = nl_floor_frac * bscale_inst;
        omega = (a.nl_relax > 0.0 && a.nl_relax <= 1.0) ? a.nl_relax : 1.0;
        const double is0 = s_first > 0.0 ? 1.0 / s_first : 1.0;
        s_nld[0] = is0;
        s_nlf[0] = (float)fmin(is0, 1e30);
    }
    __syncthreads();
    double inv_s = s_nld[0];      // every thread's copy follows thread 0's
    float inv_sf = s_nlf[0];

    // Double-word residual constants.  On the uniform mesh the 1D factors are exact multiples
    // of [1 d 1] (mass, d = 4 inside, 2 at an end) and [-1 e -1] (stiffness, e = 2 / 1), so
    //   A zeta = -C1 U + i C2 V - C3 Wk + i C5 Tm0 [transmission edge] + c zeta,
    // with Tm = [1 dy 1] zeta and Tk = [-1 ey -1] zeta along y, U = [-1 ex -1] Tm,
    // V = [1 dx 1] Tm, Wk = [1 dx 1] Tk along x (exact weights: powers of two), and
    // C1 = hy/(6hx), C2 = alpha hx hy/36, C3 = hx/(6hy), C5 = p hy/6, c = w W + w kappa|zeta|^2.
    dw nC1{}, nC2{}, C2{}, nC3{}, nC5{}, C5{}, C5r{}, C6{};
    float C6f = 0.f;
    const float cfacf = a.nl_picard ? 1.f : 2.f;
    if constexpr (DW) {
        // double-word constants split on the host (Geom::fill_coefficients; no FP64 conversion here)
        nC1 = {g.dwk[0], g.dwk[1]};
        C2 = {g.dwk[2], g.dwk[3]};
        nC2 = dw_neg(C2);
        nC3 = {g.dwk[4], g.dwk[5]};
        // edge coefficient rho hy/6: i p hy/6 (Robin, per instance) or (rho_re + i rho_im) hy/6 (S_pade)
        if constexpr (PADE) {
            C5r = {a.dwrho[0], a.dwrho[1]};
            C5 = {a.dwrho[2], a.dwrho[3]};
        } else {
            C5 = {g.dwk[6], g.dwk[7]};
        }
        nC5 = dw_neg(C5);
        if (a.mode == 0) C6 = {g.dwk[8], g.dwk[9]};
        C6f = C6.h;
        // zeta, b = (2i/dt) M h - M^Gamma Q^T (l; r) and w W in double-word form, ||b||^2.
        // Integer splits away from the edge columns (no FP64 instruction there); ||b||^2 in
        // FP32 in units of the first correction's scale, edge columns apart.
        const dw HXHY = {g.dwk[10], g.dwk[11]};
        const float bsc = (float)inv_s;
        float bb = 0.f, be = 0.f;
        auto edge_b = [&](int ix, int iy, long long idx) {
            const Coef1<double> cy = coef1<double>(iy, ny, KYd);
            double2 b = rhs0 ? rhs0[idx] : make_double2(0.0, 0.0);
            b = csub(b, edge_term(ix, iy, cy));
            const cdw bv = {dw_from(b.x), dw_from(b.y)};
            cdw_st(bdw + idx, bv);
            const float bxs = bv.x.h * bsc, bys = bv.y.h * bsc;
            be += bxs * bxs + bys * bys;
        };
        // zeta, its accumulated correction and w W of one node in double-word form
        auto init_node = [&](int ix, int iy, long long idx) {
            const double2 zv = zeta[idx];
            cdw_st(zdw + idx, {dw_from_bits(zv.x), dw_from_bits(zv.y)});
            if (a.dw_mode == 0) cdw_st(ddw + idx, cdw_zero());
            const float qxy = ((ix > 0 && ix < c) ? 1.f : 0.5f) * ((iy > 0 && iy < ny) ? 1.f : 0.5f);
            const dw wv = Wn ? dw_pow2(dw_mul(dw_from_bits(Wn[idx]), HXHY), qxy) : dw{0.f, 0.f};
            a.wdw[sbase + idx] = make_float2(wv.h, wv.l);
        };
        // the 2 nyn edge nodes (FP64 data term) in equal shares over the strip's blocks
        const int ne = 2 * nyn, epc = (ne + bps - 1) / bps;
        for (int t = rank * epc + threadIdx.x; t < min(ne, (rank + 1) * epc); t += blockDim.x) {
            const int ix = t < nyn ? 0 : c, iy = t < nyn ? t : t - nyn;
            const long long idx = (long long)ix * P + iy;
            edge_b(ix, iy, idx);
            if (a.dw_mode != 2) init_node(ix, iy, idx);
        }
        // the state and b off the edges: this step's already in dw_mode 2
        if (a.dw_mode != 2) {
            for (int n = it_first(Ns); n < it_end(Ns); n += it_step) {
                int ix, iy;
                split_node(n, nyn, inv_nyn, ix, iy);
                if (ix == 0 || ix == c) continue;
                const long long idx = (long long)ix * P + iy;
                const double2 b = rhs0 ? rhs0[idx] : make_double2(0.0, 0.0);
                const cdw bv = {dw_from_bits(b.x), dw_from_bits(b.y)};
                cdw_st(bdw + idx, bv);
                const float bxs = bv.x.h * bsc, bys = bv.y.h * bsc;
                bb += bxs * bxs + bys * bys;
                init_node(ix, iy, idx);
            }
        }
        float lbT[2] = {bb, be};
        dw lb2[2];
        block_sum_dw<2>(lbT, lb2, (float*)s_red);
        double lb[4] = {0.0, 0.0, 0.0, 0.0}, tb[4];
        if (threadIdx.x == 0) {
            const double bs2 = (double)bsc * (double)bsc;
            lb[0] = dw_to(lb2[0]) / bs2;
            lb[1] = dw_to(lb2[1]) / bs2;
        }
        if (!strip_sum4(lb, tb)) status = DD_NLS_ETIMEOUT;
        if (!status && threadIdx.x == 0) {
            if (a.dw_mode == 2) tb[0] = a.bint2[j];
            else if (a.dw_mode == 1 && rank == 0) a.bint2[j] = tb[0];
            bnorm = sqrt(tb[0] + tb[1]);
        }
        lap(0);
    }
    // The double-word residual resolves about 1e-14 of ||b||: below kDWFinish the strip folds
    // its accumulated correction into the FP64 zeta and finishes with the FP64 residual (only
    // with zeta as the state, dw_mode 0; the host keeps tighter tolerances out of modes 1 and 2).
    bool dwr = DW;

    for (; !status; ++nl_it) {
        // ---------------- phase R: coefficients c = w (W + kappa|zeta|^2) and FP64 residual
        // A work item is a run of RX consecutive x-nodes at one y: the y-direction sums
        // (My zeta, Ky zeta) of each column are formed once and used by the three nodes that
        // need them.  ||b||^2 only in the launch's first residual (b is fixed in a launch).
        double loc[4] = {0.0, 0.0, 0.0, 0.0};   // ||res||^2, ||b||^2, rho = r^T z (re, im)
        T rz_re = 0, rz_im = 0;
        float rr_f = 0.f;                        // double-word residual: ||res||^2 partial
        const bool need_b = !DW && nl_it == 0;
        for (int n = it_first(NRall); n < it_end(NRall); n += it_step) {
            if (DW && dwr && (!PADE || n < NR)) {
                const int seg = n / nyn;
                const int iy = n - seg * nyn;
                const int x0 = seg * RX, x1 = min(x0 + RX, g.nxs);
                const bool ylo = iy > 0, yhi = iy < ny;
                const float dY = (ylo && yhi) ? 4.f : 2.f, eY = (ylo && yhi) ? 2.f : 1.f;
                const float qy = (ylo && yhi) ? 1.f : 0.5f;
                const Coef1<T> cyT = coef1<T>(iy, ny, KYt);
                // exact-weight y sums of column ix at row iy
                auto colsum = [&](int ix, cdw& Tm, cdw& Tk, cdw& zc) {
                    const float4* col = zdw + (long long)ix * P + iy;
                    zc = cdw_ld(col);
                    const cdw S = (ylo && yhi) ? cdw_add_s(cdw_ld(col - 1), cdw_ld(col + 1)) : cdw_ld(ylo ? col - 1 : col + 1);
                    Tm = cdw_add_s(S, cdw_pow2(zc, dY));
                    Tk = cdw_sub_s(cdw_pow2(zc, eY), S);
                };
                cdw Tmm = cdw_zero(), Tkm = cdw_zero(), Tm0, Tk0, z0, zdum;
                if (x0 > 0) colsum(x0 - 1, Tmm, Tkm, zdum);
                colsum(x0, Tm0, Tk0, z0);
                for (int ix = x0; ix < x1; ++ix) {
                    cdw Tmp = cdw_zero(), Tkp = cdw_zero(), zp = cdw_zero();
                    if (ix < c) colsum(ix + 1, Tmp, Tkp, zp);
                    const bool xlo = ix > 0, xhi = ix < c;
                    const float dX = (xlo && xhi) ? 4.f : 2.f, eX = (xlo && xhi) ? 2.f : 1.f;
                    const float qxy = ((xlo && xhi) ? 1.f : 0.5f) * qy;
                    const cdw Q = (xlo && xhi) ? cdw_add_s(Tmm, Tmp) : (xlo ? Tmm : Tmp);
                    const cdw Kq = (xlo && xhi) ? cdw_add_s(Tkm, Tkp) : (xlo ? Tkm : Tkp);
                    const cdw U = cdw_sub_s(cdw_pow2(Tm0, eX), Q);
                    const cdw V = cdw_add_s(Q, cdw_pow2(Tm0, dX));
                    const cdw Wk = cdw_add_s(Kq, cdw_pow2(Tk0, dX));
                    dw ax = dw_add_s(dw_add_s(dw_mul(nC1, U.x), dw_mul(nC2, V.y)), dw_mul(nC3, Wk.x));
                    dw ay = dw_add_s(dw_add_s(dw_mul(nC1, U.y), dw_mul(C2, V.x)), dw_mul(nC3, Wk.y));
                    const long long idx = (long long)ix * P + iy;
                    if ((ix == 0 && ltc) || (ix == c && rtc)) {
                        ax = dw_add_s(ax, dw_mul(nC5, Tm0.y));
                        ay = dw_add_s(ay, dw_mul(C5, Tm0.x));
                        if constexpr (PADE) {
                            ax = dw_add_s(ax, dw_mul(C5r, Tm0.x));
                            ay = dw_add_s(ay, dw_mul(C5r, Tm0.y));
                            // B_s phi_s = -i a_s d_s M^G phi_s on the edge rows (FP64; 2(ny+1) nodes)
                            const int e = ix == 0 ? 0 : 1;
                            const Coef1<double> cyd = coef1<double>(iy, ny, KYd);
                            double2 cpl = make_double2(0.0, 0.0);
                            for (int s2 = 0; s2 < m; ++s2)
                                cpl = cadd(cpl, cmul(sig_of(s2), edge_mass<double, double2>(phi + ((long long)e * m + s2) * P, iy, ny, cyd)));
                            ax = dw_sub_s(ax, dw_from(cpl.x));
                            ay = dw_sub_s(ay, dw_from(cpl.y));
                        }
                    }
                    const dw a2 = dw_add_s(dw_mul(z0.x, z0.x), dw_mul(z0.y, z0.y));
                    const float2 wv2 = wdw[idx];
                    const dw cd = dw_add_s(dw{wv2.x, wv2.y}, dw_mul(dw_pow2(C6, qxy), a2));
                    ax = dw_add_s(ax, dw_mul(cd, z0.x));
                    ay = dw_add_s(ay, dw_mul(cd, z0.y));
                    const cdw bv = cdw_ld(bdw + idx);
                    const dw rx = dw_sub_s(bv.x, ax), ry = dw_sub_s(bv.y, ay);
                    // the correction's operator in the inner precision
                    const T cop = wv2.x + cfacf * (C6f * qxy) * a2.h;
                    T rre, rim;
                    rho_atT(ix, rre, rim);
                    const Coef1<T> cxT = coef1<T>(ix, c, KXt);
                    T2 rT;
                    rT.x = rx.h * inv_sf;
                    rT.y = ry.h * inv_sf;
                    rr_f += rT.x * rT.x + rT.y * rT.y;    // scaled: no underflow of tiny residuals
                    const T2 di = diag_inv<T>(cxT, cyT, alphaT, rre, rim, cop);
                    const T2 zT = cmul(di, rT);
                    cT[idx] = cop;
                    r[idx] = rT;
                    if constexpr (SR) dv[idx] = di;
                    if (!use_sr) {
                        z[idx] = zT;
                        x[idx] = mk<T2>(0.0, 0.0);
                        p[idx] = mk<T2>(0.0, 0.0);
                        q[idx] = mk<T2>(0.0, 0.0);
                    }
                    rz_re += rT.x * zT.x - rT.y * zT.y;
                    rz_im += rT.x * zT.y + rT.y * zT.x;
                    Tmm = Tm0; Tkm = Tk0;
                    Tm0 = Tmp; Tk0 = Tkp; z0 = zp;
                }
            } else if (!PADE || n < NR) {
                const int seg = n / nyn;
                const int iy = n - seg * nyn;
                const int x0 = seg * RX, x1 = min(x0 + RX, g.nxs);
                const Coef1<double> cy = coef1<double>(iy, ny, KYd);
                const Coef1<T> cyT = coef1<T>(iy, ny, KYt);
                const double wy = wq(iy, ny, g.hy);
                // y-direction sums of column ix at row iy
                auto colsum = [&](int ix, double2& tM, double2& tK, double2& zc) {
                    const double2* col = zeta + (long long)ix * P + iy;
                    zc = col[0];
                    const double2 am = iy > 0 ? col[-1] : make_double2(0.0, 0.0);
                    const double2 ap = iy < ny ? col[1] : make_double2(0.0, 0.0);
                    tM.x = cy.m[0] * am.x + cy.m[1] * zc.x + cy.m[2] * ap.x;
                    tM.y = cy.m[0] * am.y + cy.m[1] * zc.y + cy.m[2] * ap.y;
                    tK.x = cy.k[0] * am.x + cy.k[1] * zc.x + cy.k[2] * ap.x;
                    tK.y = cy.k[0] * am.y + cy.k[1] * zc.y + cy.k[2] * ap.y;
                };
                double2 tMm = make_double2(0.0, 0.0), tKm = tMm, tM0, tK0, z0, zdum;
                if (x0 > 0) colsum(x0 - 1, tMm, tKm, zdum);
                colsum(x0, tM0, tK0, z0);
                for (int ix = x0; ix < x1; ++ix) {
                    double2 tMp = make_double2(0.0, 0.0), tKp = tMp, zp = tMp;
                    if (ix < c) colsum(ix + 1, tMp, tKp, zp);
                    const Coef1<double> cx = coef1<double>(ix, c, KXd);
                    double rre, rim;
                    rho_at(ix, rre, rim);
                    // sum over dx of (Bx(ix, ix+dx) tM - Mx(ix, ix+dx) tK), Bx = -Kx + i alpha Mx + rho E
                    double2 Az = make_double2(0.0, 0.0);
                    {
                        const double bre = -cx.k[0], bim = g.alpha * cx.m[0];
                        Az.x += bre * tMm.x - bim * tMm.y - cx.m[0] * tKm.x;
                        Az.y += bre * tMm.y + bim * tMm.x - cx.m[0] * tKm.y;
                    }
                    {
                        const double bre = -cx.k[1] + rre, bim = g.alpha * cx.m[1] + rim;
                        Az.x += bre * tM0.x - bim * tM0.y - cx.m[1] * tK0.x;
                        Az.y += bre * tM0.y + bim * tM0.x - cx.m[1] * tK0.y;
                    }
                    {
                        const double bre = -cx.k[2], bim = g.alpha * cx.m[2];
                        Az.x += bre * tMp.x - bim * tMp.y - cx.m[2] * tKp.x;
                        Az.y += bre * tMp.y + bim * tMp.x - cx.m[2] * tKp.y;
                    }
                    const long long idx = (long long)ix * P + iy;
                    const double W = Wn ? Wn[idx] : 0.0;
                    const double wxy = wq(ix, c, g.hx) * wy, a2 = z0.x * z0.x + z0.y * z0.y;
                    const double cdiag = wxy * (W + kap * a2);                 // the residual's operator
                    const double cop = wxy * (W + cfac * kap * a2);            // the correction's operator
                    Az.x += cdiag * z0.x;
                    Az.y += cdiag * z0.y;
                    if (PADE) {
                        const int e = tc_edge(ix);
                        if (e >= 0)            // B_s phi_s = -i a_s d_s M^G phi_s on the edge rows
                            for (int s2 = 0; s2 < m; ++s2) {
                                const double2 mph = edge_mass<double, double2>(phi + ((long long)e * m + s2) * P, iy, ny, cy);
                                Az = csub(Az, cmul(sig_of(s2), mph));
                            }
                    }
                    double2 b = rhs0 ? rhs0[idx] : make_double2(0.0, 0.0);
                    if (ix == 0 || ix == c || unit_side >= 0) b = csub(b, edge_term(ix, iy, cy));
                    const double2 res = csub(b, Az);
                    loc[0] += res.x * res.x + res.y * res.y;
                    if (need_b) loc[1] += b.x * b.x + b.y * b.y;
                    const Coef1<T> cxT = coef1<T>(ix, c, KXt);
                    const T2 rT = cfrom<T2>(make_double2(res.x * inv_s, res.y * inv_s));
                    const T2 di = diag_inv<T>(cxT, cyT, alphaT, (T)rre, (T)rim, (T)cop);
                    const T2 zT = cmul(di, rT);
                    cT[idx] = (T)cop;
                    r[idx] = rT;
                    if (use_sr) {
                        dv[idx] = di;
                    } else {
                        z[idx] = zT;
                        x[idx] = mk<T2>(0.0, 0.0);
                        p[idx] = mk<T2>(0.0, 0.0);
                        q[idx] = mk<T2>(0.0, 0.0);
                    }
                    rz_re += rT.x * zT.x - rT.y * zT.y;
                    rz_im += rT.x * zT.y + rT.y * zT.x;
                    tMm = tM0; tKm = tK0;
                    tM0 = tMp; tK0 = tKp; z0 = zp;
                }
            } else {
                int e, s2, iy;
                split_phi(n - NR + Ns, e, s2, iy);
                if (!(e == 0 ? ltc : rtc)) continue;
                const int ixe = e == 0 ? 0 : c;
                const long long fi = ((long long)e * m + s2) * P + iy;
                const Coef1<double> cy = coef1<double>(iy, ny, KYd);
                // the edge column of the strip state: zeta, or the double-word fields while they are it
                auto zedge = [&](int yy) -> double2 {
                    if constexpr (DW) {
                        if (dwr) {
                            const cdw q = cdw_ld(zdw + (long long)ixe * P + yy);
                            return make_double2(dw_to(q.x), dw_to(q.y));
                        }
                    }
                    return zeta[(long long)ixe * P + yy];
                };
                const double2 ze = zedge(iy);
                const double2 zem = iy > 0 ? zedge(iy - 1) : make_double2(0.0, 0.0);
                const double2 zep = iy < ny ? zedge(iy + 1) : make_double2(0.0, 0.0);
                const double W = Wn ? Wn[(long long)ixe * P + iy] : 0.0;
                const double ae2 = ze.x * ze.x + ze.y * ze.y;
                const double cphi = wq(iy, ny, g.hy) * (W + kap * ae2);
                const double cphi_op = wq(iy, ny, g.hy) * (W + cfac * kap * ae2);
                const double2 gam = gam_of(s2), sig = sig_of(s2);
                const double2 res = make_double2(0.0, 0.0);
                const double2 J = phi_row_v<double, double2>(zem, ze, zep, phi + ((long long)e * m + s2) * P, iy, ny,
                                                             cy, gam, sig, cphi);
                const double2 rs = csub(res, J);
                const Coef1<T> cyT = coef1<T>(iy, ny, KYt);
                const T2 rT = cfrom<T2>(make_double2(rs.x * inv_s, rs.y * inv_s));
                if (DW && dwr) rr_f += rT.x * rT.x + rT.y * rT.y;   // the double-word pass's scaled sum
                else loc[0] += rs.x * rs.x + rs.y * rs.y;
                const T2 di = phi_diag_inv<T, T2>(cyT, cfrom<T2>(gam), cfrom<T2>(sig), (T)cphi_op);
                const T2 zT = cmul(di, rT);
                if (s2 == 0) cTf[(long long)e * P + iy] = (T)cphi_op;
                rf[fi] = rT;
                zf[fi] = zT;
                xf[fi] = mk<T2>(0.0, 0.0);
                pf[fi] = mk<T2>(0.0, 0.0);
                qf[fi] = mk<T2>(0.0, 0.0);
                rz_re += rT.x * zT.x - rT.y * zT.y;
                rz_im += rT.x * zT.y + rT.y * zT.x;
            }
        }
        bool fp32_sums = false;
        if constexpr (DW) fp32_sums = dwr;
        if (fp32_sums) {
            // the double-word residual's partials are FP32 (scaled units): block sum in double
            // words on the FP32 pipe, conversion to FP64 by thread 0 alone
            float lT[3] = {rr_f, (float)rz_re, (float)rz_im};
            dw l3[3];
            block_sum_dw<3>(lT, l3, (float*)s_red);
            if (threadIdx.x == 0) {
                const double isf = (double)inv_sf;
                loc[0] = dw_to(l3[0]) / (isf * isf);
                loc[1] = 0.0;
                loc[2] = dw_to(l3[1]);
                loc[3] = dw_to(l3[2]);
            }
        } else {
            loc[2] = (double)rz_re;
            loc[3] = (double)rz_im;
            block_sum<4>(loc, s_red);
        }
        lap(0);
        double tot[4];
        if (!strip_sum4(loc, tot)) { status = DD_NLS_ETIMEOUT; break; }
        lap(4);
        // thread 0 decides: 0 go on, 1 converged, 2 error (status), 3 leave the double-word residual
        if (threadIdx.x == 0) {
            const double rnorm = sqrt(tot[0]);
            if (need_b) bnorm = sqrt(tot[1]);
            nres = bnorm > 0.0 ? rnorm / bnorm : rnorm;
            int ctl = 0, st = 0;
            if (!isfinite(tot[0]) || !isfinite(tot[1])) {
                ctl = 2;
                st = DD_NLS_ENONFINITE;
            } else if (nres <= nl_tol || rnorm <= floor_abs || rnorm == 0.0) {
                ctl = 1;
            } else if (nl_it >= a.max_nl) {
                ctl = 2;
                st = DD_NLS_ENOCONV;
            } else if (DW && dwr && a.dw_mode == 0 && nres <= kDWFinish) {
                ctl = 3;
                inv_s = 1.0 / rnorm;
                rprev = INFINITY;
                s_nld[0] = inv_s;
                s_nlf[0] = (float)fmin(inv_s, 1e30);
            } else {
                if (nl_it > 0 && rnorm > 0.9 * rprev) omega = fmax(0.25, 0.6 * omega);
                rprev = rnorm;
                rnorm0 = rnorm;
                rho_r = tot[2];
                rho_i = tot[3];
                // inner stopping test in the scaled units of r
                target = fmax(a.inner_tol * rnorm, fmax(inner_floor * bnorm, 0.1 * floor_abs)) * inv_s;
                // r holds res * inv_s, scaled for the launch's first correction; a later one (a
                // strip near convergence) is far smaller, and FP32 squares of the on-chip
                // recurrences (|delta|^2, ||r||^2) would underflow: the power of two sf2 brings
                // ||r|| to [1/2, 1) there (exact; the correction's scale takes the same factor)
                int e2 = 0;
                (void)frexp(rnorm * inv_s, &e2);
                e2 = max(-120, min(120, e2));
                s_nlf[1] = __int_as_float((127 - e2) << 23);   // 2^-e2
            }
            s_nli[0] = ctl;
            s_nli[1] = st;
        }
        __syncthreads();
        {
            const int ctl = s_nli[0];
            if (ctl == 1) break;
            if (ctl == 2) { status = s_nli[1]; break; }
        }
        if (DW && dwr && s_nli[0] == 3) {
            for (int n = it_first(Ns); n < it_end(Ns); n += it_step) {
                int ix, iy;
                split_node(n, nyn, inv_nyn, ix, iy);
                const long long idx = (long long)ix * P + iy;
                const cdw d = cdw_ld(ddw + idx);
                const double2 zv = zeta[idx];
                zeta[idx] = make_double2(zv.x + dw_to(d.x), zv.y + dw_to(d.y));
            }
            dwr = false;
            inv_s = s_nld[0];
            inv_sf = s_nlf[0];
            if (!strip_barrier()) { status = DD_NLS_ETIMEOUT; break; }
            continue;       // the next residual is the FP64 one
        }

        // ---------------- inner COCG on A(c) delta = res, Jacobi preconditioner
        if (CLU && use_sr) {
            if constexpr (CLU) {
            // ---- single-reduction COCG with the Krylov state on chip (one strip per cluster).
            // Slab of this CTA: rows [y0, y1) of every column; node m < M of the slab is column
            // m / h, row y0 + m % h, and node k of this thread is m = threadIdx.x + k BS.
            const int H = (nyn + kClusterCTAs - 1) / kClusterCTAs;
            const int y0 = min(nyn, rank * H), y1 = min(nyn, y0 + H), h = y1 - y0;
            const int M = h * g.nxs, ZP = H + 2, NX = g.nxs;
            const float inv_h = h > 0 ? 1.0f / (float)h : 0.f;
            // disjoint arrays of the dynamic shared memory (restrict: loads of one node may be
            // scheduled ahead of the stores of the previous one)
            float2* __restrict__ Zs = (float2*)s_dyn;                  // z with halo rows: [NX][H + 2]
            float2* __restrict__ Ws = (float2*)s_dyn + (size_t)NX * ZP;            // [NX][H]
            float2* __restrict__ Ps = (float2*)s_dyn + (size_t)NX * (ZP + H);
            float2* __restrict__ Ss = (float2*)s_dyn + (size_t)NX * (ZP + 2 * H);
            float2* __restrict__ Ds = (float2*)s_dyn + (size_t)NX * (ZP + 3 * H);  // D^-1
            float2* __restrict__ Ex = (float2*)s_dyn + (size_t)NX * (ZP + 4 * H);  // exported rows [2 parity][2 side][r w s][NX]
            float2* __restrict__ Dh = Ex + (size_t)12 * NX;            // D^-1 of the halo rows [up, down][NX]
            float* __restrict__ Cs = (float*)(Ex + (size_t)16 * NX);   // c of A(c)
            auto exp_at = [&](int par, int side, int arr, int ix) { return Ex + ((size_t)(par * 2 + side) * 3 + arr) * NX + ix; };
            const Interior9<T2> W9 = interior9<T, T2>(KXt, KYt, alphaT);
            // w = A(c) z at slab node (ix, iy): the interior stencil off the edges, else the general one
            auto apply_at = [&](int ix, int iy, int zo, T cdg) -> T2 {
                if (ix > 0 && ix < c && iy > 0 && iy < ny) return apply_interior<T, T2>(Zs, zo, ZP, W9, cdg);
                const Coef1<T> cxT = coef1<T>(ix, c, KXt), cyT = coef1<T>(iy, ny, KYt);
                T rre, rim;
                rho_atT(ix, rre, rim);
                return apply_op<T, T2>(Zs, zo, ix, iy, c, ny, ZP, cxT, cyT, alphaT, rre, rim, cdg);
            };
            const bool has_up = y0 > 0 && h > 0, has_dn = y1 < nyn && h > 0;
            const unsigned nb_up = (unsigned)(rank - 1), nb_dn = (unsigned)(rank + 1);
            T2 rreg[kOnChipNPT], xreg[kOnChipNPT];
            const T2 zeroT = mk<T2>(0.0, 0.0);
            // r rescaled by the power of two sf2 (thread 0's choice above)
            const float sf2 = s_nlf[1];
            const T2 sf2v = T2{sf2, 0.f};
            // load r_0 (scaled residual), D^-1, c of the residual pass; x = p = s_{-1} = 0
#pragma unroll
            for (int k = 0; k < kOnChipNPT; ++k) {
                const int mm = threadIdx.x + k * BS;
                rreg[k] = zeroT;
                xreg[k] = zeroT;
                if (mm >= M) continue;
                int ix, il;
                split_node(mm, h, inv_h, ix, il);
                const long long idx = (long long)ix * P + y0 + il;
                const int o = ix * H + il;
                const T2 dvv = dv[idx];
                const T2 r0 = r[idx];
                rreg[k] = T2{r0.x * sf2, r0.y * sf2};
                Ds[o] = dvv;
                Cs[o] = cT[idx];
                Ps[o] = zeroT;
                Ss[o] = zeroT;
                Zs[ix * ZP + il + 1] = cmul(dvv, rreg[k]);
            }
            // halo rows of z_0 = D^-1 r_0 and their D^-1 (fixed during the solve) from global memory
            // (written by the residual pass)
            for (int ix = threadIdx.x; ix < NX; ix += BS) {
                if (has_up) {
                    const T2 du = dv[(long long)ix * P + y0 - 1];
                    Dh[ix] = du;
                    Zs[ix * ZP] = cmul(cmul(du, r[(long long)ix * P + y0 - 1]), sf2v);
                }
                if (has_dn) {
                    const T2 dd = dv[(long long)ix * P + y1];
                    Dh[NX + ix] = dd;
                    Zs[ix * ZP + h + 1] = cmul(cmul(dd, r[(long long)ix * P + y1]), sf2v);
                }
            }
            __syncthreads();
            // w_0 = A z_0, delta_0 = w_0^T z_0; export the slab's first and last rows (parity 0)
            T d0r = 0, d0i = 0;
#pragma unroll
            for (int k = 0; k < kOnChipNPT; ++k) {
                const int mm = threadIdx.x + k * BS;
                if (mm >= M) continue;
                int ix, il;
                split_node(mm, h, inv_h, ix, il);
                const int iy = y0 + il, o = ix * H + il, zo = ix * ZP + il + 1;
                const T2 w0 = apply_at(ix, iy, zo, Cs[o]);
                const T2 zo_v = Zs[zo];
                Ws[o] = w0;
                d0r += w0.x * zo_v.x - w0.y * zo_v.y;
                d0i += w0.x * zo_v.y + w0.y * zo_v.x;
                if (il == 0) {
                    *exp_at(0, 0, 0, ix) = rreg[k]; *exp_at(0, 0, 1, ix) = w0; *exp_at(0, 0, 2, ix) = zeroT;
                }
                if (il == h - 1) {
                    *exp_at(0, 1, 0, ix) = rreg[k]; *exp_at(0, 1, 1, ix) = w0; *exp_at(0, 1, 2, ix) = zeroT;
                }
            }
            // thread-0 state of the recurrences, in double words (no FP64 on the iteration path),
            // kept in shared memory (no registers in the other threads): gamma_k, 1/gamma_k,
            // q_k = 1/(gamma_k alpha_k), alpha_k, beta_k, the stopping bound and the stagnation guard
            cdw& gam = *reinterpret_cast<cdw*>(s_kr);
            cdw& ig = *reinterpret_cast<cdw*>(s_kr + 4);
            cdw& qk = *reinterpret_cast<cdw*>(s_kr + 8);
            cdw& al = *reinterpret_cast<cdw*>(s_kr + 12);
            cdw& be = *reinterpret_cast<cdw*>(s_kr + 16);
            float& target2 = s_kr[20];
            float& best2 = s_kr[21];      // least ||r||^2 so far
            int& since = s_kri;           // iterations since it fell by 1%
            if (threadIdx.x == 0) {
                const double sf2d = (double)sf2;
                gam = {dw_from(rho_r * sf2d * sf2d), dw_from(rho_i * sf2d * sf2d)};
                ig = qk = al = be = cdw_zero();
                target2 = (float)((target * sf2d) * (target * sf2d));
                best2 = INFINITY;
                since = 0;
                inv_s *= sf2d;      // x is the correction in units of 1/(inv_s sf2)
            }
            float* s_outf = (float*)s_out;
            {
                float lT[2] = {d0r, d0i};
                dw l2[2];
                block_sum_dw<2>(lT, l2, (float*)s_red);
                lap(1);
                dw dl[2];
                if (!cluster_allreduce_dw<2>(s_cld, l2, dl, ++cepoch, bps, a.err, wait_ns, s_outf, &s_flag)) {
                    status = DD_NLS_ETIMEOUT;
                    break;
                }
                if (threadIdx.x == 0) {
                    const cdw del = {dl[0], dl[1]};
                    const float dd2 = cdw_abs2(del).h;
                    int ctl = 0, st = 0;
                    if (!(dd2 > 0.f) || !isfinite(dd2)) {
                        ctl = 2;
                        st = isfinite(dd2) ? DD_NLS_EBREAKDOWN : DD_NLS_ENONFINITE;
                    } else {
                        al = cdw_mul(gam, cdw_recip(del));     // alpha_0 = gamma_0 / delta_0
                        if (cdw_nonzero(gam)) {
                            const cdw rg2 = cdw_recip(cdw_mul(gam, gam));
                            ig = cdw_mul(gam, rg2);
                            qk = cdw_mul(del, rg2);
                        }
                    }
                    s_ctl[0] = ctl;
                    s_ctl[1] = st;
                    s_sc[0] = al.x.h;
                    s_sc[1] = al.y.h;
                }
            }
            __syncthreads();
            lap(4);
            if (s_ctl[0]) { status = s_ctl[1]; break; }
            T2 alT = T2{s_sc[0], s_sc[1]}, beT = T2{0, 0};
            int cstat = 0;
            for (int it = 0; it < a.max_inner; ++it) {
                const int pin = it & 1, pout = pin ^ 1;
                // phase 1: p_k = z_k + beta p_{k-1}, s_k = w_k + beta s_{k-1}, x += alpha p_k,
                // r_{k+1} = r_k - alpha s_k, z_{k+1} = D^-1 r_{k+1}
#pragma unroll
                for (int k = 0; k < kOnChipNPT; ++k) {
                    const int mm = threadIdx.x + k * BS;
                    if (mm >= M) continue;
                    int ix, il;
                    split_node(mm, h, inv_h, ix, il);
                    const int o = ix * H + il;
                    const T2 dvv = Ds[o];
                    const T2 pn = cfma(beT, Ps[o], cmul(dvv, rreg[k]));
                    T2 sn;
                    rreg[k] = rnext_v(rreg[k], Ws[o], Ss[o], alT, beT, sn);
                    xreg[k] = cfma(alT, pn, xreg[k]);
                    Ps[o] = pn;
                    Ss[o] = sn;
                    Zs[ix * ZP + il + 1] = cmul(dvv, rreg[k]);
                }
                // halo rows of z_{k+1}, rebuilt from the neighbours' exported r_k, w_k, s_{k-1}
                for (int ix = threadIdx.x; ix < NX; ix += BS) {
                    if (has_up) {
                        T2 sv;
                        const T2 rr = rnext_v(ld_cluster_f2(mapa(smem_addr(exp_at(pin, 1, 0, ix)), nb_up)),
                                              ld_cluster_f2(mapa(smem_addr(exp_at(pin, 1, 1, ix)), nb_up)),
                                              ld_cluster_f2(mapa(smem_addr(exp_at(pin, 1, 2, ix)), nb_up)), alT, beT, sv);
                        Zs[ix * ZP] = cmul(Dh[ix], rr);
                    }
                    if (has_dn) {
                        T2 sv;
                        const T2 rr = rnext_v(ld_cluster_f2(mapa(smem_addr(exp_at(pin, 0, 0, ix)), nb_dn)),
                                              ld_cluster_f2(mapa(smem_addr(exp_at(pin, 0, 1, ix)), nb_dn)),
                                              ld_cluster_f2(mapa(smem_addr(exp_at(pin, 0, 2, ix)), nb_dn)), alT, beT, sv);
                        Zs[ix * ZP + h + 1] = cmul(Dh[NX + ix], rr);
                    }
                }
                __syncthreads();
                // phase 2: w_{k+1} = A z_{k+1}; gamma = r^T z, delta = w^T z, ||r||^2; export rows
                T g_r = 0, g_i = 0, dlt_r = 0, dlt_i = 0, rr2 = 0;
#pragma unroll
                for (int k = 0; k < kOnChipNPT; ++k) {
                    const int mm = threadIdx.x + k * BS;
                    if (mm >= M) continue;
                    int ix, il;
                    split_node(mm, h, inv_h, ix, il);
                    const int iy = y0 + il, o = ix * H + il, zo = ix * ZP + il + 1;
                    const T2 wn = apply_at(ix, iy, zo, Cs[o]);
                    const T2 zz = Zs[zo], rv = rreg[k];
                    Ws[o] = wn;
                    g_r += rv.x * zz.x - rv.y * zz.y;
                    g_i += rv.x * zz.y + rv.y * zz.x;
                    dlt_r += wn.x * zz.x - wn.y * zz.y;
                    dlt_i += wn.x * zz.y + wn.y * zz.x;
                    rr2 += rv.x * rv.x + rv.y * rv.y;
                    if (il == 0) {
                        *exp_at(pout, 0, 0, ix) = rv; *exp_at(pout, 0, 1, ix) = wn; *exp_at(pout, 0, 2, ix) = Ss[o];
                    }
                    if (il == h - 1) {
                        *exp_at(pout, 1, 0, ix) = rv; *exp_at(pout, 1, 1, ix) = wn; *exp_at(pout, 1, 2, ix) = Ss[o];
                    }
                }
                float lT[5] = {g_r, g_i, dlt_r, dlt_i, rr2};
                dw l5[5];
                block_sum_dw<5>(lT, l5, (float*)s_red);
                lap(2);
                // one exchange per iteration: gamma, delta and ||r||^2; the rows exported above are
                // visible to the neighbours once it completes
                dw gg[5];
                if (!cluster_allreduce_dw<5>(s_cld, l5, gg, ++cepoch, bps, a.err, wait_ns, s_outf, &s_flag)) {
                    cstat = DD_NLS_ETIMEOUT;
                    break;
                }
                if (threadIdx.x == 0) {
                    int ctl = 0, st = 0;
                    const cdw gk = {gg[0], gg[1]}, dk = {gg[2], gg[3]};
                    const float rr = gg[4].h;
                    if (!isfinite(rr) || !isfinite(gk.x.h) || !isfinite(gk.y.h) || !isfinite(dk.x.h) || !isfinite(dk.y.h)) {
                        ctl = 2;
                        st = DD_NLS_ENONFINITE;
                    } else if (rr <= target2) {
                        ctl = 1;          // x was advanced in this pass; the solution is complete
                    } else {
                        // a breakdown of the recurrences after the first step, or 32 steps without a
                        // 1% gain in ||r||, ends the inner solve with the x reached (ctl 3)
                        if (rr < 0.9801f * best2) {
                            best2 = rr;
                            since = 0;
                        } else if (++since >= 32) {
                            ctl = 3;
                        }
                        if (!ctl && !cdw_nonzero(gam)) ctl = 3;
                        if (!ctl) {
                            // beta_{k+1} = gamma_{k+1}/gamma_k and
                            // alpha_{k+1} = gamma_{k+1}/(delta_{k+1} - beta_{k+1} gamma_{k+1}/alpha_k),
                            // the latter as gamma_{k+1}/(delta_{k+1} - gamma_{k+1}^2 q_k): two
                            // independent reciprocals per step instead of three chained quotients
                            const cdw g2 = cdw_mul(gk, gk);
                            const cdw den = cdw_sub(dk, cdw_mul(g2, qk));
                            if (!cdw_finite(den) || !cdw_finite(g2)) {
                                ctl = 2;
                                st = DD_NLS_ENONFINITE;
                            } else if (!cdw_nonzero(den) || !cdw_nonzero(g2)) {
                                ctl = 3;
                            } else {
                                const cdw r1 = cdw_recip(den), r2 = cdw_recip(g2);
                                be = cdw_mul(gk, ig);
                                al = cdw_mul(gk, r1);
                                qk = cdw_mul(den, r2);
                                ig = cdw_mul(gk, r2);
                                gam = gk;
                            }
                        }
                    }
                    s_ctl[0] = ctl;
                    s_ctl[1] = st;
                    s_sc[0] = al.x.h;
                    s_sc[1] = al.y.h;
                    s_sc[2] = be.x.h;
                    s_sc[3] = be.y.h;
                }
                __syncthreads();
                lap(4);
                ++kry;
                if (s_ctl[0]) {
                    if (s_ctl[0] == 2) cstat = s_ctl[1];
                    if (s_ctl[0] == 3) use_sr = false;   // keep x; two-reduction loop from now on
                    break;
                }
                alT = T2{s_sc[0], s_sc[1]};
                beT = T2{s_sc[2], s_sc[3]};
            }
            // x of the slab back to global memory, then every CTA sees the whole correction
#pragma unroll
            for (int k = 0; k < kOnChipNPT; ++k) {
                const int mm = threadIdx.x + k * BS;
                if (mm >= M) continue;
                int ix, il;
                split_node(mm, h, inv_h, ix, il);
                x[(long long)ix * P + y0 + il] = xreg[k];
            }
            if (cstat) { status = cstat; break; }
            if (!strip_barrier()) { status = DD_NLS_ETIMEOUT; break; }
            }
        } else if (use_sr) {
            // Single-reduction COCG (the Chronopoulos-Gear arrangement of CG with the unconjugated
            // bilinear form): s = A p is carried, w = A z is formed in the same pass as the updates
            // with z_{k+1} rebuilt at the stencil neighbours, so one reduction (gamma = r^T z,
            // delta = w^T z, ||r||^2) and one barrier per iteration.
            // w_0 = A z_0, delta_0 = w_0^T z_0
            T d0r = 0, d0i = 0;
            const T2 zeroT = mk<T2>(0.0, 0.0);
            for (int n = it_first(Ns); n < it_end(Ns); n += it_step) {
                int ix, iy;
                split_node(n, nyn, inv_nyn, ix, iy);
                const long long idx = (long long)ix * P + iy;
                const Coef1<T> cxT = coef1<T>(ix, c, KXt), cyT = coef1<T>(iy, ny, KYt);
                T rre, rim;
                rho_atT(ix, rre, rim);
                T2 zo;
                // z_0 = D^-1 r_0 (the rebuild with alpha = beta = 0 reads r only)
                const T2 w0 = apply_op_znext<T, T2>(rbuf[0], rbuf[0], rbuf[0], dv, idx, ix, iy, c, ny, P, cxT, cyT, alphaT,
                                                    rre, rim, cT[idx], zeroT, zeroT, zo);
                wbuf[0][idx] = w0;
                // the residual pass leaves these to the strips that correct: x = p = s_{-1} = 0
                x[idx] = zeroT;
                p[idx] = zeroT;
                sbuf[1][idx] = zeroT;
                d0r += w0.x * zo.x - w0.y * zo.y;
                d0i += w0.x * zo.y + w0.y * zo.x;
            }
            {
                T lT[2] = {d0r, d0i};
                double l2[2];
                block_sum_t<T, 2>(lT, l2, s_red);
                if (threadIdx.x == 0) { double* sp = slot_ptr(epoch + 1); sp[0] = l2[0]; sp[1] = l2[1]; sp[2] = 0; sp[3] = 0; }
            }
            ++epoch;
            lap(1);
            if (!gbar(epoch * bps)) { status = DD_NLS_ETIMEOUT; break; }
            // thread-0 state of the recurrences
            double gam_r = rho_r, gam_i = rho_i, al_r = 0.0, al_i = 0.0, be_r = 0.0, be_i = 0.0;
            double best = INFINITY;     // stagnation guard: least ||r|| so far, iterations since
            int since = 0;
            if (threadIdx.x < 32) {
                double dl[4];
                group_sum_w0<4>(group_ptr(epoch), bps, dl);
                if (threadIdx.x == 0) {
                    const double del_r = dl[0], del_i = dl[1];
                    const double dd2 = del_r * del_r + del_i * del_i;
                    int ctl = 0, st = 0;
                    if (!(dd2 > 0.0) || !isfinite(dd2)) {
                        ctl = 2;
                        st = isfinite(dd2) ? DD_NLS_EBREAKDOWN : DD_NLS_ENONFINITE;
                    } else {
                        al_r = (gam_r * del_r + gam_i * del_i) / dd2;
                        al_i = (gam_i * del_r - gam_r * del_i) / dd2;
                    }
                    s_ctl[0] = ctl;
                    s_ctl[1] = st;
                    s_sc[0] = (T)al_r;
                    s_sc[1] = (T)al_i;
                }
            }
            __syncthreads();
            lap(4);
            if (s_ctl[0]) { status = s_ctl[1]; break; }
            T2 alT = T2{s_sc[0], s_sc[1]}, beT = T2{0, 0};
            for (int it = 0; it < a.max_inner; ++it) {
                const int cur = it & 1, nxt = cur ^ 1;
                const T2* rc = rbuf[cur];
                const T2* wc = wbuf[cur];
                const T2* sp = sbuf[nxt];          // s_{k-1}
                T2* so = sbuf[cur];                // s_k
                T2* rn_b = rbuf[nxt];
                T2* wn_b = wbuf[nxt];
                T g_r = 0, g_i = 0, dlt_r = 0, dlt_i = 0, rr2 = 0;
                for (int n = it_first(Ns); n < it_end(Ns); n += it_step) {
                    int ix, iy;
                    split_node(n, nyn, inv_nyn, ix, iy);
                    const long long idx = (long long)ix * P + iy;
                    const Coef1<T> cxT = coef1<T>(ix, c, KXt), cyT = coef1<T>(iy, ny, KYt);
                    const T2 zc = cmul(dv[idx], rc[idx]);
                    const T2 pn = cfma(beT, p[idx], zc);           // p_k = z_k + beta p_{k-1}
                    const T2 sn = cfma(beT, sp[idx], wc[idx]);     // s_k = w_k + beta s_{k-1}
                    x[idx] = cfma(alT, pn, x[idx]);
                    p[idx] = pn;
                    so[idx] = sn;
                    T2 rnew = rc[idx];
                    rnew.x -= alT.x * sn.x - alT.y * sn.y;
                    rnew.y -= alT.x * sn.y + alT.y * sn.x;
                    rn_b[idx] = rnew;
                    T rre, rim;
                    rho_atT(ix, rre, rim);
                    T2 zo;
                    const T2 wn = apply_op_znext<T, T2>(rc, wc, sp, dv, idx, ix, iy, c, ny, P, cxT, cyT, alphaT, rre, rim,
                                                        cT[idx], alT, beT, zo);
                    wn_b[idx] = wn;
                    g_r += rnew.x * zo.x - rnew.y * zo.y;
                    g_i += rnew.x * zo.y + rnew.y * zo.x;
                    dlt_r += wn.x * zo.x - wn.y * zo.y;
                    dlt_i += wn.x * zo.y + wn.y * zo.x;
                    rr2 += rnew.x * rnew.x + rnew.y * rnew.y;
                }
                T lT[4] = {g_r, g_i, dlt_r, dlt_i};
                double l4[4];
                block_sum_t<T, 4>(lT, l4, s_red);
                T lr[1] = {rr2};
                double l1[1];
                block_sum_t<T, 1>(lr, l1, s_red);
                if (threadIdx.x == 0) {
                    double* spp = slot_ptr(epoch + 1);
                    spp[0] = l4[0]; spp[1] = l4[1]; spp[2] = l4[2]; spp[3] = l4[3];
                    // ||r||^2 travels in the other half of the slot ring (slot epoch+3, unused now)
                    slot_ptr(epoch + 3)[0] = l1[0];
                }
                ++epoch;
                lap(2);
                if (!gbar(epoch * bps)) { status = DD_NLS_ETIMEOUT; break; }
                if (threadIdx.x < 32) {
                    double gg[4], rq[1];
                    group_sum_w0<4>(group_ptr(epoch), bps, gg);
                    group_sum_w0<1>(group_ptr(epoch + 2), bps, rq);
                    if (threadIdx.x == 0) {
                        int ctl = 0, st = 0;
                        const double rk = sqrt(rq[0]);
                        if (!isfinite(rq[0]) || !isfinite(gg[0]) || !isfinite(gg[2])) {
                            ctl = 2;
                            st = DD_NLS_ENONFINITE;
                        } else if (rk <= target) {
                            ctl = 1;          // x was advanced in this pass; the solution is complete
                        } else {
                            // A breakdown of the recurrences after the first step, or 32 steps
                            // without a 1% gain, ends the inner solve with the x reached: the
                            // nonlinear loop recomputes the exact residual and continues with the
                            // two-reduction loop (ctl 3).
                            if (rk < 0.99 * best) {
                                best = rk;
                                since = 0;
                            } else if (++since >= 32) {
                                ctl = 3;
                            }
                            // beta_{k+1} = gamma_{k+1}/gamma_k,
                            // alpha_{k+1} = gamma_{k+1}/(delta_{k+1} - beta_{k+1} gamma_{k+1}/alpha_k)
                            const double gk2 = gam_r * gam_r + gam_i * gam_i;
                            if (!ctl && !(gk2 > 0.0)) ctl = 3;
                            if (!ctl) {
                                const double nb_r = (gg[0] * gam_r + gg[1] * gam_i) / gk2;
                                const double nb_i = (gg[1] * gam_r - gg[0] * gam_i) / gk2;
                                const double a2 = al_r * al_r + al_i * al_i;
                                const double bg_r = nb_r * gg[0] - nb_i * gg[1], bg_i = nb_r * gg[1] + nb_i * gg[0];
                                const double t_r = (bg_r * al_r + bg_i * al_i) / a2, t_i = (bg_i * al_r - bg_r * al_i) / a2;
                                const double den_r = gg[2] - t_r, den_i = gg[3] - t_i;
                                const double den2 = den_r * den_r + den_i * den_i;
                                if (!isfinite(den2)) {
                                    ctl = 2;
                                    st = DD_NLS_ENONFINITE;
                                } else if (!(den2 > 0.0)) {
                                    ctl = 3;
                                } else {
                                    al_r = (gg[0] * den_r + gg[1] * den_i) / den2;
                                    al_i = (gg[1] * den_r - gg[0] * den_i) / den2;
                                    be_r = nb_r;
                                    be_i = nb_i;
                                    gam_r = gg[0];
                                    gam_i = gg[1];
                                }
                            }
                        }
                        s_ctl[0] = ctl;
                        s_ctl[1] = st;
                        s_sc[0] = (T)al_r;
                        s_sc[1] = (T)al_i;
                        s_sc[2] = (T)be_r;
                        s_sc[3] = (T)be_i;
                    }
                }
                __syncthreads();
                lap(4);
                ++kry;
                if (s_ctl[0]) {
                    if (s_ctl[0] == 2) status = s_ctl[1];
                    if (s_ctl[0] == 3) use_sr = false;   // keep x; two-reduction loop from now on
                    break;
                }
                alT = T2{s_sc[0], s_sc[1]};
                beT = T2{s_sc[2], s_sc[3]};
            }
        } else {
        T2 bT = T2{0, 0};
        for (int it = 0; it < a.max_inner; ++it) {
            // phase A: q = A z + beta q, p = z + beta p, partial mu = p^T q
            // (per-thread partials in T: the FP64 pipe is ~1/64 of FP32 on this part)
            T am_re = 0, am_im = 0;
            for (int n = it_first(Nall); n < it_end(Nall); n += it_step) {
                if (!PADE || n < Ns) {
                    int ix, iy;
                    split_node(n, nyn, inv_nyn, ix, iy);
                    const long long idx = (long long)ix * P + iy;
                    const Coef1<T> cxT = coef1<T>(ix, c, KXt), cyT = coef1<T>(iy, ny, KYt);
                    T rre, rim;
                    rho_atT(ix, rre, rim);
                    T2 Az = apply_op<T, T2>(z, idx, ix, iy, c, ny, P, cxT, cyT, alphaT, rre, rim, cT[idx]);
                    if (PADE) {
                        const int e = tc_edge(ix);
                        if (e >= 0)
                            for (int s2 = 0; s2 < m; ++s2) {
                                const T2 mph = edge_mass<T, T2>(zf + ((long long)e * m + s2) * P, iy, ny, cyT);
                                Az = csub(Az, cmul(s_psig[s2], mph));
                            }
                    }
                    const T2 qn = cfma(bT, q[idx], Az);
                    const T2 pn = cfma(bT, p[idx], z[idx]);
                    q[idx] = qn;
                    p[idx] = pn;
                    am_re += pn.x * qn.x - pn.y * qn.y;
                    am_im += pn.x * qn.y + pn.y * qn.x;
                } else {
                    int e, s2, iy;
                    split_phi(n, e, s2, iy);
                    if (!(e == 0 ? ltc : rtc)) continue;
                    const int ixe = e == 0 ? 0 : c;
                    const long long fi = ((long long)e * m + s2) * P + iy;
                    const Coef1<T> cyT = coef1<T>(iy, ny, KYt);
                    const T2 J = phi_row<T, T2>(z + (long long)ixe * P, zf + ((long long)e * m + s2) * P, iy, ny, cyT,
                                                s_pgam[s2], s_psig[s2], cTf[(long long)e * P + iy]);
                    const T2 qn = cfma(bT, qf[fi], J);
                    const T2 pn = cfma(bT, pf[fi], zf[fi]);
                    qf[fi] = qn;
                    pf[fi] = pn;
                    am_re += pn.x * qn.x - pn.y * qn.y;
                    am_im += pn.x * qn.y + pn.y * qn.x;
                }
            }
            T lmT[2] = {am_re, am_im};
            double lm[2];
            block_sum_t<T, 2>(lmT, lm, s_red);
            lap(1);
            double mu[4];
            if constexpr (CLU) {
                const double lm4[4] = {lm[0], lm[1], 0.0, 0.0};
                if (!strip_sum4(lm4, mu)) { status = DD_NLS_ETIMEOUT; break; }
            } else {
                if (threadIdx.x == 0) { double* sp = slot_ptr(epoch + 1); sp[0] = lm[0]; sp[1] = lm[1]; sp[2] = 0; sp[3] = 0; }
                ++epoch;
                if (!gbar(epoch * bps)) { status = DD_NLS_ETIMEOUT; break; }
                if (threadIdx.x < 32) group_sum_w0<4>(group_ptr(epoch), bps, mu);
            }
            if (threadIdx.x < 32) {
                if (threadIdx.x == 0) {
                    const double mu2 = mu[0] * mu[0] + mu[1] * mu[1];
                    int ctl = 0, st = 0;
                    if (!(mu2 > 0.0) || !isfinite(mu2)) {
                        ctl = 2;
                        st = isfinite(mu2) ? DD_NLS_EBREAKDOWN : DD_NLS_ENONFINITE;
                    }
                    // a = rho / mu
                    s_ctl[0] = ctl;
                    s_ctl[1] = st;
                    s_sc[0] = (T)((rho_r * mu[0] + rho_i * mu[1]) / mu2);
                    s_sc[1] = (T)((rho_i * mu[0] - rho_r * mu[1]) / mu2);
                }
            }
            __syncthreads();
            lap(4);
            if (s_ctl[0]) { status = s_ctl[1]; break; }
            const T2 alT = T2{s_sc[0], s_sc[1]};
            const T2 malT = T2{-s_sc[0], -s_sc[1]};
            // phase B: x += a p, r -= a q, z = D^-1 r, partials rho' = r^T z, ||r||^2
            T b0s = 0, b1s = 0, b2s = 0;
            for (int n = it_first(Nall); n < it_end(Nall); n += it_step) {
                T2 rn, zn;
                if (!PADE || n < Ns) {
                    int ix, iy;
                    split_node(n, nyn, inv_nyn, ix, iy);
                    const long long idx = (long long)ix * P + iy;
                    const Coef1<T> cxT = coef1<T>(ix, c, KXt), cyT = coef1<T>(iy, ny, KYt);
                    const T2 pc = p[idx];
                    x[idx] = cfma(alT, pc, x[idx]);
                    rn = cfma(malT, q[idx], r[idx]);
                    r[idx] = rn;
                    T rre, rim;
                    rho_atT(ix, rre, rim);
                    const T2 di = diag_inv<T>(cxT, cyT, alphaT, rre, rim, cT[idx]);
                    zn = cmul(di, rn);
                    z[idx] = zn;
                } else {
                    int e, s2, iy;
                    split_phi(n, e, s2, iy);
                    if (!(e == 0 ? ltc : rtc)) continue;
                    const long long fi = ((long long)e * m + s2) * P + iy;
                    const Coef1<T> cyT = coef1<T>(iy, ny, KYt);
                    xf[fi] = cfma(alT, pf[fi], xf[fi]);
                    rn = cfma(malT, qf[fi], rf[fi]);
                    rf[fi] = rn;
                    const T2 di = phi_diag_inv<T, T2>(cyT, s_pgam[s2], s_psig[s2], cTf[(long long)e * P + iy]);
                    zn = cmul(di, rn);
                    zf[fi] = zn;
                }
                b0s += rn.x * zn.x - rn.y * zn.y;
                b1s += rn.x * zn.y + rn.y * zn.x;
                b2s += rn.x * rn.x + rn.y * rn.y;
            }
            T lbT[3] = {b0s, b1s, b2s};
            double lb[3];
            block_sum_t<T, 3>(lbT, lb, s_red);
            lap(2);
            double rb[4];
            if constexpr (CLU) {
                const double lb4[4] = {lb[0], lb[1], lb[2], 0.0};
                if (!strip_sum4(lb4, rb)) { status = DD_NLS_ETIMEOUT; break; }
            } else {
                if (threadIdx.x == 0) { double* sp = slot_ptr(epoch + 1); sp[0] = lb[0]; sp[1] = lb[1]; sp[2] = lb[2]; sp[3] = 0; }
                ++epoch;
                if (!gbar(epoch * bps)) { status = DD_NLS_ETIMEOUT; break; }
                if (threadIdx.x < 32) group_sum_w0<4>(group_ptr(epoch), bps, rb);
            }
            if (threadIdx.x < 32) {
                if (threadIdx.x == 0) {
                    int ctl = 0, st = 0;
                    const double rr2 = rho_r * rho_r + rho_i * rho_i;
                    if (!isfinite(rb[2])) {
                        ctl = 2;
                        st = DD_NLS_ENONFINITE;
                    } else if (sqrt(rb[2]) <= target) {
                        ctl = 1;
                    } else if (!(rr2 > 0.0)) {
                        ctl = 2;
                        st = DD_NLS_EBREAKDOWN;
                    } else {
                        const double b_re = (rb[0] * rho_r + rb[1] * rho_i) / rr2;
                        const double b_im = (rb[1] * rho_r - rb[0] * rho_i) / rr2;
                        rho_r = rb[0];
                        rho_i = rb[1];
                        s_sc[2] = (T)b_re;
                        s_sc[3] = (T)b_im;
                    }
                    s_ctl[0] = ctl;
                    s_ctl[1] = st;
                }
            }
            __syncthreads();
            lap(4);
            ++kry;
            if (s_ctl[0]) {
                if (s_ctl[0] == 2) status = s_ctl[1];
                break;
            }
            bT = T2{s_sc[2], s_sc[3]};
        }
        }
        if (status) break;
        // ---------------- zeta += delta (FP64), then every block must see the new zeta
        // thread 0: the correction's scale sc = omega / inv_s and the next correction's inv_s
        if (threadIdx.x == 0) {
            const double sc0 = omega / inv_s;
            const dw scd0 = dw_from(sc0);
            s_nld[1] = sc0;
            s_nlf[2] = scd0.h;
            s_nlf[3] = scd0.l;
            inv_s = 1.0 / rnorm0;
            s_nld[0] = inv_s;
            s_nlf[0] = (float)fmin(inv_s, 1e30);
        }
        __syncthreads();
        const double sc = s_nld[1];
        if (DW && dwr) {
            // double-word zeta and the correction accumulated over the launch
            const dw scd = {s_nlf[2], s_nlf[3]};
            for (int n = it_first(Ns); n < it_end(Ns); n += it_step) {
                int ix, iy;
                split_node(n, nyn, inv_nyn, ix, iy);
                const long long idx = (long long)ix * P + iy;
                const T2 dx = x[idx];
                const cdw cc = {dw_mul_f(scd, dx.x), dw_mul_f(scd, dx.y)};
                cdw_st(zdw + idx, cdw_add(cdw_ld(zdw + idx), cc));
                if (a.dw_mode == 0) cdw_st(ddw + idx, cdw_add(cdw_ld(ddw + idx), cc));
            }
            if constexpr (PADE) {
                // the phi unknowns stay FP64
                for (int n = it_first(Nall); n < it_end(Nall); n += it_step) {
                    if (n < Ns) continue;
                    int e, s2, iy;
                    split_phi(n, e, s2, iy);
                    if (!(e == 0 ? ltc : rtc)) continue;
                    const long long fi = ((long long)e * m + s2) * P + iy;
                    const double2 dx = cd(xf[fi]);
                    phi[fi] = make_double2(phi[fi].x + sc * dx.x, phi[fi].y + sc * dx.y);
                }
            }
        } else
        for (int n = it_first(Nall); n < it_end(Nall); n += it_step) {
            if (!PADE || n < Ns) {
                int ix, iy;
                split_node(n, nyn, inv_nyn, ix, iy);
                const long long idx = (long long)ix * P + iy;
                const double2 dx = cd(x[idx]);
                zeta[idx] = make_double2(zeta[idx].x + sc * dx.x, zeta[idx].y + sc * dx.y);
            } else {
                int e, s2, iy;
                split_phi(n, e, s2, iy);
                if (!(e == 0 ? ltc : rtc)) continue;
                const long long fi = ((long long)e * m + s2) * P + iy;
                const double2 dx = cd(xf[fi]);
                phi[fi] = make_double2(phi[fi].x + sc * dx.x, phi[fi].y + sc * dx.y);
            }
        }
        inv_s = s_nld[0];              // scale of the next correction
        inv_sf = s_nlf[0];
        lap(3);
        if (!strip_barrier()) { status = DD_NLS_ETIMEOUT; break; }
        lap(4);
    }
    if (DW && dwr && a.dw_mode != 0) {
        // the double-word fields stay the state; the trace exchange reads the edge columns
        for (int t = rank * blockDim.x + threadIdx.x; t < 2 * nyn; t += bps * blockDim.x) {
            const int ix = t < nyn ? 0 : c, iy = t < nyn ? t : t - nyn;
            const long long idx = (long long)ix * P + iy;
            const cdw zv = cdw_ld(zdw + idx);
            zeta[idx] = make_double2(dw_to(zv.x), dw_to(zv.y));
        }
    } else if (DW && dwr) {
        // zeta (FP64) += the launch's accumulated correction, own nodes only
        for (int n = it_first(Ns); n < it_end(Ns); n += it_step) {
            int ix, iy;
            split_node(n, nyn, inv_nyn, ix, iy);
            const long long idx = (long long)ix * P + iy;
            const cdw d = cdw_ld(ddw + idx);
            const double2 zv = zeta[idx];
            zeta[idx] = make_double2(zv.x + dw_to(d.x), zv.y + dw_to(d.y));
        }
    }
    if (a.pcyc && threadIdx.x == 0)
        for (int k = 0; k < 5; ++k) a.pcyc[(size_t)blockIdx.x * 8 + k] = cyc[k];
    if (rank == 0 && threadIdx.x == 0) {
        a.status[j] = status;
        a.nl_its[j] = nl_it;
        a.kry_its[j] = kry;
        a.nl_res[j] = nres;
    }
    // no CTA leaves while another may still read its shared memory or push into it
    if constexpr (CLU) cluster_sync_all();
}

void fill_fp32_constants(StripSolveArgs& a, double rho_re, double rho_im, double hy) {
    a.rho_f[0] = (float)rho_re;
    a.rho_f[1] = (float)rho_im;
    const double v[2] = {rho_re * hy / 6.0, rho_im * hy / 6.0};
    for (int i = 0; i < 2; ++i) {
        a.dwrho[2 * i] = (float)v[i];
        a.dwrho[2 * i + 1] = (float)(v[i] - (double)a.dwrho[2 * i]);
    }
}

unsigned strip_cluster_smem(int nxs, int nyn) {
    const long long H = (nyn + kClusterCTAs - 1) / kClusterCTAs;
    if ((long long)nxs * H > 512LL * kOnChipNPT) return 0;
    const long long bytes = 8LL * nxs * (H + 2) + 4 * 8LL * nxs * H + 16 * 8LL * nxs + 4LL * nxs * H;
    return bytes <= 200 * 1024 ? (unsigned)bytes : 0u;
}

// Cluster kernels: opt in to 16-CTA clusters and to the dynamic shared memory they need.
static void* cluster_kernel(bool dw) {
    return dw ? (void*)strip_solve_kernel<float, false, 512, true, true>
              : (void*)strip_solve_kernel<float, false, 512, false, true>;
}
static cudaError_t cluster_prepare(bool dw, unsigned smem) {
    const void* k = cluster_kernel(dw);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e;
}
static void cluster_config(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* at, int nstrips, unsigned smem, cudaStream_t s) {
    cfg = cudaLaunchConfig_t{};
    cfg.gridDim = dim3(nstrips * kClusterCTAs);
    cfg.blockDim = dim3(512);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kClusterCTAs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
}
int strip_cluster_capacity(bool dw, unsigned smem) {
    if (smem == 0 || cluster_prepare(dw, smem) != cudaSuccess) { cudaGetLastError(); return 0; }
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[1];
    cluster_config(cfg, at, 1, smem, nullptr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, cluster_kernel(dw), &cfg) != cudaSuccess) { cudaGetLastError(); return 0; }
    return n;
}

template <typename T>
static cudaError_t launch_strip_solve_t(const StripSolveArgs& args, int nblocks, int bs, cudaStream_t s) {
    StripSolveArgs a = args;
    void* params[] = {&a};
    dim3 grid(nblocks), block(bs);
    count_launches(1);
    if (sizeof(T) == 4 && a.cluster && a.mode == 0 && a.pade_m == 0 && !a.geoms && !a.sinfo) {
        // nblocks = strips: one cluster per strip, clusters independent (no cooperative launch)
        const bool dw = a.zdw != nullptr;
        cudaError_t e = cluster_prepare(dw, a.cluster_smem);
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg;
        cudaLaunchAttribute at[1];
        cluster_config(cfg, at, nblocks, a.cluster_smem, s);
        return dw ? cudaLaunchKernelEx(&cfg, strip_solve_kernel<float, false, 512, true, true>, a)
                  : cudaLaunchKernelEx(&cfg, strip_solve_kernel<float, false, 512, false, true>, a);
    }
    if (a.pade_m > 0) {
        if (a.geoms || a.sinfo) return cudaErrorInvalidValue;   // S_pade strips are never batched
        if (sizeof(T) == 4 && a.zdw && a.mode == 0)
            return cudaLaunchCooperativeKernel((const void*)strip_solve_kernel<float, true, 256, true>, grid, dim3(256), params, 0, s);
        return cudaLaunchCooperativeKernel((const void*)strip_solve_kernel<T, true, 256>, grid, dim3(256), params, 0, s);
    }
    if (sizeof(T) == 4 && a.zdw && a.mode == 0)
        return cudaLaunchCooperativeKernel((const void*)strip_solve_kernel<float, false, 256, true>, grid, dim3(256), params, 0, s);
    if (bs == 128)
        return cudaLaunchCooperativeKernel((const void*)strip_solve_kernel<T, false, 128>, grid, block, params, 0, s);
    return cudaLaunchCooperativeKernel((const void*)strip_solve_kernel<T, false, 256>, grid, dim3(256), params, 0, s);
}

cudaError_t launch_strip_solve(const StripSolveArgs& a, int nblocks, bool fp32, cudaStream_t s, int block_size) {
    return fp32 ? launch_strip_solve_t<float>(a, nblocks, block_size, s)
                : launch_strip_solve_t<double>(a, nblocks, block_size, s);
}

__global__ void dw_to_zeta_kernel(Geom g, const float4* __restrict__ zdw, double2* __restrict__ zeta) {
    const long long total = (long long)g.N * g.sstride();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        if ((int)(i % g.P) >= g.nyn) continue;
        const cdw v = cdw_ld(zdw + i);
        zeta[i] = make_double2(dw_to(v.x), dw_to(v.y));
    }
}
cudaError_t launch_dw_to_zeta(const Geom& g, const float4* zdw, double2* zeta, cudaStream_t s) {
    count_launches(1);
    const long long total = (long long)g.N * g.sstride();
    const int nb = (int)std::min<long long>((total + 255) / 256, 152LL * 8);
    dw_to_zeta_kernel<<<nb, 256, 0, s>>>(g, zdw, zeta);
    return cudaGetLastError();
}

int strip_solve_max_blocks_bs(bool fp32, int bs) {
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (bs == 128) {
        if (fp32) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, strip_solve_kernel<float, false, 128>, 128, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, strip_solve_kernel<double, false, 128>, 128, 0);
        return per * nsm;
    }
    return strip_solve_max_blocks(fp32);
}

int strip_solve_max_blocks(bool fp32) {
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // the smaller of the Robin and S_pade instances, so one schedule fits both
    int per2 = 0, per3 = 0;
    if (fp32) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, strip_solve_kernel<float, false, 256>, 256, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, strip_solve_kernel<float, true, 256>, 256, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per3, strip_solve_kernel<float, false, 256, true>, 256, 0);
        per2 = std::min(per2, per3);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per3, strip_solve_kernel<float, true, 256, true>, 256, 0);
        per2 = std::min(per2, per3);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, strip_solve_kernel<double, false, 256>, 256, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, strip_solve_kernel<double, true, 256>, 256, 0);
    }
    return std::min(per, per2) * nsm;
}

}  // namespace ddnls
