// Internal launch interface between the host runtime (api.cu) and the kernels.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace ddnls {

// Error text returned by dd_nls_last_error(NULL) (api.cu).
void set_handle_free_error(const char* msg);

// Kernels launched by this library since load (every launch_* wrapper adds its count).
long long kernel_launch_count();
void count_launches(int n);

constexpr int kMaxPade = 96;   // largest Pade order m of eq. (TCS) the kernels take

struct StripSolveArgs;
// Fill the FP32 edge coefficient of a strip-solver launch: rho = rho_re + i rho_im on a mesh of
// y spacing hy.
void fill_fp32_constants(StripSolveArgs& a, double rho_re, double rho_im, double hy);

// Batched instances: strip j of the launch belongs to instance `inst` (its own geometry),
// is strip `jloc` of that instance, and its fields start at element `off` of the field arrays;
// the instance's interface vector starts at element `goff` of gtr.
struct StripInfo {
    int inst, jloc;
    long long off, goff;
};

struct StripSolveArgs {
    Geom g;
    const Geom* geoms;       // batched: [instances] geometry, else NULL (use g)
    const StripInfo* sinfo;  // batched: [strips] descriptors, else NULL
    int bps;                 // unused when blk_strip is set
    const int* blk_strip;    // [gridDim] strip of each block
    const int* blk_start;    // [strips+1] first block of each strip
    const double* bnorm0;    // [strips] ||(2i/dt) M h|| per strip (scale of the first correction), or NULL
    int mode;                // 0: Schwarz strips; 1: unit data on free strips (L_h setup)
    int unit_base;           // mode 1: first unit column (side*nyn + pos) of this launch
    int unit_ltc, unit_rtc;  // mode 1: edge kinds of the strip type
    double2* zeta;           // FP64 strip fields, in/out
    const double2* rhs0;     // (2i/dt) M h per strip, or NULL (zero)
    const double* Wn;        // V/lap per strip node, or NULL (zero)
    const double2* gtr;      // interface traces [2(N-1)][P]
    void *x, *r, *z, *p, *q; // inner Krylov vectors (float2 or double2)
    void *w1, *s0, *s1, *dv; // single-reduction COCG (Robin): second w buffer, s ping-pong, D^-1
    // double-word residual (FP32 Robin, mode 0), all NULL otherwise: zeta and its accumulated
    // correction (float4 {re.h, re.l, im.h, im.l} per node), the right side b, w W (float2)
    float4 *zdw, *ddw, *bdw;
    float2* wdw;
    // 0: zeta (FP64) is the state: set up the double-word fields from it and add the launch's
    //    correction back at the end.  1: first launch of a step whose strip tolerances stay at
    //    or above kDWFinish: full set-up, then the double-word fields are the state and only
    //    the edge columns of zeta (what the trace exchange reads) are written back.
    //    2: later such launches: only the edge columns of b are refreshed.
    int dw_mode;
    double* bint2;           // [strips] ||b||^2 off the edge columns (set in mode 1, read in 2)
    void* cT;                // c = w (W + kappa|zeta|^2) in inner precision
    double nl_tol, inner_tol, inner_floor;
    const double* nl_tol_strip;   // batched: per-strip nonlinear tolerance (device), or NULL
    const double* bscale;    // ||(2i/dt) M u_{n-1}|| over all strips, one per instance (device), or NULL
    double nl_floor_frac;    // strips stop once ||res|| <= nl_floor_frac * (*bscale)
    int max_nl, max_inner;
    double nl_relax;         // first relaxation factor of the fixed point (adaptive below it)
    int nl_picard;           // 1: corrections with the fixed point's operator; 0: Jacobian diagonal
    double* part;            // [4][gridDim][4] partial sums
    unsigned* bar;           // [strips] barrier counters, zeroed before the launch
    int* status;             // [strips]
    int* nl_its;             // [strips]
    long long* kry_its;      // [strips]
    double* nl_res;          // [strips]
    int* err;                // launch-wide error word
    unsigned long long wait_ns;   // bound of every device-side wait (0: two seconds)
    int test_skip_arrival;   // > 0: block test_skip_arrival - 1 skips its first barrier arrival (tests
                             // of the time-out path); 0 otherwise
    // cluster mode (FP32 Robin, mode 0): one strip per cluster of kClusterCTAs CTAs of 512 threads,
    // blk_strip[c] = strip of cluster c, cluster_smem bytes of dynamic shared memory per CTA
    int cluster;
    unsigned cluster_smem;
    // the S_pade edge coefficient i sum a_s (re, im) rounded to FP32 on the host, and rho hy/6 in
    // double words (re hi, re lo, im hi, im lo) for the double-word residual
    float rho_f[2];
    float dwrho[4];
    long long* pcyc;         // [gridDim][8] phase cycles (R, A, B, epilogue, waits) or NULL
    // S_pade^m transmission (eq. TCS): auxiliary unknowns phi_{e,s} on both vertical edges
    int pade_m;              // 0: Robin
    double2* phi;            // [strips][2][m][P] FP64 state
    void *xf, *rf, *zf, *pf, *qf;   // their inner Krylov vectors
    void* cTf;               // [strips][2][P] w_y (W + kappa|zeta|^2) on each edge, inner precision
    double2 pade_a[kMaxPade], pade_d[kMaxPade];
};

// cooperative launch of nblocks blocks (a.blk_strip / a.blk_start map blocks to strips)
cudaError_t launch_strip_solve(const StripSolveArgs& a, int nblocks, bool fp32, cudaStream_t s, int block_size = 256);
// zeta = the double-word state, every strip node (ends a step run with dw_mode 1/2)
cudaError_t launch_dw_to_zeta(const Geom& g, const float4* zdw, double2* zeta, cudaStream_t s);
// The double-word residual resolves about 1e-14 of ||b||: a strip tolerance below this needs the
// FP64 finish, i.e. dw_mode 0.
constexpr double kDWFinish = 1e-12;
int strip_solve_max_blocks(bool fp32);
// Cluster mode: dynamic shared memory of one CTA for a strip of nxs x nyn nodes, 0 when the strip's
// slab does not fit on chip; clusters that can be resident at once (0: cluster mode unavailable).
unsigned strip_cluster_smem(int nxs, int nyn);
int strip_cluster_capacity(bool dw, unsigned smem);
int strip_solve_max_blocks_bs(bool fp32, int block_size);   // Robin kernel with 128 or 256 threads

// ---- auxiliary kernels (aux_kernels.cu)
using AuxGeom = Geom;

// nodal (ny+1)x(nx+1) x-fastest  <->  strip layout
cudaError_t launch_scatter_u(const AuxGeom& g, const double2* glob, double2* strips, cudaStream_t s);
cudaError_t launch_gather_u(const AuxGeom& g, const double2* strips, double2* glob, cudaStream_t s);
cudaError_t launch_scatter_real(const AuxGeom& g, const double* glob, double scale, double* strips, cudaStream_t s);
// out[j] = ||rhs0|| over strip j (one block per strip)
// ||rhs0|| per strip; part: scratch of part_cap doubles (at least N)
cudaError_t launch_strip_norms(const AuxGeom& g, const double2* rhs0, double* out, double* part, int part_cap,
                               cudaStream_t s);
// rhs0 = i alpha M h (per strip); partial sums of ||rhs0||^2 into part[nblk][1]
cudaError_t launch_rhs0(const AuxGeom& g, const double2* h, double2* rhs0, double* part, int* nblk_out, cudaStream_t s);
// interface flux update, eq. (fluxlr): writes gnew, partial norms into part[nblk][2].
// Robin when pade_m == 0, else S v = -i sum a_s v + i sum a_s d_s phi_s (eq. TCSdist).
cudaError_t launch_traces(const AuxGeom& g, const double2* zeta, const double2* gtr, double2* gnew,
                          double* part, int* nblk_out, cudaStream_t s, int pade_m = 0,
                          const double2* phi = nullptr, const double2* pa = nullptr, const double2* pd = nullptr);
// v[0] = sqrt(v[0]) on the device
cudaError_t launch_sqrt(double* v, cudaStream_t s);
// sum part[nblk][k] (k < nv) in fixed order into out[k]
cudaError_t launch_finalize(const double* part, int nblk, int nv, double* out, cudaStream_t s);
// u_n = 2 zeta - u_{n-1}, interface columns from the left strip
cudaError_t launch_commit(const AuxGeom& g, const double2* zeta, double2* u, cudaStream_t s);
// mass u^H M u and energy parts; partial sums part[nblk][4]
cudaError_t launch_diagnostics(const AuxGeom& g, const double2* u, const double* Wn, double* part,
                               int* nblk_out, cudaStream_t s);
// L_h block extraction from unit-datum solutions (mode 1 of the strip solver)
cudaError_t launch_extract_blocks(const AuxGeom& g, const double2* zeta, int nvirt, int unit_base,
                                  double2* X, cudaStream_t s);
// y = x - L x  (P of eq. algo_pd) with per-strip block sets X[btype[j]] (4 blocks each)
cudaError_t launch_apply_P(const AuxGeom& g, const void* X, bool fp32, const int* btype_dev,
                           const double2* x, double2* y, double2* work, cudaStream_t s);
cudaError_t launch_convert_blocks(const double2* X, float2* Xf, long long n, cudaStream_t s);

// exact P^{-1} in the cosine basis (modal.cu)
cudaError_t launch_modal_setup(const AuxGeom& g, int ntypes, const int* tkind_dev, const int* btype_dev,
                               double* Cf, double* Ci, float* Cf32, float* Ci32, double2* xm, double2* fac,
                               double2* work, cudaStream_t s, int pade_m = 0, const double2* pa = nullptr,
                               const double2* pd = nullptr);
cudaError_t launch_to_float(const double* a, float* b, long long n, cudaStream_t s);
// g_new = g_k - P^{-1}(g_k - R(g_k)) (eq. algo_pd) with the modal P^-1: five launches (the
// subtractions fused into the transforms).  kmax > 0: modes k >= kmax take P = I.
// g_new and tmp may alias rg.
cudaError_t launch_modal_update(const Geom& g, bool fp32, const double* Cf, const double* Ci, const float* Cf32,
                                const float* Ci32, const double2* fac, const float2* fac32, const double2* gk,
                                const double2* rg, double2* gnew, double2* tmp, void* cpart, int kmax, cudaStream_t s);

// ---- rotating frame of the GPE (rotating.cu)
// Wout = Ws + (w0 trap(t0) + w1 trap(t1)) inv_lap, trap(t) = -(gx2 x^2 + gy2 y^2)/2 at A(t) x~,
// with (c_k, s_k) = (cos w t_k, sin w t_k)
struct TrapArgs {
    double gx2, gy2, inv_lap;
    double c0, s0, w0, c1, s1, w1;
};
cudaError_t launch_trap_potential(const Geom& g, const double* Ws, double* Wout, const TrapArgs& t, cudaStream_t s);
// <u, L_z u> partial sums into part[b*4 + slot], nblk blocks
cudaError_t launch_lz(const Geom& g, const double2* u, double* part, int nblk, int slot, cudaStream_t s);
// Q1 interpolant of u (strip layout) at A^T (x, y) on (nxo+1) x (nyo+1) points of (x0,x1) x (y0,y1)
cudaError_t launch_lab_frame(const Geom& g, const double2* u, int nxo, int nyo, double x0, double x1, double y0,
                             double y1, double c, double s, double2* out, cudaStream_t st);

// GMRES helpers on vectors of length n (complex, FP64)
cudaError_t launch_dots(const double2* V, long long ld, int k, const double2* w, long long n, double2* out,
                        double* scratch, cudaStream_t s);
cudaError_t launch_axpy_multi(const double2* V, long long ld, int k, const double2* h, double2* w, long long n,
                              cudaStream_t s);
cudaError_t launch_nrm2(const double2* w, long long n, double* out, double* scratch, cudaStream_t s);
cudaError_t launch_scale(double2* y, const double2* x, const double* inv_from, long long n, cudaStream_t s);
cudaError_t launch_sub(double2* y, const double2* a, const double2* b, long long n, cudaStream_t s);
cudaError_t launch_copy(double2* y, const double2* x, long long n, cudaStream_t s);

}  // namespace ddnls
