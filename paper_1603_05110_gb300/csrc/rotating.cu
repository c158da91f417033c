// The GPE in the rotating frame (Sec. 5.2.1 of the paper, eq. x1Ax, GPE_Trans, u1u):
//  - the time-dependent trap V_t(t, x~) = V(A(t) x~) and the potential of one time step,
//    W_n = (V_n + V_{n-1})/2 (eq. CNS), written on every strip node;
//  - the angular momentum <u, L_z u>, L_z = -i (x d_y - y d_x), for the energy of eq. (GPE);
//  - the lab-frame field u(t, x, y) = u~(t, A(t)^T (x, y)) on the valid zone, by Q1 interpolation.
// A(t) = [[cos wt, sin wt], [-sin wt, cos wt]]; the trap of eq. (GPE) is
// V = (gx^2 x^2 + gy^2 y^2)/2, which enters eq. (Sch) with the opposite sign.
#include "common.cuh"
#include "kernels.h"

#include <algorithm>

namespace ddnls {

// -(gx2 x^2 + gy2 y^2)/2 at (x, y) = A (xt, yt), A = [[c, s], [-s, c]]
__device__ __forceinline__ double trap_at(double xt, double yt, double c, double s, double gx2, double gy2) {
    const double x = c * xt + s * yt, y = -s * xt + c * yt;
    return -0.5 * (gx2 * x * x + gy2 * y * y);
}

// Wout = Ws + (w0 trap(t0) + w1 trap(t1)) / lap on every strip node (Ws nullable: zero)
__global__ void trap_potential_kernel(Geom g, const double* __restrict__ Ws, double* __restrict__ Wout, TrapArgs t) {
    const long long total = (long long)g.N * g.nxs * g.nyn;
    const int c = g.nxs - 1;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total; q += (long long)gridDim.x * blockDim.x) {
        int j, ix, iy;
        split_strip_node(q, g.nxs, g.nyn, j, ix, iy);
        const double xt = g.xl + (double)(j * c + ix) * g.hx, yt = g.yb + (double)iy * g.hy;
        const long long idx = (long long)(j * g.nxs + ix) * g.P + iy;
        double v = t.w0 * trap_at(xt, yt, t.c0, t.s0, t.gx2, t.gy2);
        if (t.w1 != 0.0) v += t.w1 * trap_at(xt, yt, t.c1, t.s1, t.gx2, t.gy2);
        Wout[idx] = (Ws ? Ws[idx] : 0.0) + v * t.inv_lap;
    }
}
cudaError_t launch_trap_potential(const Geom& g, const double* Ws, double* Wout, const TrapArgs& t, cudaStream_t s) {
    count_launches(1);
    trap_potential_kernel<<<1024, 256, 0, s>>>(g, Ws, Wout, t);
    return cudaGetLastError();
}

// <u, L_z u> per block into part[b*4 + slot]: nodal weights (halves on the duplicated interface
// columns, each strip counting its copy), central differences (one-sided at the ends of Omega;
// across an interface the neighbour strip's column), real part.
__global__ void lz_kernel(Geom g, const double2* __restrict__ u, double* __restrict__ part, int slot) {
    __shared__ double sm[64];
    const int c = g.nxs - 1, ny = g.nyn - 1;
    const long long total = (long long)g.N * g.nxs * g.nyn;
    double v[1] = {0.0};
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total; q += (long long)gridDim.x * blockDim.x) {
        int j, ix, iy;
        split_strip_node(q, g.nxs, g.nyn, j, ix, iy);
        const long long col = (long long)(j * g.nxs + ix) * g.P;
        const double2 u0 = u[col + iy];
        // d/dy in the column
        double2 dy;
        if (ny == 0) dy = make_double2(0.0, 0.0);
        else if (iy == 0) dy = cscale(csub(u[col + 1], u0), 1.0 / g.hy);
        else if (iy == ny) dy = cscale(csub(u0, u[col + iy - 1]), 1.0 / g.hy);
        else dy = cscale(csub(u[col + iy + 1], u[col + iy - 1]), 0.5 / g.hy);
        // d/dx along the row, across strips
        const int ixg = j * c + ix;
        auto at = [&](int xg) {                  // u at global column xg, row iy
            const int jj = xg >= g.nx ? g.N - 1 : xg / c;
            return u[(long long)(jj * g.nxs + (xg - jj * c)) * g.P + iy];
        };
        double2 dx;
        if (g.nx == 0) dx = make_double2(0.0, 0.0);
        else if (ixg == 0) dx = cscale(csub(at(1), u0), 1.0 / g.hx);
        else if (ixg == g.nx) dx = cscale(csub(u0, at(g.nx - 1)), 1.0 / g.hx);
        else dx = cscale(csub(at(ixg + 1), at(ixg - 1)), 0.5 / g.hx);
        const double x = g.xl + (double)ixg * g.hx, y = g.yb + (double)iy * g.hy;
        // L u = -i (x dy - y dx);  Re(conj(u0) L u) = Im(conj(u0) (x dy - y dx))
        const double2 d = make_double2(x * dy.x - y * dx.x, x * dy.y - y * dx.y);
        const double w = wq(ix, c, g.hx) * wq(iy, ny, g.hy);
        v[0] += w * (u0.x * d.y - u0.y * d.x);
    }
    block_sum<1>(v, sm);
    if (threadIdx.x == 0) part[blockIdx.x * 4 + slot] = v[0];
}
cudaError_t launch_lz(const Geom& g, const double2* u, double* part, int nblk, int slot, cudaStream_t s) {
    count_launches(1);
    lz_kernel<<<nblk, 256, 0, s>>>(g, u, part, slot);
    return cudaGetLastError();
}

// out[iy][ix] (x fastest, (nxo+1) x (nyo+1) points on the valid zone (x0,x1) x (y0,y1)) =
// the Q1 interpolant of u~ at A^T (x, y), A^T = [[c, -s], [s, c]]
__global__ void lab_frame_kernel(Geom g, const double2* __restrict__ u, int nxo, int nyo, double x0, double x1,
                                 double y0, double y1, double c, double s, double2* __restrict__ out) {
    const long long total = (long long)(nxo + 1) * (nyo + 1);
    const int cc = g.nxs - 1, ny = g.nyn - 1;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total; q += (long long)gridDim.x * blockDim.x) {
        const int ox = (int)(q % (nxo + 1)), oy = (int)(q / (nxo + 1));
        const double x = nxo > 0 ? x0 + (x1 - x0) * (double)ox / (double)nxo : x0;
        const double y = nyo > 0 ? y0 + (y1 - y0) * (double)oy / (double)nyo : y0;
        const double xt = c * x - s * y, yt = s * x + c * y;
        const double fx = (xt - g.xl) / g.hx, fy = (yt - g.yb) / g.hy;
        int ixg = (int)floor(fx), iy = (int)floor(fy);
        ixg = min(max(ixg, 0), g.nx - 1);
        iy = min(max(iy, 0), max(ny - 1, 0));
        const double sx = fx - ixg, sy = ny > 0 ? fy - iy : 0.0;
        // the cell [ixg, ixg+1] lies inside one strip
        const int j = ixg / cc, ix = ixg - j * cc;
        const double2* col0 = u + (long long)(j * g.nxs + ix) * g.P;
        const double2* col1 = col0 + g.P;
        const int iy1 = ny > 0 ? iy + 1 : iy;
        const double2 a = col0[iy], b = col1[iy], cq = col0[iy1], d = col1[iy1];
        const double wa = (1 - sx) * (1 - sy), wb = sx * (1 - sy), wc = (1 - sx) * sy, wd = sx * sy;
        out[q] = make_double2(wa * a.x + wb * b.x + wc * cq.x + wd * d.x, wa * a.y + wb * b.y + wc * cq.y + wd * d.y);
    }
}
cudaError_t launch_lab_frame(const Geom& g, const double2* u, int nxo, int nyo, double x0, double x1, double y0,
                             double y1, double c, double s, double2* out, cudaStream_t st) {
    const long long total = (long long)(nxo + 1) * (nyo + 1);
    const int nb = (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, 152LL * 8));
    count_launches(1);
    lab_frame_kernel<<<nb, 256, 0, st>>>(g, u, nxo, nyo, x0, x1, y0, y1, c, s, out);
    return cudaGetLastError();
}

}  // namespace ddnls
