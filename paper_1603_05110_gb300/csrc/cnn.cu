// Learned initial interface guess: a small CNN on the stacked interface traces.
//
// The paper starts each step from the previous step's converged interface vector
// (g_n^0 = g_{n-1}, Sec. 5).  Here a 4-layer convolutional network predicts the next vector
// from the last three: the input image has H = 2(N-1) rows (the traces of g, in the order of
// Sec. 2.3) and W = ny+1 columns, and 6 channels
//     g_{n-1}/s0,  (g_{n-1} - g_{n-2})/s1,  (g_{n-2} - g_{n-3})/s1    (real and imaginary parts),
// s0 = rms(g_{n-1}), s1 = rms(g_{n-1} - g_{n-2}).  The network (3x3 convolutions 6->32->32->32->2,
// ReLU between) outputs a correction to a base guess, linear extrapolation (e = 1, default) or
// the paper's previous-step vector (e = 0, dd_cnn_set_base):
//     g_n^0 = g_{n-1} + e (g_{n-1} - g_{n-2}) + s1 * out.
// With zero last-layer weights it is the base; trained on converged vectors of the plain solver
// it learns the rest.  The Schwarz iteration converges from any guess, so the guess
// only changes the iteration count.
//
// Arithmetic: activations and weights in BF16, accumulation in FP32, on the tensor cores through
// mma.sync m16n8k16 (implicit GEMM: pixels x output channels, K = input channels x 9).  The
// input gradient is the same forward convolution with the kernels rotated by 180 degrees and
// the channel roles swapped; the weight gradient is a GEMM over pixels with deterministic
// per-chunk partial sums.  Master weights and Adam moments are FP32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dd_nls.h"
#include "common.cuh"
#include "kernels.h"

namespace ddnls {

constexpr int kLayers = 4;
constexpr int kChunk = 1024;     // pixels per weight-gradient partial

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<unsigned*>(&v);
}

// D += A (16x16, row-major) * B (16x8, col-major), BF16 in, FP32 accumulate.
__device__ __forceinline__ void mma16816(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// im2col value: input channel ci, tap r (kh = r/3, kw = r%3) at pixel p of an H x W image
__device__ __forceinline__ float im2col(const __nv_bfloat16* __restrict__ X, int H, int W, int p, int k, int K) {
    if (p >= H * W || k >= K) return 0.f;
    const int ci = k / 9, r = k - ci * 9;
    const int h = p / W + r / 3 - 1, w = p % W + r % 3 - 1;
    if (h < 0 || h >= H || w < 0 || w >= W) return 0.f;
    return __bfloat162float(X[(long long)ci * H * W + (long long)h * W + w]);
}

// Y[co][p] = sum_k Wt[co][k] im2col(X)[p][k] + bias[co]   (one warp: 16 pixels x all channels)
// Outputs: pre (FP32, nullable), act = bf16(relu(pre)) (nullable), or for the last layer pre only.
template <int NT>
__global__ void conv_fwd_kernel(const __nv_bfloat16* __restrict__ X, int Cin, int H, int W,
                                const __nv_bfloat16* __restrict__ Wt, const float* __restrict__ bias, int Cout,
                                float* __restrict__ pre, __nv_bfloat16* __restrict__ act) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int HW = H * W;
    const int p0 = (int)(warp * 16);
    if (p0 >= HW) return;
    const int g = lane >> 2, t = lane & 3;
    const int K = Cin * 9, K16 = (K + 15) / 16;
    float acc[NT][4];
#pragma unroll
    for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
    const int pa = p0 + g, pb = p0 + g + 8;
    for (int kk = 0; kk < K16; ++kk) {
        const int k0 = kk * 16 + 2 * t, k1 = k0 + 8;
        unsigned a[4];
        a[0] = pack_bf16(im2col(X, H, W, pa, k0, K), im2col(X, H, W, pa, k0 + 1, K));
        a[1] = pack_bf16(im2col(X, H, W, pb, k0, K), im2col(X, H, W, pb, k0 + 1, K));
        a[2] = pack_bf16(im2col(X, H, W, pa, k1, K), im2col(X, H, W, pa, k1 + 1, K));
        a[3] = pack_bf16(im2col(X, H, W, pb, k1, K), im2col(X, H, W, pb, k1 + 1, K));
#pragma unroll
        for (int n = 0; n < NT; ++n) {
            const int co = n * 8 + g;
            unsigned b[2];
            auto wv = [&](int k) { return (co < Cout && k < K) ? __bfloat162float(Wt[(long long)co * K + k]) : 0.f; };
            b[0] = pack_bf16(wv(k0), wv(k0 + 1));
            b[1] = pack_bf16(wv(k1), wv(k1 + 1));
            mma16816(acc[n], a, b);
        }
    }
#pragma unroll
    for (int n = 0; n < NT; ++n) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int co = n * 8 + 2 * t + (e & 1);
            const int p = (e < 2) ? pa : pb;
            if (co >= Cout || p >= HW) continue;
            const float v = acc[n][e] + (bias ? bias[co] : 0.f);
            if (pre) pre[(long long)co * HW + p] = v;
            if (act) act[(long long)co * HW + p] = __float2bfloat16(v > 0.f ? v : 0.f);
        }
    }
}

// Partial weight gradients: P[chunk][co][k] = sum_{p in chunk} dY[co][p] im2col(X)[p][k].
// Block (4 warps): co tile of 16 (blockIdx.z), k range of 64 (blockIdx.y), pixel chunk (blockIdx.x).
__global__ void conv_wgrad_kernel(const __nv_bfloat16* __restrict__ dY, int Cout, const __nv_bfloat16* __restrict__ X,
                                  int Cin, int H, int W, float* __restrict__ part) {
    __shared__ float red[4][16][64];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int HW = H * W, K = Cin * 9;
    const int co0 = blockIdx.z * 16, kb = blockIdx.y * 64;
    const int c0 = blockIdx.x * kChunk;
    float acc[8][4];
#pragma unroll
    for (int n = 0; n < 8; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
    auto dy = [&](int co, int p) { return (co < Cout && p < HW) ? __bfloat162float(dY[(long long)co * HW + p]) : 0.f; };
    for (int pp = c0 + wid * 16; pp < min(c0 + kChunk, HW); pp += 64) {
        unsigned a[4];
        a[0] = pack_bf16(dy(co0 + g, pp + 2 * t), dy(co0 + g, pp + 2 * t + 1));
        a[1] = pack_bf16(dy(co0 + g + 8, pp + 2 * t), dy(co0 + g + 8, pp + 2 * t + 1));
        a[2] = pack_bf16(dy(co0 + g, pp + 2 * t + 8), dy(co0 + g, pp + 2 * t + 9));
        a[3] = pack_bf16(dy(co0 + g + 8, pp + 2 * t + 8), dy(co0 + g + 8, pp + 2 * t + 9));
#pragma unroll
        for (int n = 0; n < 8; ++n) {
            const int k = kb + n * 8 + g;
            unsigned b[2];
            b[0] = pack_bf16(im2col(X, H, W, pp + 2 * t, k, K), im2col(X, H, W, pp + 2 * t + 1, k, K));
            b[1] = pack_bf16(im2col(X, H, W, pp + 2 * t + 8, k, K), im2col(X, H, W, pp + 2 * t + 9, k, K));
            mma16816(acc[n], a, b);
        }
    }
#pragma unroll
    for (int n = 0; n < 8; ++n)
#pragma unroll
        for (int e = 0; e < 4; ++e) red[wid][g + (e >= 2 ? 8 : 0)][n * 8 + 2 * t + (e & 1)] = acc[n][e];
    __syncthreads();
    for (int i = threadIdx.x; i < 16 * 64; i += blockDim.x) {
        const int r = i / 64, cc = i % 64;
        const int co = co0 + r, k = kb + cc;
        if (co >= Cout || k >= K) continue;
        const float s = red[0][r][cc] + red[1][r][cc] + red[2][r][cc] + red[3][r][cc];
        part[((long long)blockIdx.x * Cout + co) * K + k] = s;
    }
}

// grad[i] = sum_chunk part[chunk][i]  (fixed order), and bias gradients db[co] = sum_p dY[co][p]
__global__ void reduce_chunks_kernel(const float* __restrict__ part, int nchunk, int n, float* __restrict__ grad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.f;
    for (int c = 0; c < nchunk; ++c) s += part[(long long)c * n + i];
    grad[i] = s;
}
__global__ void bias_grad_kernel(const __nv_bfloat16* __restrict__ dY, int HW, float* __restrict__ db) {
    __shared__ double sm[64];
    const int co = blockIdx.x;
    double v[1] = {0.0};
    for (int p = threadIdx.x; p < HW; p += blockDim.x) v[0] += __bfloat162float(dY[(long long)co * HW + p]);
    block_sum<1>(v, sm);
    if (threadIdx.x == 0) db[co] = (float)v[0];
}

// W2[ci][co*9 + r] = Wt[co][ci*9 + 8 - r]: the input gradient as a forward convolution
__global__ void rotate_weights_kernel(const __nv_bfloat16* __restrict__ Wt, int Cout, int Cin,
                                      __nv_bfloat16* __restrict__ W2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = Cout * Cin * 9;
    if (i >= n) return;
    const int ci = i / (Cout * 9), rem = i - ci * Cout * 9, co = rem / 9, r = rem - co * 9;
    W2[i] = Wt[(long long)co * Cin * 9 + ci * 9 + 8 - r];
}

// dX (FP32 from the transposed convolution) times relu'(pre) -> BF16
__global__ void relu_back_kernel(const float* __restrict__ dX, const float* __restrict__ pre, long long n,
                                 __nv_bfloat16* __restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16(pre[i] > 0.f ? dX[i] : 0.f);
}

// loss = mean (out - tgt)^2 over the 2 x HW outputs; dY = 2 (out - tgt) / count (BF16)
__global__ void mse_kernel(const float* __restrict__ out, const float* __restrict__ tgt, long long n,
                           __nv_bfloat16* __restrict__ dY, double* __restrict__ loss_part) {
    __shared__ double sm[64];
    double v[1] = {0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = out[i] - tgt[i];
        v[0] += (double)d * d;
        dY[i] = __float2bfloat16(2.f * d / (float)n);
    }
    block_sum<1>(v, sm);
    if (threadIdx.x == 0) loss_part[blockIdx.x * 4] = v[0] / (double)n;
}

// Adam on the FP32 master weights; refreshes the BF16 copy
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ gr, float* __restrict__ m,
                            float* __restrict__ v, __nv_bfloat16* __restrict__ wb, long long n, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = gr[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        wb[i] = __float2bfloat16(wi);
    }
}
__global__ void to_bf16_kernel(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = __float2bfloat16(a[i]);
}

// ---------------------------------------------------------------- features and guess
// Interface vectors: ntr traces of nyn complex values (unpadded, the ABI layout).
// part[0] = sum |g1|^2, part[1] = sum |g1 - g2|^2 (one block per reduction, fixed order)
__global__ void guess_norms_kernel(const double2* __restrict__ g1, const double2* __restrict__ g2, long long n,
                                   double* __restrict__ out) {
    __shared__ double sm[64];
    double v[2] = {0.0, 0.0};
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        const double2 a = g1[i], b = g2[i];
        v[0] += a.x * a.x + a.y * a.y;
        v[1] += (a.x - b.x) * (a.x - b.x) + (a.y - b.y) * (a.y - b.y);
    }
    block_sum<2>(v, sm);
    if (threadIdx.x == 0) {
        const double nn = (double)(n > 0 ? n : 1);
        out[0] = sqrt(v[0] / nn) + 1e-300;      // s0
        out[1] = sqrt(v[1] / nn) + 1e-300;      // s1
    }
}
// x[6][n] (bf16) and, when gt != NULL, the training target tgt[2][n] = (gt - g1 - e (g1 - g2))/s1
__global__ void guess_features_kernel(const double2* __restrict__ g1, const double2* __restrict__ g2,
                                      const double2* __restrict__ g3, const double2* __restrict__ gt, long long n,
                                      const double* __restrict__ s, double e, __nv_bfloat16* __restrict__ x,
                                      float* __restrict__ tgt) {
    const double s0 = s[0], s1 = s[1];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double2 a = g1[i], b = g2[i], c = g3[i];
        x[0 * n + i] = __float2bfloat16((float)(a.x / s0));
        x[1 * n + i] = __float2bfloat16((float)(a.y / s0));
        x[2 * n + i] = __float2bfloat16((float)((a.x - b.x) / s1));
        x[3 * n + i] = __float2bfloat16((float)((a.y - b.y) / s1));
        x[4 * n + i] = __float2bfloat16((float)((b.x - c.x) / s1));
        x[5 * n + i] = __float2bfloat16((float)((b.y - c.y) / s1));
        if (gt) {
            const double2 t = gt[i];
            tgt[0 * n + i] = (float)((t.x - a.x - e * (a.x - b.x)) / s1);
            tgt[1 * n + i] = (float)((t.y - a.y - e * (a.y - b.y)) / s1);
        }
    }
}
// g0 = g1 + e (g1 - g2) + s1 * out
__global__ void guess_apply_kernel(const double2* __restrict__ g1, const double2* __restrict__ g2, const float* __restrict__ out,
                                   long long n, const double* __restrict__ s, double e, double2* __restrict__ g0) {
    const double s1 = s[1];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double2 a = g1[i], b = g2[i];
        g0[i] = make_double2(a.x + e * (a.x - b.x) + s1 * out[0 * n + i], a.y + e * (a.y - b.y) + s1 * out[1 * n + i]);
    }
}

}  // namespace ddnls

using namespace ddnls;

static const int kCin[kLayers] = {6, 32, 32, 32};
static const int kCout[kLayers] = {32, 32, 32, 2};

struct dd_cnn {
    int H = 0, W = 0;           // image: H = number of traces, W = nodes per trace
    double e = 1.0;             // base guess: 1 linear extrapolation, 0 the previous vector
    long long HW = 0;
    cudaStream_t s = nullptr;
    long long nparam = 0;
    long long woff[kLayers], boff[kLayers];
    float *w = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;   // FP32 master, Adam, gradient
    __nv_bfloat16* wb = nullptr;                                         // BF16 copy (same layout)
    __nv_bfloat16* w2 = nullptr;                                         // rotated kernels (scratch)
    __nv_bfloat16 *x = nullptr, *act[kLayers] = {nullptr, nullptr, nullptr, nullptr};
    float* pre[kLayers] = {nullptr, nullptr, nullptr, nullptr};
    __nv_bfloat16 *dya = nullptr, *dyb = nullptr;
    float *dx = nullptr, *tgt = nullptr, *part = nullptr;
    double *sc = nullptr, *lossp = nullptr, *hloss = nullptr;
    long long adam_t = 0;
    std::string error;
};

static int cfail(dd_cnn* c, int code, const std::string& msg) {
    if (c) c->error = msg;
    else set_handle_free_error(msg.c_str());
    return code;
}
#define CCK(call)                                                                                \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return cfail(c, DD_NLS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

static int nblk(long long n, int b) { long long v = (n + b - 1) / b; return (int)(v > 4096 ? 4096 : (v < 1 ? 1 : v)); }

static cudaError_t conv_forward(dd_cnn* c, const __nv_bfloat16* X, int Cin, const __nv_bfloat16* Wt, const float* bias,
                                int Cout, float* pre, __nv_bfloat16* act) {
    const long long warps = (c->HW + 15) / 16;
    const int grid = (int)((warps * 32 + 127) / 128);
    count_launches(1);
    if (Cout > 8)
        conv_fwd_kernel<4><<<grid, 128, 0, c->s>>>(X, Cin, c->H, c->W, Wt, bias, Cout, pre, act);
    else
        conv_fwd_kernel<1><<<grid, 128, 0, c->s>>>(X, Cin, c->H, c->W, Wt, bias, Cout, pre, act);
    return cudaGetLastError();
}

// forward pass from c->x; out in c->pre[3]
static int cnn_forward(dd_cnn* c) {
    const __nv_bfloat16* in = c->x;
    for (int l = 0; l < kLayers; ++l) {
        const bool last = l == kLayers - 1;
        CCK(conv_forward(c, in, kCin[l], c->wb + c->woff[l], c->w + c->boff[l], kCout[l], c->pre[l], last ? nullptr : c->act[l]));
        in = c->act[l];
    }
    return DD_NLS_OK;
}

// loss and gradients of the last forward pass against c->tgt; gradients into c->grad
static int cnn_backward(dd_cnn* c, double* loss) {
    const long long nout = 2 * c->HW;
    count_launches(1);
    mse_kernel<<<256, 256, 0, c->s>>>(c->pre[kLayers - 1], c->tgt, nout, c->dya, c->lossp);
    CCK(cudaGetLastError());
    CCK(launch_finalize(c->lossp, 256, 1, c->sc + 4, c->s));
    const int nchunk = (int)((c->HW + kChunk - 1) / kChunk);
    __nv_bfloat16* dy = c->dya;
    __nv_bfloat16* dnext = c->dyb;
    for (int l = kLayers - 1; l >= 0; --l) {
        const int Cin = kCin[l], Cout = kCout[l], K = Cin * 9;
        const __nv_bfloat16* X = l == 0 ? c->x : c->act[l - 1];
        dim3 grid(nchunk, (K + 63) / 64, (Cout + 15) / 16);
        count_launches(3);
        conv_wgrad_kernel<<<grid, 128, 0, c->s>>>(dy, Cout, X, Cin, c->H, c->W, c->part);
        reduce_chunks_kernel<<<(Cout * K + 255) / 256, 256, 0, c->s>>>(c->part, nchunk, Cout * K, c->grad + c->woff[l]);
        bias_grad_kernel<<<Cout, 256, 0, c->s>>>(dy, (int)c->HW, c->grad + c->boff[l]);
        CCK(cudaGetLastError());
        if (l == 0) break;
        // input gradient: forward convolution with rotated kernels, then relu' of layer l-1
        count_launches(1);
        rotate_weights_kernel<<<(Cout * Cin * 9 + 255) / 256, 256, 0, c->s>>>(c->wb + c->woff[l], Cout, Cin, c->w2);
        CCK(cudaGetLastError());
        CCK(conv_forward(c, dy, Cout, c->w2, nullptr, Cin, c->dx, nullptr));
        count_launches(1);
        relu_back_kernel<<<nblk((long long)Cin * c->HW, 256), 256, 0, c->s>>>(c->dx, c->pre[l - 1], (long long)Cin * c->HW, dnext);
        CCK(cudaGetLastError());
        std::swap(dy, dnext);
    }
    if (loss) {
        CCK(cudaMemcpyAsync(c->hloss, c->sc + 4, sizeof(double), cudaMemcpyDeviceToHost, c->s));
        CCK(cudaStreamSynchronize(c->s));
        *loss = c->hloss[0];
    }
    return DD_NLS_OK;
}

static int cnn_features(dd_cnn* c, const double* g1, const double* g2, const double* g3, const double* gt) {
    const long long n = c->HW;
    count_launches(2);
    guess_norms_kernel<<<1, 512, 0, c->s>>>((const double2*)g1, (const double2*)g2, n, c->sc);
    guess_features_kernel<<<nblk(n, 256), 256, 0, c->s>>>((const double2*)g1, (const double2*)g2, (const double2*)g3,
                                                         (const double2*)gt, n, c->sc, c->e, c->x, c->tgt);
    CCK(cudaGetLastError());
    return DD_NLS_OK;
}

extern "C" int dd_cnn_create(int n_traces, int nodes_per_trace, void* stream, dd_cnn** out) {
    dd_cnn* c = nullptr;
    if (n_traces < 1 || nodes_per_trace < 1 || !out) return cfail(nullptr, DD_NLS_EINVAL, "dd_cnn_create: bad sizes");
    if ((long long)n_traces * nodes_per_trace > (1LL << 28))      // the kernels index an image with 32-bit ints
        return cfail(nullptr, DD_NLS_EINVAL, "dd_cnn_create: n_traces x nodes_per_trace above 2^28");
    *out = nullptr;
    c = new dd_cnn();
    c->H = n_traces;
    c->W = nodes_per_trace;
    c->HW = (long long)n_traces * nodes_per_trace;
    c->s = (cudaStream_t)stream;
    long long off = 0;
    for (int l = 0; l < kLayers; ++l) {
        c->woff[l] = off;
        off += (long long)kCout[l] * kCin[l] * 9;
        c->boff[l] = off;
        off += kCout[l];
    }
    c->nparam = off;
    const long long nchunk = (c->HW + kChunk - 1) / kChunk;
    cudaError_t e = cudaSuccess;
    auto A = [&](void** p, size_t bytes) { if (!e) { e = cudaMalloc(p, bytes); if (!e) e = cudaMemset(*p, 0, bytes); } };
    A((void**)&c->w, sizeof(float) * off);
    A((void**)&c->m, sizeof(float) * off);
    A((void**)&c->v, sizeof(float) * off);
    A((void**)&c->grad, sizeof(float) * off);
    A((void**)&c->wb, sizeof(__nv_bfloat16) * off);
    A((void**)&c->w2, sizeof(__nv_bfloat16) * 32 * 32 * 9);
    A((void**)&c->x, sizeof(__nv_bfloat16) * 6 * c->HW);
    for (int l = 0; l < kLayers; ++l) {
        A((void**)&c->pre[l], sizeof(float) * kCout[l] * c->HW);
        if (l < kLayers - 1) A((void**)&c->act[l], sizeof(__nv_bfloat16) * kCout[l] * c->HW);
    }
    A((void**)&c->dya, sizeof(__nv_bfloat16) * 32 * c->HW);
    A((void**)&c->dyb, sizeof(__nv_bfloat16) * 32 * c->HW);
    A((void**)&c->dx, sizeof(float) * 32 * c->HW);
    A((void**)&c->tgt, sizeof(float) * 2 * c->HW);
    A((void**)&c->part, sizeof(float) * nchunk * 32 * 32 * 9);
    A((void**)&c->sc, sizeof(double) * 8);
    A((void**)&c->lossp, sizeof(double) * 4 * 256);
    if (!e) e = cudaMallocHost((void**)&c->hloss, sizeof(double) * 2);
    if (e) {
        std::string msg = std::string("dd_cnn_create: ") + cudaGetErrorString(e);
        dd_cnn_destroy(c);
        return cfail(nullptr, DD_NLS_ENOMEM, msg);
    }
    *out = c;
    return DD_NLS_OK;
}

extern "C" long long dd_cnn_num_params(const dd_cnn* c) { return c ? c->nparam : 0; }

extern "C" int dd_cnn_set_base(dd_cnn* c, int base) {
    if (!c || (base != DD_CNN_BASE_PREVIOUS && base != DD_CNN_BASE_EXTRAPOLATE))
        return DD_NLS_EINVAL;
    c->e = base == DD_CNN_BASE_EXTRAPOLATE ? 1.0 : 0.0;
    return DD_NLS_OK;
}

extern "C" int dd_cnn_set_params(dd_cnn* c, const float* w, int ptr_kind) {
    if (!c || !w) return cfail(c, DD_NLS_EINVAL, "dd_cnn_set_params: NULL argument");
    if (ptr_kind != DD_NLS_PTR_HOST && ptr_kind != DD_NLS_PTR_DEVICE) return cfail(c, DD_NLS_EINVAL, "dd_cnn_set_params: unknown ptr_kind");
    CCK(cudaMemcpyAsync(c->w, w, sizeof(float) * c->nparam,
                        ptr_kind == DD_NLS_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->s));
    CCK(cudaMemsetAsync(c->m, 0, sizeof(float) * c->nparam, c->s));
    CCK(cudaMemsetAsync(c->v, 0, sizeof(float) * c->nparam, c->s));
    count_launches(1);
    to_bf16_kernel<<<nblk(c->nparam, 256), 256, 0, c->s>>>(c->w, c->wb, c->nparam);
    CCK(cudaGetLastError());
    CCK(cudaStreamSynchronize(c->s));
    c->adam_t = 0;
    return DD_NLS_OK;
}

extern "C" int dd_cnn_get_params(dd_cnn* c, float* w, int ptr_kind) {
    if (!c || !w) return cfail(c, DD_NLS_EINVAL, "dd_cnn_get_params: NULL argument");
    if (ptr_kind != DD_NLS_PTR_HOST && ptr_kind != DD_NLS_PTR_DEVICE) return cfail(c, DD_NLS_EINVAL, "dd_cnn_get_params: unknown ptr_kind");
    CCK(cudaMemcpyAsync(w, c->w, sizeof(float) * c->nparam,
                        ptr_kind == DD_NLS_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->s));
    CCK(cudaStreamSynchronize(c->s));
    return DD_NLS_OK;
}

extern "C" int dd_cnn_guess(dd_cnn* c, const double* g1, const double* g2, const double* g3, double* g0) {
    if (!c || !g1 || !g2 || !g3 || !g0) return cfail(c, DD_NLS_EINVAL, "dd_cnn_guess: NULL argument");
    int rc = cnn_features(c, g1, g2, g3, nullptr);
    if (rc) return rc;
    rc = cnn_forward(c);
    if (rc) return rc;
    count_launches(1);
    guess_apply_kernel<<<nblk(c->HW, 256), 256, 0, c->s>>>((const double2*)g1, (const double2*)g2, c->pre[kLayers - 1],
                                                          c->HW, c->sc, c->e, (double2*)g0);
    CCK(cudaGetLastError());
    CCK(cudaStreamSynchronize(c->s));
    return DD_NLS_OK;
}

extern "C" int dd_cnn_loss_grad(dd_cnn* c, const double* g1, const double* g2, const double* g3, const double* gt,
                                float* grad, double* loss, int ptr_kind) {
    if (!c || !g1 || !g2 || !g3 || !gt) return cfail(c, DD_NLS_EINVAL, "dd_cnn_loss_grad: NULL argument");
    if (ptr_kind != DD_NLS_PTR_HOST && ptr_kind != DD_NLS_PTR_DEVICE) return cfail(c, DD_NLS_EINVAL, "dd_cnn_loss_grad: unknown ptr_kind");
    int rc = cnn_features(c, g1, g2, g3, gt);
    if (!rc) rc = cnn_forward(c);
    if (!rc) rc = cnn_backward(c, loss);
    if (rc) return rc;
    if (grad)
        CCK(cudaMemcpyAsync(grad, c->grad, sizeof(float) * c->nparam,
                            ptr_kind == DD_NLS_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->s));
    CCK(cudaStreamSynchronize(c->s));
    return DD_NLS_OK;
}

extern "C" int dd_cnn_train_step(dd_cnn* c, const double* g1, const double* g2, const double* g3, const double* gt,
                                 float lr, double* loss) {
    if (!c || !g1 || !g2 || !g3 || !gt) return cfail(c, DD_NLS_EINVAL, "dd_cnn_train_step: NULL argument");
    int rc = cnn_features(c, g1, g2, g3, gt);
    if (!rc) rc = cnn_forward(c);
    if (!rc) rc = cnn_backward(c, loss);
    if (rc) return rc;
    c->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)c->adam_t), c2 = 1.f - powf(b2, (float)c->adam_t);
    count_launches(1);
    adam_kernel<<<nblk(c->nparam, 256), 256, 0, c->s>>>(c->w, c->grad, c->m, c->v, c->wb, c->nparam, lr, b1, b2, 1e-8f, c1, c2);
    CCK(cudaGetLastError());
    if (!loss) CCK(cudaStreamSynchronize(c->s));
    return DD_NLS_OK;
}

extern "C" const char* dd_cnn_last_error(const dd_cnn* c) { return c ? c->error.c_str() : dd_nls_last_error(nullptr); }

extern "C" void dd_cnn_destroy(dd_cnn* c) {
    if (!c) return;
    if (c->s) cudaStreamSynchronize(c->s);
    void* p[] = {c->w, c->m, c->v, c->grad, c->wb, c->w2, c->x, c->pre[0], c->pre[1], c->pre[2], c->pre[3], c->act[0],
                 c->act[1], c->act[2], c->dya, c->dyb, c->dx, c->tgt, c->part, c->sc, c->lossp};
    for (void* q : p)
        if (q) cudaFree(q);
    if (c->hloss) cudaFreeHost(c->hloss);
    delete c;
}
