// mlp.cu -- the learned control variate's network on the device.
//
// The estimator of Eq. (7b) is a plain Monte Carlo mean (Sec. 4). A control
// variate subtracts from every path the sum of G(s_j, X_j) . sqrt(2) dW_j over
// the sub-steps it takes; any G keeps the mean, a G close to the solution's
// gradient removes most of the variance. Here G is the spatial gradient of a
// network g(x, y, t, w, |grad w| / w): two tanh layers of 64 units, one
// network per field, fitted by least squares to the method's own single-path
// scores. This file holds its kernels:
//
//   k_node_r / k_node_features  the node fields the network reads: w, r =
//                               |grad w| / w and their gradients, by the
//                               finite differences of the drift (FP64);
//   k_cv_scatter                training rows from single-path estimates;
//   k_moments / k_norm          feature standardisation (two-pass, FP64);
//   k_mlp_grad                  forward and backward pass over a tile of 64
//                               rows in shared memory, FP32 SIMT; per-tile
//                               partial gradients, reduced in a fixed order;
//   k_mlp_reduce / k_mlp_adam   the batch gradient; Adam (Kingma & Ba 2015);
//   k_cv_tabulate               the table G at every node and time slice by
//                               forward-mode differentiation; the 64 x 64 layer
//                               on the tensor cores (tcgen05.mma, BF16 in, FP32
//                               accumulate in tensor memory), everything else FP32.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace sdd {
namespace {

constexpr int H = kMlpHidden;
constexpr int D = kMlpInputs;
constexpr int OW1 = 0, OB1 = H * D, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H, OB3 = OW3 + H;
static_assert(OB3 + 1 == kMlpParams, "parameter layout");

constexpr int TILE = 64;     // rows per block of the training kernel
constexpr int LD = 68;       // row stride of the activation tiles (16-byte rows, conflict-free float4 reads)
constexpr int GRAD_THREADS = 256;

// ---------------------------------------------------------------- node fields

__device__ __forceinline__ double fd_x(const double* f, int nx, int i, int j, double rx)
{
    const double* row = f + (long long)j * nx;
    if (i == 0) return (-3.0 * row[0] + 4.0 * row[1] - row[2]) * rx;
    if (i == nx - 1) return (3.0 * row[nx - 1] - 4.0 * row[nx - 2] + row[nx - 3]) * rx;
    return (row[i + 1] - row[i - 1]) * rx;
}

__device__ __forceinline__ double fd_y(const double* f, int nx, int ny, int i, int j, double ry)
{
    const double* col = f + i;
    if (j == 0) return (-3.0 * col[0] + 4.0 * col[(long long)nx] - col[2LL * nx]) * ry;
    if (j == ny - 1)
        return (3.0 * col[(long long)(ny - 1) * nx] - 4.0 * col[(long long)(ny - 2) * nx] +
                col[(long long)(ny - 3) * nx]) * ry;
    return (col[(long long)(j + 1) * nx] - col[(long long)(j - 1) * nx]) * ry;
}

__global__ void k_node_w64(const float* __restrict__ w, long long n, double* __restrict__ w64)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        w64[k] = (double)w[k];
}

// grad w and r = |grad w| / w at every node (FP64).
__global__ void k_node_r(const double* __restrict__ w64, int nx, int ny, double* __restrict__ r64,
                         double2* __restrict__ gw)
{
    const long long n = (long long)nx * ny;
    const double rx = 0.5 * (nx - 1), ry = 0.5 * (ny - 1);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k % nx), j = (int)(k / nx);
        const double wx = fd_x(w64, nx, i, j, rx), wy = fd_y(w64, nx, ny, i, j, ry);
        gw[k] = make_double2(wx, wy);
        r64[k] = sqrt(wx * wx + wy * wy) / w64[k];
    }
}

// nfa = (w, r, dw/dx, dw/dy), nfb = (dr/dx, dr/dy) in FP32.
__global__ void k_node_features(const double* __restrict__ w64, const double* __restrict__ r64,
                                const double2* __restrict__ gw, int nx, int ny, float4* __restrict__ nfa,
                                float2* __restrict__ nfb)
{
    const long long n = (long long)nx * ny;
    const double rx = 0.5 * (nx - 1), ry = 0.5 * (ny - 1);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k % nx), j = (int)(k / nx);
        nfa[k] = make_float4((float)w64[k], (float)r64[k], (float)gw[k].x, (float)gw[k].y);
        nfb[k] = make_float2((float)fd_x(r64, nx, i, j, rx), (float)fd_y(r64, nx, ny, i, j, ry));
    }
}

// The control variate's model from the fields at t_{n-1} themselves: one
// slice, (d xi/dx, d xi/dy, d eta/dx, d eta/dy) at every node by the same
// finite differences. Over a short mesh step the solution's gradient stays
// close to the previous field's.
__global__ void k_field_grad(const double* __restrict__ xi, const double* __restrict__ eta, int nx, int ny,
                             double* __restrict__ table)
{
    const long long n = (long long)nx * ny;
    const double rx = 0.5 * (nx - 1), ry = 0.5 * (ny - 1);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k % nx), j = (int)(k / nx);
        double* o = table + 4 * k;
        o[0] = fd_x(xi, nx, i, j, rx);
        o[1] = fd_y(xi, nx, ny, i, j, ry);
        o[2] = fd_x(eta, nx, i, j, rx);
        o[3] = fd_y(eta, nx, ny, i, j, ry);
    }
}

// Weights C(order, m) 2^-order of the binomial filter, in single precision
// (exact up to order 24; rounded beyond), and the order.
struct BinomWeights {
    float w[kCvMaxOrder + 1];
    int order;
};

// Pass along x: tmp[j (nx - 1) + i] = sum_m w_m table[j][clamp(i - r + m)], all four components,
// for the cells i < nx - 1 along x and the node rows j < ny.
__global__ void k_cv_smooth_x(const double* __restrict__ table, int nx, int ny, const BinomWeights W,
                              float4* __restrict__ tmp)
{
    const long long n = (long long)(nx - 1) * ny;
    const int r = (W.order - 1) / 2;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k % (nx - 1)), j = (int)(k / (nx - 1));
        const double* row = table + 4LL * j * nx;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int m = 0; m <= W.order; ++m) {
            const int q = min(max(i - r + m, 0), nx - 1);
            const double2 u = *reinterpret_cast<const double2*>(row + 4LL * q);
            const double2 v = *reinterpret_cast<const double2*>(row + 4LL * q + 2);
            const float wm = W.w[m];
            acc.x = fmaf(wm, (float)u.x, acc.x);
            acc.y = fmaf(wm, (float)u.y, acc.y);
            acc.z = fmaf(wm, (float)v.x, acc.z);
            acc.w = fmaf(wm, (float)v.y, acc.w);
        }
        tmp[k] = acc;
    }
}

// Pass along y: cells[j (nx - 1) + i] = sum_m w_m tmp[clamp(j - r + m)][i], j < ny - 1.
__global__ void k_cv_smooth_y(const float4* __restrict__ tmp, int nx, int ny, const BinomWeights W,
                              float4* __restrict__ cells)
{
    const long long n = (long long)(nx - 1) * (ny - 1);
    const int r = (W.order - 1) / 2;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k % (nx - 1)), j = (int)(k / (nx - 1));
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int m = 0; m <= W.order; ++m) {
            const int q = min(max(j - r + m, 0), ny - 1);
            const float4 v = tmp[(long long)q * (nx - 1) + i];
            const float wm = W.w[m];
            acc.x = fmaf(wm, v.x, acc.x);
            acc.y = fmaf(wm, v.y, acc.y);
            acc.z = fmaf(wm, v.z, acc.z);
            acc.w = fmaf(wm, v.w, acc.w);
        }
        cells[k] = acc;
    }
}

// ---------------------------------------------------------------- training rows

__device__ __forceinline__ float bilin(const float4* __restrict__ nfa, int nx, int ny, double x, double y, int comp)
{
    double u = x * (nx - 1), v = y * (ny - 1);
    u = fmin(fmax(u, 0.0), nx - 1.0);
    v = fmin(fmax(v, 0.0), ny - 1.0);
    const int i = min((int)floor(u), nx - 2), j = min((int)floor(v), ny - 2);
    const double s = u - i, t = v - j;
    const long long k = (long long)j * nx + i;
    auto get = [&](long long q) { const float4 a = nfa[q]; return (double)(comp == 0 ? a.x : a.y); };
    return (float)((1 - s) * (1 - t) * get(k) + s * (1 - t) * get(k + 1) + (1 - s) * t * get(k + nx) +
                   s * t * get(k + nx + 1));
}

// Horizon k (1-based) of K, M samples: sample m goes to row m K + k - 1.
__global__ void k_cv_scatter(const double* __restrict__ xs, const double* __restrict__ ys,
                             const double* __restrict__ yxi, const double* __restrict__ yeta,
                             const float4* __restrict__ nfa, int nx, int ny, int k, int K, int M,
                             float* __restrict__ feats, float* __restrict__ targets)
{
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
        const long long row = (long long)m * K + (k - 1);
        float* f = feats + row * D;
        f[0] = (float)xs[m];
        f[1] = (float)ys[m];
        f[2] = (float)((double)k / (double)K);
        f[3] = bilin(nfa, nx, ny, xs[m], ys[m], 0);
        f[4] = bilin(nfa, nx, ny, xs[m], ys[m], 1);
        targets[2 * row + 0] = (float)yxi[m];
        targets[2 * row + 1] = (float)yeta[m];
    }
}

// ---------------------------------------------------------------- standardisation

constexpr int MOM_BLOCKS = 256;

// pass 0: per-block sums of f; pass 1: per-block sums of (f - mu)^2.
__global__ void k_moments(const float* __restrict__ feats, long long n, const double* __restrict__ mu, int pass,
                          double* __restrict__ part)
{
    __shared__ double red[D][256 / 32];
    double acc[D];
#pragma unroll
    for (int c = 0; c < D; ++c) acc[c] = 0.0;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const double v = (double)feats[r * D + c];
            const double d = pass ? v - mu[c] : v;
            acc[c] += pass ? d * d : d;
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        double v = acc[c];
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[c][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < D) {
        double v = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) v += red[threadIdx.x][q];
        part[blockIdx.x * D + threadIdx.x] = v;
    }
}

// mu (pass 0) or s (pass 1) from the block sums, in block order.
__global__ void k_norm(const double* __restrict__ part, int nblk, long long n, double* __restrict__ mu, int pass,
                       float* __restrict__ norm)
{
    const int c = threadIdx.x;
    if (c >= D) return;
    double v = 0.0;
    for (int b = 0; b < nblk; ++b) v += part[b * D + c];
    v /= (double)n;
    if (pass == 0) {
        mu[c] = v;
        norm[c] = (float)v;
    } else {
        const double sd = sqrt(v);
        const double m = fabs(mu[c]);
        norm[D + c] = sd > 1e-6 * fmax(1.0, m) ? (float)(1.0 / sd) : 0.0f;
    }
}

// ---------------------------------------------------------------- training

struct GradSmem {
    float th[kMlpStride];      // the network's parameters
    float w2t[H * H];          // W2 transposed: [k][j]
    float z[TILE * D];
    float y[TILE];
    float d[TILE];
    float h1[TILE * LD];       // tanh(a1), later dL/da1
    float h2[TILE * LD];       // tanh(a2), later dL/da2
    float red[GRAD_THREADS / 32];
};

// One 64-row tile of one network (blockIdx.y): forward, backward, and the
// tile's share of the gradient of the batch loss (1 / batch) sum (g - y)^2,
// written to part[(f nblk + tile) stride + p]; part[.. + kMlpParams] = the
// tile's sum of squared errors.
__global__ void __launch_bounds__(GRAD_THREADS) k_mlp_grad(const float* __restrict__ theta,
                                                           const float* __restrict__ norm,
                                                           const float* __restrict__ feats,
                                                           const float* __restrict__ targets, long long row0,
                                                           float inv_batch, float* __restrict__ part)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GradSmem& S = *reinterpret_cast<GradSmem*>(smem_raw);
    const int f = blockIdx.y, tile = blockIdx.x, nblk = gridDim.x, t = threadIdx.x;
    const float* th = theta + (long long)f * kMlpStride;
    for (int p = t; p < kMlpParams; p += GRAD_THREADS) S.th[p] = th[p];
    for (int p = t; p < H * H; p += GRAD_THREADS) {
        const int j = p >> 6, k = p & 63;
        S.w2t[k * H + j] = th[OW2 + p];
    }
    const long long r0 = row0 + (long long)tile * TILE;
    for (int p = t; p < TILE * D; p += GRAD_THREADS) {
        const int c = p % D;
        S.z[p] = (feats[r0 * D + p] - norm[c]) * norm[D + c];
    }
    for (int i = t; i < TILE; i += GRAD_THREADS) S.y[i] = targets[2 * (r0 + i) + f];
    __syncthreads();

    // layer 1: thread owns unit j and rows (t >> 6) + 4 m
    {
        const int j = t & 63;
        float wj[D];
#pragma unroll
        for (int c = 0; c < D; ++c) wj[c] = S.th[OW1 + j * D + c];
        const float bj = S.th[OB1 + j];
#pragma unroll 4
        for (int i = t >> 6; i < TILE; i += 4) {
            float a = bj;
#pragma unroll
            for (int c = 0; c < D; ++c) a = fmaf(wj[c], S.z[i * D + c], a);
            S.h1[i * LD + j] = tanhf(a);
        }
    }
    __syncthreads();

    const int tx = t & 15, ty = t >> 4;   // 4 x 4 blocks of the 64 x 64 tiles
    // layer 2: a2[i][j] = b2[j] + sum_k h1[i][k] W2[j][k], rows 4 ty.., units 4 tx..
    {
        float acc[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = S.th[OB2 + 4 * tx + c];
#pragma unroll 8
        for (int k = 0; k < H; ++k) {
            const float4 wv = *reinterpret_cast<const float4*>(&S.w2t[k * H + 4 * tx]);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const float h = S.h1[(4 * ty + r) * LD + k];
                acc[r][0] = fmaf(h, wv.x, acc[r][0]);
                acc[r][1] = fmaf(h, wv.y, acc[r][1]);
                acc[r][2] = fmaf(h, wv.z, acc[r][2]);
                acc[r][3] = fmaf(h, wv.w, acc[r][3]);
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) S.h2[(4 * ty + r) * LD + 4 * tx + c] = tanhf(acc[r][c]);
    }
    __syncthreads();

    // output and dL/dg: one warp per 8 rows, lanes split the 64 units
    const int lane = t & 31, wid = t >> 5;
    {
        float sq = 0.f;
        for (int i = wid * 8; i < wid * 8 + 8; ++i) {
            float v = S.th[OW3 + lane] * S.h2[i * LD + lane] + S.th[OW3 + lane + 32] * S.h2[i * LD + lane + 32];
            for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            const float e = v + S.th[OB3] - S.y[i];
            if (lane == 0) S.d[i] = 2.f * e * inv_batch;
            sq = fmaf(e, e, sq);
        }
        if (lane == 0) S.red[wid] = sq;
    }
    __syncthreads();
    float* out = part + ((long long)f * nblk + tile) * kMlpStride;
    // dL/dw3[j] = sum_i d_i h2[i][j], dL/db3 = sum_i d_i, loss
    if (t < H) {
        float a = 0.f;
        for (int i = 0; i < TILE; ++i) a = fmaf(S.d[i], S.h2[i * LD + t], a);
        out[OW3 + t] = a;
    } else if (t == H) {
        float a = 0.f;
        for (int i = 0; i < TILE; ++i) a += S.d[i];
        out[OB3] = a;
    } else if (t == H + 1) {
        float a = 0.f;
        for (int q = 0; q < GRAD_THREADS / 32; ++q) a += S.red[q];
        out[kMlpParams] = a;
    }
    __syncthreads();
    // dL/da2 = d_i w3_j (1 - h2^2), in place
    {
        const int j = t & 63;
        const float w3 = S.th[OW3 + j];
        for (int i = t >> 6; i < TILE; i += 4) {
            const float h = S.h2[i * LD + j];
            S.h2[i * LD + j] = S.d[i] * w3 * (1.f - h * h);
        }
    }
    __syncthreads();
    // dL/dW2[j][k] = sum_i g2[i][j] h1[i][k] (units 4 ty.., inputs 4 tx..), dL/db2
    {
        float acc[4][4] = {};
        float db[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
        for (int i = 0; i < TILE; ++i) {
            const float4 g = *reinterpret_cast<const float4*>(&S.h2[i * LD + 4 * ty]);
            const float4 h = *reinterpret_cast<const float4*>(&S.h1[i * LD + 4 * tx]);
            const float gv[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                acc[r][0] = fmaf(gv[r], h.x, acc[r][0]);
                acc[r][1] = fmaf(gv[r], h.y, acc[r][1]);
                acc[r][2] = fmaf(gv[r], h.z, acc[r][2]);
                acc[r][3] = fmaf(gv[r], h.w, acc[r][3]);
                db[r] += gv[r];
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            *reinterpret_cast<float4*>(&out[OW2 + (4 * ty + r) * H + 4 * tx]) =
                make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
            if (tx == 0) out[OB2 + 4 * ty + r] = db[r];
        }
    }
    // dL/da1[i][k] = (sum_j g2[i][j] W2[j][k]) (1 - h1[i][k]^2), rows 4 ty.., inputs 4 tx..;
    // each thread overwrites only its own h1 entries, which no other thread reads in this phase
    __syncthreads();
    {
        float acc[4][4] = {};
#pragma unroll 8
        for (int j = 0; j < H; ++j) {
            const float4 wv = *reinterpret_cast<const float4*>(&S.th[OW2 + j * H + 4 * tx]);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const float g = S.h2[(4 * ty + r) * LD + j];
                acc[r][0] = fmaf(g, wv.x, acc[r][0]);
                acc[r][1] = fmaf(g, wv.y, acc[r][1]);
                acc[r][2] = fmaf(g, wv.z, acc[r][2]);
                acc[r][3] = fmaf(g, wv.w, acc[r][3]);
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float& h = S.h1[(4 * ty + r) * LD + 4 * tx + c];
                h = acc[r][c] * (1.f - h * h);
            }
    }
    __syncthreads();
    // dL/dW1[j][c] = sum_i g1[i][j] z[i][c], dL/db1[j] = sum_i g1[i][j]
    for (int o = t; o < H * (D + 1); o += GRAD_THREADS) {
        const int j = o & 63, c = o >> 6;
        float a = 0.f;
        if (c < D) {
            for (int i = 0; i < TILE; ++i) a = fmaf(S.h1[i * LD + j], S.z[i * D + c], a);
            out[OW1 + j * D + c] = a;
        } else {
            for (int i = 0; i < TILE; ++i) a += S.h1[i * LD + j];
            out[OB1 + j] = a;
        }
    }
}

// Sum of the tiles' partials in tile order (FP64): the batch gradient and mean loss.
__global__ void k_mlp_reduce(const float* __restrict__ part, int nblk, float inv_rows, float* __restrict__ grad,
                             float* __restrict__ loss)
{
    const int f = blockIdx.y;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > kMlpParams) return;
    double a = 0.0;
    for (int b = 0; b < nblk; ++b) a += (double)part[((long long)f * nblk + b) * kMlpStride + p];
    if (p < kMlpParams) {
        grad[(long long)f * kMlpStride + p] = (float)a;
    } else if (loss) {
        loss[f] = (float)(a * inv_rows);
    }
}

struct AdamArgs {
    float lr;        // step size of this update
    float c1, c2;    // 1 / (1 - beta1^t), 1 / (1 - beta2^t)
    float beta1, beta2, eps;
    float inv_rows;
    int nblk;
    long long step;  // index into the loss record
};

// Adam (Kingma & Ba 2015, Algorithm 1) on the batch gradient, reduced from
// the tiles' partials in tile order.
__global__ void k_mlp_adam(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ part, AdamArgs a, float* __restrict__ losses, long long steps)
{
    const int f = blockIdx.y;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > kMlpParams) return;
    double s = 0.0;
    for (int b = 0; b < a.nblk; ++b) s += (double)part[((long long)f * a.nblk + b) * kMlpStride + p];
    if (p == kMlpParams) {
        if (losses) losses[(long long)f * steps + a.step] = (float)(s * a.inv_rows);
        return;
    }
    const long long q = (long long)f * kMlpStride + p;
    const float g = (float)s;
    const float mm = a.beta1 * m[q] + (1.f - a.beta1) * g;
    const float vv = a.beta2 * v[q] + (1.f - a.beta2) * g * g;
    m[q] = mm;
    v[q] = vv;
    theta[q] -= a.lr * (mm * a.c1) / (sqrtf(vv * a.c2) + a.eps);
}

// ---------------------------------------------------------------- tabulation

__device__ __forceinline__ float tanh_approx(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

struct TabArgs {
    const float* theta;     // [2][kMlpStride]
    const float* norm;      // mu[5], s[5]
    const float4* nfa;      // (w, r, dw/dx, dw/dy) per node
    const float2* nfb;      // (dr/dx, dr/dy) per node
    int nx, ny, slices;
    double* table;          // (slices, ny, nx, 4)
    int* status;            // STATUS_TIMEOUT if a bounded wait runs out
    float tfrac[kMaxCvSlices];
};

// ---- the 64 x 64 layer on the fifth-generation tensor cores
//
// A CTA of 256 threads takes tiles of 128 points (point p = slice * nodes +
// node). Threads t and t + 128 share point t % 128, each with half of the 64
// units: they compute layer 1 and write three BF16 rows into shared memory: h1 = tanh(a1), u1 = (1 - h1^2) W1 dz/dx, v1 = (1 - h1^2) W1
// dz/dy. One thread issues the three products h1 W2^T, u1 W2^T, v1 W2^T as
// tcgen05.mma (M = 128, N = 64, K = 16, BF16 in, FP32 accumulate) into three
// 64-column accumulators in tensor memory, committed to an mbarrier; then
// warp w reads lanes 32 (w % 4) .. 32 (w % 4) + 31 (its threads' points),
// its half of the columns, back with tcgen05.ld and forms its half of
// d/dx = sum_j w3_j (1 - tanh(a2_j)^2) (W2 u1)_j, d/dy likewise; the halves
// meet in shared memory.
//
// Operands are K-major without swizzle: 8 x 8 BF16 core matrices of 128
// contiguous bytes (a row's 8 consecutive k at 16-byte pitch); core matrices
// adjacent in k are 128 B apart (leading byte offset), 8-row groups 1024 B
// (stride byte offset). Byte offset of (row r, k): (r / 8) 1024 + (k / 8) 128
// + (r % 8) 16 + (k % 8) 2.

constexpr int TC_ROWS = 128;                         // points per tile = MMA M
constexpr int TC_THREADS = 2 * TC_ROWS;              // two threads per point
constexpr int TC_OPERAND_BYTES = TC_ROWS * H * 2;    // one 128 x 64 BF16 operand
constexpr int TC_W2_BYTES = H * H * 2;
constexpr int TC_TMEM_COLS = 256;                    // three 64-column FP32 accumulators, rounded to a power of two
// Dynamic shared memory requested per CTA: above a third of the SM's 228 KB,
// so that at most two CTAs (2 x 256 tensor-memory columns of 512) share an SM
// and tcgen05.alloc never waits.
constexpr int TC_SMEM_REQUEST = 100 * 1024;
constexpr long long TC_WAIT_LIMIT = 1LL << 26;       // polls of the MMA mbarrier before giving up

struct TcSmem {
    alignas(1024) unsigned char a[3][TC_OPERAND_BYTES];
    alignas(1024) unsigned char b[TC_W2_BYTES];
    float w1[H * D], b1[H], b2[H], w3[H];
    float2 half_g[TC_ROWS];   // the second half's (d/dx, d/dy) partial sums
    alignas(8) unsigned long long mbar;
    uint32_t tmem;
    int abort;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t core_off(int r, int k) { return (r >> 3) * 1024 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2; }

// Shared-memory matrix descriptor: start, leading and stride byte offsets (all
// >> 4), the fixed 0b001 at bits 46-48, no swizzle (bits 61-63 zero).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ULL << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A
// and B (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits
// 17-22, M >> 4 at bits 24-28.
constexpr uint32_t tc_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        :: "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc) : "memory");
}

// 16 consecutive accumulator columns of the thread's lane; the wait is in the
// same statement, so no use of the registers can be scheduled before it.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n\ttcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

__global__ void __launch_bounds__(TC_THREADS) k_cv_tabulate(const TabArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    TcSmem& S = *reinterpret_cast<TcSmem*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const int f = blockIdx.y;
    const int t = threadIdx.x, warp = t >> 5;
    const int row = t % TC_ROWS, half = t / TC_ROWS;   // the point and the half of the units
    const float* th = a.theta + (long long)f * kMlpStride;

    // weights: layer 1 and the biases in FP32, W2 (B operand, rows n, k-major) in BF16
    for (int p = t; p < H * D; p += TC_THREADS) S.w1[p] = th[OW1 + p];
    for (int p = t; p < H; p += TC_THREADS) {
        S.b1[p] = th[OB1 + p];
        S.b2[p] = th[OB2 + p];
        S.w3[p] = th[OW3 + p];
    }
    for (int p = t; p < H * H / 8; p += TC_THREADS) {
        const int n = p / (H / 8), k0 = (p % (H / 8)) * 8;
        const float* wr = th + OW2 + n * H + k0;
        const uint4 v = make_uint4(pack_bf16(wr[0], wr[1]), pack_bf16(wr[2], wr[3]), pack_bf16(wr[4], wr[5]),
                                   pack_bf16(wr[6], wr[7]));
        *reinterpret_cast<uint4*>(S.b + core_off(n, k0)) = v;
    }
    if (t == 0) {
        S.abort = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&S.mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&S.tmem)), "n"(TC_TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = S.tmem;

    float mu[D], sc[D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
        mu[c] = a.norm[c];
        sc[c] = a.norm[D + c];
    }
    const long long nn = (long long)a.nx * a.ny;
    const long long points = nn * a.slices;
    const long long tiles = (points + TC_ROWS - 1) / TC_ROWS;
    constexpr uint32_t idesc = tc_idesc(TC_ROWS, H);
    uint32_t phase = 0;
    for (long long tl = blockIdx.x; tl < tiles; tl += gridDim.x) {
        // layer 1 of this thread's point (clamped in the ragged last tile; not written)
        const long long pt = tl * TC_ROWS + row;
        const long long pc = pt < points ? pt : points - 1;
        const int sl = (int)(pc / nn);
        const long long node = pc - (long long)sl * nn;
        {
            const int i = (int)(node % a.nx), j = (int)(node / a.nx);
            const float4 fa = a.nfa[node];
            const float2 fb = a.nfb[node];
            float z[D], dzx[D], dzy[D];
            z[0] = ((float)i / (float)(a.nx - 1) - mu[0]) * sc[0];
            z[1] = ((float)j / (float)(a.ny - 1) - mu[1]) * sc[1];
            z[2] = (a.tfrac[sl] - mu[2]) * sc[2];
            z[3] = (fa.x - mu[3]) * sc[3];
            z[4] = (fa.y - mu[4]) * sc[4];
            dzx[0] = sc[0]; dzx[1] = 0.f; dzx[2] = 0.f; dzx[3] = fa.z * sc[3]; dzx[4] = fb.x * sc[4];
            dzy[0] = 0.f; dzy[1] = sc[1]; dzy[2] = 0.f; dzy[3] = fa.w * sc[3]; dzy[4] = fb.y * sc[4];
#pragma unroll 1
            for (int k0 = half * (H / 2); k0 < (half + 1) * (H / 2); k0 += 8) {
                uint32_t ph[4], pu[4], pv[4];
#pragma unroll
                for (int e = 0; e < 8; e += 2) {
                    float hv[2], uv[2], vv[2];
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const float* w1 = S.w1 + (k0 + e + q) * D;
                        float a1 = S.b1[k0 + e + q];
#pragma unroll
                        for (int c = 0; c < D; ++c) a1 = fmaf(w1[c], z[c], a1);
                        const float t1 = tanh_approx(a1);
                        const float k1 = 1.f - t1 * t1;
                        float ux = 0.f, uy = 0.f;
#pragma unroll
                        for (int c = 0; c < D; ++c) {
                            ux = fmaf(w1[c], dzx[c], ux);
                            uy = fmaf(w1[c], dzy[c], uy);
                        }
                        hv[q] = t1;
                        uv[q] = k1 * ux;
                        vv[q] = k1 * uy;
                    }
                    ph[e / 2] = pack_bf16(hv[0], hv[1]);
                    pu[e / 2] = pack_bf16(uv[0], uv[1]);
                    pv[e / 2] = pack_bf16(vv[0], vv[1]);
                }
                const uint32_t o = core_off(row, k0);
                *reinterpret_cast<uint4*>(S.a[0] + o) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
                *reinterpret_cast<uint4*>(S.a[1] + o) = make_uint4(pu[0], pu[1], pu[2], pu[3]);
                *reinterpret_cast<uint4*>(S.a[2] + o) = make_uint4(pv[0], pv[1], pv[2], pv[3]);
            }
        }
        // the operands, written through the generic proxy, become visible to the tensor cores
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t bbase = smem_u32(S.b);
#pragma unroll
            for (int g = 0; g < 3; ++g) {
                const uint32_t abase = smem_u32(S.a[g]);
#pragma unroll
                for (int kk = 0; kk < H / 16; ++kk)
                    tc_mma(tmem + (uint32_t)(H * g), smem_desc(abase + 256 * kk, 128, 1024),
                           smem_desc(bbase + 256 * kk, 128, 1024), idesc, kk > 0 ? 1u : 0u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(&S.mbar)) : "memory");
        }
        // wait for the products (bounded)
        {
            uint32_t done = 0;
            for (long long it = 0; it < TC_WAIT_LIMIT && !done; ++it)
                asm volatile(
                    "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                    "selp.u32 %0, 1, 0, p;\n\t}"
                    : "=r"(done) : "r"(smem_u32(&S.mbar)), "r"(phase) : "memory");
            if (!done) S.abort = 1;
        }
        phase ^= 1u;
        __syncthreads();
        if (S.abort) {
            if (t == 0) atomicOr(a.status, STATUS_TIMEOUT);
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // epilogue: this thread's row from the three accumulators, 16 columns at a time
        float gx = 0.f, gy = 0.f;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
#pragma unroll 1
        for (int c0 = half * (H / 2); c0 < (half + 1) * (H / 2); c0 += 16) {
            float vh[16], vu[16], vv[16];
            tc_ld16(lane_base + (uint32_t)c0, vh);
            tc_ld16(lane_base + (uint32_t)(H + c0), vu);
            tc_ld16(lane_base + (uint32_t)(2 * H + c0), vv);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const float h2 = tanh_approx(vh[k] + S.b2[c0 + k]);
                const float wq = S.w3[c0 + k] * (1.f - h2 * h2);
                gx = fmaf(wq, vu[k], gx);
                gy = fmaf(wq, vv[k], gy);
            }
        }
        if (half == 1) S.half_g[row] = make_float2(gx, gy);
        __syncthreads();
        if (half == 0 && pt < points) {
            const float2 o2 = S.half_g[row];
            double* o = a.table + pt * 4 + 2 * f;
            o[0] = (double)(gx + o2.x);
            o[1] = (double)(gy + o2.y);
        }
        // every warp is done with the accumulators and the operands before the next tile
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "n"(TC_TMEM_COLS));
    }
}

int grid_for(long long n, int block)
{
    const long long b = (n + block - 1) / block;
    return (int)std::min<long long>(std::max<long long>(b, 1), 4096);
}

}  // namespace

// ---------------------------------------------------------------- launchers

cudaError_t launch_node_features(const float* w, int nx, int ny, double* w64, double* r64, double2* gw, float4* nfa,
                                 float2* nfb, cudaStream_t s)
{
    const long long n = (long long)nx * ny;
    k_node_w64<<<grid_for(n, 256), 256, 0, s>>>(w, n, w64);
    k_node_r<<<grid_for(n, 256), 256, 0, s>>>(w64, nx, ny, r64, gw);
    k_node_features<<<grid_for(n, 256), 256, 0, s>>>(w64, r64, gw, nx, ny, nfa, nfb);
    return cudaGetLastError();
}

cudaError_t launch_field_grad(const double* xi, const double* eta, int nx, int ny, double* table, cudaStream_t s)
{
    const long long n = (long long)nx * ny;
    k_field_grad<<<grid_for(n, 256), 256, 0, s>>>(xi, eta, nx, ny, table);
    return cudaGetLastError();
}

cudaError_t launch_cv_smooth(const double* table, int nx, int ny, int order, float4* tmp, float4* cells,
                             cudaStream_t s)
{
    if (order < 1 || order > kCvMaxOrder || (order & 1) == 0) return cudaErrorInvalidValue;
    BinomWeights W{};
    W.order = order;
    double c = 1.0;   // C(order, m)
    for (int m = 0; m <= order; ++m) {
        W.w[m] = (float)std::ldexp(c, -order);
        c = c * (double)(order - m) / (double)(m + 1);
    }
    const long long nxr = (long long)(nx - 1) * ny, nc = (long long)(nx - 1) * (ny - 1);
    k_cv_smooth_x<<<grid_for(nxr, 256), 256, 0, s>>>(table, nx, ny, W, tmp);
    k_cv_smooth_y<<<grid_for(nc, 256), 256, 0, s>>>(tmp, nx, ny, W, cells);
    return cudaGetLastError();
}

cudaError_t launch_cv_scatter(const double* xs, const double* ys, const double* yxi, const double* yeta,
                              const float4* nfa, int nx, int ny, int k, int K, int M, float* feats, float* targets,
                              cudaStream_t s)
{
    k_cv_scatter<<<grid_for(M, 256), 256, 0, s>>>(xs, ys, yxi, yeta, nfa, nx, ny, k, K, M, feats, targets);
    return cudaGetLastError();
}

size_t mlp_norm_scratch_doubles() { return (size_t)MOM_BLOCKS * D + D; }

cudaError_t launch_mlp_norm(const float* feats, long long n, double* scratch, float* norm, cudaStream_t s)
{
    double* part = scratch;
    double* mu = scratch + MOM_BLOCKS * D;
    const int nb = (int)std::min<long long>(MOM_BLOCKS, std::max<long long>(1, (n + 255) / 256));
    k_moments<<<nb, 256, 0, s>>>(feats, n, mu, 0, part);
    k_norm<<<1, 32, 0, s>>>(part, nb, n, mu, 0, norm);
    k_moments<<<nb, 256, 0, s>>>(feats, n, mu, 1, part);
    k_norm<<<1, 32, 0, s>>>(part, nb, n, mu, 1, norm);
    return cudaGetLastError();
}

int mlp_tile_rows() { return TILE; }

cudaError_t launch_mlp_grad(const float* theta, const float* norm, const float* feats, const float* targets,
                            long long row0, long long rows, float inv_batch, float* part, cudaStream_t s)
{
    const size_t smem = sizeof(GradSmem);
    cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)(rows / TILE), 2);
    k_mlp_grad<<<grid, GRAD_THREADS, smem, s>>>(theta, norm, feats, targets, row0, inv_batch, part);
    return cudaGetLastError();
}

cudaError_t launch_mlp_reduce(const float* part, int nblk, float inv_rows, float* grad, float* loss, cudaStream_t s)
{
    const dim3 grid((kMlpParams + 1 + 255) / 256, 2);
    k_mlp_reduce<<<grid, 256, 0, s>>>(part, nblk, inv_rows, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* theta, float* m, float* v, const float* part, int nblk, double lr, long long t,
                            float inv_rows, float* losses, long long steps, long long step, cudaStream_t s)
{
    AdamArgs a;
    const double b1 = 0.9, b2 = 0.999;
    a.lr = (float)lr;
    a.c1 = (float)(1.0 / (1.0 - std::pow(b1, (double)t)));
    a.c2 = (float)(1.0 / (1.0 - std::pow(b2, (double)t)));
    a.beta1 = (float)b1;
    a.beta2 = (float)b2;
    a.eps = 1e-8f;
    a.inv_rows = inv_rows;
    a.nblk = nblk;
    a.step = step;
    const dim3 grid((kMlpParams + 1 + 255) / 256, 2);
    k_mlp_adam<<<grid, 256, 0, s>>>(theta, m, v, part, a, losses, steps);
    return cudaGetLastError();
}

cudaError_t launch_cv_tabulate(const float* theta, const float* norm, const float4* nfa, const float2* nfb, int nx,
                               int ny, int slices, const float* tfrac, double* table, int* status, int sm_count,
                               cudaStream_t s)
{
    static_assert(sizeof(TcSmem) + 1024 <= TC_SMEM_REQUEST, "tabulation shared memory");
    TabArgs a{};
    a.theta = theta;
    a.norm = norm;
    a.nfa = nfa;
    a.nfb = nfb;
    a.nx = nx;
    a.ny = ny;
    a.slices = slices;
    a.table = table;
    a.status = status;
    for (int q = 0; q < slices && q < kMaxCvSlices; ++q) a.tfrac[q] = tfrac[q];
    const long long tiles = ((long long)nx * ny * slices + TC_ROWS - 1) / TC_ROWS;
    if (tiles <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_cv_tabulate, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_REQUEST);
    if (e != cudaSuccess) return e;
    // two CTAs per SM and network at most (tensor-memory columns), both networks side by side
    const int grid = (int)std::min<long long>(tiles, (long long)sm_count);
    k_cv_tabulate<<<dim3(grid, 2), TC_THREADS, TC_SMEM_REQUEST, s>>>(a);
    return cudaGetLastError();
}

}  // namespace sdd
