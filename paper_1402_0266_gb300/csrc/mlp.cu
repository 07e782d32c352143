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
//                               on the tensor cores (BF16 in, FP32 accumulate,
//                               mma.sync m16n8k16), everything else FP32.
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

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

struct TabArgs {
    const float* theta;     // [2][kMlpStride]
    const float* norm;      // mu[5], s[5]
    const float4* nfa;      // (w, r, dw/dx, dw/dy) per node
    const float2* nfb;      // (dr/dx, dr/dy) per node
    int nx, ny, slices;
    double* table;          // (slices, ny, nx, 4)
    float tfrac[kMaxCvSlices];
};

constexpr int TAB_WARPS = 4;

// One warp evaluates 16 nodes at a time for one network (blockIdx.y). Rows of
// the m16n8k16 A operand are nodes; three operands per tile: h1 = tanh(a1),
// u1 = (1 - h1^2) W1 dz/dx, v1 = (1 - h1^2) W1 dz/dy. Lane (g, q) = (lane / 4,
// lane % 4) holds rows g, g + 8 and, per 16-wide k step kk, the units
// 16 kk + 2 q + {0, 1, 8, 9} of A, and after the MMA the units 8 n + 2 q + {0, 1}
// of every 8-wide n tile. W2 (B operand, B[k][n] = W2[n][k]) stays in registers.
__global__ void __launch_bounds__(TAB_WARPS * 32) k_cv_tabulate(const TabArgs a)
{
    __shared__ float sw1[H * D], sb1[H], sb2[H], sw3[H];
    const int f = blockIdx.y;
    const float* th = a.theta + (long long)f * kMlpStride;
    for (int p = threadIdx.x; p < H * D; p += blockDim.x) sw1[p] = th[OW1 + p];
    for (int p = threadIdx.x; p < H; p += blockDim.x) {
        sb1[p] = th[OB1 + p];
        sb2[p] = th[OB2 + p];
        sw3[p] = th[OW3 + p];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    uint32_t B[8][4][2];
#pragma unroll
    for (int n = 0; n < 8; ++n)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const float* wr = th + OW2 + (8 * n + g) * H + 16 * kk + 2 * q;
            B[n][kk][0] = pack_bf16(wr[0], wr[1]);
            B[n][kk][1] = pack_bf16(wr[8], wr[9]);
        }
    float mu[D], sc[D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
        mu[c] = a.norm[c];
        sc[c] = a.norm[D + c];
    }
    const long long nn = (long long)a.nx * a.ny;
    const long long tiles = (nn + 15) / 16;
    const long long warp0 = (long long)blockIdx.x * TAB_WARPS + (threadIdx.x >> 5);
    const long long nwarps = (long long)gridDim.x * TAB_WARPS;
    for (long long tl = warp0; tl < tiles; tl += nwarps) {
        // the lane's two nodes (clamped in the ragged last tile; their results are not written)
        long long node[2];
        float z[2][D], dzx[2][D], dzy[2][D];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            node[h] = tl * 16 + g + 8 * h;
            const long long k = node[h] < nn ? node[h] : nn - 1;
            const int i = (int)(k % a.nx), j = (int)(k / a.nx);
            const float4 fa = a.nfa[k];
            const float2 fb = a.nfb[k];
            z[h][2] = 0.f;   // the time input is per slice
            z[h][0] = ((float)i / (float)(a.nx - 1) - mu[0]) * sc[0];
            z[h][1] = ((float)j / (float)(a.ny - 1) - mu[1]) * sc[1];
            z[h][3] = (fa.x - mu[3]) * sc[3];
            z[h][4] = (fa.y - mu[4]) * sc[4];
            dzx[h][0] = sc[0]; dzx[h][1] = 0.f; dzx[h][2] = 0.f; dzx[h][3] = fa.z * sc[3]; dzx[h][4] = fb.x * sc[4];
            dzy[h][0] = 0.f; dzy[h][1] = sc[1]; dzy[h][2] = 0.f; dzy[h][3] = fa.w * sc[3]; dzy[h][4] = fb.y * sc[4];
        }
        for (int sl = 0; sl < a.slices; ++sl) {
            const float zt = (a.tfrac[sl] - mu[2]) * sc[2];
            // layer 1 for the lane's units, packed straight into the A operands
            uint32_t Ah[4][4], Au[4][4], Av[4][4];
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
#pragma unroll
                for (int hi = 0; hi < 2; ++hi)       // units +0,+1 (hi = 0) or +8,+9 (hi = 1)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {    // row g or g + 8
                        float hv[2], uv[2], vv[2];
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const int j = 16 * kk + 2 * q + 8 * hi + e;
                            const float* w1 = sw1 + j * D;
                            float a1 = sb1[j];
                            a1 = fmaf(w1[0], z[h][0], a1);
                            a1 = fmaf(w1[1], z[h][1], a1);
                            a1 = fmaf(w1[2], zt, a1);
                            a1 = fmaf(w1[3], z[h][3], a1);
                            a1 = fmaf(w1[4], z[h][4], a1);
                            const float t1 = tanh_approx(a1);
                            const float k1 = 1.f - t1 * t1;
                            float ux = w1[0] * dzx[h][0] + w1[3] * dzx[h][3] + w1[4] * dzx[h][4];
                            float uy = w1[1] * dzy[h][1] + w1[3] * dzy[h][3] + w1[4] * dzy[h][4];
                            hv[e] = t1;
                            uv[e] = k1 * ux;
                            vv[e] = k1 * uy;
                        }
                        const int r = 2 * hi + h;    // register order: (g, lo) (g+8, lo) (g, hi) (g+8, hi)
                        Ah[kk][r] = pack_bf16(hv[0], hv[1]);
                        Au[kk][r] = pack_bf16(uv[0], uv[1]);
                        Av[kk][r] = pack_bf16(vv[0], vv[1]);
                    }
            // layer 2: h1 W2^T, then the lane's w3_j (1 - h2_j^2) weights
            float wq[8][4];
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) mma_bf16(c, Ah[kk], B[n][kk][0], B[n][kk][1]);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int j = 8 * n + 2 * q + (e & 1);
                    const float h2 = tanh_approx(c[e] + sb2[j]);
                    wq[n][e] = sw3[j] * (1.f - h2 * h2);
                }
            }
            // d/dx and d/dy: sum_j w3_j (1 - h2_j^2) (W2 u1)_j, likewise for v1
            float gx[2] = {0.f, 0.f}, gy[2] = {0.f, 0.f};
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                float cu[4] = {0.f, 0.f, 0.f, 0.f}, cv[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    mma_bf16(cu, Au[kk], B[n][kk][0], B[n][kk][1]);
                    mma_bf16(cv, Av[kk], B[n][kk][0], B[n][kk][1]);
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    gx[e >> 1] = fmaf(wq[n][e], cu[e], gx[e >> 1]);
                    gy[e >> 1] = fmaf(wq[n][e], cv[e], gy[e >> 1]);
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                gx[h] += __shfl_xor_sync(0xffffffffu, gx[h], 1);
                gx[h] += __shfl_xor_sync(0xffffffffu, gx[h], 2);
                gy[h] += __shfl_xor_sync(0xffffffffu, gy[h], 1);
                gy[h] += __shfl_xor_sync(0xffffffffu, gy[h], 2);
            }
            if (q == 0) {
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    if (node[h] < nn) {
                        double* o = a.table + ((long long)sl * nn + node[h]) * 4 + 2 * f;
                        o[0] = (double)gx[h];
                        o[1] = (double)gy[h];
                    }
            }
        }
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
                               int ny, int slices, const float* tfrac, double* table, int sm_count, cudaStream_t s)
{
    TabArgs a{};
    a.theta = theta;
    a.norm = norm;
    a.nfa = nfa;
    a.nfb = nfb;
    a.nx = nx;
    a.ny = ny;
    a.slices = slices;
    a.table = table;
    for (int q = 0; q < slices && q < kMaxCvSlices; ++q) a.tfrac[q] = tfrac[q];
    const long long tiles = ((long long)nx * ny + 15) / 16;
    const long long blocks = (tiles + TAB_WARPS - 1) / TAB_WARPS;
    const int grid = (int)std::min<long long>(blocks, (long long)sm_count * 8);
    k_cv_tabulate<<<dim3(grid, 2), TAB_WARPS * 32, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace sdd
