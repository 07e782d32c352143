// fields.cu -- per-mesh-step field preparation (the path kernel's tables).
//
//  * drift b = -grad w / w at the grid nodes by finite differences (Eq. 6;
//    Sec. 4 "derivatives ... approximated using finite differences"):
//    second-order central differences inside, second-order one-sided
//    differences (-3 w0 + 4 w1 - w2) / 2h on the edges, in double precision;
//  * per cell, the bilinear interpolant of b and of (xi, eta) written as
//    a0 + a1 s + a2 t + a3 s t over the cell's local coordinates (s, t), with
//    a0 = f00, a1 = f10 - f00, a2 = f01 - f00, a3 = f11 - f10 - f01 + f00,
//    formed in double and stored in single precision, the two components
//    interleaved (Sec. 4: bilinear interpolation between grid points);
//  * the boundary data of Sec. 3: xi = 0 / 1 on x = 0 / 1, eta = 0 / 1 on
//    y = 0 / 1, and on the other faces the 1D Winslow solution
//    int_0^s w / int_0^1 w (cumulative trapezoid, double precision).
#include <cuda_fp16.h>

#include "common.cuh"

namespace sdd {

namespace {

__device__ __forceinline__ double2 node_drift(const float* __restrict__ w, int nx, int ny, int i, int j,
                                              double rx, double ry)
{
    // rx = 1 / (2 hx) = (nx - 1) / 2, ry likewise
    const float* row = w + (long long)j * nx;
    double wx, wy;
    if (i == 0)
        wx = (-3.0 * (double)row[0] + 4.0 * (double)row[1] - (double)row[2]) * rx;
    else if (i == nx - 1)
        wx = (3.0 * (double)row[nx - 1] - 4.0 * (double)row[nx - 2] + (double)row[nx - 3]) * rx;
    else
        wx = ((double)row[i + 1] - (double)row[i - 1]) * rx;
    const float* col = w + i;
    if (j == 0)
        wy = (-3.0 * (double)col[0] + 4.0 * (double)col[(long long)nx] - (double)col[2LL * nx]) * ry;
    else if (j == ny - 1)
        wy = (3.0 * (double)col[(long long)(ny - 1) * nx] - 4.0 * (double)col[(long long)(ny - 2) * nx] +
              (double)col[(long long)(ny - 3) * nx]) * ry;
    else
        wy = ((double)col[(long long)(j + 1) * nx] - (double)col[(long long)(j - 1) * nx]) * ry;
    const double wc = (double)row[i];
    return make_double2(-wx / wc, -wy / wc);
}

// Bilinear coefficients of two fields u, v on one cell, interleaved so that one
// paired single-precision FMA evaluates both: (a0u, a0v, a1u, a1v) and
// (a2u, a2v, a3u, a3v).
__device__ __forceinline__ void bilinear_coefs2(double u00, double u10, double u01, double u11, double v00,
                                                double v10, double v01, double v11, float4& lo, float4& hi)
{
    lo = make_float4((float)u00, (float)v00, (float)(u10 - u00), (float)(v10 - v00));
    hi = make_float4((float)(u01 - u00), (float)(v01 - v00), (float)((u11 - u10) - (u01 - u00)),
                     (float)((v11 - v10) - (v01 - v00)));
}

__device__ __forceinline__ bool bad_w(float v) { return !(v > 0.0f) || !isfinite(v); }

// One block per 32 x 8 cells: the drift at the tile's 33 x 9 nodes once (in
// shared memory, double precision), then each cell's records.
constexpr int PREP_TX = 32, PREP_TY = 8;

__global__ void __launch_bounds__(PREP_TX * PREP_TY) k_prep_cells(const float* __restrict__ w,
                                                                  const double* __restrict__ xi,
                                                                  const double* __restrict__ eta, int nx, int ny,
                                                                  float4* __restrict__ bcoef,
                                                                  float4* __restrict__ fcoef, int* status)
{
    __shared__ double2 bn[PREP_TY + 1][PREP_TX + 1];
    const int ix0 = blockIdx.x * PREP_TX, iy0 = blockIdx.y * PREP_TY;
    const int ix = ix0 + threadIdx.x, iy = iy0 + threadIdx.y;
    const bool cell_in = ix < nx - 1 && iy < ny - 1;
    if (bcoef) {
        const double rx = 0.5 * (double)(nx - 1), ry = 0.5 * (double)(ny - 1);
        const int tid = threadIdx.y * PREP_TX + threadIdx.x;
        for (int k = tid; k < (PREP_TX + 1) * (PREP_TY + 1); k += PREP_TX * PREP_TY) {
            const int ti = k % (PREP_TX + 1), tj = k / (PREP_TX + 1);
            const int i = ix0 + ti, j = iy0 + tj;
            if (i < nx && j < ny) bn[tj][ti] = node_drift(w, nx, ny, i, j, rx, ry);
        }
        __syncthreads();
        if (cell_in) {
            // every node is checked by the cell that has it as lower-left corner,
            // the last row and column by the cells next to them
            bool bad = bad_w(w[(long long)iy * nx + ix]);
            if (ix == nx - 2) bad |= bad_w(w[(long long)iy * nx + ix + 1]);
            if (iy == ny - 2) bad |= bad_w(w[(long long)(iy + 1) * nx + ix]);
            if (ix == nx - 2 && iy == ny - 2) bad |= bad_w(w[(long long)(iy + 1) * nx + ix + 1]);
            if (bad) atomicOr(status, STATUS_BAD_W);
            const int tx = threadIdx.x, ty = threadIdx.y;
            const double2 b00 = bn[ty][tx], b10 = bn[ty][tx + 1], b01 = bn[ty + 1][tx], b11 = bn[ty + 1][tx + 1];
            const long long cell = (long long)iy * (nx - 1) + ix;
            bilinear_coefs2(b00.x, b10.x, b01.x, b11.x, b00.y, b10.y, b01.y, b11.y, bcoef[2 * cell + 0],
                            bcoef[2 * cell + 1]);
        }
    }
    if (fcoef && cell_in) {
        const long long cell = (long long)iy * (nx - 1) + ix;
        const long long n00 = (long long)iy * nx + ix;
        const long long n01 = n00 + nx;
        bilinear_coefs2(xi[n00], xi[n00 + 1], xi[n01], xi[n01 + 1], eta[n00], eta[n00 + 1], eta[n01], eta[n01 + 1],
                        fcoef[2 * cell + 0], fcoef[2 * cell + 1]);
    }
}

// Control-variate table: node values (slice, j, i, 4) of the two models'
// gradients -> one 32-byte record per slice and cell holding the cell's four
// corner values in half precision (round to nearest even): the xi model's
// (d/dx, d/dy) at corners 00, 10, 01, 11, then the eta model's. The model the
// estimator uses is the bilinear interpolation of these rounded node values
// (continuous across cells: neighbouring cells hold the same rounded values).
__global__ void k_cv_cells(const double* __restrict__ g, int slices, int nx, int ny, uint4* __restrict__ cv)
{
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int iy = blockIdx.y * blockDim.y + threadIdx.y;
    const int q = blockIdx.z;
    if (ix >= nx - 1 || iy >= ny - 1 || q >= slices) return;
    const double* T = g + (long long)q * nx * ny * 4;
    const long long n00 = (long long)iy * nx + ix;
    const long long corner[4] = {n00, n00 + 1, n00 + nx, n00 + nx + 1};
    const long long cell = (long long)q * (nx - 1) * (ny - 1) + (long long)iy * (nx - 1) + ix;
    uint32_t w[8];
    for (int f = 0; f < 2; ++f)
        for (int k = 0; k < 4; ++k) {
            const double* v = T + 4 * corner[k] + 2 * f;
            const __half hx = __double2half(v[0]), hy = __double2half(v[1]);
            w[4 * f + k] = (uint32_t)__half_as_ushort(hx) | ((uint32_t)__half_as_ushort(hy) << 16);
        }
    cv[2 * cell + 0] = make_uint4(w[0], w[1], w[2], w[3]);
    cv[2 * cell + 1] = make_uint4(w[4], w[5], w[6], w[7]);
}

// Cumulative trapezoid of one line of w, normalised by its total, by one warp:
// each lane sums a contiguous run of intervals, the run totals are scanned
// across the warp, then each lane writes its run.
__device__ void warp_cumtrapz(const float* __restrict__ v, long long stride, int n, double* __restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int intervals = n - 1;
    const int run = (intervals + 31) / 32;
    const int k0 = 1 + lane * run;
    const int k1 = min(k0 + run, n);
    double mine = 0.0;
    for (int k = k0; k < k1; ++k) mine += 0.5 * ((double)v[(k - 1) * stride] + (double)v[k * stride]);
    double incl = mine;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const double o = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += o;
    }
    const double total = __shfl_sync(0xffffffffu, incl, 31);
    double acc = incl - mine;
    if (lane == 0) out[0] = 0.0;
    for (int k = k0; k < k1; ++k) {
        acc += 0.5 * ((double)v[(k - 1) * stride] + (double)v[k * stride]);
        out[k] = acc / total;
    }
}

__global__ void k_winslow_faces(const float* __restrict__ w, int nx, int ny, double* __restrict__ faces,
                                float* __restrict__ faces32)
{
    const long long per_field = 2LL * ny + 2LL * nx;
    double* xl = faces;
    double* xr = faces + ny;
    double* xb = faces + 2LL * ny;
    double* xt = faces + 2LL * ny + nx;
    double* el = faces + per_field;
    double* er = faces + per_field + ny;
    double* eb = faces + per_field + 2LL * ny;
    double* et = faces + per_field + 2LL * ny + nx;
    const int warp = threadIdx.x >> 5;
    if (warp == 0) warp_cumtrapz(w, 1, nx, xb);                                   // xi on y = 0
    if (warp == 1) warp_cumtrapz(w + (long long)(ny - 1) * nx, 1, nx, xt);        // xi on y = 1
    if (warp == 2) warp_cumtrapz(w, nx, ny, el);                                  // eta on x = 0
    if (warp == 3) warp_cumtrapz(w + (nx - 1), nx, ny, er);                       // eta on x = 1
    for (int k = threadIdx.x; k < ny; k += blockDim.x) {
        xl[k] = 0.0;
        xr[k] = 1.0;
    }
    for (int k = threadIdx.x; k < nx; k += blockDim.x) {
        eb[k] = 0.0;
        et[k] = 1.0;
    }
    if (faces32) {
        // the single-precision copy the path kernel scores exits with
        __syncthreads();
        for (long long k = threadIdx.x; k < 2 * per_field; k += blockDim.x) faces32[k] = (float)faces[k];
    }
}

__global__ void k_faces32(const double* __restrict__ f64, float* __restrict__ f32, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) f32[k] = (float)f64[k];
}

// Zero map of the drift records: one block per map word (32 segments of 2^zshift consecutive cells in
// row-major order); bit k set when a record of segment k has a nonzero coefficient. The last word's bits
// past the last cell stay clear (no path reaches those cells).
__global__ void __launch_bounds__(256) k_drift_zmap(const float4* __restrict__ bcoef, long long cells,
                                                    uint32_t zshift, uint32_t* __restrict__ zmap)
{
    __shared__ int nz[32];
    if (threadIdx.x < 32) nz[threadIdx.x] = 0;
    __syncthreads();
    const long long c0 = (long long)blockIdx.x << (zshift + 5);
    const long long span = 32LL << zshift;
    for (long long k = threadIdx.x; k < span; k += blockDim.x) {
        const long long c = c0 + k;
        if (c >= cells) break;
        const float4 lo = bcoef[2 * c], hi = bcoef[2 * c + 1];
        if (lo.x != 0.f || lo.y != 0.f || lo.z != 0.f || lo.w != 0.f || hi.x != 0.f || hi.y != 0.f ||
            hi.z != 0.f || hi.w != 0.f)
            nz[k >> zshift] = 1;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const unsigned word = __ballot_sync(0xffffffffu, nz[threadIdx.x] != 0);
        if (threadIdx.x == 0) zmap[blockIdx.x] = word;
    }
}

}  // namespace

cudaError_t launch_prep_cells(const float* w, const double* xi, const double* eta, int nx, int ny, float4* bcoef,
                              float4* fcoef, int* status, cudaStream_t s, uint32_t* zmap, uint32_t zshift)
{
    const dim3 block(PREP_TX, PREP_TY);
    const dim3 grid((nx - 1 + PREP_TX - 1) / PREP_TX, (ny - 1 + PREP_TY - 1) / PREP_TY);
    k_prep_cells<<<grid, block, 0, s>>>(w, xi, eta, nx, ny, bcoef, fcoef, status);
    if (bcoef && zmap) {
        const long long cells = (long long)(nx - 1) * (ny - 1);
        k_drift_zmap<<<zmap_words(cells, zshift), 256, 0, s>>>(bcoef, cells, zshift, zmap);
    }
    return cudaGetLastError();
}

cudaError_t launch_cv_cells(const double* grad, int slices, int nx, int ny, uint4* cvcoef, cudaStream_t s)
{
    const dim3 block(32, 8);
    const dim3 grid((nx - 1 + 31) / 32, (ny - 1 + 7) / 8, slices);
    k_cv_cells<<<grid, block, 0, s>>>(grad, slices, nx, ny, cvcoef);
    return cudaGetLastError();
}

cudaError_t launch_winslow_faces(const float* w, int nx, int ny, double* faces64, float* faces32, cudaStream_t s)
{
    k_winslow_faces<<<1, 128, 0, s>>>(w, nx, ny, faces64, faces32);
    return cudaGetLastError();
}

cudaError_t launch_faces32(const double* faces64, float* faces32, int n, cudaStream_t s)
{
    k_faces32<<<(n + 255) / 256, 256, 0, s>>>(faces64, faces32, n);
    return cudaGetLastError();
}

}  // namespace sdd
