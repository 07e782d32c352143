// solve.cu -- the deterministic single-domain solves (Sec. 4).
//
// The paper solves an implicit finite-difference discretisation of Eq. (3)
// on each subdomain, with the interface values as Dirichlet data, and gives no
// stencil. Since -(1/w) grad w . grad xi + lap xi = w div((1/w) grad xi), the
// implicit Euler step multiplied by 1/w reads, at an unknown node,
//
//   xi_ij / (w_ij Dt) + sum_nb c_nb (xi_ij - xi_nb) = xi^{n-1}_ij / (w_ij Dt),
//   c_nb = 1 / (wbar h^2),  wbar = (w_ij + w_nb) / 2,
//
// a symmetric positive definite M-matrix, solved here per subdomain and field
// by Jacobi-preconditioned conjugate gradients in double precision. Each
// system is one thread block running the whole iteration; the block's
// unknowns never leave L1/L2. The iteration stops at ||r|| <= rtol ||b|| or
// after max_iter iterations (then a status bit is set; it never hangs).
#include "common.cuh"

namespace sdd {

namespace {

constexpr int SOLVE_THREADS = 1024;

__global__ void k_solve_setup(const float* __restrict__ w, const double* __restrict__ pxi,
                              const double* __restrict__ peta, int nx, int ny, double Dt, double* __restrict__ cx,
                              double* __restrict__ cy, double* __restrict__ dg, double* __restrict__ rhs0)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= nx || j >= ny) return;
    const long long n = (long long)j * nx + i;
    const double ihx2 = (double)(nx - 1) * (double)(nx - 1);
    const double ihy2 = (double)(ny - 1) * (double)(ny - 1);
    const double wc = (double)w[n];
    const double e = (i + 1 < nx) ? ihx2 / (0.5 * (wc + (double)w[n + 1])) : 0.0;
    const double no = (j + 1 < ny) ? ihy2 / (0.5 * (wc + (double)w[n + nx])) : 0.0;
    cx[n] = e;
    cy[n] = no;
    double d = 1.0 / (wc * Dt);
    rhs0[n] = pxi[n] * d;
    rhs0[(long long)nx * ny + n] = peta[n] * d;
    if (i > 0 && i + 1 < nx && j > 0 && j + 1 < ny) {
        const double wwest = (double)w[n - 1], wsouth = (double)w[n - nx];
        d += e + no + ihx2 / (0.5 * (wc + wwest)) + ihy2 / (0.5 * (wc + wsouth));
    }
    dg[n] = d;
}

// Dirichlet data of the new fields: the face data on the outer boundary, the
// interface estimates on the interface lines, and the previous values
// (initial guess) elsewhere.
__global__ void k_dirichlet(const double* __restrict__ faces, const double* __restrict__ pxi,
                            const double* __restrict__ peta, int nx, int ny, double* __restrict__ xo,
                            double* __restrict__ eo)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= nx || j >= ny) return;
    const long long n = (long long)j * nx + i;
    const long long per_field = 2LL * ny + 2LL * nx;
    double a = pxi[n], b = peta[n];
    // faces: left (x = 0, by j), right, bottom (y = 0, by i), top; first match wins
    if (i == 0) { a = faces[j]; b = faces[per_field + j]; }
    else if (i == nx - 1) { a = faces[ny + j]; b = faces[per_field + ny + j]; }
    else if (j == 0) { a = faces[2LL * ny + i]; b = faces[per_field + 2LL * ny + i]; }
    else if (j == ny - 1) { a = faces[2LL * ny + nx + i]; b = faces[per_field + 2LL * ny + nx + i]; }
    xo[n] = a;
    eo[n] = b;
}

__global__ void k_scatter_iface(const double* __restrict__ vx, const double* __restrict__ ve,
                                const int32_t* __restrict__ idx, int n, double* __restrict__ xo,
                                double* __restrict__ eo)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    xo[idx[k]] = vx[k];
    eo[idx[k]] = ve[k];
}

__device__ __forceinline__ double block_sum(double v, double* sh)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    const int nw = blockDim.x >> 5;
    for (int k = 0; k < nw; ++k) t += sh[k];  // same order in every thread
    return t;
}

__device__ __forceinline__ void block_sum2(double& a, double& b, double* sh)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, off);
        b += __shfl_xor_sync(0xffffffffu, b, off);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) {
        sh[warp] = a;
        sh[32 + warp] = b;
    }
    __syncthreads();
    double ta = 0.0, tb = 0.0;
    const int nw = blockDim.x >> 5;
    for (int k = 0; k < nw; ++k) {
        ta += sh[k];
        tb += sh[32 + k];
    }
    a = ta;
    b = tb;
}

__global__ void __launch_bounds__(SOLVE_THREADS) k_pcg(const SolveArgs a)
{
    __shared__ double sh[64];
    const SolveSys S = a.sys[blockIdx.x];
    const int nx = a.nx;
    const int mx = S.i1 - S.i0, my = S.j1 - S.j0;
    const int m = mx * my;
    double* __restrict__ x = a.x[S.field];
    double* __restrict__ r = a.r[S.field];
    double* __restrict__ p = a.p[S.field];
    double* __restrict__ q = a.q[S.field];
    const double* __restrict__ rhs = a.rhs0 + (long long)S.field * nx * a.ny;
    const double* __restrict__ cx = a.cx;
    const double* __restrict__ cy = a.cy;
    const double* __restrict__ dg = a.dg;

    // r = b - A x over the block, with x's Dirichlet ring fixed; z = r / diag; p = z
    double bb = 0.0, rz = 0.0;
    for (int u = threadIdx.x; u < m; u += blockDim.x) {
        const int i = S.i0 + u % mx, j = S.j0 + u / mx;
        const long long n = (long long)j * nx + i;
        // b: the rhs plus the Dirichlet neighbours
        double b = rhs[n];
        const double ax = dg[n] * x[n] - cx[n - 1] * x[n - 1] - cx[n] * x[n + 1] - cy[n - nx] * x[n - nx] -
                          cy[n] * x[n + nx];
        double bd = 0.0;
        if (i == S.i0) bd += cx[n - 1] * x[n - 1];
        if (i == S.i1 - 1) bd += cx[n] * x[n + 1];
        if (j == S.j0) bd += cy[n - nx] * x[n - nx];
        if (j == S.j1 - 1) bd += cy[n] * x[n + nx];
        b += bd;
        const double rr = rhs[n] - ax;
        const double z = rr / dg[n];
        r[n] = rr;
        p[n] = z;
        bb += b * b;
        rz += rr * z;
    }
    block_sum2(bb, rz, sh);
    const double bnorm = sqrt(bb);
    double rr_norm2 = 0.0;
    {
        double t = 0.0;
        for (int u = threadIdx.x; u < m; u += blockDim.x) {
            const int i = S.i0 + u % mx, j = S.j0 + u / mx;
            const double v = r[(long long)j * nx + i];
            t += v * v;
        }
        rr_norm2 = block_sum(t, sh);
    }
    int it = 0;
    if (sqrt(rr_norm2) > a.rtol * bnorm) {
        for (it = 1; it <= a.max_iter; ++it) {
            __syncthreads();  // p complete
            double pq = 0.0;
            for (int u = threadIdx.x; u < m; u += blockDim.x) {
                const int i = S.i0 + u % mx, j = S.j0 + u / mx;
                const long long n = (long long)j * nx + i;
                // p is zero outside the block (Dirichlet nodes): only block neighbours count
                double v = dg[n] * p[n];
                if (i > S.i0) v -= cx[n - 1] * p[n - 1];
                if (i < S.i1 - 1) v -= cx[n] * p[n + 1];
                if (j > S.j0) v -= cy[n - nx] * p[n - nx];
                if (j < S.j1 - 1) v -= cy[n] * p[n + nx];
                q[n] = v;
                pq += p[n] * v;
            }
            pq = block_sum(pq, sh);
            const double alpha = rz / pq;
            double rz_new = 0.0, r2 = 0.0;
            for (int u = threadIdx.x; u < m; u += blockDim.x) {
                const int i = S.i0 + u % mx, j = S.j0 + u / mx;
                const long long n = (long long)j * nx + i;
                x[n] += alpha * p[n];
                const double rn = r[n] - alpha * q[n];
                r[n] = rn;
                const double z = rn / dg[n];
                rz_new += rn * z;
                r2 += rn * rn;
            }
            block_sum2(rz_new, r2, sh);
            if (sqrt(r2) <= a.rtol * bnorm) break;
            const double beta = rz_new / rz;
            rz = rz_new;
            for (int u = threadIdx.x; u < m; u += blockDim.x) {
                const int i = S.i0 + u % mx, j = S.j0 + u / mx;
                const long long n = (long long)j * nx + i;
                p[n] = r[n] / dg[n] + beta * p[n];
            }
        }
    }
    if (threadIdx.x == 0) {
        a.iters[blockIdx.x] = it;
        if (it > a.max_iter) atomicOr(a.status, STATUS_NOCONV);
    }
}

__global__ void k_bump_step(uint32_t* step)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *step += 1u;
}

}  // namespace

cudaError_t launch_solve_setup(const float* w, const double* prev_xi, const double* prev_eta, int nx, int ny,
                               double Dt, double* cx, double* cy, double* dg, double* rhs0, cudaStream_t s)
{
    const dim3 block(32, 8);
    const dim3 grid((nx + 31) / 32, (ny + 7) / 8);
    k_solve_setup<<<grid, block, 0, s>>>(w, prev_xi, prev_eta, nx, ny, Dt, cx, cy, dg, rhs0);
    return cudaGetLastError();
}

cudaError_t launch_dirichlet(const double* faces64, const double* prev_xi, const double* prev_eta,
                             const double* iface_xi, const double* iface_eta, const int32_t* iface_idx,
                             int n_iface, int nx, int ny, double* xi_out, double* eta_out, cudaStream_t s)
{
    const dim3 block(32, 8);
    const dim3 grid((nx + 31) / 32, (ny + 7) / 8);
    k_dirichlet<<<grid, block, 0, s>>>(faces64, prev_xi, prev_eta, nx, ny, xi_out, eta_out);
    if (n_iface > 0)
        k_scatter_iface<<<(n_iface + 255) / 256, 256, 0, s>>>(iface_xi, iface_eta, iface_idx, n_iface, xi_out,
                                                             eta_out);
    return cudaGetLastError();
}

cudaError_t launch_pcg(const SolveArgs& a, cudaStream_t s)
{
    if (a.nsys > 0) k_pcg<<<a.nsys, SOLVE_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bump_step(uint32_t* step, cudaStream_t s)
{
    k_bump_step<<<1, 32, 0, s>>>(step);
    return cudaGetLastError();
}

}  // namespace sdd
