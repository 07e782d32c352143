// mg.cu -- multigrid-preconditioned conjugate gradients for large subdomains.
//
// The subdomain systems of Sec. 4 (the implicit step of Eq. (3) in the
// symmetric form xi / (w Dt) + sum_nb c_nb (xi - xi_nb) = rhs, an SPD
// M-matrix) become ill-conditioned as the grid is refined: Jacobi-PCG needs
// O(sqrt(Dt) / h) iterations, about 1,800 at 2049^2 with Dt = 1e-3. A
// geometric multigrid V-cycle as preconditioner brings that to a few tens.
//
// Levels: every system is a box of mx x my unknowns with a Dirichlet frame;
// while both sizes are odd and at least 3, the next level keeps every second
// node (M = (m - 1) / 2; coarse node I sits on fine node 2I). Coarse
// operators are rediscretised from the fine coefficients: the mass term
// 1 / (w Dt) is sampled, a coarse face's coefficient is the series
// combination of the two fine faces it spans, (1/2) c1 c2 / (c1 + c2), which
// keeps the scaling c / H^2 = c / (4 h^2) of a uniform medium. Smoother:
// red-black Gauss-Seidel, two sweeps before (red, black) and after (black,
// red) the coarse correction; restriction full weighting, prolongation
// bilinear (restriction = transpose / 4), so the V-cycle is symmetric. Levels
// of at most 4096 unknowns run inside one block per system.
//
// Precision, as in the Jacobi-PCG kernels: the residual b - A x and the
// update x += d are double precision; the inner conjugate gradients on A d = r
// and the V-cycle are single precision (iterative refinement). Every dot
// product is reduced per block, then in block order; every loop count is
// fixed on the host, and systems (and fields) that have converged stop
// changing, so the whole solve is a fixed sequence of launches that a CUDA
// graph can hold.
#include <algorithm>

#include "common.cuh"

namespace sdd {
namespace {

constexpr int MG_THREADS = 256;
constexpr int TAIL_THREADS = 1024;

// padded index -> (i, j) of level l
struct Lv {
    int W, H, mx, my;
    long long off;   // this system's first element
};

__device__ __forceinline__ Lv level(const MgArgs& a, int l, int s)
{
    Lv v;
    v.mx = a.mx[l];
    v.my = a.my[l];
    v.W = v.mx + 2;
    v.H = v.my + 2;
    v.off = a.off[l] + (long long)s * v.W * v.H;
    return v;
}

__device__ __forceinline__ bool any_active(const MgArgs& a, int s)
{
    return a.act_i[2 * s] | a.act_i[2 * s + 1];
}

// ---------------------------------------------------------------- setup

// Level 0 from the grid: D and the face coefficients (single precision
// copies), the mass term, and every level-0 vector zeroed (the frame stays
// zero for the whole solve).
__global__ void k_mg_coef0(const MgArgs a)
{
    const int s = blockIdx.y;
    const SolveSys S = a.sys[s];
    const Lv v = level(a, 0, s);
    const int P = v.W * v.H;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < P; idx += gridDim.x * blockDim.x) {
        const int ip = idx % v.W, jp = idx / v.W;
        const long long g = (long long)(S.j0 - 1 + jp) * a.nx + (S.i0 - 1 + ip);
        const bool in = ip >= 1 && ip <= v.mx && jp >= 1 && jp <= v.my;
        const long long e = v.off + idx;
        a.D[e] = in ? a.dgf[g] : 0.f;
        a.MS[e] = in ? (float)(1.0 / ((double)a.w[g] * a.Dt)) : 0.f;
        a.CX[e] = (ip <= v.mx && jp >= 1 && jp <= v.my) ? a.cxf[g] : 0.f;
        a.CY[e] = (jp <= v.my && ip >= 1 && ip <= v.mx) ? a.cyf[g] : 0.f;
        for (int f = 0; f < 2; ++f) {
            a.U[f][e] = 0.f;
            a.F[f][e] = 0.f;
            a.Pv[f][idx + (long long)s * P] = 0.f;
            a.Qv[f][idx + (long long)s * P] = 0.f;
            a.Cv[f][idx + (long long)s * P] = 0.f;
        }
    }
}

__device__ __forceinline__ float series(float c1, float c2)
{
    return (c1 > 0.f && c2 > 0.f) ? 0.5f * c1 * c2 / (c1 + c2) : 0.f;
}

// Level l + 1 from level l (see the header: sampled mass, series faces).
__global__ void k_mg_coarsen(const MgArgs a, int l)
{
    const int s = blockIdx.y;
    const Lv h = level(a, l, s), c = level(a, l + 1, s);
    const int P = c.W * c.H;
    const float* CXh = a.CX + h.off;
    const float* CYh = a.CY + h.off;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < P; idx += gridDim.x * blockDim.x) {
        const int I = idx % c.W, J = idx / c.W;
        const int fi = 2 * I, fj = 2 * J;   // fine padded coordinates of the coarse node
        auto cxH = [&](int Ic, int Jc) { return series(CXh[2 * Jc * h.W + 2 * Ic], CXh[2 * Jc * h.W + 2 * Ic + 1]); };
        auto cyH = [&](int Ic, int Jc) {
            return series(CYh[2 * Jc * h.W + 2 * Ic], CYh[(2 * Jc + 1) * h.W + 2 * Ic]);
        };
        const bool in = I >= 1 && I <= c.mx && J >= 1 && J <= c.my;
        const long long e = c.off + idx;
        a.CX[e] = (I <= c.mx && J >= 1 && J <= c.my) ? cxH(I, J) : 0.f;
        a.CY[e] = (J <= c.my && I >= 1 && I <= c.mx) ? cyH(I, J) : 0.f;
        if (in) {
            const float ms = a.MS[h.off + (long long)fj * h.W + fi];
            a.MS[e] = ms;
            a.D[e] = ms + cxH(I - 1, J) + cxH(I, J) + cyH(I, J - 1) + cyH(I, J);
        } else {
            a.MS[e] = 0.f;
            a.D[e] = 0.f;
        }
        a.U[0][e] = a.U[1][e] = 0.f;
        a.F[0][e] = a.F[1][e] = 0.f;
    }
}

// ---------------------------------------------------------------- V-cycle pieces

// One red (color 0) or black (color 1) Gauss-Seidel half-sweep on level l.
__device__ __forceinline__ void smooth_node(const MgArgs& a, const Lv& v, int idx)
{
    const long long e = v.off + idx;
    const float d = a.D[e];
    const float cw = a.CX[e - 1], ce = a.CX[e], cs = a.CY[e - v.W], cn = a.CY[e];
    const float id = 1.f / d;
#pragma unroll
    for (int f = 0; f < 2; ++f) {
        const float* U = a.U[f];
        const float t = a.F[f][e] + cw * U[e - 1] + ce * U[e + 1] + cs * U[e - v.W] + cn * U[e + v.W];
        a.U[f][e] = t * id;
    }
}

__global__ void __launch_bounds__(MG_THREADS) k_mg_smooth(const MgArgs a, int l, int color)
{
    const int s = blockIdx.y;
    if (!any_active(a, s)) return;
    const Lv v = level(a, l, s);
    // interior nodes of one color, enumerated row by row: row jp has ceil/floor(mx / 2) of them
    const int per_row = (v.mx + 1) / 2;
    const int n = per_row * v.my;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int jp = 1 + k / per_row;
        const int ip = 1 + 2 * (k % per_row) + ((jp + 1 + color) & 1);   // (ip + jp) & 1 == color
        if (ip > v.mx) continue;
        smooth_node(a, v, jp * v.W + ip);
    }
}

__device__ __forceinline__ float residual_at(const MgArgs& a, const Lv& v, int f, long long e)
{
    const float* U = a.U[f];
    return a.F[f][e] - (a.D[e] * U[e] - a.CX[e - 1] * U[e - 1] - a.CX[e] * U[e + 1] - a.CY[e - v.W] * U[e - v.W] -
                        a.CY[e] * U[e + v.W]);
}

// F_{l+1} = full weighting of F_l - A_l U_l; U_{l+1} = 0.
__global__ void __launch_bounds__(MG_THREADS) k_mg_restrict(const MgArgs a, int l)
{
    const int s = blockIdx.y;
    if (!any_active(a, s)) return;
    const Lv h = level(a, l, s), c = level(a, l + 1, s);
    const int P = c.W * c.H;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < P; idx += gridDim.x * blockDim.x) {
        const int I = idx % c.W, J = idx / c.W;
        const long long e = c.off + idx;
        a.U[0][e] = a.U[1][e] = 0.f;
        if (I < 1 || I > c.mx || J < 1 || J > c.my) continue;
        const long long fc = h.off + (long long)(2 * J) * h.W + 2 * I;
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            float acc = 4.f * residual_at(a, h, f, fc);
            acc += 2.f * (residual_at(a, h, f, fc - 1) + residual_at(a, h, f, fc + 1) + residual_at(a, h, f, fc - h.W) +
                          residual_at(a, h, f, fc + h.W));
            acc += residual_at(a, h, f, fc - h.W - 1) + residual_at(a, h, f, fc - h.W + 1) +
                   residual_at(a, h, f, fc + h.W - 1) + residual_at(a, h, f, fc + h.W + 1);
            a.F[f][e] = acc * (1.f / 16.f);
        }
    }
}

// U_l += bilinear interpolation of U_{l+1} (its frame is zero).
__global__ void __launch_bounds__(MG_THREADS) k_mg_prolong(const MgArgs a, int l)
{
    const int s = blockIdx.y;
    if (!any_active(a, s)) return;
    const Lv h = level(a, l, s), c = level(a, l + 1, s);
    const int n = h.mx * h.my;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int ip = 1 + k % h.mx, jp = 1 + k / h.mx;
        const int I0 = ip >> 1, J0 = jp >> 1;          // coarse node at or left/below of the fine node
        const int I1 = (ip + 1) >> 1, J1 = (jp + 1) >> 1; // coarse node at or right/above
        const long long e = h.off + (long long)jp * h.W + ip;
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            const float* Uc = a.U[f] + c.off;
            const float v = 0.25f * (Uc[J0 * c.W + I0] + Uc[J0 * c.W + I1] + Uc[J1 * c.W + I0] + Uc[J1 * c.W + I1]);
            a.U[f][e] += v;
        }
    }
}

// The levels from lt down to the coarsest and back, by the calling block
// (system s); U_lt starts at zero.
__device__ void vcycle_block(const MgArgs& a, int s, int lt)
{
    auto sweep = [&](int l, int color) {
        const Lv v = level(a, l, s);
        const int per_row = (v.mx + 1) / 2;
        const int n = per_row * v.my;
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const int jp = 1 + k / per_row;
            const int ip = 1 + 2 * (k % per_row) + ((jp + 1 + color) & 1);
            if (ip <= v.mx) smooth_node(a, v, jp * v.W + ip);
        }
        __syncthreads();
    };
    const int L = a.levels;
    for (int l = lt; l < L - 1; ++l) {
        for (int k = 0; k < a.nu; ++k) {
            sweep(l, 0);
            sweep(l, 1);
        }
        const Lv h = level(a, l, s), c = level(a, l + 1, s);
        const int P = c.W * c.H;
        for (int idx = threadIdx.x; idx < P; idx += blockDim.x) {
            const int I = idx % c.W, J = idx / c.W;
            const long long e = c.off + idx;
            a.U[0][e] = a.U[1][e] = 0.f;
            if (I < 1 || I > c.mx || J < 1 || J > c.my) continue;
            const long long fc = h.off + (long long)(2 * J) * h.W + 2 * I;
            for (int f = 0; f < 2; ++f) {
                float acc = 4.f * residual_at(a, h, f, fc);
                acc += 2.f * (residual_at(a, h, f, fc - 1) + residual_at(a, h, f, fc + 1) +
                              residual_at(a, h, f, fc - h.W) + residual_at(a, h, f, fc + h.W));
                acc += residual_at(a, h, f, fc - h.W - 1) + residual_at(a, h, f, fc - h.W + 1) +
                       residual_at(a, h, f, fc + h.W - 1) + residual_at(a, h, f, fc + h.W + 1);
                a.F[f][e] = acc * (1.f / 16.f);
            }
        }
        __syncthreads();
    }
    // coarsest level: one unknown is solved exactly, a larger box by many sweeps
    {
        const Lv v = level(a, L - 1, s);
        if (v.mx == 1 && v.my == 1) {
            if (threadIdx.x < 2) {
                const long long e = v.off + v.W + 1;
                a.U[threadIdx.x][e] = a.F[threadIdx.x][e] / a.D[e];
            }
            __syncthreads();
        } else {
            for (int k = 0; k < a.coarse_sweeps; ++k) {
                sweep(L - 1, 0);
                sweep(L - 1, 1);
            }
            for (int k = 0; k < a.coarse_sweeps; ++k) {
                sweep(L - 1, 1);
                sweep(L - 1, 0);
            }
        }
    }
    for (int l = L - 2; l >= lt; --l) {
        const Lv h = level(a, l, s), c = level(a, l + 1, s);
        const int n = h.mx * h.my;
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const int ip = 1 + k % h.mx, jp = 1 + k / h.mx;
            const int I0 = ip >> 1, J0 = jp >> 1, I1 = (ip + 1) >> 1, J1 = (jp + 1) >> 1;
            const long long e = h.off + (long long)jp * h.W + ip;
            for (int f = 0; f < 2; ++f) {
                const float* Uc = a.U[f] + c.off;
                a.U[f][e] += 0.25f * (Uc[J0 * c.W + I0] + Uc[J0 * c.W + I1] + Uc[J1 * c.W + I0] + Uc[J1 * c.W + I1]);
            }
        }
        __syncthreads();
        for (int k = 0; k < a.nu; ++k) {
            sweep(l, 1);
            sweep(l, 0);
        }
    }
}

__global__ void __launch_bounds__(TAIL_THREADS) k_mg_tail(const MgArgs a, int lt)
{
    const int s = blockIdx.x;
    if (!any_active(a, s)) return;
    vcycle_block(a, s, lt);
}

// ---------------------------------------------------------------- Krylov pieces (level-0 vectors)

// Per-block sums of two values per field -> part[s][block][4].
__device__ __forceinline__ void block_sum4(float v0, float v1, float v2, float v3, float* out)
{
    __shared__ float red[4][MG_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float v[4] = {v0, v1, v2, v3};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        for (int o = 16; o; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
        if (lane == 0) red[k][warp] = v[k];
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        float t = 0.f;
        for (int q = 0; q < MG_THREADS / 32; ++q) t += red[threadIdx.x][q];
        out[threadIdx.x] = t;
    }
}

__device__ __forceinline__ void block_sum4d(double v0, double v1, double v2, double v3, double* out)
{
    __shared__ double red[4][MG_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double v[4] = {v0, v1, v2, v3};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        for (int o = 16; o; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
        if (lane == 0) red[k][warp] = v[k];
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int q = 0; q < MG_THREADS / 32; ++q) t += red[threadIdx.x][q];
        out[threadIdx.x] = t;
    }
}

// sum over the system's blocks, in block order
__device__ __forceinline__ float sum_part(const MgArgs& a, int s, int k)
{
    float t = 0.f;
    for (int b = 0; b < a.B0; ++b) t += a.part[((long long)s * a.B0 + b) * 4 + k];
    return t;
}

// Double-precision residual of the current fields on every unknown; writes it
// (single precision) as the V-cycle's level-0 right-hand side, zeroes the
// correction and the V-cycle's level-0 iterate; per-block sums of ||r||^2 and
// ||b||^2 (b = rhs + the Dirichlet neighbours' terms).
__global__ void __launch_bounds__(MG_THREADS) k_mg_res64(const MgArgs a)
{
    const int s = blockIdx.y;
    const SolveSys S = a.sys[s];
    const Lv v = level(a, 0, s);
    const int n = v.mx * v.my;
    const int nx = a.nx;
    double rr[2] = {0.0, 0.0}, bb[2] = {0.0, 0.0};
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int ip = 1 + k % v.mx, jp = 1 + k / v.mx;
        const int i = S.i0 - 1 + ip, j = S.j0 - 1 + jp;
        const long long g = (long long)j * nx + i;
        const long long e = (long long)jp * v.W + ip;
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            const double* x = a.x[f];
            const double* rhs = a.rhs0 + (long long)f * nx * a.ny;
            const double ax = a.dg[g] * x[g] - a.cx[g - 1] * x[g - 1] - a.cx[g] * x[g + 1] - a.cy[g - nx] * x[g - nx] -
                              a.cy[g] * x[g + nx];
            const double r = rhs[g] - ax;
            double b = rhs[g];
            if (i == S.i0) b += a.cx[g - 1] * x[g - 1];
            if (i == S.i1 - 1) b += a.cx[g] * x[g + 1];
            if (j == S.j0) b += a.cy[g - nx] * x[g - nx];
            if (j == S.j1 - 1) b += a.cy[g] * x[g + nx];
            rr[f] += r * r;
            bb[f] += b * b;
            a.F[f][v.off + e] = (float)r;
            a.U[f][v.off + e] = 0.f;
            a.Cv[f][(long long)s * v.W * v.H + e] = 0.f;
        }
    }
    block_sum4d(rr[0], rr[1], bb[0], bb[1], a.part64 + ((long long)s * a.B0 + blockIdx.x) * 4);
}

// Per system and field: outer convergence. first: stop2 = rtol^2 ||b||^2 and
// every field starts active. final: the status and iteration counts. The two
// fields of a system are neighbouring lanes of one warp.
__global__ void k_mg_outer(const MgArgs a, int first, int final)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = t < 2 * a.nsys;
    const int s = t >> 1, f = t & 1;
    double rr = 0.0, bb = 0.0;
    if (valid)
        for (int b = 0; b < a.B0; ++b) {
            rr += a.part64[((long long)s * a.B0 + b) * 4 + f];
            bb += a.part64[((long long)s * a.B0 + b) * 4 + 2 + f];
        }
    if (valid && first) {
        a.stop2[t] = a.rtol * a.rtol * bb;
        a.act_o[t] = 1;
        a.iters[t] = 0;
    }
    const bool conv = valid ? rr <= a.stop2[t] : true;
    if (final) {
        const unsigned other = __shfl_xor_sync(0xffffffffu, conv ? 1u : 0u, 1);
        const int it_other = __shfl_xor_sync(0xffffffffu, valid ? a.iters[t] : 0, 1);
        if (!valid) return;
        if (!conv) atomicOr(a.status, STATUS_NOCONV);
        if (f == 0) a.sys_iters[s] = (conv && other) ? max(a.iters[t], it_other) : a.max_iter + 1;
        return;
    }
    if (!valid) return;
    if (conv) a.act_o[t] = 0;
    a.act_i[t] = a.act_o[t];
    a.rr0[t] = (float)rr;
}

// Level-0 vectors of a system: z (the V-cycle's U), r (its F), p, q, d.
struct V0 {
    long long off, base;
    int W, H, mx, my;
};

__device__ __forceinline__ V0 v0(const MgArgs& a, int s)
{
    V0 v;
    v.mx = a.mx[0];
    v.my = a.my[0];
    v.W = v.mx + 2;
    v.H = v.my + 2;
    v.base = (long long)s * v.W * v.H;
    v.off = a.off[0] + v.base;
    return v;
}

// rz = (r, z) partials
__global__ void __launch_bounds__(MG_THREADS) k_mg_rz(const MgArgs a)
{
    const int s = blockIdx.y;
    const V0 v = v0(a, s);
    const int n = v.mx * v.my;
    float t[2] = {0.f, 0.f};
    if (any_active(a, s))
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
            const long long e = (long long)(1 + k / v.mx) * v.W + 1 + k % v.mx;
#pragma unroll
            for (int f = 0; f < 2; ++f) t[f] += a.F[f][v.off + e] * a.U[f][v.off + e];
        }
    block_sum4(t[0], t[1], 0.f, 0.f, a.part + ((long long)s * a.B0 + blockIdx.x) * 4);
}

// p = z + beta p with beta = rz_new / rz_old (first: p = z); rz slots by parity.
__global__ void __launch_bounds__(MG_THREADS) k_mg_pupdate(const MgArgs a, int first, int parity)
{
    const int s = blockIdx.y;
    if (!any_active(a, s)) return;
    if (parity < 0) parity = a.loop[1] & 1;   // inside a graph loop: the inner iteration counter
    const V0 v = v0(a, s);
    const int n = v.mx * v.my;
    float beta[2];
#pragma unroll
    for (int f = 0; f < 2; ++f) {
        const float rz_new = sum_part(a, s, f);
        const float rz_old = a.rz[(2 * s + f) * 2 + (parity ^ 1)];
        beta[f] = (!first && a.act_i[2 * s + f] && rz_old > 0.f) ? rz_new / rz_old : 0.f;
        if (blockIdx.x == 0 && threadIdx.x == 0) a.rz[(2 * s + f) * 2 + parity] = rz_new;
    }
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const long long e = (long long)(1 + k / v.mx) * v.W + 1 + k % v.mx;
#pragma unroll
        for (int f = 0; f < 2; ++f) a.Pv[f][v.base + e] = a.U[f][v.off + e] + beta[f] * a.Pv[f][v.base + e];
    }
}

// q = A p (level 0, single precision), (p, q) partials
__global__ void __launch_bounds__(MG_THREADS) k_mg_spmv(const MgArgs a)
{
    const int s = blockIdx.y;
    const V0 v = v0(a, s);
    const int n = v.mx * v.my;
    float t[2] = {0.f, 0.f};
    if (any_active(a, s))
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
            const long long e = (long long)(1 + k / v.mx) * v.W + 1 + k % v.mx;
            const long long c = v.off + e;
            const float d = a.D[c], cw = a.CX[c - 1], ce = a.CX[c], cs = a.CY[c - v.W], cn = a.CY[c];
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                const float* p = a.Pv[f] + v.base;
                const float q = d * p[e] - cw * p[e - 1] - ce * p[e + 1] - cs * p[e - v.W] - cn * p[e + v.W];
                a.Qv[f][v.base + e] = q;
                t[f] += p[e] * q;
            }
        }
    block_sum4(t[0], t[1], 0.f, 0.f, a.part + ((long long)s * a.B0 + blockIdx.x) * 4);
}

// d += alpha p, r -= alpha q, z = 0 (the next V-cycle starts from zero); (r, r) partials.
__global__ void __launch_bounds__(MG_THREADS) k_mg_update(const MgArgs a, int parity)
{
    const int s = blockIdx.y;
    if (parity < 0) parity = a.loop[1] & 1;
    const V0 v = v0(a, s);
    const int n = v.mx * v.my;
    float t[2] = {0.f, 0.f};
    if (any_active(a, s)) {
        float alpha[2];
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            const float pq = sum_part(a, s, f);
            const float rz = a.rz[(2 * s + f) * 2 + parity];
            alpha[f] = (a.act_i[2 * s + f] && pq > 0.f) ? rz / pq : 0.f;
        }
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
            const long long e = (long long)(1 + k / v.mx) * v.W + 1 + k % v.mx;
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                a.Cv[f][v.base + e] += alpha[f] * a.Pv[f][v.base + e];
                const float r = a.F[f][v.off + e] - alpha[f] * a.Qv[f][v.base + e];
                a.F[f][v.off + e] = r;
                a.U[f][v.off + e] = 0.f;
                t[f] += r * r;
            }
        }
    }
    block_sum4(t[0], t[1], 0.f, 0.f, a.part + ((long long)s * a.B0 + blockIdx.x) * 4);
}

// Inner convergence: a field stops once ||r||^2 <= inner_tol^2 ||r_0||^2 (or on a breakdown).
__global__ void k_mg_inner(const MgArgs a)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * a.nsys) return;
    if (!a.act_i[t]) return;
    const float rr = sum_part(a, t >> 1, t & 1);
    a.iters[t] += 1;
    if (!(rr > a.inner_tol * a.inner_tol * a.rr0[t])) a.act_i[t] = 0;
}

// Loop control inside a graph: counter `which` (0 refinement sweeps, 1 inner
// iterations) counts this pass, and the while-node's condition becomes "some
// field still active (act_o for 0, act_i for 1) and fewer than cap passes".
__global__ void k_mg_cond(const MgArgs a, cudaGraphConditionalHandle h, int which, int cap, int body_kernels)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (a.launches) *a.launches += body_kernels;   // the pass of the loop body that ends here
    const int32_t* act = which == 0 ? a.act_o : a.act_i;
    int any = 0;
    for (int t = 0; t < 2 * a.nsys; ++t) any |= act[t];
    const int c = a.loop[which] + 1;
    a.loop[which] = c;
    cudaGraphSetConditional(h, (any && c < cap) ? 1u : 0u);
}

// Start a loop: counter `which` to zero and the loop's condition to "some field active".
__global__ void k_mg_loop_reset(const MgArgs a, cudaGraphConditionalHandle h, int which)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (which == 0 && a.launches) *a.launches = 0;
    const int32_t* act = which == 0 ? a.act_o : a.act_i;
    int any = 0;
    for (int t = 0; t < 2 * a.nsys; ++t) any |= act[t];
    a.loop[which] = 0;
    cudaGraphSetConditional(h, any ? 1u : 0u);
}

// x += d (double precision) on every unknown of the fields still iterating
__global__ void __launch_bounds__(MG_THREADS) k_mg_xupdate(const MgArgs a)
{
    const int s = blockIdx.y;
    const SolveSys S = a.sys[s];
    const V0 v = v0(a, s);
    const int n = v.mx * v.my;
    const bool on[2] = {a.act_o[2 * s] != 0, a.act_o[2 * s + 1] != 0};
    if (!on[0] && !on[1]) return;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int ip = 1 + k % v.mx, jp = 1 + k / v.mx;
        const long long g = (long long)(S.j0 - 1 + jp) * a.nx + (S.i0 - 1 + ip);
        const long long e = (long long)jp * v.W + ip;
#pragma unroll
        for (int f = 0; f < 2; ++f)
            if (on[f]) a.x[f][g] += (double)a.Cv[f][v.base + e];
    }
}

int blocks_for(long long n)
{
    const long long b = (n + MG_THREADS * 4 - 1) / (MG_THREADS * 4);
    return (int)std::max<long long>(1, std::min<long long>(b, 64));
}

}  // namespace

// ---------------------------------------------------------------- host side

bool mg_levels(int mx, int my, MgArgs& a)
{
    if (mx < 1 || my < 1) return false;
    int L = 1;
    a.mx[0] = mx;
    a.my[0] = my;
    while (L < kMgMaxLevels && (a.mx[L - 1] & 1) && (a.my[L - 1] & 1) && a.mx[L - 1] >= 3 && a.my[L - 1] >= 3) {
        a.mx[L] = (a.mx[L - 1] - 1) / 2;
        a.my[L] = (a.my[L - 1] - 1) / 2;
        ++L;
    }
    a.levels = L;
    // the coarsest level is solved by sweeps; only worthwhile when it is small
    if ((long long)a.mx[L - 1] * a.my[L - 1] > 64) return false;
    a.tail = 0;
    while (a.tail < L - 1 && (long long)a.mx[a.tail] * a.my[a.tail] > 4096) ++a.tail;
    return L >= 2;
}

long long mg_layout(MgArgs& a, int nsys)
{
    long long off = 0;
    for (int l = 0; l < a.levels; ++l) {
        a.off[l] = off;
        off += (long long)nsys * (a.mx[l] + 2) * (a.my[l] + 2);
    }
    a.nsys = nsys;
    a.B0 = blocks_for((long long)a.mx[0] * a.my[0]);
    return off;
}

cudaError_t launch_mg_setup(const MgArgs& a, cudaStream_t s)
{
    const long long P0 = (long long)(a.mx[0] + 2) * (a.my[0] + 2);
    k_mg_coef0<<<dim3(blocks_for(P0), a.nsys), MG_THREADS, 0, s>>>(a);
    for (int l = 0; l + 1 < a.levels; ++l) {
        const long long P = (long long)(a.mx[l + 1] + 2) * (a.my[l + 1] + 2);
        k_mg_coarsen<<<dim3(blocks_for(P), a.nsys), MG_THREADS, 0, s>>>(a, l);
    }
    return cudaGetLastError();
}

// kernels one V-cycle launches
static int vcycle_kernels(const MgArgs& a) { return a.tail * (4 * a.nu + 2) + 1; }

static void vcycle(const MgArgs& a, cudaStream_t s)
{
    for (int l = 0; l < a.tail; ++l) {
        const dim3 g(blocks_for(((long long)a.mx[l] * a.my[l] + 1) / 2), a.nsys);
        for (int k = 0; k < a.nu; ++k) {
            k_mg_smooth<<<g, MG_THREADS, 0, s>>>(a, l, 0);
            k_mg_smooth<<<g, MG_THREADS, 0, s>>>(a, l, 1);
        }
        const long long Pc = (long long)(a.mx[l + 1] + 2) * (a.my[l + 1] + 2);
        k_mg_restrict<<<dim3(blocks_for(Pc), a.nsys), MG_THREADS, 0, s>>>(a, l);
    }
    k_mg_tail<<<a.nsys, TAIL_THREADS, 0, s>>>(a, a.tail);
    for (int l = a.tail - 1; l >= 0; --l) {
        const dim3 g(blocks_for(((long long)a.mx[l] * a.my[l] + 1) / 2), a.nsys);
        k_mg_prolong<<<dim3(blocks_for((long long)a.mx[l] * a.my[l]), a.nsys), MG_THREADS, 0, s>>>(a, l);
        for (int k = 0; k < a.nu; ++k) {
            k_mg_smooth<<<g, MG_THREADS, 0, s>>>(a, l, 1);
            k_mg_smooth<<<g, MG_THREADS, 0, s>>>(a, l, 0);
        }
    }
}

cudaError_t launch_mg_solve(const MgArgs& a, cudaStream_t s)
{
    const dim3 g0(a.B0, a.nsys);
    const int sc = (2 * a.nsys + 127) / 128;
    for (int o = 0; o < a.outer; ++o) {
        k_mg_res64<<<g0, MG_THREADS, 0, s>>>(a);
        k_mg_outer<<<sc, 128, 0, s>>>(a, o == 0, 0);
        vcycle(a, s);
        k_mg_rz<<<g0, MG_THREADS, 0, s>>>(a);
        k_mg_pupdate<<<g0, MG_THREADS, 0, s>>>(a, 1, 0);
        int parity = 0;
        for (int it = 0; it < a.inner; ++it) {
            k_mg_spmv<<<g0, MG_THREADS, 0, s>>>(a);
            k_mg_update<<<g0, MG_THREADS, 0, s>>>(a, parity);
            k_mg_inner<<<sc, 128, 0, s>>>(a);
            if (it + 1 == a.inner) break;
            vcycle(a, s);
            k_mg_rz<<<g0, MG_THREADS, 0, s>>>(a);
            parity ^= 1;
            k_mg_pupdate<<<g0, MG_THREADS, 0, s>>>(a, 0, parity);
        }
        k_mg_xupdate<<<g0, MG_THREADS, 0, s>>>(a);
    }
    k_mg_res64<<<g0, MG_THREADS, 0, s>>>(a);
    k_mg_outer<<<sc, 128, 0, s>>>(a, 0, 1);
    return cudaGetLastError();
}

// A condition handle of the graph that stream s is capturing into. The
// handle's default (1) applies only when the whole graph is launched, so a
// loop entered more than once per launch has its handle set by a kernel first.
static cudaError_t make_handle(cudaStream_t s, cudaGraphConditionalHandle* h)
{
    cudaStreamCaptureStatus st;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, &g, nullptr, nullptr, nullptr);
    if (e != cudaSuccess) return e;
    if (st != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureImplicit;
    return cudaGraphConditionalHandleCreate(h, g, 1, cudaGraphCondAssignDefault);
}

// Add a while-node on handle h after the capture's current dependencies on
// stream s and start capturing its body on stream b.
static cudaError_t begin_while(cudaStream_t s, cudaStream_t b, cudaGraphConditionalHandle h, cudaGraphNode_t* node)
{
    cudaStreamCaptureStatus st;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd);
    if (e != cudaSuccess) return e;
    if (st != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureImplicit;
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    if ((e = cudaGraphAddNode(node, g, deps, nullptr, nd, &p)) != cudaSuccess) return e;
    return cudaStreamBeginCaptureToGraph(b, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeRelaxed);
}

// Close the body captured on b; s continues after the while-node.
static cudaError_t end_while(cudaStream_t s, cudaStream_t b, cudaGraphNode_t node)
{
    cudaGraph_t body = nullptr;
    cudaError_t e = cudaStreamEndCapture(b, &body);
    if (e != cudaSuccess) return e;
    return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

static cudaError_t mg_graph_body(const MgArgs& a, cudaStream_t s, cudaStream_t s2, cudaStream_t s3)
{
    const dim3 g0(a.B0, a.nsys);
    const int sc = (2 * a.nsys + 127) / 128;
    cudaError_t e;
    cudaGraphConditionalHandle ho, hi;
    cudaGraphNode_t no, ni;
    k_mg_res64<<<g0, MG_THREADS, 0, s>>>(a);
    k_mg_outer<<<sc, 128, 0, s>>>(a, 1, 0);
    if ((e = make_handle(s, &ho)) != cudaSuccess) return e;
    k_mg_loop_reset<<<1, 32, 0, s>>>(a, ho, 0);
    if ((e = begin_while(s, s2, ho, &no)) != cudaSuccess) return e;
    // one refinement sweep: the inner PCG on A d = r, then x += d and the new residual
    vcycle(a, s2);
    k_mg_rz<<<g0, MG_THREADS, 0, s2>>>(a);
    if ((e = make_handle(s2, &hi)) != cudaSuccess) return e;
    k_mg_loop_reset<<<1, 32, 0, s2>>>(a, hi, 1);
    k_mg_pupdate<<<g0, MG_THREADS, 0, s2>>>(a, 1, -1);
    if ((e = begin_while(s2, s3, hi, &ni)) != cudaSuccess) return e;
    k_mg_spmv<<<g0, MG_THREADS, 0, s3>>>(a);
    k_mg_update<<<g0, MG_THREADS, 0, s3>>>(a, -1);
    k_mg_inner<<<sc, 128, 0, s3>>>(a);
    k_mg_cond<<<1, 32, 0, s3>>>(a, hi, 1, a.inner, 6 + vcycle_kernels(a));
    vcycle(a, s3);
    k_mg_rz<<<g0, MG_THREADS, 0, s3>>>(a);
    k_mg_pupdate<<<g0, MG_THREADS, 0, s3>>>(a, 0, -1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = end_while(s2, s3, ni)) != cudaSuccess) return e;
    k_mg_xupdate<<<g0, MG_THREADS, 0, s2>>>(a);
    k_mg_res64<<<g0, MG_THREADS, 0, s2>>>(a);
    k_mg_outer<<<sc, 128, 0, s2>>>(a, 0, 0);
    k_mg_cond<<<1, 32, 0, s2>>>(a, ho, 0, a.outer, 8 + vcycle_kernels(a));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = end_while(s, s2, no)) != cudaSuccess) return e;
    k_mg_outer<<<sc, 128, 0, s>>>(a, 0, 1);
    return cudaGetLastError();
}

// The same solve for a stream that is being captured: the refinement sweeps
// and the inner iterations are while-nodes whose condition kernels stop them
// once every field has converged (at most outer x inner passes), so a graph
// replay runs only the iterations the systems need.
cudaError_t launch_mg_solve_graph(const MgArgs& a, cudaStream_t s, cudaStream_t s2, cudaStream_t s3)
{
    const cudaError_t e = mg_graph_body(a, s, s2, s3);
    if (e != cudaSuccess) {
        // leave no body capture open: the caller ends (and discards) the main capture
        for (cudaStream_t b : {s3, s2}) {
            cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(b, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
                cudaGraph_t g = nullptr;
                cudaStreamEndCapture(b, &g);
                if (g) cudaGraphDestroy(g);
            }
        }
    }
    return e;
}

}  // namespace sdd
