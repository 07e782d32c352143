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
// a symmetric positive definite M-matrix, solved per subdomain and field by
// Jacobi-preconditioned conjugate gradients.
//
// Precision: the solution and its residual are double precision; the
// conjugate-gradient sweeps run on the residual equation A d = r in single
// precision (iterative refinement): each sweep reduces ||r|| by inner_tol,
// then x += d and r = b - A x are formed again in double precision, until
// ||r|| <= rtol ||b||. On GB300 double-precision arithmetic runs at a small
// fraction of the single-precision rate; only the residuals use it.
//
// Execution: one thread-block cluster per system; each block owns a band of
// the subdomain's rows. Dot products are reduced inside each block, then
// across the cluster through distributed shared memory, in a fixed order, so
// every block takes the same branch. All loops are bounded by max_iter and
// max_outer; non-convergence sets a status bit.
#include <cooperative_groups.h>

#include "cluster.cuh"
#include "common.cuh"

namespace cg = cooperative_groups;

namespace sdd {

namespace {


__global__ void k_solve_setup(const float* __restrict__ w, const double* __restrict__ pxi,
                              const double* __restrict__ peta, int nx, int ny, double Dt, double* __restrict__ cx,
                              double* __restrict__ cy, double* __restrict__ dg, double* __restrict__ rhs0,
                              float* __restrict__ cxf, float* __restrict__ cyf, float* __restrict__ dgf,
                              float* __restrict__ dinvf)
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
    cxf[n] = (float)e;
    cyf[n] = (float)no;
    double d = 1.0 / (wc * Dt);
    rhs0[n] = pxi[n] * d;
    rhs0[(long long)nx * ny + n] = peta[n] * d;
    if (i > 0 && i + 1 < nx && j > 0 && j + 1 < ny) {
        const double wwest = (double)w[n - 1], wsouth = (double)w[n - nx];
        d += e + no + ihx2 / (0.5 * (wc + wwest)) + ihy2 / (0.5 * (wc + wsouth));
    }
    dg[n] = d;
    dgf[n] = (float)d;
    dinvf[n] = (float)(1.0 / d);
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
                                double* __restrict__ eo, uint32_t* step)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (step && k == 0) *step += 1u;   // the mesh step counter, when this closes the step
    if (k >= n) return;
    xo[idx[k]] = vx[k];
    eo[idx[k]] = ve[k];
}

__global__ void __launch_bounds__(SOLVE_THREADS) k_pcg_cluster(const SolveArgs a)
{
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const SolveSys S = a.sys[blockIdx.x / C];
    const int nx = a.nx;
    const int mx = S.i1 - S.i0, my = S.j1 - S.j0;
    const int row0 = S.j0 + (my * rank) / C, row1 = S.j0 + (my * (rank + 1)) / C;
    const int m = (row1 - row0) * mx;  // unknowns of this block
    double* __restrict__ x = a.x[S.field];
    float* __restrict__ r = a.r[S.field];
    float* __restrict__ p = a.p[S.field];
    float* __restrict__ q = a.q[S.field];
    float* __restrict__ d = a.d[S.field];
    const double* __restrict__ rhs = a.rhs0 + (long long)S.field * nx * a.ny;

    __shared__ ClusterSlots<double> red64[2];
    __shared__ ClusterSlots<float> red32[2];
    int seq = 0;  // one counter for both slot types: consecutive calls never share a slot set

    auto node = [&](int u) -> long long { return (long long)(row0 + u / mx) * nx + (S.i0 + u % mx); };

    // ||b||^2 with b = rhs + the Dirichlet neighbours' terms
    double bb = 0.0, unused = 0.0;
    for (int u = threadIdx.x; u < m; u += SOLVE_THREADS) {
        const long long n = node(u);
        const int i = S.i0 + u % mx, j = row0 + u / mx;
        double b = rhs[n];
        if (i == S.i0) b += a.cx[n - 1] * x[n - 1];
        if (i == S.i1 - 1) b += a.cx[n] * x[n + 1];
        if (j == S.j0) b += a.cy[n - nx] * x[n - nx];
        if (j == S.j1 - 1) b += a.cy[n] * x[n + nx];
        bb += b * b;
    }
    cluster_sum2(cl, red64, seq, bb, unused);
    const double stop2 = a.rtol * a.rtol * bb;

    int total = 0;
    bool converged = false;
    for (int outer = 0; outer < a.max_outer; ++outer) {
        // double-precision residual r = b - A x (x complete on every block: cluster-synchronised)
        double rr64 = 0.0, unused64 = 0.0;
        for (int u = threadIdx.x; u < m; u += SOLVE_THREADS) {
            const long long n = node(u);
            const double ax = a.dg[n] * x[n] - a.cx[n - 1] * x[n - 1] - a.cx[n] * x[n + 1] -
                              a.cy[n - nx] * x[n - nx] - a.cy[n] * x[n + nx];
            const double res = rhs[n] - ax;
            rr64 += res * res;
            const float rf = (float)res;
            r[n] = rf;
            d[n] = 0.0f;
            p[n] = rf * a.dinvf[n];
        }
        cluster_sum2(cl, red64, seq, rr64, unused64);
        if (rr64 <= stop2) {
            converged = true;
            break;
        }
        if (total >= a.max_iter) break;
        // single-precision PCG on A d = r, from d = 0 with p = z = r / diag
        float rz = 0.0f, rr = 0.0f;
        for (int u = threadIdx.x; u < m; u += SOLVE_THREADS) {
            const long long n = node(u);
            rz += r[n] * p[n];
            rr += r[n] * r[n];
        }
        cluster_sum2(cl, red32, seq, rz, rr);  // its barrier also publishes p to the neighbouring blocks
        if (!(rr > 0.0f)) continue;
        const float stop_in = a.inner_tol * a.inner_tol * rr;
        while (total < a.max_iter) {
            ++total;
            float pq = 0.0f, unused32 = 0.0f;
            for (int u = threadIdx.x; u < m; u += SOLVE_THREADS) {
                const long long n = node(u);
                // p is zero on every node that is not an unknown
                const float v = a.dgf[n] * p[n] - a.cxf[n - 1] * p[n - 1] - a.cxf[n] * p[n + 1] -
                                a.cyf[n - nx] * p[n - nx] - a.cyf[n] * p[n + nx];
                q[n] = v;
                pq += p[n] * v;
            }
            cluster_sum2(cl, red32, seq, pq, unused32);
            const float alpha = rz / pq;
            float rz_new = 0.0f, rr_new = 0.0f;
            for (int u = threadIdx.x; u < m; u += SOLVE_THREADS) {
                const long long n = node(u);
                d[n] += alpha * p[n];
                const float rn = r[n] - alpha * q[n];
                r[n] = rn;
                rz_new += rn * rn * a.dinvf[n];
                rr_new += rn * rn;
            }
            cluster_sum2(cl, red32, seq, rz_new, rr_new);
            if (rr_new <= stop_in) break;
            const float beta = rz_new / rz;
            rz = rz_new;
            for (int u = threadIdx.x; u < m; u += SOLVE_THREADS) {
                const long long n = node(u);
                p[n] = r[n] * a.dinvf[n] + beta * p[n];
            }
            cl.sync();  // p complete before the next product
        }
        // x += d in double precision; the next residual reads the neighbours' x
        for (int u = threadIdx.x; u < m; u += SOLVE_THREADS) {
            const long long n = node(u);
            x[n] += (double)d[n];
        }
        cl.sync();
    }
    if (threadIdx.x == 0 && rank == 0) {
        a.iters[blockIdx.x / C] = converged ? total : a.max_iter + 1;
        if (!converged) atomicOr(a.status, STATUS_NOCONV);
    }
    cl.sync();  // no block leaves while others may still read its shared memory
}

// Register-resident variant for subdomains whose band fits in the block:
// one cluster solves both fields of a subdomain (same matrix, two right-hand
// sides), so the cluster barriers are shared by the two solves. Each thread
// keeps UPT unknowns (coefficients and, per field, the CG vectors) in
// registers; the preconditioned residuals u live in shared memory with a
// halo row above and below. The inner iteration is the Chronopoulos--Gear
// form of preconditioned CG (Chronopoulos & Gear, "s-step iterative methods
// for symmetric linear systems", 1989): one fused reduction per iteration
// ((r,u), (w,u), (r,r) of both fields) after the product w = A u. Blocks push
// the edge rows of u and their reduction partials straight into the
// neighbours' shared memory before a cluster barrier, so an iteration is two
// barriers and no read crosses blocks. Halo rows and partial slots are
// double-buffered by the iteration's parity; a buffer is rewritten only two
// barriers after it was read. A field that has converged stops changing
// while the other one finishes.
template <int UPT>
__global__ void __launch_bounds__(SOLVE_THREADS) k_pcg_cg2(const SolveArgs a, int rows_max)
{
    extern __shared__ float m_s[];  // u: [parity][field] planes of (rows_max + 2) x (mx + 2), zero frame
    __shared__ float4 slots[2][16][2];  // [parity][block]: (gamma, delta, rr) of field 0, then field 1
    __shared__ float warp_part[6][SOLVE_WARPS];
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const SolveSys S = a.sys[blockIdx.x / C];
    const int nx = a.nx;
    const int mx = S.i1 - S.i0, my = S.j1 - S.j0;
    const int row0 = S.j0 + (my * rank) / C, row1 = S.j0 + (my * (rank + 1)) / C;
    const int rows = row1 - row0;
    const int m = rows * mx;
    const int W = mx + 2;
    const int plane = (rows_max + 2) * W;
    const int rows_below = rank > 0 ? ((my * rank) / C) - ((my * (rank - 1)) / C) : 0;
    double* __restrict__ x0 = a.x[0];
    double* __restrict__ x1 = a.x[1];
    const double* __restrict__ rhs0 = a.rhs0;
    const double* __restrict__ rhs1 = a.rhs0 + (long long)nx * a.ny;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    __shared__ ClusterSlots<double> red64[2];
    int seq = 0;

    for (int k = threadIdx.x; k < 4 * plane; k += SOLVE_THREADS) m_s[k] = 0.0f;
    float* nb_lo = (C > 1 && rank > 0) ? cl.map_shared_rank(m_s, rank - 1) : nullptr;     // block below
    float* nb_hi = (C > 1 && rank < C - 1) ? cl.map_shared_rank(m_s, rank + 1) : nullptr; // block above

    int n_[UPT];      // grid index of the unknown
    int sidx[UPT];    // its place in a plane of m_s
    int lc_[UPT];     // its column in the band
    int edge[UPT];    // 1: first row of the band, 2: last row
    bool own[UPT];
    float cw[UPT], ce[UPT], cs[UPT], cn[UPT], dgv[UPT], dinv[UPT];
    float r[2][UPT], u[2][UPT], w[2][UPT], s[2][UPT], p[2][UPT], d[2][UPT];
#pragma unroll
    for (int k = 0; k < UPT; ++k) {
        const int uu0 = threadIdx.x + k * SOLVE_THREADS;
        own[k] = uu0 < m;
        const int uu = own[k] ? uu0 : 0;
        const int lr = uu / mx;
        lc_[k] = uu % mx;
        n_[k] = (row0 + lr) * nx + (S.i0 + lc_[k]);
        sidx[k] = (lr + 1) * W + (lc_[k] + 1);
        edge[k] = (lr == 0 ? 1 : 0) | (lr == rows - 1 ? 2 : 0);
        if (own[k]) {
            const int n = n_[k];
            cw[k] = a.cxf[n - 1];
            ce[k] = a.cxf[n];
            cs[k] = a.cyf[n - nx];
            cn[k] = a.cyf[n];
            dgv[k] = a.dgf[n];
            dinv[k] = a.dinvf[n];
        } else {
            cw[k] = ce[k] = cs[k] = cn[k] = dgv[k] = dinv[k] = 0.0f;
        }
#pragma unroll
        for (int f = 0; f < 2; ++f) r[f][k] = u[f][k] = w[f][k] = s[f][k] = p[f][k] = d[f][k] = 0.0f;
    }

    // write both fields' u into buffer b and push their edge rows to the neighbours' halos
    auto publish = [&](int b) {
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            float* mine = m_s + (2 * b + f) * plane;
            const int off = (2 * b + f) * plane;
#pragma unroll
            for (int k = 0; k < UPT; ++k) {
                if (!own[k]) continue;
                mine[sidx[k]] = u[f][k];
                if ((edge[k] & 1) && nb_lo) nb_lo[off + (rows_below + 1) * W + lc_[k] + 1] = u[f][k];
                if ((edge[k] & 2) && nb_hi) nb_hi[off + lc_[k] + 1] = u[f][k];
            }
        }
    };
    auto apply_A = [&](int b, int f, int k) -> float {
        const float* v = m_s + (2 * b + f) * plane;
        const int c0 = sidx[k];
        return dgv[k] * v[c0] - cw[k] * v[c0 - 1] - ce[k] * v[c0 + 1] - cs[k] * v[c0 - W] - cn[k] * v[c0 + W];
    };
    // block partials of six sums, pushed to every block's slot [b][rank]; the barrier follows
    auto push6 = [&](int b, float (&v)[6]) {
#pragma unroll
        for (int q = 0; q < 6; ++q) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
            if (lane == 0) warp_part[q][warp] = v[q];
        }
        __syncthreads();
        if (warp == 0) {
            float t[6];
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                t[q] = lane < SOLVE_WARPS ? warp_part[q][lane] : 0.f;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) t[q] += __shfl_xor_sync(0xffffffffu, t[q], off);
            }
            if (lane < C) {
                float4* dst = cl.map_shared_rank(&slots[b][rank][0], lane);
                dst[0] = make_float4(t[0], t[1], t[2], 0.f);
                dst[1] = make_float4(t[3], t[4], t[5], 0.f);
            }
        }
    };
    // after the barrier, in every warp: lane q takes block q's partials, then a fixed butterfly
    auto read6 = [&](int b, float (&v)[6]) {
        float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
        if (lane < C) {
            a0 = slots[b][lane][0];
            a1 = slots[b][lane][1];
        }
        v[0] = a0.x; v[1] = a0.y; v[2] = a0.z; v[3] = a1.x; v[4] = a1.y; v[5] = a1.z;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
        }
    };

    // ||b||^2 of both fields
    double bb[2] = {0.0, 0.0};
#pragma unroll
    for (int k = 0; k < UPT; ++k) {
        if (!own[k]) continue;
        const int n = n_[k];
        const int i = S.i0 + lc_[k], j = n / nx;
        double b0 = rhs0[n], b1 = rhs1[n];
        if (i == S.i0) { b0 += a.cx[n - 1] * x0[n - 1]; b1 += a.cx[n - 1] * x1[n - 1]; }
        if (i == S.i1 - 1) { b0 += a.cx[n] * x0[n + 1]; b1 += a.cx[n] * x1[n + 1]; }
        if (j == S.j0) { b0 += a.cy[n - nx] * x0[n - nx]; b1 += a.cy[n - nx] * x1[n - nx]; }
        if (j == S.j1 - 1) { b0 += a.cy[n] * x0[n + nx]; b1 += a.cy[n] * x1[n + nx]; }
        bb[0] += b0 * b0;
        bb[1] += b1 * b1;
    }
    cluster_sum2(cl, red64, seq, bb[0], bb[1]);
    const double stop2[2] = {a.rtol * a.rtol * bb[0], a.rtol * a.rtol * bb[1]};

    int total = 0, it = 0;
    bool converged = false;
    for (int outer = 0; outer < a.max_outer; ++outer) {
        double rr64[2] = {0.0, 0.0};
#pragma unroll
        for (int k = 0; k < UPT; ++k) {
            if (!own[k]) continue;
            const int n = n_[k];
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                const double* xf = f ? x1 : x0;
                const double ax = a.dg[n] * xf[n] - a.cx[n - 1] * xf[n - 1] - a.cx[n] * xf[n + 1] -
                                  a.cy[n - nx] * xf[n - nx] - a.cy[n] * xf[n + nx];
                const double res = (f ? rhs1[n] : rhs0[n]) - ax;
                rr64[f] += res * res;
                r[f][k] = (float)res;
                d[f][k] = 0.0f;
                u[f][k] = r[f][k] * dinv[k];
                s[f][k] = p[f][k] = 0.0f;
            }
        }
        cluster_sum2(cl, red64, seq, rr64[0], rr64[1]);
        bool active[2] = {!(rr64[0] <= stop2[0]), !(rr64[1] <= stop2[1])};
        if (!active[0] && !active[1]) {
            converged = true;
            break;
        }
        if (total >= a.max_iter) break;
        // a converged field has d = 0 and a zero residual in this sweep
#pragma unroll
        for (int f = 0; f < 2; ++f)
            if (!active[f]) {
#pragma unroll
                for (int k = 0; k < UPT; ++k) r[f][k] = u[f][k] = 0.0f;
            }
        // Chronopoulos--Gear iterations on A d = r from d = 0, u = M^-1 r, both fields in step
        float alpha[2] = {0.f, 0.f}, beta[2] = {0.f, 0.f}, gam_old[2] = {1.f, 1.f}, rr0[2] = {0.f, 0.f};
        bool first = true;
        for (;;) {
            if (!first) {
#pragma unroll
                for (int f = 0; f < 2; ++f) {
                    if (!active[f]) continue;
#pragma unroll
                    for (int k = 0; k < UPT; ++k) {
                        p[f][k] = u[f][k] + beta[f] * p[f][k];
                        s[f][k] = w[f][k] + beta[f] * s[f][k];
                        d[f][k] += alpha[f] * p[f][k];
                        r[f][k] -= alpha[f] * s[f][k];
                        u[f][k] = r[f][k] * dinv[k];
                    }
                }
            }
            const int b = it & 1;
            ++it;
            publish(b);
            cl.sync();
            float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int f = 0; f < 2; ++f) {
#pragma unroll
                for (int k = 0; k < UPT; ++k) {
                    w[f][k] = own[k] ? apply_A(b, f, k) : 0.f;
                    v[3 * f + 0] += r[f][k] * u[f][k];
                    v[3 * f + 1] += w[f][k] * u[f][k];
                    v[3 * f + 2] += r[f][k] * r[f][k];
                }
            }
            push6(b, v);
            cl.sync();
            read6(b, v);
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                if (!active[f]) continue;
                const float gam = v[3 * f + 0], del = v[3 * f + 1], rr = v[3 * f + 2];
                if (first) {
                    rr0[f] = rr;
                    if (!(rr0[f] > 0.f) || !(del > 0.f)) {
                        active[f] = false;
                        continue;
                    }
                    alpha[f] = gam / del;
                    beta[f] = 0.f;
                } else {
                    if (rr <= a.inner_tol * a.inner_tol * rr0[f]) {
                        active[f] = false;
                        continue;
                    }
                    beta[f] = gam / gam_old[f];
                    alpha[f] = gam / (del - beta[f] * gam / alpha[f]);
                }
                gam_old[f] = gam;
            }
            first = false;
            if (!active[0] && !active[1]) break;
            if (total >= a.max_iter) break;
            ++total;
        }
        // x += d in double precision; the next residual reads the neighbours' x
#pragma unroll
        for (int k = 0; k < UPT; ++k)
            if (own[k]) {
                x0[n_[k]] += (double)d[0][k];
                x1[n_[k]] += (double)d[1][k];
            }
        cl.sync();
    }
    if (threadIdx.x == 0 && rank == 0) {
        a.iters[blockIdx.x / C] = converged ? total : a.max_iter + 1;
        if (!converged) atomicOr(a.status, STATUS_NOCONV);
    }
    cl.sync();  // no block leaves while others may still write into its shared memory
}

__global__ void k_bump_step(uint32_t* step)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *step += 1u;
}

}  // namespace

cudaError_t launch_solve_setup(const float* w, const double* prev_xi, const double* prev_eta, int nx, int ny,
                               double Dt, double* cx, double* cy, double* dg, double* rhs0, float* cxf, float* cyf,
                               float* dgf, float* dinvf, cudaStream_t s)
{
    const dim3 block(32, 8);
    const dim3 grid((nx + 31) / 32, (ny + 7) / 8);
    k_solve_setup<<<grid, block, 0, s>>>(w, prev_xi, prev_eta, nx, ny, Dt, cx, cy, dg, rhs0, cxf, cyf, dgf, dinvf);
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
                                                             eta_out, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_dirichlet_faces(const double* faces64, const double* prev_xi, const double* prev_eta, int nx,
                                   int ny, double* xi_out, double* eta_out, cudaStream_t s)
{
    const dim3 block(32, 8);
    const dim3 grid((nx + 31) / 32, (ny + 7) / 8);
    k_dirichlet<<<grid, block, 0, s>>>(faces64, prev_xi, prev_eta, nx, ny, xi_out, eta_out);
    return cudaGetLastError();
}

cudaError_t launch_scatter_iface(const double* iface_xi, const double* iface_eta, const int32_t* iface_idx,
                                 int n_iface, double* xi_out, double* eta_out, uint32_t* step, cudaStream_t s)
{
    const int n = n_iface > 0 ? n_iface : 1;
    k_scatter_iface<<<(n + 255) / 256, 256, 0, s>>>(iface_xi, iface_eta, iface_idx, n_iface, xi_out, eta_out, step);
    return cudaGetLastError();
}

// Blocks per system: a power of two up to 16, no more than the SMs allow for
// all systems at once and no more than the smallest system's rows.
int solve_cluster_size(int nsys, int min_rows, int sm_count)
{
    static int max_c = -1;
    if (max_c < 0) {
        max_c = 8;
        if (cudaFuncSetAttribute(k_pcg_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(16);
            cfg.blockDim = dim3(SOLVE_THREADS);
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = 16;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, k_pcg_cluster, &cfg) == cudaSuccess && n > 0) max_c = 16;
        }
        cudaGetLastError();
    }
    int c = 1;
    while (c * 2 <= max_c && (long long)c * 2 * nsys <= sm_count && c * 2 <= min_rows) c *= 2;
    return c;
}

static cudaLaunchConfig_t cluster_config(const SolveArgs& a, size_t smem, cudaStream_t s, cudaLaunchAttribute* at)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(a.nsys * a.cluster));
    cfg.blockDim = dim3(SOLVE_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)a.cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}

template <int UPT>
static cudaError_t launch_reg(const SolveArgs& a, int rows_max, int max_mx, cudaStream_t s)
{
    const size_t smem = 4 * (size_t)(rows_max + 2) * (size_t)(max_mx + 2) * sizeof(float);
    if (a.cluster > 8) cudaFuncSetAttribute(k_pcg_cg2<UPT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_pcg_cg2<UPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = cluster_config(a, smem, s, at);
    return cudaLaunchKernelEx(&cfg, k_pcg_cg2<UPT>, a, rows_max);
}

// Unknowns per thread of the register-resident kernel for these systems
// (0: too large, use the general kernel).
int solve_reg_upt(int max_band_unknowns)
{
    const int need = (max_band_unknowns + SOLVE_THREADS - 1) / SOLVE_THREADS;
    if (need <= 1) return 1;
    if (need <= 2) return 2;
    if (need <= 4) return 4;
    return 0;
}

cudaError_t launch_pcg(const SolveArgs& a, int upt, int rows_max, int max_mx, cudaStream_t s)
{
    if (a.nsys <= 0) return cudaSuccess;
    switch (upt) {
    case 1: return launch_reg<1>(a, rows_max, max_mx, s);
    case 2: return launch_reg<2>(a, rows_max, max_mx, s);
    case 4: return launch_reg<4>(a, rows_max, max_mx, s);
    default: {
        cudaLaunchAttribute at[1];
        cudaLaunchConfig_t cfg = cluster_config(a, 0, s, at);
        return cudaLaunchKernelEx(&cfg, k_pcg_cluster, a);
    }
    }
}

cudaError_t launch_bump_step(uint32_t* step, cudaStream_t s)
{
    k_bump_step<<<1, 32, 0, s>>>(step);
    return cudaGetLastError();
}

}  // namespace sdd
