// mgc.cu -- multigrid-preconditioned CG inside one thread-block cluster per subdomain.
//
// The same solver as mg.cu (double-precision refinement around single-
// precision conjugate gradients preconditioned by a symmetric V-cycle:
// red-black Gauss-Seidel, full weighting, bilinear prolongation,
// rediscretised coarse operators built by mg.cu's setup), laid out for
// subdomains of up to about 140 x 140 unknowns, where a chain of grid-wide
// launches spends its time in launch latency:
//
//   * the cluster's blocks split the subdomain's rows; every thread keeps one
//     to four unknowns of the finest level in registers (coefficients, the
//     residual r, the product q, the correction d); the V-cycle iterate z,
//     the search direction p and the fine residual live in shared memory, and
//     a block reads its neighbours' edge rows straight from their shared
//     memory (distributed shared memory) after a cluster barrier;
//   * the coarser levels (second finest and below) live in the shared memory
//     of the cluster's first block, which runs that part of every V-cycle
//     alone while the others wait; the other blocks write their share of the
//     restricted residual into it and read the coarse correction back from it;
//     the levels are described by offsets into the shared memory, kept once
//     per block in shared memory, and the kernel uses no local memory (with
//     up to 210 KB of shared memory per block the L1 cannot hold 512 threads'
//     stack frames, and every local access would go to L2);
//   * dot products are reduced inside each block, then across the cluster in
//     a fixed order (every block takes the same branch); the loop counts are
//     bounded (max_outer refinement sweeps, max_iter inner iterations).
//
// One launch per solve: the whole iteration runs inside the kernel.
#include <cooperative_groups.h>

#include "cluster.cuh"
#include "common.cuh"

namespace sdd {
namespace {

// The kernel's dynamic shared memory.
extern __shared__ float mgc_sm[];

// a coarse level in the first block's shared memory: its arrays as offsets
// into the dynamic shared memory, so that every access is a shared-memory load
struct SLv {
    int D, CX, CY, U[2], F[2];
    int mx, my, W;
};

// floor(k / d) for 0 <= k from the single-precision product (k + 1/2) fl(1/d):
// (k + 1/2) / d lies at least 1/(2d) from every integer, and the two roundings
// move the product by less than (k + 1/2) 2^-23, so the quotient is exact while
// (k + 1/2) d < 2^22 (mgc_config admits only levels within that bound).
__device__ __forceinline__ int qdiv(int k, float rd) { return __float2int_rz(__fmul_rn((float)k + 0.5f, rd)); }

// One point of a red-black sweep: the level's offsets and row length are
// passed as values, so no descriptor is re-read after the stores.
__device__ __forceinline__ void s_smooth(int oD, int oCX, int oCY, int oU0, int oU1, int oF0, int oF1, int W, int idx)
{
    const float id = 1.f / mgc_sm[oD + idx];
    const float cw = mgc_sm[oCX + idx - 1], ce = mgc_sm[oCX + idx], cs = mgc_sm[oCY + idx - W], cn = mgc_sm[oCY + idx];
    const float n0 = mgc_sm[oF0 + idx] + cw * mgc_sm[oU0 + idx - 1] + ce * mgc_sm[oU0 + idx + 1] +
                     cs * mgc_sm[oU0 + idx - W] + cn * mgc_sm[oU0 + idx + W];
    const float n1 = mgc_sm[oF1 + idx] + cw * mgc_sm[oU1 + idx - 1] + ce * mgc_sm[oU1 + idx + 1] +
                     cs * mgc_sm[oU1 + idx - W] + cn * mgc_sm[oU1 + idx + W];
    mgc_sm[oU0 + idx] = n0 * id;
    mgc_sm[oU1 + idx] = n1 * id;
}

__device__ __forceinline__ float s_res(const SLv& v, int f, int idx)
{
    const float* U = mgc_sm + v.U[f];
    const float* D = mgc_sm + v.D;
    const float* CX = mgc_sm + v.CX;
    const float* CY = mgc_sm + v.CY;
    return mgc_sm[v.F[f] + idx] - (D[idx] * U[idx] - CX[idx - 1] * U[idx - 1] - CX[idx] * U[idx + 1] -
                                   CY[idx - v.W] * U[idx - v.W] - CY[idx] * U[idx + v.W]);
}

// One red-black half-sweep of level v (the points of one colour), then a block barrier.
__device__ __forceinline__ void s_sweep(const SLv& v, int color)
{
    const int mxl = v.mx, W = v.W;
    const int oD = v.D, oCX = v.CX, oCY = v.CY, oU0 = v.U[0], oU1 = v.U[1], oF0 = v.F[0], oF1 = v.F[1];
    const int per_row = (mxl + 1) >> 1;
    const int n = per_row * v.my;
    const float rpr = 1.f / (float)per_row;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int q = qdiv(k, rpr);
        const int jp = 1 + q;
        const int ip = 1 + 2 * (k - q * per_row) + ((jp + 1 + color) & 1);
        if (ip <= mxl) s_smooth(oD, oCX, oCY, oU0, oU1, oF0, oF1, W, jp * W + ip);
    }
    __syncthreads();
}

// The V-cycle below the finest level, by one block on its shared memory
// (levels 1 .. L-1 of lv; U of level 1 starts at zero, F of level 1 is given).
__device__ void coarse_cycle(const SLv* lv, int L, int nu, int coarse_sweeps)
{
    for (int l = 1; l < L - 1; ++l) {
        const SLv& h = lv[l];
        const SLv& c = lv[l + 1];
        for (int k = 0; k < nu; ++k) {
            s_sweep(h, 0);
            s_sweep(h, 1);
        }
        const int P = c.W * (c.my + 2);
        const float rW = 1.f / (float)c.W;
        for (int idx = threadIdx.x; idx < P; idx += blockDim.x) {
            const int J = qdiv(idx, rW), I = idx - J * c.W;
            mgc_sm[c.U[0] + idx] = mgc_sm[c.U[1] + idx] = 0.f;
            if (I < 1 || I > c.mx || J < 1 || J > c.my) continue;
            const int fc = 2 * J * h.W + 2 * I;
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                float acc = 4.f * s_res(h, f, fc);
                acc += 2.f * (s_res(h, f, fc - 1) + s_res(h, f, fc + 1) + s_res(h, f, fc - h.W) + s_res(h, f, fc + h.W));
                acc += s_res(h, f, fc - h.W - 1) + s_res(h, f, fc - h.W + 1) + s_res(h, f, fc + h.W - 1) +
                       s_res(h, f, fc + h.W + 1);
                mgc_sm[c.F[f] + idx] = acc * (1.f / 16.f);
            }
        }
        __syncthreads();
    }
    {
        const SLv& v = lv[L - 1];
        if (v.mx == 1 && v.my == 1) {
            if (threadIdx.x < 2)
                mgc_sm[v.U[threadIdx.x] + v.W + 1] = mgc_sm[v.F[threadIdx.x] + v.W + 1] / mgc_sm[v.D + v.W + 1];
            __syncthreads();
        } else {
            for (int k = 0; k < coarse_sweeps; ++k) {
                s_sweep(v, 0);
                s_sweep(v, 1);
            }
            for (int k = 0; k < coarse_sweeps; ++k) {
                s_sweep(v, 1);
                s_sweep(v, 0);
            }
        }
    }
    for (int l = L - 2; l >= 1; --l) {
        const SLv& h = lv[l];
        const SLv& c = lv[l + 1];
        const int n = h.mx * h.my;
        const float rmx = 1.f / (float)h.mx;
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const int q = qdiv(k, rmx);
            const int jp = 1 + q, ip = 1 + k - q * h.mx;
            const int I0 = ip >> 1, J0 = jp >> 1, I1 = (ip + 1) >> 1, J1 = (jp + 1) >> 1;
            const int e = jp * h.W + ip;
            float corr[2];
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                const float* Uc = mgc_sm + c.U[f];
                corr[f] = mgc_sm[h.U[f] + e] +
                          0.25f * (Uc[J0 * c.W + I0] + Uc[J0 * c.W + I1] + Uc[J1 * c.W + I0] + Uc[J1 * c.W + I1]);
            }
            mgc_sm[h.U[0] + e] = corr[0];
            mgc_sm[h.U[1] + e] = corr[1];
        }
        __syncthreads();
        for (int k = 0; k < nu; ++k) {
            s_sweep(h, 1);
            s_sweep(h, 0);
        }
    }
}

template <int UPT>
__global__ void __launch_bounds__(SOLVE_THREADS, 1) k_mgc(const MgArgs a, int rows_max)
{
    float* const sm = mgc_sm;
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int sys = blockIdx.x / C;
    const SolveSys S = a.sys[sys];
    const int mx = a.mx[0], my = a.my[0];
    const int W = mx + 2;
    const int r0 = (my * rank) / C, r1 = (my * (rank + 1)) / C;   // rows of this block (interior, 0-based)
    const int rows = r1 - r0;
    const int rows_lo = rank > 0 ? r0 - (my * (rank - 1)) / C : 0;  // rows of the block below
    const int nx = a.nx;
    const int plane = rows_max * W;
    // finest-level vectors with their frame columns (zero): [field][row][column]
    float* Zs = sm;                  // V-cycle iterate z
    float* Ps = sm + 2 * plane;      // search direction p
    float* Rs = sm + 4 * plane;      // residual f - A z inside the V-cycle
    // coarse levels, in every block at the same offsets (only the first block's are used).
    // One copy of their descriptors per block, in shared memory: a per-thread copy would
    // sit in local memory, which the L1 left beside this kernel's shared memory cannot hold.
    __shared__ SLv lv[kMgMaxLevels];
    if (threadIdx.x == 0) {
        int q = 6 * plane;
        for (int l = 1; l < a.levels; ++l) {
            const int Wl = a.mx[l] + 2, P = Wl * (a.my[l] + 2);
            lv[l].mx = a.mx[l];
            lv[l].my = a.my[l];
            lv[l].W = Wl;
            lv[l].D = q;
            lv[l].CX = q + P;
            lv[l].CY = q + 2 * P;
            lv[l].U[0] = q + 3 * P;
            lv[l].U[1] = q + 4 * P;
            lv[l].F[0] = q + 5 * P;
            lv[l].F[1] = q + 6 * P;
            q += 7 * P;
        }
    }
    __syncthreads();
    // the neighbours' planes and the first block's level-1 arrays, at the same offsets
    // from the mapped base of each block's shared memory
    const float* Z_lo = rank > 0 ? cl.map_shared_rank(Zs, rank - 1) : nullptr;
    const float* Z_hi = rank < C - 1 ? cl.map_shared_rank(Zs, rank + 1) : nullptr;
    const float* P_lo = Z_lo ? Z_lo + 2 * plane : nullptr;
    const float* P_hi = Z_hi ? Z_hi + 2 * plane : nullptr;
    const float* R_lo = Z_lo ? Z_lo + 4 * plane : nullptr;
    const float* R_hi = Z_hi ? Z_hi + 4 * plane : nullptr;
    float* const B0 = cl.map_shared_rank(sm, 0);
    float* F1_0 = a.levels > 1 ? B0 + lv[1].F[0] : nullptr;   // the first block's level-1 rhs
    float* F1_1 = a.levels > 1 ? B0 + lv[1].F[1] : nullptr;
    const float* U1_0 = a.levels > 1 ? B0 + lv[1].U[0] : nullptr;
    const float* U1_1 = a.levels > 1 ? B0 + lv[1].U[1] : nullptr;

    __shared__ ClusterSlots4<double> red64[2];
    __shared__ ClusterSlots<float> red32[2];
    int seq = 0, seq64 = 0;

    // zero the finest-level planes; the first block loads the coarse coefficients
    for (int k = threadIdx.x; k < 6 * plane; k += blockDim.x) sm[k] = 0.f;
    if (rank == 0) {
        for (int l = 1; l < a.levels; ++l) {
            const SLv& v = lv[l];
            const int P = v.W * (v.my + 2);
            const long long off = a.off[l] + (long long)sys * P;
            for (int k = threadIdx.x; k < P; k += blockDim.x) {
                sm[v.D + k] = a.D[off + k];
                sm[v.CX + k] = a.CX[off + k];
                sm[v.CY + k] = a.CY[off + k];
                sm[v.U[0] + k] = sm[v.U[1] + k] = 0.f;
                sm[v.F[0] + k] = sm[v.F[1] + k] = 0.f;
            }
        }
    }

    // this thread's unknowns: row lr of the band, padded column c
    int lr_[UPT], c_[UPT];
    bool own[UPT];
#pragma unroll
    for (int k = 0; k < UPT; ++k) {
        const int u0 = threadIdx.x + k * SOLVE_THREADS;
        own[k] = u0 < rows * mx;
        const int u = own[k] ? u0 : 0;
        lr_[k] = u / mx;
        c_[k] = u % mx + 1;
    }
    // global index of unknown k (recomputed where needed rather than held in registers)
    auto gidx = [&](int k) -> long long { return (long long)(S.j0 + r0 + lr_[k]) * nx + (S.i0 + c_[k] - 1); };
    float dg[UPT], cw[UPT], ce[UPT], cs[UPT], cn[UPT], dinv[UPT];
    float r[2][UPT], q[2][UPT], d[2][UPT];
#pragma unroll
    for (int k = 0; k < UPT; ++k) {
        if (own[k]) {
            const long long g = gidx(k);
            dg[k] = a.dgf[g];
            cw[k] = a.cxf[g - 1];
            ce[k] = a.cxf[g];
            cs[k] = a.cyf[g - nx];
            cn[k] = a.cyf[g];
        } else {
            dg[k] = 1.f;
            cw[k] = ce[k] = cs[k] = cn[k] = 0.f;
        }
        dinv[k] = 1.f / dg[k];
#pragma unroll
        for (int f = 0; f < 2; ++f) r[f][k] = q[f][k] = d[f][k] = 0.f;
    }
    cl.sync();

    // neighbour sums of a finest-level plane (frame rows and columns are zero)
    auto nb = [&](const float* V, const float* Vlo, const float* Vhi, int f, int k) -> float {
        const float* row = V + (f * rows_max + lr_[k]) * W;
        const int c = c_[k];
        float s = cw[k] * row[c - 1] + ce[k] * row[c + 1];
        if (lr_[k] > 0) s += cs[k] * row[c - W];
        else if (Vlo) s += cs[k] * Vlo[(f * rows_max + rows_lo - 1) * W + c];
        if (lr_[k] < rows - 1) s += cn[k] * row[c + W];
        else if (Vhi) s += cn[k] * Vhi[(f * rows_max) * W + c];
        return s;
    };
    auto at = [&](float* V, int f, int k) -> float& { return V[(f * rows_max + lr_[k]) * W + c_[k]]; };

    // z = V-cycle(r)
    auto vcycle = [&]() {
#pragma unroll
        for (int k = 0; k < UPT; ++k)
            if (own[k]) at(Zs, 0, k) = at(Zs, 1, k) = 0.f;
        cl.sync();
        // The points of one colour read only the other's: a thread loads its
        // points before it stores them (all of them with up to two per thread;
        // with four, both fields of one point at a time, within the registers).
        auto half = [&](int color) {
            if constexpr (UPT <= 2) {
                float z0[UPT], z1[UPT];
#pragma unroll
                for (int k = 0; k < UPT; ++k)
                    if (own[k] && ((r0 + lr_[k] + c_[k] - 1) & 1) == color) {
                        z0[k] = (r[0][k] + nb(Zs, Z_lo, Z_hi, 0, k)) * dinv[k];
                        z1[k] = (r[1][k] + nb(Zs, Z_lo, Z_hi, 1, k)) * dinv[k];
                    }
#pragma unroll
                for (int k = 0; k < UPT; ++k)
                    if (own[k] && ((r0 + lr_[k] + c_[k] - 1) & 1) == color) {
                        at(Zs, 0, k) = z0[k];
                        at(Zs, 1, k) = z1[k];
                    }
            } else {
#pragma unroll
                for (int k = 0; k < UPT; ++k)
                    if (own[k] && ((r0 + lr_[k] + c_[k] - 1) & 1) == color) {
                        const float z0 = (r[0][k] + nb(Zs, Z_lo, Z_hi, 0, k)) * dinv[k];
                        const float z1 = (r[1][k] + nb(Zs, Z_lo, Z_hi, 1, k)) * dinv[k];
                        at(Zs, 0, k) = z0;
                        at(Zs, 1, k) = z1;
                    }
            }
            cl.sync();
        };
        for (int s = 0; s < a.nu; ++s) {
            half(0);
            half(1);
        }
        if (a.levels > 1) {
            // the fine residual, then its full weighting into the first block's level-1 rhs
#pragma unroll
            for (int k = 0; k < UPT; ++k)
                if (own[k])
#pragma unroll
                    for (int f = 0; f < 2; ++f)
                        at(Rs, f, k) = r[f][k] - (dg[k] * at(Zs, f, k) - nb(Zs, Z_lo, Z_hi, f, k));
            cl.sync();
            const SLv& c1 = lv[1];
            // coarse rows J whose centre fine row 2J - 1 (0-based) lies in this band
            const int J0 = (r0 + 2) / 2, J1 = r1 / 2;   // J with r0 <= 2J - 1 < r1
            const int ncr = J1 - J0 + 1 > 0 ? J1 - J0 + 1 : 0;
            for (int t = threadIdx.x; t < ncr * c1.mx; t += blockDim.x) {
                const int J = J0 + t / c1.mx, I = 1 + t % c1.mx;
                const int lr = 2 * J - 1 - r0;          // centre row in the band
                const int col = 2 * I;                  // padded fine column of the centre
                for (int f = 0; f < 2; ++f) {
                    auto R = [&](int dr, int dc) -> float {
                        const int rr = lr + dr;
                        if (rr < 0) return R_lo ? R_lo[(f * rows_max + rows_lo - 1) * W + col + dc] : 0.f;
                        if (rr >= rows) return R_hi ? R_hi[(f * rows_max) * W + col + dc] : 0.f;
                        return Rs[(f * rows_max + rr) * W + col + dc];
                    };
                    float acc = 4.f * R(0, 0);
                    acc += 2.f * (R(0, -1) + R(0, 1) + R(-1, 0) + R(1, 0));
                    acc += R(-1, -1) + R(-1, 1) + R(1, -1) + R(1, 1);
                    (f == 0 ? F1_0 : F1_1)[J * c1.W + I] = acc * (1.f / 16.f);
                }
            }
            cl.sync();
            if (rank == 0) {
                const int P1 = c1.W * (c1.my + 2);
                for (int k = threadIdx.x; k < P1; k += blockDim.x) sm[c1.U[0] + k] = sm[c1.U[1] + k] = 0.f;
                __syncthreads();
                coarse_cycle(lv, a.levels, a.nu, a.coarse_sweeps);
            }
            cl.sync();
            // z += bilinear interpolation of the level-1 correction
            const int W1 = c1.W;
#pragma unroll
            for (int k = 0; k < UPT; ++k)
                if (own[k]) {
                    const int i = c_[k], j = r0 + lr_[k] + 1;   // 1-based interior coordinates
                    const int I0 = i >> 1, I1 = (i + 1) >> 1, J0c = j >> 1, J1c = (j + 1) >> 1;
                    at(Zs, 0, k) += 0.25f * (U1_0[J0c * W1 + I0] + U1_0[J0c * W1 + I1] + U1_0[J1c * W1 + I0] +
                                             U1_0[J1c * W1 + I1]);
                    at(Zs, 1, k) += 0.25f * (U1_1[J0c * W1 + I0] + U1_1[J0c * W1 + I1] + U1_1[J1c * W1 + I0] +
                                             U1_1[J1c * W1 + I1]);
                }
            cl.sync();
        }
        for (int s = 0; s < a.nu; ++s) {
            half(1);
            half(0);
        }
    };

    // double-precision residual of x into r (single precision), ||r||^2 and ||b||^2
    auto residual64 = [&](double& rr0, double& rr1, double& bb0, double& bb1) {
        double t[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int k = 0; k < UPT; ++k) {
            if (!own[k]) continue;
            const long long g = gidx(k);
            const int i = S.i0 + c_[k] - 1, j = S.j0 + r0 + lr_[k];
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                const double* x = a.x[f];
                const double* rhs = a.rhs0 + (long long)f * nx * a.ny;
                const double ax = a.dg[g] * x[g] - a.cx[g - 1] * x[g - 1] - a.cx[g] * x[g + 1] -
                                  a.cy[g - nx] * x[g - nx] - a.cy[g] * x[g + nx];
                const double res = rhs[g] - ax;
                double b = rhs[g];
                if (i == S.i0) b += a.cx[g - 1] * x[g - 1];
                if (i == S.i1 - 1) b += a.cx[g] * x[g + 1];
                if (j == S.j0) b += a.cy[g - nx] * x[g - nx];
                if (j == S.j1 - 1) b += a.cy[g] * x[g + nx];
                t[f] += res * res;
                t[2 + f] += b * b;
                r[f][k] = (float)res;
                d[f][k] = 0.f;
            }
        }
        cluster_sum4(cl, red64, seq64, t);
        rr0 = t[0];
        rr1 = t[1];
        bb0 = t[2];
        bb1 = t[3];
    };

    double rr[2], bb[2];
    residual64(rr[0], rr[1], bb[0], bb[1]);
    const double stop2[2] = {a.rtol * a.rtol * bb[0], a.rtol * a.rtol * bb[1]};
    bool conv[2] = {rr[0] <= stop2[0], rr[1] <= stop2[1]};
    int iters[2] = {0, 0}, total = 0;
    for (int outer = 0; outer < a.outer && !(conv[0] && conv[1]) && total < a.max_iter; ++outer) {
        bool act[2] = {!conv[0], !conv[1]};
        const float rr0[2] = {(float)rr[0], (float)rr[1]};
        vcycle();
        float rz[2] = {0.f, 0.f};
#pragma unroll
        for (int k = 0; k < UPT; ++k)
            if (own[k])
#pragma unroll
                for (int f = 0; f < 2; ++f) {
                    at(Ps, f, k) = at(Zs, f, k);
                    rz[f] += r[f][k] * at(Zs, f, k);
                }
        cluster_sum2(cl, red32, seq, rz[0], rz[1]);   // its barrier also publishes p
        while ((act[0] || act[1]) && total < a.max_iter) {
            ++total;
            float pq[2] = {0.f, 0.f};
#pragma unroll
            for (int k = 0; k < UPT; ++k)
                if (own[k])
#pragma unroll
                    for (int f = 0; f < 2; ++f) {
                        q[f][k] = dg[k] * at(Ps, f, k) - nb(Ps, P_lo, P_hi, f, k);
                        pq[f] += at(Ps, f, k) * q[f][k];
                    }
            cluster_sum2(cl, red32, seq, pq[0], pq[1]);
            float alpha[2];
#pragma unroll
            for (int f = 0; f < 2; ++f) alpha[f] = (act[f] && pq[f] > 0.f) ? rz[f] / pq[f] : 0.f;
            float rn[2] = {0.f, 0.f};
#pragma unroll
            for (int k = 0; k < UPT; ++k)
                if (own[k])
#pragma unroll
                    for (int f = 0; f < 2; ++f) {
                        d[f][k] += alpha[f] * at(Ps, f, k);
                        r[f][k] -= alpha[f] * q[f][k];
                        rn[f] += r[f][k] * r[f][k];
                    }
            cluster_sum2(cl, red32, seq, rn[0], rn[1]);
#pragma unroll
            for (int f = 0; f < 2; ++f)
                if (act[f]) {
                    ++iters[f];
                    if (!(rn[f] > a.inner_tol * a.inner_tol * rr0[f])) act[f] = false;
                }
            if (!(act[0] || act[1])) break;
            vcycle();
            float rz_new[2] = {0.f, 0.f};
#pragma unroll
            for (int k = 0; k < UPT; ++k)
                if (own[k])
#pragma unroll
                    for (int f = 0; f < 2; ++f) rz_new[f] += r[f][k] * at(Zs, f, k);
            cluster_sum2(cl, red32, seq, rz_new[0], rz_new[1]);
            float beta[2];
#pragma unroll
            for (int f = 0; f < 2; ++f) beta[f] = (act[f] && rz[f] > 0.f) ? rz_new[f] / rz[f] : 0.f;
#pragma unroll
            for (int k = 0; k < UPT; ++k)
                if (own[k])
#pragma unroll
                    for (int f = 0; f < 2; ++f) at(Ps, f, k) = at(Zs, f, k) + beta[f] * at(Ps, f, k);
            rz[0] = rz_new[0];
            rz[1] = rz_new[1];
            cl.sync();   // p complete before the next product
        }
        // x += d (double precision) where still short of rtol; the next residual reads neighbours' x
#pragma unroll
        for (int k = 0; k < UPT; ++k)
            if (own[k])
#pragma unroll
                for (int f = 0; f < 2; ++f)
                    if (!conv[f]) a.x[f][gidx(k)] += (double)d[f][k];
        cl.sync();
        residual64(rr[0], rr[1], bb[0], bb[1]);
        conv[0] = rr[0] <= stop2[0];
        conv[1] = rr[1] <= stop2[1];
    }
    if (threadIdx.x == 0 && rank == 0) {
        const bool ok = conv[0] && conv[1];
        a.sys_iters[sys] = ok ? max(iters[0], iters[1]) : a.max_iter + 1;
        if (!ok) atomicOr(a.status, STATUS_NOCONV);
    }
    cl.sync();   // no block leaves while others may still read its shared memory
}

template <int UPT>
cudaError_t launch_mgc_t(const MgArgs& a, int C, int rows_max, size_t smem, cudaStream_t s)
{
    if (C > 8) cudaFuncSetAttribute(k_mgc<UPT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaError_t e = cudaFuncSetAttribute(k_mgc<UPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(a.nsys * C));
    cfg.blockDim = dim3(SOLVE_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_mgc<UPT>, a, rows_max);
}

}  // namespace

// Cluster shape for the in-cluster solver: C blocks (a power of two, at most
// 16) such that a block's band fits max_upt (2 or 4) unknowns per thread; 0
// when the subdomain is too large (band or shared memory). Four unknowns per
// thread halve the SMs the solve holds (for a solve that runs beside other
// work) at some cost in its own time.
int mgc_config(const MgArgs& a, int* C_out, int* rows_max_out, size_t* smem_out, int max_upt)
{
    const int mx = a.mx[0], my = a.my[0];
    const int per_block = (max_upt >= 4 ? 4 : 2) * SOLVE_THREADS;
    int C = 1;
    while (C < 16 && (((my + C - 1) / C) * mx > per_block)) C *= 2;
    const int rows_max = (my + C - 1) / C;
    if (rows_max * mx > per_block || C > my) return 0;
    // the coarse levels' index quotients are exact in single precision (qdiv) below this size
    for (int l = 1; l < a.levels; ++l) {
        const long long Wl = a.mx[l] + 2;
        if (Wl * Wl * (a.my[l] + 2) >= (1LL << 21)) return 0;
    }
    size_t floats = 6 * (size_t)rows_max * (mx + 2);
    for (int l = 1; l < a.levels; ++l) floats += 7 * (size_t)(a.mx[l] + 2) * (a.my[l] + 2);
    const size_t smem = floats * sizeof(float);
    if (smem > 220 * 1024) return 0;
    *C_out = C;
    *rows_max_out = rows_max;
    *smem_out = smem;
    const int band = rows_max * mx;
    return band > 2 * SOLVE_THREADS ? 4 : band > SOLVE_THREADS ? 2 : 1;
}

cudaError_t launch_mgc(const MgArgs& a, int upt, int C, int rows_max, size_t smem, cudaStream_t s)
{
    if (upt == 1) return launch_mgc_t<1>(a, C, rows_max, smem, s);
    if (upt == 4) return launch_mgc_t<4>(a, C, rows_max, smem, s);
    return launch_mgc_t<2>(a, C, rows_max, smem, s);
}

}  // namespace sdd
