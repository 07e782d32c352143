// chol.cu -- direct subdomain solves for small subdomains (Sec. 4).
//
// The paper solves each subdomain's implicit system directly (LU). The system
// of solve.cu (symmetric positive definite, five-point) is, in the natural
// row-major order of a subdomain's mx x my unknowns, banded with bandwidth mx;
// for mx <= 32 and a band that fits in shared memory one block per subdomain
// factors it, A = L D L^T (right-looking banded LDL^T, no square roots), and
// solves both fields, one warp per field, by forward, diagonal and backward
// substitution.
//
// Precision: as the iterative solvers, the factorisation and the
// substitutions run in single precision (GB300's double-precision units are
// few and their dependency chains long) inside an iterative refinement in
// double precision: x += (L D L^T)^-1 r, r = b - A x formed in double precision
// from the double-precision coefficients, until ||r|| <= rtol ||b|| for both
// fields (at most CHOL_SWEEPS sweeps; each gains about -log10(cond(A) 2^-24)
// digits); a field that does not get there sets the status bit.
//
// Speed: the factorisation is m sequential column steps (one block barrier
// each) and every substitution 2 m sequential steps; on 19 x 19 subdomains a
// solve with its set-up takes 176 us against 159 us for Jacobi-PCG (51
// iterations), on 31 x 31 605 against 222 us. It is the exact solve the
// paper uses, offered on request, not the automatic choice.
//
// Layout in shared memory: row k of the band holds, at d = 0 .. mx, the
// factorisation's working values S(k, k - d) (single precision): d = 0 the
// pivot D(k), d > 0 the unscaled column entries, L(k, k - d) = S(k, k - d) /
// D(k - d); then 1 / D(k); per field the right-hand side b, the solution x
// (double precision) and the correction (single precision); the (p, q) pairs
// of the trailing update's triangle.
#include "chol.cuh"

namespace sdd {
namespace {

constexpr int CHOL_THREADS = 256;
constexpr int CHOL_MAX_BW = 32;
constexpr int CHOL_SWEEPS = 6;

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(CHOL_THREADS) k_chol(const SolveArgs a)
{
    extern __shared__ double sh[];
    __shared__ int bad;
    __shared__ double red[CHOL_THREADS / 32][4];
    __shared__ int done;
    const SolveSys S = a.sys[blockIdx.x];
    const int mx = S.i1 - S.i0, my = S.j1 - S.j0, m = mx * my, bw = mx, W = bw + 1;
    const int nx = a.nx;
    const long long plane = (long long)nx * a.ny;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double* bv = sh;                                             // [2][m] right-hand sides
    double* xv = bv + 2 * (size_t)m;                             // [2][m] solutions
    float* L = reinterpret_cast<float*>(xv + 2 * (size_t)m);     // [m][W]
    float* dinv = L + (size_t)m * W;                             // [m]
    float* cv = dinv + m;                                        // [2][m] corrections
    const size_t fl = (size_t)m * W + 3 * (size_t)m;            // floats before the pairs: padded to 8 bytes
    int2* tri = reinterpret_cast<int2*>(L + fl + (fl & 1));    // [bw (bw + 1) / 2]
    auto gidx = [&](int k) {
        const int jj = k / mx, ii = k - jj * mx;
        return (long long)(S.j0 + jj) * nx + (S.i0 + ii);
    };

    // the band of A (lower part), the right-hand sides with the Dirichlet neighbours
    if (tid == 0) {
        bad = 0;
        done = 0;
    }
    for (int k = tid; k < m; k += CHOL_THREADS) {
        const int jj = k / mx, ii = k - jj * mx;
        const long long g = gidx(k);
        float* row = L + (size_t)k * W;
        for (int d = 0; d <= bw; ++d) row[d] = 0.f;
        row[0] = (float)a.dg[g];
        if (ii > 0) row[1] = (float)-a.cx[g - 1];
        if (jj > 0) row[bw] = (float)-a.cy[g - nx];
        for (int f = 0; f < 2; ++f) {
            const double* x = a.x[f];
            double b = a.rhs0[f * plane + g];
            if (ii == 0) b += a.cx[g - 1] * x[g - 1];
            if (ii == mx - 1) b += a.cx[g] * x[g + 1];
            if (jj == 0) b += a.cy[g - nx] * x[g - nx];
            if (jj == my - 1) b += a.cy[g] * x[g + nx];
            bv[f * m + k] = b;
            xv[f * m + k] = 0.0;
            cv[f * m + k] = (float)b;     // the first correction solves A x = b itself
        }
    }
    // the trailing update's pairs (p, q), 1 <= q <= p <= bw, row by row: the first
    // nb (nb + 1) / 2 of them are the pairs with p <= nb
    for (int p = 1 + tid; p <= bw; p += CHOL_THREADS)
        for (int q = 1; q <= p; ++q) tri[p * (p - 1) / 2 + q - 1] = make_int2(p, q);
    __syncthreads();

    // A = L D L^T, column by column: every thread forms 1 / D(c) from the pivot, then
    // the trailing window S(i, t) -= S(i, c) S(t, c) / D(c), c < t <= i <= c + nb
    for (int c = 0; c < m; ++c) {
        const float d = L[(size_t)c * W];
        const float r = 1.f / d;
        if (tid == 0) {
            if (!(d > 0.f)) bad = 1;
            dinv[c] = r;
        }
        const int nb = min(bw, m - 1 - c);
        const int ne = nb * (nb + 1) / 2;
        for (int e = tid; e < ne; e += CHOL_THREADS) {
            const int2 pq = tri[e];
            const int i = c + pq.x, t = c + pq.y;
            L[(size_t)i * W + (i - t)] -= L[(size_t)i * W + pq.x] * (L[(size_t)t * W + pq.y] * r);
        }
        __syncthreads();
    }

    double t4[4] = {0.0, 0.0, 0.0, 0.0};
    for (int sweep = 0; sweep < CHOL_SWEEPS; ++sweep) {
        // the correction: L y = r, D z = y, L^T e = z in place, one warp per field
        // (bw <= 32: a lane per band entry); L(i, c) = S(i, c) / D(c)
        if (warp < 2) {
            float* e = cv + (size_t)warp * m;
            for (int c = 0; c < m; ++c) {
                const float yc = e[c] * dinv[c];   // L(i, c) y(c) = S(i, c) (y(c) / D(c))
                const int i = c + 1 + lane;
                if (lane < bw && i < m) e[i] -= L[(size_t)i * W + (i - c)] * yc;
                __syncwarp();
            }
            for (int k = lane; k < m; k += 32) e[k] *= dinv[k];
            __syncwarp();
            for (int c = m - 1; c >= 0; --c) {
                const float xc = e[c];
                const int i = c - 1 - lane;
                if (lane < bw && i >= 0) e[i] -= (L[(size_t)c * W + (c - i)] * dinv[i]) * xc;
                __syncwarp();
            }
        }
        __syncthreads();
        // x += e, then r = b - A x in double precision (the next correction's right-hand side)
        for (int k = tid; k < 2 * m; k += CHOL_THREADS) xv[k] += (double)cv[k];
        __syncthreads();
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int k = tid; k < m; k += CHOL_THREADS) {
            const int jj = k / mx, ii = k - jj * mx;
            const long long g = gidx(k);
            for (int f = 0; f < 2; ++f) {
                const double* x = xv + (size_t)f * m;
                double ax = a.dg[g] * x[k];
                if (ii > 0) ax -= a.cx[g - 1] * x[k - 1];
                if (ii < mx - 1) ax -= a.cx[g] * x[k + 1];
                if (jj > 0) ax -= a.cy[g - nx] * x[k - mx];
                if (jj < my - 1) ax -= a.cy[g] * x[k + mx];
                const double r = bv[f * m + k] - ax;
                cv[f * m + k] = (float)r;
                acc[f] += r * r;
                acc[2 + f] += bv[f * m + k] * bv[f * m + k];
            }
        }
        for (int q = 0; q < 4; ++q) acc[q] = warp_sum_d(acc[q]);
        if (lane == 0)
            for (int q = 0; q < 4; ++q) red[warp][q] = acc[q];
        __syncthreads();
        if (tid == 0) {
            for (int q = 0; q < 4; ++q) t4[q] = 0.0;
            for (int w = 0; w < CHOL_THREADS / 32; ++w)
                for (int q = 0; q < 4; ++q) t4[q] += red[w][q];
            const double tol2 = a.rtol * a.rtol;
            done = bad || (t4[0] <= tol2 * t4[2] && t4[1] <= tol2 * t4[3]);
        }
        __syncthreads();
        if (done) break;   // uniform over the block
    }

    // the solutions into the fields; after a pivot that is not positive (or not a number) the
    // fields keep their previous values and only the status reports the failure
    for (int k = tid; k < m && !bad; k += CHOL_THREADS) {
        const long long g = gidx(k);
        a.x[0][g] = xv[k];
        a.x[1][g] = xv[(size_t)m + k];
    }
    if (tid == 0) {
        const double tol2 = a.rtol * a.rtol;
        const bool ok = !bad && t4[0] <= tol2 * t4[2] && t4[1] <= tol2 * t4[3];
        a.iters[blockIdx.x] = ok ? 1 : a.max_iter + 1;
        if (!ok) atomicOr(a.status, STATUS_NOCONV);
    }
}

size_t chol_smem(int mx, int my)
{
    const size_t m = (size_t)mx * my;
    const size_t floats = m * (mx + 1) + m + 2 * m + 1;   // band, 1 / D, corrections, alignment
    return 4 * m * sizeof(double) + floats * sizeof(float) + (size_t)mx * (mx + 1) / 2 * sizeof(int2);
}

}  // namespace

bool chol_fits(int mx, int my) { return mx >= 1 && my >= 1 && mx <= CHOL_MAX_BW && chol_smem(mx, my) <= 200 * 1024; }

cudaError_t launch_chol(const SolveArgs& a, int mx_max, int my_max, cudaStream_t s)
{
    if (a.nsys <= 0) return cudaSuccess;
    const size_t smem = chol_smem(mx_max, my_max);
    cudaError_t e = cudaFuncSetAttribute(k_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_chol<<<a.nsys, CHOL_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace sdd
