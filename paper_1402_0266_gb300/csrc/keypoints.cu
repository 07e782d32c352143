// keypoints.cu -- key-point placement and interface fill (Sec. 4, Sec. 5).
//
// Sec. 4 evaluates the stochastic solution only near the maxima and minima of
// rho_x, rho_xx along the horizontal interfaces and of rho_y, rho_yy along the
// vertical ones (rho = 1 / w as in Sec. 5); Sec. 5 fills the other interface
// points by piecewise cubic Hermite interpolation. Along a line with positions
// t = 0 .. n - 1 (t = 0 and n - 1 on the boundary):
//
//   D1(t) = rho(t + 1) - rho(t - 1),  D2(t) = (rho(t + 1) - rho(t)) - (rho(t) - rho(t - 1))
//
// for t = 1 .. n - 2 in double precision (undivided: the grid spacing does not
// move an extremum). A position t in 2 .. n - 3 is a key point when D1 or D2
// has a local extremum there (p(t) > p(t - 1) and p(t) >= p(t + 1), or the
// mirror) of size |p(t)| >= max |p| / 100 (smaller ones are rounding noise
// where rho is flat); crossings of a vertical and a horizontal line are
// always key points, and so, with a spacing g > 0, is every position t with
// t mod g = 0 (the mesh also moves where rho is flat along a line). The fill is the monotone PCHIP interpolant (Fritsch &
// Carlson's scheme with Fritsch & Butland's derivative formula) through the
// line's two boundary values and its key points' estimates.
#include <algorithm>

#include "common.cuh"

namespace sdd {
namespace {

constexpr int KP_THREADS = 1024;

__device__ __forceinline__ long long line_node(const KeyLine& L, int nx, int t)
{
    // vertical line: column fixed, row t; horizontal line: row fixed, column t
    return L.orient == 0 ? (long long)t * nx + L.fixed : (long long)L.fixed * nx + t;
}

// One block per line: the profiles in shared memory, their largest sizes, then
// the extremum test at every position the line owns.
__global__ void __launch_bounds__(KP_THREADS) k_keypoints(const float* __restrict__ w, int nx,
                                                           const KeyLine* __restrict__ lines,
                                                           const int32_t* __restrict__ pos_idx,
                                                           const uint8_t* __restrict__ pos_cross,
                                                           int spacing, uint8_t* __restrict__ mask)
{
    extern __shared__ double prof[];   // D1 at [0, n), D2 at [n, 2n): entry t for t = 1 .. n - 2
    __shared__ double red[2][KP_THREADS / 32];
    const KeyLine L = lines[blockIdx.x];
    const int n = L.n;
    double m1 = 0.0, m2 = 0.0;
    for (int t = 1 + threadIdx.x; t <= n - 2; t += blockDim.x) {
        const double rm = 1.0 / (double)w[line_node(L, nx, t - 1)];
        const double r0 = 1.0 / (double)w[line_node(L, nx, t)];
        const double rp = 1.0 / (double)w[line_node(L, nx, t + 1)];
        const double d1 = rp - rm;
        const double d2 = (rp - r0) - (r0 - rm);
        prof[t] = d1;
        prof[n + t] = d2;
        m1 = fmax(m1, fabs(d1));
        m2 = fmax(m2, fabs(d2));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o; o >>= 1) {
        m1 = fmax(m1, __shfl_xor_sync(0xffffffffu, m1, o));
        m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
    }
    if (lane == 0) {
        red[0][wid] = m1;
        red[1][wid] = m2;
    }
    __syncthreads();
    double big[2] = {0.0, 0.0};
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
        big[0] = fmax(big[0], red[0][q]);
        big[1] = fmax(big[1], red[1][q]);
    }
    for (int t = 1 + threadIdx.x; t <= n - 2; t += blockDim.x) {
        const int k = L.start + t - 1;
        if (pos_cross[k]) {
            if (L.orient == 0) mask[pos_idx[k]] = 1;   // a crossing belongs to its vertical line
            continue;
        }
        uint8_t key = (spacing > 0 && t % spacing == 0) ? 1 : 0;
        if (t >= 2 && t <= n - 3) {
            for (int q = 0; q < 2; ++q) {
                const double* p = prof + q * n;
                const double pm = p[t - 1], p0 = p[t], pp = p[t + 1];
                if (big[q] == 0.0 || fabs(p0) * 100.0 < big[q]) continue;
                if ((p0 > pm && p0 >= pp) || (p0 < pm && p0 <= pp)) key = 1;
            }
        }
        mask[pos_idx[k]] = key;
    }
}

// PCHIP of one field along one line (the calling thread alone): anchors
// (ax, ay) at the line's two ends and its key points, their derivatives ad,
// then the positions the line owns that are not key points. key(t), val(t),
// idx(t) and cross(t) describe interior position t = 1 .. n - 2.
template <typename Key, typename Val, typename Idx, typename Cross, typename IT, typename DT>
__device__ __forceinline__ void pchip_line(const KeyLine& L, double y_start, double y_end, Key key, Val val, Idx idx,
                                           Cross cross, IT* ax, DT* ay, DT* ad, double* __restrict__ mean)
{
    const int n = L.n;
    int m = 0;
    ax[m] = 0;
    ay[m++] = y_start;
    for (int t = 1; t <= n - 2; ++t)
        if (key(t)) {
            ax[m] = t;
            ay[m++] = val(t);
        }
    ax[m] = n - 1;
    ay[m++] = y_end;
    // derivatives (Fritsch-Butland weighted harmonic mean inside, shape-preserving three-point ends)
    if (m == 2) {
        ad[0] = ad[1] = (ay[1] - ay[0]) / (double)(ax[1] - ax[0]);
    } else {
        for (int k = 1; k < m - 1; ++k) {
            const double h0 = (double)(ax[k] - ax[k - 1]), h1 = (double)(ax[k + 1] - ax[k]);
            const double s0 = (ay[k] - ay[k - 1]) / h0, s1 = (ay[k + 1] - ay[k]) / h1;
            if (s0 == 0.0 || s1 == 0.0 || (s0 > 0.0) != (s1 > 0.0)) {
                ad[k] = 0.0;
            } else {
                const double w1 = 2.0 * h1 + h0, w2 = h1 + 2.0 * h0;
                ad[k] = (w1 + w2) / (w1 / s0 + w2 / s1);
            }
        }
        for (int e = 0; e < 2; ++e) {
            // end derivative from the first (last) two intervals
            const int a = e == 0 ? 0 : m - 1, b = e == 0 ? 1 : m - 2, c = e == 0 ? 2 : m - 3;
            const double h0 = fabs((double)(ax[b] - ax[a])), h1 = fabs((double)(ax[c] - ax[b]));
            const double s0 = (ay[b] - ay[a]) / (double)(ax[b] - ax[a]), s1 = (ay[c] - ay[b]) / (double)(ax[c] - ax[b]);
            double d = ((2.0 * h0 + h1) * s0 - h0 * s1) / (h0 + h1);
            const auto sgn = [](double v) { return (v > 0.0) - (v < 0.0); };
            if (sgn(d) != sgn(s0)) d = 0.0;
            else if (sgn(s0) != sgn(s1) && fabs(d) > fabs(3.0 * s0)) d = 3.0 * s0;
            ad[a] = d;
        }
    }
    // evaluate at the positions this line owns that are not key points
    int seg = 0;
    for (int t = 1; t <= n - 2; ++t) {
        if (key(t) || (L.orient == 1 && cross(t))) continue;
        const double x = (double)t;
        while (seg < m - 2 && (double)ax[seg + 1] < x) ++seg;
        const double h = (double)(ax[seg + 1] - ax[seg]);
        const double s = (ay[seg + 1] - ay[seg]) / h;
        const double c3 = (ad[seg] + ad[seg + 1] - 2.0 * s) / (h * h);
        const double c2 = (s - ad[seg]) / h - (ad[seg] + ad[seg + 1] - 2.0 * s) / h;
        const double u = x - (double)ax[seg];
        mean[idx(t)] = ((c3 * u + c2) * u + ad[seg]) * u + ay[seg];
    }
}

// The boundary values of field f at the two ends of line L.
__device__ __forceinline__ void line_ends(const KeyLine& L, const double* faces, int f, int nx, int ny, double& y0,
                                          double& y1)
{
    // face data: per field left[ny] right[ny] bottom[nx] top[nx]
    const double* F = faces + (long long)f * (2LL * ny + 2LL * nx);
    y0 = L.orient == 0 ? F[2 * ny + L.fixed] : F[L.fixed];
    y1 = L.orient == 0 ? F[2 * ny + nx + L.fixed] : F[ny + L.fixed];
}

constexpr int PCHIP_THREADS = 64;

// Shared-memory bytes of k_pchip_smem for lines of up to n positions.
size_t pchip_smem_bytes(int n) { return (size_t)n * (6 * sizeof(double) + 3 * sizeof(int32_t) + 1); }

// One block per line: the block stages the line's node indices, key and
// crossing flags and key-point estimates in shared memory (in parallel), then
// thread f < 2 interpolates field f there.
__global__ void __launch_bounds__(PCHIP_THREADS) k_pchip_smem(const KeyLine* __restrict__ lines,
                                                              const int32_t* __restrict__ pos_idx,
                                                              const uint8_t* __restrict__ pos_cross,
                                                              const uint8_t* __restrict__ mask,
                                                              const double* __restrict__ faces, int nx, int ny,
                                                              double* __restrict__ mean_xi,
                                                              double* __restrict__ mean_eta, int max_n)
{
    extern __shared__ double sp[];
    const KeyLine L = lines[blockIdx.x];
    const int n = L.n;
    double* val = sp;                                   // [2][max_n] key-point estimates
    double* ay = sp + 2LL * max_n;                      // [2][max_n]
    double* ad = sp + 4LL * max_n;                      // [2][max_n]
    int32_t* ax = reinterpret_cast<int32_t*>(sp + 6LL * max_n);   // [2][max_n]
    int32_t* idx = ax + 2LL * max_n;                    // [max_n]
    uint8_t* flag = reinterpret_cast<uint8_t*>(idx + max_n);     // [max_n]: bit 0 key, bit 1 crossing
    for (int t = 1 + threadIdx.x; t <= n - 2; t += blockDim.x) {
        const int k = L.start + t - 1;
        const int i = pos_idx[k];
        const uint8_t key = mask[i];
        idx[t] = i;
        flag[t] = (uint8_t)((key ? 1 : 0) | (pos_cross[k] ? 2 : 0));
        if (key) {
            val[t] = mean_xi[i];
            val[max_n + t] = mean_eta[i];
        }
    }
    __syncthreads();
    const int f = threadIdx.x;
    if (f >= 2) return;
    double y0, y1;
    line_ends(L, faces, f, nx, ny, y0, y1);
    const double* v = val + (long long)f * max_n;
    pchip_line(
        L, y0, y1, [&](int t) { return (flag[t] & 1) != 0; }, [&](int t) { return v[t]; },
        [&](int t) { return idx[t]; }, [&](int t) { return (flag[t] & 2) != 0; }, ax + (long long)f * max_n,
        ay + (long long)f * max_n, ad + (long long)f * max_n, f == 0 ? mean_xi : mean_eta);
}

// Lines too long for shared memory: one block per line, thread f < 2
// interpolates field f with its anchors in global scratch.
__global__ void k_pchip(const KeyLine* __restrict__ lines, const int32_t* __restrict__ pos_idx,
                        const uint8_t* __restrict__ pos_cross, const uint8_t* __restrict__ mask,
                        const double* __restrict__ faces, int nx, int ny, double* __restrict__ mean_xi,
                        double* __restrict__ mean_eta, double* __restrict__ scratch)
{
    const int f = threadIdx.x;
    if (f >= 2) return;
    const KeyLine L = lines[blockIdx.x];
    const int n = L.n;
    double* mean = f == 0 ? mean_xi : mean_eta;
    double y0, y1;
    line_ends(L, faces, f, nx, ny, y0, y1);
    // anchors: (x, y) and their derivatives, in this line's scratch region (three arrays of n per field;
    // the lines before this one hold L.start + 2 blockIdx.x positions in all)
    double* ax = scratch + 6LL * (L.start + 2LL * blockIdx.x) + 3LL * f * n;
    double* ay = ax + n;
    double* ad = ay + n;
    pchip_line(
        L, y0, y1, [&](int t) { return mask[pos_idx[L.start + t - 1]] != 0; },
        [&](int t) { return mean[pos_idx[L.start + t - 1]]; }, [&](int t) { return pos_idx[L.start + t - 1]; },
        [&](int t) { return pos_cross[L.start + t - 1] != 0; }, ax, ay, ad, mean);
}

}  // namespace

cudaError_t launch_keypoints(const float* w, int nx, const KeyLine* lines, int nlines, int max_n,
                             const int32_t* pos_idx, const uint8_t* pos_cross, int spacing, uint8_t* mask,
                             cudaStream_t s)
{
    if (nlines <= 0) return cudaSuccess;
    const size_t smem = 2 * (size_t)max_n * sizeof(double);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_keypoints, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_keypoints<<<nlines, KP_THREADS, smem, s>>>(w, nx, lines, pos_idx, pos_cross, spacing, mask);
    return cudaGetLastError();
}

size_t pchip_scratch_doubles(long long total_positions, int nlines)
{
    return (size_t)(6 * (total_positions + 2LL * nlines) + 16);
}

cudaError_t launch_pchip(const KeyLine* lines, int nlines, int max_n, const int32_t* pos_idx,
                         const uint8_t* pos_cross, const uint8_t* mask, const double* faces, int nx, int ny,
                         double* mean_xi, double* mean_eta, double* scratch, cudaStream_t s)
{
    if (nlines <= 0) return cudaSuccess;
    const size_t smem = pchip_smem_bytes(max_n);
    if (smem <= 200 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_pchip_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_pchip_smem<<<nlines, PCHIP_THREADS, smem, s>>>(lines, pos_idx, pos_cross, mask, faces, nx, ny, mean_xi,
                                                         mean_eta, max_n);
    } else {
        k_pchip<<<nlines, 32, 0, s>>>(lines, pos_idx, pos_cross, mask, faces, nx, ny, mean_xi, mean_eta, scratch);
    }
    return cudaGetLastError();
}

}  // namespace sdd
