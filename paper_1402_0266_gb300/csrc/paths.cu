// paths.cu -- the interface Monte Carlo path kernel and the per-node reduction.
//
// Each path solves dX = -(1/w) grad w dt + sqrt(2) dW (Eq. 7a with the
// Winslow coefficients of Eq. 6) from its node by Euler--Maruyama over the K
// sub-steps of one mesh step (Sec. 4), with dW = sqrt(dt) N(0,1), the drift
// interpolated bilinearly between the grid nodes, and a boundary test after
// every sub-step. A path that leaves scores the boundary data f, g at its exit
// point; a path that stays scores xi, eta of the start of the mesh step at its
// end point (Eq. 7b). The node's estimate is the mean over its paths (Sec. 4).
//
// Execution: a persistent grid; each warp repeatedly takes a task (one node,
// a contiguous range of its paths) from a counter, on its own. Each lane runs one path at
// a time and, when its path ends, takes the task's next unstarted path, so
// lanes stay busy when paths leave early. In the paper's (plain) exit mode one
// Philox block supplies the normals of two consecutive sub-steps, so paths are
// only started at even sub-step boundaries. Scores are summed per lane with
// compensation (single precision, shifted by the node's start coordinates),
// then per warp in double precision; the per-node reduction over tasks runs in
// a fixed order, so results do not depend on scheduling.
//
// Deferred scoring: when the fields of the step's start are still being
// computed beside the path kernel (pipelined mesh steps), a surviving path
// leaves its end point (and control-variate sums) in a record array instead,
// and so does a path that leaves by the plain test (the sub-step that crossed
// the boundary: scoring it here would hold its warp on the face-table loads);
// k_score_surv scores the records once the fields are final, then runs the
// per-node reduction.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"

namespace sdd {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// Positions and both components of every bilinear field travel as float2 so
// that GB300's paired single-precision instructions (FFMA2, FADD2, FMUL2)
// handle x and y together.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

struct Cell {
    float2 st;        // local coordinates (s, t) in [0, 1)
    uint32_t idx;     // row-major cell index
};

// Cell of pos and local coordinates. floor() through a directed add of 2^23:
// for 0 <= g < 2^23, (g + 2^23) rounded down is 2^23 + floor(g) exactly, and
// its bits are 0x4B000000 + floor(g); cell_bias removes that offset from the
// row-major cell index in 32-bit wrap-around arithmetic.
__device__ __forceinline__ Cell locate(const InstDev& I, float2 pos)
{
    float2 g = __fmul2_rn(pos, f2(I.sx, I.sy));
    g.x = fminf(g.x, I.gxmax);
    g.y = fminf(g.y, I.gymax);
    const float2 t = __fadd2_rd(g, f2(8388608.0f, 8388608.0f));
    const uint32_t cell = __float_as_uint(t.y) * (uint32_t)(I.nx - 1) + __float_as_uint(t.x) - I.cell_bias;
    const float2 fl = __fadd2_rn(t, f2(-8388608.0f, -8388608.0f));    // floor(g), exact
    Cell c;
    c.st = __ffma2_rn(fl, f2(-1.0f, -1.0f), g);                        // g - floor(g), exact
    c.idx = cell;
    return c;
}

// The two coefficient records of cell idx in a table of cell records.
__device__ __forceinline__ const float4* rec2(const float4* base, uint32_t idx) { return base + 2 * (size_t)idx; }

// The drift records of a cell. With the zero map (ZM), a cell of a segment
// whose drift records are all zero (w constant around it: b = -grad w / w = 0
// exactly) reads the all-zero record at index zcell instead: the same values,
// so the same arithmetic and results, but every lane of a warp that is in such
// a segment reads the same 32 bytes, one L1 wavefront for all of them, where
// each lane's own cell would cost one wavefront per lane. zsm: the map in
// shared memory, bit k of word k / 32 set when a record of cells
// [k 2^zshift, (k + 1) 2^zshift) is nonzero; word w sits at zmap_slot(w).
// Shared-memory slot of map word w: the word's bank (its low five bits) xored
// with the next five bits. A warp's lanes sit in nearby rows of cells, whose
// words lie a multiple of 32 apart where rows are 32 words long or a divisor
// of that: unswizzled they would share a bank and serialise the load.
__device__ __forceinline__ uint32_t zmap_slot(uint32_t w) { return w ^ ((w >> 5) & 31u); }

template <bool ZM>
__device__ __forceinline__ const float4* drift_rec(const InstDev& I, const Cell& c, const uint32_t* zsm,
                                                   const PathArgs& a)
{
    uint32_t idx = c.idx;
    if (ZM) {
        const uint32_t seg = idx >> a.zshift;
        if (!((zsm[zmap_slot(seg >> 5)] >> (seg & 31u)) & 1u)) idx = a.zcell;
    }
    return rec2(I.bcoef, idx);
}

// A cell's two records in one 256-bit read-only load (records are 32-byte
// aligned): one L1 request per gather instead of two for the same sector.
__device__ __forceinline__ void load_cell(const float4* p, float4& lo, float4& hi)
{
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(lo.x), "=f"(lo.y), "=f"(lo.z), "=f"(lo.w), "=f"(hi.x), "=f"(hi.y), "=f"(hi.z), "=f"(hi.w)
        : "l"(p));
}

// Both components of a bilinear field from the cell's records
// lo = (a0u, a0v, a1u, a1v), hi = (a2u, a2v, a3u, a3v): (a0 + a1 s) + t (a2 + a3 s).
__device__ __forceinline__ float2 eval2(const float4& lo, const float4& hi, float2 st)
{
    const float2 ss = f2(st.x, st.x), tt = f2(st.y, st.y);
    const float2 r = __ffma2_rn(f2(lo.z, lo.w), ss, f2(lo.x, lo.y));
    const float2 q = __ffma2_rn(f2(hi.z, hi.w), ss, f2(hi.x, hi.y));
    return __ffma2_rn(q, tt, r);
}

// One Euler--Maruyama sub-step from pos with increment z = sqrt(2 dt) N(0,1)^2:
// pos + b(pos) dt + z, b bilinear from the cell's drift records.
__device__ __forceinline__ float2 em(const float4& lo, const float4& hi, float2 st, float2 pos, float2 dt2, float2 z)
{
    return __fadd2_rn(__ffma2_rn(eval2(lo, hi, st), dt2, pos), z);
}

// Strictly inside the unit square: x - x^2 > 0 and y - y^2 > 0. Each is one
// rounding of the exact value, whose sign it keeps (barring underflow below
// 2^-126, which no position of a path reaches).
__device__ __forceinline__ bool inside2(float2 p)
{
    const float2 q = __ffma2_rn(f2(-p.x, -p.y), p, p);
    return fminf(q.x, q.y) > 0.0f;
}

// Face `face` at tangential coordinate s: the offset of its table (field 0;
// field 1 follows 2 ny + 2 nx entries later), the interval k and the fraction f.
__device__ __forceinline__ void face_interval(const InstDev& I, int face, float s, long long& off, int& k, float& f)
{
    const int n = (face < 2) ? I.ny : I.nx;
    off = 0;
    if (face >= 1) off += I.ny;
    if (face >= 2) off += I.ny;
    if (face >= 3) off += I.nx;
    const float g = s * (float)(n - 1);
    k = (int)floorf(g);
    k = max(0, min(k, n - 2));
    f = g - (float)k;
}

// Linear interpolation of face `face` of `field` at tangential coordinate s.
__device__ __forceinline__ float face_value(const InstDev& I, int field, int face, float s)
{
    long long off;
    int k;
    float f;
    face_interval(I, face, s, off, k, f);
    const float* v = I.faces32 + off + (long long)field * (2LL * I.ny + 2LL * I.nx);
    return fmaf(f, v[k + 1] - v[k], v[k]);
}

// The boundary crossing of the sub-step X_j = (x, y) -> X_{j+1} = (xn, yn):
// the segment is cut at the smallest crossing fraction over the violated
// faces, ties to the face listed first (left, right, bottom, top); t is the
// tangential coordinate of the crossing on that face.
__device__ __forceinline__ void exit_crossing(float x, float y, float xn, float yn, int& face, float& t)
{
    float best = 2.0f;
    int f = -1;
    if (xn <= 0.0f) { const float s = x / (x - xn); if (s < best) { best = s; f = 0; } }
    if (xn >= 1.0f) { const float s = (1.0f - x) / (xn - x); if (s < best) { best = s; f = 1; } }
    if (yn <= 0.0f) { const float s = y / (y - yn); if (s < best) { best = s; f = 2; } }
    if (yn >= 1.0f) { const float s = (1.0f - y) / (yn - y); if (s < best) { best = s; f = 3; } }
    if (f < 0) { f = 0; best = 0.0f; }  // only for a non-finite position
    float tt = (f < 2) ? fmaf(best, yn - y, y) : fmaf(best, xn - x, x);
    t = fminf(fmaxf(tt, 0.0f), 1.0f);
    face = f;
}

// Exit through the boundary between X_j and X_{j+1}: the boundary data at the crossing.
__device__ __forceinline__ void plain_exit(const InstDev& I, float x, float y, float xn, float yn, int& face,
                                        float& yxi, float& yeta, float& xe, float& ye)
{
    float t;
    exit_crossing(x, y, xn, yn, face, t);
    yxi = face_value(I, 0, face, t);
    yeta = face_value(I, 1, face, t);
    xe = (face == 0) ? 0.0f : (face == 1) ? 1.0f : t;
    ye = (face == 2) ? 0.0f : (face == 3) ? 1.0f : t;
}

// Brownian-bridge test between two inside points: the half plane behind face
// k is touched with probability exp(-d0 d1 / dt) (sigma^2 = 2); the faces
// combine as 1 - prod (1 - p_k). On exit: the face of largest p_k, at the
// projection of the sub-step midpoint.
__device__ __forceinline__ bool bridge_exit(const InstDev& I, float x, float y, float xn, float yn, float dt, float u,
                                         int& face, float& yxi, float& yeta, float& xe, float& ye)
{
    const float d0[4] = {x, 1.0f - x, y, 1.0f - y};
    const float d1[4] = {xn, 1.0f - xn, yn, 1.0f - yn};
    const float inv = 1.0f / dt;
    float stay = 1.0f, pmax = -1.0f;
    int f = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float p = __expf(-d0[k] * d1[k] * inv);
        stay *= (1.0f - p);
        if (p > pmax) { pmax = p; f = k; }
    }
    if (!(u < 1.0f - stay)) return false;
    float t = (f < 2) ? 0.5f * (y + yn) : 0.5f * (x + xn);
    t = fminf(fmaxf(t, 0.0f), 1.0f);
    face = f;
    yxi = face_value(I, 0, f, t);
    yeta = face_value(I, 1, f, t);
    xe = (f == 0) ? 0.0f : (f == 1) ? 1.0f : t;
    ye = (f == 2) ? 0.0f : (f == 3) ? 1.0f : t;
    return true;
}

// 32 bytes through the non-coherent path as eight words.
__device__ __forceinline__ void load_words(const uint4* p, uint4& lo, uint4& hi)
{
    asm("ld.global.nc.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(lo.x), "=r"(lo.y), "=r"(lo.z), "=r"(lo.w), "=r"(hi.x), "=r"(hi.y), "=r"(hi.z), "=r"(hi.w)
        : "l"(p));
}

__device__ __forceinline__ float2 half2_to_float2(uint32_t u)
{
    __half2 h;
    memcpy(&h, &u, sizeof h);
    return __half22float2(h);
}

// Bilinear interpolation of four corner values (00, 10, 01, 11) at (s, t):
// ((1 - s) f00 + s f10) (1 - t) + ((1 - s) f01 + s f11) t, both components.
__device__ __forceinline__ float2 corners2(const uint4& r, float2 ss, float2 oms, float2 tt, float2 omt)
{
    const float2 r0 = __ffma2_rn(ss, half2_to_float2(r.y), __fmul2_rn(oms, half2_to_float2(r.x)));
    const float2 r1 = __ffma2_rn(ss, half2_to_float2(r.w), __fmul2_rn(oms, half2_to_float2(r.z)));
    return __ffma2_rn(tt, r1, __fmul2_rn(omt, r0));
}

// Control variate: the model gradients of xi and eta at the cell's point
// (slice q), gxi = (d/dx, d/dy) of the xi model, geta of the eta model.
__device__ __forceinline__ void cv_eval(const InstDev& I, const Cell& c, int q, float2& gxi, float2& geta)
{
    const uint4* r = I.cvcoef + 2 * ((size_t)q * (size_t)(I.nx - 1) * (size_t)(I.ny - 1) + c.idx);
    uint4 gx, ge;
    load_words(r, gx, ge);
    const float2 ss = f2(c.st.x, c.st.x), tt = f2(c.st.y, c.st.y);
    const float2 oms = f2(1.f - c.st.x, 1.f - c.st.x), omt = f2(1.f - c.st.y, 1.f - c.st.y);
    gxi = corners2(gx, ss, oms, tt, omt);
    geta = corners2(ge, ss, oms, tt, omt);
}

// Control variate of one value per cell: (d/dx, d/dy) of xi, then of eta, on
// the cell holding the point, in one 128-bit read-only load.
__device__ __forceinline__ void cv_cell(const InstDev& I, const Cell& c, float2& gxi, float2& geta)
{
    const float4 g = __ldg(I.cvcell + c.idx);
    gxi = f2(g.x, g.y);
    geta = f2(g.z, g.w);
}

// The gradients times the sub-step's increment z = sqrt(2 dt) N(0,1)^2, added to
// the running sums (acc_xi, acc_eta hold the x and y parts separately).
__device__ __forceinline__ void cv_acc(float2 gxi, float2 geta, float2 z, float2& acc_xi, float2& acc_eta)
{
    acc_xi = __ffma2_rn(gxi, z, acc_xi);
    acc_eta = __ffma2_rn(geta, z, acc_eta);
}

struct Acc {
    float s, cs, q, cq;
    __device__ __forceinline__ void add(float v)
    {
        float y1 = v - cs;
        float t1 = s + y1;
        cs = (t1 - s) - y1;
        s = t1;
        const float v2 = v * v;
        float y2 = v2 - cq;
        float t2 = q + y2;
        cq = (t2 - q) - y2;
        q = t2;
    }
    __device__ __forceinline__ double sum() const { return (double)s - (double)cs; }
    __device__ __forceinline__ double sumsq() const { return (double)q - (double)cq; }
};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
    return v;
}

__device__ __forceinline__ long long warp_sum_ll(long long v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
    return v;
}

// Deferred scoring: a path's record in the survivor buffer, one float2 (two
// with CV, the second holding the control-variate sums): a survivor leaves its
// end point (x, y), x > 0; a path that left by the plain test the crossing of
// its last sub-step with the boundary, (-1 - face, t) with t the tangential
// coordinate on that face (the face data are interpolated there later); a path
// scored in the kernel (bridge exits) REC_SKIP. No point inside the square has
// a negative x, so the sign tells the kinds apart.
constexpr float REC_SKIP = -8.0f;

template <bool CV>
__device__ __forceinline__ void put_record(void* surv, long long i, float2 r, float cxi, float ceta)
{
    float2* q = static_cast<float2*>(surv) + (CV ? 2 * i : i);
    q[0] = r;
    if (CV) q[1] = f2(cxi, ceta);
}

// The record of a plain exit through the sub-step (x, y) -> (xn, yn).
__device__ __forceinline__ float2 exit_record(float x, float y, float xn, float yn)
{
    int face;
    float t;
    exit_crossing(x, y, xn, yn, face, t);
    return f2(-1.0f - (float)face, t);
}

// Lanes refilled together below this count spend a loop pass drawing their
// first normals instead of a divergent Philox block (front257: 2.7% faster).
constexpr int WARM_MIN = 8;

// MODE 0: the paper's test, sub-step pairs; MODE 1: with the bridge test;
// MODE 2: as MODE 0 when K is even (every pair has both sub-steps).
// CVM: 0 no control variate; otherwise subtract sum_j G(s_j, X_j) . sqrt(2) dW_j
// from both scores, G from node values interpolated bilinearly in time slices
// (1, cv_eval) or one value per cell (2, cv_cell).
// Kernel variants by where the tables come from: VAR_MULTI, each task's
// instance from the instance table (batches); VAR_ONE, a single instance whose
// tables are kernel parameters (no registers held for them); VAR_ZM, VAR_ONE
// with the zero map of the drift records. Launch shapes: a single instance's
// kernel fits 40 registers (48 warps per SM; 64 with the control variate of
// node values, 48 with that of cell values), the batch kernel 64 (32 warps;
// 80 with a control variate).
constexpr int VAR_MULTI = 0, VAR_ONE = 1, VAR_ZM = 2;
constexpr int kCvCellBlocks = 5;   // cell-valued control variate, single instance: 48 registers, 40 warps per SM
constexpr int kOneMaxBlock = 256;
constexpr int paths_max_block(int cvm, int var) { return cvm ? kCvMaxBlock : var != VAR_MULTI ? kOneMaxBlock : 512; }
constexpr int paths_min_blocks(int cvm, int var)
{
    return cvm == 2 ? (var != VAR_MULTI ? kCvCellBlocks : 3) : cvm ? (var != VAR_MULTI ? 4 : 3)
                                                                    : (var != VAR_MULTI ? 6 : 2);
}

template <int MODE, bool RECORD, int CVM, int VAR>
__global__ void __launch_bounds__(paths_max_block(CVM, VAR), paths_min_blocks(CVM, VAR))
    k_paths(const PathArgs a)
{
    constexpr bool ZM = VAR == VAR_ZM;
    constexpr bool CV = CVM != 0;
    constexpr bool CVT = CVM == 1;   // node values in time slices
    extern __shared__ uint32_t zsm[];   // the zero map of the drift records (ZM)
    if (ZM) {
        for (int k = threadIdx.x; k < a.zwords; k += blockDim.x) zsm[zmap_slot((uint32_t)k)] = a.zmap[k];
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const uint32_t step = a.step_ptr ? *a.step_ptr : a.step_index;
    const int K = a.K;
    const float dt = a.dt;
    constexpr bool PAIRS = MODE != 1;

    // Each warp takes the next task as soon as its last one is done (no wait
    // for the block's other warps); tasks go node by node, so warps started
    // together share the node's neighbourhood in L1.
    for (;;) {
        int tq = 0;
        if (lane == 0) tq = atomicAdd(a.queue, 1);
        const int t = __shfl_sync(FULL, tq, 0);
        if (t >= a.ntasks) return;

        const Task task = a.tasks[t];
        if (a.node_mask && !a.node_mask[task.node]) continue;   // not a key point this step
        const NodeDev& nd = a.nodes[task.node];
        // a single instance's tables come from the kernel parameters (no registers held for them)
        InstDev Iloc;
        if (VAR == VAR_MULTI) Iloc = a.inst[nd.inst];
        const InstDev& I = VAR != VAR_MULTI ? a.one : Iloc;
        const float x0 = nd.xf, y0 = nd.yf;
        const uint32_t nctr = nd.ctr;
        const int end = task.path0 + task.npaths;
        int next = task.path0 + 32;
        int path = task.path0 + lane;
        bool alive = path < end;
        float2 pos = f2(x0, y0);
        int m = 0;  // draw index: the sub-step pair (plain mode) or the sub-step (bridge mode)
        // normals of draw m, already scaled by sqrt(2 dt): zA for the first
        // sub-step, zB for the second (plain mode); ub the bridge uniform
        float2 zA = f2(0.f, 0.f), zB = f2(0.f, 0.f);
        float ub = 1.f;
        float2 cvx = f2(0.f, 0.f), cve = f2(0.f, 0.f);  // control-variate sums of the path
        int cvq = 0, cvn = CVT ? a.cv_bound[1] : 0;      // slice of the current sub-step, start of the next
        const float2 dt2 = f2(dt, dt);
        auto first_draw = [&]() {
            uint4 r = make_uint4((uint32_t)path, nctr, 0u, step);
            philox_rounds_rk<0, 10>(r, a.keys);
            if (PAIRS) {
                box_muller2(r, a.bm_scale, zA, zB);
            } else {
                box_muller(r.x, r.y, a.bm_scale, zA.x, zA.y);
                ub = uniform_pos(r.z);
            }
        };
        if (alive) first_draw();
        Acc ax{0.f, 0.f, 0.f, 0.f}, ae{0.f, 0.f, 0.f, 0.f};
        int exits = 0, steps = 0;

        while (__any_sync(FULL, alive)) {
            if (alive) {
                bool done = false;
                int code = -1, taken = 0;
                float yxi = 0.f, yeta = 0.f, xe = 0.f, ye = 0.f;
                const bool warm = m < 0;   // draw -1: the pass draws the path's first normals
                float2 seg = f2(REC_SKIP, 0.f);   // a plain exit's crossing, scored later
                // sub-step A: gather, then the next draw's first rounds while the gather is in flight
                const Cell cA = locate(I, pos);
                float4 gA0, gA1;
                load_cell(drift_rec<ZM>(I, cA, zsm, a), gA0, gA1);
                if (CV) {
                    float2 gxA, geA;   // the model at X_j
                    if (CVT) {
                        const int j = PAIRS ? 2 * m : m;
                        if (j >= cvn) cvn = a.cv_bound[++cvq + 1];
                        cv_eval(I, cA, cvq, gxA, geA);
                    } else {
                        cv_cell(I, cA, gxA, geA);
                    }
                    cv_acc(gxA, geA, zA, cvx, cve);
                }
                uint4 r = make_uint4((uint32_t)path, nctr, (uint32_t)(m + 1), step);
                philox_rounds_rk<0, 5>(r, a.keys);
                const float2 pa = em(gA0, gA1, cA.st, pos, dt2, zA);
                const bool outA = !inside2(pa);
                if (PAIRS) {
                    // sub-step B from the point A reached (or from X_j when A left: harmless, in bounds)
                    const float2 pq = outA ? pos : pa;
                    const Cell cB = locate(I, pq);
                    float4 gB0, gB1;
                    load_cell(drift_rec<ZM>(I, cB, zsm, a), gB0, gB1);
                    philox_rounds_rk<5, 10>(r, a.keys);
                    float2 nA, nB;
                    box_muller2(r, a.bm_scale, nA, nB);
                    const float2 pb = em(gB0, gB1, cB.st, pq, dt2, zB);
                    const bool haveB = (MODE == 2) || 2 * m + 1 < K;
                    const bool outB = haveB && !outA && !inside2(pb);
                    if (CV) {
                        // the second sub-step counts only when the path takes it
                        const float2 zt = (haveB && !outA) ? zB : f2(0.f, 0.f);
                        float2 gxB, geB;
                        if (CVT) {
                            if (haveB && 2 * m + 1 >= cvn) cvn = a.cv_bound[++cvq + 1];
                            cv_eval(I, cB, cvq, gxB, geB);
                        } else {
                            cv_cell(I, cB, gxB, geB);
                        }
                        cv_acc(gxB, geB, zt, cvx, cve);
                    }
                    if (warm) {
                        // a path taken up mid-task: this pass only drew its first normals
                    } else if (outA) {
                        if (a.surv) seg = exit_record(pos.x, pos.y, pa.x, pa.y), code = 0;
                        else plain_exit(I, pos.x, pos.y, pa.x, pa.y, code, yxi, yeta, xe, ye);
                        done = true;
                        taken = 2 * m + 1;
                    } else if (outB) {
                        if (a.surv) seg = exit_record(pa.x, pa.y, pb.x, pb.y), code = 0;
                        else plain_exit(I, pa.x, pa.y, pb.x, pb.y, code, yxi, yeta, xe, ye);
                        done = true;
                        taken = 2 * m + 2;
                    } else {
                        pos = haveB ? pb : pa;
                    }
                    zA = nA;
                    zB = nB;
                    ++m;
                    if (!warm && !done && 2 * m >= K) {
                        done = true;
                        taken = K;
                    }
                } else {
                    philox_rounds_rk<5, 10>(r, a.keys);
                    float2 nA;
                    box_muller(r.x, r.y, a.bm_scale, nA.x, nA.y);
                    const float nub = uniform_pos(r.z);
                    if (warm) {
                        // a path taken up mid-task: this pass only drew its first normals
                    } else if (outA) {
                        if (a.surv) seg = exit_record(pos.x, pos.y, pa.x, pa.y), code = 0;
                        else plain_exit(I, pos.x, pos.y, pa.x, pa.y, code, yxi, yeta, xe, ye);
                        done = true;
                    } else {
                        const float dm0 = fminf(fminf(pos.x, 1.0f - pos.x), fminf(pos.y, 1.0f - pos.y));
                        const float dm1 = fminf(fminf(pa.x, 1.0f - pa.x), fminf(pa.y, 1.0f - pa.y));
                        if (dm0 * dm1 < a.bridge_cut &&
                            bridge_exit(I, pos.x, pos.y, pa.x, pa.y, dt, ub, code, yxi, yeta, xe, ye)) {
                            code += 4;
                            done = true;
                        } else {
                            pos = pa;
                        }
                    }
                    zA = nA;
                    ub = nub;
                    ++m;
                    taken = m;
                    if (!warm && !done && m >= K) done = true;
                }
                if (done) {
                    bool later = false;   // scored by k_score_surv once the fields are final
                    if (code < 0) {
                        if (a.surv) {
                            later = true;
                            put_record<CV>(a.surv, nd.rec0 + path, pos, cvx.x + cvx.y, cve.x + cve.y);
                        } else {
                            // survived the mesh step: xi, eta of its start at the end point
                            const Cell c = locate(I, pos);
                            float4 f0, f1;
                            load_cell(rec2(I.fcoef, c.idx), f0, f1);
                            const float2 v = eval2(f0, f1, c.st);
                            yxi = v.x;
                            yeta = v.y;
                            xe = pos.x;
                            ye = pos.y;
                        }
                    } else {
                        ++exits;
                        if (a.surv) {
                            // a plain exit leaves its sub-step, a bridge exit (scored here) the skip mark
                            later = seg.x != REC_SKIP;
                            put_record<CV>(a.surv, nd.rec0 + path, seg, cvx.x + cvx.y, cve.x + cve.y);
                        }
                    }
                    if (!later) {
                        if (CV) {
                            yxi -= cvx.x + cvx.y;
                            yeta -= cve.x + cve.y;
                        }
                        ax.add(yxi - x0);
                        ae.add(yeta - y0);
                    }
                    steps += taken;
                    if (RECORD) {
                        const long long ri = nd.rec0 + path;
                        if (a.rec.steps) a.rec.steps[ri] = taken;
                        if (a.rec.code) a.rec.code[ri] = code;
                        if (a.rec.score_xi) a.rec.score_xi[ri] = yxi;
                        if (a.rec.score_eta) a.rec.score_eta[ri] = yeta;
                        if (a.rec.x_end) a.rec.x_end[ri] = xe;
                        if (a.rec.y_end) a.rec.y_end[ri] = ye;
                    }
                    alive = false;
                }
            }
            // lanes whose path ended take the task's next paths, in lane order
            const unsigned need = __ballot_sync(FULL, !alive);
            if (need != 0u && next < end) {
                const int cand = next + __popc(need & below);
                if (!alive && cand < end) {
                    path = cand;
                    alive = true;
                    pos = f2(x0, y0);
                    m = 0;
                    if (CV) cvx = cve = f2(0.f, 0.f);
                    if (CVT) {
                        cvq = 0;
                        cvn = a.cv_bound[1];
                    }
                    if (__popc(need) >= WARM_MIN) {
                        first_draw();
                    } else {
                        // few lanes refill: rather than run the first draw's Philox block
                        // with the others idle, the lane spends the next pass drawing it
                        m = -1;
                        zA = zB = f2(0.f, 0.f);
                        ub = 1.f;
                    }
                }
                next += __popc(need);
            }
        }

        const double sx = warp_sum(ax.sum()), qx = warp_sum(ax.sumsq());
        const double se = warp_sum(ae.sum()), qe = warp_sum(ae.sumsq());
        const long long ex = warp_sum_ll(exits), st = warp_sum_ll(steps);
        if (lane == 0) {
            Partial p;
            p.s_xi = sx;
            p.q_xi = qx;
            p.s_eta = se;
            p.q_eta = qe;
            p.exits = ex;
            p.steps = st;
            a.partials[t] = p;
        }
    }
}

// Exponential time-stepping (exit_mode 2), the alternative integrator Sec. 4
// names: sub-step j of a path has length tau_j = -dt ln u with u = (2^23 - m)
// 2^-23 from word 3 of the block (path, node, j, step), cut at the end of the
// mesh step (and after 4K + 16 sub-steps); normals from words 0, 1 scaled by
// sqrt(2 tau_j); the plain test, then the Brownian-bridge test over tau_j with
// the uniform of word 2. No software pipelining: one block per sub-step.
template <bool RECORD>
__global__ void __launch_bounds__(512, 2) k_paths_exp(const PathArgs a)
{
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const uint32_t step = a.step_ptr ? *a.step_ptr : a.step_index;
    const int K = a.K;
    const int cap = 4 * K + 16;
    const float T = a.horizon;
    const float ln2dt = a.dt * 0.69314718055994530942f;
    for (;;) {
        int tq = 0;
        if (lane == 0) tq = atomicAdd(a.queue, 1);
        const int t = __shfl_sync(FULL, tq, 0);
        if (t >= a.ntasks) return;
        const Task task = a.tasks[t];
        if (a.node_mask && !a.node_mask[task.node]) continue;
        const NodeDev& nd = a.nodes[task.node];
        const InstDev I = a.inst[nd.inst];
        const float x0 = nd.xf, y0 = nd.yf;
        const uint32_t nctr = nd.ctr;
        const int end = task.path0 + task.npaths;
        int next = task.path0 + 32;
        int path = task.path0 + lane;
        bool alive = path < end;
        float2 pos = f2(x0, y0);
        int j = 0;
        float tm = 0.f;
        Acc ax{0.f, 0.f, 0.f, 0.f}, ae{0.f, 0.f, 0.f, 0.f};
        int exits = 0, steps = 0;
        while (__any_sync(FULL, alive)) {
            if (alive) {
                uint4 r = make_uint4((uint32_t)path, nctr, (uint32_t)j, step);
                philox_rounds_rk<0, 10>(r, a.keys);
                const float u3 = 2.0f - __uint_as_float(0x3F800000u | (r.w & 0x7FFFFFu));
                float tau = -ln2dt * __log2f(u3);
                bool last = false;
                if (tm + tau >= T || j + 1 >= cap) {
                    tau = T - tm;
                    last = true;
                }
                float2 z;
                box_muller(r.x, r.y, -2.77258872223978123767f * tau, z.x, z.y);   // -4 ln 2 tau: sqrt(2 tau) N(0,1)
                const float ub = uniform_pos(r.z);
                const Cell c = locate(I, pos);
                float4 g0, g1;
                load_cell(rec2(I.bcoef, c.idx), g0, g1);
                const float2 pn = em(g0, g1, c.st, pos, f2(tau, tau), z);
                bool done = false;
                int code = -1;
                float yxi = 0.f, yeta = 0.f, xe = 0.f, ye = 0.f;
                float2 seg = f2(REC_SKIP, 0.f);
                if (!inside2(pn)) {
                    if (a.surv) seg = exit_record(pos.x, pos.y, pn.x, pn.y), code = 0;
                    else plain_exit(I, pos.x, pos.y, pn.x, pn.y, code, yxi, yeta, xe, ye);
                    done = true;
                } else {
                    const float dm0 = fminf(fminf(pos.x, 1.0f - pos.x), fminf(pos.y, 1.0f - pos.y));
                    const float dm1 = fminf(fminf(pn.x, 1.0f - pn.x), fminf(pn.y, 1.0f - pn.y));
                    if (dm0 * dm1 < 18.0f * tau && bridge_exit(I, pos.x, pos.y, pn.x, pn.y, tau, ub, code, yxi, yeta, xe, ye)) {
                        code += 4;
                        done = true;
                    } else {
                        pos = pn;
                        tm += tau;
                        if (last) done = true;
                    }
                }
                ++j;
                if (done) {
                    bool later = false;
                    if (code < 0) {
                        if (a.surv) {
                            later = true;
                            put_record<false>(a.surv, nd.rec0 + path, pos, 0.f, 0.f);
                        } else {
                            const Cell cf = locate(I, pos);
                            float4 f0, f1;
                            load_cell(rec2(I.fcoef, cf.idx), f0, f1);
                            const float2 v = eval2(f0, f1, cf.st);
                            yxi = v.x;
                            yeta = v.y;
                            xe = pos.x;
                            ye = pos.y;
                        }
                    } else {
                        ++exits;
                        if (a.surv) {
                            later = seg.x != REC_SKIP;
                            put_record<false>(a.surv, nd.rec0 + path, seg, 0.f, 0.f);
                        }
                    }
                    if (!later) {
                        ax.add(yxi - x0);
                        ae.add(yeta - y0);
                    }
                    steps += j;
                    if (RECORD) {
                        const long long ri = nd.rec0 + path;
                        if (a.rec.steps) a.rec.steps[ri] = j;
                        if (a.rec.code) a.rec.code[ri] = code;
                        if (a.rec.score_xi) a.rec.score_xi[ri] = yxi;
                        if (a.rec.score_eta) a.rec.score_eta[ri] = yeta;
                        if (a.rec.x_end) a.rec.x_end[ri] = xe;
                        if (a.rec.y_end) a.rec.y_end[ri] = ye;
                    }
                    alive = false;
                }
            }
            const unsigned need = __ballot_sync(FULL, !alive);
            if (need != 0u && next < end) {
                const int cand = next + __popc(need & below);
                if (!alive && cand < end) {
                    path = cand;
                    alive = true;
                    pos = f2(x0, y0);
                    j = 0;
                    tm = 0.f;
                }
                next += __popc(need);
            }
        }
        const double sx = warp_sum(ax.sum()), qx = warp_sum(ax.sumsq());
        const double se = warp_sum(ae.sum()), qe = warp_sum(ae.sumsq());
        const long long ex = warp_sum_ll(exits), st = warp_sum_ll(steps);
        if (lane == 0) {
            Partial p;
            p.s_xi = sx;
            p.q_xi = qx;
            p.s_eta = se;
            p.q_eta = qe;
            p.exits = ex;
            p.steps = st;
            a.partials[t] = p;
        }
    }
}

// Scores of the paths that survived a mesh step, once the fields of the step's
// start are final (the estimate of the next mesh step runs beside the
// subdomain solve that produces them). One block per node: the node's paths
// end in one neighbourhood, so its gathers share L1; thread k takes paths k,
// k + T, ... SCORE_BATCH at a time (records, then gathers, in flight
// together) and sums xi and eta at the end points minus the paths'
// control-variate sums; the block's sums, in warp order, join the partial
// sums of the node's first task in the node's reduction, which the block's
// first warp then runs (the mean and standard error of every node, boundary
// and masked nodes included). The next batch's records are read while the
// current batch's gathers are in flight. T = 256 threads at 64 registers puts
// four blocks on an SM (many nodes: one wave for up to four per SM); with no
// more nodes than SMs, T = 1024 gives each node's paths four times the threads.
constexpr int SCORE_BATCH = 2;

__device__ void finalize_node(const FinalArgs& a, int node, int lane, const double* add0);

template <bool CV, int SCORE_THREADS>
__global__ void __launch_bounds__(SCORE_THREADS, 1024 / SCORE_THREADS) k_score_surv(const ScoreArgs a)
{
    __shared__ double red[SCORE_THREADS / 32][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int node = blockIdx.x;
    const NodeDev& nd = a.nodes[node];
    if (nd.ntasks == 0 || (a.fin.node_mask && !a.fin.node_mask[node])) {
        // a boundary node or one left to the interface fill: no paths to score
        if (warp == 0) finalize_node(a.fin, node, lane, nullptr);
        return;   // uniform over the block
    }
    const InstDev I = a.inst[nd.inst];
    const float x0 = nd.xf, y0 = nd.yf;
    const int end = nd.n_paths;
    Acc ax{0.f, 0.f, 0.f, 0.f}, ae{0.f, 0.f, 0.f, 0.f};
    // the records of the batch that starts at path p0 (past the end: the skip mark)
    auto load_batch = [&](int p0, float2 (&r)[SCORE_BATCH], float2 (&cvs)[SCORE_BATCH]) {
#pragma unroll
        for (int u = 0; u < SCORE_BATCH; ++u) {
            const int p = p0 + u * SCORE_THREADS;
            r[u] = f2(REC_SKIP, 0.f);
            cvs[u] = f2(0.f, 0.f);
            if (p < end) {
                const long long si = nd.rec0 + p;
                const float2* q = static_cast<const float2*>(a.surv) + (CV ? 2 * si : si);
                r[u] = q[0];
                if (CV) cvs[u] = q[1];
            }
        }
    };
    float2 r[SCORE_BATCH];
    float2 cvs[SCORE_BATCH];
    load_batch(threadIdx.x, r, cvs);
    for (int p0 = threadIdx.x; p0 < end; p0 += SCORE_BATCH * SCORE_THREADS) {
        // one round of loads for the batch: a survivor gathers the field record at its
        // end point, a plain exit the face data on both sides of its crossing
        // (f0 = xi[k], xi[k + 1], eta[k], eta[k + 1]; st.x the fraction)
        float4 f0[SCORE_BATCH], f1[SCORE_BATCH];
        float2 st[SCORE_BATCH];
#pragma unroll
        for (int u = 0; u < SCORE_BATCH; ++u) {
            if (r[u].x >= 0.f) {
                const Cell c = locate(I, r[u]);
                load_cell(rec2(I.fcoef, c.idx), f0[u], f1[u]);
                st[u] = c.st;
            } else if (r[u].x != REC_SKIP) {
                int k;
                float f;
                long long off;
                const int face = (int)(-1.0f - r[u].x);
                face_interval(I, face, r[u].y, off, k, f);
                const float* v0 = I.faces32 + off + k;
                const float* v1 = v0 + (2LL * I.ny + 2LL * I.nx);
                f0[u] = make_float4(v0[0], v0[1], v1[0], v1[1]);
                st[u] = f2(f, 0.f);
            }
        }
        // the next batch's records while this batch's gathers are in flight
        float2 rn[SCORE_BATCH];
        float2 cn[SCORE_BATCH];
        load_batch(p0 + SCORE_BATCH * SCORE_THREADS, rn, cn);
#pragma unroll
        for (int u = 0; u < SCORE_BATCH; ++u) {
            if (r[u].x == REC_SKIP) continue;   // scored in the path kernel, or past the end
            float yxi, yeta;
            if (r[u].x >= 0.f) {
                const float2 v = eval2(f0[u], f1[u], st[u]);
                yxi = v.x;
                yeta = v.y;
            } else {
                // left the domain in the sub-step (x0, y0) -> (x1, y1): the boundary data there,
                // as face_value interpolates it
                yxi = fmaf(st[u].x, f0[u].y - f0[u].x, f0[u].x);
                yeta = fmaf(st[u].x, f0[u].w - f0[u].z, f0[u].z);
            }
            ax.add(yxi - cvs[u].x - x0);
            ae.add(yeta - cvs[u].y - y0);
        }
#pragma unroll
        for (int u = 0; u < SCORE_BATCH; ++u) {
            r[u] = rn[u];
            cvs[u] = cn[u];
        }
    }
    const double v[4] = {warp_sum(ax.sum()), warp_sum(ax.sumsq()), warp_sum(ae.sum()), warp_sum(ae.sumsq())};
    if (lane == 0)
        for (int q = 0; q < 4; ++q) red[warp][q] = v[q];
    __syncthreads();
    if (warp == 0) {
        double tot[4] = {0.0, 0.0, 0.0, 0.0};
        for (int g = 0; g < SCORE_THREADS / 32; ++g)
            for (int q = 0; q < 4; ++q) tot[q] += red[g][q];
        finalize_node(a.fin, node, lane, tot);   // the node's mean and standard error
    }
}

__device__ __forceinline__ double face_value64(const InstDev& I, int field, int face, double s)
{
    const int n = (face < 2) ? I.ny : I.nx;
    long long off = (long long)field * (2LL * I.ny + 2LL * I.nx);
    if (face >= 1) off += I.ny;
    if (face >= 2) off += I.ny;
    if (face >= 3) off += I.nx;
    const double* v = I.faces64 + off;
    const double g = s * (double)(n - 1);
    int k = (int)floor(g);
    k = max(0, min(k, n - 2));
    const double f = g - (double)k;
    return (1.0 - f) * v[k] + f * v[k + 1];
}

// One warp per node: compensated sums of the node's task partials (each lane a
// fixed stride of tasks; add0, if non-null, added to the first task's), a
// fixed butterfly across the warp, then the mean and the standard error
// s / sqrt(N), s^2 = (Q - S^2 / N) / (N - 1) of the shifted scores.
__device__ void finalize_node(const FinalArgs& a, int node, int lane, const double* add0)
{
    const NodeDev nd = a.nodes[node];
    const OutDev o = a.out_table ? a.out_table[nd.inst] : a.out0;
    const int k = nd.local;
    if (a.node_mask && !a.node_mask[node]) {
        // not estimated this step: no paths; the interface fill writes its value
        if (lane == 0) {
            if (o.mean_xi) o.mean_xi[k] = 0.0;
            if (o.mean_eta) o.mean_eta[k] = 0.0;
            if (o.se_xi) o.se_xi[k] = 0.0;
            if (o.se_eta) o.se_eta[k] = 0.0;
            if (o.n_exit) o.n_exit[k] = 0;
            if (o.path_steps) o.path_steps[k] = 0;
        }
        return;
    }
    if (nd.ntasks == 0) {
        // a node on the boundary: its Dirichlet value, every path exits at time 0
        const InstDev I = a.inst[nd.inst];
        int face;
        double tg;
        if (nd.x <= 0.0) { face = 0; tg = nd.y; }
        else if (nd.x >= 1.0) { face = 1; tg = nd.y; }
        else if (nd.y <= 0.0) { face = 2; tg = nd.x; }
        else { face = 3; tg = nd.x; }
        const double vx = face_value64(I, 0, face, tg), ve = face_value64(I, 1, face, tg);
        if (lane == 0) {
            if (o.mean_xi) o.mean_xi[k] = vx;
            if (o.mean_eta) o.mean_eta[k] = ve;
            if (o.se_xi) o.se_xi[k] = 0.0;
            if (o.se_eta) o.se_eta[k] = 0.0;
            if (o.n_exit) o.n_exit[k] = nd.n_paths;
            if (o.path_steps) o.path_steps[k] = 0;
        }
        for (int p = lane; p < nd.n_paths; p += 32) {
            const long long ri = nd.rec0 + p;
            if (a.rec.steps) a.rec.steps[ri] = 0;
            if (a.rec.code) a.rec.code[ri] = face;
            if (a.rec.score_xi) a.rec.score_xi[ri] = (float)vx;
            if (a.rec.score_eta) a.rec.score_eta[ri] = (float)ve;
            if (a.rec.x_end) a.rec.x_end[ri] = nd.xf;
            if (a.rec.y_end) a.rec.y_end[ri] = nd.yf;
        }
        return;
    }
    double v[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0};
    long long ex = 0, st = 0;
    for (int t = nd.task0 + lane; t < nd.task0 + nd.ntasks; t += 32) {
        const Partial p = a.partials[t];
        double in[4] = {p.s_xi, p.q_xi, p.s_eta, p.q_eta};
        if (add0 && t == nd.task0)
#pragma unroll
            for (int q = 0; q < 4; ++q) in[q] += add0[q];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const double y = in[q] - c[q];
            const double tt = v[q] + y;
            c[q] = (tt - v[q]) - y;
            v[q] = tt;
        }
        ex += p.exits;
        st += p.steps;
    }
    double tot[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) tot[q] = warp_sum(v[q] - c[q]);
    ex = warp_sum_ll(ex);
    st = warp_sum_ll(st);
    if (lane == 0) {
        const double N = (double)nd.n_paths;
        const double mx = tot[0] / N, me = tot[2] / N;
        double vx = 0.0, ve = 0.0;
        if (nd.n_paths > 1) {
            vx = fmax(0.0, (tot[1] - tot[0] * mx) / (N - 1.0));
            ve = fmax(0.0, (tot[3] - tot[2] * me) / (N - 1.0));
        }
        if (o.mean_xi) o.mean_xi[k] = (double)nd.xf + mx;
        if (o.mean_eta) o.mean_eta[k] = (double)nd.yf + me;
        if (o.se_xi) o.se_xi[k] = sqrt(vx / N);
        if (o.se_eta) o.se_eta[k] = sqrt(ve / N);
        if (o.n_exit) o.n_exit[k] = ex;
        if (o.path_steps) o.path_steps[k] = st;
    }
}

__global__ void k_finalize(const FinalArgs a)
{
    const int node = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (node >= a.nnodes) return;
    finalize_node(a, node, lane, nullptr);
}

__global__ void k_rng_draw(uint64_t seed, const uint32_t* __restrict__ ctrs, long long count,
                           uint32_t* __restrict__ words, float* __restrict__ normals)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= count) return;
    const uint4 c = make_uint4(ctrs[4 * i], ctrs[4 * i + 1], ctrs[4 * i + 2], ctrs[4 * i + 3]);
    const uint4 r = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    words[4 * i + 0] = r.x;
    words[4 * i + 1] = r.y;
    words[4 * i + 2] = r.z;
    words[4 * i + 3] = r.w;
    if (normals) {
        const float scale = -1.38629436111989061883f;  // -2 ln 2: unit variance
        float z0, z1, z2, z3;
        box_muller(r.x, r.y, scale, z0, z1);
        box_muller(r.z, r.w, scale, z2, z3);
        normals[4 * i + 0] = z0;
        normals[4 * i + 1] = z1;
        normals[4 * i + 2] = z2;
        normals[4 * i + 3] = z3;
    }
}

template <int MODE, bool RECORD, int CVM, int VAR>
const void* kernel_ptr()
{
    return (const void*)k_paths<MODE, RECORD, CVM, VAR>;
}

template <int CVM, int VAR>
const void* pick_cv(int mode, bool record)
{
    if (mode == 3) return record ? (const void*)k_paths_exp<true> : (const void*)k_paths_exp<false>;
    if (mode == 0) return record ? kernel_ptr<0, true, CVM, VAR>() : kernel_ptr<0, false, CVM, VAR>();
    if (mode == 2) return record ? kernel_ptr<2, true, CVM, VAR>() : kernel_ptr<2, false, CVM, VAR>();
    return record ? kernel_ptr<1, true, CVM, VAR>() : kernel_ptr<1, false, CVM, VAR>();
}

template <int VAR>
const void* pick_var(int mode, bool record, int cvm)
{
    if (cvm == 2) return pick_cv<2, VAR>(mode, record);
    return cvm ? pick_cv<1, VAR>(mode, record) : pick_cv<0, VAR>(mode, record);
}

// cvm: 0 no control variate, 1 node values in time slices, 2 one value per cell
const void* pick(int mode, bool record, int cvm, int var)
{
    if (var == VAR_ZM) return pick_var<VAR_ZM>(mode, record, cvm);
    if (var == VAR_ONE) return pick_var<VAR_ONE>(mode, record, cvm);
    return pick_var<VAR_MULTI>(mode, record, cvm);
}

// The variant of a launch: the zero map where the arguments carry one, else the single instance's
// tables as parameters where the launch has one instance.
int path_var(const PathArgs& a)
{
    if (a.zwords > 0 && a.zmap != nullptr) return VAR_ZM;
    return a.single ? VAR_ONE : VAR_MULTI;
}

}  // namespace

static void prefer_l1();

int path_kernel_max_block(int exit_mode, int cvm, bool single)
{
    return exit_mode == 2 ? 512 : paths_max_block(cvm, single ? VAR_ONE : VAR_MULTI);
}

int path_kernel_blocks_per_sm(int exit_mode, bool record, int block, int cvm, int zwords, bool single)
{
    prefer_l1();
    int n = 0;
    // the even-K kernel has the same footprint class; size the grid for the larger of the two
    const int mode = exit_mode == 2 ? 3 : exit_mode == 1 ? 1 : 0;
    const int var = zwords > 0 ? VAR_ZM : single ? VAR_ONE : VAR_MULTI;
    const size_t smem = var == VAR_ZM && mode != 3 ? zmap_smem_bytes(zwords) : 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pick(mode, record, cvm, var), block, smem) !=
        cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

// The shared-memory carveout (percent of the SM's largest) that holds `blocks` blocks of `smem`
// dynamic bytes each, so that the zero map costs the launch no occupancy and L1 keeps the rest.
static unsigned carveout_pct(int blocks, size_t smem)
{
    int dev = 0, most = 0, resv = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&most, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (most <= 0) return 100;
    const double need = (double)blocks * (double)(smem + (size_t)resv);
    const int pct = (int)std::ceil(100.0 * need / (double)most);
    return (unsigned)std::min(100, std::max(0, pct));
}

static int kernel_mode(int exit_mode, int K)
{
    if (exit_mode == 2) return 3;   // exponential time-stepping
    return exit_mode == 1 ? 1 : ((K & 1) == 0 ? 2 : 0);
}

// Without the zero map the path kernel keeps no data in shared memory: give L1 the whole carveout.
// The kernels with the map prefer the largest carveout (so that occupancy queries see the blocks the
// registers allow); each launch then asks, by a launch attribute, for the carveout its blocks need.
static void prefer_l1()
{
    static bool done = false;
    if (done) return;
    done = true;
    for (int mode : {0, 1, 2, 3})
        for (bool rec : {false, true})
            for (int cvm : {0, 1, 2})
                for (int var : {VAR_MULTI, VAR_ONE, VAR_ZM})
                    cudaFuncSetAttribute(pick(mode, rec, cvm, var), cudaFuncAttributePreferredSharedMemoryCarveout,
                                         var == VAR_ZM && mode != 3 ? 100 : 0);
    cudaGetLastError();
}

// A launch of a kernel with the zero map: dynamic shared memory for the map, and the carveout that the
// blocks the registers allow need (with less, the CUDA runtime may fit fewer blocks; with more, L1 shrinks).
// The preference is the function's, set before each launch (launches of one function inside a step
// graph share one shape, so they need the same value).
static void launch_zm(const void* fn, const PathArgs& a, int grid, int block, size_t smem, cudaStream_t s)
{
    struct Pref {
        const void* fn;
        int block;
        size_t smem;
        int pct;
    };
    static Pref cache[64];
    static int ncache = 0;
    int pct = -1;
    for (int k = 0; k < ncache; ++k)
        if (cache[k].fn == fn && cache[k].block == block && cache[k].smem == smem) pct = cache[k].pct;
    if (pct < 0) {
        int n = 1;
        cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, block, smem) != cudaSuccess || n < 1) n = 1;
        pct = (int)carveout_pct(n, smem);
        if (ncache < 64) cache[ncache++] = Pref{fn, block, smem, pct};
    }
    cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
    void* args[] = {(void*)&a};
    cudaLaunchKernel(fn, dim3((unsigned)grid), dim3((unsigned)block), args, smem, s);
}

template <int CVM, int VAR>
static void launch_mode(const PathArgs& a, int mode, bool record, int grid, int block, size_t smem, cudaStream_t s)
{
    if (VAR == VAR_ZM && mode != 3) {
        launch_zm(pick(mode, record, CVM, VAR_ZM), a, grid, block, smem, s);
        return;
    }
    switch (mode) {
    case 3:
        if (record) k_paths_exp<true><<<grid, block, 0, s>>>(a);
        else k_paths_exp<false><<<grid, block, 0, s>>>(a);
        break;
    case 0:
        if (record) k_paths<0, true, CVM, VAR><<<grid, block, smem, s>>>(a);
        else k_paths<0, false, CVM, VAR><<<grid, block, smem, s>>>(a);
        break;
    case 2:
        if (record) k_paths<2, true, CVM, VAR><<<grid, block, smem, s>>>(a);
        else k_paths<2, false, CVM, VAR><<<grid, block, smem, s>>>(a);
        break;
    default:
        if (record) k_paths<1, true, CVM, VAR><<<grid, block, smem, s>>>(a);
        else k_paths<1, false, CVM, VAR><<<grid, block, smem, s>>>(a);
    }
}


cudaError_t launch_paths(const PathArgs& a, int exit_mode, bool record, int grid, int block, cudaStream_t s, int cvm)
{
    prefer_l1();
    const int mode = kernel_mode(exit_mode, a.K);
    const int var = path_var(a);
    const size_t smem = var == VAR_ZM && mode != 3 ? zmap_smem_bytes(a.zwords) : 0;
    switch (var * 3 + cvm) {
    case VAR_ZM * 3 + 0: launch_mode<0, VAR_ZM>(a, mode, record, grid, block, smem, s); break;
    case VAR_ZM * 3 + 1: launch_mode<1, VAR_ZM>(a, mode, record, grid, block, smem, s); break;
    case VAR_ZM * 3 + 2: launch_mode<2, VAR_ZM>(a, mode, record, grid, block, smem, s); break;
    case VAR_ONE * 3 + 0: launch_mode<0, VAR_ONE>(a, mode, record, grid, block, 0, s); break;
    case VAR_ONE * 3 + 1: launch_mode<1, VAR_ONE>(a, mode, record, grid, block, 0, s); break;
    case VAR_ONE * 3 + 2: launch_mode<2, VAR_ONE>(a, mode, record, grid, block, 0, s); break;
    case VAR_MULTI * 3 + 0: launch_mode<0, VAR_MULTI>(a, mode, record, grid, block, 0, s); break;
    case VAR_MULTI * 3 + 1: launch_mode<1, VAR_MULTI>(a, mode, record, grid, block, 0, s); break;
    default: launch_mode<2, VAR_MULTI>(a, mode, record, grid, block, 0, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_score_surv(const ScoreArgs& a, bool cv, cudaStream_t s)
{
    if (a.nnodes <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (a.nnodes <= sms) {
        if (cv) k_score_surv<true, 1024><<<a.nnodes, 1024, 0, s>>>(a);
        else k_score_surv<false, 1024><<<a.nnodes, 1024, 0, s>>>(a);
    } else {
        if (cv) k_score_surv<true, 256><<<a.nnodes, 256, 0, s>>>(a);
        else k_score_surv<false, 256><<<a.nnodes, 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalArgs& a, cudaStream_t s)
{
    const int block = 256;
    const long long threads = (long long)a.nnodes * 32;
    const int grid = (int)((threads + block - 1) / block);
    if (grid > 0) k_finalize<<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_rng_draw(uint64_t seed, const uint32_t* ctrs, long long count, uint32_t* words, float* normals,
                            cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    const int block = 256;
    k_rng_draw<<<(unsigned)((count + block - 1) / block), block, 0, s>>>(seed, ctrs, count, words, normals);
    return cudaGetLastError();
}

}  // namespace sdd
