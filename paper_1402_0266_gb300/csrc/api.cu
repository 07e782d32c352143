// api.cu -- the C ABI of libsdd (include/sdd.h): contexts, node plans, launches,
// the subdomain solve and the per-mesh-step CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sdd.h"
#include "chol.cuh"
#include "common.cuh"

using namespace sdd;

namespace {

template <typename T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    cudaError_t alloc(size_t count)
    {
        if (count <= n && p) return cudaSuccess;
        release();
        if (count == 0) return cudaSuccess;
        cudaError_t e = cudaMalloc((void**)&p, count * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            n = 0;
            return e;
        }
        n = count;
        return cudaSuccess;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
};

// A node set turned into tasks, with the device tables the kernels read.
struct Plan {
    std::vector<double> hx, hy;
    std::vector<int64_t> hp;
    std::vector<int64_t> seg_key;
    int ppt_req = -1, block_req = -1, exit_mode = -1;
    bool valid = false;

    int block = 256, grid = 0, ppt = 0;
    int zero_map = 1;   // single-instance launches: read the drift through the zero map (1) or not (0)
    bool zero_map_auto = true;   // zero_map is the tuner's choice for the plain kernel (not the caller's)
    int64_t nnodes = 0, ntasks = 0, total_paths = 0;
    std::vector<NodeDev> nodes;
    std::vector<Task> tasks;
    DevBuf<NodeDev> d_nodes;
    DevBuf<Task> d_tasks;
    DevBuf<Partial> d_partials;
    DevBuf<int> d_queue;

};

// Launch shapes chosen by the autotuner, keyed by a hash of the node set and
// the parameters that change the work (K, exit mode).
struct TunedShape {
    uint64_t key;
    int block, ppt;
    float ms;
    int zero_map;   // 1: the zero map's kernel was the faster (single instance)
};

struct GraphSlot {
    cudaGraphExec_t exec = nullptr;
    void release()
    {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
    }
};

// One implicit subdomain step: the kernels' arguments and the solver choice,
// fixed when its set-up is enqueued (the iterations may run later).
struct SolveCall {
    SolveArgs a{};
    MgArgs m{};
    bool use_mg = false;
    bool use_chol = false;      // direct (banded Cholesky) solves
    int mgc_upt = 0, mgc_C = 0, mgc_rows = 0;
    size_t mgc_smem = 0;
    const float* w = nullptr;                        // w of the step's start
    const double* px = nullptr, *pe = nullptr;        // the fields of the step's start
    double Dt = 0.0;
};

}  // namespace

struct sdd_ctx {
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    int nx = 0, ny = 0, sub_x = 1, sub_y = 1;

    DevBuf<float> w;
    DevBuf<double> fld[2][2];  // [buffer][field]: the current fields are fld[cur]
    int cur = 0;
    DevBuf<double> faces64;
    DevBuf<float> faces32;
    DevBuf<float4> bcoef, fcoef;  // bcoef holds one more record, all zero, after the cells'
    DevBuf<uint32_t> zmap;        // zero map of the drift records (see PathArgs)
    uint32_t zshift = 0;
    int zwords = 0;
    DevBuf<uint4> cvcoef;      // control-variate table (per slice and cell, half-precision corners)
    int cv_slices = 0;
    int cv_mode = 0;           // 0 off, 1 the table as set, 2 the model re-tabulated per estimate, 3 field gradient
    int cv_model_slices = 0;   // time slices of the model's table
    DevBuf<float4> cv_tmp, cv_cell;   // field gradient (mode 3): the smoothing's scratch, the cell values
    int cv_order = 0;                 // its binomial smoothing order (0: by the grid, cv_fields_order)

    // learned control variate: node features, training data, model, scratch
    DevBuf<double> cv_w64, cv_r64, cv_table64, cv_norm_scratch, cv_sxy, cv_smean[2];
    DevBuf<double2> cv_gw;
    DevBuf<float4> cv_nfa;
    DevBuf<float2> cv_nfb;
    DevBuf<float> cv_feats, cv_targets, cv_theta, cv_norm, cv_m, cv_v, cv_part, cv_losses, cv_grad_part;
    int64_t cv_rows = 0;
    int64_t cv_loss_steps = 0;
    bool cv_model = false;
    Plan sample_plan;
    DevBuf<InstDev> d_inst;
    DevBuf<int> d_status;
    DevBuf<uint32_t> d_step;
    bool user_faces = false;
    bool dirty_w = true, dirty_fields = true;

    Plan mc_plan;     // sdd_interface_mc
    Plan step_plan;   // the interface nodes of sdd_step
    std::vector<TunedShape> tuned;
    std::vector<double> iface_x, iface_y;
    std::vector<int32_t> iface_idx;
    DevBuf<int32_t> d_iface_idx;
    DevBuf<double> iface_stats[4];  // mean_xi, mean_eta, se_xi, se_eta
    DevBuf<long long> iface_counts[2];

    // solver
    DevBuf<double> cx, cy, dg, rhs0;
    DevBuf<float> cxf, cyf, dgf, dinvf, r32[2], p32[2], q32[2], d32[2];
    std::vector<SolveSys> systems;
    int solve_cluster = 1, solve_upt = 0, solve_rows_max = 0, solve_mx_max = 0;
    DevBuf<SolveSys> d_systems;
    DevBuf<int32_t> d_iters;
    // key points (Sec. 4) and the interface fill
    int keypoints = 0;
    int key_spacing = 0;
    std::vector<KeyLine> klines;
    std::vector<int32_t> kpos_idx;
    std::vector<uint8_t> kpos_cross;
    int kmax_n = 0;
    DevBuf<KeyLine> d_klines;
    DevBuf<int32_t> d_kpos_idx;
    DevBuf<uint8_t> d_kpos_cross, d_kmask;
    DevBuf<double> d_kscratch;
    // multigrid-preconditioned solver (every subdomain the same size)
    bool mg_ok = false;
    MgArgs mg{};
    int solver = 0;                 // 0 automatic, 1 Jacobi-PCG, 2 multigrid-PCG, 3 direct
    size_t solve_nsys_used = 0;     // systems of the last enqueued solve (entries of d_iters)
    DevBuf<SolveSys> mg_sys;
    DevBuf<float> mg_lv[8], mg_kv[6], mg_part, mg_rz, mg_rr0;
    DevBuf<double> mg_part64, mg_stop2;
    DevBuf<int32_t> mg_flags, mg_loop;
    cudaStream_t mg_s2 = nullptr, mg_s3 = nullptr;   // streams capturing the solve's loop bodies
    // direct solves (banded Cholesky, small subdomains): one system per subdomain
    bool chol_ok = false;
    int chol_mx = 0, chol_my = 0;
    int chol_nsys = 0;
    DevBuf<SolveSys> chol_sys;
    bool graph_mg_loops = false;    // the step graphs hold the multigrid while-loops

    // step graph (one per parity of the current field buffer)
    GraphSlot graph[2];
    int graph_kernels = 0;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // step start, paths start/end, estimate end, step end
    sdd_step_params graph_params{};
    bool graph_ok = false;
    uint32_t step_index = 0;

    // Pipelined mesh steps: the iterations of step n's subdomain solve run in
    // step n + 1's graph beside its paths, whose survivors are scored once the
    // solve is done. graph_p[parity] begins with the pending iterations.
    bool pipe_allowed = true;       // sdd_set_pipeline
    bool defer = false;             // the step graphs score survivors and plain exits after the path kernel
    bool pipe = false;              // the step graphs defer the iterations
    bool pending = false;           // iterations of the last step not enqueued yet
    SolveCall step_call[2];         // the solve set up by graph[parity] / graph_p[parity]
    SolveCall pend_call;
    GraphSlot graph_p[2];
    int graph_kernels_p = 0;
    bool last_had_pending = false;  // the last launched graph ran deferred iterations
    DevBuf<float4> surv;            // the step's path records (8 bytes per path, 16 with the control variate)
    cudaStream_t pipe_stream = nullptr;  // the side branch (highest priority)
    cudaStream_t faces_stream = nullptr; // the face data beside the drift records
    cudaEvent_t fev[2] = {nullptr, nullptr};
    // fork, join of the field records, iterations start, end, join of the systems
    cudaEvent_t pev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};

    std::string err;
};

namespace {

sdd_status vfail(std::string* err, sdd_status s, const char* fmt, va_list ap)
{
    if (err) {
        char buf[512];
        vsnprintf(buf, sizeof buf, fmt, ap);
        *err = buf;
    }
    return s;
}

sdd_status fail(std::string* err, sdd_status s, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vfail(err, s, fmt, ap);
    va_end(ap);
    return s;
}

sdd_status fail(sdd_ctx* c, sdd_status s, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vfail(c ? &c->err : nullptr, s, fmt, ap);
    va_end(ap);
    return s;
}

#define CU(c, expr)                                                                                       \
    do {                                                                                                  \
        cudaError_t e_ = (expr);                                                                          \
        if (e_ != cudaSuccess)                                                                            \
            return fail((c), e_ == cudaErrorMemoryAllocation ? SDD_ENOMEM : SDD_ECUDA, "%s: %s (%s:%d)", \
                        #expr, cudaGetErrorString(e_), __FILE__, __LINE__);                               \
    } while (0)

std::vector<int> interface_lines(int n, int parts)
{
    std::vector<int> v;
    for (int k = 1; k < parts; ++k) v.push_back((int)std::lround((double)k * (n - 1) / parts));
    return v;
}

std::vector<int> block_edges(int n, int parts)
{
    std::vector<int> v{0};
    for (int k : interface_lines(n, parts)) v.push_back(k);
    v.push_back(n - 1);
    return v;
}


// The zero map of a single instance's drift records (map null: launches without it).
struct ZmapRef {
    bool single = false;   // one instance: its tables go to the kernel as parameters
    InstDev inst{};        // the instance's tables (host copy of inst[0])
    const uint32_t* map = nullptr;   // null: no zero map
    int words = 0;
    uint32_t shift = 0;
    uint32_t cell = 0;
};

InstDev inst_host(const sdd_ctx* c)
{
    InstDev I{};
    I.bcoef = c->bcoef.p;
    I.fcoef = c->fcoef.p;
    I.faces32 = c->faces32.p;
    I.faces64 = c->faces64.p;
    I.nx = c->nx;
    I.ny = c->ny;
    I.sx = (float)(c->nx - 1);
    I.sy = (float)(c->ny - 1);
    I.gxmax = std::nextafter((float)(c->nx - 1), 0.0f);
    I.gymax = std::nextafter((float)(c->ny - 1), 0.0f);
    I.cell_bias = 0x4B000000u * (uint32_t)c->nx;
    I.cv_slices = c->cv_slices;
    I.cvcoef = c->cvcoef.p;
    I.cvcell = c->cv_cell.p;
    return I;
}

ZmapRef ctx_zmap(const sdd_ctx* c, bool use_map = true)
{
    ZmapRef z;
    z.single = true;
    z.inst = inst_host(c);
    if (!use_map) return z;
    z.map = c->zmap.p;
    z.words = c->zwords;
    z.shift = c->zshift;
    z.cell = (uint32_t)((size_t)(c->nx - 1) * (c->ny - 1));
    return z;
}

sdd_status upload_inst(sdd_ctx* c)
{
    const InstDev I = inst_host(c);
    CU(c, c->d_inst.alloc(1));
    CU(c, cudaMemcpy(c->d_inst.p, &I, sizeof I, cudaMemcpyHostToDevice));
    return SDD_OK;
}

int64_t faces_len(const sdd_ctx* c) { return 2LL * (2LL * c->nx + 2LL * c->ny); }

// Field tables for the current w, fields and face data (enqueued on s).
// The tables of the current w (faces, drift records) and fields (field
// records) on stream s, where they changed since they were last built.
sdd_status prepare_parts(sdd_ctx* c, cudaStream_t s, bool w_part, bool f_part)
{
    const bool dw = w_part && c->dirty_w, df = f_part && c->dirty_fields;
    if (dw && !c->user_faces) {
        CU(c, launch_winslow_faces(c->w.p, c->nx, c->ny, c->faces64.p, c->faces32.p, s));
    }
    if (dw || df) {
        CU(c, launch_prep_cells(c->w.p, c->fld[c->cur][0].p, c->fld[c->cur][1].p, c->nx, c->ny,
                                dw ? c->bcoef.p : nullptr, df ? c->fcoef.p : nullptr, c->d_status.p, s, c->zmap.p,
                                c->zshift));
    }
    if (w_part) c->dirty_w = false;
    if (f_part) c->dirty_fields = false;
    return SDD_OK;
}

sdd_status prepare(sdd_ctx* c, cudaStream_t s)
{
    if (c->dirty_w && c->dirty_fields) {
        // both record sets in one pass
        if (!c->user_faces) {
            CU(c, launch_winslow_faces(c->w.p, c->nx, c->ny, c->faces64.p, c->faces32.p, s));
        }
        CU(c, launch_prep_cells(c->w.p, c->fld[c->cur][0].p, c->fld[c->cur][1].p, c->nx, c->ny, c->bcoef.p,
                                c->fcoef.p, c->d_status.p, s, c->zmap.p, c->zshift));
        c->dirty_w = c->dirty_fields = false;
        return SDD_OK;
    }
    return prepare_parts(c, s, true, true);
}

bool valid_params(sdd_ctx* c, double dt, double Dt, int exit_mode, int* K)
{
    if (!(dt > 0.0) || !(Dt > 0.0) || !std::isfinite(dt) || !std::isfinite(Dt)) return false;
    const double k = Dt / dt;
    const double kr = std::round(k);
    if (kr < 1.0 || kr > (double)(1 << 20) || std::fabs(kr - k) > 1e-9 * k) return false;
    if (exit_mode != 0 && exit_mode != 1 && exit_mode != 2) return false;
    *K = (int)kr;
    (void)c;
    return true;
}

// One node list of one instance inside a plan.
struct NodeSeg {
    const double* x;
    const double* y;
    const int64_t* np;
    int64_t count;
    int32_t inst;   // instance index (tables, outputs)
    uint32_t ctr0;  // node word of the Philox counter of its first node
};

// Position of a point of the unit square along a Hilbert curve through the
// 4096 x 4096 grid of squares of side 2^-12 (24 bits). Consecutive positions
// are neighbouring squares, so nodes taken in this order lie close together.
uint64_t hilbert_key(double xf, double yf)
{
    constexpr uint32_t n = 4096;
    uint32_t x = (uint32_t)std::min<double>(std::max(xf, 0.0) * n, n - 1);
    uint32_t y = (uint32_t)std::min<double>(std::max(yf, 0.0) * n, n - 1);
    uint64_t d = 0;
    for (uint32_t s = n / 2; s > 0; s >>= 1) {
        const uint32_t qx = (x & s) ? 1u : 0u, qy = (y & s) ? 1u : 0u;
        // quadrants in curve order: (0,0), (0,1), (1,1), (1,0)
        d += (uint64_t)s * s * (qx ? (qy ? 2u : 3u) : (qy ? 1u : 0u));
        if (!qy) {
            // the lower quadrants are traversed transposed, the right one also mirrored
            if (qx) {
                x ^= s - 1;
                y ^= s - 1;
            }
            std::swap(x, y);
        }
        x &= s - 1;
        y &= s - 1;
    }
    return d;
}

// Build (or reuse) the plan of one or more node lists.
sdd_status build_plan_segs(std::string* err, int sm_count, Plan& P, const std::vector<NodeSeg>& segs, int ppt_req,
                           int block_req, int exit_mode, bool record)
{
    int64_t count = 0;
    for (const NodeSeg& g : segs) {
        if (g.count < 0 || g.count > (1LL << 30)) return fail(err, SDD_EINVAL, "node count out of range");
        for (int64_t k = 0; k < g.count; ++k) {
            if (!(g.x[k] >= 0.0 && g.x[k] <= 1.0 && g.y[k] >= 0.0 && g.y[k] <= 1.0))
                return fail(err, SDD_EINVAL, "node %lld of instance %d lies outside the unit square", (long long)k,
                            g.inst);
            if (g.np[k] < 1 || g.np[k] > 0x7fffffffLL)
                return fail(err, SDD_EINVAL, "node %lld of instance %d: n_paths out of range", (long long)k, g.inst);
        }
        count += g.count;
    }
    if (count > (1LL << 30)) return fail(err, SDD_EINVAL, "node count out of range");
    if (block_req != 0 && block_req != 64 && block_req != 128 && block_req != 256 && block_req != 512)
        return fail(err, SDD_EINVAL, "block_threads must be 0, 64, 128, 256 or 512");
    if (ppt_req < 0 || (ppt_req % 32) != 0) return fail(err, SDD_EINVAL, "paths_per_task must be a multiple of 32");

    std::vector<int64_t> key;
    key.reserve(3 * segs.size());
    for (const NodeSeg& g : segs) {
        key.push_back(g.count);
        key.push_back(g.inst);
        key.push_back(g.ctr0);
    }
    bool same = P.valid && P.ppt_req == ppt_req && P.block_req == block_req && P.exit_mode == exit_mode &&
                (int64_t)P.hx.size() == count && P.seg_key == key;
    if (same) {
        int64_t o = 0;
        for (const NodeSeg& g : segs) {
            same = same && std::equal(g.x, g.x + g.count, P.hx.begin() + o) &&
                   std::equal(g.y, g.y + g.count, P.hy.begin() + o) && std::equal(g.np, g.np + g.count, P.hp.begin() + o);
            o += g.count;
        }
    }
    if (same) return SDD_OK;

    P.hx.clear();
    P.hy.clear();
    P.hp.clear();
    for (const NodeSeg& g : segs) {
        P.hx.insert(P.hx.end(), g.x, g.x + g.count);
        P.hy.insert(P.hy.end(), g.y, g.y + g.count);
        P.hp.insert(P.hp.end(), g.np, g.np + g.count);
    }
    P.seg_key = key;
    P.ppt_req = ppt_req;
    P.block_req = block_req;
    P.exit_mode = exit_mode;
    P.valid = false;

    int64_t total = 0;
    for (int64_t k = 0; k < count; ++k) total += P.hp[k];
    P.block = std::min(block_req ? block_req : 256, path_kernel_max_block(exit_mode));
    const int per_sm = path_kernel_blocks_per_sm(exit_mode, record, P.block);
    P.grid = sm_count * per_sm;
    if (ppt_req) {
        P.ppt = ppt_req;
    } else {
        // about 8 tasks per resident warp, 32..2048 paths per task
        const int64_t warps = (int64_t)P.grid * (P.block / 32);
        int64_t q = total / (32LL * 8 * std::max<int64_t>(warps, 1));
        q = std::min<int64_t>(std::max<int64_t>(q, 1), 64);
        P.ppt = (int)(32 * q);
    }
    P.nodes.resize(count);
    P.tasks.clear();
    std::vector<int32_t> inst_of(count), local_of(count);
    std::vector<uint32_t> ctr_of(count);
    {
        int64_t o = 0, rec = 0;
        for (const NodeSeg& g : segs)
            for (int64_t k = 0; k < g.count; ++k, ++o) {
                P.nodes[o].rec0 = rec;
                rec += g.np[k];
                inst_of[o] = g.inst;
                local_of[o] = (int32_t)k;
                ctr_of[o] = g.ctr0 + (uint32_t)k;
            }
    }
    const double* x = P.hx.data();
    const double* y = P.hy.data();
    const int64_t* np = P.hp.data();
    // Tasks go node by node, the nodes of each instance along a Hilbert curve:
    // the nodes whose paths run at the same time lie close together, and so
    // do the cells their paths read (L2 keeps that neighbourhood; in the order
    // of the nodes' distance from the boundary the nodes in flight lay around
    // the whole square and the cell tables of a large grid spilled to DRAM).
    std::vector<int64_t> order(count);
    for (int64_t k = 0; k < count; ++k) order[k] = k;
    std::vector<uint64_t> hk(count);
    for (int64_t k = 0; k < count; ++k) hk[k] = ((uint64_t)(uint32_t)inst_of[k] << 26) | hilbert_key(x[k], y[k]);
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return hk[a] < hk[b]; });
    for (int64_t k : order) {
        NodeDev& nd = P.nodes[k];
        nd.x = x[k];
        nd.y = y[k];
        nd.xf = (float)x[k];
        nd.yf = (float)y[k];
        nd.inst = inst_of[k];
        nd.ctr = ctr_of[k];
        nd.n_paths = (int32_t)np[k];
        nd.local = local_of[k];
        const bool bnd = x[k] <= 0.0 || x[k] >= 1.0 || y[k] <= 0.0 || y[k] >= 1.0;
        nd.task0 = (int32_t)P.tasks.size();
        if (bnd) {
            nd.ntasks = 0;
            continue;
        }
        for (int64_t p0 = 0; p0 < np[k]; p0 += P.ppt) {
            Task t{};
            t.node = (int32_t)k;
            t.path0 = (int32_t)p0;
            t.npaths = (int32_t)std::min<int64_t>(P.ppt, np[k] - p0);
            P.tasks.push_back(t);
        }
        nd.ntasks = (int32_t)(P.tasks.size() - nd.task0);
        if (P.tasks.size() > 0x7fffffffULL) return fail(err, SDD_EINVAL, "too many tasks");
    }
    P.nnodes = count;
    P.ntasks = (int64_t)P.tasks.size();
    P.total_paths = total;
    // an earlier launch of this plan may still read its buffers on a stream
    // that does not wait for the synchronous copies below
    CU(err, cudaDeviceSynchronize());
    CU(err, P.d_nodes.alloc(std::max<int64_t>(count, 1)));
    CU(err, P.d_tasks.alloc(std::max<int64_t>(P.ntasks, 1)));
    CU(err, P.d_partials.alloc(std::max<int64_t>(P.ntasks, 1)));
    CU(err, P.d_queue.alloc(1));
    if (count) CU(err, cudaMemcpy(P.d_nodes.p, P.nodes.data(), count * sizeof(NodeDev), cudaMemcpyHostToDevice));
    if (P.ntasks)
        CU(err, cudaMemcpy(P.d_tasks.p, P.tasks.data(), P.ntasks * sizeof(Task), cudaMemcpyHostToDevice));
    P.valid = true;
    return SDD_OK;
}

uint64_t shape_key(const std::vector<NodeSeg>& segs, int K, int exit_mode)
{
    uint64_t h = 1469598103934665603ULL;
    auto mix = [&](const void* p, size_t n) {
        const unsigned char* b = (const unsigned char*)p;
        for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ULL;
    };
    for (const NodeSeg& g : segs) {
        mix(&g.count, sizeof g.count);
        mix(&g.inst, sizeof g.inst);
        mix(g.x, g.count * sizeof(double));
        mix(g.y, g.count * sizeof(double));
        mix(g.np, g.count * sizeof(int64_t));
    }
    mix(&K, sizeof K);
    mix(&exit_mode, sizeof exit_mode);
    return h;
}

sdd_status run_plan_on(std::string* err, Plan& P, const InstDev* inst, const OutDev* outs, const OutDev& out0, double dt,
                       int K, uint64_t seed, uint32_t step_index, const uint32_t* step_ptr, int exit_mode,
                       const RecDev* rec, cudaStream_t s, cudaEvent_t ev_a, cudaEvent_t ev_b, int cv_slices = 0,
                       const uint8_t* node_mask = nullptr, void* surv = nullptr, cudaEvent_t join = nullptr,
                       ZmapRef zm = ZmapRef{}, bool cv_cell = false);

const TunedShape* find_tuned(const std::vector<TunedShape>& t, uint64_t key)
{
    for (const TunedShape& s : t)
        if (s.key == key) return &s;
    return nullptr;
}

// Time every candidate launch shape on this node set (outputs discarded) and
// keep the fastest: block sizes 128 / 256 / 512 x paths per task 32 .. 1024.
sdd_status autotune_plan(std::string* err, int sm_count, const std::vector<NodeSeg>& segs, const InstDev* inst,
                         int ninst, int K, double dt, int exit_mode, cudaStream_t s, std::vector<TunedShape>& cache,
                         TunedShape* best_out, ZmapRef zm = ZmapRef{})
{
    int64_t count = 0;
    for (const NodeSeg& g : segs) count += g.count;
    DevBuf<double> dmean;
    DevBuf<OutDev> dout;
    CU(err, dmean.alloc(std::max<int64_t>(count, 1)));
    std::vector<OutDev> outs(ninst);
    {
        int64_t o = 0;
        for (int k = 0; k < ninst; ++k) {
            outs[k] = OutDev{};
            outs[k].mean_xi = dmean.p + o;  // only the means are written, each instance its own slice
            o += segs[k].count;
        }
    }
    CU(err, dout.alloc(ninst));
    CU(err, cudaMemcpy(dout.p, outs.data(), ninst * sizeof(OutDev), cudaMemcpyHostToDevice));
    cudaEvent_t e0, e1;
    CU(err, cudaEventCreate(&e0));
    CU(err, cudaEventCreate(&e1));
    TunedShape best{shape_key(segs, K, exit_mode), 256, 0, 1e30f, zm.map != nullptr ? 1 : 0};
    sdd_status st = SDD_OK;
    // a single instance: the kernel with the zero map and the one without (it saves the map's
    // instructions where the drift has few zero cells)
    for (int use_map = zm.map != nullptr ? 1 : 0; use_map >= 0 && st == SDD_OK; --use_map) {
        ZmapRef z = zm;
        if (!use_map) z.map = nullptr;
        for (int block : {128, 256, 512}) {
            if (block > path_kernel_max_block(exit_mode, 0, z.single)) continue;
            for (int ppt : {32, 64, 128, 256, 512, 1024}) {
                Plan P;
                st = build_plan_segs(err, sm_count, P, segs, ppt, block, exit_mode, false);
                if (st != SDD_OK) break;
                // one untimed run, then the mean of two timed runs
                st = run_plan_on(err, P, inst, dout.p, OutDev{}, dt, K, 0x5EEDULL, 0, nullptr, exit_mode, nullptr, s,
                                 nullptr, nullptr, 0, nullptr, nullptr, nullptr, z);
                if (st == SDD_OK && cudaEventRecord(e0, s) != cudaSuccess) st = fail(err, SDD_ECUDA, "event record");
                for (int r = 0; r < 2 && st == SDD_OK; ++r)
                    st = run_plan_on(err, P, inst, dout.p, OutDev{}, dt, K, 0x5EEDULL + r, 0, nullptr, exit_mode,
                                     nullptr, s, nullptr, nullptr, 0, nullptr, nullptr, nullptr, z);
                if (st == SDD_OK && cudaEventRecord(e1, s) != cudaSuccess) st = fail(err, SDD_ECUDA, "event record");
                if (st == SDD_OK && cudaEventSynchronize(e1) != cudaSuccess) st = fail(err, SDD_ECUDA, "event sync");
                if (st != SDD_OK) break;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                ms *= 0.5f;
                if (ms < best.ms) {
                    best.block = block;
                    best.ppt = ppt;
                    best.ms = ms;
                    best.zero_map = use_map;
                }
            }
            if (st != SDD_OK) break;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SDD_OK) return st;
    for (TunedShape& t : cache)
        if (t.key == best.key) {
            t = best;
            *best_out = best;
            return SDD_OK;
        }
    cache.push_back(best);
    *best_out = best;
    return SDD_OK;
}

sdd_status build_plan(sdd_ctx* c, Plan& P, const double* x, const double* y, const int64_t* np, int64_t count,
                      int ppt_req, int block_req, int exit_mode, bool record, uint32_t ctr0 = 0)
{
    std::vector<NodeSeg> segs(1);
    segs[0] = NodeSeg{x, y, np, count, 0, ctr0};
    return build_plan_segs(&c->err, c->sm_count, P, segs, ppt_req, block_req, exit_mode, record);
}

// Enqueue the estimate for a built plan. inst: the instance table; outs:
// per-instance outputs (null: every node writes to out0). surv: if non-null,
// the survivors' scores are deferred to a second kernel that runs once event
// `join` (if non-null) has completed: P.total_paths records of float2, or of
// float4 with the control variate.
sdd_status run_plan_on(std::string* err, Plan& P, const InstDev* inst, const OutDev* outs, const OutDev& out0, double dt,
                       int K, uint64_t seed, uint32_t step_index, const uint32_t* step_ptr, int exit_mode,
                       const RecDev* rec, cudaStream_t s, cudaEvent_t ev_a, cudaEvent_t ev_b, int cv_slices,
                       const uint8_t* node_mask, void* surv, cudaEvent_t join, ZmapRef zm, bool cv_cell)
{
    if (surv && rec) return fail(err, SDD_EINVAL, "per-path records with deferred survivor scores");
    if (P.nnodes == 0 || P.ntasks == 0) {
        if (join) CU(err, cudaStreamWaitEvent(s, join, 0));
        if (P.nnodes == 0) return SDD_OK;
    }
    if (P.ntasks > 0) {
        PathArgs a{};
        a.inst = inst;
        a.nodes = P.d_nodes.p;
        a.tasks = P.d_tasks.p;
        a.partials = P.d_partials.p;
        a.queue = P.d_queue.p;
        a.ntasks = (int32_t)P.ntasks;
        a.K = K;
        a.dt = (float)dt;
        a.bm_scale = (float)(-4.0 * dt * std::log(2.0));
        a.bridge_cut = (float)(18.0 * dt);
        a.horizon = (float)((double)K * dt);
        a.keys = philox_keys(seed);
        a.step_index = step_index;
        a.step_ptr = step_ptr;
        if (rec) a.rec = *rec;
        a.node_mask = node_mask;
        a.surv = surv;
        if (zm.single) {
            a.single = 1;
            a.one = zm.inst;
            if (zm.map && zm.words > 0 && zm.words <= kZmapMaxWords) {
                a.zmap = zm.map;
                a.zwords = zm.words;
                a.zshift = zm.shift;
                a.zcell = zm.cell;
            }
        }
        const bool cv = cv_slices > 0;
        const int cvm = !cv ? 0 : cv_cell ? 2 : 1;
        if (cv && cv_slices > K) return fail(err, SDD_EINVAL, "more control-variate slices than sub-steps per step");
        if (cv && exit_mode == 2)
            return fail(err, SDD_EINVAL, "the control variate needs fixed sub-steps (exit_mode 0 or 1)");
        for (int q = 0; q <= kMaxCvSlices; ++q)
            a.cv_bound[q] = cv && q <= cv_slices ? (int32_t)(((int64_t)q * K + cv_slices - 1) / cv_slices) : K + 1;
        CU(err, cudaMemsetAsync(P.d_queue.p, 0, sizeof(int), s));
        // each path kernel is compiled for at most path_kernel_max_block threads per block
        const int block = std::min(P.block, path_kernel_max_block(exit_mode, cvm, a.single != 0));
        const int64_t per_block = block / 32;
        int grid_max = P.grid;
        if (block != P.block || cv || a.single) {
            int dev = 0, sms = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            grid_max = sms * path_kernel_blocks_per_sm(exit_mode, rec != nullptr, block, cvm, a.zwords, a.single != 0);
        }
        const int grid = (int)std::min<int64_t>(grid_max, std::max<int64_t>(1, (P.ntasks + per_block - 1) / per_block));
        if (ev_a) CU(err, cudaEventRecordWithFlags(ev_a, s, cudaEventRecordExternal));
        CU(err, launch_paths(a, exit_mode, rec != nullptr, grid, block, s, cvm));
        if (ev_b) CU(err, cudaEventRecordWithFlags(ev_b, s, cudaEventRecordExternal));
        if (join) CU(err, cudaStreamWaitEvent(s, join, 0));
    }
    FinalArgs f{};
    f.inst = inst;
    f.nodes = P.d_nodes.p;
    f.partials = P.d_partials.p;
    f.out_table = outs;
    f.out0 = out0;
    f.nnodes = (int32_t)P.nnodes;
    if (rec) f.rec = *rec;
    f.node_mask = node_mask;
    if (surv && P.ntasks > 0) {
        // the survivors' scores and the per-node reduction in one launch
        ScoreArgs sa{};
        sa.inst = inst;
        sa.nodes = P.d_nodes.p;
        sa.surv = surv;
        sa.nnodes = (int32_t)P.nnodes;
        sa.fin = f;
        const bool cv = cv_slices > 0;
        CU(err, launch_score_surv(sa, cv, s));
        return SDD_OK;
    }
    CU(err, launch_finalize(f, s));
    return SDD_OK;
}

// The tuner times the plain kernel; where it left the zero map off (the plain kernel is no faster
// with it) a control-variate launch still takes it: that kernel is bound by L1 wavefronts, which
// the map saves wherever a warp's lanes share the all-zero record.
sdd_status run_plan(sdd_ctx* c, Plan& P, double dt, int K, uint64_t seed, uint32_t step_index,
                    const uint32_t* step_ptr, int exit_mode, const OutDev& out, const RecDev* rec, cudaStream_t s,
                    cudaEvent_t ev_a = nullptr, cudaEvent_t ev_b = nullptr, const uint8_t* node_mask = nullptr,
                    void* surv = nullptr, cudaEvent_t join = nullptr)
{
    return run_plan_on(&c->err, P, c->d_inst.p, nullptr, out, dt, K, seed, step_index, step_ptr, exit_mode, rec, s,
                       ev_a, ev_b, c->cv_mode ? c->cv_slices : 0, node_mask, surv, join,
                       ctx_zmap(c, P.zero_map != 0 || (P.zero_map_auto && c->cv_mode != 0)), c->cv_mode == SDD_CV_FIELDS);
}

// Launch shape for a plan: explicit requests win, else a tuned shape for this node set, else the heuristic.
// zero_map (if non-null): the caller's request (0 automatic: the tuned choice, else on; 1 on; 2 off) in,
// 1 (use the zero map) or 0 out.
void pick_shape(const std::vector<TunedShape>& cache, const std::vector<NodeSeg>& segs, int K, int exit_mode,
                int* ppt, int* block, int* zero_map = nullptr)
{
    const TunedShape* t = find_tuned(cache, shape_key(segs, K, exit_mode));
    if (zero_map) *zero_map = *zero_map == 0 ? (t ? t->zero_map : 1) : (*zero_map == 1 ? 1 : 0);
    if (*ppt || *block) return;
    if (t) {
        *ppt = t->ppt;
        *block = t->block;
    }
}

sdd_status setup_solver(sdd_ctx* c)
{
    const size_t N = (size_t)c->nx * c->ny;
    CU(c, c->cx.alloc(N));
    CU(c, c->cy.alloc(N));
    CU(c, c->dg.alloc(N));
    CU(c, c->rhs0.alloc(2 * N));
    CU(c, c->cxf.alloc(N));
    CU(c, c->cyf.alloc(N));
    CU(c, c->dgf.alloc(N));
    CU(c, c->dinvf.alloc(N));
    for (int f = 0; f < 2; ++f) {
        CU(c, c->r32[f].alloc(N));
        CU(c, c->p32[f].alloc(N));
        CU(c, c->q32[f].alloc(N));
        CU(c, c->d32[f].alloc(N));
        // the search direction stays zero on the boundary and interface nodes
        CU(c, cudaMemset(c->p32[f].p, 0, N * sizeof(float)));
    }
    const std::vector<int> xs = block_edges(c->nx, c->sub_x), ys = block_edges(c->ny, c->sub_y);
    // subdomains (both fields solved together by the register-resident kernel)
    std::vector<SolveSys> subs;
    int min_rows = 1 << 30;
    for (int b = 0; b < c->sub_y; ++b)
        for (int a = 0; a < c->sub_x; ++a) {
            SolveSys S{};
            S.i0 = xs[a] + 1;
            S.i1 = xs[a + 1];
            S.j0 = ys[b] + 1;
            S.j1 = ys[b + 1];
            S.field = -1;
            if (S.i1 > S.i0 && S.j1 > S.j0) {
                subs.push_back(S);
                min_rows = std::min(min_rows, S.j1 - S.j0);
            }
        }
    c->solve_upt = 0;
    if (!subs.empty()) {
        const int C = solve_cluster_size((int)subs.size(), min_rows, c->sm_count);
        int band_max = 0, rows_max = 0, mx_max = 0;
        for (const SolveSys& S : subs) {
            const int my = S.j1 - S.j0, mx = S.i1 - S.i0;
            for (int rk = 0; rk < C; ++rk) {
                const int rows = (my * (rk + 1)) / C - (my * rk) / C;
                rows_max = std::max(rows_max, rows);
                band_max = std::max(band_max, rows * mx);
            }
            mx_max = std::max(mx_max, mx);
        }
        c->solve_upt = solve_reg_upt(band_max);
        if (4 * (size_t)(rows_max + 2) * (mx_max + 2) * sizeof(float) > 200 * 1024 || C > 16) c->solve_upt = 0;
        if (c->solve_upt) {
            c->systems = subs;
            c->solve_cluster = C;
            c->solve_rows_max = rows_max;
            c->solve_mx_max = mx_max;
        }
    }
    if (!c->solve_upt) {
        // general kernel: one system per subdomain and field
        c->systems.clear();
        for (int field = 0; field < 2; ++field)
            for (const SolveSys& S0 : subs) {
                SolveSys S = S0;
                S.field = field;
                c->systems.push_back(S);
            }
        c->solve_cluster = c->systems.empty() ? 1 : solve_cluster_size((int)c->systems.size(), min_rows, c->sm_count);
    }
    CU(c, c->d_systems.alloc(std::max<size_t>(c->systems.size(), 1)));
    if (!c->systems.empty())
        CU(c, cudaMemcpy(c->d_systems.p, c->systems.data(), c->systems.size() * sizeof(SolveSys),
                         cudaMemcpyHostToDevice));
    CU(c, c->d_iters.alloc(std::max<size_t>(std::max(c->systems.size(), subs.size()), 1)));

    // multigrid: every subdomain the same odd sizes, coarsening down to a small box
    c->mg_ok = false;
    bool same = !subs.empty();
    for (const SolveSys& S : subs)
        same = same && (S.i1 - S.i0) == (subs[0].i1 - subs[0].i0) && (S.j1 - S.j0) == (subs[0].j1 - subs[0].j0);
    MgArgs m{};
    if (same && mg_levels(subs[0].i1 - subs[0].i0, subs[0].j1 - subs[0].j0, m)) {
        const long long total = mg_layout(m, (int)subs.size());
        const long long P0 = (long long)(m.mx[0] + 2) * (m.my[0] + 2) * (long long)subs.size();
        for (auto& b : c->mg_lv) CU(c, b.alloc((size_t)total));
        for (auto& b : c->mg_kv) CU(c, b.alloc((size_t)P0));
        const size_t ns = subs.size();
        CU(c, c->mg_part.alloc(ns * m.B0 * 4));
        CU(c, c->mg_part64.alloc(ns * m.B0 * 4));
        CU(c, c->mg_stop2.alloc(2 * ns));
        CU(c, c->mg_rz.alloc(4 * ns));
        CU(c, c->mg_rr0.alloc(2 * ns));
        CU(c, c->mg_flags.alloc(6 * ns));
        CU(c, c->mg_loop.alloc(3));
        CU(c, cudaMemset(c->mg_loop.p, 0, 3 * sizeof(int32_t)));
        if (!c->mg_s2) CU(c, cudaStreamCreateWithFlags(&c->mg_s2, cudaStreamNonBlocking));
        if (!c->mg_s3) CU(c, cudaStreamCreateWithFlags(&c->mg_s3, cudaStreamNonBlocking));
        CU(c, cudaMemset(c->mg_rz.p, 0, 4 * ns * sizeof(float)));
        CU(c, cudaMemset(c->mg_flags.p, 0, 6 * ns * sizeof(int32_t)));
        CU(c, c->mg_sys.alloc(ns));
        CU(c, cudaMemcpy(c->mg_sys.p, subs.data(), ns * sizeof(SolveSys), cudaMemcpyHostToDevice));
        c->mg = m;
        c->mg_ok = true;
    }

    // direct solves where every subdomain's band fits one block's shared memory
    c->chol_ok = !subs.empty();
    c->chol_mx = c->chol_my = 0;
    for (const SolveSys& S : subs) {
        c->chol_ok = c->chol_ok && chol_fits(S.i1 - S.i0, S.j1 - S.j0);
        c->chol_mx = std::max(c->chol_mx, S.i1 - S.i0);
        c->chol_my = std::max(c->chol_my, S.j1 - S.j0);
    }
    c->chol_ok = c->chol_ok && chol_fits(c->chol_mx, c->chol_my);
    if (c->chol_ok) {
        c->chol_nsys = (int)subs.size();
        CU(c, c->chol_sys.alloc(subs.size()));
        CU(c, cudaMemcpy(c->chol_sys.p, subs.data(), subs.size() * sizeof(SolveSys), cudaMemcpyHostToDevice));
    }
    return SDD_OK;
}

void build_interface(sdd_ctx* c)
{
    const std::vector<int> vi = interface_lines(c->nx, c->sub_x), hj = interface_lines(c->ny, c->sub_y);
    c->iface_x.clear();
    c->iface_y.clear();
    c->iface_idx.clear();
    for (int I : vi)
        for (int j = 1; j < c->ny - 1; ++j) {
            c->iface_x.push_back((double)I / (c->nx - 1));
            c->iface_y.push_back((double)j / (c->ny - 1));
            c->iface_idx.push_back(j * c->nx + I);
        }
    for (int J : hj)
        for (int i = 1; i < c->nx - 1; ++i) {
            bool on_v = false;
            for (int I : vi) on_v |= (I == i);
            if (on_v) continue;
            c->iface_x.push_back((double)i / (c->nx - 1));
            c->iface_y.push_back((double)J / (c->ny - 1));
            c->iface_idx.push_back(J * c->nx + i);
        }
    // the interface lines as key-point lines: interior positions -> interface-node index
    c->klines.clear();
    c->kpos_idx.clear();
    c->kpos_cross.clear();
    c->kmax_n = 0;
    const int nv = c->ny - 2;
    for (size_t a = 0; a < vi.size(); ++a) {
        KeyLine L{0, vi[a], c->ny, (int32_t)c->kpos_idx.size()};
        for (int j = 1; j < c->ny - 1; ++j) {
            bool cross = false;
            for (int J : hj) cross |= (J == j);
            c->kpos_idx.push_back((int32_t)(a * nv + (j - 1)));
            c->kpos_cross.push_back(cross ? 1 : 0);
        }
        c->klines.push_back(L);
        c->kmax_n = std::max(c->kmax_n, c->ny);
    }
    int32_t next = (int32_t)(vi.size() * nv);
    for (int J : hj) {
        KeyLine L{1, J, c->nx, (int32_t)c->kpos_idx.size()};
        for (int i = 1; i < c->nx - 1; ++i) {
            int a_cross = -1;
            for (size_t a = 0; a < vi.size(); ++a)
                if (vi[a] == i) a_cross = (int)a;
            if (a_cross >= 0) {
                c->kpos_idx.push_back((int32_t)(a_cross * nv + (J - 1)));
                c->kpos_cross.push_back(1);
            } else {
                c->kpos_idx.push_back(next++);
                c->kpos_cross.push_back(0);
            }
        }
        c->klines.push_back(L);
        c->kmax_n = std::max(c->kmax_n, c->nx);
    }
}

// Key-point mask of the current w (one byte per interface node) on stream s.
sdd_status enqueue_keypoints(sdd_ctx* c, uint8_t* mask, cudaStream_t s)
{
    CU(c, launch_keypoints(c->w.p, c->nx, c->d_klines.p, (int)c->klines.size(), c->kmax_n, c->d_kpos_idx.p,
                           c->d_kpos_cross.p, c->key_spacing, mask, s));
    return SDD_OK;
}

// Automatic solver choice: multigrid where the register-resident Jacobi kernel
// does not fit, and from 10,000 unknowns per subdomain (127^2: 1.32 against
// 1.56 ms per step at 257^2 with 2 x 2 subdomains; 19^2: Jacobi is faster).
bool mg_auto(const sdd_ctx* c)
{
    return c->solve_upt == 0 || (long long)c->mg.mx[0] * c->mg.my[0] >= 10000;
}

// The solver the next solve uses: 3 direct, 2 multigrid-PCG, 1 Jacobi-PCG. The
// direct solve is taken only on request: its column and substitution chains
// are sequential, and Jacobi-PCG is faster on every subdomain it fits (19^2:
// 159 against 176 us per solve with the set-up, 31^2: 222 against 605 us).
int solver_choice(const sdd_ctx* c)
{
    if (c->solver == 3 && c->chol_ok) return 3;
    if (c->mg_ok && (c->solver == 2 || (c->solver == 0 && mg_auto(c)))) return 2;
    return 1;
}

SolveCall make_solve_call(sdd_ctx* c, double Dt, double rtol, int max_iter, double* xo, double* eo,
                          const float* w, const double* px, const double* pe, bool narrow = false)
{
    SolveCall k;
    k.w = w;
    k.px = px;
    k.pe = pe;
    k.Dt = Dt;
    SolveArgs& a = k.a;
    a.nx = c->nx;
    a.ny = c->ny;
    a.cx = c->cx.p;
    a.cy = c->cy.p;
    a.dg = c->dg.p;
    a.rhs0 = c->rhs0.p;
    a.cxf = c->cxf.p;
    a.cyf = c->cyf.p;
    a.dgf = c->dgf.p;
    a.dinvf = c->dinvf.p;
    a.x[0] = xo;
    a.x[1] = eo;
    for (int f = 0; f < 2; ++f) {
        a.r[f] = c->r32[f].p;
        a.p[f] = c->p32[f].p;
        a.q[f] = c->q32[f].p;
        a.d[f] = c->d32[f].p;
    }
    a.sys = c->d_systems.p;
    a.nsys = (int32_t)c->systems.size();
    a.cluster = c->solve_cluster;
    a.max_iter = max_iter;
    a.max_outer = 12;
    a.rtol = rtol;
    a.inner_tol = 1e-4f;
    a.iters = c->d_iters.p;
    a.status = c->d_status.p;
    k.use_chol = solver_choice(c) == 3;
    k.use_mg = !k.use_chol && solver_choice(c) == 2;
    if (k.use_mg) {
        MgArgs& m = k.m;
        m = c->mg;
        m.nx = c->nx;
        m.ny = c->ny;
        m.cx = c->cx.p;
        m.cy = c->cy.p;
        m.dg = c->dg.p;
        m.rhs0 = c->rhs0.p;
        m.cxf = c->cxf.p;
        m.cyf = c->cyf.p;
        m.dgf = c->dgf.p;
        m.w = w;
        m.Dt = Dt;
        m.x[0] = xo;
        m.x[1] = eo;
        m.sys = c->mg_sys.p;
        m.D = c->mg_lv[0].p;
        m.CX = c->mg_lv[1].p;
        m.CY = c->mg_lv[2].p;
        m.MS = c->mg_lv[3].p;
        m.U[0] = c->mg_lv[4].p;
        m.U[1] = c->mg_lv[5].p;
        m.F[0] = c->mg_lv[6].p;
        m.F[1] = c->mg_lv[7].p;
        for (int f = 0; f < 2; ++f) {
            m.Pv[f] = c->mg_kv[f].p;
            m.Qv[f] = c->mg_kv[2 + f].p;
            m.Cv[f] = c->mg_kv[4 + f].p;
        }
        const size_t ns = (size_t)m.nsys;
        m.part = c->mg_part.p;
        m.part64 = c->mg_part64.p;
        m.stop2 = c->mg_stop2.p;
        m.rz = c->mg_rz.p;
        m.rr0 = c->mg_rr0.p;
        m.act_o = c->mg_flags.p;
        m.act_i = c->mg_flags.p + 2 * ns;
        m.iters = c->mg_flags.p + 4 * ns;
        m.sys_iters = c->d_iters.p;
        m.loop = c->mg_loop.p;
        m.launches = c->mg_loop.p + 2;
        m.status = c->d_status.p;
        m.nu = 2;
        m.coarse_sweeps = 20;
        m.max_iter = max_iter;
        m.rtol = rtol;
        m.inner_tol = 1e-5f;
        k.mgc_upt = mgc_config(m, &k.mgc_C, &k.mgc_rows, &k.mgc_smem, narrow ? 4 : 2);
        if (k.mgc_upt > 0) m.outer = 8;
    }
    return k;
}

// The iterations are one kernel launch (the cluster multigrid solve or the
// Jacobi-PCG kernels), so they can run beside other work.
bool solve_single_launch(const SolveCall& k) { return k.use_chol || !k.use_mg || k.mgc_upt > 0; }

// The Dirichlet data of an implicit subdomain step on stream s: the faces and
// the interface values written into the new fields, the old fields inside.
sdd_status enqueue_solve_dirichlet(sdd_ctx* c, const SolveCall& k, const double* ix, const double* ie,
                                   cudaStream_t s)
{
    CU(c, launch_dirichlet(c->faces64.p, k.px, k.pe, ix, ie, c->d_iface_idx.p, (int)c->iface_idx.size(), c->nx,
                           c->ny, k.a.x[0], k.a.x[1], s));
    return SDD_OK;
}

// The systems of an implicit subdomain step on stream s: coefficients and
// right-hand sides from w and the fields of the step's start, the multigrid
// hierarchy.
sdd_status enqueue_solve_system(sdd_ctx* c, const SolveCall& k, cudaStream_t s)
{
    CU(c, launch_solve_setup(k.w, k.px, k.pe, c->nx, c->ny, k.Dt, c->cx.p, c->cy.p, c->dg.p, c->rhs0.p, c->cxf.p,
                             c->cyf.p, c->dgf.p, c->dinvf.p, s));
    if (k.use_mg) CU(c, launch_mg_setup(k.m, s));
    return SDD_OK;
}

// The iterations of the implicit subdomain step on stream s: the new fields.
sdd_status enqueue_solve_iterate(sdd_ctx* c, const SolveCall& k, cudaStream_t s)
{
    if (k.use_chol) {
        SolveArgs a = k.a;
        a.sys = c->chol_sys.p;
        a.nsys = c->chol_nsys;
        CU(c, launch_chol(a, c->chol_mx, c->chol_my, s));
        c->solve_nsys_used = (size_t)c->chol_nsys;
        return SDD_OK;
    }
    if (k.use_mg) {
        MgArgs m = k.m;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        CU(c, cudaStreamIsCapturing(s, &cs));
        if (k.mgc_upt > 0) {
            // subdomains that fit one cluster: the whole solve in one launch
            CU(c, launch_mgc(m, k.mgc_upt, k.mgc_C, k.mgc_rows, k.mgc_smem, s));
        } else if (cs == cudaStreamCaptureStatusActive) {
            // inside the step's graph: while-loops that stop once every field has converged
            m.inner = std::max(1, std::min(30, m.max_iter));
            m.outer = std::max(1, std::min(8, m.max_iter / m.inner));
            CU(c, launch_mg_solve_graph(m, s, c->mg_s2, c->mg_s3));
            c->graph_mg_loops = true;
        } else {
            // a direct call: a fixed number of passes (5 inner iterations x 6 sweeps at most)
            m.inner = std::max(1, std::min(5, m.max_iter));
            m.outer = std::max(1, std::min(6, m.max_iter / m.inner));
            CU(c, launch_mg_solve(m, s));
        }
        c->solve_nsys_used = (size_t)m.nsys;
        return SDD_OK;
    }
    CU(c, launch_pcg(k.a, c->solve_upt, c->solve_rows_max, c->solve_mx_max, s));
    c->solve_nsys_used = c->systems.size();
    return SDD_OK;
}

// The implicit subdomain step on stream s, set-up and iterations. xo/eo
// receive the new fields.
sdd_status enqueue_solve(sdd_ctx* c, double Dt, const double* ix, const double* ie, double rtol, int max_iter,
                         double* xo, double* eo, cudaStream_t s)
{
    const SolveCall k = make_solve_call(c, Dt, rtol, max_iter, xo, eo, c->w.p, c->fld[c->cur][0].p,
                                        c->fld[c->cur][1].p);
    sdd_status st = enqueue_solve_system(c, k, s);
    if (st == SDD_OK) st = enqueue_solve_dirichlet(c, k, ix, ie, s);
    if (st != SDD_OK) return st;
    return enqueue_solve_iterate(c, k, s);
}


// Enqueue the deferred iterations of the last mesh step's solve on the
// context's stream: afterwards the current fields are final.
sdd_status flush_pending(sdd_ctx* c)
{
    if (!c->pending) return SDD_OK;
    c->pending = false;
    return enqueue_solve_iterate(c, c->pend_call, c->stream);
}

void drop_graphs_fn(sdd_ctx* c)
{
    c->graph[0].release();
    c->graph[1].release();
    c->graph_p[0].release();
    c->graph_p[1].release();
    c->graph_ok = false;
    c->graph_mg_loops = false;
}

// ---------------------------------------------------------------- learned control variate (host side)

constexpr uint32_t kInitWord = 0x494E4954u;        // counter word of the initial weights
constexpr uint32_t kSampleStepWord = 0xFFFFFFFFu;  // step word of the training paths

// u = ((bits >> 8) + 0.5) 2^-24: a uniform in (0, 1) with 24 significant bits
double unit_open(uint32_t bits) { return ((double)(bits >> 8) + 0.5) * (1.0 / 16777216.0); }

// Glorot-uniform weights, zero biases; weight p of network f from word 0 of
// the Philox block with counter (p, f, kInitWord, 0).
void init_params_host(uint64_t seed, std::vector<float>& th)
{
    th.assign(2 * (size_t)kMlpStride, 0.f);
    const int H = kMlpHidden, D = kMlpInputs;
    struct Seg { int a, b, fan_in, fan_out; };
    const Seg segs[3] = {{0, H * D, D, H}, {H * D + H, H * D + H + H * H, H, H},
                         {H * D + 2 * H + H * H, H * D + 3 * H + H * H, H, 1}};
    for (int f = 0; f < 2; ++f)
        for (const Seg& g : segs) {
            const double limit = std::sqrt(6.0 / (double)(g.fan_in + g.fan_out));
            for (int p = g.a; p < g.b; ++p) {
                const uint4 r = philox4x32_10(make_uint4((uint32_t)p, (uint32_t)f, kInitWord, 0u), (uint32_t)seed,
                                              (uint32_t)(seed >> 32));
                th[(size_t)f * kMlpStride + p] = (float)((2.0 * unit_open(r.x) - 1.0) * limit);
            }
        }
}

sdd_status ensure_node_features(sdd_ctx* c)
{
    const size_t n = (size_t)c->nx * c->ny;
    CU(c, c->cv_w64.alloc(n));
    CU(c, c->cv_r64.alloc(n));
    CU(c, c->cv_gw.alloc(n));
    CU(c, c->cv_nfa.alloc(n));
    CU(c, c->cv_nfb.alloc(n));
    CU(c, launch_node_features(c->w.p, c->nx, c->ny, c->cv_w64.p, c->cv_r64.p, c->cv_gw.p, c->cv_nfa.p, c->cv_nfb.p,
                               c->stream));
    return SDD_OK;
}

// Time left, as a fraction of Dt, at the middle sub-step of each slice.
void slice_fracs(int K, int S, float* out)
{
    for (int q = 0; q < S; ++q) {
        const int64_t b0 = ((int64_t)q * K + S - 1) / S, b1 = ((int64_t)(q + 1) * K + S - 1) / S;
        out[q] = (float)(((double)K - 0.5 * (double)(b0 + b1 - 1)) / (double)K);
    }
}

sdd_status cv_mode_buffers(sdd_ctx* c, int mode);

sdd_status set_table_from64(sdd_ctx* c, int slices)
{
    const size_t cells = (size_t)(c->nx - 1) * (c->ny - 1);
    CU(c, c->cvcoef.alloc(2 * cells * (size_t)slices));
    CU(c, launch_cv_cells(c->cv_table64.p, slices, c->nx, c->ny, c->cvcoef.p, c->stream));
    c->cv_slices = slices;
    CU(c, cudaStreamSynchronize(c->stream));
    // a mode that rebuilds its table per estimate keeps its own slice count
    if (c->cv_mode >= 2) return cv_mode_buffers(c, c->cv_mode);
    return upload_inst(c);
}

sdd_status train_loop(sdd_ctx* c, float* theta, const float* norm, const float* feats, const float* targets,
                      int64_t n, const sdd_train_params* p, float* losses, int64_t* steps_out)
{
    const int tile = mlp_tile_rows();
    if (p->epochs < 1 || p->batch < tile || p->batch % tile != 0 || p->batch > (1 << 24))
        return fail(c, SDD_EINVAL, "epochs must be >= 1 and batch a positive multiple of %d", tile);
    if (!(p->lr > 0.0) || !std::isfinite(p->lr)) return fail(c, SDD_EINVAL, "lr must be positive");
    const int64_t nb = n / p->batch;
    if (nb < 1) return fail(c, SDD_EINVAL, "fewer rows than one batch");
    int64_t total = (int64_t)p->epochs * nb;
    const int64_t run = p->max_steps > 0 ? std::min<int64_t>(p->max_steps, total) : total;
    const int nblk = p->batch / tile;
    CU(c, c->cv_m.alloc(2 * (size_t)kMlpStride));
    CU(c, c->cv_v.alloc(2 * (size_t)kMlpStride));
    CU(c, c->cv_part.alloc(2 * (size_t)nblk * kMlpStride));
    CU(c, cudaMemsetAsync(c->cv_m.p, 0, 2 * (size_t)kMlpStride * sizeof(float), c->stream));
    CU(c, cudaMemsetAsync(c->cv_v.p, 0, 2 * (size_t)kMlpStride * sizeof(float), c->stream));
    const float inv = 1.0f / (float)p->batch;
    for (int64_t t = 0; t < run; ++t) {
        const int64_t b = t % nb;
        const double lr = p->lr * 0.5 * (1.0 + std::cos(M_PI * (double)t / (double)total));
        CU(c, launch_mlp_grad(theta, norm, feats, targets, b * p->batch, p->batch, inv, c->cv_part.p, c->stream));
        CU(c, launch_mlp_adam(theta, c->cv_m.p, c->cv_v.p, c->cv_part.p, nblk, lr, t + 1, inv, losses, run, t,
                              c->stream));
    }
    if (steps_out) *steps_out = run;
    return SDD_OK;
}

sdd_status samples_into(sdd_ctx* c, const sdd_sample_params* p, float* feats, float* targets)
{
    int K = 0;
    if (!valid_params(c, p->dt, p->Dt, p->exit_mode, &K))
        return fail(c, SDD_EINVAL, "dt, Dt or exit_mode rejected (Dt / dt must be an integer in [1, 2^20])");
    const int64_t M = p->per_horizon;
    if (M < 1 || M * (int64_t)K > (int64_t)1 << 28)
        return fail(c, SDD_EINVAL, "per_horizon must be >= 1 and per_horizon * K <= 2^28");
    sdd_status st = prepare(c, c->stream);
    if (st != SDD_OK) return st;
    if ((st = ensure_node_features(c)) != SDD_OK) return st;
    CU(c, c->cv_sxy.alloc(2 * (size_t)M));
    CU(c, c->cv_smean[0].alloc((size_t)M));
    CU(c, c->cv_smean[1].alloc((size_t)M));
    std::vector<double> xs(M), ys(M);
    std::vector<int64_t> np(M, 1);
    OutDev out{};
    out.mean_xi = c->cv_smean[0].p;
    out.mean_eta = c->cv_smean[1].p;
    for (int k = 1; k <= K; ++k) {
        const uint32_t word0 = (uint32_t)((int64_t)(k - 1) * M);
        for (int64_t m = 0; m < M; ++m) {
            const uint4 r = philox4x32_10(make_uint4(1u, word0 + (uint32_t)m, 0u, kSampleStepWord), (uint32_t)p->seed,
                                          (uint32_t)(p->seed >> 32));
            xs[m] = unit_open(r.x);
            ys[m] = unit_open(r.y);
        }
        // the previous horizon's launch and scatter read the buffers refilled here
        CU(c, cudaStreamSynchronize(c->stream));
        std::vector<NodeSeg> segs(1);
        segs[0] = NodeSeg{xs.data(), ys.data(), np.data(), M, 0, word0};
        if ((st = build_plan_segs(&c->err, c->sm_count, c->sample_plan, segs, 0, 0, p->exit_mode, false)) != SDD_OK)
            return st;
        CU(c, cudaMemcpyAsync(c->cv_sxy.p, xs.data(), M * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        CU(c, cudaMemcpyAsync(c->cv_sxy.p + M, ys.data(), M * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        if ((st = run_plan_on(&c->err, c->sample_plan, c->d_inst.p, nullptr, out, p->dt, k, p->seed, kSampleStepWord,
                              nullptr, p->exit_mode, nullptr, c->stream, nullptr, nullptr, 0, nullptr, nullptr,
                              nullptr, ctx_zmap(c))) != SDD_OK)
            return st;
        CU(c, launch_cv_scatter(c->cv_sxy.p, c->cv_sxy.p + M, out.mean_xi, out.mean_eta, c->cv_nfa.p, c->nx, c->ny, k,
                                K, (int)M, feats, targets, c->stream));
    }
    CU(c, cudaStreamSynchronize(c->stream));
    return SDD_OK;
}

sdd_status tabulate_into_ctx(sdd_ctx* c, const float* theta, const float* norm, int slices, double dt, double Dt)
{
    int K = 0;
    if (!valid_params(c, dt, Dt, 0, &K)) return fail(c, SDD_EINVAL, "dt, Dt rejected");
    if (slices < 1 || slices > kMaxCvSlices || slices > K)
        return fail(c, SDD_EINVAL, "slices must be in [1, min(K, %d)]", kMaxCvSlices);
    sdd_status st = ensure_node_features(c);
    if (st != SDD_OK) return st;
    const size_t nn = (size_t)c->nx * c->ny;
    CU(c, c->cv_table64.alloc(4 * nn * (size_t)slices));
    float tf[kMaxCvSlices];
    slice_fracs(K, slices, tf);
    CU(c, launch_cv_tabulate(theta, norm, c->cv_nfa.p, c->cv_nfb.p, c->nx, c->ny, slices, tf, c->cv_table64.p,
                             c->d_status.p, c->sm_count, c->stream));
    if ((st = set_table_from64(c, slices)) != SDD_OK) return st;
    drop_graphs_fn(c);
    return SDD_OK;
}

// The binomial smoothing order of the field-gradient control variate: the one
// set, else by the grid: 2 floor((m - 1)^2 / 16384) - 1 for the larger side of
// m nodes, within 1..33 (129: 1, 257: 7, 513: 31, from 1025: 33). The
// interface values' Monte Carlo error leaves noise on the grid's scale in the
// fields' differences, which the filter removes; on finer grids the
// solution's own structure spans more cells, so the filter can be wider.
int cv_fields_order(const sdd_ctx* c)
{
    if (c->cv_order > 0) return c->cv_order;
    const double m = (double)std::max(c->nx, c->ny) - 1.0;
    const int o = 2 * (int)std::floor(m * m / 16384.0) - 1;
    return std::max(1, std::min(o, 33));
}

// Buffers of a control-variate mode, allocated before any capture.
sdd_status cv_mode_buffers(sdd_ctx* c, int mode)
{
    const size_t nn = (size_t)c->nx * c->ny, cells = (size_t)(c->nx - 1) * (c->ny - 1);
    const int slices = mode == 2 ? c->cv_model_slices : mode == 3 ? 1 : c->cv_slices;
    if (mode == 2) {
        const size_t n = (size_t)c->nx * c->ny;
        CU(c, c->cv_w64.alloc(n));
        CU(c, c->cv_r64.alloc(n));
        CU(c, c->cv_gw.alloc(n));
        CU(c, c->cv_nfa.alloc(n));
        CU(c, c->cv_nfb.alloc(n));
        CU(c, c->cv_table64.alloc(4 * nn * (size_t)slices));
        CU(c, c->cvcoef.alloc(2 * cells * (size_t)slices));
        c->cv_slices = slices;
        return upload_inst(c);
    }
    if (mode == 3) {
        CU(c, c->cv_table64.alloc(4 * nn));
        CU(c, c->cv_tmp.alloc((size_t)(c->nx - 1) * c->ny));
        CU(c, c->cv_cell.alloc(cells));
        c->cv_slices = 1;
        return upload_inst(c);
    }
    return SDD_OK;
}

// The per-estimate part of modes 2 and 3: the table from the current w (model)
// or the current fields (field gradient), then its cell records.
sdd_status enqueue_cv_refresh(sdd_ctx* c, int K, cudaStream_t s)
{
    if (c->cv_mode == 2) {
        if (c->cv_slices > K) return fail(c, SDD_EINVAL, "more control-variate slices than sub-steps per step");
        float tf[kMaxCvSlices];
        slice_fracs(K, c->cv_slices, tf);
        CU(c, launch_node_features(c->w.p, c->nx, c->ny, c->cv_w64.p, c->cv_r64.p, c->cv_gw.p, c->cv_nfa.p,
                                   c->cv_nfb.p, s));
        CU(c, launch_cv_tabulate(c->cv_theta.p, c->cv_norm.p, c->cv_nfa.p, c->cv_nfb.p, c->nx, c->ny, c->cv_slices,
                                 tf, c->cv_table64.p, c->d_status.p, c->sm_count, s));
        CU(c, launch_cv_cells(c->cv_table64.p, c->cv_slices, c->nx, c->ny, c->cvcoef.p, s));
    } else if (c->cv_mode == 3) {
        CU(c, launch_field_grad(c->fld[c->cur][0].p, c->fld[c->cur][1].p, c->nx, c->ny, c->cv_table64.p, s));
        CU(c, launch_cv_smooth(c->cv_table64.p, c->nx, c->ny, cv_fields_order(c), c->cv_tmp.p, c->cv_cell.p, s));
    }
    return SDD_OK;
}

OutDev out_from(const sdd_node_stats* o)
{
    OutDev d{};
    if (o) {
        d.mean_xi = o->mean_xi;
        d.mean_eta = o->mean_eta;
        d.se_xi = o->se_xi;
        d.se_eta = o->se_eta;
        d.n_exit = (long long*)o->n_exit;
        d.path_steps = (long long*)o->path_steps;
    }
    return d;
}

}  // namespace

extern "C" {

sdd_status sdd_init(sdd_ctx** out, const sdd_grid* g, const float* w, const double* xi0, const double* eta0,
                    void* stream)
{
    if (!out || !g) return SDD_EINVAL;
    *out = nullptr;
    if (g->nx < 3 || g->ny < 3 || g->nx > 32768 || g->ny > 32768) return SDD_EINVAL;
    if (g->sub_x < 1 || g->sub_y < 1 || g->sub_x > g->nx - 1 || g->sub_y > g->ny - 1) return SDD_EINVAL;
    if ((long long)g->nx * g->ny > (1LL << 30)) return SDD_EINVAL;
    sdd_ctx* c = new (std::nothrow) sdd_ctx();
    if (!c) return SDD_ENOMEM;
    c->nx = g->nx;
    c->ny = g->ny;
    c->sub_x = g->sub_x;
    c->sub_y = g->sub_y;
    c->stream = (cudaStream_t)stream;
    sdd_status st = SDD_OK;
    auto bail = [&](sdd_status s) {
        sdd_destroy(c);
        return s;
    };
#define INIT_CU(expr)                                                             \
    do {                                                                          \
        cudaError_t e_ = (expr);                                                  \
        if (e_ != cudaSuccess)                                                    \
            return bail(e_ == cudaErrorMemoryAllocation ? SDD_ENOMEM : SDD_ECUDA); \
    } while (0)
    INIT_CU(cudaGetDevice(&c->device));
    INIT_CU(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device));
    INIT_CU(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    for (int k = 0; k < 5; ++k) INIT_CU(cudaEventCreate(&c->ev[k]));
    const size_t N = (size_t)c->nx * c->ny;
    const size_t cells = (size_t)(c->nx - 1) * (c->ny - 1);
    INIT_CU(c->w.alloc(N));
    for (int b = 0; b < 2; ++b)
        for (int f = 0; f < 2; ++f) INIT_CU(c->fld[b][f].alloc(N));
    INIT_CU(c->faces64.alloc(faces_len(c)));
    INIT_CU(c->faces32.alloc(faces_len(c)));
    INIT_CU(c->bcoef.alloc(2 * (cells + 1)));
    INIT_CU(cudaMemset(c->bcoef.p + 2 * cells, 0, 2 * sizeof(float4)));   // the all-zero record
    c->zshift = zmap_shift((long long)cells);
    c->zwords = zmap_words((long long)cells, c->zshift);
    INIT_CU(c->zmap.alloc(c->zwords));
    INIT_CU(c->fcoef.alloc(2 * cells));
    INIT_CU(c->d_status.alloc(1));
    INIT_CU(c->d_step.alloc(1));
    INIT_CU(cudaMemset(c->d_status.p, 0, sizeof(int)));
    INIT_CU(cudaMemset(c->d_step.p, 0, sizeof(uint32_t)));
    // inputs (defaults: w = 1, xi = x, eta = y)
    {
        std::vector<float> hw;
        std::vector<double> hx, hy;
        if (!w) hw.assign(N, 1.0f);
        if (!xi0 || !eta0) {
            hx.resize(N);
            hy.resize(N);
            for (int j = 0; j < c->ny; ++j)
                for (int i = 0; i < c->nx; ++i) {
                    hx[(size_t)j * c->nx + i] = (double)i / (c->nx - 1);
                    hy[(size_t)j * c->nx + i] = (double)j / (c->ny - 1);
                }
        }
        INIT_CU(cudaMemcpy(c->w.p, w ? (const void*)w : (const void*)hw.data(), N * sizeof(float),
                           w ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
        INIT_CU(cudaMemcpy(c->fld[0][0].p, xi0 ? (const void*)xi0 : (const void*)hx.data(), N * sizeof(double),
                           xi0 ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
        INIT_CU(cudaMemcpy(c->fld[0][1].p, eta0 ? (const void*)eta0 : (const void*)hy.data(), N * sizeof(double),
                           eta0 ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
    }
    if ((st = upload_inst(c)) != SDD_OK) return bail(st);
    if ((st = setup_solver(c)) != SDD_OK) return bail(st);
    build_interface(c);
    INIT_CU(c->d_iface_idx.alloc(std::max<size_t>(c->iface_idx.size(), 1)));
    if (!c->iface_idx.empty())
        INIT_CU(cudaMemcpy(c->d_iface_idx.p, c->iface_idx.data(), c->iface_idx.size() * sizeof(int32_t),
                           cudaMemcpyHostToDevice));
    INIT_CU(c->d_klines.alloc(std::max<size_t>(c->klines.size(), 1)));
    INIT_CU(c->d_kpos_idx.alloc(std::max<size_t>(c->kpos_idx.size(), 1)));
    INIT_CU(c->d_kpos_cross.alloc(std::max<size_t>(c->kpos_cross.size(), 1)));
    INIT_CU(c->d_kmask.alloc(std::max<size_t>(c->iface_idx.size(), 1)));
    INIT_CU(c->d_kscratch.alloc(pchip_scratch_doubles((long long)c->kpos_idx.size(), (int)c->klines.size())));
    if (!c->klines.empty()) {
        INIT_CU(cudaMemcpy(c->d_klines.p, c->klines.data(), c->klines.size() * sizeof(KeyLine), cudaMemcpyHostToDevice));
        INIT_CU(cudaMemcpy(c->d_kpos_idx.p, c->kpos_idx.data(), c->kpos_idx.size() * sizeof(int32_t),
                           cudaMemcpyHostToDevice));
        INIT_CU(cudaMemcpy(c->d_kpos_cross.p, c->kpos_cross.data(), c->kpos_cross.size(), cudaMemcpyHostToDevice));
    }
    for (int k = 0; k < 4; ++k) INIT_CU(c->iface_stats[k].alloc(std::max<size_t>(c->iface_idx.size(), 1)));
    for (int k = 0; k < 2; ++k) INIT_CU(c->iface_counts[k].alloc(std::max<size_t>(c->iface_idx.size(), 1)));
    c->dirty_w = c->dirty_fields = true;
    if ((st = prepare(c, c->stream)) != SDD_OK) return bail(st);
    INIT_CU(cudaStreamSynchronize(c->stream));
#undef INIT_CU
    *out = c;
    return SDD_OK;
}

static void drop_graphs(sdd_ctx* c) { drop_graphs_fn(c); }

sdd_status sdd_set_w(sdd_ctx* c, const float* w)
{
    if (!c || !w) return fail(c, SDD_EINVAL, "null argument");
    CU(c, cudaMemcpyAsync(c->w.p, w, (size_t)c->nx * c->ny * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
    c->dirty_w = true;
    return SDD_OK;
}

sdd_status sdd_set_w_host(sdd_ctx* c, const float* w)
{
    if (!c || !w) return fail(c, SDD_EINVAL, "null argument");
    CU(c, cudaMemcpyAsync(c->w.p, w, (size_t)c->nx * c->ny * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    c->dirty_w = true;
    return SDD_OK;
}

sdd_status sdd_set_fields(sdd_ctx* c, const double* xi, const double* eta)
{
    if (!c || !xi || !eta) return fail(c, SDD_EINVAL, "null argument");
    {
        const sdd_status fs = flush_pending(c);
        if (fs != SDD_OK) return fs;
    }
    const size_t bytes = (size_t)c->nx * c->ny * sizeof(double);
    CU(c, cudaMemcpyAsync(c->fld[c->cur][0].p, xi, bytes, cudaMemcpyDeviceToDevice, c->stream));
    CU(c, cudaMemcpyAsync(c->fld[c->cur][1].p, eta, bytes, cudaMemcpyDeviceToDevice, c->stream));
    c->dirty_fields = true;
    return SDD_OK;
}

sdd_status sdd_set_boundary(sdd_ctx* c, const double* faces)
{
    if (!c) return SDD_EINVAL;
    if (faces) {
        CU(c, cudaMemcpyAsync(c->faces64.p, faces, faces_len(c) * sizeof(double), cudaMemcpyDeviceToDevice,
                              c->stream));
        CU(c, launch_faces32(c->faces64.p, c->faces32.p, (int)faces_len(c), c->stream));
        c->user_faces = true;
    } else {
        c->user_faces = false;
        c->dirty_w = true;  // recompute the paper's data from w
    }
    drop_graphs(c);
    return SDD_OK;
}

sdd_status sdd_get_faces(sdd_ctx* c, double* faces)
{
    if (!c || !faces) return fail(c, SDD_EINVAL, "null argument");
    sdd_status st = prepare(c, c->stream);
    if (st != SDD_OK) return st;
    CU(c, cudaMemcpyAsync(faces, c->faces64.p, faces_len(c) * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    return SDD_OK;
}

sdd_status sdd_get_fields(sdd_ctx* c, double* xi, double* eta)
{
    if (!c || !xi || !eta) return fail(c, SDD_EINVAL, "null argument");
    {
        const sdd_status fs = flush_pending(c);
        if (fs != SDD_OK) return fs;
    }
    const size_t bytes = (size_t)c->nx * c->ny * sizeof(double);
    CU(c, cudaMemcpyAsync(xi, c->fld[c->cur][0].p, bytes, cudaMemcpyDefault, c->stream));
    CU(c, cudaMemcpyAsync(eta, c->fld[c->cur][1].p, bytes, cudaMemcpyDefault, c->stream));
    return SDD_OK;
}

sdd_status sdd_get_fields_host(sdd_ctx* c, double* xi, double* eta)
{
    sdd_status st = sdd_get_fields(c, xi, eta);
    if (st != SDD_OK) return st;
    CU(c, cudaStreamSynchronize(c->stream));
    return SDD_OK;
}

static sdd_status mc_common(sdd_ctx* c, const sdd_nodes* nodes, const sdd_mc_params* p, sdd_node_stats* out,
                            const sdd_path_records* rec)
{
    if (!c || !nodes || !p) return fail(c, SDD_EINVAL, "null argument");
    {
        const sdd_status fs = flush_pending(c);
        if (fs != SDD_OK) return fs;
    }
    if (nodes->count > 0 && (!nodes->x || !nodes->y || !nodes->n_paths)) return fail(c, SDD_EINVAL, "null node array");
    int K = 0;
    if (!valid_params(c, p->dt, p->Dt, p->exit_mode, &K))
        return fail(c, SDD_EINVAL, "dt, Dt or exit_mode rejected (Dt / dt must be an integer in [1, 2^20])");
    if (p->zero_map < 0 || p->zero_map > 2) return fail(c, SDD_EINVAL, "zero_map must be 0, 1 or 2");
    int ppt = p->paths_per_task, block = p->block_threads, zmap = p->zero_map;
    {
        std::vector<NodeSeg> segs(1);
        segs[0] = NodeSeg{nodes->x, nodes->y, nodes->n_paths, nodes->count, 0, p->node_word0};
        pick_shape(c->tuned, segs, K, p->exit_mode, &ppt, &block, &zmap);
    }
    sdd_status st = build_plan(c, c->mc_plan, nodes->x, nodes->y, nodes->n_paths, nodes->count, ppt, block,
                               p->exit_mode, rec != nullptr, p->node_word0);
    if (st != SDD_OK) return st;
    c->mc_plan.zero_map = zmap;
    c->mc_plan.zero_map_auto = p->zero_map == 0;
    if ((st = prepare(c, c->stream)) != SDD_OK) return st;
    if ((st = enqueue_cv_refresh(c, K, c->stream)) != SDD_OK) return st;
    RecDev rd{};
    if (rec) {
        rd.steps = rec->steps;
        rd.code = rec->code;
        rd.score_xi = rec->score_xi;
        rd.score_eta = rec->score_eta;
        rd.x_end = rec->x_end;
        rd.y_end = rec->y_end;
    }
    return run_plan(c, c->mc_plan, p->dt, K, p->seed, p->step_index, nullptr, p->exit_mode, out_from(out),
                    rec ? &rd : nullptr, c->stream);
}

sdd_status sdd_interface_mc(sdd_ctx* c, const sdd_nodes* nodes, const sdd_mc_params* p, sdd_node_stats* out)
{
    return mc_common(c, nodes, p, out, nullptr);
}

sdd_status sdd_interface_mc_record(sdd_ctx* c, const sdd_nodes* nodes, const sdd_mc_params* p, sdd_node_stats* out,
                                   const sdd_path_records* rec)
{
    if (!rec) return fail(c, SDD_EINVAL, "null records");
    return mc_common(c, nodes, p, out, rec);
}

sdd_status sdd_set_keypoints(sdd_ctx* c, int32_t on, int32_t spacing)
{
    if (!c) return SDD_EINVAL;
    if (spacing < 0) return fail(c, SDD_EINVAL, "spacing must be >= 0");
    if ((on != 0) != (c->keypoints != 0) || spacing != c->key_spacing) drop_graphs(c);
    c->keypoints = on != 0;
    c->key_spacing = spacing;
    return SDD_OK;
}

sdd_status sdd_keypoint_mask(sdd_ctx* c, uint8_t* mask)
{
    if (!c || !mask) return fail(c, SDD_EINVAL, "null argument");
    return enqueue_keypoints(c, mask, c->stream);
}

sdd_status sdd_keypoint_fill(sdd_ctx* c, const uint8_t* mask, double* values_xi, double* values_eta)
{
    if (!c || !mask || !values_xi || !values_eta) return fail(c, SDD_EINVAL, "null argument");
    // the line ends are the face data of the current w
    sdd_status st = prepare_parts(c, c->stream, true, false);
    if (st != SDD_OK) return st;
    CU(c, launch_pchip(c->d_klines.p, (int)c->klines.size(), c->kmax_n, c->d_kpos_idx.p, c->d_kpos_cross.p, mask,
                       c->faces64.p, c->nx, c->ny, values_xi, values_eta, c->d_kscratch.p, c->stream));
    return SDD_OK;
}

sdd_status sdd_set_solver(sdd_ctx* c, int32_t solver)
{
    if (!c) return SDD_EINVAL;
    if (solver < 0 || solver > 3) return fail(c, SDD_EINVAL, "solver must be 0, 1, 2 or 3");
    if (solver == 2 && !c->mg_ok)
        return fail(c, SDD_EINVAL, "multigrid needs subdomains of one size, odd, coarsening to at most 64 unknowns");
    if (solver == 3 && !c->chol_ok)
        return fail(c, SDD_EINVAL, "the direct solve needs subdomains of at most 32 columns whose band fits 200 KB");
    if (solver != c->solver) drop_graphs(c);
    c->solver = solver;
    return SDD_OK;
}

int32_t sdd_solver_in_use(const sdd_ctx* c)
{
    if (!c) return -1;
    return solver_choice(c);
}

sdd_status sdd_cv_set_table(sdd_ctx* c, const double* grad, int32_t slices)
{
    if (!c || !grad) return fail(c, SDD_EINVAL, "null argument");
    if (slices < 1 || slices > kMaxCvSlices) return fail(c, SDD_EINVAL, "slices must be in [1, %d]", kMaxCvSlices);
    const size_t n = 4 * (size_t)c->nx * c->ny * (size_t)slices;
    CU(c, c->cv_table64.alloc(n));
    CU(c, cudaMemcpyAsync(c->cv_table64.p, grad, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    sdd_status st = set_table_from64(c, slices);
    if (st != SDD_OK) return st;
    drop_graphs(c);
    return SDD_OK;
}

sdd_status sdd_cv_get_table(sdd_ctx* c, double* grad)
{
    if (!c || !grad) return fail(c, SDD_EINVAL, "null argument");
    if (c->cv_slices < 1) return fail(c, SDD_EINVAL, "no control-variate table has been set");
    const size_t n = 4 * (size_t)c->nx * c->ny * (size_t)c->cv_slices;
    CU(c, cudaMemcpyAsync(grad, c->cv_table64.p, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    return SDD_OK;
}

sdd_status sdd_cv_set_fields_order(sdd_ctx* c, int32_t order)
{
    if (!c) return SDD_EINVAL;
    if (order != 0 && (order < 1 || order > kCvMaxOrder || (order & 1) == 0))
        return fail(c, SDD_EINVAL, "the smoothing order must be 0 or odd in 1..%d", kCvMaxOrder);
    if (order != c->cv_order) drop_graphs(c);
    c->cv_order = order;
    return SDD_OK;
}

int32_t sdd_cv_fields_order(const sdd_ctx* c) { return c ? cv_fields_order(c) : 0; }

sdd_status sdd_cv_get_cells(sdd_ctx* c, float* cells)
{
    if (!c || !cells) return fail(c, SDD_EINVAL, "null argument");
    if (c->cv_mode != 3) return fail(c, SDD_EINVAL, "the field-gradient control variate is not enabled");
    {
        const sdd_status fs = flush_pending(c);
        if (fs != SDD_OK) return fs;
    }
    CU(c, launch_field_grad(c->fld[c->cur][0].p, c->fld[c->cur][1].p, c->nx, c->ny, c->cv_table64.p, c->stream));
    CU(c, launch_cv_smooth(c->cv_table64.p, c->nx, c->ny, cv_fields_order(c), c->cv_tmp.p, c->cv_cell.p, c->stream));
    CU(c, cudaMemcpyAsync(cells, c->cv_cell.p, 4 * sizeof(float) * (size_t)(c->nx - 1) * (c->ny - 1),
                          cudaMemcpyDeviceToDevice, c->stream));
    return SDD_OK;
}

sdd_status sdd_cv_enable(sdd_ctx* c, int32_t mode)
{
    if (!c) return SDD_EINVAL;
    if (mode < 0 || mode > 3) return fail(c, SDD_EINVAL, "control-variate mode must be 0..3");
    if (mode == 1 && c->cv_slices < 1) return fail(c, SDD_EINVAL, "no control-variate table has been set");
    if (mode == 2 && !c->cv_model) return fail(c, SDD_EINVAL, "no control-variate model has been trained or set");
    sdd_status st = cv_mode_buffers(c, mode);
    if (st != SDD_OK) return st;
    if (mode != c->cv_mode) drop_graphs(c);
    c->cv_mode = mode;
    return SDD_OK;
}

sdd_status sdd_mlp_init(sdd_ctx* c, uint64_t seed, float* theta)
{
    if (!c || !theta) return fail(c, SDD_EINVAL, "null argument");
    std::vector<float> th;
    init_params_host(seed, th);
    CU(c, cudaMemcpyAsync(theta, th.data(), th.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    CU(c, cudaStreamSynchronize(c->stream));
    return SDD_OK;
}

sdd_status sdd_cv_samples(sdd_ctx* c, const sdd_sample_params* p, float* feats, float* targets)
{
    if (!c || !p || !feats || !targets) return fail(c, SDD_EINVAL, "null argument");
    {
        const sdd_status fs = flush_pending(c);
        if (fs != SDD_OK) return fs;
    }
    return samples_into(c, p, feats, targets);
}

sdd_status sdd_mlp_norm(sdd_ctx* c, const float* feats, int64_t n, float* norm)
{
    if (!c || !feats || !norm) return fail(c, SDD_EINVAL, "null argument");
    if (n < 1) return fail(c, SDD_EINVAL, "no rows");
    CU(c, c->cv_norm_scratch.alloc(mlp_norm_scratch_doubles()));
    CU(c, launch_mlp_norm(feats, n, c->cv_norm_scratch.p, norm, c->stream));
    return SDD_OK;
}

sdd_status sdd_mlp_grad(sdd_ctx* c, const float* theta, const float* norm, const float* feats, const float* targets,
                        int64_t rows, float* grad, float* loss)
{
    if (!c || !theta || !norm || !feats || !targets || !grad) return fail(c, SDD_EINVAL, "null argument");
    const int tile = mlp_tile_rows();
    if (rows < tile || rows % tile != 0 || rows > (1LL << 28))
        return fail(c, SDD_EINVAL, "rows must be a positive multiple of %d", tile);
    const int nblk = (int)(rows / tile);
    CU(c, c->cv_grad_part.alloc(2 * (size_t)nblk * kMlpStride));
    const float inv = (float)(1.0 / (double)rows);
    CU(c, launch_mlp_grad(theta, norm, feats, targets, 0, rows, inv, c->cv_grad_part.p, c->stream));
    CU(c, launch_mlp_reduce(c->cv_grad_part.p, nblk, inv, grad, loss, c->stream));
    return SDD_OK;
}

sdd_status sdd_mlp_train(sdd_ctx* c, float* theta, const float* norm, const float* feats, const float* targets,
                         int64_t n, const sdd_train_params* p, float* losses)
{
    if (!c || !theta || !norm || !feats || !targets || !p) return fail(c, SDD_EINVAL, "null argument");
    return train_loop(c, theta, norm, feats, targets, n, p, losses, nullptr);
}

sdd_status sdd_cv_tabulate(sdd_ctx* c, const float* theta, const float* norm, int32_t slices, double dt, double Dt)
{
    if (!c || !theta || !norm) return fail(c, SDD_EINVAL, "null argument");
    return tabulate_into_ctx(c, theta, norm, slices, dt, Dt);
}

sdd_status sdd_cv_train(sdd_ctx* c, const sdd_cv_train_params* p, sdd_cv_train_info* info)
{
    if (!c || !p) return fail(c, SDD_EINVAL, "null argument");
    {
        const sdd_status fs = flush_pending(c);
        if (fs != SDD_OK) return fs;
    }
    int K = 0;
    if (!valid_params(c, p->samples.dt, p->samples.Dt, p->samples.exit_mode, &K))
        return fail(c, SDD_EINVAL, "dt, Dt or exit_mode rejected");
    const int slices = p->slices > 0 ? p->slices : std::min(K, kMaxCvSlices);
    if (slices > K || slices > kMaxCvSlices) return fail(c, SDD_EINVAL, "slices must be in [1, min(K, %d)]", kMaxCvSlices);
    const int64_t n = (int64_t)p->samples.per_horizon * K;
    if (p->samples.per_horizon < 1 || n > (1LL << 28)) return fail(c, SDD_EINVAL, "per_horizon out of range");
    if (n < p->train.batch) return fail(c, SDD_EINVAL, "fewer training rows than one batch");
    cudaEvent_t ev[4] = {};
    for (auto& e : ev) CU(c, cudaEventCreate(&e));
    struct Guard {
        cudaEvent_t* e;
        ~Guard() { for (int k = 0; k < 4; ++k) if (e[k]) cudaEventDestroy(e[k]); }
    } guard{ev};
    CU(c, c->cv_feats.alloc((size_t)n * kMlpInputs));
    CU(c, c->cv_targets.alloc((size_t)n * 2));
    CU(c, c->cv_theta.alloc(2 * (size_t)kMlpStride));
    CU(c, c->cv_norm.alloc(16));
    CU(c, cudaEventRecord(ev[0], c->stream));
    sdd_status st = samples_into(c, &p->samples, c->cv_feats.p, c->cv_targets.p);
    if (st != SDD_OK) return st;
    CU(c, cudaEventRecord(ev[1], c->stream));
    if (!(p->warm_start && c->cv_model)) {
        std::vector<float> th;
        init_params_host(p->init_seed, th);
        CU(c, cudaMemcpyAsync(c->cv_theta.p, th.data(), th.size() * sizeof(float), cudaMemcpyHostToDevice,
                              c->stream));
        CU(c, cudaStreamSynchronize(c->stream));
        CU(c, c->cv_norm_scratch.alloc(mlp_norm_scratch_doubles()));
        CU(c, launch_mlp_norm(c->cv_feats.p, n, c->cv_norm_scratch.p, c->cv_norm.p, c->stream));
    }
    int64_t steps = 0;
    const int64_t nb = n / p->train.batch;
    const int64_t planned = (int64_t)p->train.epochs * nb;
    const int64_t run = p->train.max_steps > 0 ? std::min<int64_t>(p->train.max_steps, planned) : planned;
    CU(c, c->cv_losses.alloc(2 * (size_t)std::max<int64_t>(run, 1)));
    if ((st = train_loop(c, c->cv_theta.p, c->cv_norm.p, c->cv_feats.p, c->cv_targets.p, n, &p->train,
                         c->cv_losses.p, &steps)) != SDD_OK)
        return st;
    CU(c, cudaEventRecord(ev[2], c->stream));
    c->cv_model = true;
    c->cv_model_slices = slices;
    c->cv_rows = n;
    c->cv_loss_steps = steps;
    if ((st = tabulate_into_ctx(c, c->cv_theta.p, c->cv_norm.p, slices, p->samples.dt, p->samples.Dt)) != SDD_OK)
        return st;
    CU(c, cudaEventRecord(ev[3], c->stream));
    CU(c, cudaEventSynchronize(ev[3]));
    if (info) {
        std::memset(info, 0, sizeof *info);
        CU(c, cudaEventElapsedTime(&info->samples_ms, ev[0], ev[1]));
        CU(c, cudaEventElapsedTime(&info->train_ms, ev[1], ev[2]));
        CU(c, cudaEventElapsedTime(&info->tabulate_ms, ev[2], ev[3]));
        info->rows = n;
        info->steps = steps;
        info->slices = slices;
        if (steps > 0) {
            float l[2];
            CU(c, cudaMemcpy(&l[0], c->cv_losses.p + (steps - 1), sizeof(float), cudaMemcpyDeviceToHost));
            CU(c, cudaMemcpy(&l[1], c->cv_losses.p + steps + (steps - 1), sizeof(float), cudaMemcpyDeviceToHost));
            info->loss_xi = l[0];
            info->loss_eta = l[1];
        }
    }
    return SDD_OK;
}

sdd_status sdd_cv_set_model(sdd_ctx* c, const float* theta, const float* norm, int32_t slices)
{
    if (!c || !theta || !norm) return fail(c, SDD_EINVAL, "null argument");
    if (slices < 1 || slices > kMaxCvSlices) return fail(c, SDD_EINVAL, "slices must be in [1, %d]", kMaxCvSlices);
    CU(c, c->cv_theta.alloc(2 * (size_t)kMlpStride));
    CU(c, c->cv_norm.alloc(16));
    CU(c, cudaMemcpyAsync(c->cv_theta.p, theta, 2 * (size_t)kMlpStride * sizeof(float), cudaMemcpyDeviceToDevice,
                          c->stream));
    CU(c, cudaMemcpyAsync(c->cv_norm.p, norm, 2 * kMlpInputs * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
    c->cv_model = true;
    c->cv_model_slices = slices;
    if (c->cv_mode == 2) {
        sdd_status st = cv_mode_buffers(c, 2);
        if (st != SDD_OK) return st;
        drop_graphs(c);
    }
    return SDD_OK;
}

sdd_status sdd_cv_get_model(sdd_ctx* c, float* theta, float* norm)
{
    if (!c) return SDD_EINVAL;
    if (!c->cv_model) return fail(c, SDD_EINVAL, "no trained model");
    if (theta)
        CU(c, cudaMemcpyAsync(theta, c->cv_theta.p, 2 * (size_t)kMlpStride * sizeof(float), cudaMemcpyDeviceToDevice,
                              c->stream));
    if (norm) CU(c, cudaMemcpyAsync(norm, c->cv_norm.p, 2 * kMlpInputs * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
    return SDD_OK;
}

sdd_status sdd_cv_losses(sdd_ctx* c, float* losses, int64_t count)
{
    if (!c || !losses) return fail(c, SDD_EINVAL, "null argument");
    if (!c->cv_model) return fail(c, SDD_EINVAL, "no trained model");
    const int64_t have = c->cv_loss_steps;
    if (count < 0 || count > have) return fail(c, SDD_EINVAL, "count exceeds the recorded steps");
    CU(c, cudaMemcpyAsync(losses, c->cv_losses.p, (size_t)count * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
    CU(c, cudaMemcpyAsync(losses + count, c->cv_losses.p + have, (size_t)count * sizeof(float),
                          cudaMemcpyDeviceToDevice, c->stream));
    return SDD_OK;
}

sdd_status sdd_autotune(sdd_ctx* c, const sdd_nodes* nodes, const sdd_mc_params* p, sdd_launch_shape* out)
{
    if (!c || !nodes || !p) return fail(c, SDD_EINVAL, "null argument");
    {
        const sdd_status fs = flush_pending(c);
        if (fs != SDD_OK) return fs;
    }
    if (nodes->count > 0 && (!nodes->x || !nodes->y || !nodes->n_paths)) return fail(c, SDD_EINVAL, "null node array");
    int K = 0;
    if (!valid_params(c, p->dt, p->Dt, p->exit_mode, &K)) return fail(c, SDD_EINVAL, "dt, Dt or exit_mode rejected");
    sdd_status st = prepare(c, c->stream);
    if (st != SDD_OK) return st;
    std::vector<NodeSeg> segs(1);
    segs[0] = NodeSeg{nodes->x, nodes->y, nodes->n_paths, nodes->count, 0, p->node_word0};
    TunedShape best{};
    st = autotune_plan(&c->err, c->sm_count, segs, c->d_inst.p, 1, K, p->dt, p->exit_mode, c->stream, c->tuned, &best,
                       ctx_zmap(c));
    if (st != SDD_OK) return st;
    if (out) {
        out->block_threads = best.block;
        out->paths_per_task = best.ppt;
        out->ms = best.ms;
        out->zero_map = best.zero_map ? 1 : 2;
    }
    return SDD_OK;
}

sdd_status sdd_interface_nodes(sdd_ctx* c, double* x, double* y, int64_t* count)
{
    if (!c || !count) return fail(c, SDD_EINVAL, "null argument");
    *count = (int64_t)c->iface_x.size();
    if (x) std::memcpy(x, c->iface_x.data(), c->iface_x.size() * sizeof(double));
    if (y) std::memcpy(y, c->iface_y.data(), c->iface_y.size() * sizeof(double));
    return SDD_OK;
}

sdd_status sdd_subdomain_solve(sdd_ctx* c, double Dt, const double* iface_xi, const double* iface_eta, double rtol,
                               int32_t max_iter, double* xi_out, double* eta_out, int32_t* iters_out)
{
    if (!c || !xi_out || !eta_out) return fail(c, SDD_EINVAL, "null argument");
    {
        const sdd_status fs = flush_pending(c);
        if (fs != SDD_OK) return fs;
    }
    if (!c->iface_idx.empty() && (!iface_xi || !iface_eta)) return fail(c, SDD_EINVAL, "null interface values");
    if (!(Dt > 0.0) || !(rtol >= 0.0) || max_iter < 0) return fail(c, SDD_EINVAL, "Dt, rtol or max_iter rejected");
    sdd_status st = prepare(c, c->stream);
    if (st != SDD_OK) return st;
    if ((st = enqueue_solve(c, Dt, iface_xi, iface_eta, rtol, max_iter, xi_out, eta_out, c->stream)) != SDD_OK)
        return st;
    if (iters_out) {
        const size_t ns = c->solve_nsys_used;
        std::vector<int32_t> it(std::max<size_t>(ns, 1), 0);
        CU(c, cudaMemcpyAsync(it.data(), c->d_iters.p, ns * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
        CU(c, cudaStreamSynchronize(c->stream));
        int32_t mx = 0;
        for (size_t k = 0; k < ns; ++k) mx = std::max(mx, it[k]);
        *iters_out = mx;
        if (mx > max_iter) return fail(c, SDD_ENOCONV, "subdomain solve did not reach rtol in max_iter iterations");
    }
    return SDD_OK;
}

// Record one mesh step into a graph on the capture stream: field tables, the
// interface estimate, the Dirichlet data, the subdomain solve and the step
// counter. Pipelined (c->pipe), a second branch beside the drift records, key
// points and paths runs the previous step's solve iterations (with_pending),
// the field records and this step's systems (from w and the fields of the
// step's start); the survivors are scored after the field records, and this
// step's iterations are left for the next step's graph (or sdd_flush).
static sdd_status capture_step(sdd_ctx* c, const sdd_step_params* p, int K, int parity, bool with_pending)
{
    cudaStream_t s = c->cap_stream;
    cudaGraph_t g = nullptr;
    CU(c, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    // the graph always recomputes the tables: w and the fields change every step
    const bool keep_w = c->dirty_w, keep_f = c->dirty_fields;
    c->dirty_w = true;
    c->dirty_fields = true;
    const int saved = c->cur;
    c->cur = parity;
    sdd_status st = SDD_OK;
    auto rec_ext = [&](cudaEvent_t e, cudaStream_t on) {
        if (st != SDD_OK) return;
        cudaError_t r = cudaEventRecordWithFlags(e, on, cudaEventRecordExternal);
        if (r != cudaSuccess) st = fail(c, SDD_ECUDA, "event: %s", cudaGetErrorString(r));
    };
    auto cu = [&](cudaError_t r) {
        if (st == SDD_OK && r != cudaSuccess) st = fail(c, SDD_ECUDA, "%s", cudaGetErrorString(r));
    };
    rec_ext(c->ev[0], s);
    // pipelined, the cluster solve takes half the SMs (four unknowns per thread): it runs beside the paths
    c->step_call[parity] = make_solve_call(c, p->Dt, p->rtol, p->max_iter, c->fld[1 - parity][0].p,
                                           c->fld[1 - parity][1].p, c->w.p, c->fld[parity][0].p,
                                           c->fld[parity][1].p, c->pipe);
    cudaEvent_t join = nullptr;
    if (c->pipe && !c->user_faces) {
        // the face data (one small block's prefix sums) on a third branch, beside the drift records
        cu(cudaEventRecord(c->fev[0], s));
        cu(cudaStreamWaitEvent(c->faces_stream, c->fev[0], 0));
        cu(launch_winslow_faces(c->w.p, c->nx, c->ny, c->faces64.p, c->faces32.p, c->faces_stream));
        cu(cudaEventRecord(c->fev[1], c->faces_stream));
    }
    if (c->pipe) {
        cudaStream_t q = c->pipe_stream;
        cu(cudaEventRecord(c->pev[0], s));
        cu(cudaStreamWaitEvent(q, c->pev[0], 0));
        if (with_pending) {
            // the previous step's iterations write this step's fields
            rec_ext(c->pev[2], q);
            if (st == SDD_OK) st = enqueue_solve_iterate(c, c->step_call[1 - parity], q);
            rec_ext(c->pev[3], q);
        }
        if (st == SDD_OK) st = prepare_parts(c, q, false, true);
        // with the plain test the path kernel reads no face data (its exits are scored later):
        // the face data join the main branch here, before the scoring
        if (!c->user_faces && p->exit_mode == 0) cu(cudaStreamWaitEvent(q, c->fev[1], 0));
        cu(cudaEventRecord(c->pev[1], q));
        join = c->pev[1];
        if (st == SDD_OK) st = enqueue_solve_system(c, c->step_call[parity], q);
        // the new fields' faces and interior start (this step's face data, made on the third branch)
        if (!c->user_faces) cu(cudaStreamWaitEvent(q, c->fev[1], 0));
        const SolveCall& k = c->step_call[parity];
        cu(launch_dirichlet_faces(c->faces64.p, k.px, k.pe, c->nx, c->ny, k.a.x[0], k.a.x[1], q));
        cu(cudaEventRecord(c->pev[4], q));
    }
    if (st == SDD_OK && c->pipe) {
        // the drift records; the face data come from the third branch forked above
        cu(launch_prep_cells(c->w.p, nullptr, nullptr, c->nx, c->ny, c->bcoef.p, nullptr, c->d_status.p, s, c->zmap.p,
                             c->zshift));
        if (!c->user_faces && p->exit_mode != 0) cu(cudaStreamWaitEvent(s, c->fev[1], 0));
        c->dirty_w = false;
    } else if (st == SDD_OK) {
        st = prepare(c, s);
    }
    if (st == SDD_OK) st = enqueue_cv_refresh(c, K, s);
    OutDev o{};
    o.mean_xi = c->iface_stats[0].p;
    o.mean_eta = c->iface_stats[1].p;
    o.se_xi = c->iface_stats[2].p;
    o.se_eta = c->iface_stats[3].p;
    o.n_exit = c->iface_counts[0].p;
    o.path_steps = c->iface_counts[1].p;
    const uint8_t* kmask = c->keypoints ? c->d_kmask.p : nullptr;
    if (st == SDD_OK && kmask) st = enqueue_keypoints(c, c->d_kmask.p, s);
    if (st == SDD_OK)
        st = run_plan(c, c->step_plan, p->dt, K, p->seed, 0, c->d_step.p, p->exit_mode, o, nullptr, s, c->ev[1],
                      c->ev[2], kmask, c->defer ? (void*)c->surv.p : nullptr, join);
    if (st == SDD_OK && kmask) {
        cudaError_t e = launch_pchip(c->d_klines.p, (int)c->klines.size(), c->kmax_n, c->d_kpos_idx.p,
                                     c->d_kpos_cross.p, kmask, c->faces64.p, c->nx, c->ny, o.mean_xi, o.mean_eta,
                                     c->d_kscratch.p, s);
        if (e != cudaSuccess) st = fail(c, SDD_ECUDA, "interface fill: %s", cudaGetErrorString(e));
    }
    rec_ext(c->ev[3], s);
    if (st == SDD_OK && c->pipe) {
        // the systems and the faces of the new fields were made beside the paths; the interface
        // values close the step, with the step counter
        cu(cudaStreamWaitEvent(s, c->pev[4], 0));
        const SolveCall& k = c->step_call[parity];
        cu(launch_scatter_iface(o.mean_xi, o.mean_eta, c->d_iface_idx.p, (int)c->iface_idx.size(), k.a.x[0],
                                k.a.x[1], c->d_step.p, s));
    } else if (st == SDD_OK) {
        st = enqueue_solve_dirichlet(c, c->step_call[parity], o.mean_xi, o.mean_eta, s);
        if (st == SDD_OK) st = enqueue_solve_system(c, c->step_call[parity], s);
        if (st == SDD_OK) st = enqueue_solve_iterate(c, c->step_call[parity], s);
        if (st == SDD_OK) cu(launch_bump_step(c->d_step.p, s));
    }
    rec_ext(c->ev[4], s);
    c->cur = saved;
    c->dirty_w = keep_w;
    c->dirty_fields = keep_f;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (st != SDD_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return fail(c, SDD_ECUDA, "capture: %s", cudaGetErrorString(e));
    GraphSlot& slot = with_pending ? c->graph_p[parity] : c->graph[parity];
    slot.release();
    {
        size_t nn = 0;
        if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn > 0) {
            std::vector<cudaGraphNode_t> nodes(nn);
            int kernels = 0;
            if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
                for (size_t k = 0; k < nn; ++k) {
                    cudaGraphNodeType t;
                    if (cudaGraphNodeGetType(nodes[k], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
                }
            (with_pending ? c->graph_kernels_p : c->graph_kernels) = kernels;
        }
    }
    e = cudaGraphInstantiate(&slot.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        slot.exec = nullptr;
        return fail(c, SDD_ECUDA, "instantiate: %s", cudaGetErrorString(e));
    }
    return SDD_OK;
}

sdd_status sdd_step(sdd_ctx* c, const sdd_step_params* p)
{
    if (!c || !p) return fail(c, SDD_EINVAL, "null argument");
    int K = 0;
    if (!valid_params(c, p->dt, p->Dt, p->exit_mode, &K)) return fail(c, SDD_EINVAL, "dt, Dt or exit_mode rejected");
    if (p->paths_per_node < 1 || p->paths_per_node > 0x7fffffffLL || p->max_iter < 0 || !(p->rtol >= 0.0))
        return fail(c, SDD_EINVAL, "paths_per_node, max_iter or rtol rejected");
    const bool same = c->graph_ok && std::memcmp(&c->graph_params, p, sizeof *p) == 0;
    if (!same) {
        sdd_status st0 = flush_pending(c);
        if (st0 != SDD_OK) return st0;
        drop_graphs(c);
        std::vector<int64_t> np(c->iface_x.size(), p->paths_per_node);
        std::vector<NodeSeg> segs(1);
        segs[0] = NodeSeg{c->iface_x.data(), c->iface_y.data(), np.data(), (int64_t)np.size(), 0, 0u};
        if (p->tune && !find_tuned(c->tuned, shape_key(segs, K, p->exit_mode))) {
            sdd_status st0 = prepare(c, c->stream);
            if (st0 != SDD_OK) return st0;
            TunedShape best{};
            st0 = autotune_plan(&c->err, c->sm_count, segs, c->d_inst.p, 1, K, p->dt, p->exit_mode, c->stream, c->tuned,
                                &best, ctx_zmap(c));
            if (st0 != SDD_OK) return st0;
        }
        int ppt = 0, block = 0, zmap = 0;
        pick_shape(c->tuned, segs, K, p->exit_mode, &ppt, &block, &zmap);
        sdd_status st = build_plan(c, c->step_plan, c->iface_x.data(), c->iface_y.data(), np.data(),
                                   (int64_t)np.size(), ppt, block, p->exit_mode, false);
        if (st != SDD_OK) return st;
        c->step_plan.zero_map = zmap;
        c->step_plan.zero_map_auto = true;
        CU(c, cudaStreamSynchronize(c->stream));
        // pipelined steps where the solve's iterations are one launch and the
        // paths do not read the fields (the field-gradient control variate does)
        const SolveCall probe = make_solve_call(c, p->Dt, p->rtol, p->max_iter, nullptr, nullptr, nullptr, nullptr,
                                                nullptr, true);
        // deferred scoring (survivors and plain exits scored after the path kernel) where the
        // records fit; pipelining needs it
        const size_t rec_bytes = (c->cv_mode ? 2 : 1) * sizeof(float2);
        c->defer = c->step_plan.ntasks > 0 && (size_t)c->step_plan.total_paths * rec_bytes <= (8ULL << 30);
        c->pipe = c->pipe_allowed && solve_single_launch(probe) && c->cv_mode != SDD_CV_FIELDS && c->defer;
        if (c->defer)
            CU(c, c->surv.alloc(((size_t)c->step_plan.total_paths * rec_bytes + sizeof(float4) - 1) / sizeof(float4)));
        if (c->pipe) {
            if (!c->pipe_stream) {
                // its kernels take SMs before the waiting blocks of the path kernel
                int least = 0, greatest = 0;
                CU(c, cudaDeviceGetStreamPriorityRange(&least, &greatest));
                CU(c, cudaStreamCreateWithPriority(&c->pipe_stream, cudaStreamNonBlocking, greatest));
            }
            for (cudaEvent_t& e : c->pev)
                if (!e) CU(c, cudaEventCreate(&e));
            if (!c->faces_stream) CU(c, cudaStreamCreateWithFlags(&c->faces_stream, cudaStreamNonBlocking));
            for (cudaEvent_t& e : c->fev)
                if (!e) CU(c, cudaEventCreate(&e));
        }
        for (int parity = 0; parity < 2; ++parity)
            if ((st = capture_step(c, p, K, parity, false)) != SDD_OK) return st;
        if (c->pipe)
            for (int parity = 0; parity < 2; ++parity)
                if ((st = capture_step(c, p, K, parity, true)) != SDD_OK) return st;
        c->graph_params = *p;
        c->graph_ok = true;
    }
    // the step counter lives on the device; make sure it holds n
    CU(c, cudaMemcpyAsync(c->d_step.p, &c->step_index, sizeof(uint32_t), cudaMemcpyHostToDevice, c->stream));
    const bool with_pending = c->pipe && c->pending;
    CU(c, cudaGraphLaunch((with_pending ? c->graph_p : c->graph)[c->cur].exec, c->stream));
    c->last_had_pending = with_pending;
    if (c->pipe) {
        c->pend_call = c->step_call[c->cur];
        c->pending = true;
    }
    c->cur = 1 - c->cur;
    c->step_index += 1;
    c->dirty_w = false;
    c->dirty_fields = true;  // the new fields need their tables before a direct estimate
    return SDD_OK;
}

sdd_status sdd_last_interface_stats(sdd_ctx* c, sdd_node_stats* out)
{
    if (!c || !out) return fail(c, SDD_EINVAL, "null argument");
    const size_t n = c->iface_idx.size();
    double* dst[4] = {out->mean_xi, out->mean_eta, out->se_xi, out->se_eta};
    for (int k = 0; k < 4; ++k)
        if (dst[k] && n) CU(c, cudaMemcpyAsync(dst[k], c->iface_stats[k].p, n * sizeof(double), cudaMemcpyDefault, c->stream));
    int64_t* ci[2] = {out->n_exit, out->path_steps};
    for (int k = 0; k < 2; ++k)
        if (ci[k] && n) CU(c, cudaMemcpyAsync(ci[k], c->iface_counts[k].p, n * sizeof(int64_t), cudaMemcpyDefault, c->stream));
    return SDD_OK;
}

sdd_status sdd_last_step_info(sdd_ctx* c, sdd_step_info* out)
{
    if (!c || !out) return fail(c, SDD_EINVAL, "null argument");
    if (!c->graph_ok) return fail(c, SDD_EINVAL, "no step has run");
    CU(c, cudaStreamSynchronize(c->stream));
    out->kernel_nodes = c->last_had_pending ? c->graph_kernels_p : c->graph_kernels;
    if (c->graph_mg_loops) {
        // kernel nodes of the graph itself plus the kernels its loop bodies ran in this step
        int32_t body = 0;
        CU(c, cudaMemcpy(&body, c->mg_loop.p + 2, sizeof body, cudaMemcpyDeviceToHost));
        out->kernel_nodes += body;
    }
    CU(c, cudaEventElapsedTime(&out->paths_ms, c->ev[1], c->ev[2]));
    CU(c, cudaEventElapsedTime(&out->estimate_ms, c->ev[0], c->ev[3]));
    CU(c, cudaEventElapsedTime(&out->solve_ms, c->ev[3], c->ev[4]));
    if (c->last_had_pending) {
        // the iterations this graph ran (the previous step's) beside the paths
        float it = 0.f;
        CU(c, cudaEventElapsedTime(&it, c->pev[2], c->pev[3]));
        out->solve_ms += it;
    }
    CU(c, cudaEventElapsedTime(&out->step_ms, c->ev[0], c->ev[4]));
    return SDD_OK;
}

sdd_status sdd_set_step_index(sdd_ctx* c, uint32_t n)
{
    if (!c) return SDD_EINVAL;
    c->step_index = n;
    return SDD_OK;
}

uint32_t sdd_get_step_index(const sdd_ctx* c) { return c ? c->step_index : 0u; }

sdd_status sdd_set_pipeline(sdd_ctx* c, int32_t on)
{
    if (!c) return SDD_EINVAL;
    const sdd_status fs = flush_pending(c);
    if (fs != SDD_OK) return fs;
    if (c->pipe_allowed != (on != 0)) drop_graphs(c);
    c->pipe_allowed = on != 0;
    return SDD_OK;
}

int32_t sdd_pipeline_in_use(const sdd_ctx* c) { return c && c->graph_ok && c->pipe ? 1 : 0; }

sdd_status sdd_flush(sdd_ctx* c)
{
    if (!c) return SDD_EINVAL;
    return flush_pending(c);
}

sdd_status sdd_sync(sdd_ctx* c)
{
    if (!c) return SDD_EINVAL;
    {
        const sdd_status fs = flush_pending(c);
        if (fs != SDD_OK) return fs;
    }
    CU(c, cudaStreamSynchronize(c->stream));
    int status = 0;
    CU(c, cudaMemcpy(&status, c->d_status.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (status) {
        CU(c, cudaMemset(c->d_status.p, 0, sizeof(int)));
        if (status & STATUS_BAD_W) return fail(c, SDD_EDEVICE, "w has a value that is not finite and positive");
        if (status & STATUS_TIMEOUT) return fail(c, SDD_ETIMEOUT, "a bounded device wait ran out");
        if (status & STATUS_NOCONV) return fail(c, SDD_ENOCONV, "a subdomain solve stopped at max_iter");
    }
    return SDD_OK;
}

const char* sdd_last_error(const sdd_ctx* c) { return c ? c->err.c_str() : "null context"; }

void sdd_destroy(sdd_ctx* c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    for (int k = 0; k < 5; ++k)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->mg_s2) cudaStreamDestroy(c->mg_s2);
    if (c->mg_s3) cudaStreamDestroy(c->mg_s3);
    if (c->pipe_stream) cudaStreamDestroy(c->pipe_stream);
    for (cudaEvent_t e : c->pev)
        if (e) cudaEventDestroy(e);
    if (c->faces_stream) cudaStreamDestroy(c->faces_stream);
    for (cudaEvent_t e : c->fev)
        if (e) cudaEventDestroy(e);
    delete c;  // device buffers are freed by their destructors
}

}  // extern "C"

struct sdd_batch {
    std::vector<sdd_ctx*> ctxs;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    int device = 0;
    int sm_count = 0;
    DevBuf<InstDev> d_inst;
    DevBuf<OutDev> d_out;       // outputs of sdd_batch_interface_mc
    DevBuf<OutDev> d_step_out;  // each instance's interface statistics of sdd_batch_step
    DevBuf<uint32_t> d_step;
    Plan mc_plan;
    Plan step_plan;
    std::vector<TunedShape> tuned;
    GraphSlot graph[2];
    std::vector<int> graph_parity[2];
    sdd_step_params graph_params{};
    bool graph_ok = false;
    int graph_kernels = 0;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    uint32_t step_index = 0;
    std::string err;
};

namespace {

void drop_batch_graphs(sdd_batch* b)
{
    for (int k = 0; k < 2; ++k) {
        b->graph[k].release();
        b->graph_parity[k].clear();
    }
    b->graph_ok = false;
}

// the step graph of the batch for the instances' current field buffers
sdd_status capture_batch_step(sdd_batch* b, const sdd_step_params* p, int K, int slot)
{
    cudaStream_t s = b->cap_stream;
    cudaGraph_t g = nullptr;
    CU(&b->err, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    sdd_status st = SDD_OK;
    std::vector<char> keep_w(b->ctxs.size()), keep_f(b->ctxs.size());
    for (size_t k = 0; k < b->ctxs.size(); ++k) {
        keep_w[k] = b->ctxs[k]->dirty_w;
        keep_f[k] = b->ctxs[k]->dirty_fields;
    }
    auto rec_ev = [&](int k) {
        if (st != SDD_OK) return;
        cudaError_t e = cudaEventRecordWithFlags(b->ev[k], s, cudaEventRecordExternal);
        if (e != cudaSuccess) st = fail(&b->err, SDD_ECUDA, "event: %s", cudaGetErrorString(e));
    };
    rec_ev(0);
    for (sdd_ctx* c : b->ctxs) {
        if (st != SDD_OK) break;
        c->dirty_w = c->dirty_fields = true;
        st = prepare(c, s);
        if (st != SDD_OK) b->err = c->err;
    }
    if (st == SDD_OK)
        st = run_plan_on(&b->err, b->step_plan, b->d_inst.p, b->d_step_out.p, OutDev{}, p->dt, K, p->seed, 0,
                         b->d_step.p, p->exit_mode, nullptr, s, b->ev[1], b->ev[2]);
    rec_ev(3);
    for (sdd_ctx* c : b->ctxs) {
        if (st != SDD_OK) break;
        st = enqueue_solve(c, p->Dt, c->iface_stats[0].p, c->iface_stats[1].p, p->rtol, p->max_iter,
                           c->fld[1 - c->cur][0].p, c->fld[1 - c->cur][1].p, s);
        if (st != SDD_OK) b->err = c->err;
    }
    if (st == SDD_OK) {
        cudaError_t e = launch_bump_step(b->d_step.p, s);
        if (e != cudaSuccess) st = fail(&b->err, SDD_ECUDA, "%s", cudaGetErrorString(e));
    }
    rec_ev(4);
    for (size_t k = 0; k < b->ctxs.size(); ++k) {
        b->ctxs[k]->dirty_w = keep_w[k];
        b->ctxs[k]->dirty_fields = keep_f[k];
    }
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (st != SDD_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return fail(&b->err, SDD_ECUDA, "capture: %s", cudaGetErrorString(e));
    b->graph[slot].release();
    size_t nn = 0;
    if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn > 0) {
        std::vector<cudaGraphNode_t> nodes(nn);
        int kernels = 0;
        if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
            for (size_t k = 0; k < nn; ++k) {
                cudaGraphNodeType t;
                if (cudaGraphNodeGetType(nodes[k], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
            }
        b->graph_kernels = kernels;
    }
    e = cudaGraphInstantiate(&b->graph[slot].exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->graph[slot].exec = nullptr;
        return fail(&b->err, SDD_ECUDA, "instantiate: %s", cudaGetErrorString(e));
    }
    b->graph_parity[slot].clear();
    for (sdd_ctx* c : b->ctxs) b->graph_parity[slot].push_back(c->cur);
    return SDD_OK;
}

}  // namespace

extern "C" {

sdd_status sdd_batch_create(sdd_batch** out, sdd_ctx* const* ctxs, int32_t count, void* stream)
{
    if (!out || !ctxs || count < 1) return SDD_EINVAL;
    *out = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SDD_ECUDA;
    for (int32_t k = 0; k < count; ++k)
        if (!ctxs[k] || ctxs[k]->device != dev) return SDD_EINVAL;
    for (int32_t a = 0; a < count; ++a)
        for (int32_t c = a + 1; c < count; ++c)
            if (ctxs[a] == ctxs[c]) return SDD_EINVAL;
    for (int32_t k = 0; k < count; ++k) {
        // a context's own pipelined step may have left its solve's iterations pending
        if (ctxs[k]->pending) {
            const sdd_status fs = flush_pending(ctxs[k]);
            if (fs != SDD_OK) return fs;
            if (cudaStreamSynchronize(ctxs[k]->stream) != cudaSuccess) return SDD_ECUDA;
        }
    }
    sdd_batch* b = new (std::nothrow) sdd_batch();
    if (!b) return SDD_ENOMEM;
    b->ctxs.assign(ctxs, ctxs + count);
    b->stream = (cudaStream_t)stream;
    b->device = dev;
    b->sm_count = ctxs[0]->sm_count;
    auto bail = [&](sdd_status st) {
        sdd_batch_destroy(b);
        return st;
    };
    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) return bail(SDD_ECUDA);
    for (int k = 0; k < 5; ++k)
        if (cudaEventCreate(&b->ev[k]) != cudaSuccess) return bail(SDD_ECUDA);
    std::vector<InstDev> inst(count);
    std::vector<OutDev> outs(count);
    for (int32_t k = 0; k < count; ++k) {
        inst[k] = inst_host(ctxs[k]);
        sdd_ctx* c = ctxs[k];
        outs[k].mean_xi = c->iface_stats[0].p;
        outs[k].mean_eta = c->iface_stats[1].p;
        outs[k].se_xi = c->iface_stats[2].p;
        outs[k].se_eta = c->iface_stats[3].p;
        outs[k].n_exit = c->iface_counts[0].p;
        outs[k].path_steps = c->iface_counts[1].p;
    }
    if (b->d_inst.alloc(count) != cudaSuccess || b->d_out.alloc(count) != cudaSuccess ||
        b->d_step_out.alloc(count) != cudaSuccess || b->d_step.alloc(1) != cudaSuccess)
        return bail(SDD_ENOMEM);
    if (cudaMemcpy(b->d_inst.p, inst.data(), count * sizeof(InstDev), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_step_out.p, outs.data(), count * sizeof(OutDev), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->d_step.p, 0, sizeof(uint32_t)) != cudaSuccess)
        return bail(SDD_ECUDA);
    *out = b;
    return SDD_OK;
}

// A context stepped on its own may have left its solve's iterations pending:
// run them (on its stream) before the batch uses its fields.
static sdd_status flush_batch(sdd_batch* b)
{
    for (sdd_ctx* c : b->ctxs) {
        if (!c->pending) continue;
        const sdd_status fs = flush_pending(c);
        if (fs != SDD_OK) return fail(&b->err, fs, "%s", c->err.c_str());
        CU(&b->err, cudaStreamSynchronize(c->stream));
    }
    return SDD_OK;
}

sdd_status sdd_batch_interface_mc(sdd_batch* b, const sdd_nodes* nodes, const sdd_mc_params* p, sdd_node_stats* out)
{
    if (!b || !nodes || !p || !out) return b ? fail(&b->err, SDD_EINVAL, "null argument") : SDD_EINVAL;
    {
        const sdd_status fs = flush_batch(b);
        if (fs != SDD_OK) return fs;
    }
    int K = 0;
    if (!valid_params(nullptr, p->dt, p->Dt, p->exit_mode, &K))
        return fail(&b->err, SDD_EINVAL, "dt, Dt or exit_mode rejected (Dt / dt must be an integer in [1, 2^20])");
    const int32_t n = (int32_t)b->ctxs.size();
    std::vector<NodeSeg> segs(n);
    uint32_t ctr = p->node_word0;
    for (int32_t k = 0; k < n; ++k) {
        if (nodes[k].count > 0 && (!nodes[k].x || !nodes[k].y || !nodes[k].n_paths))
            return fail(&b->err, SDD_EINVAL, "null node array for instance %d", k);
        segs[k] = NodeSeg{nodes[k].x, nodes[k].y, nodes[k].n_paths, nodes[k].count, k, ctr};
        ctr += (uint32_t)nodes[k].count;
    }
    int ppt = p->paths_per_task, block = p->block_threads;
    pick_shape(b->tuned, segs, K, p->exit_mode, &ppt, &block);
    sdd_status st = build_plan_segs(&b->err, b->sm_count, b->mc_plan, segs, ppt, block, p->exit_mode, false);
    if (st != SDD_OK) return st;
    for (sdd_ctx* c : b->ctxs)
        if ((st = prepare(c, b->stream)) != SDD_OK) return fail(&b->err, st, "%s", c->err.c_str());
    std::vector<OutDev> outs(n);
    for (int32_t k = 0; k < n; ++k) outs[k] = out_from(&out[k]);
    CU(&b->err, cudaMemcpyAsync(b->d_out.p, outs.data(), n * sizeof(OutDev), cudaMemcpyHostToDevice, b->stream));
    return run_plan_on(&b->err, b->mc_plan, b->d_inst.p, b->d_out.p, OutDev{}, p->dt, K, p->seed, p->step_index,
                       nullptr, p->exit_mode, nullptr, b->stream, nullptr, nullptr);
}

sdd_status sdd_batch_step(sdd_batch* b, const sdd_step_params* p)
{
    if (!b || !p) return b ? fail(&b->err, SDD_EINVAL, "null argument") : SDD_EINVAL;
    {
        const sdd_status fs = flush_batch(b);
        if (fs != SDD_OK) return fs;
    }
    int K = 0;
    if (!valid_params(nullptr, p->dt, p->Dt, p->exit_mode, &K)) return fail(&b->err, SDD_EINVAL, "dt, Dt or exit_mode rejected");
    if (p->paths_per_node < 1 || p->paths_per_node > 0x7fffffffLL || p->max_iter < 0 || !(p->rtol >= 0.0))
        return fail(&b->err, SDD_EINVAL, "paths_per_node, max_iter or rtol rejected");
    const bool same = b->graph_ok && std::memcmp(&b->graph_params, p, sizeof *p) == 0;
    if (!same) {
        drop_batch_graphs(b);
        const int32_t n = (int32_t)b->ctxs.size();
        std::vector<std::vector<int64_t>> np(n);
        std::vector<NodeSeg> segs(n);
        uint32_t ctr = 0;
        for (int32_t k = 0; k < n; ++k) {
            sdd_ctx* c = b->ctxs[k];
            np[k].assign(c->iface_x.size(), p->paths_per_node);
            segs[k] = NodeSeg{c->iface_x.data(), c->iface_y.data(), np[k].data(), (int64_t)np[k].size(), k, ctr};
            ctr += (uint32_t)np[k].size();
        }
        if (p->tune && !find_tuned(b->tuned, shape_key(segs, K, p->exit_mode))) {
            for (sdd_ctx* c : b->ctxs) {
                sdd_status st0 = prepare(c, b->stream);
                if (st0 != SDD_OK) return fail(&b->err, st0, "%s", c->err.c_str());
            }
            TunedShape best{};
            sdd_status st0 = autotune_plan(&b->err, b->sm_count, segs, b->d_inst.p, n, K, p->dt, p->exit_mode,
                                           b->stream, b->tuned, &best);
            if (st0 != SDD_OK) return st0;
        }
        int ppt = 0, block = 0;
        pick_shape(b->tuned, segs, K, p->exit_mode, &ppt, &block);
        sdd_status st = build_plan_segs(&b->err, b->sm_count, b->step_plan, segs, ppt, block, p->exit_mode, false);
        if (st != SDD_OK) return st;
        b->graph_params = *p;
        b->graph_ok = true;
    }
    // the graph whose field buffers match the instances' current ones
    int slot = -1;
    for (int k = 0; k < 2 && slot < 0; ++k) {
        if (!b->graph[k].exec || b->graph_parity[k].size() != b->ctxs.size()) continue;
        bool match = true;
        for (size_t i = 0; i < b->ctxs.size(); ++i) match = match && b->graph_parity[k][i] == b->ctxs[i]->cur;
        if (match) slot = k;
    }
    if (slot < 0) {
        slot = b->graph[0].exec ? 1 : 0;
        if (b->graph[0].exec && b->graph[1].exec) slot = 0;
        CU(&b->err, cudaStreamSynchronize(b->stream));
        sdd_status st = capture_batch_step(b, p, K, slot);
        if (st != SDD_OK) return st;
    }
    CU(&b->err, cudaMemcpyAsync(b->d_step.p, &b->step_index, sizeof(uint32_t), cudaMemcpyHostToDevice, b->stream));
    CU(&b->err, cudaGraphLaunch(b->graph[slot].exec, b->stream));
    for (sdd_ctx* c : b->ctxs) {
        c->cur = 1 - c->cur;
        c->step_index = b->step_index + 1;
        c->dirty_w = false;
        c->dirty_fields = true;
    }
    b->step_index += 1;
    return SDD_OK;
}

sdd_status sdd_batch_autotune(sdd_batch* b, const sdd_nodes* nodes, const sdd_mc_params* p, sdd_launch_shape* out)
{
    if (!b || !nodes || !p) return b ? fail(&b->err, SDD_EINVAL, "null argument") : SDD_EINVAL;
    int K = 0;
    if (!valid_params(nullptr, p->dt, p->Dt, p->exit_mode, &K)) return fail(&b->err, SDD_EINVAL, "dt, Dt or exit_mode rejected");
    const int32_t n = (int32_t)b->ctxs.size();
    std::vector<NodeSeg> segs(n);
    uint32_t ctr = p->node_word0;
    for (int32_t k = 0; k < n; ++k) {
        if (nodes[k].count > 0 && (!nodes[k].x || !nodes[k].y || !nodes[k].n_paths))
            return fail(&b->err, SDD_EINVAL, "null node array for instance %d", k);
        segs[k] = NodeSeg{nodes[k].x, nodes[k].y, nodes[k].n_paths, nodes[k].count, k, ctr};
        ctr += (uint32_t)nodes[k].count;
    }
    for (sdd_ctx* c : b->ctxs) {
        sdd_status st = prepare(c, b->stream);
        if (st != SDD_OK) return fail(&b->err, st, "%s", c->err.c_str());
    }
    TunedShape best{};
    sdd_status st = autotune_plan(&b->err, b->sm_count, segs, b->d_inst.p, n, K, p->dt, p->exit_mode, b->stream,
                                  b->tuned, &best);
    if (st != SDD_OK) return st;
    if (out) {
        out->block_threads = best.block;
        out->paths_per_task = best.ppt;
        out->ms = best.ms;
        out->zero_map = best.zero_map ? 1 : 2;
    }
    return SDD_OK;
}

sdd_status sdd_batch_last_step_info(sdd_batch* b, sdd_step_info* out)
{
    if (!b || !out) return SDD_EINVAL;
    if (!b->graph_ok) return fail(&b->err, SDD_EINVAL, "no step has run");
    CU(&b->err, cudaStreamSynchronize(b->stream));
    out->kernel_nodes = b->graph_kernels;
    CU(&b->err, cudaEventElapsedTime(&out->paths_ms, b->ev[1], b->ev[2]));
    CU(&b->err, cudaEventElapsedTime(&out->estimate_ms, b->ev[0], b->ev[3]));
    CU(&b->err, cudaEventElapsedTime(&out->solve_ms, b->ev[3], b->ev[4]));
    CU(&b->err, cudaEventElapsedTime(&out->step_ms, b->ev[0], b->ev[4]));
    return SDD_OK;
}

sdd_status sdd_batch_set_step_index(sdd_batch* b, uint32_t n)
{
    if (!b) return SDD_EINVAL;
    b->step_index = n;
    for (sdd_ctx* c : b->ctxs) c->step_index = n;
    return SDD_OK;
}

sdd_status sdd_batch_sync(sdd_batch* b)
{
    if (!b) return SDD_EINVAL;
    CU(&b->err, cudaStreamSynchronize(b->stream));
    for (sdd_ctx* c : b->ctxs) {
        sdd_status st = sdd_sync(c);
        if (st != SDD_OK) return fail(&b->err, st, "%s", c->err.c_str());
    }
    return SDD_OK;
}

const char* sdd_batch_last_error(const sdd_batch* b) { return b ? b->err.c_str() : "null batch"; }

void sdd_batch_destroy(sdd_batch* b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    drop_batch_graphs(b);
    for (int k = 0; k < 5; ++k)
        if (b->ev[k]) cudaEventDestroy(b->ev[k]);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete b;
}

sdd_status sdd_rng_draw(uint64_t seed, const uint32_t* ctrs, int64_t count, uint32_t* words, float* normals,
                        void* stream)
{
    if (count < 0 || (count > 0 && (!ctrs || !words))) return SDD_EINVAL;
    cudaError_t e = launch_rng_draw(seed, ctrs, count, words, normals, (cudaStream_t)stream);
    return e == cudaSuccess ? SDD_OK : SDD_ECUDA;
}

}  // extern "C"
