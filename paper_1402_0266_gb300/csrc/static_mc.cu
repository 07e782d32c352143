// static_mc.cu -- the interface estimate with every piece of working memory in
// one fixed array of static device memory, for callers that cannot allocate.
//
// Who needs it: code that runs where allocating device memory is not allowed
// or not wanted -- a real-time loop that must not call into the allocator
// after start-up, a host application whose memory pool hands out only fixed
// buffers, a plugin that is given device pointers and a stream and nothing
// else. Such a caller still passes its inputs (w, xi, eta, optional face data,
// the nodes) and its output arrays; the tables the estimate needs (cell
// records of the drift and of xi, eta, the face data, the node and task lists,
// the per-task sums and the work counter) live in g_static_scratch below.
//
// The array is file-scope __device__ memory, so every GPU that loads the
// library holds its kStaticScratchBytes until the process exits. Host code
// cannot use the array's name as a device address: the first call on each
// device looks the address up with cudaGetSymbolAddress (with that device
// current) and keeps it; make that first call before any stream capture.
// Every call shares the array and it keeps the previous call's contents: the
// work counter and the status word are cleared on every call, everything else
// is rewritten before it is read. Calls whose work overlaps on the GPU (other
// streams, other host threads) race on the array and must not be issued.
//
// Device-side errors (a w that is not finite and positive) set the status word
// in the array; the call hands it to the caller: copied into the caller's
// device word at the end of the call's work, or, without one, read back after
// waiting for the stream and returned as SDD_EDEVICE.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/sdd.h"
#include "common.cuh"

using namespace sdd;

namespace {

// Limits of the static variant.
constexpr int kStaticMaxSide = 257;                                      // nx, ny <= 257
constexpr int kStaticMaxCells = (kStaticMaxSide - 1) * (kStaticMaxSide - 1);
constexpr int kStaticMaxFaces = 2 * (2 * kStaticMaxSide + 2 * kStaticMaxSide);
constexpr int kStaticMaxNodes = 8192;
constexpr int kStaticMaxTasks = 65536;

constexpr size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Byte offsets of the regions inside the array.
constexpr size_t kOffQueue = 0;
constexpr size_t kOffStatus = kOffQueue + 256;
constexpr size_t kOffInst = kOffStatus + 256;
constexpr size_t kOffNodes = kOffInst + align256(sizeof(InstDev));
constexpr size_t kOffTasks = kOffNodes + align256(sizeof(NodeDev) * kStaticMaxNodes);
constexpr size_t kOffPartials = kOffTasks + align256(sizeof(Task) * kStaticMaxTasks);
constexpr size_t kOffBcoef = kOffPartials + align256(sizeof(Partial) * kStaticMaxTasks);
constexpr size_t kOffFcoef = kOffBcoef + align256(2 * sizeof(float4) * kStaticMaxCells);
constexpr size_t kOffFaces64 = kOffFcoef + align256(2 * sizeof(float4) * kStaticMaxCells);
constexpr size_t kOffFaces32 = kOffFaces64 + align256(sizeof(double) * kStaticMaxFaces);
constexpr size_t kStaticScratchBytes = kOffFaces32 + align256(sizeof(float) * kStaticMaxFaces);

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_lock;
unsigned char* g_static_ptr[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};

// Host staging of the node and task lists (host static memory: no allocation).
NodeDev g_nodes_host[kStaticMaxNodes];
Task g_tasks_host[kStaticMaxTasks];
InstDev g_inst_host;
int g_status_host;

// Address of this device's array, looked up once per device.
cudaError_t static_scratch(unsigned char** out, int* sm_count)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_setup_lock);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        if (!p) return cudaErrorInvalidSymbol;
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        g_static_ptr[dev] = (unsigned char*)p;
        g_sm_count[dev] = sms;
    }
    *out = g_static_ptr[dev];
    *sm_count = g_sm_count[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" {

int64_t sdd_static_scratch_bytes(void) { return (int64_t)kStaticScratchBytes; }

sdd_status sdd_interface_mc_static(const sdd_fields* f, const sdd_nodes* nodes, const sdd_mc_params* p,
                                   sdd_node_stats* out, int32_t* status_out, void* stream)
{
    if (!f || !nodes || !p || !out) return SDD_EINVAL;
    const int nx = f->nx, ny = f->ny;
    if (nx < 3 || ny < 3 || nx > kStaticMaxSide || ny > kStaticMaxSide) return SDD_EINVAL;
    if (!f->w || !f->xi || !f->eta) return SDD_EINVAL;
    const int64_t count = nodes->count;
    if (count < 0 || count > kStaticMaxNodes) return SDD_EINVAL;
    if (count > 0 && (!nodes->x || !nodes->y || !nodes->n_paths)) return SDD_EINVAL;
    if (!(p->dt > 0.0) || !(p->Dt > 0.0) || !std::isfinite(p->dt) || !std::isfinite(p->Dt)) return SDD_EINVAL;
    const double kq = p->Dt / p->dt, kr = std::round(kq);
    if (kr < 1.0 || kr > (double)(1 << 20) || std::fabs(kr - kq) > 1e-9 * kq) return SDD_EINVAL;
    if (p->exit_mode != 0 && p->exit_mode != 1 && p->exit_mode != 2) return SDD_EINVAL;
    if (p->paths_per_task < 0 || (p->paths_per_task % 32) != 0) return SDD_EINVAL;
    const int block_req = p->block_threads ? p->block_threads : 256;
    if (block_req != 64 && block_req != 128 && block_req != 256 && block_req != 512) return SDD_EINVAL;
    const int block = std::min(block_req, path_kernel_max_block(p->exit_mode));
    const int K = (int)kr;
    for (int64_t k = 0; k < count; ++k) {
        if (!(nodes->x[k] >= 0.0 && nodes->x[k] <= 1.0 && nodes->y[k] >= 0.0 && nodes->y[k] <= 1.0)) return SDD_EINVAL;
        if (nodes->n_paths[k] < 1 || nodes->n_paths[k] > 0x7fffffffLL) return SDD_EINVAL;
    }
    // paths per task: as requested, else the smallest multiple of 128 that keeps the task list within its limit
    auto tasks_for = [&](int64_t q) {
        int64_t t = 0;
        for (int64_t k = 0; k < count; ++k) {
            const double x = nodes->x[k], y = nodes->y[k];
            if (x <= 0.0 || x >= 1.0 || y <= 0.0 || y >= 1.0) continue;
            t += (nodes->n_paths[k] + q - 1) / q;
        }
        return t;
    };
    int64_t ppt = p->paths_per_task;
    if (ppt) {
        if (tasks_for(ppt) > kStaticMaxTasks) return SDD_EINVAL;  // the requested task size does not fit
    } else {
        // the task count falls as the task size grows: bisect over multiples of 128 (at the largest
        // node's path count every node is one task, and count <= kStaticMaxNodes < kStaticMaxTasks)
        int64_t most = 1;
        for (int64_t k = 0; k < count; ++k) most = std::max<int64_t>(most, nodes->n_paths[k]);
        int64_t lo = 1, hi = (most + 127) / 128;
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo) / 2;
            if (tasks_for(128 * mid) <= kStaticMaxTasks) hi = mid;
            else lo = mid + 1;
        }
        ppt = 128 * lo;
    }

    unsigned char* base = nullptr;
    int sm_count = 0;
    if (static_scratch(&base, &sm_count) != cudaSuccess) return SDD_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    int* queue = (int*)(base + kOffQueue);
    int* status = (int*)(base + kOffStatus);
    InstDev* inst = (InstDev*)(base + kOffInst);
    NodeDev* dnodes = (NodeDev*)(base + kOffNodes);
    Task* dtasks = (Task*)(base + kOffTasks);
    Partial* partials = (Partial*)(base + kOffPartials);
    float4* bcoef = (float4*)(base + kOffBcoef);
    float4* fcoef = (float4*)(base + kOffFcoef);
    double* faces64 = (double*)(base + kOffFaces64);
    float* faces32 = (float*)(base + kOffFaces32);
    const int nfaces = 2 * (2 * nx + 2 * ny);

    // node and task lists, in the caller's node order
    int64_t t = 0, rec = 0;
    for (int64_t k = 0; k < count; ++k) {
        NodeDev& nd = g_nodes_host[k];
        std::memset(&nd, 0, sizeof nd);
        nd.x = nodes->x[k];
        nd.y = nodes->y[k];
        nd.xf = (float)nd.x;
        nd.yf = (float)nd.y;
        nd.inst = 0;
        nd.ctr = p->node_word0 + (uint32_t)k;
        nd.n_paths = (int32_t)nodes->n_paths[k];
        nd.local = (int32_t)k;
        nd.rec0 = rec;
        rec += nodes->n_paths[k];
        nd.task0 = (int32_t)t;
        const bool bnd = nd.x <= 0.0 || nd.x >= 1.0 || nd.y <= 0.0 || nd.y >= 1.0;
        if (!bnd) {
            for (int64_t p0 = 0; p0 < nodes->n_paths[k]; p0 += ppt) {
                Task& tk = g_tasks_host[t++];
                tk.node = (int32_t)k;
                tk.path0 = (int32_t)p0;
                tk.npaths = (int32_t)std::min<int64_t>(ppt, nodes->n_paths[k] - p0);
                tk.pad = 0;
            }
        }
        nd.ntasks = (int32_t)(t - nd.task0);
    }
    std::memset(&g_inst_host, 0, sizeof g_inst_host);
    g_inst_host.bcoef = bcoef;
    g_inst_host.fcoef = fcoef;
    g_inst_host.faces32 = faces32;
    g_inst_host.faces64 = faces64;
    g_inst_host.nx = nx;
    g_inst_host.ny = ny;
    g_inst_host.sx = (float)(nx - 1);
    g_inst_host.sy = (float)(ny - 1);
    g_inst_host.gxmax = std::nextafter((float)(nx - 1), 0.0f);
    g_inst_host.gymax = std::nextafter((float)(ny - 1), 0.0f);
    g_inst_host.cell_bias = 0x4B000000u * (uint32_t)nx;

#define STATIC_CU(expr)                             \
    do {                                            \
        if ((expr) != cudaSuccess) return SDD_ECUDA; \
    } while (0)
    // pageable copies return once the host data is staged, so the host lists may be reused by the next call
    STATIC_CU(cudaMemcpyAsync(inst, &g_inst_host, sizeof g_inst_host, cudaMemcpyHostToDevice, s));
    if (count) STATIC_CU(cudaMemcpyAsync(dnodes, g_nodes_host, count * sizeof(NodeDev), cudaMemcpyHostToDevice, s));
    if (t) STATIC_CU(cudaMemcpyAsync(dtasks, g_tasks_host, t * sizeof(Task), cudaMemcpyHostToDevice, s));
    STATIC_CU(cudaMemsetAsync(status, 0, sizeof(int), s));
    // the tables of the estimate
    if (f->faces) STATIC_CU(cudaMemcpyAsync(faces64, f->faces, nfaces * sizeof(double), cudaMemcpyDeviceToDevice, s));
    else STATIC_CU(launch_winslow_faces(f->w, nx, ny, faces64, nullptr, s));
    STATIC_CU(launch_faces32(faces64, faces32, nfaces, s));
    STATIC_CU(launch_prep_cells(f->w, f->xi, f->eta, nx, ny, bcoef, fcoef, status, s));
    // the paths, then the per-node means
    if (t > 0) {
        PathArgs a{};
        a.inst = inst;
        a.nodes = dnodes;
        a.tasks = dtasks;
        a.partials = partials;
        a.queue = queue;
        a.ntasks = (int32_t)t;
        a.K = K;
        a.dt = (float)p->dt;
        a.bm_scale = (float)(-4.0 * p->dt * std::log(2.0));
        a.bridge_cut = (float)(18.0 * p->dt);
        a.horizon = (float)((double)a.K * p->dt);
        a.keys = philox_keys(p->seed);
        a.step_index = p->step_index;
        a.step_ptr = nullptr;
        STATIC_CU(cudaMemsetAsync(queue, 0, sizeof(int), s));
        const int per_block = block / 32;
        const int grid_max = sm_count * path_kernel_blocks_per_sm(p->exit_mode, false, block);
        const int grid = (int)std::min<int64_t>(grid_max, std::max<int64_t>(1, (t + per_block - 1) / per_block));
        STATIC_CU(launch_paths(a, p->exit_mode, false, grid, block, s));
    }
    if (count > 0) {
        FinalArgs fa{};
        fa.inst = inst;
        fa.nodes = dnodes;
        fa.partials = partials;
        fa.out_table = nullptr;
        fa.out0.mean_xi = out->mean_xi;
        fa.out0.mean_eta = out->mean_eta;
        fa.out0.se_xi = out->se_xi;
        fa.out0.se_eta = out->se_eta;
        fa.out0.n_exit = (long long*)out->n_exit;
        fa.out0.path_steps = (long long*)out->path_steps;
        fa.nnodes = (int32_t)count;
        STATIC_CU(launch_finalize(fa, s));
    }
    // the call's device status: into the caller's word, or read here after the stream's work
    if (status_out) {
        STATIC_CU(cudaMemcpyAsync(status_out, status, sizeof(int), cudaMemcpyDeviceToDevice, s));
    } else {
        STATIC_CU(cudaStreamSynchronize(s));
        STATIC_CU(cudaMemcpy(&g_status_host, status, sizeof(int), cudaMemcpyDeviceToHost));
        if (g_status_host != 0) return SDD_EDEVICE;
    }
#undef STATIC_CU
    return SDD_OK;
}

}  // extern "C"
