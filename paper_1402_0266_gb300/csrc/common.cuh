// common.cuh -- device-side data layout shared by the kernels of libsdd.
//
// One "instance" is one mesh problem (grid, w, xi, eta, face data). A single
// context is one instance; a batched launch runs many. Work is cut into tasks
// (a node and a contiguous range of its paths); persistent warps take tasks
// from a counter in device memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rng.cuh"

namespace sdd {

constexpr int kMaxCvSlices = 128;  // time slices of a control-variate table
constexpr int kCvMaxBlock = 256;   // threads per block of the path kernel with a control variate
constexpr int kCvMaxOrder = 255;   // largest order of the binomial smoothing of the field-gradient control variate

// The control variate's network: 5 inputs, two tanh layers of 64, one output;
// parameters W1 (64 x 5), b1, W2 (64 x 64, [out][in]), b2, w3, b3 in this order.
constexpr int kMlpInputs = 5;
constexpr int kMlpHidden = 64;
constexpr int kMlpParams = 4609;
constexpr int kMlpStride = 4616;   // floats between the two networks (xi, eta) of a parameter block

// Geometry and field tables of one instance, as the path kernel reads them.
struct InstDev {
    const float4* bcoef;   // 2 float4 per cell: (a0x, a0y, a1x, a1y), (a2x, a2y, a3x, a3y) of b = (b_x, b_y)
    const float4* fcoef;   // 2 float4 per cell: the same for (xi, eta)
    const float* faces32;  // face data, single precision (layout of sdd.h)
    const double* faces64; // face data, double precision
    int32_t nx, ny;
    float sx, sy;          // nx - 1, ny - 1 (inverse spacings)
    float gxmax, gymax;    // largest floats below nx - 1, ny - 1
    uint32_t cell_bias;    // 0x4B000000 * nx (mod 2^32): cell index from the float bits of 2^23 + floor(g)
    int32_t cv_slices;     // slices of the control-variate table (0: none)
    const uint4* cvcoef;   // per slice and cell 2 uint4: corner values (half precision) of the xi model's gradient, then the eta model's
    const float4* cvcell;  // per cell: (d/dx, d/dy) of the xi model, then of the eta model (one value per cell)
};

// Output arrays of one instance (device pointers; any may be null).
struct OutDev {
    double* mean_xi;
    double* mean_eta;
    double* se_xi;
    double* se_eta;
    long long* n_exit;
    long long* path_steps;
};

// One evaluation node.
struct NodeDev {
    double x, y;        // as given
    float xf, yf;       // start point of the paths (single precision)
    int32_t inst;       // instance index
    uint32_t ctr;       // node word of the Philox counter (numbers the nodes of all instances)
    int32_t n_paths;
    int32_t task0;      // first task of this node
    int32_t ntasks;     // 0 for a node on the boundary
    int32_t local;      // index into the instance's output arrays
    long long rec0;     // first per-path record of this node
};

struct Task {
    int32_t node;
    int32_t path0;
    int32_t npaths;
    int32_t pad;
};

// Per-task sums, shifted by the node's start coordinates (xi by x, eta by y):
// s = sum (Y - c), q = sum (Y - c)^2.
struct Partial {
    double s_xi, q_xi, s_eta, q_eta;
    long long exits, steps;
};

struct RecDev {
    int32_t* steps;
    int32_t* code;
    float* score_xi;
    float* score_eta;
    float* x_end;
    float* y_end;
};

struct PathArgs {
    const InstDev* inst;
    const NodeDev* nodes;
    const Task* tasks;
    Partial* partials;
    int* queue;              // next task (zeroed before the launch)
    int32_t ntasks;
    int32_t K;               // sub-steps per mesh step
    float dt;
    float bm_scale;          // -4 dt ln 2: r = sqrt(bm_scale * log2(u1)) = sqrt(2 dt) sqrt(-2 ln u1)
    float bridge_cut;        // skip the bridge test when dmin0 * dmin1 exceeds this
    float horizon;           // the mesh step K dt (exponential time-stepping)
    PhiloxKeys keys;         // round keys of the seed
    int32_t cv_bound[kMaxCvSlices + 1];  // control variate: slice q serves sub-steps cv_bound[q] <= j < cv_bound[q + 1]
    uint32_t step_index;
    const uint32_t* step_ptr; // if non-null, read the step index here
    RecDev rec;
    const uint8_t* node_mask; // if non-null, only nodes with a nonzero entry run their paths
    void* surv;               // if non-null, survivors and plain exits leave records here, scored later (rec0 + path)
    // zero map of the drift records (single-instance launches; zwords = 0: none): bit k of word k / 32
    // set when a drift record of cells [k 2^zshift, (k + 1) 2^zshift) is nonzero; record zcell is all zero
    const uint32_t* zmap;
    int32_t zwords;
    uint32_t zshift;
    uint32_t zcell;
    InstDev one;              // single: the one instance's tables (inst[0]), read as parameters
    int32_t single;           // 1: every task is of instance 0 and `one` holds its tables
};

// The zero map's size: at most kZmapMaxWords words (16 KB of shared memory per block of the path kernel).
constexpr int kZmapMaxWords = 4096;
inline uint32_t zmap_shift(long long cells)
{
    uint32_t s = 0;
    while (((cells + (1LL << s) - 1) >> s) > 32LL * kZmapMaxWords) ++s;
    return s;
}
inline int zmap_words(long long cells, uint32_t shift) { return (int)((((cells + (1LL << shift) - 1) >> shift) + 31) / 32); }
// Shared memory for a map of `words` words: whole groups of 32, as the kernel's slots permute each group.
inline size_t zmap_smem_bytes(int words) { return sizeof(uint32_t) * (size_t)((words + 31) / 32 * 32); }

struct FinalArgs {
    const InstDev* inst;
    const NodeDev* nodes;
    const Partial* partials;
    const OutDev* out_table;  // per instance; if null every node writes to out0
    OutDev out0;
    int32_t nnodes;
    RecDev rec;               // per-path records of boundary nodes (may be all null)
    const uint8_t* node_mask; // if non-null, nodes with a zero entry report no paths (filled later)
};

// Deferred scoring of the survivors, then the per-node reduction (k_score_surv).
struct ScoreArgs {
    const InstDev* inst;
    const NodeDev* nodes;
    const void* surv;
    int32_t nnodes;
    FinalArgs fin;            // the per-node reduction (nodes, partials, outputs, mask)
};

// Device status word bits.
enum : int {
    STATUS_BAD_W = 1,
    STATUS_NOCONV = 2,
    STATUS_TIMEOUT = 4,
};

// Launchers (defined in the .cu files; all asynchronous on `s`).
// cvm: the control variate's form, 0 none, 1 cvcoef (node values, time slices), 2 cvcell (cell values)
cudaError_t launch_paths(const PathArgs& a, int exit_mode, bool record, int grid, int block, cudaStream_t s,
                         int cvm = 0);
// exit_mode 0 with an even number of sub-steps has its own kernel (no odd last pair)
cudaError_t launch_finalize(const FinalArgs& a, cudaStream_t s);
cudaError_t launch_score_surv(const ScoreArgs& a, bool cv, cudaStream_t s);
int path_kernel_blocks_per_sm(int exit_mode, bool record, int block, int cvm = 0, int zwords = 0,
                              bool single = false);
// the largest block the path kernel of this exit mode is compiled for (single: one instance)
int path_kernel_max_block(int exit_mode, int cvm = 0, bool single = false);

// Cell records of the drift (from w; bcoef null: skipped) and of the fields
// (from xi, eta; fcoef null: skipped); with the drift records, if zmap is
// non-null, their zero map (zmap_words(cells, zshift) words, see PathArgs).
cudaError_t launch_prep_cells(const float* w, const double* xi, const double* eta, int nx, int ny, float4* bcoef,
                              float4* fcoef, int* status, cudaStream_t s, uint32_t* zmap = nullptr,
                              uint32_t zshift = 0);
// The paper's boundary data from w (faces64) and, if faces32 is non-null, its single-precision copy.
cudaError_t launch_winslow_faces(const float* w, int nx, int ny, double* faces64, float* faces32, cudaStream_t s);
cudaError_t launch_cv_cells(const double* grad, int slices, int nx, int ny, uint4* cvcoef, cudaStream_t s);
cudaError_t launch_faces32(const double* faces64, float* faces32, int n, cudaStream_t s);

// Key points and interface fill (keypoints.cu). One interface line: vertical
// (orient 0, column fixed) or horizontal (orient 1, row fixed), n nodes along
// it (both ends on the boundary); its interior positions t = 1 .. n - 2 are
// entries start + t - 1 of the position arrays (interface-node index, crossing flag).
struct KeyLine {
    int32_t orient, fixed, n, start;
};
cudaError_t launch_keypoints(const float* w, int nx, const KeyLine* lines, int nlines, int max_n,
                             const int32_t* pos_idx, const uint8_t* pos_cross, int spacing, uint8_t* mask,
                             cudaStream_t s);
size_t pchip_scratch_doubles(long long total_positions, int nlines);
cudaError_t launch_pchip(const KeyLine* lines, int nlines, int max_n, const int32_t* pos_idx,
                         const uint8_t* pos_cross, const uint8_t* mask, const double* faces, int nx, int ny,
                         double* mean_xi, double* mean_eta, double* scratch, cudaStream_t s);

// Learned control variate (mlp.cu).
cudaError_t launch_node_features(const float* w, int nx, int ny, double* w64, double* r64, double2* gw, float4* nfa,
                                 float2* nfb, cudaStream_t s);
cudaError_t launch_field_grad(const double* xi, const double* eta, int nx, int ny, double* table, cudaStream_t s);
// The field-gradient control variate's cell values from the node table of launch_field_grad:
// each component smoothed by the binomial filter of odd order `order` (<= kCvMaxOrder) along x,
// then along y, centred on the cells (cell i: node i - r + m with weight C(order, m) 2^-order,
// m = 0..order, r = (order - 1) / 2, nodes past an edge read as the edge node). tmp: (nx - 1) ny
// float4 of scratch; cells: (nx - 1) (ny - 1) float4.
cudaError_t launch_cv_smooth(const double* table, int nx, int ny, int order, float4* tmp, float4* cells,
                             cudaStream_t s);
cudaError_t launch_cv_scatter(const double* xs, const double* ys, const double* yxi, const double* yeta,
                              const float4* nfa, int nx, int ny, int k, int K, int M, float* feats, float* targets,
                              cudaStream_t s);
size_t mlp_norm_scratch_doubles();
cudaError_t launch_mlp_norm(const float* feats, long long n, double* scratch, float* norm, cudaStream_t s);
int mlp_tile_rows();
cudaError_t launch_mlp_grad(const float* theta, const float* norm, const float* feats, const float* targets,
                            long long row0, long long rows, float inv_batch, float* part, cudaStream_t s);
cudaError_t launch_mlp_reduce(const float* part, int nblk, float inv_rows, float* grad, float* loss, cudaStream_t s);
cudaError_t launch_mlp_adam(float* theta, float* m, float* v, const float* part, int nblk, double lr, long long t,
                            float inv_rows, float* losses, long long steps, long long step, cudaStream_t s);
cudaError_t launch_cv_tabulate(const float* theta, const float* norm, const float4* nfa, const float2* nfb, int nx,
                               int ny, int slices, const float* tfrac, double* table, int* status, int sm_count,
                               cudaStream_t s);

cudaError_t launch_rng_draw(uint64_t seed, const uint32_t* ctrs, long long count, uint32_t* words, float* normals,
                            cudaStream_t s);

// Subdomain solve.
struct SolveSys {
    int32_t i0, i1, j0, j1;   // unknown block [i0, i1) x [j0, j1)
    int32_t field;            // 0 xi, 1 eta
    int32_t pad;
};

struct SolveArgs {
    int32_t nx, ny;
    const double* cx;        // face coefficient between (i, j) and (i + 1, j)
    const double* cy;        // face coefficient between (i, j) and (i, j + 1)
    const double* dg;        // diagonal
    const double* rhs0;      // 2 fields: prev / (w Dt)
    const float* cxf;        // single-precision copies for the inner iterations
    const float* cyf;
    const float* dgf;
    const float* dinvf;      // 1 / diagonal (Jacobi)
    double* x[2];            // solution fields (full grid, Dirichlet entries set)
    float* r[2];             // inner residual
    float* p[2];             // search direction (zero on every node that is not an unknown)
    float* q[2];             // A p
    float* d[2];             // inner correction
    const SolveSys* sys;
    int32_t nsys;
    int32_t cluster;         // thread blocks per system
    int32_t max_iter;        // total inner iterations allowed
    int32_t max_outer;       // refinement sweeps allowed
    double rtol;             // on the double-precision residual, relative to ||b||
    float inner_tol;         // inner reduction of ||r|| per refinement sweep
    int32_t* iters;          // per system: total inner iterations (max_iter + 1 when not converged)
    int* status;
};

// Multigrid-preconditioned solves (mg.cu): every subdomain a system of the same
// mx x my unknowns, both fields together.
constexpr int kMgMaxLevels = 10;
struct MgArgs {
    // grid data (as SolveArgs)
    int32_t nx, ny;
    const double* cx;
    const double* cy;
    const double* dg;
    const double* rhs0;
    const float* cxf;
    const float* cyf;
    const float* dgf;
    const float* w;
    double Dt;
    double* x[2];
    const SolveSys* sys;     // subdomain boxes
    int32_t nsys;
    // levels: interior sizes, first element of each level in the level arrays
    int32_t levels, tail;    // number of levels; first level handled inside one block per system
    int32_t mx[kMgMaxLevels], my[kMgMaxLevels];
    long long off[kMgMaxLevels];
    int32_t B0;              // blocks per system for level-0 vectors (partial sums)
    // level arrays (all levels, padded boxes with a zero frame)
    float* D;
    float* CX;               // coefficient between a node and its east neighbour
    float* CY;               // ... and its north neighbour
    float* MS;               // mass term 1 / (w Dt)
    float* U[2];             // V-cycle iterate (level 0: the preconditioned residual z)
    float* F[2];             // V-cycle right-hand side (level 0: the residual r)
    // level-0 Krylov vectors: search direction, product, correction
    float* Pv[2];
    float* Qv[2];
    float* Cv[2];
    float* part;             // [nsys][B0][4] single-precision partial sums
    double* part64;          // [nsys][B0][4] double-precision partial sums
    double* stop2;           // [nsys][2]
    float* rz;               // [nsys][2][2] (r, z) by parity
    float* rr0;              // [nsys][2]
    int32_t* act_o;          // [nsys][2] field still short of rtol
    int32_t* act_i;          // [nsys][2] inner iteration still running
    int32_t* iters;          // [nsys][2]
    int32_t* sys_iters;      // [nsys] inner iterations of the system (max_iter + 1: not converged)
    int32_t* loop;           // [2] pass counters of the graph loops (refinement sweeps, inner iterations)
    int32_t* launches;       // kernels the graph loops' bodies launched in this solve (or null)
    int* status;
    int32_t outer, inner, nu, coarse_sweeps, max_iter;
    double rtol;
    float inner_tol;
};
bool mg_levels(int mx, int my, MgArgs& a);
long long mg_layout(MgArgs& a, int nsys);
cudaError_t launch_mg_setup(const MgArgs& a, cudaStream_t s);
cudaError_t launch_mg_solve(const MgArgs& a, cudaStream_t s);
cudaError_t launch_mg_solve_graph(const MgArgs& a, cudaStream_t s, cudaStream_t s2, cudaStream_t s3);
// the same solve inside one thread-block cluster per subdomain (mgc.cu); mgc_config returns the unknowns
// per thread (0: subdomains too large) and the cluster shape
int mgc_config(const MgArgs& a, int* C, int* rows_max, size_t* smem, int max_upt = 2);
cudaError_t launch_mgc(const MgArgs& a, int upt, int C, int rows_max, size_t smem, cudaStream_t s);

cudaError_t launch_solve_setup(const float* w, const double* prev_xi, const double* prev_eta, int nx, int ny,
                               double Dt, double* cx, double* cy, double* dg, double* rhs0, float* cxf, float* cyf,
                               float* dgf, float* dinvf, cudaStream_t s);
int solve_cluster_size(int nsys, int min_rows, int sm_count);
cudaError_t launch_dirichlet(const double* faces64, const double* prev_xi, const double* prev_eta,
                             const double* iface_xi, const double* iface_eta, const int32_t* iface_idx,
                             int n_iface, int nx, int ny, double* xi_out, double* eta_out, cudaStream_t s);
// The two halves of launch_dirichlet: the faces and the old interior into the
// new fields; the interface values into them (and, if step is non-null, the
// mesh step counter increased by one).
cudaError_t launch_dirichlet_faces(const double* faces64, const double* prev_xi, const double* prev_eta, int nx,
                                   int ny, double* xi_out, double* eta_out, cudaStream_t s);
cudaError_t launch_scatter_iface(const double* iface_xi, const double* iface_eta, const int32_t* iface_idx,
                                 int n_iface, double* xi_out, double* eta_out, uint32_t* step, cudaStream_t s);
cudaError_t launch_pcg(const SolveArgs& a, int upt, int rows_max, int max_mx, cudaStream_t s);
int solve_reg_upt(int max_band_unknowns);
cudaError_t launch_bump_step(uint32_t* step, cudaStream_t s);

}  // namespace sdd
