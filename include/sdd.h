/*
 * sdd.h -- C ABI of the GB300 interface Monte Carlo library (libsdd.so).
 *
 * The library evaluates, at subdomain-interface nodes, the stochastic
 * (Feynman--Kac) representation of the relaxed Winslow mesh PDE
 *
 *     xi_t = -(1/w) grad w . grad xi + lap xi,   eta likewise          (Eq. 3)
 *
 * from Bihlo & Haynes, "A stochastic domain decomposition method for time
 * dependent mesh generation" (arXiv:1402.0266), and runs the implicit
 * per-subdomain solves that the interface values feed (Sec. 4).
 *
 * Conventions (all entry points):
 *   - The domain is the unit square; a grid has nx x ny nodes, node (i, j) at
 *     (i / (nx-1), j / (ny-1)). Grid arrays are row-major, x fastest:
 *     a[j * nx + i].
 *   - "DEVICE" pointers are CUDA device (or managed) memory on the device the
 *     context was created on; "HOST" pointers are ordinary host memory.
 *     The caller owns every pointer it passes; the library never frees them
 *     and keeps none of them after the call returns.
 *   - Work is enqueued on the context's stream (a cudaStream_t passed as
 *     void*; NULL means the legacy default stream) and runs asynchronously.
 *     Output buffers are valid once the stream has reached the call.
 *   - A rejected argument returns SDD_EINVAL and enqueues nothing. A failed
 *     CUDA call returns SDD_ECUDA; sdd_last_error() then names it. Errors
 *     found on the device are reported by sdd_sync() and by the next call.
 *   - No entry point is thread-safe for one context; distinct contexts may be
 *     used from distinct threads.
 */
#ifndef SDD_H
#define SDD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sdd_ctx sdd_ctx;

typedef enum {
    SDD_OK = 0,
    SDD_EINVAL = 1,   /* argument rejected on the host; nothing enqueued        */
    SDD_ENOMEM = 2,   /* a device or host allocation failed                      */
    SDD_ECUDA = 3,    /* a CUDA runtime call failed                              */
    SDD_ENOCONV = 4,  /* a subdomain solve stopped at max_iter before rtol       */
    SDD_ETIMEOUT = 5, /* a bounded device wait ran out                           */
    SDD_EDEVICE = 6   /* a device-side check failed                              */
} sdd_status;

/* Grid and domain decomposition. The interface lines sit on the grid columns
 * round(k (nx-1) / sub_x), k = 1 .. sub_x-1, and the grid rows
 * round(k (ny-1) / sub_y); a value of 1 means no interface in that direction.
 * nx, ny >= 3; 1 <= sub_x <= nx-1; 1 <= sub_y <= ny-1. */
typedef struct {
    int32_t nx, ny;
    int32_t sub_x, sub_y;
} sdd_grid;

/* A set of evaluation nodes (HOST arrays of `count` entries). Coordinates must
 * lie in [0, 1]; a node on the boundary returns its Dirichlet value with a
 * standard error of 0 and no path steps. n_paths[k] in [1, 2^31 - 1]. The
 * node's position k in the arrays is its index in the random stream (offset
 * by sdd_mc_params.node_word0). */
typedef struct {
    const double* x;
    const double* y;
    const int64_t* n_paths;
    int64_t count;
} sdd_nodes;

/* Per-node results (DEVICE arrays of `count` entries; any may be NULL):
 * the Monte Carlo means of the two scored fields (Sec. 4, "the expected values
 * are then replaced by arithmetic means"), their standard errors
 * s / sqrt(N) with s^2 the N-1 sample variance, the number of paths that left
 * the domain and the number of Euler--Maruyama sub-steps taken in total. */
typedef struct {
    double* mean_xi;
    double* mean_eta;
    double* se_xi;
    double* se_eta;
    int64_t* n_exit;
    int64_t* path_steps;
} sdd_node_stats;

/* Per-path records (DEVICE arrays, one entry per path, node after node in the
 * order of sdd_nodes; any may be NULL): sub-steps taken; exit code (-1 survived
 * the mesh step, 0..3 left through face left/right/bottom/top at a sub-step
 * end, 4..7 left through face k-4 by the bridge test); the two scores; the end
 * point (exit point or X at the end of the step). The paths of a node on the
 * boundary take 0 steps, the code of its face (first of left, right, bottom,
 * top that holds), its Dirichlet values and the node as end point. */
typedef struct {
    int32_t* steps;
    int32_t* code;
    float* score_xi;
    float* score_eta;
    float* x_end;
    float* y_end;
} sdd_path_records;

/* Parameters of one evaluation over a mesh step (Sec. 4).
 *   dt          Euler--Maruyama sub-step, > 0.
 *   Dt          the mesh step; Dt / dt must be an integer K within 1e-9
 *               relative, 1 <= K <= 2^20.
 *   seed        Philox key: key = (seed low 32 bits, seed high 32 bits).
 *   step_index  mesh step number n, the last word of the Philox counter
 *               (counter = (path, node, draw, n)).
 *   exit_mode   0: the paper's boundary test after every sub-step;
 *               1: that test plus a Brownian-bridge test between sub-steps;
 *               2: exponential time-stepping, the alternative Sec. 4 names:
 *                  sub-step j lasts tau_j = -dt ln u (u from word 3 of the
 *                  sub-step's Philox block (path, node, j, n): (2^23 - m)
 *                  2^-23, m its low 23 bits), the last one cut at the end
 *                  of the mesh step (and after 4K + 16 sub-steps); normals
 *                  scaled by sqrt(2 tau_j); both tests over tau_j. Not with
 *                  the control variate (SDD_EINVAL).
 *   block_threads, paths_per_task: launch shape; 0 picks the tuned default.
 *               block_threads in {64, 128, 256, 512}; paths_per_task a
 *               multiple of 32.
 *   node_word0  node word of the first node: node k of the call takes
 *               node_word0 + k as the node word of its Philox counters
 *               (0: the call's own numbering). A caller that splits a node
 *               list into ranges (one range per GPU, say) passes each
 *               range's first index: with the same paths_per_task every
 *               node's results are then those of the whole list, bit for
 *               bit. A batch numbers its nodes from node_word0 on.
 *   zero_map    0: automatic (the autotuner's choice for the node set, else
 *               on; always on with a control variate); 1 on; 2 off. With it
 *               on, the path kernel of a context
 *               reads one shared all-zero drift record wherever the drift
 *               records of a stretch of cells are all zero (w constant
 *               there): the same values, so the same results bit for bit,
 *               with fewer L1 wavefronts and a few more instructions per
 *               sub-step. Batches ignore it. */
typedef struct {
    double dt;
    double Dt;
    uint64_t seed;
    uint32_t step_index;
    int32_t exit_mode;
    int32_t block_threads;
    int32_t paths_per_task;
    uint32_t node_word0;
    int32_t zero_map;
} sdd_mc_params;

/* Create a context on the current CUDA device.
 *   g        grid and decomposition (HOST).
 *   w        DEVICE nx*ny float, the mesh density at the start of the first
 *            mesh step; every value finite and > 0. NULL means w = 1.
 *   xi0,eta0 DEVICE nx*ny double, the computational coordinates at the start
 *            of the first mesh step. NULL means the uniform mesh xi = x,
 *            eta = y (Sec. 3, initial conditions).
 *   stream   cudaStream_t for all work of this context.
 * Boundary data default to the paper's (Sec. 3): xi = 0 / 1 on x = 0 / 1,
 * eta = 0 / 1 on y = 0 / 1, the 1D Winslow solution on the other faces.
 * The inputs are copied; the call waits for the copies. */
sdd_status sdd_init(sdd_ctx** out, const sdd_grid* g, const float* w, const double* xi0, const double* eta0,
                    void* stream);

/* Replace the mesh density (held fixed over a mesh step, Sec. 4). DEVICE
 * nx*ny floats; copied on the context stream. Values are checked on the device
 * (finite and > 0); a violation is reported as SDD_EDEVICE. */
sdd_status sdd_set_w(sdd_ctx* ctx, const float* w);

/* As sdd_set_w, from HOST memory (pinned memory copies asynchronously). */
sdd_status sdd_set_w_host(sdd_ctx* ctx, const float* w);

/* Replace xi and eta at the start of the next mesh step (DEVICE nx*ny doubles). */
sdd_status sdd_set_fields(sdd_ctx* ctx, const double* xi, const double* eta);

/* Boundary data f, g (Sec. 3). faces: DEVICE doubles in the layout
 *   xi_left[ny] xi_right[ny] xi_bottom[nx] xi_top[nx]
 *   eta_left[ny] eta_right[ny] eta_bottom[nx] eta_top[nx]
 * (left/right: x = 0 / 1, indexed by j; bottom/top: y = 0 / 1, indexed by i),
 * linear between nodes. NULL returns to the paper's data, recomputed from w
 * whenever w changes. The values are copied. */
sdd_status sdd_set_boundary(sdd_ctx* ctx, const double* faces);

/* The face data in use (DEVICE output, 2 (2 nx + 2 ny) doubles, layout above). */
sdd_status sdd_get_faces(sdd_ctx* ctx, double* faces);

/* Copy out xi, eta at the start of the next mesh step (DEVICE or HOST outputs,
 * nx*ny doubles each; the _host form waits for the copy). */
sdd_status sdd_get_fields(sdd_ctx* ctx, double* xi, double* eta);
sdd_status sdd_get_fields_host(sdd_ctx* ctx, double* xi, double* eta);

/* The Monte Carlo estimate of Eq. (7b) at the given nodes over one mesh step
 * (Sec. 4): from each node, n_paths Euler--Maruyama paths of
 * dX = -(1/w) grad w dt + sqrt(2) dW (Eq. 7a) with drift from finite
 * differences of w at the nodes and bilinear interpolation between them,
 * K = Dt / dt sub-steps and a boundary test after each; a path that leaves
 * scores the boundary data at its exit point, a path that stays scores the
 * bilinear interpolant of xi, eta at its end point; the means and standard
 * errors go to `out`. Uses the context's current w, xi, eta and face data. */
sdd_status sdd_interface_mc(sdd_ctx* ctx, const sdd_nodes* nodes, const sdd_mc_params* p, sdd_node_stats* out);

/* As sdd_interface_mc, and also write every path's record. */
sdd_status sdd_interface_mc_record(sdd_ctx* ctx, const sdd_nodes* nodes, const sdd_mc_params* p,
                                   sdd_node_stats* out, const sdd_path_records* rec);

/* Control variate (a model of the solution's gradient; the paper notes that
 * Monte Carlo converges slowly, Sec. 4). With it enabled, every path's scores
 * become Y - sum_{j < kappa} G(s_j, X_j) . sqrt(2) dW_j: the model gradient at
 * the start of each sub-step the path takes times the sub-step's Brownian
 * increment. The sum has zero mean for any model (a martingale stopped at a
 * bounded time), so the estimate stays unbiased; a good model shrinks the
 * variance.
 * sdd_cv_set_table gives the model as a table:
 *   grad    DEVICE doubles, shape (slices, ny, nx, 4): at every node the
 *           d/dx, d/dy of the xi model and of the eta model; slice q serves
 *           the sub-steps j with floor(j * slices / K) = q and is interpolated
 *           bilinearly in space. 1 <= slices <= 128, and an estimate with
 *           more slices than sub-steps K fails with SDD_EINVAL. Copied into
 *           the context (the call waits for it). The estimator reads the node
 *           values rounded to half precision (nearest even): the model is the
 *           bilinear interpolation of the rounded values, so one 32-byte
 *           record per cell and slice serves a sub-step.
 * sdd_cv_enable chooses the model of every later estimate and mesh step of
 * the context (batched calls run without one):
 *   SDD_CV_OFF     the plain estimator;
 *   SDD_CV_TABLE   the table last set or tabulated;
 *   SDD_CV_MODEL   the trained network (sdd_cv_train or sdd_cv_set_model),
 *                  tabulated again from the context's w before every
 *                  estimate (inside the mesh step's graph);
 *   SDD_CV_FIELDS  one value per cell from the fields at t_{n-1} (no
 *                  training; over a short mesh step the solution's gradient
 *                  stays close to theirs): the finite-difference gradients of
 *                  xi and eta at the nodes (the table sdd_cv_get_table then
 *                  returns, one slice), smoothed by the binomial filter of
 *                  odd order o along x, then along y, centred on the cells
 *                  (cell i takes node i - r + m with weight C(o, m) 2^-o,
 *                  m = 0..o, r = (o - 1) / 2, nodes past an edge read as the
 *                  edge node), in single precision. G at a point is the value
 *                  of its cell, read at every sub-step. The smoothing removes
 *                  the grid-scale noise that the interface values' Monte
 *                  Carlo error leaves in the fields' differences. o: see
 *                  sdd_cv_set_fields_order. */
#define SDD_CV_OFF 0
#define SDD_CV_TABLE 1
#define SDD_CV_MODEL 2
#define SDD_CV_FIELDS 3
sdd_status sdd_cv_set_table(sdd_ctx* ctx, const double* grad, int32_t slices);
sdd_status sdd_cv_enable(sdd_ctx* ctx, int32_t mode);

/* A copy of the context's current table in the layout of sdd_cv_set_table
 * (DEVICE, slices * ny * nx * 4 doubles; slices as last set or tabulated). */
sdd_status sdd_cv_get_table(sdd_ctx* ctx, double* grad);

/* The smoothing order o of SDD_CV_FIELDS: odd, 1..255, or 0 (the default) for
 * the grid's order 2 floor((m - 1)^2 / 16384) - 1 within 1..33, m the larger
 * side's node count (129: 1, 257: 7, 513: 31, from 1025: 33).
 * SDD_EINVAL for any other value. sdd_cv_fields_order returns the order in
 * use (0 for a null context). */
sdd_status sdd_cv_set_fields_order(sdd_ctx* ctx, int32_t order);
int32_t sdd_cv_fields_order(const sdd_ctx* ctx);

/* With SDD_CV_FIELDS enabled: the cell values from the context's current
 * fields, written to `cells` (DEVICE, (ny - 1) * (nx - 1) * 4 floats, row-major
 * cells, each (d xi/dx, d xi/dy, d eta/dx, d eta/dy)), asynchronously on the
 * context's stream. SDD_EINVAL when the mode is another. */
sdd_status sdd_cv_get_cells(sdd_ctx* ctx, float* cells);

/* ------------------------------------------------------------------------
 * Learned control variate.
 *
 * The model G of the control variate above is the spatial gradient of a
 * network g, fitted to the method's own paths (the paper's estimator is the
 * plain mean of Sec. 4; the network and its training have no counterpart in
 * the paper). One network per field:
 *   features  f = (x, y, t / Dt, w(x, y), r(x, y)) with t the time left in
 *             the mesh step and r = |grad w| / w; w and r are node fields
 *             (finite differences of the drift, Sec. 4) interpolated
 *             bilinearly;
 *   input     z = (f - mu) * s, the standardisation of the training set
 *             (mu the mean, s the inverse population standard deviation, 0
 *             for a feature whose deviation is below 1e-6 max(1, |mu|));
 *   network   g(z) = w3 . tanh(W2 tanh(W1 z + b1) + b2) + b3, widths
 *             5 -> 64 -> 64 -> 1, FP32;
 *   loss      the mean of (g - Y)^2 over a batch of single-path scores Y;
 *   optimiser Adam (beta1 0.9, beta2 0.999, eps 1e-8) with the step decayed
 *             as lr (1 + cos(pi t / T)) / 2 over the T planned updates.
 * A parameter block (DEVICE float) holds the xi network at offset 0 and the
 * eta network at offset SDD_MLP_STRIDE; each is W1 (64 x 5, row-major,
 * [unit][input]), b1 (64), W2 (64 x 64, [unit][input]), b2 (64), w3 (64),
 * b3 (1). A normalisation (DEVICE float) is mu[5] then s[5].
 * All calls below run on the context's stream; those that return values on
 * the host, or that refill context buffers, wait for it. */
#define SDD_MLP_INPUTS 5
#define SDD_MLP_HIDDEN 64
#define SDD_MLP_PARAMS 4609
#define SDD_MLP_STRIDE 4616

/* Initial weights: Glorot-uniform, limit sqrt(6 / (fan_in + fan_out)), and
 * zero biases. Weight p of network f (0 xi, 1 eta) is (2u - 1) limit rounded
 * to float, u = ((word >> 8) + 0.5) 2^-24 with `word` word 0 of the Philox
 * block of key `seed` and counter (p, f, 0x494E4954, 0). theta: DEVICE block
 * of 2 * SDD_MLP_STRIDE floats (the padding is zeroed). */
sdd_status sdd_mlp_init(sdd_ctx* ctx, uint64_t seed, float* theta);

/* Training data generated by the method itself on the context's current w,
 * fields and face data: for every horizon k = 1..K (K = Dt / dt) and
 * m = 0..per_horizon-1, one path of the plain estimator (no control variate)
 * run k sub-steps from a start point uniform in the unit square. Its node
 * word is (k - 1) per_horizon + m, its step word 0xFFFFFFFF; the start point
 * is (u(word 0), u(word 1)) of the Philox block with counter (1, node word,
 * 0, 0xFFFFFFFF), u as for sdd_mlp_init. Row m K + k - 1 of
 * feats (DEVICE float, 5 per row) holds its raw features, with t / Dt = k / K,
 * and of targets (DEVICE float, 2 per row) its two scores.
 * per_horizon * K <= 2^28 rows. */
typedef struct {
    int32_t per_horizon;
    int32_t exit_mode;
    double dt;
    double Dt;
    uint64_t seed;
} sdd_sample_params;

sdd_status sdd_cv_samples(sdd_ctx* ctx, const sdd_sample_params* p, float* feats, float* targets);

/* The standardisation of n feature rows (DEVICE, 5 floats each) into norm
 * (DEVICE, 10 floats): two passes, sums in double. */
sdd_status sdd_mlp_norm(sdd_ctx* ctx, const float* feats, int64_t n, float* norm);

/* Gradient of the mean squared error over rows 0..rows-1 (a positive multiple
 * of 64) for both networks: grad (DEVICE, 2 * SDD_MLP_STRIDE floats, same
 * layout as theta; the padding is not written) and loss (DEVICE, 2 floats, or
 * NULL). targets: DEVICE, 2 floats per row (xi score, eta score). */
sdd_status sdd_mlp_grad(sdd_ctx* ctx, const float* theta, const float* norm, const float* feats,
                        const float* targets, int64_t rows, float* grad, float* loss);

/* Minibatch Adam over the rows in their stored order: epoch after epoch, update
 * t uses rows [(t mod B) batch, (t mod B + 1) batch), B = floor(n / batch);
 * batch a positive multiple of 64. max_steps > 0 stops early (the schedule
 * still spans epochs * B updates). theta (DEVICE) is updated in place;
 * losses (DEVICE, 2 x updates floats, xi then eta, or NULL) receives each
 * update's batch loss before the update. */
typedef struct {
    int32_t epochs;
    int32_t batch;
    double lr;
    int64_t max_steps;
} sdd_train_params;

sdd_status sdd_mlp_train(sdd_ctx* ctx, float* theta, const float* norm, const float* feats, const float* targets,
                         int64_t n, const sdd_train_params* p, float* losses);

/* Tabulate the model of the control variate from a parameter block and
 * normalisation on the context's current w: at every node and every time
 * slice q (1 <= slices <= min(K, 128), slice q serving the sub-steps j with
 * floor(j slices / K) = q, evaluated at the time left at its middle sub-step)
 * the total derivatives d g / dx, d g / dy of both networks, by forward-mode
 * differentiation through the features. The 64 x 64 layer runs on the tensor
 * cores with BF16 operands and FP32 sums. The result replaces the context's
 * table (as sdd_cv_set_table); sdd_cv_enable still decides whether it is used. */
sdd_status sdd_cv_tabulate(sdd_ctx* ctx, const float* theta, const float* norm, int32_t slices, double dt, double Dt);

/* All of the above in one call, into buffers the context owns: samples,
 * standardisation and initial weights (init_seed) -- or, with warm_start and
 * a model already trained, the previous weights and standardisation --
 * training, tabulation (slices 0: one per sub-step up to 128). The control
 * variate is not switched on. info (HOST, may be NULL) receives the times of
 * the three phases, the rows, the updates, the slices and the last batch
 * losses. */
typedef struct {
    sdd_sample_params samples;
    sdd_train_params train;
    int32_t slices;
    int32_t warm_start;
    uint64_t init_seed;
} sdd_cv_train_params;

typedef struct {
    float samples_ms;
    float train_ms;
    float tabulate_ms;
    float loss_xi;
    float loss_eta;
    int32_t slices;
    int64_t rows;
    int64_t steps;
} sdd_cv_train_info;

sdd_status sdd_cv_train(sdd_ctx* ctx, const sdd_cv_train_params* p, sdd_cv_train_info* info);

/* Copies of the model trained by sdd_cv_train (DEVICE; either may be NULL)
 * and of its first `count` batch losses per network (DEVICE, xi then eta).
 * sdd_cv_set_model makes a parameter block and normalisation (DEVICE, copied)
 * the context's model, tabulated at `slices` time slices in SDD_CV_MODEL. */
sdd_status sdd_cv_set_model(sdd_ctx* ctx, const float* theta, const float* norm, int32_t slices);
sdd_status sdd_cv_get_model(sdd_ctx* ctx, float* theta, float* norm);
sdd_status sdd_cv_losses(sdd_ctx* ctx, float* losses, int64_t count);

/* Launch shape of the path kernel: threads per block and paths per task (a
 * task is a node and a run of its paths that one warp computes). */
typedef struct {
    int32_t block_threads;
    int32_t paths_per_task;
    float ms;           /* measured time of one estimate with this shape */
    int32_t zero_map;   /* 1: with the drift's zero map, 2: without (see sdd_mc_params) */
} sdd_launch_shape;

/* Autotuner: time the interface estimate of this node set and these
 * parameters with every candidate launch shape (128, 256, 512 threads x 32 ..
 * 1024 paths per task, 512 only where the kernel takes it; with and without
 * the zero map; outputs discarded; uses the context's current tables),
 * keep the fastest, and use it for later calls on the same node set, K and
 * exit mode that leave block_threads and paths_per_task at 0. Waits for the
 * stream. `out` (HOST, may be NULL) receives the chosen shape. */
sdd_status sdd_autotune(sdd_ctx* ctx, const sdd_nodes* nodes, const sdd_mc_params* p, sdd_launch_shape* out);

/* The interface nodes of the context's decomposition (each once): first the
 * vertical lines left to right, each bottom to top (j = 1 .. ny-2), then the
 * horizontal lines bottom to top, each left to right (i = 1 .. nx-2), skipping
 * nodes already listed. With x, y NULL only the count is returned. HOST
 * outputs of *count entries. */
sdd_status sdd_interface_nodes(sdd_ctx* ctx, double* x, double* y, int64_t* count);

/* Deterministic single-domain solves (Sec. 4): one implicit Euler step of
 * Eq. (3) on every subdomain, in the symmetric form
 *   (xi_ij - xi^{n-1}_ij) / (w_ij Dt) = sum_nb (xi_nb - xi_ij) / (wbar h^2),
 * wbar the average of w over the two nodes, with Dirichlet data from the face
 * data on the outer boundary and from iface_xi / iface_eta (DEVICE, one
 * double per interface node in the order of sdd_interface_nodes) on the
 * interfaces. Solved in double precision by Jacobi-preconditioned conjugate
 * gradients to ||r|| <= rtol ||b|| or max_iter iterations.
 * Outputs xi_out, eta_out: DEVICE nx*ny doubles (full fields). iters_out
 * (HOST, may be NULL): the largest iteration count over the systems; asking
 * for it waits for the solve. The context's fields are not changed.
 * Non-convergence returns SDD_ENOCONV when iters_out is given, else it is
 * reported by sdd_sync(). */
sdd_status sdd_subdomain_solve(sdd_ctx* ctx, double Dt, const double* iface_xi, const double* iface_eta,
                               double rtol, int32_t max_iter, double* xi_out, double* eta_out,
                               int32_t* iters_out);

/* Key points (Sec. 4) and interface fill (Sec. 5). With key points on, each
 * mesh step of sdd_step estimates only at the key points of the interface
 * lines and fills the other interface nodes, line by line, by monotone PCHIP
 * interpolation (Fritsch-Carlson, Fritsch-Butland derivatives) through the
 * line's two boundary values (face data) and the key points' estimates; the
 * filled nodes report a standard error of 0 and no path steps. Key points of
 * a line (rho = 1 / w at its nodes t = 0 .. n - 1, t = 0, n - 1 on the
 * boundary): the positions t in 2 .. n - 3 where D1(t) = rho(t+1) - rho(t-1)
 * or D2(t) = (rho(t+1) - rho(t)) - (rho(t) - rho(t-1)) (computed in double
 * precision for t = 1 .. n - 2) has a local extremum (p(t) > p(t-1) and
 * p(t) >= p(t+1), or the mirror) of size |p(t)| >= max |p| / 100, every
 * crossing of a vertical and a horizontal line, and, with spacing > 0, every
 * position t with t mod spacing = 0 (the mesh also moves where rho is flat
 * along a line; 0 keeps the extrema alone).
 * sdd_keypoint_mask writes the mask of the context's current w (DEVICE, one
 * byte per interface node in the order of sdd_interface_nodes) on the
 * context's stream. */
sdd_status sdd_set_keypoints(sdd_ctx* ctx, int32_t on, int32_t spacing);
sdd_status sdd_keypoint_mask(sdd_ctx* ctx, uint8_t* mask);

/* The interface fill of a mesh step with key points, on given values:
 * values_xi, values_eta (DEVICE, one double per interface node in the order of
 * sdd_interface_nodes) keep their entries where `mask` (DEVICE, one byte per
 * interface node) is nonzero, and every other entry is overwritten, line by
 * line, by the PCHIP interpolant (as above) through the line's two face values
 * of the context's current w and its masked entries. A crossing of a vertical
 * and a horizontal line that the mask leaves out is filled along its vertical
 * line. Enqueued on the context's stream; SDD_EINVAL for null arguments. */
sdd_status sdd_keypoint_fill(sdd_ctx* ctx, const uint8_t* mask, double* values_xi, double* values_eta);

/* The solver of the subdomain systems (sdd_subdomain_solve and sdd_step).
 * The paper uses LU (Sec. 4); the GPU solves the same symmetric system either
 * directly or by conjugate gradients refined in double precision to rtol:
 *   SDD_SOLVER_DIRECT  a banded L D L^T factorisation per subdomain (one block,
 *                      single precision) inside an iterative refinement in
 *                      double precision to rtol (available when every
 *                      subdomain has at most 32 columns and its band fits
 *                      200 KB of shared memory, e.g. 31 x 31; else
 *                      SDD_EINVAL; status bit when rtol is missed, and
 *                      after a pivot that is not positive the subdomain's
 *                      fields keep their previous values); slower than
 *                      Jacobi-PCG on these sizes, so never chosen automatically;
 *   SDD_SOLVER_JACOBI  Jacobi preconditioner; one thread-block cluster per
 *                      subdomain, register-resident when the subdomain fits;
 *   SDD_SOLVER_MG      a geometric multigrid V-cycle as preconditioner
 *                      (available when every subdomain has the same odd
 *                      sizes that halve, (m - 1) / 2, down to a box of at
 *                      most 64 unknowns; else SDD_EINVAL);
 *   SDD_SOLVER_AUTO    multigrid where it is available and the subdomains are
 *                      too large for the register-resident Jacobi kernel or
 *                      hold at least 10,000 unknowns; else Jacobi.
 * With multigrid, max_iter caps the inner iterations: inside sdd_step's graph
 * the refinement sweeps and inner iterations are graph while-loops that stop
 * once every field has converged (at most 30 inner iterations per sweep and
 * 8 sweeps, within max_iter); a direct sdd_subdomain_solve runs a fixed 5 x 6.
 * sdd_solver_in_use returns the solver the next solve will use (1 Jacobi,
 * 2 multigrid, 3 direct). */
#define SDD_SOLVER_AUTO 0
#define SDD_SOLVER_JACOBI 1
#define SDD_SOLVER_MG 2
#define SDD_SOLVER_DIRECT 3
sdd_status sdd_set_solver(sdd_ctx* ctx, int32_t solver);
int32_t sdd_solver_in_use(const sdd_ctx* ctx);

/* One mesh step t_{n-1} -> t_n (Sec. 4): the interface estimate at every
 * interface node with paths_per_node paths, the subdomain solves with those
 * values, then xi, eta advance and the step counter n (the Philox counter's
 * last word) increases by one. The sequence is recorded once into a CUDA
 * graph and replayed while the parameters stay the same. The interface
 * statistics of the step can be read with sdd_last_interface_stats.
 *
 * Pipelining: where the subdomain solve's iterations are one kernel launch
 * (the cluster multigrid or Jacobi-PCG kernels) and the paths do not read the
 * fields (no SDD_CV_FIELDS), the iterations of step n's solve run inside step
 * n + 1's graph, beside its paths; the paths that survive step n + 1 are
 * scored once they are done. Every call that reads or writes the fields
 * (sdd_get_fields, sdd_set_fields, sdd_interface_mc, sdd_subdomain_solve,
 * sdd_cv_samples, sdd_cv_train, sdd_autotune, sdd_sync, the batch calls) or
 * changes the step's parameters first enqueues the pending iterations, and
 * sdd_flush does so alone. The results are those of the unpipelined
 * sequence; only the order of the floating-point sums over a task's paths
 * differs. */
typedef struct {
    double dt;
    double Dt;
    uint64_t seed;
    int64_t paths_per_node;
    int32_t exit_mode;
    int32_t max_iter;
    double rtol;
    int32_t tune;   /* nonzero: autotune the path kernel's launch shape for this step (see sdd_autotune) */
    int32_t pad;
} sdd_step_params;

sdd_status sdd_step(sdd_ctx* ctx, const sdd_step_params* p);

/* Statistics of the interface nodes from the last sdd_step (DEVICE outputs in
 * the order of sdd_interface_nodes). */
sdd_status sdd_last_interface_stats(sdd_ctx* ctx, sdd_node_stats* out);

/* Facts about the last sdd_step, for profiling (waits for the stream):
 * the number of kernel launches in the step graph and the device time of the
 * step's parts, taken with events recorded inside the graph. */
typedef struct {
    int32_t kernel_nodes;  /* kernels the last step launched (the graph's kernel nodes
                              and the kernels its solver loops ran)                */
    float paths_ms;        /* the path kernel                                    */
    float estimate_ms;     /* the whole interface estimate (tables, paths, means) */
    float solve_ms;        /* the subdomain solves (pipelined: this step's set-up and
                              the previous step's iterations, run beside the paths) */
    float step_ms;         /* the whole step                                     */
} sdd_step_info;

sdd_status sdd_last_step_info(sdd_ctx* ctx, sdd_step_info* out);

/* Mesh step counter n. */
sdd_status sdd_set_step_index(sdd_ctx* ctx, uint32_t n);
uint32_t sdd_get_step_index(const sdd_ctx* ctx);

/* Allow (on != 0, the default) or forbid pipelined mesh steps (see sdd_step;
 * Sec. 4 orders a mesh step as the interface estimate, then the subdomain
 * solves, which both settings keep); enqueues any pending iterations first and
 * drops the step graphs when the setting changes. SDD_EINVAL for a null
 * context, else the status of enqueuing the pending iterations.
 * sdd_pipeline_in_use: 1 if the current step graphs are pipelined (known after
 * the first sdd_step with these parameters), 0 otherwise or for a null context. */
sdd_status sdd_set_pipeline(sdd_ctx* ctx, int32_t on);
int32_t sdd_pipeline_in_use(const sdd_ctx* ctx);

/* Enqueue the pending iterations of the last pipelined mesh step's solve
 * (asynchronous, on the context stream; SDD_OK when none is pending, SDD_EINVAL
 * for a null context, SDD_ECUDA if the launch fails). After it the fields of
 * the last step are complete once the stream reaches it; a non-convergence of
 * those iterations is reported by the next sdd_sync. */
sdd_status sdd_flush(sdd_ctx* ctx);

/* Enqueue any pending solve (sdd_flush), wait for the context stream and
 * return the first device-side error since the last sdd_sync (SDD_EDEVICE,
 * SDD_ENOCONV, SDD_ETIMEOUT) or SDD_OK. */
sdd_status sdd_sync(sdd_ctx* ctx);

/* Last error message of the context (static storage until the next call). */
const char* sdd_last_error(const sdd_ctx* ctx);

/* Release the context and everything it allocated (waits for its stream). */
void sdd_destroy(sdd_ctx* ctx);

/* Many mesh instances through one launch (the paper's method applied to
 * independent problems at once; Sec. 4 "fully parallel"). A batch groups
 * contexts (each its own grid, w, fields and face data) created on the same
 * device; the contexts must outlive the batch and must not be destroyed or
 * re-initialised while it exists. Work is enqueued on the batch's stream;
 * order it after earlier work on the contexts' streams (e.g. use one stream).
 * In a batch the node word of the Philox counter numbers the nodes of all
 * instances in order: instance k's node j is node (sum of the counts of the
 * instances before k) + j. */
typedef struct sdd_batch sdd_batch;

sdd_status sdd_batch_create(sdd_batch** out, sdd_ctx* const* ctxs, int32_t count, void* stream);

/* The interface estimate of every instance in one persistent launch: nodes[k]
 * and out[k] (count entries each, as in sdd_interface_mc) belong to
 * instance k; dt, Dt, seed and step_index are shared. */
sdd_status sdd_batch_interface_mc(sdd_batch* b, const sdd_nodes* nodes, const sdd_mc_params* p, sdd_node_stats* out);

/* One mesh step of every instance (as sdd_step, paths_per_node paths at every
 * interface node of each instance): the field tables of each instance, one
 * persistent path-kernel launch over all instances' interface nodes, then each
 * instance's subdomain solves; recorded once into a CUDA graph and replayed.
 * The batch's step counter (shared by the instances) advances by one. */
sdd_status sdd_batch_step(sdd_batch* b, const sdd_step_params* p);

/* As sdd_autotune for the batched estimate (nodes: one list per instance). */
sdd_status sdd_batch_autotune(sdd_batch* b, const sdd_nodes* nodes, const sdd_mc_params* p, sdd_launch_shape* out);

/* As sdd_last_step_info, for the last sdd_batch_step (waits for the stream). */
sdd_status sdd_batch_last_step_info(sdd_batch* b, sdd_step_info* out);

sdd_status sdd_batch_set_step_index(sdd_batch* b, uint32_t n);

/* Wait for the batch stream; then sdd_sync of every instance. */
sdd_status sdd_batch_sync(sdd_batch* b);
const char* sdd_batch_last_error(const sdd_batch* b);

/* Release the batch (not its contexts). */
void sdd_batch_destroy(sdd_batch* b);

/* The inputs of one mesh step, for entry points that take them directly
 * (DEVICE arrays of nx*ny entries, row-major): w (float), xi and eta (double);
 * faces: DEVICE face data in the layout of sdd_set_boundary, or NULL for the
 * paper's data computed from w. */
typedef struct {
    int32_t nx, ny;
    const float* w;
    const double* xi;
    const double* eta;
    const double* faces;
} sdd_fields;

/* The interface estimate of sdd_interface_mc without any allocation: no
 * context, no cudaMalloc or cudaFree, nothing allocated on the host heap.
 * This entry point has no counterpart in the paper; it exists for callers
 * that are not allowed to allocate device memory once they are running (a
 * real-time loop, a host application that hands out only fixed buffers, a
 * plugin given pointers and a stream). They pass the inputs (`f`, DEVICE;
 * `nodes`, HOST, as in sdd_interface_mc) and the output arrays (`out`,
 * DEVICE); all working memory -- the cell tables, the face data, the node
 * and task lists, the per-task sums and the work counter -- is one static
 * device array of sdd_static_scratch_bytes() bytes that every GPU loading the
 * library holds until the process exits.
 * Limits (else SDD_EINVAL, nothing enqueued): nx, ny <= 257; at most 8192
 * nodes and 65536 tasks (paths_per_task as requested, else chosen to fit).
 * The first call on a device looks up the array's device address (so make it
 * before any stream capture). Every call shares the array: calls whose work
 * can overlap on the GPU (different streams or host threads) race and must
 * not be made; one call at a time per process. Results equal those of
 * sdd_interface_mc for the same inputs, parameters and paths_per_task.
 * Work is enqueued on `stream`.
 * Device errors: `status_out` (DEVICE, one int32, caller-owned) receives the
 * call's device status word once the call's work has run on `stream` (0 when
 * none; bit 0 set when w is not finite and positive somewhere, and then the
 * outputs are meaningless); the caller reads it after its own stream sync.
 * With status_out = NULL the call instead waits for `stream` and returns
 * SDD_EDEVICE when the word is nonzero. */
sdd_status sdd_interface_mc_static(const sdd_fields* f, const sdd_nodes* nodes, const sdd_mc_params* p,
                                   sdd_node_stats* out, int32_t* status_out, void* stream);

/* Size in bytes of the static array used by sdd_interface_mc_static. */
int64_t sdd_static_scratch_bytes(void);

/* The variates of the estimator, for checking: for each counter
 * (path, node, draw, step) in `ctrs` (DEVICE, 4 uint32 per entry), the Philox
 * block (`words`, DEVICE, 4 uint32 per entry) and the four normals of its two
 * Box--Muller pairs, unscaled (`normals`, DEVICE, 4 float per entry; may be
 * NULL). key = (seed low 32 bits, seed high 32 bits). */
sdd_status sdd_rng_draw(uint64_t seed, const uint32_t* ctrs, int64_t count, uint32_t* words, float* normals,
                        void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SDD_H */
