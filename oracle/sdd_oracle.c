/*
 * sdd_oracle.c -- FP64 CPU oracle for the interface Monte Carlo estimator of
 * Bihlo & Haynes, "A stochastic domain decomposition method for time dependent
 * mesh generation" (arXiv:1402.0266).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links, loads or
 * calls this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark do. It shares no code, header, table or constant
 * generator with the CUDA path.
 *
 * Everything here is a plain, slow restatement of the paper's method, step by
 * step and in the paper's order, in double precision:
 *
 *   - the SDE dX = -(1/w) grad w dt + sqrt(2) dW            (Eq. 7a, with the
 *     Winslow coefficients of Eq. 6: a = I_2, b = -grad w / w)
 *   - the scored estimator xi = E[xi0(X(t)) 1{tau>t}] + E[f(X(tau)) 1{tau<t}]
 *                                                           (Eq. 7b; Eq. 5)
 *   - Euler--Maruyama with dW = sqrt(dt) N(0,1)             (Sec. 4)
 *   - drift from finite differences of w at grid points, bilinear in between
 *                                                           (Sec. 4)
 *   - sub-steps of the mesh step with a boundary test after each (Sec. 4)
 *   - arithmetic means over paths                           (Sec. 4)
 *   - boundary data xi = int_0^x w / int_0^1 w on the faces (Sec. 3, the 1D
 *     version of Eq. 2 along the boundary)
 *
 * Readings where the paper is silent are numbered R1..R19 in the design notes
 * and restated where they are used.
 *
 * Normal variates: the paper only asks for N(0,1) numbers (Sec. 4). The
 * estimator draws them from Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11) through the
 * Box--Muller transform (Box & Muller, 1958), keyed and countered so that the
 * CUDA path can draw the very same stream from its own implementation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11, Sec. 4.2 of that paper): ten rounds of two 32x32->64 */
/* multiplies whose halves are xored with the other counter words and the   */
/* round key; the key is bumped by the Weyl constants between rounds.        */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Stream layout (reading R9): key = (seed_lo, seed_hi), counter = (path,
 * node, draw, mesh step); the node word numbers the nodes of all instances
 * evaluated together. */
static void draw_words(uint64_t seed, uint32_t path, uint32_t node, uint32_t draw, uint32_t step,
                       uint32_t out[4])
{
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {path, node, draw, step};
    orc_philox4x32_10(ctr, key, out);
}

/* Uniforms from a 32-bit word: the low 23 bits m give
 *   u_open0  = (2^23 - m) / 2^23  in (0, 1]   (argument of the logarithm)
 *   u_closed = m / 2^23           in [0, 1)   (angle)
 *   u_pos    = (m + 1) / 2^23     in (0, 1]   (bridge exit test)
 * All three are exact in both single and double precision. */
static double u_open0(uint32_t w) { return (double)(8388608u - (w & 0x7FFFFFu)) / 8388608.0; }
static double u_closed(uint32_t w) { return (double)(w & 0x7FFFFFu) / 8388608.0; }
static double u_pos(uint32_t w) { return (double)((w & 0x7FFFFFu) + 1u) / 8388608.0; }

/* Box--Muller: R = sqrt(-2 ln U1), Z0 = R cos(2 pi U2), Z1 = R sin(2 pi U2). */
void orc_box_muller(uint32_t a, uint32_t b, double* z0, double* z1)
{
    double u1 = u_open0(a);
    double u2 = u_closed(b);
    double r = sqrt(-2.0 * log(u1));
    *z0 = r * cos(2.0 * M_PI * u2);
    *z1 = r * sin(2.0 * M_PI * u2);
}

/* ------------------------------------------------------------------------ */
/* Grid fields. Unit square, nx x ny nodes, node (i, j) at (i hx, j hy),     */
/* row-major with x fastest: f[j * nx + i].                                  */
/* ------------------------------------------------------------------------ */

/* Drift b = -grad w / w at the grid nodes (Eq. 6; Sec. 4: "derivatives in
 * grad w are approximated using finite differences"). Reading R4: second
 * order central differences inside, second order one-sided differences
 * (-3 w0 + 4 w1 - w2) / 2h on the edges. Needs nx, ny >= 3. */
void orc_drift_field(int nx, int ny, const double* w, double* bx, double* by)
{
    double hx = 1.0 / (double)(nx - 1), hy = 1.0 / (double)(ny - 1);
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            double wx, wy;
            if (i == 0)
                wx = (-3.0 * w[j * nx + 0] + 4.0 * w[j * nx + 1] - w[j * nx + 2]) / (2.0 * hx);
            else if (i == nx - 1)
                wx = (3.0 * w[j * nx + nx - 1] - 4.0 * w[j * nx + nx - 2] + w[j * nx + nx - 3]) / (2.0 * hx);
            else
                wx = (w[j * nx + i + 1] - w[j * nx + i - 1]) / (2.0 * hx);
            if (j == 0)
                wy = (-3.0 * w[0 * nx + i] + 4.0 * w[1 * nx + i] - w[2 * nx + i]) / (2.0 * hy);
            else if (j == ny - 1)
                wy = (3.0 * w[(ny - 1) * nx + i] - 4.0 * w[(ny - 2) * nx + i] + w[(ny - 3) * nx + i]) / (2.0 * hy);
            else
                wy = (w[(j + 1) * nx + i] - w[(j - 1) * nx + i]) / (2.0 * hy);
            bx[j * nx + i] = -wx / w[j * nx + i];
            by[j * nx + i] = -wy / w[j * nx + i];
        }
    }
}

/* Bilinear interpolation of a grid field at (x, y) in [0,1]^2 (Sec. 4):
 * cell c = floor(x / h) clamped to [0, n-2], local fractions s, t, and the
 * four corner weights (1-s)(1-t), s(1-t), (1-s)t, st. */
double orc_bilinear(int nx, int ny, const double* f, double x, double y)
{
    double gx = x * (double)(nx - 1), gy = y * (double)(ny - 1);
    int i = (int)floor(gx), j = (int)floor(gy);
    if (i < 0) i = 0;
    if (i > nx - 2) i = nx - 2;
    if (j < 0) j = 0;
    if (j > ny - 2) j = ny - 2;
    double s = gx - (double)i, t = gy - (double)j;
    double f00 = f[j * nx + i], f10 = f[j * nx + i + 1];
    double f01 = f[(j + 1) * nx + i], f11 = f[(j + 1) * nx + i + 1];
    return (1.0 - s) * (1.0 - t) * f00 + s * (1.0 - t) * f10 + (1.0 - s) * t * f01 + s * t * f11;
}

/* Row-major index j (nx - 1) + i of the cell holding (x, y): the cell of
 * orc_bilinear. */
static int64_t cell_index(int nx, int ny, double x, double y)
{
    int i = (int)floor(x * (double)(nx - 1)), j = (int)floor(y * (double)(ny - 1));
    if (i < 0) i = 0;
    if (i > nx - 2) i = nx - 2;
    if (j < 0) j = 0;
    if (j > ny - 2) j = ny - 2;
    return (int64_t)j * (nx - 1) + i;
}

/* Bilinear interpolation of a node table whose values are strided by 4
 * (one of the four components of a control-variate slice). */
static double cv_bilinear(int nx, int ny, const double* f, double x, double y)
{
    double gx = x * (double)(nx - 1), gy = y * (double)(ny - 1);
    int i = (int)floor(gx), j = (int)floor(gy);
    if (i < 0) i = 0;
    if (i > nx - 2) i = nx - 2;
    if (j < 0) j = 0;
    if (j > ny - 2) j = ny - 2;
    double s = gx - (double)i, t = gy - (double)j;
    double f00 = f[4 * (j * nx + i)], f10 = f[4 * (j * nx + i + 1)];
    double f01 = f[4 * ((j + 1) * nx + i)], f11 = f[4 * ((j + 1) * nx + i + 1)];
    return (1.0 - s) * (1.0 - t) * f00 + s * (1.0 - t) * f10 + (1.0 - s) * t * f01 + s * t * f11;
}

/* Face tables. Layout (8 segments, back to back):
 *   xi_left[ny] xi_right[ny] xi_bottom[nx] xi_top[nx]
 *   eta_left[ny] eta_right[ny] eta_bottom[nx] eta_top[nx]
 * left/right faces (x = 0, x = 1) are indexed by j, bottom/top (y = 0, 1) by i.
 * Face numbering used throughout: 0 = left, 1 = right, 2 = bottom, 3 = top. */
static int64_t face_offset(int nx, int ny, int field, int face)
{
    int64_t per_field = 2 * (int64_t)ny + 2 * (int64_t)nx;
    int64_t off = (int64_t)field * per_field;
    if (face >= 1) off += ny;
    if (face >= 2) off += ny;
    if (face >= 3) off += nx;
    return off;
}

int64_t orc_faces_len(int nx, int ny) { return 2 * (2 * (int64_t)ny + 2 * (int64_t)nx); }

/* Cumulative trapezoid of v[0..n-1] on a uniform grid, normalised by the
 * total: out[k] = int_0^{s_k} v / int_0^1 v (the 1D solution of Eq. 2). */
static void cumulative_trapezoid_normalised(int n, const double* v, int64_t stride, double* out)
{
    double acc = 0.0;
    out[0] = 0.0;
    for (int k = 1; k < n; ++k) {
        acc += 0.5 * (v[(int64_t)(k - 1) * stride] + v[(int64_t)k * stride]);
        out[k] = acc;
    }
    for (int k = 0; k < n; ++k) out[k] /= acc;
}

/* Boundary data of Sec. 3 (reading R12): xi = 0 on x = 0, xi = 1 on x = 1,
 * eta = 0 on y = 0, eta = 1 on y = 1; the other faces carry the 1D Winslow
 * solution xi(x) = int_0^x w / int_0^1 w along the face (eta likewise in y). */
void orc_winslow_faces(int nx, int ny, const double* w, double* faces)
{
    double* xl = faces + face_offset(nx, ny, 0, 0);
    double* xr = faces + face_offset(nx, ny, 0, 1);
    double* xb = faces + face_offset(nx, ny, 0, 2);
    double* xt = faces + face_offset(nx, ny, 0, 3);
    double* el = faces + face_offset(nx, ny, 1, 0);
    double* er = faces + face_offset(nx, ny, 1, 1);
    double* eb = faces + face_offset(nx, ny, 1, 2);
    double* et = faces + face_offset(nx, ny, 1, 3);
    for (int j = 0; j < ny; ++j) { xl[j] = 0.0; xr[j] = 1.0; }
    cumulative_trapezoid_normalised(nx, w + 0, 1, xb);
    cumulative_trapezoid_normalised(nx, w + (int64_t)(ny - 1) * nx, 1, xt);
    for (int i = 0; i < nx; ++i) { eb[i] = 0.0; et[i] = 1.0; }
    cumulative_trapezoid_normalised(ny, w + 0, nx, el);
    cumulative_trapezoid_normalised(ny, w + (nx - 1), nx, er);
}

/* Linear interpolation of face `face` of `field` at the tangential
 * coordinate s in [0, 1]. */
double orc_face_value(int nx, int ny, const double* faces, int field, int face, double s)
{
    int n = (face < 2) ? ny : nx;
    const double* v = faces + face_offset(nx, ny, field, face);
    double g = s * (double)(n - 1);
    int k = (int)floor(g);
    if (k < 0) k = 0;
    if (k > n - 2) k = n - 2;
    double f = g - (double)k;
    return (1.0 - f) * v[k] + f * v[k + 1];
}

/* ------------------------------------------------------------------------ */
/* The estimator.                                                           */
/* ------------------------------------------------------------------------ */

typedef struct {
    int nx, ny;
    const double* bx;     /* drift at nodes, nx*ny */
    const double* by;
    const double* xi0;    /* xi at the start of the mesh step, nx*ny */
    const double* eta0;
    const double* faces;  /* face tables, orc_faces_len(nx, ny) */
    /* optional control variate: cv_slices tables of node values, each
     * nx*ny*4 doubles (d/dx, d/dy of the xi model, then of the eta model);
     * NULL or cv_slices = 0 for the plain estimator */
    const double* cv;
    int cv_slices;
    /* 1: cv holds one table of cell values, (nx-1)*(ny-1)*4 doubles, and the
     * model at a point is the value of its cell (the cell of orc_bilinear) */
    int cv_cell;
} orc_problem;

typedef struct {
    double dt;            /* sub-step */
    int32_t K;            /* sub-steps per mesh step, Delta t = K dt */
    int32_t exit_mode;    /* 0 plain test, 1 plain test + Brownian-bridge test, 2 exponential time-stepping */
    uint64_t seed;
    uint32_t step_index;  /* mesh step n */
} orc_params;

/* Exit location and face (reading R6): the segment X_j -> X_{j+1} is cut at
 * the smallest crossing fraction over the violated faces, ties going to the
 * face listed first (left, right, bottom, top). Returns the face and writes
 * the tangential coordinate of the crossing point, clamped to [0, 1]. */
static int plain_exit_point(double x, double y, double xn, double yn, double* tang)
{
    double best = 2.0;
    int face = -1;
    double s;
    if (xn <= 0.0) { s = x / (x - xn); if (s < best) { best = s; face = 0; } }
    if (xn >= 1.0) { s = (1.0 - x) / (xn - x); if (s < best) { best = s; face = 1; } }
    if (yn <= 0.0) { s = y / (y - yn); if (s < best) { best = s; face = 2; } }
    if (yn >= 1.0) { s = (1.0 - y) / (yn - y); if (s < best) { best = s; face = 3; } }
    double t = (face < 2) ? y + best * (yn - y) : x + best * (xn - x);
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    *tang = t;
    return face;
}

/* Brownian-bridge exit test (reading R7; the paper's "more sophisticated
 * boundary tests", Sec. 6). For a diffusion with sigma^2 = 2 that stays inside
 * at both ends of a sub-step, the probability of having touched the half plane
 * behind face k is exp(-2 d0 d1 / (sigma^2 dt)) = exp(-d0 d1 / dt), with d0, d1
 * the distances of X_j, X_{j+1} to that face. The faces are combined as
 * P = 1 - prod_k (1 - p_k). On exit the face with the largest p_k is taken
 * (ties: first listed) and the crossing point is the projection of the
 * sub-step midpoint onto it. */
static int bridge_exit(double x, double y, double xn, double yn, double dt, double u, double* tang)
{
    double d0[4] = {x, 1.0 - x, y, 1.0 - y};
    double d1[4] = {xn, 1.0 - xn, yn, 1.0 - yn};
    double stay = 1.0, pmax = -1.0;
    int face = -1;
    for (int k = 0; k < 4; ++k) {
        double p = exp(-d0[k] * d1[k] / dt);
        stay *= (1.0 - p);
        if (p > pmax) { pmax = p; face = k; }
    }
    double P = 1.0 - stay;
    if (!(u < P)) return -1;
    double t = (face < 2) ? 0.5 * (y + yn) : 0.5 * (x + xn);
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    *tang = t;
    return face;
}

static int on_boundary(double x, double y) { return x <= 0.0 || x >= 1.0 || y <= 0.0 || y >= 1.0; }

/* Face of a boundary point (first of left, right, bottom, top that holds) and
 * its tangential coordinate. */
static int boundary_face(double x, double y, double* tang)
{
    if (x <= 0.0) { *tang = y; return 0; }
    if (x >= 1.0) { *tang = y; return 1; }
    if (y <= 0.0) { *tang = x; return 2; }
    *tang = x;
    return 3;
}

/* Exponential time-stepping, the alternative to fixed Euler--Maruyama steps
 * that Sec. 4 names (after Jansons and Lythe): the sub-step lengths are
 * independent exponential times of mean dt, tau_j = -dt ln u with u =
 * u_open0(word 3) of the sub-step's Philox block (counter (path, node, j,
 * step)), the last one cut at the end of the mesh step T = K dt (and after at
 * most 4K + 16 sub-steps). Each sub-step is the Euler--Maruyama update over
 * tau_j (normals from words 0, 1 scaled by sqrt(2 tau_j)), followed by the
 * plain test and the Brownian-bridge test over tau_j (bridge uniform from word
 * 2). Same outputs as run_path; no control variate. */
static int32_t run_path_exp(const orc_problem* P, const orc_params* Q, uint32_t node, uint32_t path, double x0,
                            double y0, double* score_xi, double* score_eta, double* xe, double* ye, int32_t* code)
{
    const int nx = P->nx, ny = P->ny;
    const double T = (double)Q->K * Q->dt;
    const int32_t cap = 4 * Q->K + 16;
    double x = x0, y = y0, t = 0.0;
    uint32_t words[4];
    for (int32_t j = 0;; ++j) {
        draw_words(Q->seed, path, node, (uint32_t)j, Q->step_index, words);
        double zx, zy;
        orc_box_muller(words[0], words[1], &zx, &zy);
        const double ub = u_pos(words[2]);
        double tau = -Q->dt * log(u_open0(words[3]));
        int last = 0;
        if (t + tau >= T || j + 1 >= cap) {
            tau = T - t;
            last = 1;
        }
        const double bx = orc_bilinear(nx, ny, P->bx, x, y);
        const double by = orc_bilinear(nx, ny, P->by, x, y);
        const double sq = sqrt(2.0 * tau);
        const double xn = x + bx * tau + sq * zx;
        const double yn = y + by * tau + sq * zy;
        if (on_boundary(xn, yn)) {
            double tt;
            const int face = plain_exit_point(x, y, xn, yn, &tt);
            *score_xi = orc_face_value(nx, ny, P->faces, 0, face, tt);
            *score_eta = orc_face_value(nx, ny, P->faces, 1, face, tt);
            *xe = (face == 0) ? 0.0 : (face == 1) ? 1.0 : tt;
            *ye = (face == 2) ? 0.0 : (face == 3) ? 1.0 : tt;
            *code = face;
            return j + 1;
        }
        double tt;
        const int face = bridge_exit(x, y, xn, yn, tau, ub, &tt);
        if (face >= 0) {
            *score_xi = orc_face_value(nx, ny, P->faces, 0, face, tt);
            *score_eta = orc_face_value(nx, ny, P->faces, 1, face, tt);
            *xe = (face == 0) ? 0.0 : (face == 1) ? 1.0 : tt;
            *ye = (face == 2) ? 0.0 : (face == 3) ? 1.0 : tt;
            *code = 4 + face;
            return j + 1;
        }
        x = xn;
        y = yn;
        t += tau;
        if (last) {
            *score_xi = orc_bilinear(nx, ny, P->xi0, x, y);
            *score_eta = orc_bilinear(nx, ny, P->eta0, x, y);
            *xe = x;
            *ye = y;
            *code = -1;
            return j + 1;
        }
    }
}

/* One path of the estimator (Eq. 7b under Euler--Maruyama, Sec. 4). With a
 * control-variate table the scores are Y - sum_j G(j, X_j) . sqrt(2) dW_j,
 * G the table's slice q = floor(j S / K) interpolated bilinearly at X_j. 
 * Returns the number of sub-steps taken; writes the two scores, the end point
 * and the exit code (-1 survived, 0..3 plain exit through face k, 4..7 bridge
 * exit through face k-4). */
/* One path over one mesh step (Eq. 7a, 7b; Sec. 4). With margin non-null the
 * path also reports the smallest distance min(|x|, |1 - x|, |y|, |1 - y|) of
 * its points X_1 .. X_s to the boundary lines, s = min(its sub-steps, upto):
 * how close a decision of the exit test came to going the other way. */
static int32_t run_path(const orc_problem* P, const orc_params* Q, uint32_t node, uint32_t path,
                        double x0, double y0, double* score_xi, double* score_eta,
                        double* xe, double* ye, int32_t* code, double* margin, int32_t upto)
{
    double mrg = 1e300;
    const int nx = P->nx, ny = P->ny;
    const double dt = Q->dt;
    const double sq = sqrt(2.0 * dt); /* sigma = sqrt(2), dW = sqrt(dt) N(0,1) */
    double x = x0, y = y0;
    uint32_t words[4];
    const int cv_on = P->cv && P->cv_slices > 0;
    double cv_sum[2] = {0.0, 0.0};
    double g[4] = {0.0, 0.0, 0.0, 0.0};
    for (int32_t j = 0; j < Q->K; ++j) {
        double zx, zy, ub = 1.0;
        if (Q->exit_mode == 0) {
            /* one Philox block serves the sub-step pair (2m, 2m+1) */
            if ((j & 1) == 0) draw_words(Q->seed, path, node, (uint32_t)(j >> 1), Q->step_index, words);
            if ((j & 1) == 0) orc_box_muller(words[0], words[1], &zx, &zy);
            else orc_box_muller(words[2], words[3], &zx, &zy);
        } else {
            draw_words(Q->seed, path, node, (uint32_t)j, Q->step_index, words);
            orc_box_muller(words[0], words[1], &zx, &zy);
            ub = u_pos(words[2]);
        }
        /* drift at the current point, bilinear from the node values */
        double bx = orc_bilinear(nx, ny, P->bx, x, y);
        double by = orc_bilinear(nx, ny, P->by, x, y);
        /* Euler--Maruyama step */
        double xn = x + bx * dt + sq * zx;
        double yn = y + by * dt + sq * zy;
        /* control variate: the model gradient at X_j (before the increment)
         * times the increment's noise sqrt(2) dW_j, summed over the sub-steps
         * the path takes; its expectation is zero for any model whose value
         * is known before the increment. */
        if (cv_on) {
            if (P->cv_cell) {
                const double* T = P->cv + 4 * cell_index(nx, ny, x, y);
                for (int c = 0; c < 4; ++c) g[c] = T[c];
            } else {
                int q = (int)(((int64_t)j * P->cv_slices) / Q->K);
                if (q > P->cv_slices - 1) q = P->cv_slices - 1;
                const double* T = P->cv + (int64_t)q * 4 * nx * ny;
                /* component c of slice q, node values strided by 4 */
                for (int c = 0; c < 4; ++c) g[c] = cv_bilinear(nx, ny, T + c, x, y);
            }
            for (int c = 0; c < 4; ++c) cv_sum[c >> 1] += g[c] * sq * ((c & 1) ? zy : zx);
        }
        if (margin && j < upto) {
            const double m = fmin(fmin(fabs(xn), fabs(1.0 - xn)), fmin(fabs(yn), fabs(1.0 - yn)));
            mrg = fmin(mrg, m);
            *margin = mrg;
        }
        /* boundary test after every sub-step; the closed boundary counts */
        if (on_boundary(xn, yn)) {
            double t;
            int face = plain_exit_point(x, y, xn, yn, &t);
            *score_xi = orc_face_value(nx, ny, P->faces, 0, face, t);
            *score_eta = orc_face_value(nx, ny, P->faces, 1, face, t);
            *xe = (face == 0) ? 0.0 : (face == 1) ? 1.0 : t;
            *ye = (face == 2) ? 0.0 : (face == 3) ? 1.0 : t;
            *code = face;
            *score_xi -= cv_sum[0];
            *score_eta -= cv_sum[1];
            return j + 1;
        }
        if (Q->exit_mode == 1) {
            double t;
            int face = bridge_exit(x, y, xn, yn, dt, ub, &t);
            if (face >= 0) {
                *score_xi = orc_face_value(nx, ny, P->faces, 0, face, t);
                *score_eta = orc_face_value(nx, ny, P->faces, 1, face, t);
                *xe = (face == 0) ? 0.0 : (face == 1) ? 1.0 : t;
                *ye = (face == 2) ? 0.0 : (face == 3) ? 1.0 : t;
                *code = 4 + face;
                *score_xi -= cv_sum[0];
                *score_eta -= cv_sum[1];
                return j + 1;
            }
        }
        x = xn;
        y = yn;
    }
    /* survived the whole mesh step: score the previous field at X(t) */
    *score_xi = orc_bilinear(nx, ny, P->xi0, x, y);
    *score_eta = orc_bilinear(nx, ny, P->eta0, x, y);
    *xe = x;
    *ye = y;
    *code = -1;
    *score_xi -= cv_sum[0];
    *score_eta -= cv_sum[1];
    return Q->K;
}

/* Mean and standard error of n samples: textbook two-pass formula, sample
 * variance with n - 1 (reading R11), SE = s / sqrt(n). */
static void mean_se(const double* v, int64_t n, double* mean, double* se)
{
    double s = 0.0;
    for (int64_t k = 0; k < n; ++k) s += v[k];
    double m = s / (double)n;
    double q = 0.0;
    for (int64_t k = 0; k < n; ++k) q += (v[k] - m) * (v[k] - m);
    *mean = m;
    *se = (n > 1) ? sqrt(q / (double)(n - 1) / (double)n) : 0.0;
}

/* The interface estimator at a list of nodes. node_ids[k] is the node's
 * index in the Philox counter. stats has 6 doubles per node:
 * mean_xi, mean_eta, se_xi, se_eta, n_exit, path_steps.
 * Per-path records (any of them may be NULL) are laid out node after node,
 * n_paths[k] entries each. Returns 0, or -1 when memory runs out. */
int orc_mc_nodes(const orc_problem* P, const orc_params* Q, int64_t count,
                 const double* xs, const double* ys, const int64_t* n_paths, const uint32_t* node_ids,
                 double* stats,
                 int32_t* rec_steps, int32_t* rec_code, double* rec_xi, double* rec_eta,
                 double* rec_x, double* rec_y)
{
    int64_t rec = 0;
    for (int64_t k = 0; k < count; ++k) {
        int64_t n = n_paths[k];
        double* out = stats + 6 * k;
        if (on_boundary(xs[k], ys[k])) {
            /* a node on the boundary takes its Dirichlet value */
            double t;
            int face = boundary_face(xs[k], ys[k], &t);
            out[0] = orc_face_value(P->nx, P->ny, P->faces, 0, face, t);
            out[1] = orc_face_value(P->nx, P->ny, P->faces, 1, face, t);
            out[2] = 0.0;
            out[3] = 0.0;
            out[4] = (double)n;
            out[5] = 0.0;
            /* every path is on the boundary at time 0: no step, the face's value */
            for (int64_t p = 0; p < n; ++p) {
                if (rec_steps) rec_steps[rec + p] = 0;
                if (rec_code) rec_code[rec + p] = face;
                if (rec_xi) rec_xi[rec + p] = out[0];
                if (rec_eta) rec_eta[rec + p] = out[1];
                if (rec_x) rec_x[rec + p] = xs[k];
                if (rec_y) rec_y[rec + p] = ys[k];
            }
            rec += n;
            continue;
        }
        double* sx = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        double* se = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        if (!sx || !se) { free(sx); free(se); return -1; }
        double exits = 0.0, steps = 0.0;
        for (int64_t p = 0; p < n; ++p) {
            double xe, ye;
            int32_t code;
            int32_t taken = Q->exit_mode == 2
                                ? run_path_exp(P, Q, node_ids[k], (uint32_t)p, xs[k], ys[k], &sx[p], &se[p], &xe, &ye,
                                               &code)
                                : run_path(P, Q, node_ids[k], (uint32_t)p, xs[k], ys[k], &sx[p], &se[p], &xe, &ye,
                                           &code, NULL, 0);
            if (code >= 0) exits += 1.0;
            steps += (double)taken;
            if (rec_steps) rec_steps[rec + p] = taken;
            if (rec_code) rec_code[rec + p] = code;
            if (rec_xi) rec_xi[rec + p] = sx[p];
            if (rec_eta) rec_eta[rec + p] = se[p];
            if (rec_x) rec_x[rec + p] = xe;
            if (rec_y) rec_y[rec + p] = ye;
        }
        if (n > 0) {
            mean_se(sx, n, &out[0], &out[2]);
            mean_se(se, n, &out[1], &out[3]);
        } else {
            out[0] = out[1] = out[2] = out[3] = 0.0;
        }
        out[4] = exits;
        out[5] = steps;
        rec += n;
        free(sx);
        free(se);
    }
    return 0;
}

/* For each (node, path) pair: the path's margin (see run_path) over its first
 * upto[i] sub-steps; fixed sub-steps only (exit_mode 0 or 1). Test support: how
 * close the oracle's path came to the boundary where another implementation's
 * exit decision differs. Returns -1 for exponential time-stepping. */
int orc_path_margins(const orc_problem* P, const orc_params* Q, int64_t count, const double* xs, const double* ys,
                     const uint32_t* node_ids, const uint32_t* paths, const int32_t* upto, double* margins)
{
    if (Q->exit_mode == 2) return -1;
    for (int64_t i = 0; i < count; ++i) {
        double sx, se, xe, ye;
        int32_t code;
        margins[i] = 1e300;
        run_path(P, Q, node_ids[i], paths[i], xs[i], ys[i], &sx, &se, &xe, &ye, &code, &margins[i], upto[i]);
    }
    return 0;
}

/* Raw access to the variates, for the generator's own checks: for each of
 * `count` counters (4 words each) the Philox block and the two normals of
 * its first word pair. */
void orc_draw(uint64_t seed, int64_t count, const uint32_t* ctrs, uint32_t* words_out, double* normals_out)
{
    for (int64_t k = 0; k < count; ++k) {
        uint32_t w[4];
        draw_words(seed, ctrs[4 * k + 0], ctrs[4 * k + 1], ctrs[4 * k + 2], ctrs[4 * k + 3], w);
        for (int q = 0; q < 4; ++q) words_out[4 * k + q] = w[q];
        if (normals_out) {
            orc_box_muller(w[0], w[1], &normals_out[4 * k + 0], &normals_out[4 * k + 1]);
            orc_box_muller(w[2], w[3], &normals_out[4 * k + 2], &normals_out[4 * k + 3]);
        }
    }
}
