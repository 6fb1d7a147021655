/*
 * Plain FP64 CPU oracle for the one-fluid pressure projection.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may call,
 * link or load this file: it exists so that tests, the smoke check and the
 * benchmark's CPU baseline can compare the CUDA path against a slow, obviously
 * correct restatement of the paper.  It shares no code, header, table or
 * helper with the CUDA path.
 *
 * What it computes (paper references are to the PARIS paper, arXiv 2012.11744):
 *   1. cell density rho = rho1*C + rho2*(1-C)                       (Eq. muH)
 *   2. face coefficient beta_f = 1/rho_f, rho_f = mean of the two cells;
 *      wall faces get beta_f = 0 ("Neumann by coefficient zeroing", Sec. 3.8)
 *   3. b = (grad^h . u*) / dt                        (Eqs. cont2, incompdisc3)
 *   4. the operator L p = grad^h . (beta grad^h p) assembled as an explicit
 *      CSR matrix of -L (the A1..A7 system form of Sec. 3.7.1 scaled by -1/tau)
 *   5. unpreconditioned conjugate gradients on (-L) x = -b         (Eq. poisson)
 *   6. u = u* - dt beta_f (grad^h p)_f                                (Eq. fotm)
 *   7. the adjoint of steps 1-6 for a loss of the corrected velocity.
 *
 * Layout (same convention as the input generator): cells (i,j,k) with linear
 * index (k*ny + j)*nx + i; face arrays store face "i-1/2" at index i and have
 * n entries along a periodic axis, n+1 along a wall axis (entries 0 and n are
 * the walls).  All arithmetic is IEEE double; the file is compiled with
 * -ffp-contract=off so that no fused multiply-add changes the rounding.
 * Reductions use a fixed block decomposition so results do not depend on the
 * number of OpenMP threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PERIODIC 0
#define OR_WALL 1

typedef struct {
    int nx, ny, nz;
    double h;
    int bc[3]; /* per axis x, y, z: OR_PERIODIC or OR_WALL */
} or_grid;

/* ------------------------------------------------------------ indexing --- */

static int64_t cell_index(const or_grid* g, int i, int j, int k) {
    return ((int64_t)k * g->ny + j) * g->nx + i;
}

/* number of faces of the face array normal to `axis` along each axis */
static void face_dims(const or_grid* g, int axis, int d[3]) {
    d[0] = g->nx; d[1] = g->ny; d[2] = g->nz;
    if (g->bc[axis] == OR_WALL) d[axis] += 1;
}

static int64_t face_index(const or_grid* g, int axis, int i, int j, int k) {
    int d[3];
    face_dims(g, axis, d);
    return ((int64_t)k * d[1] + j) * d[0] + i;
}

int64_t oracle_face_count(const or_grid* g, int axis) {
    int d[3];
    face_dims(g, axis, d);
    return (int64_t)d[0] * d[1] * d[2];
}

/* The two cells on either side of face (i,j,k) of the array normal to `axis`:
 * the face lies between cell index-1 (left, "minus") and index (right, "plus")
 * along `axis`.  Returns 0 for a wall face (no cell on one side). */
static int face_cells(const or_grid* g, int axis, int i, int j, int k,
                      int64_t* left, int64_t* right) {
    int n[3] = {g->nx, g->ny, g->nz};
    int c[3] = {i, j, k};
    int lo[3] = {i, j, k};
    lo[axis] = c[axis] - 1;
    if (g->bc[axis] == OR_WALL) {
        if (c[axis] == 0 || c[axis] == n[axis]) return 0;
    } else {
        if (lo[axis] < 0) lo[axis] += n[axis];
    }
    *left = cell_index(g, lo[0], lo[1], lo[2]);
    *right = cell_index(g, c[0], c[1], c[2]);
    return 1;
}

/* Face index of the face on side `side` (-1 or +1) of cell (i,j,k) along
 * `axis`; along a periodic axis the + face of the last cell is face 0. */
static int64_t cell_face(const or_grid* g, int axis, int side, int i, int j, int k) {
    int n[3] = {g->nx, g->ny, g->nz};
    int c[3] = {i, j, k};
    if (side > 0) {
        c[axis] += 1;
        if (g->bc[axis] == OR_PERIODIC && c[axis] == n[axis]) c[axis] = 0;
    }
    return face_index(g, axis, c[0], c[1], c[2]);
}

static int is_wall_face(const or_grid* g, int axis, int side, int i, int j, int k) {
    int n[3] = {g->nx, g->ny, g->nz};
    int c[3] = {i, j, k};
    if (g->bc[axis] != OR_WALL) return 0;
    return (side < 0 && c[axis] == 0) || (side > 0 && c[axis] == n[axis] - 1);
}

/* neighbour cell across side `side` of cell (i,j,k) along `axis`; assumes the
 * face is not a wall face */
static int64_t neighbour(const or_grid* g, int axis, int side, int i, int j, int k) {
    int n[3] = {g->nx, g->ny, g->nz};
    int c[3] = {i, j, k};
    c[axis] += side;
    if (c[axis] < 0) c[axis] += n[axis];
    if (c[axis] >= n[axis]) c[axis] -= n[axis];
    return cell_index(g, c[0], c[1], c[2]);
}

/* ------------------------------------------------- deterministic sums --- */

#define OR_BLOCK 4096

static double det_dot(int64_t n, const double* a, const double* b) {
    int64_t nb = (n + OR_BLOCK - 1) / OR_BLOCK;
    double* part = (double*)malloc(sizeof(double) * (nb > 0 ? nb : 1));
    #pragma omp parallel for schedule(static)
    for (int64_t blk = 0; blk < nb; ++blk) {
        int64_t s = blk * OR_BLOCK, e = s + OR_BLOCK < n ? s + OR_BLOCK : n;
        double acc = 0.0;
        for (int64_t q = s; q < e; ++q) acc += a[q] * b[q];
        part[blk] = acc;
    }
    double t = 0.0;
    for (int64_t blk = 0; blk < nb; ++blk) t += part[blk];
    free(part);
    return t;
}

static double det_sum(int64_t n, const double* a) {
    int64_t nb = (n + OR_BLOCK - 1) / OR_BLOCK;
    double* part = (double*)malloc(sizeof(double) * (nb > 0 ? nb : 1));
    #pragma omp parallel for schedule(static)
    for (int64_t blk = 0; blk < nb; ++blk) {
        int64_t s = blk * OR_BLOCK, e = s + OR_BLOCK < n ? s + OR_BLOCK : n;
        double acc = 0.0;
        for (int64_t q = s; q < e; ++q) acc += a[q];
        part[blk] = acc;
    }
    double t = 0.0;
    for (int64_t blk = 0; blk < nb; ++blk) t += part[blk];
    free(part);
    return t;
}

double oracle_sum(int64_t n, const double* a) { return det_sum(n, a); }
double oracle_dot(int64_t n, const double* a, const double* b) { return det_dot(n, a, b); }

/* x <- x - mean(x) */
void oracle_remove_mean(int64_t n, double* x) {
    double m = det_sum(n, x) / (double)n;
    #pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < n; ++q) x[q] -= m;
}

/* Projection onto the complement of the null space of the operator with
 * solid cells (Sec. 3.8): every coefficient of a solid cell is zeroed, so each
 * solid cell is a null vector on its own, and the constants on the fluid
 * cells are the other one (a connected fluid region).  fluid[c] = 1 outside
 * the solid (the paper's flag s), 0 inside; NULL means no solid, and the
 * projection is the mean removal above.  Fluid cells lose their mean over
 * the fluid cells, solid cells are set to 0. */
void oracle_null_project(int64_t n, double* x, const unsigned char* fluid) {
    if (!fluid) {
        oracle_remove_mean(n, x);
        return;
    }
    int64_t nb = (n + OR_BLOCK - 1) / OR_BLOCK;
    double* part = (double*)malloc(sizeof(double) * 2 * (nb > 0 ? nb : 1));
    #pragma omp parallel for schedule(static)
    for (int64_t blk = 0; blk < nb; ++blk) {
        int64_t s = blk * OR_BLOCK, e = s + OR_BLOCK < n ? s + OR_BLOCK : n;
        double acc = 0.0, cnt = 0.0;
        for (int64_t q = s; q < e; ++q)
            if (fluid[q]) { acc += x[q]; cnt += 1.0; }
        part[2 * blk] = acc;
        part[2 * blk + 1] = cnt;
    }
    double t = 0.0, c = 0.0;
    for (int64_t blk = 0; blk < nb; ++blk) { t += part[2 * blk]; c += part[2 * blk + 1]; }
    free(part);
    double m = c > 0.0 ? t / c : 0.0;
    #pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < n; ++q) x[q] = fluid[q] ? x[q] - m : 0.0;
}

/* ------------------------------------------------ face coefficients --- */

/* Eq. muH gives the cell density from the volume fraction; the paper builds
 * the Poisson coefficients from interpolations of 1/rho (Sec. 3.7.1).  Here
 * the face density is the arithmetic mean of the two cells and beta = 1/rho_f.
 * Wall faces get beta = 0: the link flags of Sec. 3.8 zero those coefficients. */
void oracle_face_coeffs(const or_grid* g, const double* C, double rho1, double rho2,
                        double* bx, double* by, double* bz) {
    double* beta[3] = {bx, by, bz};
    for (int axis = 0; axis < 3; ++axis) {
        int d[3];
        face_dims(g, axis, d);
        #pragma omp parallel for schedule(static)
        for (int k = 0; k < d[2]; ++k)
            for (int j = 0; j < d[1]; ++j)
                for (int i = 0; i < d[0]; ++i) {
                    int64_t L, R, f = face_index(g, axis, i, j, k);
                    if (!face_cells(g, axis, i, j, k, &L, &R)) {
                        beta[axis][f] = 0.0;
                        continue;
                    }
                    double rhoL = rho1 * C[L] + rho2 * (1.0 - C[L]);
                    double rhoR = rho1 * C[R] + rho2 * (1.0 - C[R]);
                    double rhof = 0.5 * (rhoL + rhoR);
                    beta[axis][f] = 1.0 / rhof;
                }
    }
}

/* --------------------------------------------------------- divergence --- */

/* (grad^h . u)_c = sum over the three axes of (u_{+face} - u_{-face}) / h
 * (Eqs. cont2 and incompdisc3: outward normal velocities summed).  Wall faces
 * carry no flux (the velocity there is blocked, Sec. 3.8), whatever value the
 * array holds.  Returns rhs = div / dt. */
void oracle_divergence(const or_grid* g, const double* u, const double* v, const double* w,
                       double dt, double* rhs) {
    const double* vel[3] = {u, v, w};
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                double div = 0.0;
                for (int axis = 0; axis < 3; ++axis) {
                    double up = is_wall_face(g, axis, +1, i, j, k) ? 0.0
                              : vel[axis][cell_face(g, axis, +1, i, j, k)];
                    double um = is_wall_face(g, axis, -1, i, j, k) ? 0.0
                              : vel[axis][cell_face(g, axis, -1, i, j, k)];
                    div += (up - um) / g->h;
                }
                rhs[cell_index(g, i, j, k)] = div / dt;
            }
}

/* ----------------------------------------------------- CSR assembly --- */

typedef struct {
    int64_t n;
    int64_t* rowptr;
    int32_t* col;
    double* val;
} or_csr;

/* Assemble A = -L = -(D B G) as CSR: for every non-wall face of a cell with
 * coefficient beta, the diagonal gains beta/h^2 and the neighbour's column
 * gets -beta/h^2.  This is the paper's A1..A7 system form (Sec. 3.7.1, with
 * A7 = sum of the six neighbour coefficients and the symmetry relations
 * A2_i = A1_{i+1} etc. following from sharing one beta per face) multiplied
 * by -1/tau.  Columns are sorted and duplicates summed, which matters when a
 * periodic axis has length 1 or 2 (both neighbours are the same cell). */
or_csr* oracle_assemble(const or_grid* g, const double* bx, const double* by, const double* bz) {
    const double* beta[3] = {bx, by, bz};
    int64_t n = (int64_t)g->nx * g->ny * g->nz;
    or_csr* A = (or_csr*)calloc(1, sizeof(or_csr));
    A->n = n;
    A->rowptr = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
    A->col = (int32_t*)malloc(sizeof(int32_t) * 7 * n);
    A->val = (double*)malloc(sizeof(double) * 7 * n);
    int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * n);
    double ih2 = 1.0 / (g->h * g->h);
    /* each row is written into its own 7-slot segment, then compacted */
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                int64_t c = cell_index(g, i, j, k);
                int32_t cols[7];
                double vals[7];
                int m = 0;
                cols[m] = (int32_t)c; vals[m] = 0.0; ++m;
                for (int axis = 0; axis < 3; ++axis)
                    for (int side = -1; side <= 1; side += 2) {
                        if (is_wall_face(g, axis, side, i, j, k)) continue;
                        double b = beta[axis][cell_face(g, axis, side, i, j, k)] * ih2;
                        int64_t nb = neighbour(g, axis, side, i, j, k);
                        vals[0] += b;
                        int found = 0;
                        for (int q = 0; q < m; ++q)
                            if (cols[q] == (int32_t)nb) { vals[q] -= b; found = 1; break; }
                        if (!found) { cols[m] = (int32_t)nb; vals[m] = -b; ++m; }
                    }
                /* insertion sort by column */
                for (int a = 1; a < m; ++a) {
                    int32_t cc = cols[a]; double vv = vals[a]; int b2 = a - 1;
                    while (b2 >= 0 && cols[b2] > cc) { cols[b2 + 1] = cols[b2]; vals[b2 + 1] = vals[b2]; --b2; }
                    cols[b2 + 1] = cc; vals[b2 + 1] = vv;
                }
                for (int q = 0; q < m; ++q) { A->col[7 * c + q] = cols[q]; A->val[7 * c + q] = vals[q]; }
                cnt[c] = m;
            }
    A->rowptr[0] = 0;
    for (int64_t c = 0; c < n; ++c) A->rowptr[c + 1] = A->rowptr[c] + cnt[c];
    /* compact in place: rows only move towards the front */
    for (int64_t c = 0; c < n; ++c) {
        int64_t dst = A->rowptr[c];
        for (int64_t q = 0; q < cnt[c]; ++q) {
            A->col[dst + q] = A->col[7 * c + q];
            A->val[dst + q] = A->val[7 * c + q];
        }
    }
    free(cnt);
    return A;
}

void oracle_csr_free(or_csr* A) {
    if (!A) return;
    free(A->rowptr); free(A->col); free(A->val); free(A);
}

int64_t oracle_csr_nnz(const or_csr* A) { return A->rowptr[A->n]; }

void oracle_csr_export(const or_csr* A, int64_t* rowptr, int32_t* col, double* val) {
    memcpy(rowptr, A->rowptr, sizeof(int64_t) * (A->n + 1));
    memcpy(col, A->col, sizeof(int32_t) * A->rowptr[A->n]);
    memcpy(val, A->val, sizeof(double) * A->rowptr[A->n]);
}

/* y = A x */
void oracle_csr_matvec(const or_csr* A, const double* x, double* y) {
    #pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < A->n; ++r) {
        double acc = 0.0;
        for (int64_t q = A->rowptr[r]; q < A->rowptr[r + 1]; ++q) acc += A->val[q] * x[A->col[q]];
        y[r] = acc;
    }
}

/* ---------------------------------------------------------------- CG --- */

typedef struct {
    int iters;           /* CG iterations taken */
    int stagnated;       /* 1 if stopped because the true residual stopped improving */
    double rel_res_l2;   /* true ||b - A x||_2 / ||b||_2 at exit */
    double rel_res_linf; /* true ||b - A x||_inf / ||b||_inf at exit */
    int n_coef;          /* number of Lanczos coefficient pairs stored */
} or_cg_stats;

static double max_abs(int64_t n, const double* a) {
    double m = 0.0;
    for (int64_t q = 0; q < n; ++q) { double v = fabs(a[q]); if (v > m) m = v; }
    return m;
}

/* Unpreconditioned conjugate gradients for A x = rhs with A = -L symmetric
 * positive semi-definite and rhs mean-free (so the system is consistent).
 * x holds the initial guess on entry.  The textbook recurrence runs with one
 * addition: after every update the residual r is projected to mean zero, i.e.
 * kept orthogonal to the null space (the constants), where the consistent
 * system's residual lies in exact arithmetic.  Every `check` iterations, and whenever the recurrence residual reaches tol,
 * x is projected to mean zero and the TRUE residual rhs - A x is computed.
 * The solve stops when ||rhs - A x||_2/||rhs||_2 <= tol.  If the recurrence
 * has converged but the true residual has not, CG restarts from the true
 * residual.  The solve also stops (flagged "stagnated") when the true residual
 * has not halved over the last OR_STALL checks or after OR_MAX_RESTARTS
 * restarts without halving it: rounding then limits the attainable accuracy.
 * A stall counts only once the true residual is at most OR_STALL_FLOOR
 * relative: the FP64 floor of these systems lies far below it, while the
 * residual of unpreconditioned CG (which minimises the A-norm of the error,
 * not the residual) can sit on a plateau, or rise, for thousands of steps
 * before it falls on strongly layered densities.
 * With solid cells (fluid != NULL, Sec. 3.8) the projections above are onto
 * the complement of the masked operator's null space (oracle_null_project).
 * The CG step lengths alpha_k and ratios beta_k of the first cycle are stored
 * in coef[2k], coef[2k+1] (up to max_coef pairs): they define the Lanczos
 * tridiagonal matrix whose eigenvalues estimate the extreme eigenvalues of A. */
#define OR_STALL 20
#define OR_MAX_RESTARTS 3
#define OR_STALL_FLOOR 1e-8
void oracle_cg_masked(const or_csr* A, const double* rhs, double* x, double tol, int max_iter,
                      int check, double* coef, int max_coef, const unsigned char* fluid,
                      or_cg_stats* st) {
    int64_t n = A->n;
    double* r = (double*)malloc(sizeof(double) * n);
    double* d = (double*)malloc(sizeof(double) * n);
    double* q = (double*)malloc(sizeof(double) * n);
    double* t = (double*)malloc(sizeof(double) * n);
    double bnorm = sqrt(det_dot(n, rhs, rhs));
    double binf = max_abs(n, rhs);
    int it = 0, ncoef = 0, stag = 0, nhist = 0, restarts = 0, first_cycle = 1;
    double hist[OR_STALL]; /* true residuals of the last OR_STALL checks (ring buffer) */
    double at_restart = INFINITY;
    if (bnorm == 0.0) {
        memset(x, 0, sizeof(double) * n);
        st->iters = 0; st->stagnated = 0; st->rel_res_l2 = 0.0; st->rel_res_linf = 0.0; st->n_coef = 0;
        free(r); free(d); free(q); free(t);
        return;
    }
    oracle_null_project(n, x, fluid);
    oracle_csr_matvec(A, x, q);
    #pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n; ++c) r[c] = rhs[c] - q[c];
    oracle_null_project(n, r, fluid);
    memcpy(d, r, sizeof(double) * n);
    double rr = det_dot(n, r, r);
    if (sqrt(rr) / bnorm > tol) {
        while (it < max_iter) {
            oracle_csr_matvec(A, d, q);
            double dq = det_dot(n, d, q);
            if (!(dq > 0.0)) break; /* d = 0: nothing left to gain */
            double alpha = rr / dq;
            #pragma omp parallel for schedule(static)
            for (int64_t c = 0; c < n; ++c) { x[c] += alpha * d[c]; r[c] -= alpha * q[c]; }
            /* keep the residual in the range of A (mean-free): the rounding of A d
             * leaves a constant part in r that A cannot remove, and over many steps
             * it grows until d . A d is no longer positive */
            oracle_null_project(n, r, fluid);
            double rr_new = det_dot(n, r, r);
            double beta = rr_new / rr;
            if (coef && first_cycle && ncoef < max_coef) {
                coef[2 * ncoef] = alpha; coef[2 * ncoef + 1] = beta; ++ncoef;
            }
            #pragma omp parallel for schedule(static)
            for (int64_t c = 0; c < n; ++c) d[c] = r[c] + beta * d[c];
            rr = rr_new;
            ++it;
            int rec_done = sqrt(rr) / bnorm <= tol;
            if (it % check == 0 || rec_done) {
                oracle_null_project(n, x, fluid);
                oracle_csr_matvec(A, x, q);
                #pragma omp parallel for schedule(static)
                for (int64_t c = 0; c < n; ++c) t[c] = rhs[c] - q[c];
                double true_rel = sqrt(det_dot(n, t, t)) / bnorm;
                if (true_rel <= tol) break;
                /* hist[nhist % OR_STALL] holds the value of OR_STALL checks ago */
                if (nhist >= OR_STALL && true_rel <= OR_STALL_FLOOR && true_rel > 0.5 * hist[nhist % OR_STALL]) {
                    stag = 1;
                    break;
                }
                hist[nhist % OR_STALL] = true_rel;
                ++nhist;
                if (rec_done) {
                    if (true_rel > 0.5 * at_restart) ++restarts; else restarts = 0;
                    if (restarts >= OR_MAX_RESTARTS) { stag = 1; break; }
                    at_restart = true_rel < at_restart ? true_rel : at_restart;
                    first_cycle = 0;
                    #pragma omp parallel for schedule(static)
                    for (int64_t c = 0; c < n; ++c) r[c] = t[c];
                    oracle_null_project(n, r, fluid);
                    memcpy(d, r, sizeof(double) * n);
                    rr = det_dot(n, r, r);
                }
            }
        }
    }
    /* final true residual */
    oracle_null_project(n, x, fluid);
    oracle_csr_matvec(A, x, q);
    for (int64_t c = 0; c < n; ++c) r[c] = rhs[c] - q[c];
    st->iters = it;
    st->stagnated = stag;
    st->rel_res_l2 = sqrt(det_dot(n, r, r)) / bnorm;
    st->rel_res_linf = max_abs(n, r) / binf;
    st->n_coef = ncoef;
    free(r); free(d); free(q); free(t);
}

void oracle_cg(const or_csr* A, const double* rhs, double* x, double tol, int max_iter,
               int check, double* coef, int max_coef, or_cg_stats* st) {
    oracle_cg_masked(A, rhs, x, tol, max_iter, check, coef, max_coef, NULL, st);
}

/* ------------------------------------------------ velocity correction --- */

/* Eq. fotm: u_f = u*_f - dt beta_f (p_R - p_L)/h on every face that is not a
 * wall; wall faces are blocked (u = 0, Sec. 3.8).  In place on u, v, w. */
void oracle_project(const or_grid* g, const double* bx, const double* by, const double* bz,
                    const double* p, double dt, double* u, double* v, double* w) {
    const double* beta[3] = {bx, by, bz};
    double* vel[3] = {u, v, w};
    for (int axis = 0; axis < 3; ++axis) {
        int d[3];
        face_dims(g, axis, d);
        #pragma omp parallel for schedule(static)
        for (int k = 0; k < d[2]; ++k)
            for (int j = 0; j < d[1]; ++j)
                for (int i = 0; i < d[0]; ++i) {
                    int64_t L, R, f = face_index(g, axis, i, j, k);
                    if (!face_cells(g, axis, i, j, k, &L, &R)) { vel[axis][f] = 0.0; continue; }
                    double grad = (p[R] - p[L]) / g->h;
                    vel[axis][f] = vel[axis][f] - dt * beta[axis][f] * grad;
                }
    }
}

/* face gradient (G p)_f = (p_R - p_L)/h on non-wall faces, 0 on wall faces */
void oracle_face_gradient(const or_grid* g, const double* p, double* gx, double* gy, double* gz) {
    double* out[3] = {gx, gy, gz};
    for (int axis = 0; axis < 3; ++axis) {
        int d[3];
        face_dims(g, axis, d);
        #pragma omp parallel for schedule(static)
        for (int k = 0; k < d[2]; ++k)
            for (int j = 0; j < d[1]; ++j)
                for (int i = 0; i < d[0]; ++i) {
                    int64_t L, R, f = face_index(g, axis, i, j, k);
                    out[axis][f] = face_cells(g, axis, i, j, k, &L, &R) ? (p[R] - p[L]) / g->h : 0.0;
                }
    }
}

/* ---------------------------------------------------------- adjoint --- */

/* Adjoint of the projection u = u* - B G L^{-1} D u* for a loss with gradient
 * g = dLoss/du (the paper has no adjoint; this follows from Eqs. fotm and
 * poisson by differentiating the linear solve).  With q the mean-free solution
 * of L q = D(B g):
 *   dLoss/du*_f   = g_f - (G q)_f                  (0 on wall faces)
 *   dLoss/dbeta_f = dt (G p)_f ((G q)_f - g_f)     (0 on wall faces)
 * The adjoint solve uses the same CSR operator A = -L, so it solves A q = -c. */
void oracle_project_adjoint(const or_grid* g, const or_csr* A,
                            const double* bx, const double* by, const double* bz,
                            const double* p, double dt,
                            const double* gu, const double* gv, const double* gw,
                            double* gus, double* gvs, double* gws,
                            double* gbx, double* gby, double* gbz,
                            double* q, double tol, int max_iter, or_cg_stats* st) {
    int64_t n = A->n;
    const double* beta[3] = {bx, by, bz};
    const double* gin[3] = {gu, gv, gw};
    double* gstar[3] = {gus, gvs, gws};
    double* gbeta[3] = {gbx, gby, gbz};
    double* bg[3];
    for (int axis = 0; axis < 3; ++axis) {
        int64_t m = oracle_face_count(g, axis);
        bg[axis] = (double*)malloc(sizeof(double) * m);
        for (int64_t f = 0; f < m; ++f) bg[axis][f] = beta[axis][f] * gin[axis][f];
    }
    double* c = (double*)malloc(sizeof(double) * n);
    oracle_divergence(g, bg[0], bg[1], bg[2], 1.0, c); /* c = D (B g) */
    for (int64_t k2 = 0; k2 < n; ++k2) c[k2] = -c[k2]; /* A q = -c  <=>  L q = c */
    oracle_remove_mean(n, c);
    memset(q, 0, sizeof(double) * n);
    oracle_cg(A, c, q, tol, max_iter, 50, NULL, 0, st);
    for (int axis = 0; axis < 3; ++axis) {
        int d[3];
        face_dims(g, axis, d);
        for (int k = 0; k < d[2]; ++k)
            for (int j = 0; j < d[1]; ++j)
                for (int i = 0; i < d[0]; ++i) {
                    int64_t L, R, f = face_index(g, axis, i, j, k);
                    if (!face_cells(g, axis, i, j, k, &L, &R)) { gstar[axis][f] = 0.0; gbeta[axis][f] = 0.0; continue; }
                    double gq = (q[R] - q[L]) / g->h;
                    double gp = (p[R] - p[L]) / g->h;
                    gstar[axis][f] = gin[axis][f] - gq;
                    gbeta[axis][f] = dt * gp * (gq - gin[axis][f]);
                }
        free(bg[axis]);
    }
    free(c);
}

/* dLoss/dC_c = sum over the non-wall faces f of cell c of
 *   dLoss/dbeta_f * dbeta_f/dC_c,  dbeta_f/dC_c = -beta_f^2 (rho1 - rho2)/2,
 * from beta_f = 1/rho_f, rho_f = (rho_L + rho_R)/2, rho = rho1 C + rho2 (1-C). */
void oracle_face_coeffs_adjoint(const or_grid* g, double rho1, double rho2,
                                const double* bx, const double* by, const double* bz,
                                const double* gbx, const double* gby, const double* gbz,
                                double* gC) {
    const double* beta[3] = {bx, by, bz};
    const double* gb[3] = {gbx, gby, gbz};
    int64_t n = (int64_t)g->nx * g->ny * g->nz;
    memset(gC, 0, sizeof(double) * n);
    for (int axis = 0; axis < 3; ++axis) {
        int d[3];
        face_dims(g, axis, d);
        for (int k = 0; k < d[2]; ++k)
            for (int j = 0; j < d[1]; ++j)
                for (int i = 0; i < d[0]; ++i) {
                    int64_t L, R, f = face_index(g, axis, i, j, k);
                    if (!face_cells(g, axis, i, j, k, &L, &R)) continue;
                    double dbdC = -beta[axis][f] * beta[axis][f] * (rho1 - rho2) * 0.5;
                    gC[L] += gb[axis][f] * dbdC;
                    gC[R] += gb[axis][f] * dbdC;
                }
    }
}
