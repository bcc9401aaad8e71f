/*
 * FP64 CPU oracle for the NeFTY implicit-Euler heat solve, its discrete adjoint
 * and the diffusivity gradient.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file.  It shares no code, header,
 * table or helper with the CUDA library; it is written directly from the
 * paper's definitions so that a reader can check it against the paper by eye:
 *
 *   - face conductance: harmonic mean a_pq = 2 a_p a_q / (a_p + a_q) / dd^2
 *     (Prop. 1; App. A.3; App. D.2 "Symmetry, sign, and diagonal dominance").
 *   - operator L(alpha): L_pq = a_pq for q ~ p, L_pp = -beta_p - sum_q a_pq,
 *     lateral periodic wrap or zero-flux walls, z adiabatic, optional Robin
 *     sink beta_p = h/dz on the back face (App. A.5; App. D.2).
 *   - implicit Euler: A = I - dt L, A T^{n+1} = T^n + dt s^n (Eq. state_eq),
 *     each system solved by a plain conjugate-gradient loop to a relative
 *     residual tolerance (default 1e-14) or by dense LU on tiny grids.
 *   - objective: J = loss_scale * sum_n || Pi T^n - That^n ||^2 (Eq. nefty_obj).
 *   - adjoint: A^T mu^n = mu^{n+1} + (d l^n / d T^n)^T, mu^{Nt+1} = 0, with A^T
 *     formed by explicit CSR transposition (Eq. adjoint_eq; App. D.3).
 *   - gradient: dJ/dalpha = dt sum_n (d(L T^n)/d alpha)^T mu^n with the sparse
 *     Jacobian d(L T^n)/d alpha assembled as a matrix from the harmonic-mean
 *     derivative d a_pq / d a_p = 2 a_q^2 / (a_p + a_q)^2 / dd^2
 *     (Eq. grad_assembly; App. D.3 "Gradient assembly").
 *   - dJ/dT^0 = mu^1 (App. D.3 "Sensitivity to initial conditions").
 *   - total variation R(alpha) (Eq. tv_discrete) and its gradient.
 *
 * The source term s^n is not in the paper (its state equation is affine-free);
 * it is the pulse-flux reading: s^n = q^n / dz on the k = 0 cell slab.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int nx, ny, nz;
    double dx, dy, dz, dt;
    int nt;
    int bc;            /* 0: zero-flux walls on all six faces; 1: periodic in x and y */
    double robin_h;    /* back-face (k = nz-1) Robin coefficient h; 0 = adiabatic */
    int obs_face;      /* 0: observe the k = 0 plane; 1: the k = nz-1 plane */
    double loss_scale; /* s in J = s * sum ||Pi T - That||^2 */
} orc_problem;

typedef struct {
    int n;
    int64_t nnz;
    int64_t *rp;
    int32_t *ci;
    double *v;
} orc_csr;

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_ENOTCONV = 3 };

static int64_t cell(const orc_problem *g, int i, int j, int k) {
    return ((int64_t)k * g->ny + j) * g->nx + i;
}

/* ---------------------------------------------------------------- faces */
/* One face joins cells p and q along axis d (0 x, 1 y, 2 z). */
typedef struct { int64_t p, q; int axis; } orc_face;

/* Enumerate the faces of the grid: the +x, +y, +z face of every cell, with
 * the lateral faces wrapping when bc == 1, and no face across z walls. */
static int64_t list_faces(const orc_problem *g, orc_face *out) {
    int64_t f = 0;
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                int64_t p = cell(g, i, j, k);
                if (i + 1 < g->nx) { out[f].p = p; out[f].q = cell(g, i + 1, j, k); out[f].axis = 0; ++f; }
                else if (g->bc == 1 && g->nx > 1) { out[f].p = p; out[f].q = cell(g, 0, j, k); out[f].axis = 0; ++f; }
                if (j + 1 < g->ny) { out[f].p = p; out[f].q = cell(g, i, j + 1, k); out[f].axis = 1; ++f; }
                else if (g->bc == 1 && g->ny > 1) { out[f].p = p; out[f].q = cell(g, i, 0, k); out[f].axis = 1; ++f; }
                if (k + 1 < g->nz) { out[f].p = p; out[f].q = cell(g, i, j, k + 1); out[f].axis = 2; ++f; }
            }
    return f;
}

static double spacing_sq(const orc_problem *g, int axis) {
    double h = axis == 0 ? g->dx : (axis == 1 ? g->dy : g->dz);
    return h * h;
}

/* Harmonic-mean face conductance (Prop. 1) divided by the squared spacing. */
static double face_conductance(double ap, double aq, double h2) {
    return 2.0 * ap * aq / (ap + aq) / h2;
}

/* ------------------------------------------------------- row builder */
/* Rows are built entry by entry; equal columns are summed and each row is
 * sorted by column when the CSR arrays are emitted. */
#define ORC_ROWCAP 16
typedef struct { int cnt; int32_t col[ORC_ROWCAP]; double val[ORC_ROWCAP]; } orc_row;

static void row_add(orc_row *rows, int64_t r, int64_t c, double v) {
    orc_row *R = &rows[r];
    for (int e = 0; e < R->cnt; ++e)
        if (R->col[e] == (int32_t)c) { R->val[e] += v; return; }
    R->col[R->cnt] = (int32_t)c;
    R->val[R->cnt] = v;
    R->cnt++;
}

static int rows_to_csr(orc_row *rows, int n, orc_csr *M) {
    int64_t nnz = 0;
    for (int r = 0; r < n; ++r) nnz += rows[r].cnt;
    M->n = n;
    M->nnz = nnz;
    M->rp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    M->ci = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz ? nnz : 1));
    M->v = (double *)malloc(sizeof(double) * (size_t)(nnz ? nnz : 1));
    if (!M->rp || !M->ci || !M->v) return ORC_ENOMEM;
    int64_t e = 0;
    M->rp[0] = 0;
    for (int r = 0; r < n; ++r) {
        orc_row *R = &rows[r];
        /* insertion sort by column */
        for (int a = 1; a < R->cnt; ++a) {
            int32_t c = R->col[a]; double v = R->val[a]; int b = a - 1;
            while (b >= 0 && R->col[b] > c) { R->col[b + 1] = R->col[b]; R->val[b + 1] = R->val[b]; --b; }
            R->col[b + 1] = c; R->val[b + 1] = v;
        }
        for (int a = 0; a < R->cnt; ++a) { M->ci[e] = R->col[a]; M->v[e] = R->val[a]; ++e; }
        M->rp[r + 1] = e;
    }
    return ORC_OK;
}

static void csr_free(orc_csr *M) {
    free(M->rp); free(M->ci); free(M->v);
    M->rp = NULL; M->ci = NULL; M->v = NULL;
}

/* L(alpha) of App. D.2: off-diagonal a_pq for every face, diagonal minus the
 * sum of the row's face conductances minus the Robin sink h/dz on k = nz-1. */
static int assemble_L(const orc_problem *g, const double *alpha, orc_csr *L) {
    int n = g->nx * g->ny * g->nz;
    orc_face *faces = (orc_face *)malloc(sizeof(orc_face) * (size_t)3 * (size_t)n);
    orc_row *rows = (orc_row *)calloc((size_t)n, sizeof(orc_row));
    if (!faces || !rows) { free(faces); free(rows); return ORC_ENOMEM; }
    for (int r = 0; r < n; ++r) row_add(rows, r, r, 0.0);
    int64_t nf = list_faces(g, faces);
    for (int64_t f = 0; f < nf; ++f) {
        int64_t p = faces[f].p, q = faces[f].q;
        if (p == q) continue;
        double a = face_conductance(alpha[p], alpha[q], spacing_sq(g, faces[f].axis));
        row_add(rows, p, q, a);
        row_add(rows, p, p, -a);
        row_add(rows, q, p, a);
        row_add(rows, q, q, -a);
    }
    if (g->robin_h != 0.0) {
        double beta = g->robin_h / g->dz;
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                int64_t p = cell(g, i, j, g->nz - 1);
                row_add(rows, p, p, -beta);
            }
    }
    int rc = rows_to_csr(rows, n, L);
    free(faces); free(rows);
    return rc;
}

/* A = I - dt L (Eq. state_eq). */
static int assemble_A(const orc_problem *g, const double *alpha, orc_csr *A) {
    orc_csr L;
    int rc = assemble_L(g, alpha, &L);
    if (rc) return rc;
    for (int r = 0; r < L.n; ++r)
        for (int64_t e = L.rp[r]; e < L.rp[r + 1]; ++e)
            L.v[e] = (L.ci[e] == r ? 1.0 : 0.0) - g->dt * L.v[e];
    *A = L;
    return ORC_OK;
}

/* Explicit transpose by counting columns. */
static int csr_transpose(const orc_csr *M, orc_csr *T) {
    int n = M->n;
    T->n = n;
    T->nnz = M->nnz;
    T->rp = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
    T->ci = (int32_t *)malloc(sizeof(int32_t) * (size_t)(M->nnz ? M->nnz : 1));
    T->v = (double *)malloc(sizeof(double) * (size_t)(M->nnz ? M->nnz : 1));
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!T->rp || !T->ci || !T->v || !next) { free(next); return ORC_ENOMEM; }
    for (int64_t e = 0; e < M->nnz; ++e) T->rp[M->ci[e] + 1]++;
    for (int r = 0; r < n; ++r) T->rp[r + 1] += T->rp[r];
    for (int r = 0; r <= n; ++r) next[r] = T->rp[r];
    for (int r = 0; r < n; ++r)
        for (int64_t e = M->rp[r]; e < M->rp[r + 1]; ++e) {
            int64_t d = next[M->ci[e]]++;
            T->ci[d] = r;
            T->v[d] = M->v[e];
        }
    free(next);
    return ORC_OK;
}

static void spmv(const orc_csr *M, const double *x, double *y) {
    #pragma omp parallel for schedule(static) if (M->n >= 200000)
    for (int r = 0; r < M->n; ++r) {
        double s = 0.0;
        for (int64_t e = M->rp[r]; e < M->rp[r + 1]; ++e) s += M->v[e] * x[M->ci[e]];
        y[r] = s;
    }
}

static double dot(int n, const double *a, const double *b) {
    double s = 0.0;
    #pragma omp parallel for reduction(+ : s) schedule(static) if (n >= 200000)
    for (int i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Jacobi-preconditioned conjugate gradients on M x = b, from the given x,
 * until ||b - M x||_2 <= tol ||b||_2 (recursively updated residual).
 * Returns the iteration count, or -1 if max_iter was reached. */
static int cg_solve(const orc_csr *M, const double *b, double *x, double tol, int max_iter) {
    int n = M->n;
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    double *dinv = (double *)malloc(sizeof(double) * (size_t)n);
    for (int i = 0; i < n; ++i) {
        double d = 0.0;
        for (int64_t e = M->rp[i]; e < M->rp[i + 1]; ++e) if (M->ci[e] == i) d = M->v[e];
        dinv[i] = 1.0 / d;
    }
    double bnorm = sqrt(dot(n, b, b));
    int it = 0;
    if (bnorm == 0.0) {
        for (int i = 0; i < n; ++i) x[i] = 0.0;
        goto done;
    }
    spmv(M, x, q);
    for (int i = 0; i < n; ++i) { r[i] = b[i] - q[i]; z[i] = dinv[i] * r[i]; p[i] = z[i]; }
    double rz = dot(n, r, z);
    while (sqrt(dot(n, r, r)) > tol * bnorm) {
        if (it >= max_iter) { it = -1; break; }
        spmv(M, p, q);
        double alpha = rz / dot(n, p, q);
        for (int i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; z[i] = dinv[i] * r[i]; }
        double rz_new = dot(n, r, z);
        double beta = rz_new / rz;
        rz = rz_new;
        for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        ++it;
    }
done:
    free(r); free(z); free(p); free(q); free(dinv);
    return it;
}

/* K sweeps of the paper's Jacobi inner solver (App. D.2, Eq. jacobi_iter):
 * x <- D^{-1} (b - R x) with M = D + R, D the diagonal of M and R the rest,
 * starting from the x given (the warm start) and with no stopping test. */
static void jacobi_solve(const orc_csr *M, const double *b, double *x, int K) {
    int n = M->n;
    double *y = (double *)malloc(sizeof(double) * (size_t)n);
    for (int kappa = 0; kappa < K; ++kappa) {
        #pragma omp parallel for schedule(static) if (n >= 200000)
        for (int r = 0; r < n; ++r) {
            double d = 0.0, rx = 0.0;
            for (int64_t e = M->rp[r]; e < M->rp[r + 1]; ++e) {
                if (M->ci[e] == r) d = M->v[e];
                else rx += M->v[e] * x[M->ci[e]];
            }
            y[r] = (b[r] - rx) / d;
        }
        memcpy(x, y, sizeof(double) * (size_t)n);
    }
    free(y);
}

/* --------------------------------------------------------- dense LU */
/* Gaussian elimination with partial pivoting on a dense copy of M; the
 * factors overwrite lu, the row permutation is stored in piv. */
static int dense_lu(const orc_csr *M, double *lu, int *piv) {
    int n = M->n;
    memset(lu, 0, sizeof(double) * (size_t)n * (size_t)n);
    for (int r = 0; r < n; ++r)
        for (int64_t e = M->rp[r]; e < M->rp[r + 1]; ++e) lu[(size_t)r * n + M->ci[e]] += M->v[e];
    for (int c = 0; c < n; ++c) {
        int best = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(lu[(size_t)r * n + c]) > fabs(lu[(size_t)best * n + c])) best = r;
        piv[c] = best;
        if (best != c)
            for (int k = 0; k < n; ++k) {
                double t = lu[(size_t)c * n + k]; lu[(size_t)c * n + k] = lu[(size_t)best * n + k]; lu[(size_t)best * n + k] = t;
            }
        double d = lu[(size_t)c * n + c];
        if (d == 0.0) return ORC_EINVAL;
        for (int r = c + 1; r < n; ++r) {
            double m = lu[(size_t)r * n + c] / d;
            lu[(size_t)r * n + c] = m;
            for (int k = c + 1; k < n; ++k) lu[(size_t)r * n + k] -= m * lu[(size_t)c * n + k];
        }
    }
    return ORC_OK;
}

static void dense_lu_solve(int n, const double *lu, const int *piv, const double *b, double *x) {
    for (int i = 0; i < n; ++i) x[i] = b[i];
    for (int c = 0; c < n; ++c) { int p = piv[c]; if (p != c) { double t = x[c]; x[c] = x[p]; x[p] = t; } }
    for (int r = 0; r < n; ++r) { double s = x[r]; for (int k = 0; k < r; ++k) s -= lu[(size_t)r * n + k] * x[k]; x[r] = s; }
    for (int r = n - 1; r >= 0; --r) {
        double s = x[r];
        for (int k = r + 1; k < n; ++k) s -= lu[(size_t)r * n + k] * x[k];
        x[r] = s / lu[(size_t)r * n + r];
    }
}

/* ------------------------------------------------------------ forcing */
/* Right-hand side of step n: b = T^n + dt * q^n / dz on the k = 0 slab, with
 * q^n = q_full[n] when given, else q_face for n < q_steps. */
static void step_rhs(const orc_problem *g, int n, const double *Tn, const double *q_face, int q_steps,
                     const double *q_full, double *b) {
    int64_t N = (int64_t)g->nx * g->ny * g->nz;
    int64_t S = (int64_t)g->nx * g->ny;
    for (int64_t i = 0; i < N; ++i) b[i] = Tn[i];
    const double *q = NULL;
    if (q_full) q = q_full + (int64_t)n * S;
    else if (q_face && n < q_steps) q = q_face;
    if (q)
        for (int64_t s = 0; s < S; ++s) b[s] += g->dt * q[s] / g->dz;
}

static int64_t obs_offset(const orc_problem *g) {
    return g->obs_face ? (int64_t)(g->nz - 1) * g->nx * g->ny : 0;
}

/* ------------------------------------------------------------- API */
int orc_assemble_A(const orc_problem *g, const double *alpha, int64_t *rp, int32_t *ci, double *v,
                   int64_t *nnz) {
    orc_csr A;
    int rc = assemble_A(g, alpha, &A);
    if (rc) return rc;
    *nnz = A.nnz;
    if (rp) { memcpy(rp, A.rp, sizeof(int64_t) * (size_t)(A.n + 1)); memcpy(ci, A.ci, sizeof(int32_t) * (size_t)A.nnz); memcpy(v, A.v, sizeof(double) * (size_t)A.nnz); }
    csr_free(&A);
    return ORC_OK;
}

/* out = L(alpha) T */
int orc_apply_L(const orc_problem *g, const double *alpha, const double *T, double *out) {
    orc_csr L;
    int rc = assemble_L(g, alpha, &L);
    if (rc) return rc;
    spmv(&L, T, out);
    csr_free(&L);
    return ORC_OK;
}

/* Forward sweep.  states (optional) receives T^0..T^nt, frames (optional)
 * receives Pi T^1..Pi T^nt, loss (optional) the objective when obs is given,
 * iters (optional) the CG iteration count of each step.  dense != 0 solves each
 * step by dense LU instead of CG; jacobi_k > 0 by jacobi_k Jacobi sweeps from
 * T^n (the paper's inner solver). */
int orc_forward(const orc_problem *g, const double *alpha, const double *T0, const double *q_face,
                int q_steps, const double *q_full, const double *obs, double *frames, double *states,
                double *loss, int *iters, double tol, int max_iter, int dense, int jacobi_k) {
    int64_t N = (int64_t)g->nx * g->ny * g->nz;
    int64_t S = (int64_t)g->nx * g->ny;
    orc_csr A;
    int rc = assemble_A(g, alpha, &A);
    if (rc) return rc;
    double *Tn = (double *)calloc((size_t)N, sizeof(double));
    double *Tn1 = (double *)calloc((size_t)N, sizeof(double));
    double *b = (double *)malloc(sizeof(double) * (size_t)N);
    double *lu = NULL; int *piv = NULL;
    if (dense) {
        lu = (double *)malloc(sizeof(double) * (size_t)N * (size_t)N);
        piv = (int *)malloc(sizeof(int) * (size_t)N);
        rc = dense_lu(&A, lu, piv);
        if (rc) goto out;
    }
    if (T0) memcpy(Tn, T0, sizeof(double) * (size_t)N);
    if (states) memcpy(states, Tn, sizeof(double) * (size_t)N);
    double J = 0.0;
    int64_t o = obs_offset(g);
    for (int n = 0; n < g->nt; ++n) {
        step_rhs(g, n, Tn, q_face, q_steps, q_full, b);
        if (dense) {
            dense_lu_solve((int)N, lu, piv, b, Tn1);
        } else if (jacobi_k > 0) {
            memcpy(Tn1, Tn, sizeof(double) * (size_t)N); /* T^(0) = T^n */
            jacobi_solve(&A, b, Tn1, jacobi_k);
            if (iters) iters[n] = jacobi_k;
        } else {
            memcpy(Tn1, Tn, sizeof(double) * (size_t)N); /* warm start x0 = T^n */
            int it = cg_solve(&A, b, Tn1, tol, max_iter);
            if (iters) iters[n] = it;
            if (it < 0) rc = ORC_ENOTCONV;
        }
        if (states) memcpy(states + (int64_t)(n + 1) * N, Tn1, sizeof(double) * (size_t)N);
        if (frames) memcpy(frames + (int64_t)n * S, Tn1 + o, sizeof(double) * (size_t)S);
        if (obs)
            for (int64_t s = 0; s < S; ++s) { double e = Tn1[o + s] - obs[(int64_t)n * S + s]; J += e * e; }
        double *t = Tn; Tn = Tn1; Tn1 = t;
    }
    if (loss) *loss = g->loss_scale * J;
out:
    free(Tn); free(Tn1); free(b); free(lu); free(piv);
    csr_free(&A);
    return rc;
}

/* d(L(alpha) T)/d alpha as an explicit N x N sparse matrix (rows: cells of
 * L T, columns: alpha).  For a face (p, q) with conductance a, row p of L T
 * holds a (T_q - T_p) and row q holds a (T_p - T_q); both depend on alpha_p
 * and alpha_q through d a / d alpha_p = 2 alpha_q^2 / (alpha_p + alpha_q)^2 / h^2. */
static int assemble_jacobian_LT(const orc_problem *g, const double *alpha, const double *T, orc_csr *Jm) {
    int n = g->nx * g->ny * g->nz;
    orc_face *faces = (orc_face *)malloc(sizeof(orc_face) * (size_t)3 * (size_t)n);
    orc_row *rows = (orc_row *)calloc((size_t)n, sizeof(orc_row));
    if (!faces || !rows) { free(faces); free(rows); return ORC_ENOMEM; }
    int64_t nf = list_faces(g, faces);
    for (int64_t f = 0; f < nf; ++f) {
        int64_t p = faces[f].p, q = faces[f].q;
        if (p == q) continue;
        double h2 = spacing_sq(g, faces[f].axis);
        double s = alpha[p] + alpha[q];
        double da_dp = 2.0 * alpha[q] * alpha[q] / (s * s) / h2;
        double da_dq = 2.0 * alpha[p] * alpha[p] / (s * s) / h2;
        row_add(rows, p, p, (T[q] - T[p]) * da_dp);
        row_add(rows, p, q, (T[q] - T[p]) * da_dq);
        row_add(rows, q, p, (T[p] - T[q]) * da_dp);
        row_add(rows, q, q, (T[p] - T[q]) * da_dq);
    }
    int rc = rows_to_csr(rows, n, Jm);
    free(faces); free(rows);
    return rc;
}

/* Forward (all states kept), then the reverse-time adjoint recurrence with
 * A^T formed by transposition, then gradient assembly.  jacobi_k > 0: every
 * forward and adjoint solve is jacobi_k Jacobi sweeps from the warm start
 * (T^n, mu^(n+1)), as the paper's inner solver. */
int orc_adjoint_grad(const orc_problem *g, const double *alpha, const double *T0, const double *q_face,
                     int q_steps, const double *q_full, const double *obs, double *loss, double *grad_alpha,
                     double *grad_T0, double tol, int max_iter, int jacobi_k) {
    int64_t N = (int64_t)g->nx * g->ny * g->nz;
    int64_t S = (int64_t)g->nx * g->ny;
    double *states = (double *)malloc(sizeof(double) * (size_t)N * (size_t)(g->nt + 1));
    if (!states) return ORC_ENOMEM;
    int rc = orc_forward(g, alpha, T0, q_face, q_steps, q_full, obs, NULL, states, loss, NULL, tol, max_iter, 0,
                         jacobi_k);
    if (rc && rc != ORC_ENOTCONV) { free(states); return rc; }
    orc_csr A, At;
    int rc2 = assemble_A(g, alpha, &A);
    if (rc2) { free(states); return rc2; }
    rc2 = csr_transpose(&A, &At);
    csr_free(&A);
    if (rc2) { free(states); return rc2; }
    double *mu_next = (double *)calloc((size_t)N, sizeof(double));
    double *mu = (double *)calloc((size_t)N, sizeof(double));
    double *rhs = (double *)malloc(sizeof(double) * (size_t)N);
    int64_t o = obs_offset(g);
    for (int64_t i = 0; i < N; ++i) grad_alpha[i] = 0.0;
    for (int n = g->nt; n >= 1; --n) {
        const double *Tn = states + (int64_t)n * N;
        /* rhs = mu^{n+1} + (d l^n / d T^n)^T, l^n = s ||Pi T^n - That^n||^2 */
        for (int64_t i = 0; i < N; ++i) rhs[i] = mu_next[i];
        if (obs)
            for (int64_t s = 0; s < S; ++s)
                rhs[o + s] += 2.0 * g->loss_scale * (Tn[o + s] - obs[(int64_t)(n - 1) * S + s]);
        memcpy(mu, mu_next, sizeof(double) * (size_t)N); /* warm start from mu^{n+1} */
        if (jacobi_k > 0) {
            jacobi_solve(&At, rhs, mu, jacobi_k);
        } else {
            int it = cg_solve(&At, rhs, mu, tol, max_iter);
            if (it < 0) rc = ORC_ENOTCONV;
        }
        /* grad += dt * J(T^n)^T mu^n, summed entry by entry */
        orc_csr Jm;
        rc2 = assemble_jacobian_LT(g, alpha, Tn, &Jm);
        if (rc2) { rc = rc2; break; }
        for (int r = 0; r < Jm.n; ++r)
            for (int64_t e = Jm.rp[r]; e < Jm.rp[r + 1]; ++e) grad_alpha[Jm.ci[e]] += g->dt * Jm.v[e] * mu[r];
        csr_free(&Jm);
        double *t = mu_next; mu_next = mu; mu = t;
    }
    if (grad_T0) memcpy(grad_T0, mu_next, sizeof(double) * (size_t)N); /* mu^1 */
    free(mu_next); free(mu); free(rhs); free(states);
    csr_free(&At);
    return rc;
}

/* Isotropic TV of Eq. tv_discrete with forward differences; lateral
 * differences wrap when bc == 1 and vanish on the last column/row otherwise;
 * the z difference vanishes on the last slice.  grad (optional) receives
 * lam * dR/dalpha.  Returns lam * R. */
double orc_tv(const orc_problem *g, const double *alpha, double lam, double eps, double *grad) {
    int64_t N = (int64_t)g->nx * g->ny * g->nz;
    double V = g->dx * g->dy * g->dz;
    double R = 0.0;
    if (grad) for (int64_t i = 0; i < N; ++i) grad[i] = 0.0;
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                int64_t p = cell(g, i, j, k);
                int64_t px = -1, py = -1, pz = -1;
                if (i + 1 < g->nx) px = cell(g, i + 1, j, k); else if (g->bc == 1) px = cell(g, 0, j, k);
                if (j + 1 < g->ny) py = cell(g, i, j + 1, k); else if (g->bc == 1) py = cell(g, i, 0, k);
                if (k + 1 < g->nz) pz = cell(g, i, j, k + 1);
                double gx = px >= 0 ? (alpha[px] - alpha[p]) / g->dx : 0.0;
                double gy = py >= 0 ? (alpha[py] - alpha[p]) / g->dy : 0.0;
                double gz = pz >= 0 ? (alpha[pz] - alpha[p]) / g->dz : 0.0;
                double t = sqrt(gx * gx + gy * gy + gz * gz + eps * eps);
                R += t;
                if (grad) {
                    double w = lam * V / t;
                    if (px >= 0) { grad[px] += w * gx / g->dx; grad[p] -= w * gx / g->dx; }
                    if (py >= 0) { grad[py] += w * gy / g->dy; grad[p] -= w * gy / g->dy; }
                    if (pz >= 0) { grad[pz] += w * gz / g->dz; grad[p] -= w * gz / g->dz; }
                }
            }
    return lam * V * R;
}
