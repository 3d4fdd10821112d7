/*
 * FP64 CPU oracle for Matching Pursuit LASSO (MPL, Algorithm 1) and its batch
 * mode (BMPL, Sec. 3).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load it.  It shares no code, header, table or
 * helper with the CUDA library, and the CUDA library never calls it.
 *
 * What it computes, per signal b (a column of B, eq. 3 separates by column):
 *
 *     x* = argmin_x  lambda*||x||_1 + 0.5*||b - A x||^2          (eq. 2)
 *
 * by running Algorithm 1 literally, in double precision:
 *   1. x = 0, residual xi = b, active set I = {} (the initialisation of Alg. 1).
 *   2. worst-case analysis: g = A^T xi (Alg. 1).  The atoms j not in
 *      I with |g_j| > lambda are ranked by |g_j| (larger first, lower index on
 *      ties) and the first rho of them form J_t; I <- I u J_t.
 *      If J_t is empty the stopping condition ||xi^T A||_inf <= lambda of
 *      Sec. 2.3 holds and the loop ends.
 *   3. master problem (eq. "primal_MPL"): the LASSO restricted to I, warm
 *      started from x_I (Alg. 1), solved by accelerated proximal
 *      gradient (Nesterov/FISTA, the paper's PG rule for lambda > 0) with a
 *      backtracking line search for the step 1/L (the line search Lemma 1
 *      takes for granted) and a function-value momentum restart that keeps f monotone,
 *      stopped by the relative-decrease rule (eq. "inner") with eps_in.
 *      The gradient A_I^T (A_I u - b) is evaluated as G u - h with
 *      G = A_I^T A_I and h = A_I^T b, which is the same quantity.
 *   4. exact finish (an addition of this oracle, so that the restricted
 *      problems are solved exactly rather than to eps_in): with the sign
 *      pattern s of the PG iterate u, solve G_PP z = h_P - lambda*s_P by
 *      Cholesky (P = nonzeros of u).  If sign(z) = s and the zero entries of I
 *      satisfy |h_i - G_iP z| <= lambda, z is the exact restricted minimiser
 *      (the optimality conditions of eq. 5 on I) and replaces u.  Otherwise
 *      PG continues with a 100x tighter eps_in and the finish is retried.
 *   5. x_I = u, xi = b - A_I x_I (the residual update of Alg. 1); back to 2.
 *
 * The worst-case analysis can alternatively use the BMPL identity
 * (eq. "batchQ"): A^T xi = beta - Q_I x_I with Q = A^T A and beta = A^T b
 * computed once, which is the batch mode of Sec. 3.
 *
 * With lambda = 0 and rho = 1 the loop is orthogonal matching pursuit
 * (Sec. 2.3, last paragraph): the restricted problem is least squares and the
 * finish solves G z = h directly.
 *
 * Subspace exploratory matching (SMPL, Algorithm 2; omega > 1): item 2 above takes
 * the omega*rho largest violators J_omega instead, the master problem is
 * solved on I u J_omega (warm started, new entries at zero), and only the rho
 * atoms of J_omega with the largest |u_i| stay (ties to the earlier-selected
 * atom); the others leave I with their entries, and x^t is u on what remains.
 *
 * Early stopping (Sec. 2.5), each rule off when its threshold is negative:
 *   eq. (stop1): before the selection, stop when ||A^T xi||_inf <= r_inf or
 *                ||xi|| <= r_2;
 *   eq. (stop_con): after the master problem of outer iteration t, stop when
 *                delta_t / |rho f(x^0)| <= eps, delta_t = f(x^{t-1}) - f(x^t),
 *                f(x^0) = 0.5 ||b||^2.
 * An early stop leaves status 3 and x = x^t.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int rho;          /* atoms added per outer iteration (varrho) */
    int max_outer;    /* cap on outer iterations (0 = m/rho + 2) */
    int s_max;        /* PG iterations per attempt */
    int max_attempts; /* PG + exact-finish attempts per outer iteration */
    int exact_finish; /* 1 = run the sign-fixed Cholesky finish */
    int corr_route;   /* 0 = g = A^T xi, 1 = g = beta - Q_I x_I (eq. batchQ) */
    double eps_in;    /* relative-decrease tolerance of eq. (inner) */
    int omega;        /* subspace search length of Algorithm 2 (1 = Algorithm 1) */
    double stop_rinf; /* eq. (stop1): r_inf (< 0: off) */
    double stop_r2;   /* eq. (stop1): r_2 (< 0: off) */
    double stop_eps;  /* eq. (stop_con): eps (< 0: off) */
} mpl_oracle_opts;

typedef struct {
    int n_outer;      /* evaluations of g (full matrix-vector products) */
    int n_inner;      /* PG iterations over all outer iterations */
    int S_size;       /* |I| at exit */
    int status;       /* 0 = stopping condition met, 1 = max_outer reached,
                         2 = met, but some restricted solve was not finished exactly,
                         3 = early stop (eq. stop1 or stop_con) */
    int nnz;          /* nonzeros of x */
    double objective; /* lambda*||x||_1 + 0.5*||b - A x||^2 */
    double kkt;       /* max KKT violation / lambda (absolute when lambda == 0) */
    double gap;       /* relative duality gap with the scaled dual point of eq. 5 */
} mpl_oracle_result;

typedef struct {
    int cap;          /* outer iterations recorded at most */
    int rho_cap;      /* entries per iteration in added/gsel */
    int* n_added;     /* [cap]            |J_t| */
    int* added;       /* [cap*rho_cap]    J_t in selection order */
    double* gsel;     /* [cap*rho_cap]    |g_j| of the selected atoms */
    double* f_prev;   /* [cap]            f(x^{t-1}) */
    double* f_first;  /* [cap]            f after the first PG step of outer t */
    double* L_first;  /* [cap]            1/step of that first PG step */
    double* f_iter;   /* [cap]            f(x^t) after the master problem */
    int* inner;       /* [cap]            PG iterations spent at outer t */
} mpl_oracle_trace;

/* ------------------------------------------------------------------ */

static double dotd(const double* a, const double* b, int n) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += a[k] * b[k];
    return s;
}

static double soft(double v, double t) {
    if (v > t) return v - t;
    if (v < -t) return v + t;
    return 0.0;
}

static double sgn(double v) { return v > 0 ? 1.0 : (v < 0 ? -1.0 : 0.0); }

/* Cholesky of the k x k symmetric positive definite matrix M (row-major, ld),
 * in place, lower triangle.  Returns 0 on success, -1 on a non-positive pivot. */
static int cholesky(double* M, int ld, int k) {
    for (int j = 0; j < k; ++j) {
        double d = M[j * ld + j];
        for (int q = 0; q < j; ++q) d -= M[j * ld + q] * M[j * ld + q];
        if (!(d > 0.0)) return -1;
        d = sqrt(d);
        M[j * ld + j] = d;
        for (int i = j + 1; i < k; ++i) {
            double s = M[i * ld + j];
            for (int q = 0; q < j; ++q) s -= M[i * ld + q] * M[j * ld + q];
            M[i * ld + j] = s / d;
        }
    }
    return 0;
}

/* Solve (L L^T) z = rhs with the factor from cholesky(). */
static void chol_solve(const double* M, int ld, int k, double* z) {
    for (int i = 0; i < k; ++i) {
        double s = z[i];
        for (int q = 0; q < i; ++q) s -= M[i * ld + q] * z[q];
        z[i] = s / M[i * ld + i];
    }
    for (int i = k - 1; i >= 0; --i) {
        double s = z[i];
        for (int q = i + 1; q < k; ++q) s -= M[q * ld + i] * z[q];
        z[i] = s / M[i * ld + i];
    }
}

/* ------------------------------------------------------------------ */
/* Per-thread workspace for one signal. */
typedef struct {
    int n, m, cap;
    double* g;      /* m */
    double* r;      /* n */
    char* inI;      /* m */
    int* I;         /* cap */
    double* G;      /* cap*cap, row-major, ld = cap */
    double* h;      /* cap */
    double* u;      /* cap */
    double* y;      /* cap */
    double* z;      /* cap */
    double* up;     /* cap */
    double* Gv;     /* cap */
    double* Gy;     /* cap */
    double* tmp;    /* cap */
    double* M;      /* cap*cap, Cholesky work */
    int* P;         /* cap */
    int* cand;      /* m */
    double* xs;     /* m, solution scratch */
} work_t;

static void work_free(work_t* w) {
    free(w->g); free(w->r); free(w->inI); free(w->I); free(w->G); free(w->h); free(w->u);
    free(w->y); free(w->z); free(w->up); free(w->Gv); free(w->Gy); free(w->tmp); free(w->M);
    free(w->P); free(w->cand); free(w->xs);
    memset(w, 0, sizeof(*w));
}

static int work_alloc(work_t* w, int n, int m, int cap) {
    memset(w, 0, sizeof(*w));
    w->n = n; w->m = m; w->cap = cap;
    w->g = malloc(sizeof(double) * (size_t)m);
    w->r = malloc(sizeof(double) * (size_t)n);
    w->inI = calloc((size_t)m, 1);
    w->cand = malloc(sizeof(int) * (size_t)m);
    w->xs = malloc(sizeof(double) * (size_t)m);
    w->I = malloc(sizeof(int) * (size_t)cap);
    w->P = malloc(sizeof(int) * (size_t)cap);
    w->G = calloc((size_t)cap * cap, sizeof(double));
    w->M = malloc(sizeof(double) * (size_t)cap * cap);
    double** vecs[] = {&w->h, &w->u, &w->y, &w->z, &w->up, &w->Gv, &w->Gy, &w->tmp};
    for (unsigned i = 0; i < sizeof(vecs) / sizeof(vecs[0]); ++i)
        *vecs[i] = calloc((size_t)cap, sizeof(double));
    if (!w->g || !w->r || !w->inI || !w->cand || !w->xs || !w->I || !w->P || !w->G || !w->M ||
        !w->h || !w->u || !w->y || !w->z || !w->up || !w->Gv || !w->Gy || !w->tmp) {
        work_free(w);
        return -1;
    }
    return 0;
}

/* Grow the per-signal capacity (keeps I, G, h, u). */
static int work_grow(work_t* w, int need) {
    if (need <= w->cap) return 0;
    int nc = w->cap;
    while (nc < need) nc *= 2;
    if (nc > w->m) nc = w->m;
    double* G = calloc((size_t)nc * nc, sizeof(double));
    double* M = malloc(sizeof(double) * (size_t)nc * nc);
    if (!G || !M) { free(G); free(M); return -1; }
    for (int i = 0; i < w->cap; ++i) memcpy(G + (size_t)i * nc, w->G + (size_t)i * w->cap, sizeof(double) * w->cap);
    free(w->G); free(w->M);
    w->G = G; w->M = M;
    int* I = realloc(w->I, sizeof(int) * nc);
    int* P = realloc(w->P, sizeof(int) * nc);
    if (!I || !P) return -1;
    w->I = I; w->P = P;
    double** vecs[] = {&w->h, &w->u, &w->y, &w->z, &w->up, &w->Gv, &w->Gy, &w->tmp};
    for (unsigned i = 0; i < sizeof(vecs) / sizeof(vecs[0]); ++i) {
        double* v = realloc(*vecs[i], sizeof(double) * nc);
        if (!v) return -1;
        for (int q = w->cap; q < nc; ++q) v[q] = 0.0;
        *vecs[i] = v;
    }
    w->cap = nc;
    return 0;
}

/* Gv = G v on the leading s x s block. */
static void gram_mv(const double* G, int ld, int s, const double* v, double* Gv) {
    for (int i = 0; i < s; ++i) Gv[i] = dotd(G + (size_t)i * ld, v, s);
}

/* Smooth part of the restricted objective without the constant 0.5*b'b:
 * 0.5 u'Gu - h'u, given Gu. */
static double smooth_part(const double* u, const double* Gu, const double* h, int s) {
    double a = 0.0, c = 0.0;
    for (int i = 0; i < s; ++i) { a += u[i] * Gu[i]; c += h[i] * u[i]; }
    return 0.5 * a - c;
}

static double l1(const double* u, int s) {
    double a = 0.0;
    for (int i = 0; i < s; ++i) a += fabs(u[i]);
    return a;
}

/* Largest eigenvalue estimate of G (power iteration); a lower bound, the
 * line search raises it when needed. */
static double power_iter(const double* G, int ld, int s, double* v, double* Gv) {
    if (s == 0) return 1.0;
    for (int i = 0; i < s; ++i) v[i] = 1.0 / sqrt((double)s);
    double theta = 0.0;
    for (int it = 0; it < 50; ++it) {
        gram_mv(G, ld, s, v, Gv);
        double nv = sqrt(dotd(Gv, Gv, s));
        theta = dotd(v, Gv, s);
        if (!(nv > 0)) return 1.0;
        for (int i = 0; i < s; ++i) v[i] = Gv[i] / nv;
    }
    return theta > 0 ? theta : 1.0;
}

/* Exact finish on the sign pattern of u (step 4 of the header). */
static int exact_finish(work_t* w, int s, double lam) {
    int* P = w->P;
    int np = 0;
    for (int i = 0; i < s; ++i)
        if (lam == 0.0 || w->u[i] != 0.0) P[np++] = i;
    if (np == 0) {
        /* u = 0: optimal iff |h_i| <= lambda for every i in I */
        for (int i = 0; i < s; ++i)
            if (fabs(w->h[i]) > lam * (1.0 + 1e-10)) return -1;
        return 0;
    }
    double* M = w->M;
    int ld = w->cap;
    for (int a = 0; a < np; ++a)
        for (int c = 0; c < np; ++c) M[(size_t)a * ld + c] = w->G[(size_t)P[a] * ld + P[c]];
    if (cholesky(M, ld, np) != 0) return -1;
    double* z = w->tmp;
    for (int a = 0; a < np; ++a) z[a] = w->h[P[a]] - lam * sgn(w->u[P[a]]);
    chol_solve(M, ld, np, z);
    if (lam > 0.0)
        for (int a = 0; a < np; ++a)
            if (!(z[a] * sgn(w->u[P[a]]) > 0.0)) return -1;
    /* candidate restricted solution */
    double* cand = w->z;
    for (int i = 0; i < s; ++i) cand[i] = 0.0;
    for (int a = 0; a < np; ++a) cand[P[a]] = z[a];
    double hmax = 0.0;
    for (int i = 0; i < s; ++i) hmax = fmax(hmax, fabs(w->h[i]));
    gram_mv(w->G, ld, s, cand, w->Gv);
    for (int i = 0; i < s; ++i) {
        if (cand[i] != 0.0) continue;
        double c = w->h[i] - w->Gv[i];
        if (fabs(c) > lam * (1.0 + 1e-10) + 1e-13 * hmax) return -1;
    }
    for (int i = 0; i < s; ++i) w->u[i] = cand[i];
    return 0;
}

/* Restricted LASSO on the first s entries of I, warm started from w->u.
 * Returns PG iterations used; *exact = 1 if the exact finish succeeded. */
static int master_problem(work_t* w, int s, double lam, const mpl_oracle_opts* o, double bb,
                          double* f_first, double* L_first, int* exact) {
    const int ld = w->cap;
    double* u = w->u;
    double* y = w->y;
    double* z = w->z;
    double* up = w->up;
    *exact = 0;
    double L = power_iter(w->G, ld, s, w->tmp, w->Gv);
    gram_mv(w->G, ld, s, u, w->Gv);
    double Fu = smooth_part(u, w->Gv, w->h, s) + lam * l1(u, s);
    const double F0 = Fu;
    int iters = 0;
    double eps = o->eps_in;
    *f_first = Fu + 0.5 * bb;
    *L_first = L;
    for (int attempt = 0; attempt < o->max_attempts; ++attempt) {
        double t = 1.0;
        memcpy(y, u, sizeof(double) * s);
        memcpy(up, u, sizeof(double) * s);
        for (int it = 0; it < o->s_max; ++it) {
            int restarted = 0;
            for (;;) {
                /* prox-gradient step from y with backtracking on L */
                gram_mv(w->G, ld, s, y, w->Gy);
                double Phy = smooth_part(y, w->Gy, w->h, s);
                for (;;) {
                    for (int i = 0; i < s; ++i) z[i] = soft(y[i] - (w->Gy[i] - w->h[i]) / L, lam / L);
                    gram_mv(w->G, ld, s, z, w->Gv);
                    double Phz = smooth_part(z, w->Gv, w->h, s);
                    double lin = 0.0, dd = 0.0;
                    for (int i = 0; i < s; ++i) {
                        double d = z[i] - y[i];
                        lin += (w->Gy[i] - w->h[i]) * d;
                        dd += d * d;
                    }
                    double tolq = 1e-15 * (fabs(Phy) + 1.0);
                    if (Phz <= Phy + lin + 0.5 * L * dd + tolq) break;
                    L *= 2.0;
                }
                double Fz = smooth_part(z, w->Gv, w->h, s) + lam * l1(z, s);
                if (Fz <= Fu || restarted) {
                    if (iters == 0) { *f_first = Fz + 0.5 * bb; *L_first = L; }
                    double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
                    double beta = restarted ? 0.0 : (t - 1.0) / tn;
                    for (int i = 0; i < s; ++i) {
                        double zi = z[i];
                        y[i] = zi + beta * (zi - u[i]);
                        up[i] = u[i];
                        u[i] = zi;
                    }
                    t = restarted ? 1.0 : tn;
                    double Fprev = Fu;
                    Fu = (Fz <= Fu) ? Fz : Fu;
                    ++iters;
                    double num = Fprev - Fu, den = F0 - Fu;
                    int stop = 0;
                    if (den <= 0.0) stop = (num <= 0.0);
                    else stop = (num / den <= eps);
                    if (stop) goto attempt_done;
                    break;
                }
                /* objective went up: restart momentum from u with a plain PG step */
                t = 1.0;
                memcpy(y, u, sizeof(double) * s);
                restarted = 1;
            }
        }
    attempt_done:
        if (!o->exact_finish) break;
        if (exact_finish(w, s, lam) == 0) { *exact = 1; break; }
        eps *= 1e-2;
        if (eps < 1e-300) eps = 0.0;
    }
    return iters;
}

/* g = A^T xi (route 0) or beta - Q_I x_I (route 1). */
static void worst_case_g(const double* At, int n, int m, const double* Q, const double* beta,
                         const work_t* w, int s, int route, double* g) {
    if (route == 0) {
        for (int j = 0; j < m; ++j) g[j] = dotd(At + (size_t)j * n, w->r, n);
    } else {
        for (int j = 0; j < m; ++j) {
            double acc = beta[j];
            const double* Qj = Q + (size_t)j * m;
            for (int a = 0; a < s; ++a) acc -= Qj[w->I[a]] * w->u[a];
            g[j] = acc;
        }
    }
}

typedef struct { double key; int idx; } rank_t;

static int rank_cmp(const void* pa, const void* pb) {
    const rank_t* a = pa;
    const rank_t* b = pb;
    if (a->key > b->key) return -1;
    if (a->key < b->key) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

/* KKT violation and duality gap of x (dense, length m) for signal b. */
static void certify(const double* At, int n, int m, const double* b, double lam, const double* x,
                    double* r, double* objective, double* kkt, double* gap, int* nnz) {
    for (int k = 0; k < n; ++k) r[k] = b[k];
    double l1x = 0.0;
    int nz = 0;
    for (int j = 0; j < m; ++j) {
        if (x[j] == 0.0) continue;
        ++nz;
        l1x += fabs(x[j]);
        const double* a = At + (size_t)j * n;
        for (int k = 0; k < n; ++k) r[k] -= a[k] * x[j];
    }
    double rr = dotd(r, r, n), rb = dotd(r, b, n);
    double worst = 0.0, ginf = 0.0;
    for (int j = 0; j < m; ++j) {
        double gj = dotd(At + (size_t)j * n, r, n);
        ginf = fmax(ginf, fabs(gj));
        double v = (x[j] != 0.0) ? fabs(gj - lam * sgn(x[j])) : fmax(fabs(gj) - lam, 0.0);
        worst = fmax(worst, v);
    }
    double P = lam * l1x + 0.5 * rr;
    double sc = (ginf > lam && ginf > 0.0) ? lam / ginf : 1.0;
    double D = -0.5 * sc * sc * rr + sc * rb;
    *objective = P;
    *kkt = lam > 0.0 ? worst / lam : worst;
    *gap = P > 0.0 ? (P - D) / P : 0.0;
    *nnz = nz;
}

typedef struct { double key; int pos; } keep_t;

static int keep_cmp(const void* pa, const void* pb) {
    const keep_t* a = pa;
    const keep_t* b = pb;
    if (a->key > b->key) return -1;
    if (a->key < b->key) return 1;
    return (a->pos > b->pos) - (a->pos < b->pos);
}

/* Algorithm 2, last steps: of the q atoms appended at positions s0..s0+q-1,
 * keep the `keep` with the largest |u| (ties to the earlier position); the
 * others leave I.  I, u, h and G are compacted in place, order preserved.
 * Returns the new |I|. */
static int smpl_prune(work_t* w, int s0, int q, int keep) {
    const int ld = w->cap;
    keep_t* k = malloc(sizeof(keep_t) * (size_t)q);
    char* stay = calloc((size_t)q, 1);
    int* from = malloc(sizeof(int) * (size_t)(s0 + q));
    if (!k || !stay || !from) { free(k); free(stay); free(from); return -1; }
    for (int a = 0; a < q; ++a) { k[a].key = fabs(w->u[s0 + a]); k[a].pos = a; }
    qsort(k, (size_t)q, sizeof(keep_t), keep_cmp);
    for (int a = 0; a < keep; ++a) stay[k[a].pos] = 1;
    int ns = 0;
    for (int a = 0; a < s0 + q; ++a)
        if (a < s0 || stay[a - s0]) from[ns++] = a;
        else w->inI[w->I[a]] = 0;
    /* forward copies: from[a] >= a, so no source is overwritten before it is read */
    for (int a = 0; a < ns; ++a) {
        const int fa = from[a];
        w->I[a] = w->I[fa];
        w->u[a] = w->u[fa];
        w->h[a] = w->h[fa];
        for (int c = 0; c < ns; ++c) w->G[(size_t)a * ld + c] = w->G[(size_t)fa * ld + from[c]];
    }
    for (int a = ns; a < s0 + q; ++a) w->u[a] = 0.0;
    free(k); free(stay); free(from);
    return ns;
}

static int solve_one(const double* At, int n, int m, const double* Q, const double* beta_in,
                     const double* b, double lam, const mpl_oracle_opts* o, work_t* w,
                     double* x, mpl_oracle_result* res, mpl_oracle_trace* tr) {
    const int rho = o->rho > 0 ? o->rho : 1;
    const int omega = o->omega > 1 ? o->omega : 1;
    const int max_outer = o->max_outer > 0 ? o->max_outer : m / rho + 2;
    memset(w->inI, 0, (size_t)m);
    for (int k = 0; k < n; ++k) w->r[k] = b[k];
    const double bb = dotd(b, b, n);
    double* beta = NULL;
    if (o->corr_route == 1) {
        beta = w->xs; /* beta = A^T b, kept for the whole solve */
        if (beta_in) memcpy(beta, beta_in, sizeof(double) * m);
        else for (int j = 0; j < m; ++j) beta[j] = dotd(At + (size_t)j * n, b, n);
    }
    int s = 0, outer = 0, inner_total = 0, status = 1, inexact = 0;
    double f_cur = 0.5 * bb;
    for (outer = 0; outer < max_outer; ++outer) {
        worst_case_g(At, n, m, Q, beta, w, s, o->corr_route, w->g);
        /* early stopping, eq. (stop1) */
        if (o->stop_rinf >= 0.0 || o->stop_r2 >= 0.0) {
            double ginf = 0.0;
            for (int j = 0; j < m; ++j) ginf = fmax(ginf, fabs(w->g[j]));
            const double rn = sqrt(dotd(w->r, w->r, n));
            if ((o->stop_rinf >= 0.0 && ginf <= o->stop_rinf) || (o->stop_r2 >= 0.0 && rn <= o->stop_r2)) {
                if (tr && outer < tr->cap) { tr->n_added[outer] = 0; tr->f_prev[outer] = f_cur; }
                status = 3;
                ++outer;
                break;
            }
        }
        /* rank the violators outside I */
        int nc = 0;
        rank_t* rk = (rank_t*)malloc(sizeof(rank_t) * (size_t)m);
        if (!rk) return -1;
        for (int j = 0; j < m; ++j) {
            if (w->inI[j]) continue;
            double a = fabs(w->g[j]);
            if (a > lam) { rk[nc].key = a; rk[nc].idx = j; ++nc; }
        }
        qsort(rk, (size_t)nc, sizeof(rank_t), rank_cmp);
        const int want = omega * rho;
        int q = nc < want ? nc : want;
        if (tr && outer < tr->cap) tr->f_prev[outer] = f_cur;
        if (q == 0) {
            free(rk);
            status = 0;
            ++outer; /* this evaluation of g counts */
            break;
        }
        if (work_grow(w, s + q) != 0) { free(rk); return -1; }
        const int ld = w->cap;
        for (int a = 0; a < q; ++a) {
            int j = rk[a].idx;
            w->inI[j] = 1;
            w->I[s + a] = j;
            w->u[s + a] = 0.0; /* warm start: new entries start at zero (Alg. 1) */
        }
        free(rk);
        /* new rows/columns of G = A_I^T A_I and new entries of h = A_I^T b */
        for (int a = s; a < s + q; ++a) {
            const double* aj = At + (size_t)w->I[a] * n;
            w->h[a] = dotd(aj, b, n);
            for (int c = 0; c <= a; ++c) {
                double v = dotd(At + (size_t)w->I[c] * n, aj, n);
                w->G[(size_t)a * ld + c] = v;
                w->G[(size_t)c * ld + a] = v;
            }
        }
        double f_first = 0.0, L_first = 0.0;
        int exact = 0;
        int it = master_problem(w, s + q, lam, o, bb, &f_first, &L_first, &exact);
        inner_total += it;
        if (!exact) inexact = 1;
        const int keep = q < rho ? q : rho;
        const int s0 = s;
        if (omega > 1 && q > keep) {
            s = smpl_prune(w, s0, q, keep);
            if (s < 0) return -1;
        } else {
            s += q;
        }
        if (tr && outer < tr->cap) {  /* J_t: the atoms that joined I, in selection order */
            tr->n_added[outer] = s - s0;
            for (int a = s0; a < s && a - s0 < tr->rho_cap; ++a) {
                tr->added[outer * tr->rho_cap + a - s0] = w->I[a];
                tr->gsel[outer * tr->rho_cap + a - s0] = fabs(w->g[w->I[a]]);
            }
        }
        /* xi = b - A_I x_I */
        for (int k = 0; k < n; ++k) w->r[k] = b[k];
        for (int a = 0; a < s; ++a) {
            double v = w->u[a];
            if (v == 0.0) continue;
            const double* aj = At + (size_t)w->I[a] * n;
            for (int k = 0; k < n; ++k) w->r[k] -= aj[k] * v;
        }
        const double f_before = f_cur;
        f_cur = lam * l1(w->u, s) + 0.5 * dotd(w->r, w->r, n);
        if (tr && outer < tr->cap) {
            tr->f_first[outer] = f_first;
            tr->L_first[outer] = L_first;
            tr->f_iter[outer] = f_cur;
            tr->inner[outer] = it;
        }
        /* early stopping, eq. (stop_con) */
        if (o->stop_eps >= 0.0 && (f_before - f_cur) / fabs((double)rho * 0.5 * bb) <= o->stop_eps) {
            status = 3;
            ++outer;
            break;
        }
    }
    for (int j = 0; j < m; ++j) x[j] = 0.0;
    for (int a = 0; a < s; ++a) x[w->I[a]] = w->u[a];
    res->n_outer = outer;
    res->n_inner = inner_total;
    res->S_size = s;
    res->status = (status == 0 && inexact) ? 2 : status;
    certify(At, n, m, b, lam, x, w->r, &res->objective, &res->kkt, &res->gap, &res->nnz);
    return 0;
}

static void default_opts(mpl_oracle_opts* o) {
    o->rho = 1; o->max_outer = 0; o->s_max = 100000; o->max_attempts = 6;
    o->exact_finish = 1; o->corr_route = 0; o->eps_in = 1e-10;
    o->omega = 1; o->stop_rinf = -1.0; o->stop_r2 = -1.0; o->stop_eps = -1.0;
}

void oracle_default_opts(mpl_oracle_opts* o) { default_opts(o); }

static int initial_cap(const mpl_oracle_opts* o, int m) {
    int c = 4 * (o->rho > 0 ? o->rho : 1);
    if (c < 16) c = 16;
    if (c > m) c = m;
    return c;
}

/* Q = A^T A (row j = A^T a_j), for the BMPL identity route. */
static double* gram_full(const double* At, int n, int m) {
    double* Q = malloc(sizeof(double) * (size_t)m * m);
    if (!Q) return NULL;
    for (int j = 0; j < m; ++j)
        for (int i = 0; i <= j; ++i) {
            double v = dotd(At + (size_t)i * n, At + (size_t)j * n, n);
            Q[(size_t)j * m + i] = v;
            Q[(size_t)i * m + j] = v;
        }
    return Q;
}

/* Single-signal MPL.  At: m x n atom-major (column-major A), b: n. */
int oracle_mpl(const double* At, int n, int m, const double* b, double lam,
               const mpl_oracle_opts* o, double* x, mpl_oracle_result* res, mpl_oracle_trace* tr) {
    if (!At || !b || !x || !res || !o || n <= 0 || m <= 0 || !(lam >= 0.0)) return -2;
    work_t w;
    if (work_alloc(&w, n, m, initial_cap(o, m)) != 0) return -1;
    double* Q = NULL;
    if (o->corr_route == 1) {
        Q = gram_full(At, n, m);
        if (!Q) { work_free(&w); return -1; }
    }
    int rc = solve_one(At, n, m, Q, NULL, b, lam, o, &w, x, res, tr);
    free(Q);
    work_free(&w);
    return rc;
}

/* Batch mode: p independent signals (eq. 3 separates by column).  B: p x n
 * (column-major n x p), lam: p, X: p x m (column-major m x p), res: p.
 * Signals run in parallel over nthreads host threads (<= 0: all). */
int oracle_bmpl(const double* At, int n, int m, const double* B, int p, const double* lam,
                const mpl_oracle_opts* o, int nthreads, double* X, mpl_oracle_result* res) {
    if (!At || !B || !lam || !X || !res || !o || n <= 0 || m <= 0 || p < 0) return -2;
    double* Q = NULL;
    if (o->corr_route == 1) {
        Q = gram_full(At, n, m);
        if (!Q) return -1;
    }
    int failed = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads) reduction(| : failed)
#endif
    {
        work_t w;
        if (work_alloc(&w, n, m, initial_cap(o, m)) != 0) {
            failed = 1;
        } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
            for (int i = 0; i < p; ++i) {
                if (solve_one(At, n, m, Q, NULL, B + (size_t)i * n, lam[i], o, &w,
                              X + (size_t)i * m, res + i, NULL) != 0)
                    failed = 1;
            }
            work_free(&w);
        }
    }
    free(Q);
    return failed ? -1 : 0;
}

/* KKT/gap certificate of a given dense x (used to score the CUDA path's
 * output in the oracle's precision).  r: n scratch. */
int oracle_certify(const double* At, int n, int m, const double* b, double lam, const double* x,
                   double* objective, double* kkt, double* gap, int* nnz) {
    double* r = malloc(sizeof(double) * (size_t)n);
    if (!r) return -1;
    certify(At, n, m, b, lam, x, r, objective, kkt, gap, nnz);
    free(r);
    return 0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
