/*
 * O2: dense bounded-variable primal simplex (test infrastructure only).
 *
 * Solves   min c.x  s.t.  A[0:m_eq] x = q[0:m_eq],  A[m_eq:m] x >= q[m_eq:m],
 *          l <= x <= u  (entries of l, u may be +-HUGE_VAL)
 * exactly (up to the 1e-9 tolerances below), giving the LP optimum that the
 * paper's PDHG only approaches (Sec. II-C: PDHG solves the relaxation and is
 * followed by crossover and simplex to reach a basic solution).  The method is
 * the textbook revised simplex with an explicit dense basis inverse:
 *
 *   standard form   A x - s = q on ">=" rows (s >= 0), plus one artificial per
 *                   row signed so that the all-artificial start is feasible;
 *   phase I         minimise the sum of artificials from x_N at a finite bound
 *                   (free columns at 0);
 *   phase II        artificials fixed to [0, 0], original costs;
 *   pricing         Dantzig (largest |reduced cost|), Bland (lowest index) after
 *                   50 consecutive degenerate pivots until progress resumes;
 *   ratio test      two-pass Harris test with bound flips;
 *   basis inverse   product-form rank-one updates, rebuilt by Gauss-Jordan
 *                   elimination every REFACTOR pivots and at phase ends.
 *
 * Output: x (n), row duals y (m; y >= 0 on ">=" rows), objective.
 * Return: 0 optimal, 1 infeasible, 2 unbounded, 3 iteration limit, -1 error.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define FEAS_TOL 1e-9
#define OPT_TOL 1e-9
#define PIV_TOL 1e-9
#define REFACTOR 1000
#define BLAND_AFTER 50

enum { AT_LO = 0, AT_HI = 1, FREE0 = 2, BASIC = 3 };

typedef struct {
    int m, N;            /* rows, total columns (structural + slack + artificial) */
    int *cp, *ri;        /* CSC of the standard-form matrix */
    double *cv;
    double *lo, *hi, *cost, *x;
    int *state, *basis, *pos;
    double *binv;        /* column-major m x m: binv[c*m + r] */
    double *pi, *d, *alpha, *work;
} Sx;

static int sx_refactor(Sx *s) {
    int m = s->m;
    double *Bm = s->work;                  /* m*m scratch, column-major */
    memset(Bm, 0, sizeof(double) * (size_t)m * m);
    for (int r = 0; r < m; r++) {
        int j = s->basis[r];
        for (int k = s->cp[j]; k < s->cp[j + 1]; k++) Bm[(size_t)r * m + s->ri[k]] = s->cv[k];
    }
    /* Gauss-Jordan on [B | I] held as B (col-major) and binv (col-major) */
    double *Iv = s->binv;
    memset(Iv, 0, sizeof(double) * (size_t)m * m);
    for (int r = 0; r < m; r++) Iv[(size_t)r * m + r] = 1.0;
    int *perm = (int *)malloc(sizeof(int) * m);
    for (int r = 0; r < m; r++) perm[r] = r;
    for (int col = 0; col < m; col++) {
        /* pivot row: largest |B[row, col]| among rows col.. (rows held in perm order) */
        int best = -1; double bv = 0.0;
        for (int rr = col; rr < m; rr++) {
            double v = fabs(Bm[(size_t)col * m + perm[rr]]);
            if (v > bv) { bv = v; best = rr; }
        }
        if (best < 0 || bv < 1e-14) { free(perm); return -1; }
        int t = perm[col]; perm[col] = perm[best]; perm[best] = t;
        int pr = perm[col];
        double piv = Bm[(size_t)col * m + pr];
        /* scale pivot row */
        for (int c = 0; c < m; c++) { Bm[(size_t)c * m + pr] /= piv; Iv[(size_t)c * m + pr] /= piv; }
        /* eliminate other rows */
        for (int rr = 0; rr < m; rr++) {
            int row = perm[rr];
            if (row == pr) continue;
            double f = Bm[(size_t)col * m + row];
            if (f == 0.0) continue;
            for (int c = 0; c < m; c++) {
                Bm[(size_t)c * m + row] -= f * Bm[(size_t)c * m + pr];
                Iv[(size_t)c * m + row] -= f * Iv[(size_t)c * m + pr];
            }
        }
    }
    /* B was reduced to a permutation P (B^-1 computed as Iv with rows permuted):
       after elimination, row perm[col] of the reduced B has its 1 in column col,
       so (P B) = I  =>  B^-1 = P-reordered Iv: row col of B^-1 = row perm[col] of Iv. */
    double *tmp = (double *)malloc(sizeof(double) * m);
    for (int c = 0; c < m; c++) {
        for (int r = 0; r < m; r++) tmp[r] = Iv[(size_t)c * m + perm[r]];
        memcpy(&Iv[(size_t)c * m], tmp, sizeof(double) * m);
    }
    free(tmp);
    free(perm);
    return 0;
}

/* x_B = B^-1 (q - N x_N) */
static void sx_recompute_xb(Sx *s, const double *rhs) {
    int m = s->m;
    double *r = s->work;
    memcpy(r, rhs, sizeof(double) * m);
    for (int j = 0; j < s->N; j++) {
        if (s->state[j] == BASIC || s->x[j] == 0.0) continue;
        for (int k = s->cp[j]; k < s->cp[j + 1]; k++) r[s->ri[k]] -= s->cv[k] * s->x[j];
    }
    for (int i = 0; i < m; i++) {
        double acc = 0.0;
        for (int c = 0; c < m; c++) acc += s->binv[(size_t)c * m + i] * r[c];
        s->x[s->basis[i]] = acc;
    }
}

/* pi^T = c_B^T B^-1 */
static void sx_recompute_pi(Sx *s) {
    int m = s->m;
    for (int c = 0; c < m; c++) {
        double acc = 0.0;
        const double *col = &s->binv[(size_t)c * m];
        for (int r = 0; r < m; r++) acc += s->cost[s->basis[r]] * col[r];
        s->pi[c] = acc;
    }
}

static double sx_reduced_cost(const Sx *s, int j) {
    double v = s->cost[j];
    for (int k = s->cp[j]; k < s->cp[j + 1]; k++) v -= s->pi[s->ri[k]] * s->cv[k];
    return v;
}

/* one phase; returns 0 optimal, 2 unbounded, 3 iteration limit, -1 numerical */
static int sx_phase(Sx *s, const double *rhs, int *iters, int max_iter) {
    int m = s->m;
    int degen = 0, bland = 0, since = 0;
    if (sx_refactor(s)) return -1;
    sx_recompute_xb(s, rhs);
    sx_recompute_pi(s);
    double cmax = 1.0;
    for (int j = 0; j < s->N; j++) if (fabs(s->cost[j]) > cmax) cmax = fabs(s->cost[j]);
    double dtol = OPT_TOL * cmax;
    for (;;) {
        if (*iters >= max_iter) return 3;
        /* pricing */
        int q = -1, dir = 0; double best = 0.0;
        for (int j = 0; j < s->N; j++) {
            int st = s->state[j];
            if (st == BASIC) continue;
            if (s->lo[j] == s->hi[j]) continue;
            double dj = sx_reduced_cost(s, j);
            int dj_dir = 0;
            if ((st == AT_LO || st == FREE0) && dj < -dtol) dj_dir = 1;
            else if ((st == AT_HI || st == FREE0) && dj > dtol) dj_dir = -1;
            if (!dj_dir) continue;
            if (bland) { q = j; dir = dj_dir; best = fabs(dj); break; }
            if (fabs(dj) > best) { best = fabs(dj); q = j; dir = dj_dir; }
        }
        if (q < 0) return 0;
        double dq = sx_reduced_cost(s, q);
        /* FTRAN: alpha = B^-1 a_q */
        memset(s->alpha, 0, sizeof(double) * m);
        for (int k = s->cp[q]; k < s->cp[q + 1]; k++) {
            const double *col = &s->binv[(size_t)s->ri[k] * m];
            double a = s->cv[k];
            for (int r = 0; r < m; r++) s->alpha[r] += a * col[r];
        }
        /* Harris ratio test */
        double theta_max = HUGE_VAL;
        for (int r = 0; r < m; r++) {
            double a = dir * s->alpha[r];
            int b = s->basis[r];
            if (a > PIV_TOL && isfinite(s->lo[b])) {
                double t = (s->x[b] - s->lo[b] + FEAS_TOL) / a;
                if (t < theta_max) theta_max = t;
            } else if (a < -PIV_TOL && isfinite(s->hi[b])) {
                double t = (s->hi[b] + FEAS_TOL - s->x[b]) / (-a);
                if (t < theta_max) theta_max = t;
            }
        }
        double flip = s->hi[q] - s->lo[q];     /* inf for free / half-bounded */
        int leave = -1; double theta = HUGE_VAL, amax = 0.0;
        for (int r = 0; r < m; r++) {
            double a = dir * s->alpha[r];
            int b = s->basis[r];
            double t;
            if (a > PIV_TOL && isfinite(s->lo[b])) t = (s->x[b] - s->lo[b]) / a;
            else if (a < -PIV_TOL && isfinite(s->hi[b])) t = (s->hi[b] - s->x[b]) / (-a);
            else continue;
            if (t <= theta_max) {
                if (bland) {
                    if (leave < 0 || t < theta - 1e-12 || (fabs(t - theta) <= 1e-12 && b < s->basis[leave])) {
                        leave = r; theta = t; amax = fabs(a);
                    }
                } else if (fabs(a) > amax) {
                    amax = fabs(a); leave = r; theta = t;
                }
            }
        }
        if (theta < 0.0) theta = 0.0;
        if (leave < 0 && !isfinite(flip)) return 2;
        (*iters)++;
        if (leave < 0 || flip <= theta) {
            /* bound flip of the entering column */
            double t = flip;
            for (int r = 0; r < m; r++) s->x[s->basis[r]] -= dir * t * s->alpha[r];
            if (dir > 0) { s->x[q] = s->hi[q]; s->state[q] = AT_HI; }
            else { s->x[q] = s->lo[q]; s->state[q] = AT_LO; }
            degen = 0; bland = 0;
            continue;
        }
        if (theta <= 1e-12) { if (++degen > BLAND_AFTER) bland = 1; }
        else { degen = 0; bland = 0; }
        /* primal update */
        for (int r = 0; r < m; r++) s->x[s->basis[r]] -= dir * theta * s->alpha[r];
        s->x[q] += dir * theta;
        int b = s->basis[leave];
        double a_r = s->alpha[leave];
        if (dir * a_r > 0) { s->x[b] = s->lo[b]; s->state[b] = AT_LO; }
        else { s->x[b] = s->hi[b]; s->state[b] = AT_HI; }
        s->pos[b] = -1;
        s->basis[leave] = q; s->pos[q] = leave; s->state[q] = BASIC;
        /* dual update with row `leave` of the old inverse: pi += (dq / a_r) rho */
        for (int c = 0; c < m; c++) s->pi[c] += (dq / a_r) * s->binv[(size_t)c * m + leave];
        /* inverse update: new row leave = old / a_r; others -= alpha_i * new row */
        for (int c = 0; c < m; c++) {
            double *col = &s->binv[(size_t)c * m];
            double t = col[leave] / a_r;
            if (t != 0.0) {
                for (int r = 0; r < m; r++) col[r] -= s->alpha[r] * t;
            }
            col[leave] = t;
        }
        if (++since >= REFACTOR) {
            since = 0;
            if (sx_refactor(s)) return -1;
            sx_recompute_xb(s, rhs);
            sx_recompute_pi(s);
        }
    }
}

int oracle_simplex(int m, int n, int m_eq,
                   const int *a_cp, const int *a_ri, const double *a_v,
                   const double *q, const double *c, const double *l, const double *u,
                   int max_iter, double *x_out, double *y_out, double *obj_out, int *iters_out) {
    Sx s;
    memset(&s, 0, sizeof s);
    int mI = m - m_eq;
    s.m = m;
    s.N = n + mI + m;
    int nnz = a_cp[n];
    s.cp = (int *)calloc(s.N + 1, sizeof(int));
    s.ri = (int *)malloc(sizeof(int) * (nnz + mI + m + 1));
    s.cv = (double *)malloc(sizeof(double) * (nnz + mI + m + 1));
    s.lo = (double *)malloc(sizeof(double) * s.N);
    s.hi = (double *)malloc(sizeof(double) * s.N);
    s.cost = (double *)calloc(s.N, sizeof(double));
    s.x = (double *)calloc(s.N, sizeof(double));
    s.state = (int *)calloc(s.N, sizeof(int));
    s.basis = (int *)malloc(sizeof(int) * m);
    s.pos = (int *)malloc(sizeof(int) * s.N);
    s.binv = (double *)malloc(sizeof(double) * (size_t)m * m);
    s.work = (double *)malloc(sizeof(double) * ((size_t)m * m + m + 1));
    s.pi = (double *)calloc(m + 1, sizeof(double));
    s.alpha = (double *)calloc(m + 1, sizeof(double));
    if (!s.cp || !s.ri || !s.cv || !s.lo || !s.hi || !s.cost || !s.x || !s.state || !s.basis ||
        !s.pos || !s.binv || !s.work || !s.pi || !s.alpha)
        return -1;
    int k = 0;
    for (int j = 0; j < n; j++) {
        s.cp[j] = k;
        for (int t = a_cp[j]; t < a_cp[j + 1]; t++) { s.ri[k] = a_ri[t]; s.cv[k] = a_v[t]; k++; }
        s.lo[j] = l[j]; s.hi[j] = u[j];
    }
    for (int i = 0; i < mI; i++) {
        int j = n + i;
        s.cp[j] = k; s.ri[k] = m_eq + i; s.cv[k] = -1.0; k++;
        s.lo[j] = 0.0; s.hi[j] = HUGE_VAL;
    }
    /* nonbasic start values */
    for (int j = 0; j < n + mI; j++) {
        if (isfinite(s.lo[j])) { s.x[j] = s.lo[j]; s.state[j] = AT_LO; }
        else if (isfinite(s.hi[j])) { s.x[j] = s.hi[j]; s.state[j] = AT_HI; }
        else { s.x[j] = 0.0; s.state[j] = FREE0; }
        s.pos[j] = -1;
    }
    double *r = (double *)malloc(sizeof(double) * m);
    memcpy(r, q, sizeof(double) * m);
    for (int j = 0; j < n + mI; j++) {
        if (s.x[j] == 0.0) continue;
        for (int t = s.cp[j]; t < s.cp[j + 1]; t++) r[s.ri[t]] -= s.cv[t] * s.x[j];
    }
    for (int i = 0; i < m; i++) {
        int j = n + mI + i;
        s.cp[j] = k; s.ri[k] = i; s.cv[k] = (r[i] >= 0.0) ? 1.0 : -1.0; k++;
        s.lo[j] = 0.0; s.hi[j] = HUGE_VAL;
        s.x[j] = fabs(r[i]);
        s.state[j] = BASIC; s.basis[i] = j; s.pos[j] = i;
        s.cost[j] = 1.0;
    }
    s.cp[s.N] = k;
    free(r);

    int iters = 0;
    int rc = sx_phase(&s, q, &iters, max_iter);
    int status = 0;
    if (rc == 3) status = 3;
    else if (rc < 0) status = -1;
    else {
        double infeas = 0.0, qmax = 1.0;
        for (int i = 0; i < m; i++) { infeas += s.x[n + mI + i]; if (fabs(q[i]) > qmax) qmax = fabs(q[i]); }
        if (infeas > 1e-7 * qmax) status = 1;
    }
    if (status == 0) {
        for (int j = 0; j < s.N; j++) s.cost[j] = 0.0;
        for (int j = 0; j < n; j++) s.cost[j] = c[j];
        for (int i = 0; i < m; i++) {
            int j = n + mI + i;
            s.hi[j] = 0.0;
            if (s.state[j] != BASIC) { s.x[j] = 0.0; s.state[j] = AT_LO; }
        }
        rc = sx_phase(&s, q, &iters, max_iter);
        if (rc == 2) status = 2;
        else if (rc == 3) status = 3;
        else if (rc < 0) status = -1;
        else {
            /* clean final solve */
            if (sx_refactor(&s)) status = -1;
            else { sx_recompute_xb(&s, q); sx_recompute_pi(&s); }
        }
    }
    double obj = 0.0;
    for (int j = 0; j < n; j++) { x_out[j] = s.x[j]; obj += c[j] * s.x[j]; }
    for (int i = 0; i < m; i++) y_out[i] = s.pi[i];
    *obj_out = obj;
    *iters_out = iters;
    free(s.cp); free(s.ri); free(s.cv); free(s.lo); free(s.hi); free(s.cost); free(s.x);
    free(s.state); free(s.basis); free(s.pos); free(s.binv); free(s.work); free(s.pi); free(s.alpha);
    return status;
}
