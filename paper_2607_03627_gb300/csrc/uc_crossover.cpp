// Crossover from a PDHG point to a vertex of the presolved LP (host).
//
// The paper's GPU arm runs PDHG, then crossover, then simplex clean-up
// (Sec. II-C, Alg. 1 "Solver 1"; Sec. III-C): PDHG gives a point near the
// optimal face, crossover turns it into a basic solution.  The paper does not
// state the crossover; this is the textbook scheme (Megiddo's primal push with
// a simplex clean-up, as in Bixby and Saltzman 1994), on the scaled presolved
// LP
//
//   min c.x   s.t.  A_E x = q_E,  A_I x - s = q_I,  l <= x <= u,  s >= 0,
//
// with a bounded revised simplex whose nonbasic variables may sit strictly
// between their bounds ("superbasic") so that it can start from the PDHG
// point itself:
//
//   1. every column is set to the PDHG value clipped to its bounds (snapped to
//      a bound within 1e-9 relative), every surplus to its row activity;
//   2. phase 1: an artificial per row carries that row's residual, and the
//      simplex drives the artificials to zero (they are then fixed at 0);
//   3. phase 2: the simplex on c.x with Dantzig pricing (Bland's rule after a
//      run of degenerate steps); superbasics move in whichever direction
//      lowers the objective;
//   4. primal push: every superbasic left (zero reduced cost) moves to one of
//      its bounds, or into the basis, by a ratio test; free columns enter the
//      basis; then phase 2 again if a push made some column attractive.
//
// The result has every nonbasic variable at a bound: a vertex.  The basis
// inverse is dense (m x m), updated by the product form at each pivot and
// recomputed from scratch (Gauss-Jordan with partial pivoting) every
// kRefactor pivots, so the crossover is for LPs with up to kMaxRows rows.

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <limits>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "uc_internal.h"

namespace uc {
namespace {

constexpr double kInf = std::numeric_limits<double>::infinity();
constexpr double kOptTol = 1e-9;      // reduced-cost optimality
constexpr double kPivTol = 1e-9;      // smallest pivot element taken
constexpr int kRefactor = 100;
constexpr int kBlandAfter = 50;       // degenerate steps before Bland's rule
constexpr int kMaxRows = 20000;

enum VarState : int8_t { BASIC = 0, AT_LOWER, AT_UPPER, SUPER };

struct Simplex {
    int m = 0, nx = 0, ns = 0, nv = 0;          // rows, columns, surplus, all variables (+ m artificials)
    // columns of [A | -I_I | artificials] in compressed form
    std::vector<int32_t> cp, ri;
    std::vector<double> cv;
    std::vector<double> lo, hi, cost, val, q;
    std::vector<int8_t> st;
    std::vector<int> head;                      // basic variable of each row position
    std::vector<double> Binv;                   // m x m, row-major
    int pivots = 0, since_refactor = 0, degenerate = 0;
    int64_t max_pivots = 0;
    const volatile int *cancel = nullptr;       // nonzero: stop at the next pivot

    void column(int j, std::vector<double> &dense) const {
        std::fill(dense.begin(), dense.end(), 0.0);
        for (int32_t e = cp[j]; e < cp[j + 1]; e++) dense[ri[e]] = cv[e];
    }
    // alpha = Binv M_j
    void ftran(int j, std::vector<double> &alpha) const {
        std::fill(alpha.begin(), alpha.end(), 0.0);
        for (int32_t e = cp[j]; e < cp[j + 1]; e++) {
            const int r = ri[e];
            const double a = cv[e];
            for (int k = 0; k < m; k++) alpha[k] += Binv[(size_t)k * m + r] * a;
        }
    }
    // recompute Binv from the basis columns; false if the basis is singular
    bool refactor() {
        std::vector<double> Bm((size_t)m * m, 0.0), col(m);
        for (int k = 0; k < m; k++) {
            column(head[k], col);
            for (int r = 0; r < m; r++) Bm[(size_t)r * m + k] = col[r];
        }
        Binv.assign((size_t)m * m, 0.0);
        for (int r = 0; r < m; r++) Binv[(size_t)r * m + r] = 1.0;
        for (int k = 0; k < m; k++) {
            int p = k;
            double best = std::fabs(Bm[(size_t)k * m + k]);
            for (int r = k + 1; r < m; r++)
                if (std::fabs(Bm[(size_t)r * m + k]) > best) { best = std::fabs(Bm[(size_t)r * m + k]); p = r; }
            if (best < 1e-12) return false;
            if (p != k)
                for (int c = 0; c < m; c++) {
                    std::swap(Bm[(size_t)k * m + c], Bm[(size_t)p * m + c]);
                    std::swap(Binv[(size_t)k * m + c], Binv[(size_t)p * m + c]);
                }
            const double inv = 1.0 / Bm[(size_t)k * m + k];
            for (int c = 0; c < m; c++) { Bm[(size_t)k * m + c] *= inv; Binv[(size_t)k * m + c] *= inv; }
            for (int r = 0; r < m; r++) {
                if (r == k) continue;
                const double f = Bm[(size_t)r * m + k];
                if (f == 0.0) continue;
                for (int c = 0; c < m; c++) {
                    Bm[(size_t)r * m + c] -= f * Bm[(size_t)k * m + c];
                    Binv[(size_t)r * m + c] -= f * Binv[(size_t)k * m + c];
                }
            }
        }
        since_refactor = 0;
        return true;
    }
    // basic values from the nonbasic ones: x_B = Binv (q - M_N x_N)
    void basic_values() {
        std::vector<double> r(q);
        for (int j = 0; j < nv; j++) {
            if (st[j] == BASIC || val[j] == 0.0) continue;
            for (int32_t e = cp[j]; e < cp[j + 1]; e++) r[ri[e]] -= cv[e] * val[j];
        }
        for (int k = 0; k < m; k++) {
            double s = 0.0;
            for (int i = 0; i < m; i++) s += Binv[(size_t)k * m + i] * r[i];
            val[head[k]] = s;
        }
    }
    // simplex multipliers y = c_B^T Binv
    void duals(std::vector<double> &y) const {
        std::fill(y.begin(), y.end(), 0.0);
        for (int k = 0; k < m; k++) {
            const double cb = cost[head[k]];
            if (cb == 0.0) continue;
            for (int i = 0; i < m; i++) y[i] += cb * Binv[(size_t)k * m + i];
        }
    }
    double reduced(int j, const std::vector<double> &y) const {
        double d = cost[j];
        for (int32_t e = cp[j]; e < cp[j + 1]; e++) d -= cv[e] * y[ri[e]];
        return d;
    }
    // Move nonbasic j in direction dir (+1 up, -1 down) as far as the bounds
    // allow.  0: moved (pivot or bound flip); 1: unbounded; 2: no step possible
    // for a free column that cannot enter.
    int step(int j, int dir, std::vector<double> &alpha) {
        ftran(j, alpha);
        double theta = dir > 0 ? hi[j] - val[j] : val[j] - lo[j];
        int leave = -1;
        double leave_piv = 0.0;
        for (int k = 0; k < m; k++) {
            const double a = dir * alpha[k];
            if (std::fabs(a) <= kPivTol) continue;
            const int b = head[k];
            const double lim = a > 0 ? (val[b] - lo[b]) / a : (hi[b] - val[b]) / -a;
            const double t = std::max(lim, 0.0);
            if (t < theta - 1e-12 || (t <= theta + 1e-12 && leave >= 0 && std::fabs(a) > leave_piv)) {
                theta = t;
                leave = k;
                leave_piv = std::fabs(a);
            }
        }
        if (!std::isfinite(theta)) return 1;
        for (int k = 0; k < m; k++) val[head[k]] -= dir * theta * alpha[k];
        val[j] += dir * theta;
        degenerate = theta <= 1e-12 ? degenerate + 1 : 0;
        if (leave < 0) {                          // bound flip
            st[j] = dir > 0 ? AT_UPPER : AT_LOWER;
            val[j] = dir > 0 ? hi[j] : lo[j];
            return 0;
        }
        const int b = head[leave];
        const double a = dir * alpha[leave];
        st[b] = a > 0 ? AT_LOWER : AT_UPPER;
        val[b] = a > 0 ? lo[b] : hi[b];
        st[j] = BASIC;
        head[leave] = j;
        // product-form update of Binv with pivot alpha[leave]
        const double piv = alpha[leave];
        double *rowk = &Binv[(size_t)leave * m];
        for (int c = 0; c < m; c++) rowk[c] /= piv;
        for (int r = 0; r < m; r++) {
            if (r == leave || alpha[r] == 0.0) continue;
            const double f = alpha[r];
            double *row = &Binv[(size_t)r * m];
            for (int c = 0; c < m; c++) row[c] -= f * rowk[c];
        }
        pivots++;
        if (++since_refactor >= kRefactor) {
            if (!refactor()) return 3;
            basic_values();
        }
        return 0;
    }
    // simplex iterations on the current cost vector: 0 optimal, 1 unbounded,
    // 3 singular basis, 4 pivot limit, 5 cancelled
    int iterate(std::vector<double> &y, std::vector<double> &alpha) {
        for (;;) {
            if (pivots >= max_pivots) return 4;
            if (cancel && *cancel) return 5;
            duals(y);
            int enter = -1, dir = 0;
            double best = kOptTol;
            const bool bland = degenerate >= kBlandAfter;
            for (int j = 0; j < nv; j++) {
                if (st[j] == BASIC || lo[j] == hi[j]) continue;
                const double d = reduced(j, y);
                int dj = 0;
                if (d < -kOptTol && (st[j] == AT_LOWER || st[j] == SUPER) && val[j] < hi[j]) dj = 1;
                else if (d > kOptTol && (st[j] == AT_UPPER || st[j] == SUPER) && val[j] > lo[j]) dj = -1;
                if (!dj) continue;
                if (bland) { enter = j; dir = dj; break; }
                if (std::fabs(d) > best) { best = std::fabs(d); enter = j; dir = dj; }
            }
            if (enter < 0) return 0;
            const int rc = step(enter, dir, alpha);
            if (rc == 1) return 1;
            if (rc == 3) return 3;
        }
    }
};

}  // namespace

// Crossover of a finished solve's returned point (see the top of the file).
int crossover(const PsData &p, const std::vector<double> &xs, int64_t max_pivots, std::vector<double> &x_out,
              std::vector<double> &y_out, int &pivots, int &superbasic_left, const volatile int *cancel) {
    const int m = p.m(), n = p.n();
    if (m > kMaxRows) {
        set_error("uc_crossover: %d rows; the dense-basis crossover takes at most %d", m, kMaxRows);
        return UC_EINVAL;
    }
    Simplex S;
    S.m = m;
    S.nx = n;
    S.ns = m - p.m_eq;
    S.nv = n + S.ns + m;
    S.max_pivots = max_pivots > 0 ? max_pivots : 50LL * (n + m);
    S.cancel = cancel;
    S.cp.assign((size_t)S.nv + 1, 0);
    // structural columns from A^T rows, surplus -e_i for ">=" rows, artificials later
    for (int j = 0; j < n; j++) {
        for (int32_t e = p.AT.rowptr[j]; e < p.AT.rowptr[j + 1]; e++) {
            S.ri.push_back(p.AT.colidx[e]);
            S.cv.push_back(p.AT.val[e]);
        }
        S.cp[j + 1] = (int32_t)S.ri.size();
    }
    for (int s = 0; s < S.ns; s++) {
        S.ri.push_back(p.m_eq + s);
        S.cv.push_back(-1.0);
        S.cp[n + s + 1] = (int32_t)S.ri.size();
    }
    S.lo.assign(S.nv, 0.0); S.hi.assign(S.nv, kInf); S.cost.assign(S.nv, 0.0); S.val.assign(S.nv, 0.0);
    S.st.assign(S.nv, AT_LOWER);
    S.q = p.q;
    for (int j = 0; j < n; j++) {
        S.lo[j] = p.l[j];
        S.hi[j] = p.u[j];
        double v = std::min(std::max(xs[j], p.l[j]), p.u[j]);
        const double tol = 1e-9 * (1.0 + std::fabs(v));
        if (std::isfinite(p.l[j]) && v - p.l[j] <= tol) { v = p.l[j]; S.st[j] = AT_LOWER; }
        else if (std::isfinite(p.u[j]) && p.u[j] - v <= tol) { v = p.u[j]; S.st[j] = AT_UPPER; }
        else S.st[j] = SUPER;
        S.val[j] = v;
    }
    // surplus = row activity - q (>= 0), snapped to 0 within the tolerance
    std::vector<double> act(m, 0.0);
    for (int i = 0; i < m; i++)
        for (int32_t e = p.A.rowptr[i]; e < p.A.rowptr[i + 1]; e++) act[i] += p.A.val[e] * S.val[p.A.colidx[e]];
    for (int s = 0; s < S.ns; s++) {
        const int i = p.m_eq + s, v = n + s;
        const double sl = act[i] - p.q[i];
        if (sl <= 1e-9 * (1.0 + std::fabs(p.q[i]))) { S.val[v] = 0.0; S.st[v] = AT_LOWER; }
        else { S.val[v] = sl; S.st[v] = SUPER; }
    }
    // artificials carry the residual q - M x, signed so that they start >= 0
    std::vector<double> res(p.q);
    for (int j = 0; j < n + S.ns; j++)
        for (int32_t e = S.cp[j]; e < S.cp[j + 1]; e++) res[S.ri[e]] -= S.cv[e] * S.val[j];
    S.head.resize(m);
    for (int i = 0; i < m; i++) {
        const int a = n + S.ns + i;
        S.ri.push_back(i);
        S.cv.push_back(res[i] >= 0.0 ? 1.0 : -1.0);
        S.cp[a + 1] = (int32_t)S.ri.size();
        S.val[a] = std::fabs(res[i]);
        S.st[a] = BASIC;
        S.head[i] = a;
        S.cost[a] = 1.0;                         // phase 1
    }
    S.Binv.assign((size_t)m * m, 0.0);
    for (int i = 0; i < m; i++) S.Binv[(size_t)i * m + i] = res[i] >= 0.0 ? 1.0 : -1.0;
    std::vector<double> y(m), alpha(m);
    int rc = S.iterate(y, alpha);
    if (rc == 5) { set_error("uc_crossover: cancelled"); return UC_ECANCELLED; }
    if (rc == 4) { set_error("uc_crossover: pivot limit in phase 1"); return UC_EITERLIMIT; }
    if (rc) { set_error("uc_crossover: phase 1 failed (%d)", rc); return UC_ENUMERIC; }
    double infeas = 0.0;
    for (int i = 0; i < m; i++) infeas += S.val[n + S.ns + i];
    if (infeas > 1e-7 * (1.0 + m)) { set_error("uc_crossover: no feasible basis (artificial sum %g)", infeas); return UC_EINFEASIBLE; }
    for (int i = 0; i < m; i++) {                // artificials are fixed at 0 from here on
        const int a = n + S.ns + i;
        S.cost[a] = 0.0;
        S.hi[a] = 0.0;
        if (S.st[a] != BASIC) { S.st[a] = AT_LOWER; S.val[a] = 0.0; }
    }
    for (int j = 0; j < n; j++) S.cost[j] = p.c[j];
    S.degenerate = 0;
    for (int round = 0; round < 4; round++) {
        rc = S.iterate(y, alpha);
        if (rc == 5) { set_error("uc_crossover: cancelled"); return UC_ECANCELLED; }
        if (rc == 4) { set_error("uc_crossover: pivot limit in phase 2"); return UC_EITERLIMIT; }
        if (rc) { set_error("uc_crossover: phase 2 failed (%d)", rc); return rc == 1 ? UC_EUNBOUNDED : UC_ENUMERIC; }
        // primal push: superbasics to a bound or into the basis
        bool pushed = false;
        for (int j = 0; j < S.nv; j++) {
            if (S.st[j] != SUPER) continue;
            const double dlo = S.val[j] - S.lo[j], dhi = S.hi[j] - S.val[j];
            const int dir = (std::isfinite(dhi) && (dhi <= dlo || !std::isfinite(dlo))) ? 1 : -1;
            if (S.step(j, dir, alpha) == 0) pushed = true;
            else if (S.step(j, -dir, alpha) == 0) pushed = true;
        }
        if (!pushed) break;
        if (!S.refactor()) { set_error("uc_crossover: singular basis"); return UC_ENUMERIC; }
        S.basic_values();
    }
    if (!S.refactor()) { set_error("uc_crossover: singular basis"); return UC_ENUMERIC; }
    S.basic_values();
    superbasic_left = 0;
    for (int j = 0; j < S.nv; j++) superbasic_left += S.st[j] == SUPER;
    x_out.assign(S.val.begin(), S.val.begin() + n);
    S.duals(y);
    y_out = y;
    pivots = S.pivots;
    return UC_OK;
}

// A vertex-optimal result of the LP by the host simplex from the cold start
// (every column at its bound nearest 0): the CPU arm of the concurrent solve.
static int simplex_result(const std::shared_ptr<const PsData> &p, int64_t max_pivots, const volatile int *cancel,
                          uc_result **out) {
    std::vector<double> x0(p->n());
    for (int j = 0; j < p->n(); j++) x0[j] = std::min(std::max(0.0, p->l[j]), p->u[j]);
    auto r = std::make_unique<uc_result>();
    r->ps = p;
    int pivots = 0, left = 0;
    const auto t0 = std::chrono::steady_clock::now();
    const int rc = crossover(*p, x0, max_pivots, r->x_ret, r->y_ret, pivots, left, cancel);
    if (rc) return rc;
    r->x_cur = r->x_avg = r->x_ret;
    r->y_cur = r->y_avg = r->y_ret;
    uc_stats &o = r->stats;
    std::memset(&o, 0, sizeof o);
    o.status = UC_OK;
    o.iters = pivots;
    o.superbasic = left;
    double pobj, dobj;
    host_kkt(*p, r->x_ret.data(), r->y_ret.data(), o.rel_primal, o.rel_dual, o.rel_gap, o.abs_primal, pobj, dobj);
    o.dual_objective = dobj + p->obj_const;
    o.abs_primal_unpolished = o.abs_primal;
    o.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = r.release();
    return UC_OK;
}

}  // namespace uc

int uc_simplex_solve(const uc_presolved *ps, int64_t max_pivots, const volatile int *cancel, uc_result **out) {
    if (!ps || !out) { uc::set_error("uc_simplex_solve: null argument"); return UC_EINVAL; }
    *out = nullptr;
    try {
        return uc::simplex_result(ps->d, max_pivots, cancel, out);
    } catch (const std::bad_alloc &) {
        uc::set_error("uc_simplex_solve: out of host memory");
        return UC_ENOMEM;
    }
}

// Alg. 1 of the paper (Sec. II-C): both arms on the same LP at once -- the
// device PDHG (uc_solve) on the calling thread and the host simplex on a
// second thread -- and the first arm to end optimal stops the other through
// its cancel flag.  An arm that ends without an optimal result (iteration
// limit, an LP too large for the dense simplex) does not stop the other.
int uc_solve_concurrent(const uc_presolved *ps, const uc_solve_opts *opts, void *stream, uc_result **out,
                        int *winner) {
    if (!ps || !out) { uc::set_error("uc_solve_concurrent: null argument"); return UC_EINVAL; }
    *out = nullptr;
    if (winner) *winner = -1;
    uc_solve_opts o;
    uc_default_solve_opts(&o);
    if (opts) o = *opts;
    volatile int stop_gpu = 0, stop_cpu = 0;
    o.cancel = &stop_gpu;
    uc_result *cpu_res = nullptr;
    int cpu_rc = UC_EINVAL;
    std::string cpu_err;
    std::thread cpu([&]() {
        cpu_rc = uc_simplex_solve(ps, 0, &stop_cpu, &cpu_res);
        if (cpu_rc == UC_OK) stop_gpu = 1;
        else cpu_err = uc_last_error();
    });
    uc_result *gpu_res = nullptr;
    const int gpu_rc = uc_solve(ps, &o, stream, &gpu_res);
    if (gpu_rc == UC_OK) stop_cpu = 1;
    cpu.join();
    std::unique_ptr<uc_result> g(gpu_res), c(cpu_res);
    if (gpu_rc == UC_OK && !(cpu_rc == UC_OK && cpu_res->stats.solve_ms < gpu_res->stats.solve_ms)) {
        if (winner) *winner = 0;
        *out = g.release();
        return UC_OK;
    }
    if (cpu_rc == UC_OK) {
        if (winner) *winner = 1;
        *out = c.release();
        return UC_OK;
    }
    if (gpu_res) {                          // neither optimal: the device result as it ended
        if (winner) *winner = 0;
        *out = g.release();
        return gpu_rc;
    }
    uc::set_error("uc_solve_concurrent: no arm returned a result (device %d; host: %s)", gpu_rc, cpu_err.c_str());
    return gpu_rc ? gpu_rc : cpu_rc;
}
