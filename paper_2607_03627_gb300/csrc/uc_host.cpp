// Host side of the unit-commitment LP solver: LP construction, presolve,
// diagonal scaling, the ||A||_2 estimate behind the PDHG step size, and
// postsolve.  None of this runs on the device; it feeds the device solve.
//
// Model (DC relaxation of the UC problem of Sec. II-A, "same relaxed problem"
// of Sec. II-C): per period t, columns [p (G), u (G), v (G), theta (B), f (L),
// shed (B)], equality rows (bus balance, line-flow definition) of all periods
// first, then ">=" rows (Pmax u - p, p - Pmin u, startup, ramp up, ramp down).
// Presolve is the reduced form of Sec. II-D's presolve that the device path
// needs; scaling is the PDLP preconditioner (Ruiz, then Pock-Chambolle).

#include <algorithm>
#include <atomic>
#include <cmath>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <limits>
#include <new>
#include <thread>

#include "uc_internal.h"

namespace uc {

static thread_local std::string g_err;

void set_error(const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

void clear_error() { g_err.clear(); }

Csr transpose(const Csr &A) {
    Csr T;
    T.rows = A.cols;
    T.cols = A.rows;
    T.rowptr.assign((size_t)A.cols + 1, 0);
    for (int32_t j : A.colidx) T.rowptr[(size_t)j + 1]++;
    for (int j = 0; j < A.cols; j++) T.rowptr[j + 1] += T.rowptr[j];
    T.colidx.resize(A.colidx.size());
    T.val.resize(A.val.size());
    std::vector<int32_t> next(T.rowptr.begin(), T.rowptr.end() - 1);
    for (int i = 0; i < A.rows; i++) {
        for (int32_t k = A.rowptr[i]; k < A.rowptr[i + 1]; k++) {
            int32_t j = A.colidx[k];
            int32_t dst = next[j]++;
            T.colidx[dst] = i;   // rows visited in order -> ascending
            T.val[dst] = A.val[k];
        }
    }
    return T;
}

// Runs fn(begin, end) over [0, n) in fixed-size chunks on `threads` workers.
template <class F>
static void parallel_for(int64_t n, int threads, F fn) {
    const int64_t chunk = 1 << 14;
    int64_t nchunks = (n + chunk - 1) / chunk;
    if (threads <= 1 || nchunks <= 1) {
        fn((int64_t)0, n);
        return;
    }
    std::atomic<int64_t> next{0};
    auto worker = [&]() {
        for (;;) {
            int64_t c = next.fetch_add(1);
            if (c >= nchunks) return;
            fn(c * chunk, std::min(n, (c + 1) * chunk));
        }
    };
    std::vector<std::thread> pool;
    int nt = (int)std::min<int64_t>(threads, nchunks);
    for (int t = 1; t < nt; t++) pool.emplace_back(worker);
    worker();
    for (auto &th : pool) th.join();
}

// Deterministic sum of squares: fixed 16384-element chunks, partials added in order.
static double sumsq(const std::vector<double> &v, int threads) {
    const int64_t chunk = 1 << 14;
    int64_t n = (int64_t)v.size();
    int64_t nch = (n + chunk - 1) / chunk;
    std::vector<double> part((size_t)std::max<int64_t>(nch, 1), 0.0);
    parallel_for(nch, threads, [&](int64_t b, int64_t e) {
        for (int64_t c = b; c < e; c++) {
            double s = 0.0;
            for (int64_t i = c * chunk; i < std::min(n, (c + 1) * chunk); i++) s += v[i] * v[i];
            part[c] = s;
        }
    });
    double s = 0.0;
    for (double p : part) s += p;
    return s;
}

// Worker threads kept for a loop of many parallel steps (the power
// iteration): run(n, fn) splits [0, n) into the same fixed 16384-element
// chunks as parallel_for and returns when every chunk is done, so results do
// not depend on the number of threads.
class Pool {
public:
    explicit Pool(int threads) {
        for (int t = 1; t < threads; t++) th_.emplace_back([this] { loop(); });
    }
    ~Pool() {
        {
            std::lock_guard<std::mutex> g(mu_);
            stop_ = true;
            gen_++;
        }
        cv_.notify_all();
        for (auto &t : th_) t.join();
    }
    void run(int64_t n, const std::function<void(int64_t, int64_t)> &fn) {
        const int64_t chunk = 1 << 14;
        const int64_t nch = (n + chunk - 1) / chunk;
        if (th_.empty() || nch <= 1) {   // the same chunks, in order, on this thread
            for (int64_t c = 0; c < nch; c++) fn(c * chunk, std::min(n, (c + 1) * chunk));
            return;
        }
        {
            std::lock_guard<std::mutex> g(mu_);
            fn_ = &fn;
            n_ = n;
            nch_ = nch;
            next_.store(0);
            busy_ = (int)th_.size();
            gen_++;
        }
        cv_.notify_all();
        work();
        std::unique_lock<std::mutex> g(mu_);
        done_.wait(g, [this] { return busy_ == 0; });
    }

private:
    void work() {
        const int64_t chunk = 1 << 14;
        for (;;) {
            const int64_t c = next_.fetch_add(1);
            if (c >= nch_) return;
            (*fn_)(c * chunk, std::min(n_, (c + 1) * chunk));
        }
    }
    void loop() {
        int seen = 0;
        for (;;) {
            {
                std::unique_lock<std::mutex> g(mu_);
                cv_.wait(g, [&] { return gen_ != seen; });
                seen = gen_;
                if (stop_) return;
            }
            work();
            {
                std::lock_guard<std::mutex> g(mu_);
                if (--busy_ == 0) done_.notify_one();
            }
        }
    }
    std::vector<std::thread> th_;
    std::mutex mu_;
    std::condition_variable cv_, done_;
    const std::function<void(int64_t, int64_t)> *fn_ = nullptr;
    int64_t n_ = 0, nch_ = 0;
    std::atomic<int64_t> next_{0};
    int busy_ = 0, gen_ = 0;
    bool stop_ = false;
};

static void spmv(const Csr &A, const std::vector<double> &x, std::vector<double> &y, int threads) {
    y.resize(A.rows);
    parallel_for(A.rows, threads, [&](int64_t b, int64_t e) {
        for (int64_t i = b; i < e; i++) {
            double s = 0.0;
            for (int32_t k = A.rowptr[i]; k < A.rowptr[i + 1]; k++) s += A.val[k] * x[A.colidx[k]];
            y[i] = s;
        }
    });
}

// ---------------------------------------------------------------------------
// LP construction
// ---------------------------------------------------------------------------
static int validate(const uc_problem *P) {
    if (!P) { set_error("uc_build_lp: null problem"); return UC_EINVAL; }
    if (P->B < 1 || P->L < 0 || P->G < 0 || P->T < 1) {
        set_error("uc_build_lp: need B >= 1, L >= 0, G >= 0, T >= 1 (got %d %d %d %d)", P->B, P->L, P->G, P->T);
        return UC_EINVAL;
    }
    if (P->ref_bus < 0 || P->ref_bus >= P->B) { set_error("uc_build_lp: ref_bus out of range"); return UC_EINVAL; }
    if ((P->L > 0 && (!P->line_from || !P->line_to || !P->x_pu || !P->fmax)) ||
        (P->G > 0 && (!P->gen_bus || !P->pmax || !P->pmin || !P->ramp || !P->c_lin || !P->c_nl ||
                      !P->c_su || !P->u0)) || !P->load) {
        set_error("uc_build_lp: null data array");
        return UC_EINVAL;
    }
    for (int l = 0; l < P->L; l++) {
        int a = P->line_from[l], b = P->line_to[l];
        if (a < 0 || a >= P->B || b < 0 || b >= P->B) { set_error("line %d: bus index out of range", l); return UC_EINVAL; }
        if (a == b) { set_error("line %d: self loop at bus %d", l, a); return UC_EINVAL; }
        if (!(P->x_pu[l] > 0.0) || !std::isfinite(P->x_pu[l])) { set_error("line %d: reactance must be > 0", l); return UC_EINVAL; }
        if (!(P->fmax[l] >= 0.0) || !std::isfinite(P->fmax[l])) { set_error("line %d: flow limit must be finite and >= 0", l); return UC_EINVAL; }
    }
    for (int g = 0; g < P->G; g++) {
        if (P->gen_bus[g] < 0 || P->gen_bus[g] >= P->B) { set_error("unit %d: bus index out of range", g); return UC_EINVAL; }
        double a = P->pmin[g], b = P->pmax[g];
        if (!(a >= 0.0) || !(b >= a) || !std::isfinite(b)) { set_error("unit %d: need 0 <= pmin <= pmax < inf", g); return UC_EINVAL; }
        if (!(P->ramp[g] >= 0.0) || !std::isfinite(P->ramp[g])) { set_error("unit %d: ramp must be finite and >= 0", g); return UC_EINVAL; }
        if (!std::isfinite(P->c_lin[g]) || !std::isfinite(P->c_nl[g]) || !std::isfinite(P->c_su[g]) ||
            !std::isfinite(P->u0[g])) { set_error("unit %d: non-finite cost or u0", g); return UC_EINVAL; }
    }
    int64_t TB = (int64_t)P->T * P->B;
    for (int64_t k = 0; k < TB; k++)
        if (!(P->load[k] >= 0.0) || !std::isfinite(P->load[k])) { set_error("load[%lld] must be finite and >= 0", (long long)k); return UC_EINVAL; }
    if (!std::isfinite(P->voll)) { set_error("voll must be finite"); return UC_EINVAL; }
    int64_t nc = 3LL * P->G + P->B + P->L + (P->voll > 0 ? P->B : 0);
    if (nc * P->T >= (1LL << 31) - 1) { set_error("problem too large for int32 indices"); return UC_EINVAL; }
    return UC_OK;
}

static int build(const uc_problem *P, RawLp &lp) {
    const int B = P->B, L = P->L, G = P->G, T = P->T;
    const bool hs = P->voll > 0.0;
    const int nc = 3 * G + B + L + (hs ? B : 0);
    const int64_t n = (int64_t)T * nc;
    lp.B = B; lp.L = L; lp.G = G; lp.T = T; lp.nc = nc; lp.has_shed = hs;
    lp.c.assign(n, 0.0); lp.l.assign(n, 0.0); lp.u.assign(n, 0.0);
    lp.col_kind.assign(n, 0); lp.col_t.assign(n, 0); lp.col_idx.assign(n, 0);
    const double inf = std::numeric_limits<double>::infinity();
    auto P_ = [&](int t, int g) { return t * nc + g; };
    auto U_ = [&](int t, int g) { return t * nc + G + g; };
    auto V_ = [&](int t, int g) { return t * nc + 2 * G + g; };
    auto TH = [&](int t, int b) { return t * nc + 3 * G + b; };
    auto F_ = [&](int t, int l) { return t * nc + 3 * G + B + l; };
    auto S_ = [&](int t, int b) { return t * nc + 3 * G + B + L + b; };
    for (int t = 0; t < T; t++) {
        for (int g = 0; g < G; g++) {
            int j = P_(t, g); lp.c[j] = P->c_lin[g]; lp.l[j] = 0; lp.u[j] = P->pmax[g];
            lp.col_kind[j] = COL_P; lp.col_t[j] = t; lp.col_idx[j] = g;
            j = U_(t, g); lp.c[j] = P->c_nl[g]; lp.l[j] = 0; lp.u[j] = 1;
            lp.col_kind[j] = COL_U; lp.col_t[j] = t; lp.col_idx[j] = g;
            j = V_(t, g); lp.c[j] = P->c_su[g]; lp.l[j] = 0; lp.u[j] = 1;
            lp.col_kind[j] = COL_V; lp.col_t[j] = t; lp.col_idx[j] = g;
        }
        for (int b = 0; b < B; b++) {
            int j = TH(t, b);
            if (b == P->ref_bus) { lp.l[j] = 0; lp.u[j] = 0; }
            else { lp.l[j] = -inf; lp.u[j] = inf; }
            lp.col_kind[j] = COL_TH; lp.col_t[j] = t; lp.col_idx[j] = b;
        }
        for (int l = 0; l < L; l++) {
            int j = F_(t, l); lp.l[j] = -P->fmax[l]; lp.u[j] = P->fmax[l];
            lp.col_kind[j] = COL_F; lp.col_t[j] = t; lp.col_idx[j] = l;
        }
        if (hs) for (int b = 0; b < B; b++) {
            int j = S_(t, b); lp.c[j] = P->voll; lp.l[j] = 0; lp.u[j] = P->load[(int64_t)t * B + b];
            lp.col_kind[j] = COL_S; lp.col_t[j] = t; lp.col_idx[j] = b;
        }
    }
    // adjacency: units and lines per bus, in index order
    std::vector<std::vector<int>> gens(B);
    std::vector<std::vector<std::pair<int, double>>> lines(B);
    for (int g = 0; g < G; g++) gens[P->gen_bus[g]].push_back(g);
    for (int l = 0; l < L; l++) {
        lines[P->line_from[l]].push_back({l, -1.0});
        lines[P->line_to[l]].push_back({l, 1.0});
    }
    for (auto &v : lines) std::sort(v.begin(), v.end());

    Csr &A = lp.A;
    A.cols = (int)n;
    A.rowptr.push_back(0);
    std::vector<std::pair<int32_t, double>> row;
    auto emit = [&](double rhs, int8_t kind, int t, int idx) {
        std::sort(row.begin(), row.end());
        for (auto &e : row)
            if (e.second != 0.0) { A.colidx.push_back(e.first); A.val.push_back(e.second); }
        A.rowptr.push_back((int32_t)A.colidx.size());
        lp.q.push_back(rhs); lp.row_kind.push_back(kind); lp.row_t.push_back(t); lp.row_idx.push_back(idx);
        row.clear();
    };
    for (int t = 0; t < T; t++) {
        for (int b = 0; b < B; b++) {
            for (int g : gens[b]) row.push_back({P_(t, g), 1.0});
            for (auto &e : lines[b]) row.push_back({F_(t, e.first), e.second});
            if (hs) row.push_back({S_(t, b), 1.0});
            emit(P->load[(int64_t)t * B + b], ROW_BAL, t, b);
        }
        for (int l = 0; l < L; l++) {
            double ix = 1.0 / P->x_pu[l];
            row.push_back({F_(t, l), 1.0});
            row.push_back({TH(t, P->line_from[l]), -ix});
            row.push_back({TH(t, P->line_to[l]), ix});
            emit(0.0, ROW_FLOW, t, l);
        }
    }
    lp.m_eq = (int)lp.q.size();
    for (int t = 0; t < T; t++) {
        for (int g = 0; g < G; g++) {
            row.push_back({P_(t, g), -1.0}); row.push_back({U_(t, g), P->pmax[g]});
            emit(0.0, ROW_GUP, t, g);
        }
        for (int g = 0; g < G; g++) {
            row.push_back({P_(t, g), 1.0}); row.push_back({U_(t, g), -P->pmin[g]});
            emit(0.0, ROW_GLO, t, g);
        }
        for (int g = 0; g < G; g++) {
            row.push_back({U_(t, g), -1.0}); row.push_back({V_(t, g), 1.0});
            if (t == 0) emit(-P->u0[g], ROW_SU, t, g);
            else { row.push_back({U_(t - 1, g), 1.0}); emit(0.0, ROW_SU, t, g); }
        }
        if (t >= 1) {
            for (int g = 0; g < G; g++) {
                row.push_back({P_(t - 1, g), 1.0}); row.push_back({P_(t, g), -1.0});
                emit(-P->ramp[g], ROW_RUP, t, g);
            }
            for (int g = 0; g < G; g++) {
                row.push_back({P_(t - 1, g), -1.0}); row.push_back({P_(t, g), 1.0});
                emit(-P->ramp[g], ROW_RDN, t, g);
            }
        }
    }
    A.rows = (int)lp.q.size();
    return UC_OK;
}

// ---------------------------------------------------------------------------
// Angle elimination (presolve option eliminate_angles).  Per period the flow
// rows f_l - inv_l (theta_a - theta_b) = 0 (a = from bus, b = to bus, inv_l =
// 1/x_l as stored) define a graph on the angle columns.  A breadth-first
// spanning tree is grown from the reference bus (the angle fixed at 0),
// visiting each bus's lines in row order.  A tree line's row gives
// theta_child - theta_parent = s f_e / inv_e (s = +1 when the child is the
// line's from end), so an angle difference is a sum of tree flows along the
// tree path.  The tree lines' rows and the angle columns leave the LP; the
// row of every other line becomes
//   f_l - inv_l (sum over a's path up of s f_e / inv_e - the same for b) = 0,
// the paths cut at their common part (its fundamental cycle).
// ---------------------------------------------------------------------------
int eliminate_angles(const RawLp &raw, RawLp &out, AngleElim &E) {
    const Csr &A = raw.A;
    const int n = A.cols, m = A.rows;
    std::vector<int> periods;
    for (int j = 0; j < n; j++)
        if (raw.col_kind[j] == COL_TH) periods.push_back(raw.col_t[j]);
    std::sort(periods.begin(), periods.end());
    periods.erase(std::unique(periods.begin(), periods.end()), periods.end());
    std::vector<std::vector<int>> th_of(periods.size()), rows_of(periods.size());
    auto pidx = [&](int t) { return (int)(std::lower_bound(periods.begin(), periods.end(), t) - periods.begin()); };
    for (int j = 0; j < n; j++)
        if (raw.col_kind[j] == COL_TH) th_of[pidx(raw.col_t[j])].push_back(j);
    for (int i = 0; i < m; i++)
        if (raw.row_kind[i] == ROW_FLOW) {
            const auto it = std::lower_bound(periods.begin(), periods.end(), raw.row_t[i]);
            if (it == periods.end() || *it != raw.row_t[i]) { set_error("eliminate_angles: flow row %d has no angles", i); return UC_EINVAL; }
            rows_of[it - periods.begin()].push_back(i);
        }
    struct Edge { int row, fc, a, b; double inv; };
    std::vector<char> drop(m, 0);
    std::vector<std::vector<std::pair<int, double>>> new_row(m);   // substituted rows (raw columns)
    std::vector<char> has_new(m, 0);
    E.roots.clear();
    E.tree.clear();
    size_t n_angles = 0;
    for (const auto &nodes : th_of) n_angles += nodes.size();
    E.tree.reserve(n_angles);
    E.tree_row.assign(n, -1);
    std::vector<int> local(n, -1);
    for (size_t p = 0; p < periods.size(); p++) {
        const std::vector<int> &nodes = th_of[p];
        int root = -1, nroot = 0;
        for (int j : nodes)
            if (raw.l[j] == 0.0 && raw.u[j] == 0.0) { root = j; nroot++; }
        if (nroot != 1) { set_error("eliminate_angles: period %d has %d angles fixed at 0, not one", periods[p], nroot); return UC_EINVAL; }
        for (size_t k = 0; k < nodes.size(); k++) local[nodes[k]] = (int)k;
        std::vector<Edge> edges;
        for (int i : rows_of[p]) {
            Edge e{i, -1, -1, -1, 0.0};
            for (int32_t k = A.rowptr[i]; k < A.rowptr[i + 1]; k++) {
                const int j = A.colidx[k];
                const double v = A.val[k];
                if (raw.col_kind[j] == COL_F) e.fc = j;
                else if (v < 0) e.a = j;
                else { e.b = j; e.inv = v; }
            }
            if (e.fc < 0 || e.a < 0 || e.b < 0 || local[e.a] < 0 || local[e.b] < 0) {
                set_error("eliminate_angles: flow row %d is not f - (theta_a - theta_b) / x", i);
                return UC_EINVAL;
            }
            edges.push_back(e);
        }
        const int nn = (int)nodes.size();
        std::vector<std::vector<std::pair<int, int>>> adj(nn);   // (local node, edge)
        for (int e = 0; e < (int)edges.size(); e++) {
            adj[local[edges[e].a]].push_back({local[edges[e].b], e});
            adj[local[edges[e].b]].push_back({local[edges[e].a], e});
        }
        std::vector<int> par(nn, -2), pedge(nn, -1), order;
        order.reserve(nn);
        par[local[root]] = -1;
        order.push_back(local[root]);
        for (size_t h = 0; h < order.size(); h++) {
            const int v = order[h];
            for (auto &we : adj[v])
                if (par[we.first] == -2) { par[we.first] = v; pedge[we.first] = we.second; order.push_back(we.first); }
        }
        if ((int)order.size() != nn) { set_error("eliminate_angles: the grid of period %d is not connected", periods[p]); return UC_EINVAL; }
        std::vector<char> in_tree(edges.size(), 0);
        for (int k = 1; k < nn; k++) in_tree[pedge[order[k]]] = 1;
        auto up = [&](int v, std::vector<std::pair<int, double>> &path) {   // (edge, s) from v to the root
            path.clear();
            while (par[v] >= 0) {
                const int e = pedge[v];
                path.push_back({e, local[edges[e].a] == v ? 1.0 : -1.0});
                v = par[v];
            }
        };
        std::vector<std::pair<int, double>> pa, pb;
        for (int e = 0; e < (int)edges.size(); e++) {
            const Edge &L = edges[e];
            if (in_tree[e]) { drop[L.row] = 1; E.tree_row[L.fc] = L.row; continue; }
            up(local[L.a], pa);
            up(local[L.b], pb);
            while (!pa.empty() && !pb.empty() && pa.back() == pb.back()) { pa.pop_back(); pb.pop_back(); }
            auto &row = new_row[L.row];
            row.reserve(1 + pa.size() + pb.size());
            row.push_back({L.fc, 1.0});
            for (auto &gs : pa) row.push_back({edges[gs.first].fc, -gs.second * L.inv / edges[gs.first].inv});
            for (auto &gs : pb) row.push_back({edges[gs.first].fc, gs.second * L.inv / edges[gs.first].inv});
            has_new[L.row] = 1;
        }
        E.roots.push_back(root);
        for (int k = 1; k < nn; k++) {
            const int w = order[k];
            const Edge &L = edges[pedge[w]];
            E.tree.push_back({nodes[w], nodes[par[w]], L.fc, local[L.a] == w ? 1.0 : -1.0, L.inv});
        }
        for (int j : nodes) local[j] = -1;
    }
    std::vector<int32_t> newcol(n, -1);
    E.col_keep.clear();
    for (int j = 0; j < n; j++)
        if (raw.col_kind[j] != COL_TH) { newcol[j] = (int32_t)E.col_keep.size(); E.col_keep.push_back(j); }
    E.row_keep.clear();
    for (int i = 0; i < m; i++)
        if (!drop[i]) E.row_keep.push_back(i);
    out = RawLp{};
    out.B = raw.B; out.L = raw.L; out.G = raw.G; out.T = raw.T; out.nc = raw.nc; out.has_shed = raw.has_shed;
    const int nk = (int)E.col_keep.size(), mk = (int)E.row_keep.size();
    out.A.rows = mk;
    out.A.cols = nk;
    int64_t nnz_new = 0;
    for (int i = 0; i < m; i++) nnz_new += has_new[i] ? (int64_t)new_row[i].size() : 0;
    out.A.rowptr.reserve((size_t)mk + 1);
    out.A.rowptr.assign(1, 0);
    out.A.colidx.reserve((size_t)(A.nnz() + nnz_new));
    out.A.val.reserve((size_t)(A.nnz() + nnz_new));
    for (auto *v : {&out.q}) v->reserve(mk);
    out.row_kind.reserve(mk); out.row_t.reserve(mk); out.row_idx.reserve(mk);
    out.c.reserve(nk); out.l.reserve(nk); out.u.reserve(nk);
    out.col_kind.reserve(nk); out.col_t.reserve(nk); out.col_idx.reserve(nk);
    std::vector<std::pair<int, double>> ents;
    for (int r = 0; r < mk; r++) {
        const int i = E.row_keep[r];
        ents.clear();
        if (has_new[i]) {
            for (auto &jv : new_row[i]) ents.push_back({newcol[jv.first], jv.second});
        } else {
            for (int32_t k = A.rowptr[i]; k < A.rowptr[i + 1]; k++) {
                if (newcol[A.colidx[k]] < 0) { set_error("eliminate_angles: row %d has an angle entry but is no flow row", i); return UC_EINVAL; }
                ents.push_back({newcol[A.colidx[k]], A.val[k]});
            }
        }
        std::sort(ents.begin(), ents.end(), [](const std::pair<int, double> &x, const std::pair<int, double> &y) { return x.first < y.first; });
        for (auto &jv : ents) { out.A.colidx.push_back(jv.first); out.A.val.push_back(jv.second); }
        out.A.rowptr.push_back((int32_t)out.A.colidx.size());
    }
    out.m_eq = 0;
    for (int i : E.row_keep) out.m_eq += i < raw.m_eq ? 1 : 0;
    for (int i : E.row_keep) {
        out.q.push_back(raw.q[i]); out.row_kind.push_back(raw.row_kind[i]);
        out.row_t.push_back(raw.row_t[i]); out.row_idx.push_back(raw.row_idx[i]);
    }
    for (int j : E.col_keep) {
        out.c.push_back(raw.c[j]); out.l.push_back(raw.l[j]); out.u.push_back(raw.u[j]);
        out.col_kind.push_back(raw.col_kind[j]); out.col_t.push_back(raw.col_t[j]); out.col_idx.push_back(raw.col_idx[j]);
    }
    return UC_OK;
}

// A point of the angle-free LP on the LP as built: the angles from the
// reference value down the tree, theta_child = theta_parent + s f_e / inv_e;
// a tree line's flow row takes the dual that keeps its flow column's reduced
// cost, sum over the substituted rows r holding f_e of (coefficient) y_r.
static void restore_angles(const AngleElim &E, const RawLp &orig, const RawLp &work, std::vector<double> &x,
                           std::vector<double> &y, bool duals) {
    std::vector<double> xo(orig.A.cols, 0.0);
    for (size_t k = 0; k < E.col_keep.size(); k++) xo[E.col_keep[k]] = x[k];
    for (int r : E.roots) xo[r] = orig.l[r];
    for (const auto &nd : E.tree) xo[nd.col] = xo[nd.parent] + nd.s * xo[nd.fcol] / nd.inv;
    x.swap(xo);
    std::vector<double> yo(orig.A.rows, 0.0);
    if (duals) {
        for (size_t k = 0; k < E.row_keep.size(); k++) yo[E.row_keep[k]] = y[k];
        const Csr &W = work.A;
        for (int r = 0; r < W.rows; r++) {
            if (work.row_kind[r] != ROW_FLOW) continue;
            for (int32_t k = W.rowptr[r]; k < W.rowptr[r + 1]; k++) {
                const int tr = E.tree_row[E.col_keep[W.colidx[k]]];
                if (tr >= 0) yo[tr] += W.val[k] * y[r];
            }
        }
    }
    y.swap(yo);
}

// ---------------------------------------------------------------------------
// Presolve
// ---------------------------------------------------------------------------
static int presolve_reduce(const RawLp &raw, PsData &ps, Csr &Ared, std::vector<double> &qr,
                           std::vector<double> &cr, std::vector<double> &lr, std::vector<double> &ur,
                           bool aggressive) {
    const Csr &A = raw.A;
    const int n = A.cols, m = A.rows;
    Csr AT = transpose(A);
    std::vector<double> l = raw.l, u = raw.u, q = raw.q, c = raw.c;
    ps.aggressive = aggressive;
    std::vector<char> col_on(n, 1), row_on(m, 1);
    ps.xfix.assign(n, 0.0);
    double obj_const = 0.0;
    const double tol = 1e-9;
    for (bool changed = true; changed;) {
        changed = false;
        for (int j = 0; j < n; j++) {                        // fixed columns
            if (!col_on[j] || l[j] != u[j]) continue;
            double v = l[j];
            for (int32_t k = AT.rowptr[j]; k < AT.rowptr[j + 1]; k++)
                if (row_on[AT.colidx[k]]) q[AT.colidx[k]] -= AT.val[k] * v;
            obj_const += c[j] * v;
            ps.xfix[j] = v;
            col_on[j] = 0;
            changed = true;
        }
        for (int i = 0; i < m; i++) {                        // empty / singleton rows
            if (!row_on[i]) continue;
            int cnt = 0, jj = -1;
            double aa = 0.0;
            for (int32_t k = A.rowptr[i]; k < A.rowptr[i + 1]; k++)
                if (col_on[A.colidx[k]]) { cnt++; jj = A.colidx[k]; aa = A.val[k]; }
            bool eq = i < raw.m_eq;
            if (cnt == 0) {
                if ((eq && std::fabs(q[i]) > tol) || (!eq && q[i] > tol)) {
                    set_error("presolve: row %d has no columns but rhs %g", i, q[i]);
                    return UC_EINFEASIBLE;
                }
                row_on[i] = 0;
                ps.removed.push_back({i, -1, 0.0, eq, false});
                changed = true;
            } else if (cnt == 1) {
                double bnd = q[i] / aa;
                bool tight = false;
                if (eq) {
                    if (bnd < l[jj] - tol || bnd > u[jj] + tol) {
                        set_error("presolve: singleton equality row %d outside the bounds of column %d", i, jj);
                        return UC_EINFEASIBLE;
                    }
                    l[jj] = bnd; u[jj] = bnd; tight = true;
                } else if (aa > 0) {
                    if (bnd > l[jj]) { l[jj] = bnd; tight = true; }
                } else {
                    if (bnd < u[jj]) { u[jj] = bnd; tight = true; }
                }
                if (l[jj] > u[jj] + tol) { set_error("presolve: bounds of column %d cross", jj); return UC_EINFEASIBLE; }
                if (l[jj] > u[jj]) u[jj] = l[jj];
                row_on[i] = 0;
                ps.removed.push_back({i, jj, aa, eq, tight});
                changed = true;
            }
        }
        // doubleton equations a_f x_f + a_s x_s = q whose x_s has no other entry
        // in an active row (aggressive presolve): solve for x_s, move its bounds
        // onto x_f and its cost into x_f's, drop the row and x_s
        auto active_entries = [&](int j) {
            int cnt = 0;
            for (int32_t k = AT.rowptr[j]; k < AT.rowptr[j + 1]; k++) cnt += row_on[AT.colidx[k]];
            return cnt;
        };
        for (int i = 0; aggressive && i < raw.m_eq; i++) {
            if (!row_on[i]) continue;
            int cnt = 0, j1 = -1, j2 = -1;
            double a1 = 0.0, a2 = 0.0;
            for (int32_t k = A.rowptr[i]; k < A.rowptr[i + 1]; k++) {
                if (!col_on[A.colidx[k]]) continue;
                if (cnt == 0) { j1 = A.colidx[k]; a1 = A.val[k]; }
                else { j2 = A.colidx[k]; a2 = A.val[k]; }
                cnt++;
            }
            if (cnt != 2) continue;
            const bool s1 = active_entries(j1) == 1, s2 = active_entries(j2) == 1;
            if (!s1 && !s2) continue;
            const int js = (s1 && s2) ? std::max(j1, j2) : (s1 ? j1 : j2);
            const int jf = js == j1 ? j2 : j1;
            const double as = js == j1 ? a1 : a2, af = js == j1 ? a2 : a1;
            const double v1 = (q[i] - as * l[js]) / af, v2 = (q[i] - as * u[js]) / af;
            const double lo = std::min(v1, v2), hi = std::max(v1, v2);
            const bool lo_from = lo > l[jf], hi_from = hi < u[jf];
            if (lo_from) l[jf] = lo;
            if (hi_from) u[jf] = hi;
            if (l[jf] > u[jf] + tol) { set_error("presolve: doubleton row %d crosses the bounds of column %d", i, jf); return UC_EINFEASIBLE; }
            if (l[jf] > u[jf]) u[jf] = l[jf];
            c[jf] = c[jf] - c[js] * af / as;
            obj_const += c[js] * q[i] / as;
            row_on[i] = 0;
            col_on[js] = 0;
            RemovedRow r{i, js, as, true, false};
            r.doubleton = true;
            r.f = jf;
            r.a_f = af;
            r.q = q[i];
            r.lo_from_s = lo_from;
            r.hi_from_s = hi_from;
            ps.removed.push_back(r);
            changed = true;
        }
        for (int j = 0; j < n; j++) {                        // empty columns
            if (!col_on[j]) continue;
            bool used = false;
            for (int32_t k = AT.rowptr[j]; k < AT.rowptr[j + 1] && !used; k++) used = row_on[AT.colidx[k]];
            if (used) continue;
            double cj = c[j], v;
            if (cj > 0) v = l[j];
            else if (cj < 0) v = u[j];
            else v = std::isfinite(l[j]) ? l[j] : (std::isfinite(u[j]) ? u[j] : 0.0);
            if (!std::isfinite(v)) { set_error("presolve: column %d is unbounded", j); return UC_EUNBOUNDED; }
            obj_const += cj * v;
            ps.xfix[j] = v;
            col_on[j] = 0;
            changed = true;
        }
    }
    std::vector<int32_t> newcol(n, -1);
    ps.col_map.reserve(n);
    ps.row_map.reserve(m);
    for (int j = 0; j < n; j++)
        if (col_on[j]) { newcol[j] = (int32_t)ps.col_map.size(); ps.col_map.push_back(j); }
    for (int i = 0; i < m; i++)
        if (row_on[i]) ps.row_map.push_back(i);
    Ared.rows = (int)ps.row_map.size();
    Ared.cols = (int)ps.col_map.size();
    Ared.rowptr.reserve(ps.row_map.size() + 1);
    Ared.rowptr.assign(1, 0);
    Ared.colidx.reserve(A.colidx.size());
    Ared.val.reserve(A.val.size());
    qr.reserve(ps.row_map.size());
    cr.reserve(ps.col_map.size()); lr.reserve(ps.col_map.size()); ur.reserve(ps.col_map.size());
    for (int32_t i : ps.row_map) {
        for (int32_t k = A.rowptr[i]; k < A.rowptr[i + 1]; k++)
            if (col_on[A.colidx[k]]) { Ared.colidx.push_back(newcol[A.colidx[k]]); Ared.val.push_back(A.val[k]); }
        Ared.rowptr.push_back((int32_t)Ared.colidx.size());
        qr.push_back(q[i]);
    }
    ps.m_eq = 0;
    for (int32_t i : ps.row_map) ps.m_eq += (i < raw.m_eq);
    for (int32_t j : ps.col_map) { cr.push_back(c[j]); lr.push_back(l[j]); ur.push_back(u[j]); }
    ps.l_tight = l;
    ps.u_tight = u;
    ps.obj_const = obj_const;
    return UC_OK;
}

// one equilibration pass: divide rows by rf, columns by cf
static void apply_scaling(Csr &A, const std::vector<double> &rf, const std::vector<double> &cf,
                          std::vector<double> &Dr, std::vector<double> &Dc, int threads) {
    parallel_for(A.rows, threads, [&](int64_t b, int64_t e) {
        for (int64_t i = b; i < e; i++)
            for (int32_t k = A.rowptr[i]; k < A.rowptr[i + 1]; k++)
                A.val[k] = A.val[k] / rf[i] / cf[A.colidx[k]];
    });
    for (int i = 0; i < A.rows; i++) Dr[i] /= rf[i];
    for (int j = 0; j < A.cols; j++) Dc[j] /= cf[j];
}

static void scale_lp(PsData &ps, const uc_presolve_opts &o, int threads) {
    Csr &A = ps.A;
    const int m = A.rows, n = A.cols;
    ps.Dr.assign(m, 1.0);
    ps.Dc.assign(n, 1.0);
    std::vector<double> rf(m), cf(n);
    // column view of A: the positions in A.val of column j's entries, rows
    // ascending (the order in which a row-by-row sweep meets them), so the
    // column sums below add in the same order as such a sweep
    std::vector<int32_t> cp((size_t)n + 1, 0), pos(A.colidx.size());
    for (int32_t j : A.colidx) cp[(size_t)j + 1]++;
    for (int j = 0; j < n; j++) cp[j + 1] += cp[j];
    {
        std::vector<int32_t> next(cp.begin(), cp.end() - 1);
        for (int i = 0; i < m; i++)
            for (int32_t k = A.rowptr[i]; k < A.rowptr[i + 1]; k++) pos[next[A.colidx[k]]++] = k;
    }
    // factor = sqrt(max |a|) (Ruiz) or sqrt(sum |a|) (Pock-Chambolle, alpha = 1)
    // of every row and column; 1 for an empty one
    auto factors = [&](bool sum) {
        parallel_for(m, threads, [&](int64_t b, int64_t e) {
            for (int64_t i = b; i < e; i++) {
                double r = 0.0;
                for (int32_t k = A.rowptr[i]; k < A.rowptr[i + 1]; k++) {
                    const double a = std::fabs(A.val[k]);
                    r = sum ? r + a : std::max(r, a);
                }
                rf[i] = r > 0 ? std::sqrt(r) : 1.0;
            }
        });
        parallel_for(n, threads, [&](int64_t b, int64_t e) {
            for (int64_t j = b; j < e; j++) {
                double r = 0.0;
                for (int32_t p = cp[j]; p < cp[j + 1]; p++) {
                    const double a = std::fabs(A.val[pos[p]]);
                    r = sum ? r + a : std::max(r, a);
                }
                cf[j] = r > 0 ? std::sqrt(r) : 1.0;
            }
        });
    };
    for (int it = 0; it < o.ruiz_iters; it++) {           // Ruiz: sqrt of row / column max
        factors(false);
        apply_scaling(A, rf, cf, ps.Dr, ps.Dc, threads);
    }
    if (o.pock_chambolle) {                                // Pock-Chambolle, alpha = 1
        factors(true);
        apply_scaling(A, rf, cf, ps.Dr, ps.Dc, threads);
    }
    for (int i = 0; i < m; i++) ps.q[i] *= ps.Dr[i];
    for (int j = 0; j < n; j++) {
        ps.c[j] *= ps.Dc[j];
        ps.l[j] /= ps.Dc[j];
        ps.u[j] /= ps.Dc[j];
    }
}

// Certified upper bound on ||A_s||_2.  After a Pock-Chambolle pass with
// alpha = 1 (row i divided by sqrt(r_i), column j by sqrt(c_j), the absolute
// row and column sums before the pass), the Schur test with weights sqrt(r_i)
// and sqrt(c_j) gives ||A_s||_2 <= 1.  Without that pass: the Schur test with
// unit weights, sqrt(max row absolute sum * max column absolute sum).
static double norm_upper_bound(const Csr &A, bool pock_chambolle) {
    if (pock_chambolle) return 1.0;
    std::vector<double> cs((size_t)A.cols, 0.0);
    double rmax = 0.0;
    for (int i = 0; i < A.rows; i++) {
        double r = 0.0;
        for (int32_t k = A.rowptr[i]; k < A.rowptr[i + 1]; k++) {
            r += std::fabs(A.val[k]);
            cs[A.colidx[k]] += std::fabs(A.val[k]);
        }
        rmax = std::max(rmax, r);
    }
    double cmax = 0.0;
    for (double v : cs) cmax = std::max(cmax, v);
    return std::sqrt(rmax * cmax);
}

// ||A||_2 by power iteration on A^T A from the unit vector 1/sqrt(n).  Every
// step runs on one pool of workers; the sum of squares adds fixed 16384-element
// chunk partials in order, so the result does not depend on the thread count.
static double power_norm(const Csr &A, const Csr &AT, int max_iter, double tol, int threads) {
    const int n = A.cols, m = A.rows;
    if (n == 0 || m == 0) return 0.0;
    std::vector<double> v(n, 1.0 / std::sqrt((double)n)), t(m), w(n);
    const int64_t chunk = 1 << 14;
    const int64_t nch = ((int64_t)n + chunk - 1) / chunk;
    std::vector<double> part((size_t)nch, 0.0);
    Pool pool(threads);
    auto mul = [](const Csr &M, const std::vector<double> &x, std::vector<double> &y) {
        return [&M, &x, &y](int64_t b, int64_t e) {
            for (int64_t i = b; i < e; i++) {
                double s = 0.0;
                for (int32_t k = M.rowptr[i]; k < M.rowptr[i + 1]; k++) s += M.val[k] * x[M.colidx[k]];
                y[i] = s;
            }
        };
    };
    const std::function<void(int64_t, int64_t)> fa = mul(A, v, t), fat = mul(AT, t, w);
    double lam = 0.0, prev = 0.0;
    const std::function<void(int64_t, int64_t)> fsq = [&](int64_t b, int64_t e) {
        double s = 0.0;
        for (int64_t i = b; i < e; i++) s += w[i] * w[i];
        part[b / chunk] = s;
    };
    const std::function<void(int64_t, int64_t)> fdiv = [&](int64_t b, int64_t e) {
        for (int64_t j = b; j < e; j++) v[j] = w[j] / lam;
    };
    for (int it = 0; it < max_iter; it++) {
        pool.run(m, fa);
        pool.run(n, fat);
        pool.run(n, fsq);
        double s = 0.0;
        for (double p : part) s += p;
        lam = std::sqrt(s);
        if (lam == 0.0) return 0.0;
        pool.run(n, fdiv);
        if (std::fabs(lam - prev) <= tol * lam) break;
        prev = lam;
    }
    return std::sqrt(lam);
}

// Relative KKT parts, the largest absolute row violation and the objectives of
// a scaled presolved point (natural order) on the unscaled presolved LP, as
// the device evaluation defines them (host loops, fixed order).
void host_kkt(const PsData &p, const double *xs, const double *ys, double &rel_p, double &rel_d,
                     double &rel_g, double &abs_p, double &pobj, double &dobj) {
    double rpu = 0.0, rdu = 0.0, qy = 0.0, cx = 0.0, bnd = 0.0;
    for (int i = 0; i < p.m(); i++) {
        double ax = 0.0;
        for (int32_t e = p.A.rowptr[i]; e < p.A.rowptr[i + 1]; e++) ax += p.A.val[e] * xs[p.A.colidx[e]];
        double r = ax - p.q[i];
        if (i >= p.m_eq && r > 0.0) r = 0.0;
        rpu = std::max(rpu, std::fabs(r) / p.Dr[i]);
        qy += p.q[i] * ys[i];
    }
    for (int j = 0; j < p.n(); j++) {
        double t = 0.0;
        for (int32_t e = p.AT.rowptr[j]; e < p.AT.rowptr[j + 1]; e++) t += p.AT.val[e] * ys[p.AT.colidx[e]];
        const double lm = p.c[j] - t;
        const bool lf = std::isfinite(p.l[j]), uf = std::isfinite(p.u[j]);
        const double lp = (lf && uf) ? lm : lf ? std::max(lm, 0.0) : uf ? std::min(lm, 0.0) : 0.0;
        rdu = std::max(rdu, std::fabs(lm - lp) / p.Dc[j]);
        cx += p.c[j] * xs[j];
        if (lf) bnd += p.l[j] * std::max(lp, 0.0);
        if (uf) bnd += p.u[j] * std::min(lp, 0.0);
    }
    pobj = cx;
    dobj = qy + bnd;
    rel_p = rpu / (1.0 + p.q_inf);
    rel_d = rdu / (1.0 + p.c_inf);
    rel_g = std::fabs(pobj - dobj) / (1.0 + std::fabs(pobj) + std::fabs(dobj));
    abs_p = rpu;
}

static void postsolve_reduced(const PsData &ps, const double *xs, const double *ys, std::vector<double> &x,
                              std::vector<double> &y);

void postsolve(const PsData &ps, const double *xs, const double *ys, std::vector<double> &x,
               std::vector<double> &y) {
    postsolve_reduced(ps, xs, ys, x, y);
    if (ps.angles) restore_angles(*ps.angles, *ps.orig, *ps.raw, x, y, ys != nullptr);
}

// to the LP the reductions started from
static void postsolve_reduced(const PsData &ps, const double *xs, const double *ys, std::vector<double> &x,
                              std::vector<double> &y) {
    const RawLp &raw = *ps.raw;
    x = ps.xfix;
    for (size_t k = 0; k < ps.col_map.size(); k++) x[ps.col_map[k]] = ps.Dc[k] * xs[k];
    for (auto it = ps.removed.rbegin(); it != ps.removed.rend(); ++it)   // substituted columns
        if (it->doubleton) x[it->col] = (it->q - it->a_f * x[it->f]) / it->a;
    y.assign(raw.A.rows, 0.0);
    if (!ys) return;
    for (size_t k = 0; k < ps.row_map.size(); k++) y[ps.row_map[k]] = ps.Dr[k] * ys[k];
    bool any = false;
    for (auto &r : ps.removed) any |= (r.col >= 0 && (r.tightened || r.doubleton));
    if (!any) return;
    Csr AT = transpose(raw.A);
    auto redcost = [&](int j) {
        double s = raw.c[j];
        for (int32_t k = AT.rowptr[j]; k < AT.rowptr[j + 1]; k++) s -= AT.val[k] * y[AT.colidx[k]];
        return s;
    };
    for (auto it = ps.removed.rbegin(); it != ps.removed.rend(); ++it) {
        if (it->doubleton) {
            // x_f at a bound that came from x_s's bounds: the row's dual zeroes
            // x_f's reduced cost (x_s then sits at its bound); otherwise x_s's
            const int f = it->f;
            const double tf = 1e-9 * (1.0 + std::fabs(x[f]));
            const bool on = (it->lo_from_s && std::fabs(x[f] - ps.l_tight[f]) <= tf) ||
                            (it->hi_from_s && std::fabs(x[f] - ps.u_tight[f]) <= tf);
            const double yi = y[it->row];
            y[it->row] = on ? (redcost(f) + it->a_f * yi) / it->a_f : (redcost(it->col) + it->a * yi) / it->a;
            continue;
        }
        if (it->col < 0 || !it->tightened) continue;
        int j = it->col;
        double lam = redcost(j);
        if (it->eq) {
            y[it->row] = lam / it->a;
        } else {
            double bnd = it->a > 0 ? ps.l_tight[j] : ps.u_tight[j];
            bool at = std::fabs(x[j] - bnd) <= 1e-9 * (1.0 + std::fabs(x[j]));
            if (at && lam / it->a > 0) y[it->row] = lam / it->a;
        }
    }
}

}  // namespace uc

using namespace uc;

// ---------------------------------------------------------------------------
// C ABI (host part)
// ---------------------------------------------------------------------------
extern "C" {

const char *uc_last_error(void) { return g_err.c_str(); }

void uc_default_presolve_opts(uc_presolve_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->ruiz_iters = 10;
    o->pock_chambolle = 1;
    o->power_max_iter = 500;
    o->power_tol = 1e-10;
    o->value_bits = 64;
    o->threads = 0;
    o->power_device = 0;
}

void uc_default_solve_opts(uc_solve_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->tol_rel_kkt = 1e-4;
    o->tol_abs_feas = 1e-5;
    o->max_iter = 100000;
    o->n_eval = 64;
    o->use_graph = 1;
    o->pw_kp = 0.5;
    o->pw_ki = 0.0;
    o->pw_kd = 0.0;
}

int uc_build_lp(const uc_problem *prob, uc_lp **out) {
    if (!out) { set_error("uc_build_lp: null out"); return UC_EINVAL; }
    *out = nullptr;
    int rc = validate(prob);
    if (rc) return rc;
    try {
        auto lp = std::make_shared<RawLp>();
        rc = build(prob, *lp);
        if (rc) return rc;
        *out = new uc_lp{lp};
    } catch (const std::bad_alloc &) {
        set_error("uc_build_lp: out of host memory");
        return UC_ENOMEM;
    }
    return UC_OK;
}

int uc_lp_dims(const uc_lp *lp, int *n, int *m, int *m_eq, int64_t *nnz) {
    if (!lp) { set_error("uc_lp_dims: null lp"); return UC_EINVAL; }
    if (n) *n = lp->d->A.cols;
    if (m) *m = lp->d->A.rows;
    if (m_eq) *m_eq = lp->d->m_eq;
    if (nnz) *nnz = lp->d->A.nnz();
    return UC_OK;
}

int uc_lp_export(const uc_lp *lp, int32_t *rowptr, int32_t *colidx, double *val, double *q,
                 double *c, double *l, double *u) {
    if (!lp) { set_error("uc_lp_export: null lp"); return UC_EINVAL; }
    const RawLp &r = *lp->d;
    if (rowptr) std::memcpy(rowptr, r.A.rowptr.data(), r.A.rowptr.size() * 4);
    if (colidx) std::memcpy(colidx, r.A.colidx.data(), r.A.colidx.size() * 4);
    if (val) std::memcpy(val, r.A.val.data(), r.A.val.size() * 8);
    if (q) std::memcpy(q, r.q.data(), r.q.size() * 8);
    if (c) std::memcpy(c, r.c.data(), r.c.size() * 8);
    if (l) std::memcpy(l, r.l.data(), r.l.size() * 8);
    if (u) std::memcpy(u, r.u.data(), r.u.size() * 8);
    return UC_OK;
}

int uc_presolve(const uc_lp *lp, const uc_presolve_opts *opts, uc_presolved **out) {
    if (!lp || !out) { set_error("uc_presolve: null argument"); return UC_EINVAL; }
    *out = nullptr;
    uc_presolve_opts o;
    uc_default_presolve_opts(&o);
    if (opts) o = *opts;
    if (o.value_bits != 64 && o.value_bits != 32) { set_error("uc_presolve: value_bits must be 32 or 64"); return UC_EINVAL; }
    if (o.ruiz_iters < 0 || o.power_max_iter < 1) { set_error("uc_presolve: bad iteration counts"); return UC_EINVAL; }
    if (o.power_device != 0 && o.power_device != 1) { set_error("uc_presolve: power_device must be 0 or 1"); return UC_EINVAL; }
    if (o.aggressive != 0 && o.aggressive != 1) { set_error("uc_presolve: aggressive must be 0 or 1"); return UC_EINVAL; }
    if (o.eliminate_angles != 0 && o.eliminate_angles != 1) { set_error("uc_presolve: eliminate_angles must be 0 or 1"); return UC_EINVAL; }
    int threads = o.threads > 0 ? o.threads : (int)std::max(1u, std::thread::hardware_concurrency());
    try {
        auto ps = std::make_shared<PsData>();
        ps->raw = ps->orig = lp->d;
        if (o.eliminate_angles) {
            auto work = std::make_shared<RawLp>();
            auto E = std::make_shared<AngleElim>();
            const int rc0 = eliminate_angles(*lp->d, *work, *E);
            if (rc0) return rc0;
            ps->raw = work;
            ps->angles = E;
        }
        int rc = presolve_reduce(*ps->raw, *ps, ps->A, ps->q, ps->c, ps->l, ps->u, o.aggressive != 0);
        if (rc) return rc;
        ps->raw_reduced_val = ps->A.val;
        double qi = 0.0, ci = 0.0;
        for (double v : ps->q) qi = std::max(qi, std::fabs(v));
        for (double v : ps->c) ci = std::max(ci, std::fabs(v));
        ps->q_inf = qi;
        ps->c_inf = ci;
        scale_lp(*ps, o, threads);
        ps->AT = transpose(ps->A);
        if (o.power_device) {
            rc = device_power_norm(ps->A, ps->AT, o.power_max_iter, o.power_tol, &ps->norm_A);
            if (rc) return rc;
        } else {
            ps->norm_A = power_norm(ps->A, ps->AT, o.power_max_iter, o.power_tol, threads);
        }
        // the step needs tau sigma ||A_s||^2 < 1 and the power estimate is a lower
        // bound, so the step takes the larger of it and a certified upper bound
        ps->norm_bound = std::max(norm_upper_bound(ps->A, o.pock_chambolle != 0), ps->norm_A);
        ps->eta = ps->norm_bound > 0 ? 0.998 / ps->norm_bound : 1.0;
        double cn = std::sqrt(sumsq(ps->c, threads)), qn = std::sqrt(sumsq(ps->q, threads));
        ps->omega0 = (cn > 1e-10 && qn > 1e-10) ? cn / qn : 1.0;
        ps->value_bits = o.value_bits;
        if (o.value_bits == 32) {
            ps->A_val32.assign(ps->A.val.begin(), ps->A.val.end());
            ps->AT_val32.assign(ps->AT.val.begin(), ps->AT.val.end());
        }
        *out = new uc_presolved{ps};
    } catch (const std::bad_alloc &) {
        set_error("uc_presolve: out of host memory");
        return UC_ENOMEM;
    }
    return UC_OK;
}

int uc_presolve_reuse(const uc_presolved *base, const uc_lp *lp, uc_presolved **out) {
    if (!base || !lp || !out) { set_error("uc_presolve_reuse: null argument"); return UC_EINVAL; }
    *out = nullptr;
    const PsData &b = *base->d;
    std::shared_ptr<const RawLp> work = lp->d;
    std::shared_ptr<AngleElim> E;
    if (b.angles) {   // the same substitution as the base's (same grid, so the same trees)
        try {
            auto w = std::make_shared<RawLp>();
            E = std::make_shared<AngleElim>();
            const int rc0 = eliminate_angles(*lp->d, *w, *E);
            if (rc0) return rc0;
            work = w;
        } catch (const std::bad_alloc &) {
            set_error("uc_presolve_reuse: out of host memory");
            return UC_ENOMEM;
        }
    }
    const RawLp &r0 = *b.raw, &r1 = *work;
    if (r0.A.rows != r1.A.rows || r0.A.cols != r1.A.cols || r0.m_eq != r1.m_eq ||
        r0.A.rowptr != r1.A.rowptr || r0.A.colidx != r1.A.colidx || r0.A.val != r1.A.val) {
        set_error("uc_presolve_reuse: the LP's matrix differs from the base LP's");
        return UC_EINVAL;
    }
    try {
        auto ps = std::make_shared<PsData>();
        ps->raw = work;
        ps->orig = lp->d;
        ps->angles = E;
        int rc = presolve_reduce(*work, *ps, ps->A, ps->q, ps->c, ps->l, ps->u, b.aggressive);
        if (rc) return rc;
        if (ps->col_map != b.col_map || ps->row_map != b.row_map || ps->A.val != b.raw_reduced_val) {
            set_error("uc_presolve_reuse: presolve removed different rows or columns than for the base LP");
            return UC_EINVAL;
        }
        double qi = 0.0, ci = 0.0;
        for (double v : ps->q) qi = std::max(qi, std::fabs(v));
        for (double v : ps->c) ci = std::max(ci, std::fabs(v));
        ps->q_inf = qi;
        ps->c_inf = ci;
        // same reduced matrix: take the base's scaling, scaled matrices and step size
        ps->A = b.A;
        ps->AT = b.AT;
        ps->A_val32 = b.A_val32;
        ps->AT_val32 = b.AT_val32;
        ps->raw_reduced_val = b.raw_reduced_val;
        ps->Dr = b.Dr;
        ps->Dc = b.Dc;
        for (size_t i = 0; i < ps->q.size(); i++) ps->q[i] *= ps->Dr[i];
        for (size_t j = 0; j < ps->c.size(); j++) {
            ps->c[j] *= ps->Dc[j];
            ps->l[j] /= ps->Dc[j];
            ps->u[j] /= ps->Dc[j];
        }
        ps->norm_A = b.norm_A;
        ps->norm_bound = b.norm_bound;
        ps->eta = b.eta;
        // same fixed-chunk sums as uc_presolve, so omega0 is bit-identical to a full presolve
        const double cn = std::sqrt(sumsq(ps->c, 1)), qn = std::sqrt(sumsq(ps->q, 1));
        ps->omega0 = (cn > 1e-10 && qn > 1e-10) ? cn / qn : 1.0;
        ps->value_bits = b.value_bits;
        *out = new uc_presolved{ps};
    } catch (const std::bad_alloc &) {
        set_error("uc_presolve_reuse: out of host memory");
        return UC_ENOMEM;
    }
    return UC_OK;
}

int uc_presolved_dims(const uc_presolved *ps, int *n, int *m, int *m_eq, int64_t *nnz) {
    if (!ps) { set_error("uc_presolved_dims: null handle"); return UC_EINVAL; }
    if (n) *n = ps->d->n();
    if (m) *m = ps->d->m();
    if (m_eq) *m_eq = ps->d->m_eq;
    if (nnz) *nnz = ps->d->A.nnz();
    return UC_OK;
}

int uc_presolved_export(const uc_presolved *h, int32_t *rowptr, int32_t *colidx, double *val,
                        double *q, double *c, double *l, double *u, double *Dr, double *Dc,
                        int32_t *col_map, int32_t *row_map, double *scalars) {
    if (!h) { set_error("uc_presolved_export: null handle"); return UC_EINVAL; }
    const PsData &p = *h->d;
    if (rowptr) std::memcpy(rowptr, p.A.rowptr.data(), p.A.rowptr.size() * 4);
    if (colidx) std::memcpy(colidx, p.A.colidx.data(), p.A.colidx.size() * 4);
    if (val) std::memcpy(val, p.A.val.data(), p.A.val.size() * 8);
    if (q) std::memcpy(q, p.q.data(), p.q.size() * 8);
    if (c) std::memcpy(c, p.c.data(), p.c.size() * 8);
    if (l) std::memcpy(l, p.l.data(), p.l.size() * 8);
    if (u) std::memcpy(u, p.u.data(), p.u.size() * 8);
    if (Dr) std::memcpy(Dr, p.Dr.data(), p.Dr.size() * 8);
    if (Dc) std::memcpy(Dc, p.Dc.data(), p.Dc.size() * 8);
    // maps into the LP as built (through the angle elimination's maps when it ran)
    for (size_t k = 0; col_map && k < p.col_map.size(); k++)
        col_map[k] = p.angles ? p.angles->col_keep[p.col_map[k]] : p.col_map[k];
    for (size_t k = 0; row_map && k < p.row_map.size(); k++)
        row_map[k] = p.angles ? p.angles->row_keep[p.row_map[k]] : p.row_map[k];
    if (scalars) {
        scalars[0] = p.eta; scalars[1] = p.omega0; scalars[2] = p.norm_A;
        scalars[3] = p.obj_const; scalars[4] = p.q_inf; scalars[5] = p.c_inf; scalars[6] = p.norm_bound;
    }
    return UC_OK;
}

int uc_result_from_point(const uc_presolved *ps, const double *x, const double *y, uc_result **out) {
    if (!ps || !x || !y || !out) { set_error("uc_result_from_point: null argument"); return UC_EINVAL; }
    *out = nullptr;
    try {
        auto r = std::make_unique<uc_result>();
        r->ps = ps->d;
        const int n = ps->d->n(), m = ps->d->m();
        r->x_ret.assign(x, x + n);
        r->y_ret.assign(y, y + m);
        r->x_cur = r->x_avg = r->x_ret;
        r->y_cur = r->y_avg = r->y_ret;
        uc_stats &o = r->stats;
        std::memset(&o, 0, sizeof o);
        double pobj, dobj;
        host_kkt(*ps->d, x, y, o.rel_primal, o.rel_dual, o.rel_gap, o.abs_primal, pobj, dobj);
        o.dual_objective = dobj + ps->d->obj_const;
        o.abs_primal_unpolished = o.abs_primal;
        o.status = UC_OK;
        *out = r.release();
    } catch (const std::bad_alloc &) {
        set_error("uc_result_from_point: out of host memory");
        return UC_ENOMEM;
    }
    return UC_OK;
}

int uc_crossover(const uc_result *res, int64_t max_pivots, uc_result **out) {
    if (!res || !out) { set_error("uc_crossover: null argument"); return UC_EINVAL; }
    *out = nullptr;
    if (res->x_ret.empty()) { set_error("uc_crossover: the result holds no returned point"); return UC_EINVAL; }
    try {
        auto v = std::make_unique<uc_result>();
        v->ps = res->ps;
        int pivots = 0, left = 0;
        const int rc = crossover(*res->ps, res->x_ret, max_pivots, v->x_ret, v->y_ret, pivots, left);
        if (rc) return rc;
        v->x_cur = v->x_avg = v->x_ret;
        v->y_cur = v->y_avg = v->y_ret;
        uc_stats &o = v->stats;
        o = res->stats;
        o.status = UC_OK;
        o.iters = pivots;
        o.superbasic = left;
        double pobj, dobj;
        host_kkt(*res->ps, v->x_ret.data(), v->y_ret.data(), o.rel_primal, o.rel_dual, o.rel_gap, o.abs_primal,
                 pobj, dobj);
        o.dual_objective = dobj + res->ps->obj_const;
        o.polish_iters = 0;
        o.abs_primal_unpolished = o.abs_primal;
        *out = v.release();
    } catch (const std::bad_alloc &) {
        set_error("uc_crossover: out of host memory");
        return UC_ENOMEM;
    }
    return UC_OK;
}

int uc_get_raw_solution(const uc_result *res, double *x, double *y) {
    if (!res) { set_error("uc_get_raw_solution: null result"); return UC_EINVAL; }
    std::vector<double> xr, yr;
    postsolve(*res->ps, res->x_ret.data(), res->y_ret.data(), xr, yr);
    if (x) std::memcpy(x, xr.data(), xr.size() * 8);
    if (y) std::memcpy(y, yr.data(), yr.size() * 8);
    return UC_OK;
}

int uc_get_solution(const uc_result *res, double *p, double *u, double *v, double *theta,
                    double *f, double *shed, double *lmp, uc_stats *stats) {
    if (!res) { set_error("uc_get_solution: null result"); return UC_EINVAL; }
    const RawLp &raw = *res->ps->orig;
    std::vector<double> xr, yr;
    postsolve(*res->ps, res->x_ret.data(), res->y_ret.data(), xr, yr);
    const int G = raw.G, B = raw.B, L = raw.L;
    if (shed) std::memset(shed, 0, sizeof(double) * (size_t)raw.T * B);
    for (size_t j = 0; j < xr.size(); j++) {
        int64_t t = raw.col_t[j], k = raw.col_idx[j];
        switch (raw.col_kind[j]) {
            case COL_P: if (p) p[t * G + k] = xr[j]; break;
            case COL_U: if (u) u[t * G + k] = xr[j]; break;
            case COL_V: if (v) v[t * G + k] = xr[j]; break;
            case COL_TH: if (theta) theta[t * B + k] = xr[j]; break;
            case COL_F: if (f) f[t * L + k] = xr[j]; break;
            case COL_S: if (shed) shed[t * B + k] = xr[j]; break;
        }
    }
    if (lmp)
        for (size_t i = 0; i < yr.size(); i++)
            if (raw.row_kind[i] == ROW_BAL) lmp[(int64_t)raw.row_t[i] * B + raw.row_idx[i]] = yr[i];
    if (stats) {
        *stats = res->stats;
        double obj = 0.0;
        for (size_t j = 0; j < xr.size(); j++) obj += raw.c[j] * xr[j];
        stats->objective = obj;
    }
    return UC_OK;
}

int uc_get_iterate(const uc_result *res, int which, double *x, double *y) {
    if (!res) { set_error("uc_get_iterate: null result"); return UC_EINVAL; }
    const std::vector<double> *xs, *ys;
    switch (which) {
        case 0: xs = &res->x_cur; ys = &res->y_cur; break;
        case 1: xs = &res->x_avg; ys = &res->y_avg; break;
        case 2: xs = &res->x_ret; ys = &res->y_ret; break;
        case 3:   // the Farkas direction of an infeasible result (x: zeros)
            if (res->y_ray.empty()) { set_error("uc_get_iterate: the result holds no infeasibility direction"); return UC_EINVAL; }
            if (x) std::memset(x, 0, res->x_ret.size() * 8);
            if (y) std::memcpy(y, res->y_ray.data(), res->y_ray.size() * 8);
            return UC_OK;
        default: set_error("uc_get_iterate: which must be 0, 1, 2 or 3"); return UC_EINVAL;
    }
    if (x) std::memcpy(x, xs->data(), xs->size() * 8);
    if (y) std::memcpy(y, ys->data(), ys->size() * 8);
    return UC_OK;
}

void uc_free_lp(uc_lp *lp) { delete lp; }
void uc_free_presolved(uc_presolved *ps) { delete ps; }
void uc_free_result(uc_result *res) { delete res; }

}  // extern "C"
