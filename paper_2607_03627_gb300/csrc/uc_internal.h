// Internal types shared by the host (presolve) and device (PDHG) translation units.
#pragma once

#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "uc_pdhg.h"

namespace uc {

void set_error(const char *fmt, ...);
void clear_error();

// Compressed sparse rows, int32 indices (every matrix here has < 2^31 entries).
struct Csr {
    int rows = 0, cols = 0;
    std::vector<int32_t> rowptr;   // rows + 1
    std::vector<int32_t> colidx;   // nnz, ascending within a row
    std::vector<double> val;       // nnz
    int64_t nnz() const { return (int64_t)colidx.size(); }
};

Csr transpose(const Csr &A);

enum ColKind : int8_t { COL_P = 0, COL_U, COL_V, COL_TH, COL_F, COL_S };
enum RowKind : int8_t { ROW_BAL = 0, ROW_FLOW, ROW_GUP, ROW_GLO, ROW_SU, ROW_RUP, ROW_RDN };

struct RawLp {
    int B = 0, L = 0, G = 0, T = 0, nc = 0;
    bool has_shed = false;
    Csr A;
    int m_eq = 0;
    std::vector<double> q, c, l, u;
    std::vector<int8_t> col_kind, row_kind;
    std::vector<int32_t> col_t, col_idx, row_t, row_idx;
};

struct RemovedRow {
    int row;          // raw row
    int col;          // raw column of a singleton row, -1 for an empty row; the
                      // substituted column s of a doubleton equation
    double a;         // its coefficient
    bool eq;
    bool tightened;   // the row moved a bound
    // doubleton equation a_f x_f + a x_s = q solved for x_s (aggressive presolve)
    bool doubleton = false;
    int f = -1;
    double a_f = 0.0, q = 0.0;
    bool lo_from_s = false, hi_from_s = false;   // x_f's bound came from x_s's
};

// The bus angles substituted out of a raw LP along a spanning tree per period
// (presolve option eliminate_angles): the angle-free LP's columns and rows are
// raw columns (all but the angles) and raw rows (all but the tree lines' flow
// rows); restore_angles maps its points back.
struct AngleElim {
    std::vector<int32_t> col_keep, row_keep;   // angle-free LP column / row -> raw
    std::vector<int32_t> roots;                // per period: the reference angle column
    struct Node { int32_t col, parent, fcol; double s, inv; };
    std::vector<Node> tree;                    // each period's non-root buses, breadth-first
    std::vector<int32_t> tree_row;             // raw n: removed flow row of a tree line's flow column, else -1
};
int eliminate_angles(const RawLp &raw, RawLp &out, AngleElim &E);

// Everything the device solve and the postsolve need.
struct PsData {
    // the LP the reductions started from (the angle-free LP when the angles
    // were eliminated), the LP as built, and what restores the angles
    std::shared_ptr<const RawLp> raw;
    std::shared_ptr<const RawLp> orig;
    std::shared_ptr<const AngleElim> angles;
    // reduced, scaled LP: A_s = diag(Dr) A diag(Dc)
    Csr A;            // m x n, FP64 scaled values
    Csr AT;           // n x m
    std::vector<float> A_val32, AT_val32;  // FP32 copies when value_bits == 32
    int m_eq = 0;
    std::vector<double> q, c, l, u;        // scaled
    std::vector<double> Dr, Dc;
    std::vector<int32_t> col_map, row_map; // reduced -> raw
    std::vector<double> xfix;              // raw n: value of fixed columns
    std::vector<double> l_tight, u_tight;  // raw n: bounds after presolve
    std::vector<RemovedRow> removed;
    std::vector<double> raw_reduced_val;   // reduced matrix values before scaling
    double eta = 1.0, omega0 = 1.0, norm_A = 0.0, obj_const = 0.0;
    double norm_bound = 0.0;               // max(certified upper bound, norm_A); eta = 0.998 / it
    bool aggressive = false;               // presolve substituted doubleton equations
    double q_inf = 0.0, c_inf = 0.0;       // unscaled infinity norms (relative KKT)
    int value_bits = 64;
    int long_cols = 0;   // device view: columns with more than kLongRow A^T entries, placed last
    int n() const { return A.cols; }
    int m() const { return A.rows; }
};

// ||A||_2 by power iteration on A^T A on the current CUDA device: the steps of
// the host power iteration (start 1/sqrt(n), lambda = ||A^T A v||, stop at
// relative change <= tol or after max_iter products), with fixed-order device
// reductions.  *out = sqrt(lambda).  UC_ECUDA when no device or a CUDA call
// fails, UC_ENOMEM when device memory is short.
int device_power_norm(const Csr &A, const Csr &AT, int max_iter, double tol, double *out);

// Relative KKT parts, largest absolute row violation and objectives of a
// scaled presolved point (natural order) on the unscaled presolved LP.
void host_kkt(const PsData &p, const double *xs, const double *ys, double &rel_p, double &rel_d,
              double &rel_g, double &abs_p, double &pobj, double &dobj);

// Crossover of a scaled presolved primal point to a vertex (uc_crossover.cpp):
// the vertex x_out, the simplex multipliers y_out (both scaled), the pivots
// taken and the variables left strictly between their bounds.
int crossover(const PsData &p, const std::vector<double> &xs, int64_t max_pivots, std::vector<double> &x_out,
              std::vector<double> &y_out, int &pivots, int &superbasic_left, const volatile int *cancel = nullptr);

// Host-side postsolve: scaled presolved (x_s, y_s) -> raw (x, y).
void postsolve(const PsData &ps, const double *xs, const double *ys, std::vector<double> &x,
               std::vector<double> &y);

}  // namespace uc

struct uc_lp {
    std::shared_ptr<uc::RawLp> d;
};

struct uc_presolved {
    std::shared_ptr<uc::PsData> d;
};

struct uc_result {
    std::shared_ptr<const uc::PsData> ps;
    std::vector<double> x_ret, y_ret;   // returned point (scaled presolved)
    std::vector<double> x_cur, y_cur;   // current iterate
    std::vector<double> x_avg, y_avg;   // average since the last restart
    std::vector<double> y_ray;          // primal infeasibility direction (infeasible status only)
    uc_stats stats{};
};
