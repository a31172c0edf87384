// rh_internal.h -- data shared by the host symbolic phase, the entry points
// and the kernels of librh.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace rh {

enum BusType : int8_t { kRef = 0, kPV = 1, kPQ = 2 };

// Result of the host symbolic phase (once per topology).
//
// Internal variable order: buses in elimination order, each contributing theta
// then (PQ only) v.  "Position" k of a bus is its place in that order; the
// slack bus has no position (no x variable).
//
// The filled matrix A = L + U of the permuted J_x is stored row-wise (CSR),
// columns ascending: [strictly lower L | diagonal | strictly upper U].  The two
// rows of a PQ bus share the same columns outside the bus (bus-level fill), so
// a kernel can walk both rows with one column list.
struct Symbolic {
    int n_bus = 0, n_branch = 0, n_gen = 0, n_pv = 0, n_pq = 0, ref = -1;
    int n_x = 0, n_p = 0, n_elim = 0;
    bool order_mf = false;                  // minimum weighted fill chosen over minimum degree

    // external index maps (documented in rh.h): -1 where absent
    std::vector<int> ix_th, ix_v, ip_v, ip_pg;
    // internal maps
    std::vector<int> ebus;          // position -> bus id
    std::vector<int> epos;          // bus id -> position (-1 for the slack)
    std::vector<int> q0;            // position -> first internal variable
    std::vector<uint8_t> nv;        // position -> 1 (PV) or 2 (PQ)
    std::vector<int> qth, qv;       // bus id -> internal variable of theta / v (-1)
    std::vector<int> perm;          // internal variable -> x index

    // bus-level patterns and schedules
    std::vector<std::vector<int>> colpat;   // position -> later positions (U side)
    std::vector<std::vector<int>> rowpat;   // position -> earlier positions (L side)
    std::vector<int> flevel, blevel;        // forward level (height) / backward level (max height - height)
    int n_flev = 0, n_blev = 0;
    std::vector<int> flev_ptr, flev_bus;    // positions grouped by forward level
    std::vector<int> blev_ptr, blev_bus;    // positions grouped by backward level
    std::vector<int> flev_maxext, blev_maxext;  // longest external row part per level

    // variable-level CSR of A
    std::vector<int> rowptr, col, diagpos;
    std::vector<int> tpos;                  // position of the transposed entry
    int64_t nnz_l = 0, nnz_u = 0;

    // Refactorisation schedule.  Buses before tail_bus0 (variables < t0) are
    // eliminated right-looking, one forward level at a time: the update step of
    // a level applies a_ij -= sum_k l_ik u_kj to every target entry of the level
    // (buses k of the level in a fixed order, theta before v), forming bus k's
    // factor entries on the fly from its final raw entries; the pivot steps,
    // which write every sparse bus's 2x2 (or 1x1) pivot block, U row and L
    // column, run once after the last level.  The trailing block [t0, n_x) is
    // then factored densely.
    int t0 = 0, tail_bus0 = 0;
    int max_tail = 0;                               // dense-tail bound in use (variables)
    int rf_n_lev = 0;
    std::vector<int> rf_lev_ptr, rf_lev_bus;        // sparse buses grouped by level
    std::vector<int64_t> rf_tgt_lev_ptr;            // level -> first target
    std::vector<int> rf_tgt_pos;                    // target position in A (-1: an empty lane)
    std::vector<int64_t> rf_tgt_gptr;               // (construction only) target -> first group
    // group (target, bus k): k's theta diagonal position dt at the first level,
    // else k itself (its pivot quantities are precomputed), k's v diagonal dv (-1
    // for a PV bus), and the positions of a_it, a_tj, a_iv, a_vj (-1, -1 for a PV
    // bus).  rf_grp holds each target's first group (six -1: none); its further
    // groups are rf_xgrp[rf_xptr[t], rf_xptr[t + 1]).
    std::vector<int> rf_grp, rf_xgrp;
    std::vector<int64_t> rf_xptr;
    // pivot jobs: level l computes the pivot quantities of buses
    // rf_piv_bus[rf_piv_lev_ptr[l] ..) from the positions rf_piv_pos (4 per job:
    // a_tt, a_tv, a_vt, a_vv; -1 for a PV bus's missing ones); job q of the level
    // owns its targets [4 q, 4 q + 4) (the entries that level updates, else empty).
    // Jobs [0, rf_piv_lev_ptr[0]) are the leaves, computed before the first level.
    std::vector<int> rf_piv_lev_ptr, rf_piv_bus, rf_piv_pos;
    // pivot steps by entry: bus, and 4 positions per entry of a U row right of the
    // bus's block: a_tj, a_vj (-1: PV), a_jt, a_jv (-1: PV)
    std::vector<int> rf_pe_bus, rf_pe_ut;
    int64_t rf_updates = 0;                         // multiply-subtracts of one refactorisation

    // admittance matrix (CSR by bus, diagonal included, parallel branches merged)
    std::vector<int> yp, yj;
    std::vector<double> G, B;
    std::vector<int> ydiag;
    std::vector<int> yrow;                          // bus of every admittance entry
    std::vector<int> pf_wb;                         // warp w of the evaluation: buses [pf_wb[w], pf_wb[w + 1])

    // J_x / J_p assembly: for every admittance entry s (bus i, neighbour-or-self j)
    // the destination of dP_i/dtheta_j, dP_i/dv_j, dQ_i/dtheta_j, dQ_i/dv_j:
    //   >= 0 : slot in A;  <= -2 : slot -(code + 2) in Jp values;  -1 : none
    std::vector<int> jac_dst;               // 4 per admittance entry
    // J_p in CSR by internal row (columns = p index), and its transpose
    std::vector<int> jp_ptr, jp_col;
    std::vector<int> jpt_ptr, jpt_row, jpt_src;
    std::vector<int> pg_slot;               // bus id -> Jp slot of its Pg column (-1)
    int64_t nnz_jx = 0;

    // Column colouring for the coloured forward-mode Jacobian (section 4.2.2):
    // J_x columns in x order and J_p columns in p order, each greedily given the
    // smallest colour not held by an earlier column that shares a row with it.
    std::vector<int> colors_x, colors_p;
    int n_colors_x = 0, n_colors_p = 0;
    // seed colour of each bus variable in the combined space [0, n_colors_x +
    // n_colors_p), J_p colours following the J_x ones; -1 where not a variable
    std::vector<int> col_th, col_v, col_pg;
    // structural J_x entries in x indices, sorted by (row, column), with their
    // slot in A; J_p rows in x indices (per internal row)
    std::vector<int> jx_slot, jx_row, jx_col, jp_xrow;
};

// Builds everything above.  Returns an empty string on success, else a message.
// level_cost: weight of one forward level when the two orders are compared
// (factor entries x n_p + level_cost x forward levels; the reading R9 of the
// paper's unstated pivot order).  max_tail: largest trailing block (variables)
// factored densely.
std::string build_symbolic(int n_bus, int n_branch, const int32_t* fr, const int32_t* to,
                           const double* r, const double* x, const double* b,
                           const int8_t* type, int64_t level_cost, Symbolic& S, int max_tail = 0);

}  // namespace rh
