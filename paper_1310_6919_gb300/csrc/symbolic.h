// Host symbolic analysis for MC-PDIPM (Sec. 2.1, Sec. 3.1): aggregate sparsity pattern,
// minimum-degree ordering, elimination tree in postorder, fundamental supernodes (the cliques
// C_r = S_r ∪ U_r in running-intersection order), the supernodal value layout shared by L̂ and
// N, and the tables the device kernels walk.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace mcsdp {

struct ProblemData {
  int n = 0, m = 0;
  std::vector<double> b;                    // length m
  // entries of A_0..A_m, upper triangle, caller's indices; A_0 already sign-converted
  std::vector<int> mat, row, col;
  std::vector<double> val;
};

struct Symbolic {
  int n = 0, m = 0;
  std::vector<int> perm, iperm;             // new -> old, old -> new
  // supernodes (cliques), in postorder = running-intersection order
  int ns = 0;
  std::vector<int> sn_col;                  // ns+1
  std::vector<int64_t> sn_rowptr;           // ns+1
  std::vector<int> rows;                    // clique rows (new indices), S_r first, ascending
  std::vector<int64_t> sn_valptr;           // ns+1
  std::vector<int64_t> sn_dptr;             // ns+1: offsets of the ncol x ncol inverse blocks
  std::vector<int> sn_parent;               // -1 for roots
  std::vector<int> sn_fdesc;                // smallest supernode index in the subtree of s
  std::vector<int> col2sn;                  // n
  int max_nrow = 0, max_ncol = 0;
  int64_t nnz_lower_E = 0;
  // height levels: supernodes with all children in lower levels
  std::vector<int> lvl_ptr, lvl_sn;
  int height = 0;
  // left-looking update lists: target t receives updates from sources upd_src[upd_ptr[t]..)
  std::vector<int> upd_ptr, upd_src, upd_p1, upd_p2;
  std::vector<int64_t> upd_relptr;
  std::vector<int> upd_rel;                 // rows(src)[p1:] positions inside rows(t)
  // aggregate-pattern slots: distinct lower positions of A_0..A_m (new indices)
  int64_t nslot = 0;
  std::vector<int> slot_i, slot_j;          // i >= j
  std::vector<int64_t> slot_off;            // layout offset
  std::vector<int> slot_ptr;                // nslot+1 into slot_k / slot_val
  std::vector<int> slot_k;                  // 0 = A_0, k = constraint k-1 (caller order)
  std::vector<double> slot_val;
  std::vector<double> slot_a0;              // value of A_0 at the slot
  // constraints (caller order): A_k . M = sum con_w * M[con_off]  (off-diagonal weight doubled)
  std::vector<int> con_ptr;                 // m+1
  std::vector<int64_t> con_off;
  std::vector<double> con_w;
  std::vector<double> con_v;                // the entry's value itself
  bool con_disjoint = false;                // no two constraints share a stored position
  // full symmetric row lists of the aggregate pattern for sparse products
  std::vector<int> arow_ptr;                // n+1
  std::vector<int> arow_col;
  std::vector<int64_t> arow_off;
  // strict-lower row structure of each row k: (column i < k, layout offset of (k, i))
  std::vector<int> rs_ptr;                  // n+1
  std::vector<int> rs_col;
  std::vector<int64_t> rs_off;
  // connected components of the aggregate sparsity pattern that carry constraints: X̂ and Y^{-1}
  // are block-diagonal over them, so B is too (B_pq = 0 for A_p, A_q in different components).
  // Internal constraint order keeps each component contiguous: component c is internal
  // [comp_cptr[c], comp_cptr[c + 1]); no SCM group spans two components
  int ncomp = 1;
  std::vector<int> comp_cptr;               // ncomp+1
  std::vector<int> grp_comp;                // ngroup: component of each group
  // SCM groups: constraints in internal order con_order, group g = internal [grp_cptr[g], ..)
  int ngroup = 0;
  std::vector<int> con_order;               // internal -> caller
  std::vector<int> con_internal;            // caller -> internal
  std::vector<int> grp_cptr;                // ngroup+1
  std::vector<int> grp_pptr;                // ngroup+1 into grp_cols
  std::vector<int> grp_cols;                // panel columns P_g (new indices, ascending)
  std::vector<int64_t> grp_rowoff;          // ngroup+1: stacked row offset of P_h
  // nonzeros of each internal constraint in local coordinates of its group's panel, both
  // triangles: (a, b, v)
  std::vector<int> anz_ptr;                 // m+1
  std::vector<int16_t> anz_a, anz_b;
  std::vector<double> anz_v;
  // per-group supernode lists: forward reach of P_g (ascending) and backward need of
  // the rows of P_h, h >= g (ascending; walked descending)
  std::vector<int64_t> reach_ptr, need_ptr;
  std::vector<int> reach_sn, need_sn;
  // max-cut shaped (every A_k = e_k e_k^T with value 1): used for the default dual start
  bool unit_diag_constraints = false;
  bool diag_constraints = false;  // every A_k (k >= 1) is diagonal
  // the last supernode is the dense root (cliques beyond the small-clique limits merged into it)
  bool dense_root = false;
  bool a0_diag_dominant_start_ok = false;
};

struct SymbolicOptions {
  int panel_max = 80;
  int group_max = 64;
  int relax = 1;          // relaxed supernode amalgamation
  int max_clique = 96;    // amalgamation never makes a clique larger than this
  // cliques with more rows / columns than these go, with their ancestors, into one dense root
  // supernode (0 = no bound of that kind; both 0 = no dense root)
  int root_rows = 112;
  int root_cols = 96;
};

// Returns empty string on success, else an error message.
std::string analyze(const ProblemData &P, const SymbolicOptions &o, Symbolic &S);

}  // namespace mcsdp
