// Internal declarations shared by the CUDA translation units of libmcsdp.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <vector>

namespace mcsdp {

// Per-update metadata of the left-looking update lists (one 32-byte record per update u):
// source supernode d's first column, width and row count, the first row p1 of its block that
// lands in the target, the block's row count np, d itself, and the offsets of the relative row
// indices and of d's values
struct alignas(16) UpdMeta {
  int dc0, dncol, dnrow, p1;
  int np, src;
  int64_t relptr, valp;
};

// Per level of the supernode tree, for sizing the staged solve kernels: largest ncol and nrow of
// its supernodes, and for the updates its targets receive, the source chunk width (<= 8 columns)
// and the largest row count of an update block
struct LsLevel {
  int nc, nr, cw, np;
};

// Reciprocal for the pivots of the serial column loops (FP64 issues one warp instruction per 64
// cycles per sub-partition here, so the chain is kept to three dependent FP64 operations).  Seed:
// the PTX approximate FP64 reciprocal (special-function unit; relative error delta about 2^-20),
// then one third-order step of the series 1/d = s / (1 - e) with e = 1 - d s:
// r = s + s (e + e^2), whose truncation error e^3 (about 2^-60 relative) is below the final
// rounding.  Outside 2^-1000 .. 2^1000, and for negative or non-finite d, the plain division.
template <class T>
__device__ __forceinline__ T pivot_rcp(T d);
template <>
__device__ __forceinline__ double pivot_rcp<double>(double d) {
  const int hi = __double2hiint(d);
  const int ex = (hi >> 20) & 0x7ff;  // biased exponent (sign bit tested separately)
  if (hi < 0 || ex < 1023 - 1000 || ex > 1023 + 1000) return 1.0 / d;
  double s;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(s) : "d"(d));
  const double e = fma(-d, s, 1.0);
  return fma(s, fma(e, e, e), s);
}
template <>
__device__ __forceinline__ float pivot_rcp<float>(float d) {
  return __frcp_rn(d);
}

// d > 0 and finite, decided on the high word with integer operations (an FP64 comparison costs
// a full FP64 issue slot); positive numbers below 2^-1042 count as zero.
__device__ __forceinline__ bool pivot_positive(double d) {
  const int hi = __double2hiint(d);
  return hi > 0 && ((hi >> 20) & 0x7ff) != 0x7ff;
}
__device__ __forceinline__ bool pivot_positive(float d) { return d > 0.f && d < __int_as_float(0x7f800000); }

// Raises a kernel's dynamic shared-memory limit to the device's opt-in maximum (less its static
// shared memory), once per (device, kernel); thread-safe, so contexts may run on several host
// threads.  The limit does not change what a launch uses (its own request does).
void smem_optin(const void *kernel);

// Device copies of the symbolic tables (all pointers into the caller's workspace).
struct DevSym {
  int n, m, ns, ngroup, max_nrow, max_ncol;
  int max_grp_nnz;  // largest number of stored nonzeros (both triangles) of one SCM group
  int max_con_nnz;  // ... of one constraint
  int64_t nnzL, nslot, nnzD;
  const int *sn_col;
  const int64_t *sn_dptr;
  const int64_t *sn_rowptr;
  const int *rows;
  const int64_t *sn_valptr;
  const int *sn_parent, *col2sn, *lvl_sn;
  const int *upd_ptr, *upd_src, *upd_p1, *upd_p2;
  const int64_t *upd_relptr;
  const int *upd_rel;
  const int *slot_i, *slot_j;
  const int64_t *slot_off;
  const int *slot_ptr, *slot_k;
  const double *slot_val, *slot_a0;
  const int *con_ptr;
  const int64_t *con_off;
  const double *con_w, *con_v;
  const int *arow_ptr, *arow_col;
  const int64_t *arow_off;
  const int *rs_ptr, *rs_col;
  const int64_t *rs_off;
  const int *con_order, *grp_cptr, *grp_pptr, *grp_cols;
  // block-diagonal SCM: row of B holding internal constraint i's right-hand side (nullptr: m)
  const int *bord;
  const int64_t *grp_rowoff;
  const int *anz_ptr;
  const int16_t *anz_a, *anz_b;
  const double *anz_v;
  const int64_t *reach_ptr, *need_ptr;
  const int *reach_sn, *need_sn;
  const int *sn_fdesc;
  // update lists split in chunks: chunk 0 of target t is upd_ptr[t] .. upd_c0end[t] (applied by
  // t's own CTA); the extra chunks xch_beg[t] .. xch_end[t] of the xch_* tables are summed in
  // parallel into slots (offset xch_slotw in rows of the solve buffer, xch_slotf in doubles of a
  // frontal partial) and added by t's CTA in chunk order
  const int *upd_c0end, *xch_beg, *xch_end;
  const int *xch_t, *xch_ub, *xch_ue;
  const int64_t *xch_slotw, *xch_slotf;
  int64_t nslotw, nslotf;
  // per (extra chunk x, tile of 32 right-hand sides): 1 if the partial slot holds a sum, 0 if
  // every update of the chunk was passed over (the slot is then neither written nor read)
  unsigned char *xvalid;
  int xv_stride;  // tiles per chunk row of xvalid
  // first extra chunk of every target that has extra chunks, level by level
  const int *xfst;
  const UpdMeta *upd_meta;
  // clique r's entries outside its own columns: layout offsets of the packed lower triangle of
  // the (nrow - ncol)^2 block, cmap_off[cmap_ptr[r] + i (i + 1) / 2 + j] for local rows i >= j
  const int64_t *cmap_ptr, *cmap_off;
  // P-MATRIX items (nw consecutive columns): union of the columns' etree paths, ascending
  const int64_t *pm_ptr;
  const int *pm_sn;
  const double *b;
  // dense root (see kern_root.cu): the forest's supernodes are 0 .. nforest - 1; when nR > 0 the
  // root is supernode ns - 1, columns [n - nR, n), a column-major nR x nR block at root_valp
  int nforest, nR;
  int64_t root_valp;
};

// Contributions of the forest's supernodes to the root block of Y (K2 at the root): entry e of
// the root block (offset ent[e] in the column-major block) receives, for c in [ptr[e],
// ptr[e + 1]), the product of rows a = ab[c] & 0xffff and b = ab[c] >> 16 of the block of update
// u[c]'s source supernode (upd_meta), summed over its columns.
struct RootGather {
  int64_t nent;
  const int64_t *ent, *ptr;
  const int *u, *ab;
};

// C(i, j) = alpha sum_{l in [klo, K)} A[l + i lda] B[l + j ldb] + beta C(i, j), C(i, j) at
// C[i cs_i + j cs_j] (kern_root.cu: k_gemm_tn)
template <class T>
struct GemmArgs {
  int M, N, K, klo;
  const T *A;
  int64_t lda;
  const T *B;
  int64_t ldb;
  T *C;
  int64_t cs_i, cs_j;
  T alpha, beta;
  int lower, mirror, tri_a;
};

// Skip rule of the level-scheduled solves: (supernode t, tile) is processed only if bit t is set
// in one of the bitmap rows tile_keys[tile].x .. tile_keys[tile].y (bits == nullptr: never skip).
struct LsSkip {
  const uint32_t *bits;
  const int2 *tile_keys;
  int words;  // 32-bit words per bitmap row
};

// Launch shape of the multi-right-hand-side supernodal solve kernels (one warp per right-hand
// side, nw warps per CTA, factor blocks staged in shared memory).
struct SolveCfg {
  int nw;          // warps (right-hand sides) per CTA
  int wsmem;       // 1: right-hand sides in shared memory, 0: in global scratch
  int cap, cap_d, cap_r;  // stage capacities: L block, D block (doubles), rows (ints)
  int grid;        // persistent CTAs
  size_t smem;     // dynamic shared memory per CTA
};

// Status word bits written by kernels (never trap).
enum : int { ST_NOT_PD = 1, ST_NUMERIC = 2, ST_TIMEOUT = 4, ST_SIZE = 8 };

// ---------------- sparse kernels (kern_sparse.cu) ----------------
// out_layout[slot] = c0 * A_0 + c1 * sum_k vec[k] A_k at every aggregate slot (others untouched)
void launch_slot_combine(const DevSym &S, double *out_layout, const double *vec, double c0,
                         double c1, cudaStream_t st);
// Left-looking supernodal Cholesky of Y_c = Ybase + alpha_c dY for ncand candidates, one level
// of the supernodal tree per launch.  Nbuf holds ncand layouts, dinv ncand n-vectors.
// Dbuf receives, per candidate, the inverses of the diagonal blocks N_SS^{-1} (sn_dptr layout).
void launch_ychol_level(const DevSym &S, int lvl_begin, int lvl_count, int ncand,
                        const double *alpha, const double *Ybase, const double *dY, double *Nbuf,
                        double *Dbuf, int *status, const double *Pf, cudaStream_t st);
// partial sums of the extra update chunks [x0, x0+nx) for ncand candidates into Pf
// (then summed per target into the slot of its first extra chunk: xfst[f0 .. f0+nf))
void launch_ychol_partials(const DevSym &S, int x0, int nx, int f0, int nf, int ncand,
                           const double *Nbuf, double *Pf, const int *status, cudaStream_t st);
size_t ychol_smem_bytes(const DevSym &S);
// Algorithm 1: L̂ from X̄ clique by clique.
void launch_alg1(const DevSym &S, const double *Xbar, double *Lhat, double *DL, int *status,
                 cudaStream_t st);
size_t alg1_smem_bytes(const DevSym &S);
// Level-scheduled supernodal solves of the columns of W (row-major n x ldw, ncolsW columns):
// forward (L^{-1}, levels bottom-up) or backward (L^{-T}, top-down).  Returns the launch count.
// lvl_xptr_host: per level, range of extra update chunks; lvl_fptr_host: per level, range of
// xfst (targets with extra chunks); Pw: partial buffer (nslotw rows of ldw); active (host, per
// level, or nullptr): the (supernode, tile) pairs the skip rule keeps, which sets the launch shape
template <class T>
int lsolve(const DevSym &S, const int *lvl_ptr_host, const int *lvl_xptr_host,
           const int *lvl_fptr_host, const LsLevel *lvl_info, int height, bool fwd,
           const T *L, const T *D, T *W, int64_t ldw, int ncolsW, const LsSkip &sk, T *Pw,
           const int64_t *active, cudaStream_t st);
template <class T>
void launch_rhs_unit(T *W, int64_t ldw, const int *rowof, int nrhs, cudaStream_t st);
// every level fits the shared-memory staged kernels for this element size
bool lsolve_staged_fits(const LsLevel *lvl_info, int height, int elem_size);
// P-MATRIX pieces for the columns [k0, k0 + nc) held in W (row-major, ld = ldw):
// Y^{-1} on lower(E) from Wy; Ww = dY Wy; M = X̂ dY Y^{-1} on E (lower and transposed) from Ww.
// T = double (FP64 form) or float (the mixed form's solves); the outputs on E are FP64.
template <class T>
void launch_extract_lowerE(const DevSym &S, const T *W, int64_t ldw, int k0, int nc,
                           double *outE, cudaStream_t st);
template <class T>
void launch_extract_upperE(const DevSym &S, const T *W, int64_t ldw, int k0, int nc,
                           double *outE, cudaStream_t st);
template <class T>
void launch_dY_times(const DevSym &S, const double *dY, const T *Wy, T *Ww, int64_t ldw, int nc,
                     cudaStream_t st);
// differentiation (mcsdp_backward): Wout = D Win for D symmetric on lower(E) (layout);
// the symmetric matrix standing for layout weights; axpy; sym(M) on E; A(M) (+ add); the SCE border
// from a caller-order vector; per-entry gradients
void launch_E_times(const DevSym &S, const double *D, const double *Win, double *Wout, int64_t ldw,
                    int nc, cudaStream_t st);
void launch_layout_sym(const DevSym &S, const double *g, double *out, cudaStream_t st);
void launch_axpy(int64_t n, double a, const double *x, double *y, cudaStream_t st);
void launch_sym_combine(const DevSym &S, const double *Mlow, const double *Mup, double *out,
                        cudaStream_t st);
void launch_con_apply(const DevSym &S, const double *M, const double *add, double *out,
                      cudaStream_t st);
void launch_border_from_user(const DevSym &S, double *B, int64_t ldb, const double *rhs,
                             cudaStream_t st);
void launch_entry_grads(int64_t nnz, const int64_t *off, const int *k, const int *pos,
                        const double *f, const double *gA0, const double *X, const double *z,
                        const double *v, double *gC, double *gA, cudaStream_t st);
// out = (float) in, n entries (FP32 copies of the factors for the mixed form's solves)
void launch_cast_f32(const double *in, float *out, int64_t n, cudaStream_t st);
// betamu_dev (may be null): beta mu read from the device instead
void launch_dx_combine(const DevSym &S, double betamu, const double *Xbar, const double *YinvE,
                       const double *Mlow, const double *Mup, double *dX, cudaStream_t st,
                       const double *betamu_dev = nullptr);
// clique-wise primal step length (eq. primal_length2): alpha_r per clique
void launch_primal_step(const DevSym &S, const double *Xbar, const double *dX, double *alpha_r,
                        int *status, cudaStream_t st);
size_t primal_step_smem_bytes(const DevSym &S);
// scalars: [0] X̄.Y, [1] A_0.X̄, [2] b.z, [3] max|A(X̄)-b|, [4] max|b|, [5] min alpha_r
// (scal holds 16 + 6 x 64 doubles: the partials of the first stage follow the 16 scalars)
void launch_measures(const DevSym &S, const double *Xbar, const double *Ylay, const double *z,
                     const double *alpha_r, double *scal, cudaStream_t st);
// steps_dev (may be null): (gamma alpha_p, gamma alpha_d, failure) from the device; a non-zero
// failure leaves the iterate unchanged
void launch_update(const DevSym &S, double *Xbar, const double *dX, double ap, double *z,
                   const double *dz, double ad, cudaStream_t st, const double *steps_dev = nullptr);
// the graph form of an iteration (device step lengths; the layout of g in kern_sparse.cu)
void launch_graph_betamu(const double *scal, int n, double beta, double *g, cudaStream_t st);
struct DualTables {
  double first[16], geo[16];
};
void launch_dual_cands(const double *g, int round, double *cand, int ncand, const DualTables &t,
                       int *cst, cudaStream_t st);
void launch_dual_update(const int *cst, const double *cand, int ncand, double *g, cudaStream_t st);
void launch_graph_steps(const double *scal, const int *status, double gamma, double *g,
                        cudaStream_t st);
// the solve graph's loop test (kern_sparse.cu k_graph_cond)
void launch_graph_cond(cudaGraphConditionalHandle h, const double *scal, const int *status,
                       const double *g, int *cnt, int n, double gap_tol, double feas_tol,
                       cudaStream_t st);
// constraints with disjoint supports: dX += sum_k c_k A_k with c_k chosen so that
// A_k . (X̄ + dX) = b_k exactly (the projection onto the primal affine set, A A^* diagonal)
void launch_project_primal(const DevSym &S, const double *Xbar, double *dX, cudaStream_t st);
void launch_set_identity(const DevSym &S, double *Xbar, cudaStream_t st);

// ---------------- dense root (kern_root.cu) ----------------
void launch_root_assemble(const DevSym &S, const RootGather &G, const double *Yb,
                          const double *dY, double alpha, double *Nbuf, cudaStream_t st);
// root = true launches it as k_root_gemm (the dense root's P-MATRIX product)
template <class T>
void gemm_tn(const GemmArgs<T> &g, cudaStream_t st, bool root = false);
// X = L^{-1} (L dense lower with its rows mirrored above the diagonal, Linv its 32 x 32 diagonal
// block inverses; work: 256 (n + 256) values); returns launches
template <class T>
int dense_trtri(const T *L, int64_t ldl, const T *Linv, T *X, int64_t ldx, int n, T *work,
                cudaStream_t st);
// lower triangle of X^T X at Z[i zs_i + j zs_j] (and mirrored)
template <class T>
int dense_lauum(const T *X, int64_t ldx, int n, T *Z, int64_t zs_i, int64_t zs_j, bool mirror,
                cudaStream_t st);
template <class Ti, class To>
void copy_square(const Ti *src, int64_t lds, To *dst, int64_t ldd, int n, cudaStream_t st);
template <class Ti, class To>
void symmetrize(const Ti *src, int64_t lds, To *dst, int64_t ldd, int n, cudaStream_t st);
template <class T>
void dotcols(const T *A, int64_t ld, int ncol, int len, int range, const double *v, double *w,
             double alpha, double beta, cudaStream_t st);
void lz_alpha(int n, double *w, const double *gvj, const double *vj, const double *vjm1,
              double *s, int j, cudaStream_t st);
void lz_reorth(int n, int jcount, double *w, const double *Qd, const double *Q, double *h,
               cudaStream_t st);
// w -= sum_c h_c Q[c n ..] (c < jcount <= 128; h on the device)
void lz_sub(int n, int jcount, double *w, const double *Q, const double *h, cudaStream_t st);
void lz_beta(int n, const double *w, const double *gw, double *vnext, double *gvnext, double *s,
             int j, cudaStream_t st);
void lz_normalise(int n, double *v, double *gv, cudaStream_t st);
void copy_lower(const double *src, int64_t lds, double *dst, int64_t ldd, int n, cudaStream_t st);
template <class T>
void launch_unit_cols(T *W, int64_t ldw, const int *colw, int k0, int nk, cudaStream_t st);
template <class T>
void launch_root_rows_from_cols(T *W, int64_t ldw, const int *colw, int nR, int nF, cudaStream_t st);
template <class T>
void launch_extract_dense(const DevSym &S, const T *W, int64_t ldw, const int *colw, double *outE,
                          cudaStream_t st);
template <class T>
void launch_times_pattern(const DevSym &S, const double *D, const T *W, T *V, int64_t ldw,
                          const int *colw, cudaStream_t st);
// the same for a D that is zero off the diagonal (dcol: ldw values of scratch)
template <class T>
void launch_times_diag(const DevSym &S, const double *D, const T *W, T *V, int64_t ldw,
                       const int *colw, T *dcol, cudaStream_t st);
template <class T>
void launch_forest_M(const DevSym &S, const T *V, const T *Wy, int64_t ldw, int ncolw,
                     double *Mlow, double *Mup, cudaStream_t st);
template <class T>
void launch_root_M(const T *M, int nR, double *Mlow_root, double *Mup_root, cudaStream_t st);
// b[i] = a[i] (FP32 to FP64), n values
void cast_f64(const float *a, double *b, int64_t n, cudaStream_t st);
// out[0] = max_j |L_jj|, out[1] = min_j |L_jj| over the layout's diagonal (device doubles)
void launch_diag_range(const DevSym &S, const double *L, double *out, cudaStream_t st);
// the root block's P-MATRIX factor T = U_RR - L_RF Z, written transposed (Tt[j nR + r] = T_rj):
// U = rows of W (root columns [0, nR)) holding dY Y^{-1}[:, R], its forest rows already replaced by
// Z = L_FF^{-1} U_F; L_RF by root row r in CSR form (ptr[r] .. ptr[r + 1]: layout offset of the
// entry of L in off, its forest row in frow)
template <class T>
void launch_root_pull(const int64_t *ptr, const int64_t *off, const int *frow, const T *L,
                      const T *U, int64_t ldw, int nF, int nR, T *Tt, cudaStream_t st);
void launch_root_dx(int nR, double betamu, const double *X, const double *YinvE, const double *Mlow,
                    const double *Mup, double *dX, cudaStream_t st);
// mirror the strict lower triangle of a column-major square into its strict upper triangle
template <class T>
void mirror_lower(T *A, int64_t ld, int n, cudaStream_t st);
// v[i] = a pseudo-random value in [-1, 1) from a counter-based hash of (i, seed)
void fill_hash(double *v, int n, unsigned seed, cudaStream_t st);
// dst[colw[k]] = src[k] (k < n)
void permute_to_cols(const double *src, const int *colw, double *dst, int n, cudaStream_t st);
// the dense Cholesky of an n x n column-major block (FP64 task queue; kern_dense.cu)
int dense_potrf(double *A, int64_t ld, int n, int *status, double *Linv, cudaStream_t st, int *sync,
                long long budget);

// ---------------- SCM assembly (kern_scm.cu) ----------------
// Tiles B[J_h, J_g] for the listed (h, g), h >= g, from WX = X̂[:, P_g] and WY = Y^{-1}[:, P_g]
// (row-major, ld = ldw, the columns of group g start at goff[g]); h_i = A_i . Y^{-1} on the
// diagonal tiles.
size_t scm_tiles_smem_bytes(const DevSym &S, int pmax);
// T = double: FP64 form; T = float: mixed form (FP32 operands and sums, entries stored in FP64)
// max-cut-shaped constraints with X̂ and Y^{-1} formed whole: B_ij = X̂(v_i, v_j) Y^{-1}(v_i, v_j) for
// internal constraints i >= j on vertices vtx[i], h_i = Y^{-1}(v_i, v_i)
template <class T>
void launch_scm_hadamard(const DevSym &S, const T *WX, const T *WY, int64_t ldw, const int *colw,
                         const int *vtx, double *B, int64_t ldb, double *hvec, cudaStream_t st);
// colmap != nullptr (dense completion): the column of vertex k is colmap[k] (goff unused)
template <class T>
void launch_scm_tiles(const DevSym &S, const int2 *tiles, int ntiles, const T *WX, const T *WY,
                      int64_t ldw, const int *goff, double *B, int64_t ldb, double *hvec,
                      int pmax, cudaStream_t st, const int *colmap = nullptr);

// ---------------- dense SCM factorisation (kern_dense.cu) ----------------
// B internal, (m+1) x m lower, column-major, ld = ldb; row m holds g^T on entry and
// (L^{-1} g)^T on exit.
// Linv: ceil(m / 32) blocks of 32 x 32 (NB x NB) values receiving the inverses of the diagonal blocks
// Streams of the blocked Cholesky with lookahead: the critical path (diagonal block, panel solve,
// update of the next block column) on a high-priority stream, the rest of every trailing update
// on a low-priority one, forked from and joined back into the caller's stream.
// The launch sequence (about four kernels per 32-column panel plus the stream dependencies) is
// the same at every iteration, so after one eager run it is captured once into a CUDA graph per
// (element type, matrix, size) and replayed.
struct CholGraph {
  const void *B = nullptr, *Linv = nullptr;
  const int *status = nullptr;
  int64_t ldb = 0;
  int m = 0, rows = 0, esize = 0, runs = 0, kernels = 0;
  cudaGraphExec_t exec = nullptr;
};
struct CholStreams {
  // synchronisation words of the FP64 task-queue factorisation (nullptr: launch per panel)
  int *dag_sync = nullptr;
  size_t dag_words = 0;
  long long dag_budget = 0;  // cycles per device wait (options.timeout_cycles; 0 = default)
  cudaStream_t chain = nullptr, rest = nullptr;
  cudaEvent_t next[2] = {}, rest_ev[2] = {}, fork = nullptr, chain_done = nullptr;
  cudaEvent_t entry = nullptr, exit = nullptr;  // caller's stream -> chain stream -> caller's
  CholGraph graphs[4];
  // FP32 factorisation with tensor-core trailing updates (kern_tc.cu): the split panel buffers
  // (tc_rows rows of TC_PANEL values, hi and lo) and the error word of its bounded waits;
  // nullptr: the FP32 factor stays on the CUDA cores
  float *tc_hi = nullptr, *tc_lo = nullptr;
  int tc_rows = 0;
  int *tc_err = nullptr;
};
void chol_graphs_destroy(CholStreams *cs);
// The diagonal blocks of a block-diagonal SCM for one task-queue launch and one batched back
// substitution (kern_dense.cu): block b at rows and columns off[b], mb[b] of them, bordered by
// the row after it; tile counters from word soff[b] of the synchronisation buffer's tile area;
// diagonal-tile inverses at loff[b]; the queue's segments (the blocks' ticket phases
// interleaved, see DagBlocks in kern_dense.cu).  Device arrays.
struct DagBlockTables {
  int nblk = 0, max_m = 0, nseg = 0;
  const int *off = nullptr, *mb = nullptr;
  const int64_t *soff = nullptr, *loff = nullptr;
  const int64_t *seg_start = nullptr, *seg_l0 = nullptr;
  const int *seg_blk = nullptr, *seg_k = nullptr;
  int64_t total = 0;        // tickets over all blocks
  size_t tile_words = 0;    // counters over all blocks (2 R_b C_b each)
  size_t words = 0;         // the synchronisation buffer (chol_dag_blocks_words)
  int64_t useful_ctas = 0;  // sum of C_b^2 / 4: tasks the blocks can have ready at once
};
// the block queue's host tables for blocks of mb[b] columns (each bordered by one row): tile
// counter offsets, the interleaved segments (see DagBlocks in kern_dense.cu), ticket total
struct DagBlockPlan {
  std::vector<int64_t> soff, seg_start, seg_l0;
  std::vector<int> seg_blk, seg_k;
  int64_t total = 0, useful_ctas = 0;
  size_t tile_words = 0, words = 0;
};
void chol_dag_block_plan(const std::vector<int> &mb, DagBlockPlan &pl);
size_t chol_dag_blocks_words(size_t tile_words);
// every block's bordered factorisation in one launch (FP64)
int dense_chol_dag_blocks(double *B, int64_t ldb, const DagBlockTables &bt, int *status,
                          double *Linv_all, cudaStream_t st, int *sync, long long budget);
// every block's back substitution in one launch (one cluster per block); -1 if a block is too
// large for the cluster kernel's shared-memory vector
int dense_backsolve_blocks(const double *B, int64_t ldb, const DagBlockTables &bt,
                           const double *Linv_all, double *x, cudaStream_t st);
// words of the task-queue factorisation's synchronisation buffer (m columns, rows rows)
size_t chol_dag_words(int m, int rows);
// cs == nullptr: everything on st, no lookahead, no graph
int dense_chol_bordered(double *B, int64_t ldb, int m, int *status, double *Linv,
                        cudaStream_t st, CholStreams *cs);
int dense_backsolve(const double *B, int64_t ldb, int m, const double *Linv, double *x,
                    cudaStream_t st);
int dense_chol_f32(float *B, int64_t ldb, int m, int *status, float *Linv, cudaStream_t st,
                   CholStreams *cs);
// Mixed precision.  mixed_factor: B made fully symmetric (strict upper <- lower^T), B32 <- FP32
// Cholesky factor of B (L^T in its strict upper triangle), g <- row m of B (the right-hand side
// border), r <- g, x <- 0.
// For m >= 4096 with dsc given, the factor is of the equilibrated S B S, S = diag(dsc),
// dsc_i = 1 / sqrt(B_ii) (a unit diagonal: the scales of B's rows no longer spend FP32 range),
// and the refinement solves through S (pass the same dsc to mixed_refine_step).  shift is added
// to the diagonal of the matrix factored (a preconditioner when the FP32 factor of B breaks down).
// tinv (may be null; m >= 4096): the inverses of the factor's diagonal blocks of 1024 rows are
// formed there for the substitutions (trsv_tinv_buffer_floats(m) floats)
int mixed_factor(double *B, int64_t ldb, int m, float *B32, float *Linv32, int *status,
                 double *g, double *r, double *x, double *dsc, double shift, float *tinv,
                 cudaStream_t st, CholStreams *cs);
int64_t trsv_tinv_floats(int m);
int64_t trsv_tinv_buffer_floats(int m);
// number of column chunks of the refinement's matrix-vector product (P, A hold chunks x m)
int mixed_chunks(int m);
// one refinement step: x += (L32 L32^T)^{-1} r, then r = g - B x (FP64) and
// norms = (max|r|, max(|B||x| + |g|)); for m >= 4096 the substitutions are blocked by panels
// of 1024 rows over all SMs (P holds their FP32 vector), below that one cluster of 8 CTAs
int mixed_refine_step(const double *B, int64_t ldb, int m, const float *L32, const float *Linv32,
                      const double *g, double *x, double *r, double *P, double *A, double *norms,
                      const double *dsc, const float *tinv, cudaStream_t st);
// GMRES form of the mixed SCE solve (m >= 4096): out = B v; w = S (L32 L32^T)^{-1} S u (the
// preconditioner: the FP32 factor of the equilibrated S B S, S = diag(dsc)); r = g - B x with
// norms = (max|r|, max(|B||x| + |g|)).  P and A are the refinement's partial-product buffers.
int mixed_matvec(const double *B, int64_t ldb, int m, const double *v, double *out, double *P,
                 double *A, cudaStream_t st);
int mixed_precond(const float *L32, int m, const float *Linv32, const double *u, double *w,
                  double *P, const double *dsc, const float *tinv, cudaStream_t st);
int mixed_residual(const double *B, int64_t ldb, int m, const double *g, const double *x,
                   double *r, double *P, double *A, double *norms, cudaStream_t st);
void launch_rhs_border(const DevSym &S, double *B, int64_t ldb, const double *hvec, double betamu,
                       cudaStream_t st, const double *betamu_dev = nullptr);
void launch_dz_to_user(const DevSym &S, const double *dz_int, double *dz_user, cudaStream_t st);
void launch_B_to_user(const DevSym &S, const double *Bint, int64_t ldi, double *Bout, int64_t ldo,
                      const double *h_int, double *h_out, cudaStream_t st);

}  // namespace mcsdp
