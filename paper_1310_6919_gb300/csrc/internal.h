// Internal declarations shared by the CUDA translation units of libmcsdp.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace mcsdp {

// Device copies of the symbolic tables (all pointers into the caller's workspace).
struct DevSym {
  int n, m, ns, ngroup, max_nrow, max_ncol;
  int64_t nnzL, nslot;
  const int *sn_col;
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
  const double *con_w;
  const int *arow_ptr, *arow_col;
  const int64_t *arow_off;
  const int *rs_ptr, *rs_col;
  const int64_t *rs_off;
  const int *con_order, *grp_cptr, *grp_pptr, *grp_cols;
  const int64_t *grp_rowoff;
  const int *anz_ptr;
  const int16_t *anz_a, *anz_b;
  const double *anz_v;
  const int64_t *reach_ptr, *need_ptr;
  const int *reach_sn, *need_sn;
  const double *b;
};

// Status word bits written by kernels (never trap).
enum : int { ST_NOT_PD = 1, ST_NUMERIC = 2, ST_TIMEOUT = 4, ST_SIZE = 8 };

// ---------------- sparse kernels (kern_sparse.cu) ----------------
// out_layout[slot] = c0 * A_0 + c1 * sum_k vec[k] A_k at every aggregate slot (others untouched)
void launch_slot_combine(const DevSym &S, double *out_layout, const double *vec, double c0,
                         double c1, cudaStream_t st);
// Left-looking supernodal Cholesky of Y_c = Ybase + alpha_c dY for ncand candidates, one level
// of the supernodal tree per launch.  Nbuf holds ncand layouts, dinv ncand n-vectors.
void launch_ychol_level(const DevSym &S, int lvl_begin, int lvl_count, int ncand,
                        const double *alpha, const double *Ybase, const double *dY, double *Nbuf,
                        double *dinv, int *status, cudaStream_t st);
size_t ychol_smem_bytes(const DevSym &S);
// Algorithm 1: L̂ from X̄ clique by clique.
void launch_alg1(const DevSym &S, const double *Xbar, double *Lhat, double *dinvL, int *status,
                 cudaStream_t st);
size_t alg1_smem_bytes(const DevSym &S);
// P-MATRIX columns (eq. newdX2): Y^{-1} on E, M = X̂ dY Y^{-1} on E (lower and transposed)
void launch_pmatrix(const DevSym &S, const double *Lhat, const double *dinvL, const double *N,
                    const double *dinvN, const double *dY, double *YinvE, double *Mlow,
                    double *Mup, cudaStream_t st);
void launch_dx_combine(const DevSym &S, double betamu, const double *Xbar, const double *YinvE,
                       const double *Mlow, const double *Mup, double *dX, cudaStream_t st);
// clique-wise primal step length (eq. primal_length2): alpha_r per clique
void launch_primal_step(const DevSym &S, const double *Xbar, const double *dX, double *alpha_r,
                        int *status, cudaStream_t st);
size_t primal_step_smem_bytes(const DevSym &S);
// scalars: [0] X̄.Y, [1] A_0.X̄, [2] b.z, [3] max|A(X̄)-b|, [4] max|b|, [5] min alpha_r
void launch_measures(const DevSym &S, const double *Xbar, const double *Ylay, const double *z,
                     const double *alpha_r, double *scal, cudaStream_t st);
void launch_update(const DevSym &S, double *Xbar, const double *dX, double ap, double *z,
                   const double *dz, double ad, cudaStream_t st);
void launch_set_identity(const DevSym &S, double *Xbar, cudaStream_t st);

// ---------------- SCM assembly (kern_scm.cu) ----------------
// Panels X̂[P_h, P_g] and Y^{-1}[P_h, P_g] (h >= g) for groups [g0, g1) by warp-per-column
// supernodal solves; panel (g, which) lives at pan + pan_off[g - g0] + which * pan_half[g - g0].
void launch_scm_panels(const DevSym &S, int g0, int g1, const double *Lhat, const double *dinvL,
                       const double *N, const double *dinvN, double *pan, const int64_t *pan_off_dev,
                       const int *rhs_grp_dev, int nrhs, cudaStream_t st);
// Tiles B[J_h, J_g] for g in [g0, g1), h >= g; h_i = A_i . Y^{-1} on the diagonal tiles.
void launch_scm_tiles(const DevSym &S, const int2 *tiles, int ntiles, int g0, const double *pan,
                      const int64_t *pan_off_dev, double *B, int64_t ldb, double *hvec, int pmax,
                      cudaStream_t st);

// ---------------- dense SCM factorisation (kern_dense.cu) ----------------
// B internal, (m+1) x m lower, column-major, ld = ldb; row m holds g^T on entry and
// (L^{-1} g)^T on exit.
int dense_chol_bordered(double *B, int64_t ldb, int m, int *status, cudaStream_t st);
int dense_backsolve(const double *B, int64_t ldb, int m, double *x, cudaStream_t st);
void launch_rhs_border(const DevSym &S, double *B, int64_t ldb, const double *hvec, double betamu,
                       cudaStream_t st);
void launch_dz_to_user(const DevSym &S, const double *dz_int, double *dz_user, cudaStream_t st);
void launch_B_to_user(const DevSym &S, const double *Bint, int64_t ldi, double *Bout, int64_t ldo,
                      const double *h_int, double *h_out, cudaStream_t st);

}  // namespace mcsdp
