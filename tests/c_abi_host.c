/* A plain C client of libmcsdp (no Python, no torch): builds the max-cut relaxation of the
 * 4-cycle in the paper's form, runs the host analysis in a host-only context and checks the
 * sizes, the exported structure and the error conventions of the C ABI.  Prints "ok" and
 * returns 0 on success; any failed check prints its line and returns 1. */
#include <stdio.h>
#include <string.h>

#include "mcsdp.h"

#define CHECK(cond)                                      \
  do {                                                   \
    if (!(cond)) {                                       \
      printf("check failed at line %d: %s\n", __LINE__, #cond); \
      return 1;                                          \
    }                                                    \
  } while (0)

int main(void) {
  /* A_0 = -L/4 of the 4-cycle (0-1-2-3-0, unit weights), A_k = e_k e_k^T, b = 1 */
  const int32_t mat[] = {0, 0, 0, 0, 0, 0, 0, 0, 1, 2, 3, 4};
  const int32_t row[] = {0, 1, 2, 3, 0, 1, 2, 0, 0, 1, 2, 3};
  const int32_t col[] = {0, 1, 2, 3, 1, 2, 3, 3, 0, 1, 2, 3};
  const double val[] = {-0.5, -0.5, -0.5, -0.5, 0.25, 0.25, 0.25, 0.25, 1, 1, 1, 1};
  const double b[] = {1, 1, 1, 1};
  mcsdp_problem p = {4, 4, 1, b, 12, mat, row, col, val};
  mcsdp_options o;
  mcsdp_default_options(&o);
  o.device = -1; /* host-only: analysis and export, no device work */
  o.relax = 0;   /* fundamental supernodes: E is exactly the filled graph */

  mcsdp_ctx *ctx = NULL;
  CHECK(mcsdp_create(&p, &o, NULL, &ctx) == MCSDP_OK);
  mcsdp_sym_info info;
  CHECK(mcsdp_sym_info_get(ctx, &info) == MCSDP_OK);
  CHECK(info.n == 4 && info.m == 4);
  /* the 4-cycle's chordal extension adds one chord: 4 diagonal + 4 edges + 1 fill */
  CHECK(info.nnz_lower_E == 9);
  CHECK(info.nslot == 8);

  int32_t perm[4], sn_col[5], sn_rows[16], con_order[4];
  int64_t sn_rowptr[5], sn_valptr[5];
  CHECK(info.nsuper >= 1 && info.nsuper <= 4);
  CHECK(mcsdp_sym_export(ctx, perm, sn_col, sn_rowptr, NULL, sn_valptr, con_order) == MCSDP_OK);
  CHECK(sn_rowptr[info.nsuper] <= 16);
  CHECK(mcsdp_sym_export(ctx, NULL, NULL, NULL, sn_rows, NULL, NULL) == MCSDP_OK);
  int seen = 0;
  for (int i = 0; i < 4; ++i) seen |= 1 << perm[i];
  CHECK(seen == 15);
  CHECK(sn_col[0] == 0 && sn_col[info.nsuper] == 4);
  CHECK(sn_valptr[info.nsuper] == info.nnz_layout);

  /* device work on a host-only context is refused with a status, not a crash */
  mcsdp_result r;
  CHECK(mcsdp_solve(ctx, &r) == MCSDP_ERR_STATE);
  CHECK(strlen(mcsdp_last_error(ctx)) > 0);
  mcsdp_destroy(ctx);

  /* input errors: an entry below the diagonal, then a duplicate entry */
  int32_t row_bad[12], col_bad[12];
  memcpy(row_bad, row, sizeof row);
  memcpy(col_bad, col, sizeof col);
  row_bad[4] = 1;                      /* A_0 entry (0, 1) given as (1, 0): row > col */
  col_bad[4] = 0;
  mcsdp_problem q = p;
  q.row = row_bad;
  q.col = col_bad;
  ctx = NULL;
  CHECK(mcsdp_create(&q, &o, NULL, &ctx) == MCSDP_ERR_ARG);
  CHECK(strstr(mcsdp_last_error(ctx), "row > col") != NULL);
  mcsdp_destroy(ctx);
  /* the last entry repeats A_3's (2, 2) in place of A_4's (3, 3) */
  const int32_t mat_dup[] = {0, 0, 0, 0, 0, 0, 0, 0, 1, 2, 3, 3};
  const int32_t row_dup[] = {0, 1, 2, 3, 0, 1, 2, 0, 0, 1, 2, 2};
  const int32_t col_dup[] = {0, 1, 2, 3, 1, 2, 3, 3, 0, 1, 2, 2};
  q = p;
  q.mat = mat_dup;
  q.row = row_dup;
  q.col = col_dup;
  ctx = NULL;
  CHECK(mcsdp_create(&q, &o, NULL, &ctx) == MCSDP_ERR_ARG);
  CHECK(strstr(mcsdp_last_error(ctx), "duplicate") != NULL);
  mcsdp_destroy(ctx);
  CHECK(mcsdp_create(NULL, &o, NULL, &ctx) == MCSDP_ERR_ARG);
  mcsdp_destroy(ctx);
  printf("ok\n");
  return 0;
}
