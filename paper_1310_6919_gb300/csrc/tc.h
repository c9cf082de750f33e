// Tensor-core (tcgen05) FP32 products of kern_tc.cu: declarations for the translation units that
// call them (the tensor-map type needs the driver API header).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace mcsdp {

// one K-major FP32 operand split into TF32 hi and lo parts, each reached by a 2-D tensor map
// (inner dimension K, outer the rows); (x, y) = tensor-map coordinates of the first element
struct TcOperand {
  CUtensorMap hi, lo;
  int x, y;
};

// tensor map of rows x kdim FP32 values, row r at base + r ld (ld a multiple of 4, base 16-byte
// aligned), boxes of 32 x 128, 128-byte swizzle, zero fill outside; false if it cannot be made
bool make_tmap_kmajor(CUtensorMap *map, const float *base, int64_t ld, int64_t kdim, int64_t rows);

// hi[c + r ldo] = tf32(a), lo[c + r ldo] = tf32(a - hi) for a = a[r lda_r + c lda_c]
// (rows x cols); tdst != nullptr: also tdst[c + r tld] = a
void split_tf32(const float *a, int64_t lda_r, int64_t lda_c, int rows, int cols, float *hi,
                float *lo, int64_t ldo, float *tdst, int64_t tld, cudaStream_t st);

// C(i, j) = alpha sum_{l < K} A(l, i) B(l, j) + beta C(i, j) for i < M, j < N on the tensor cores
// (three TF32 products per FP32 product), C(i, j) at C[i cs_i + j cs_j]; lower: i >= j only;
// mirror: C(j, i) written too; *err |= ST_TIMEOUT if a bounded wait ran out
void gemm_3xtf32(const TcOperand &A, const TcOperand &B, int M, int N, int K, float *C,
                 int64_t cs_i, int64_t cs_j, float alpha, float beta, bool lower, bool mirror,
                 int *err, cudaStream_t st);

// working storage of the tensor-core Cholesky: the split panel (tc_panel(m) x rows, hi and lo);
// wide panels for large m keep the trailing products' K long (their epilogue read-modify-write
// of C is then amortised over more MMAs), narrow ones keep small factorisations on the tensor
// cores at all
constexpr int TC_PANEL = 256, TC_PANEL_WIDE = 1024;
inline int tc_panel(int m) { return m >= 8 * TC_PANEL_WIDE ? TC_PANEL_WIDE : TC_PANEL; }
struct TcWork {
  float *hi = nullptr, *lo = nullptr;
  int rows = 0;  // capacity in rows
};

}  // namespace mcsdp
