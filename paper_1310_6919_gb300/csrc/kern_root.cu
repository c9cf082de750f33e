// Dense-root kernels.  When the chordal extension has cliques too large for the small-clique
// (shared-memory) kernels, the symbolic analysis merges them, with their ancestors, into one
// root supernode R whose clique is R itself (a dense |R| x |R| block of the layout, column-major).
// Everything below R is a forest of small cliques handled by the level-scheduled kernels; this
// file holds the dense work on R:
//   * Y = N N^T at the root (type (v) of Sec. 3.1): the root block of Y minus the forest's
//     contributions (gathered per entry in a fixed order), then a dense Cholesky;
//   * X = L^{-1} of a dense Cholesky factor (blocked, right-looking) and Z = X^T X, which give
//     (Y^{-1})_RR = N_RR^{-T} N_RR^{-1} and, for Algorithm 1 at the root, X̄_RR^{-1};
//   * one GEMM shape C = alpha A^T B + beta C with A, B column-major (both operands K-major),
//     used by the inverse, its product, and the P-MATRIX (eq. newdX2) on the root block;
//   * matrix-vector products and vector kernels for the Lanczos step-length bounds.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "internal.h"

namespace mcsdp {

// ---------------------------------------------------------------------------------------------
// K2 at the root

// N_RR = Yb_RR + alpha dY_RR over the whole column-major block (its strict upper part is unused)
__global__ void k_root_init(const double *__restrict__ Yb, const double *__restrict__ dY,
                            double alpha, double *N, int64_t cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt;
       i += (int64_t)gridDim.x * blockDim.x)
    N[i] = dY ? fma(alpha, dY[i], Yb[i]) : Yb[i];
}

// N_RR(e) -= sum over the forest supernodes d whose clique meets R of N(a, S_d) . N(b, S_d),
// (a, b) the rows of d's block landing on the entry; the contributions of every entry are
// listed in a fixed order, so the sum is reproducible bit for bit
__global__ void k_root_gather(const UpdMeta *__restrict__ meta, RootGather G,
                              const double *__restrict__ Nsrc, double *Nroot) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < G.nent;
       e += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int64_t c = G.ptr[e]; c < G.ptr[e + 1]; ++c) {
      const UpdMeta q = meta[G.u[c]];
      const int ab = G.ab[c], a = ab & 0xffff, b = ab >> 16;
      const double *col = Nsrc + q.valp;
      for (int l = 0; l < q.dncol; ++l) {
        const int64_t o = (int64_t)l * q.dnrow;
        acc = fma(col[o + a], col[o + b], acc);
      }
    }
    Nroot[G.ent[e]] -= acc;
  }
}

void launch_root_assemble(const DevSym &S, const RootGather &G, const double *Yb,
                          const double *dY, double alpha, double *Nbuf, cudaStream_t st) {
  const int64_t cnt = (int64_t)S.nR * S.nR;
  int blocks = (int)std::min<int64_t>(4096, (cnt + 255) / 256);
  k_root_init<<<blocks, 256, 0, st>>>(Yb + S.root_valp, dY ? dY + S.root_valp : nullptr, alpha,
                                      Nbuf + S.root_valp, cnt);
  if (G.nent > 0) {
    blocks = (int)std::min<int64_t>(4096, (G.nent + 255) / 256);
    k_root_gather<<<blocks, 256, 0, st>>>(S.upd_meta, G, Nbuf, Nbuf + S.root_valp);
  }
}

// ---------------------------------------------------------------------------------------------
// GEMM C(i, j) = alpha sum_{l in [klo, K)} A[l + i lda] B[l + j ldb] + beta C(i, j), i < M, j < N.
// Both operands column-major with the summation index l contiguous (C = A^T B).  C(i, j) is at
// C[i cs_i + j cs_j] (column- or row-major).  lower: only i >= j is formed (tiles above the
// diagonal skipped); mirror: C(j, i) is written too.  tri_a: A[l + i lda] = 0 for l < i (A^T
// lower triangular), so a tile's sum starts at its first row.  64 x 64 tile per CTA, 256
// threads, 4 x 4 outputs per thread, K in steps of 16 through shared memory.
constexpr int GB = 64, GK = 16;
constexpr int TRI_BLK = 256;  // block rows of the triangular inverse

template <class T>
__device__ __forceinline__ void gemm_tn_tile(const GemmArgs<T> &g) {
  __shared__ T As[2][GK][GB + 1];
  __shared__ T Bs[2][GK][GB + 1];
  const int i0 = blockIdx.x * GB, j0 = blockIdx.y * GB;
  if (g.lower && i0 + GB - 1 < j0) return;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  int klo = g.klo;
  if (g.tri_a) klo = max(klo, i0);
  T acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = T(0);
  // loader: element e = tid + 256 r (r < 4) of the 16 x 64 tile: l = e % 16, i = e / 16
  T ra[4], rb[4];
  auto load = [&](int k0) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + 256 * r, l = e & (GK - 1), ii = e >> 4;
      const int gl = k0 + l, gi = i0 + ii, gj = j0 + ii;
      ra[r] = (gl < g.K && gi < g.M) ? g.A[gl + (int64_t)gi * g.lda] : T(0);
      rb[r] = (gl < g.K && gj < g.N) ? g.B[gl + (int64_t)gj * g.ldb] : T(0);
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + 256 * r, l = e & (GK - 1), ii = e >> 4;
      As[buf][l][ii] = ra[r];
      Bs[buf][l][ii] = rb[r];
    }
  };
  int buf = 0;
  if (klo < g.K) {
    load(klo);
    store(0);
  }
  __syncthreads();
  for (int k0 = klo; k0 < g.K; k0 += GK) {
    const bool more = k0 + GK < g.K;
    if (more) load(k0 + GK);
#pragma unroll
    for (int l = 0; l < GK; ++l) {
      T a[4], b[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) a[p] = As[buf][l][ty + 16 * p];
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = Bs[buf][l][tx + 16 * q];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
    }
    if (more) {
      store(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int i = i0 + ty + 16 * p;
    if (i >= g.M) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = j0 + tx + 16 * q;
      if (j >= g.N || (g.lower && i < j)) continue;
      T *dst = g.C + (int64_t)i * g.cs_i + (int64_t)j * g.cs_j;
      const T v = g.beta == T(0) ? g.alpha * acc[p][q] : fma(g.alpha, acc[p][q], g.beta * *dst);
      *dst = v;
      if (g.mirror && i != j) g.C[(int64_t)j * g.cs_i + (int64_t)i * g.cs_j] = v;
    }
  }
}

template <class T>
__global__ void __launch_bounds__(256) k_gemm_tn(GemmArgs<T> g) {
  gemm_tn_tile<T>(g);
}
// the same product under its own name: the dense root's P-MATRIX GEMM (so that a profiler can
// select it among the other products)
template <class T>
__global__ void __launch_bounds__(256) k_root_gemm(GemmArgs<T> g) {
  gemm_tn_tile<T>(g);
}

template <class T>
void gemm_tn(const GemmArgs<T> &g, cudaStream_t st, bool root) {
  if (g.M <= 0 || g.N <= 0) return;
  dim3 grid((g.M + GB - 1) / GB, (g.N + GB - 1) / GB);
  if (root) k_root_gemm<T><<<grid, 256, 0, st>>>(g);
  else k_gemm_tn<T><<<grid, 256, 0, st>>>(g);
}

// ---------------------------------------------------------------------------------------------
// X = L^{-1} for a dense lower-triangular L (n x n, column-major, ld): L's rows are also held
// transposed in its strict upper triangle (as the dense Cholesky leaves them), and Linv holds the
// inverses of its 32 x 32 diagonal blocks (column-major, ld 32).  Blocked forward substitution of
// L X = I by block rows, right-looking: X starts as I; at step k, block row k becomes
// Linv_kk X_k (its columns 0 .. k), then the rows below are updated, X_i -= L_ik X_k, by the GEMM
// (A(l, i) = L(i, l) from the transposed copy).  Only the lower triangle of X is written.

template <class T>
__global__ void k_set_unit_lower(T *X, int64_t ld, int n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    X[i + (int64_t)j * ld] = i == j ? T(1) : T(0);
  }
}

// block row k (rows k0 .. k0 + nb): X[k0.., c0 .. c0 + 32) = Linv_k X[k0.., c0 .. c0 + 32)
template <class T>
__global__ void k_trtri_scale(const T *__restrict__ Linv_k, T *X, int64_t ld, int k0, int nb,
                              int ncol) {
  __shared__ T Ls[32][33];
  __shared__ T Xs[32][33];
  const int c0 = blockIdx.x * 32;
  const int tid = threadIdx.x;
  for (int e = tid; e < 32 * 32; e += blockDim.x) {
    const int r = e & 31, c = e >> 5;
    Ls[r][c] = (r < nb && c < nb) ? Linv_k[r + c * 32] : T(0);
    Xs[r][c] = (r < nb && c0 + c < ncol) ? X[(k0 + r) + (int64_t)(c0 + c) * ld] : T(0);
  }
  __syncthreads();
  const int r = tid & 31, cq = tid >> 5;  // 8 warps, 4 columns each
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = cq * 4 + q;
    T acc = T(0);
#pragma unroll 8
    for (int l = 0; l < 32; ++l) acc = fma(Ls[r][l], Xs[l][c], acc);
    if (r < nb && c0 + c < ncol) X[(k0 + r) + (int64_t)(c0 + c) * ld] = acc;
  }
}

// the inverse of the kb x kb diagonal block of L at (k0, k0) into X's block at (k0, k0) (X's block
// holds I on entry): 32-row steps of the substitution inside the block
template <class T>
static int trtri_diag(const T *L, int64_t ldl, const T *Linv, T *X, int64_t ldx, int k0, int kb,
                      cudaStream_t st) {
  int nl = 0;
  T *Xb = X + k0 + (int64_t)k0 * ldx;
  const T *Lb = L + k0 + (int64_t)k0 * ldl;
  for (int q0 = 0; q0 < kb; q0 += 32) {
    const int nb = std::min(32, kb - q0), ncol = q0 + nb;
    k_trtri_scale<T><<<(ncol + 31) / 32, 256, 0, st>>>(Linv + (int64_t)((k0 + q0) / 32) * 1024, Xb,
                                                       ldx, q0, nb, ncol);
    ++nl;
    const int r0 = q0 + nb;
    if (r0 >= kb) break;
    GemmArgs<T> g{};
    g.M = kb - r0;
    g.N = ncol;
    g.K = nb;
    g.A = Lb + q0 + (int64_t)r0 * ldl;  // A(l, i) = L(r0 + i, q0 + l), held transposed above
    g.lda = ldl;
    g.B = Xb + q0;
    g.ldb = ldx;
    g.C = Xb + r0;
    g.cs_i = 1;
    g.cs_j = ldx;
    g.alpha = T(-1);
    g.beta = T(1);
    gemm_tn<T>(g, st);
    ++nl;
  }
  return nl;
}

// D^T of the kb x kb lower block at D (ld) into Dt (ld 256): Dt[l + i 256] = D(i, l)
template <class T>
__global__ void k_transpose_block(const T *__restrict__ D, int64_t ld, int kb, T *Dt) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kb * kb; e += gridDim.x * blockDim.x) {
    const int i = e % kb, l = e / kb;
    Dt[l + (int64_t)i * TRI_BLK] = D[i + (int64_t)l * ld];
  }
}

// X[k0 + i, j] = T[i + j 256] for i < kb, j < ncol
template <class T>
__global__ void k_copy_rows_back(const T *__restrict__ Tm, T *X, int64_t ldx, int k0, int kb, int ncol) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)kb * ncol;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % kb), j = (int)(e / kb);
    X[k0 + i + (int64_t)j * ldx] = Tm[i + (int64_t)j * TRI_BLK];
  }
}

// Blocked in two levels: 256-row block rows (products with K = 256 keep the GEMM efficient), and
// inside each 256 x 256 diagonal block the 32-row substitution above.  Step K: the diagonal block's
// inverse D_K; the block row X_K = D_K R_K (R_K its accumulated right-hand side, columns left of
// the block) formed in work and copied back; then the rows below, R_I -= L_IK X_K.  work holds
// 256 x n values plus a 256 x 256 block.
template <class T>
int dense_trtri(const T *L, int64_t ldl, const T *Linv, T *X, int64_t ldx, int n, T *work,
                cudaStream_t st) {
  if (n <= 0) return 0;
  const int64_t cnt = (int64_t)n * n;
  const int blocks = (int)std::min<int64_t>(4096, (cnt + 255) / 256);
  k_set_unit_lower<T><<<blocks, 256, 0, st>>>(X, ldx, n);
  int nl = 1;
  T *Tm = work, *Dt = work + (size_t)TRI_BLK * n;
  for (int k0 = 0; k0 < n; k0 += TRI_BLK) {
    const int kb = std::min(TRI_BLK, n - k0);
    nl += trtri_diag<T>(L, ldl, Linv, X, ldx, k0, kb, st);
    if (k0 > 0) {
      // X_K(:, 0 .. k0) = D_K R_K(:, 0 .. k0)
      k_transpose_block<T><<<(kb * kb + 255) / 256, 256, 0, st>>>(X + k0 + (int64_t)k0 * ldx, ldx,
                                                                   kb, Dt);
      GemmArgs<T> g{};
      g.M = kb;
      g.N = k0;
      g.K = kb;
      g.A = Dt;
      g.lda = TRI_BLK;
      g.B = X + k0;
      g.ldb = ldx;
      g.C = Tm;
      g.cs_i = 1;
      g.cs_j = TRI_BLK;
      g.alpha = T(1);
      g.beta = T(0);
      gemm_tn<T>(g, st);
      k_copy_rows_back<T><<<(int)std::min<int64_t>(4096, ((int64_t)kb * k0 + 255) / 256), 256, 0,
                            st>>>(Tm, X, ldx, k0, kb, k0);
      nl += 3;
    }
    const int r0 = k0 + kb;
    if (r0 >= n) break;
    GemmArgs<T> g{};
    g.M = n - r0;
    g.N = r0;
    g.K = kb;
    g.A = L + k0 + (int64_t)r0 * ldl;  // A(l, i) = L(r0 + i, k0 + l), held transposed above
    g.lda = ldl;
    g.B = X + k0;                       // B(l, j) = X(k0 + l, j), j < r0
    g.ldb = ldx;
    g.C = X + r0;
    g.cs_i = 1;
    g.cs_j = ldx;
    g.alpha = T(-1);
    g.beta = T(1);
    gemm_tn<T>(g, st);
    ++nl;
  }
  return nl;
}

// Z = X^T X for a lower-triangular X (n x n, column-major, zero above the diagonal): the lower
// triangle of Z at Z[i zs_i + j zs_j], mirrored when mirror is set
template <class T>
int dense_lauum(const T *X, int64_t ldx, int n, T *Z, int64_t zs_i, int64_t zs_j, bool mirror,
                cudaStream_t st) {
  GemmArgs<T> g{};
  g.M = n;
  g.N = n;
  g.K = n;
  g.A = X;
  g.lda = ldx;
  g.B = X;
  g.ldb = ldx;
  g.C = Z;
  g.cs_i = zs_i;
  g.cs_j = zs_j;
  g.alpha = T(1);
  g.beta = T(0);
  g.lower = 1;
  g.mirror = mirror ? 1 : 0;
  g.tri_a = 1;
  gemm_tn<T>(g, st);
  return 1;
}

// ---------------------------------------------------------------------------------------------
// Copies and casts between the root block, the dense completion buffers and scratch

// dst[i + j ld_d] = (To) src[i + j ld_s] for i, j < n (whole square)
template <class Ti, class To>
__global__ void k_copy_square(const Ti *__restrict__ src, int64_t lds, To *dst, int64_t ldd, int n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    dst[i + (int64_t)j * ldd] = (To)src[i + (int64_t)j * lds];
  }
}

template <class Ti, class To>
void copy_square(const Ti *src, int64_t lds, To *dst, int64_t ldd, int n, cudaStream_t st) {
  if (n <= 0) return;
  const int64_t cnt = (int64_t)n * n;
  const int blocks = (int)std::min<int64_t>(4096, (cnt + 255) / 256);
  k_copy_square<Ti, To><<<blocks, 256, 0, st>>>(src, lds, dst, ldd, n);
}

// full symmetric matrix from the lower triangle of a column-major block: dst(i, j) = src(max, min)
template <class Ti, class To>
__global__ void k_symmetrize(const Ti *__restrict__ src, int64_t lds, To *dst, int64_t ldd, int n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    const int a = i > j ? i : j, b = i > j ? j : i;
    dst[i + (int64_t)j * ldd] = (To)src[a + (int64_t)b * lds];
  }
}

template <class Ti, class To>
void symmetrize(const Ti *src, int64_t lds, To *dst, int64_t ldd, int n, cudaStream_t st) {
  if (n <= 0) return;
  const int64_t cnt = (int64_t)n * n;
  const int blocks = (int)std::min<int64_t>(4096, (cnt + 255) / 256);
  k_symmetrize<Ti, To><<<blocks, 256, 0, st>>>(src, lds, dst, ldd, n);
}

// ---------------------------------------------------------------------------------------------
// Matrix-vector products for the Lanczos bounds
// w_j = beta w_j + alpha sum_{i in range(j)} A[i + j ld] v_i, one warp per column j;
// range: 0 -> [0, len), 1 -> [j, len) (A lower), 2 -> [0, j] (A upper)
template <class T>
__global__ void k_dotcols(const T *__restrict__ A, int64_t ld, int ncol, int len, int range,
                          const double *__restrict__ v, double *w, double alpha, double beta) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= ncol) return;
  const int lo = range == 1 ? j : 0, hi = range == 2 ? min(len, j + 1) : len;
  const T *col = A + (int64_t)j * ld;
  // four independent partial sums (four loads of the column in flight per lane), in T over
  // blocks of 1024 entries (FP32 in the mixed form: the matrix is FP32 and FP64 arithmetic would
  // run on the slow FP64 pipe), carried in FP64
  double acc = 0.0;
  int i = lo + lane;
  while (i + 96 < hi) {
    T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
    const int iend = min(hi - 96, i + 1024);
    for (; i < iend; i += 128) {
      a0 = fma(__ldcs(col + i), (T)v[i], a0);
      a1 = fma(__ldcs(col + i + 32), (T)v[i + 32], a1);
      a2 = fma(__ldcs(col + i + 64), (T)v[i + 64], a2);
      a3 = fma(__ldcs(col + i + 96), (T)v[i + 96], a3);
    }
    acc += (double)((a0 + a1) + (a2 + a3));
  }
  for (; i < hi; i += 32) acc = fma((double)col[i], v[i], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) w[j] = beta == 0.0 ? alpha * acc : fma(alpha, acc, beta * w[j]);
}

// the same with 16-byte loads, for columns that start on a 16-byte boundary (A aligned and
// ld sizeof(T) a multiple of 16): each lane takes runs of four consecutive entries (one float4,
// or two double2, of the column and two double2 of v) with two runs in flight; the range's
// unaligned head and the tail by single loads
template <class T>
__device__ __forceinline__ void load4(const T *p, T *o);
template <>
__device__ __forceinline__ void load4<float>(const float *p, float *o) {
  const float4 q = __ldcs(reinterpret_cast<const float4 *>(p));
  o[0] = q.x, o[1] = q.y, o[2] = q.z, o[3] = q.w;
}
template <>
__device__ __forceinline__ void load4<double>(const double *p, double *o) {
  const double2 a = __ldcs(reinterpret_cast<const double2 *>(p));
  const double2 b = __ldcs(reinterpret_cast<const double2 *>(p) + 1);
  o[0] = a.x, o[1] = a.y, o[2] = b.x, o[3] = b.y;
}

template <class T>
__global__ void k_dotcols_v4(const T *__restrict__ A, int64_t ld, int ncol, int len, int range,
                             const double *__restrict__ v, double *w, double alpha, double beta) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= ncol) return;
  const int lo = range == 1 ? j : 0, hi = range == 2 ? min(len, j + 1) : len;
  const T *col = A + (int64_t)j * ld;
  const int h0 = min(hi, (lo + 3) & ~3);
  const int hb = h0 + ((hi - h0) & ~3);
  double acc = 0.0;
  for (int i = lo + lane; i < h0; i += 32) acc = fma((double)col[i], v[i], acc);
  // runs of 4 from h0, lane-strided; partial sums in T per 1024 entries, carried in FP64
  int q = (h0 >> 2) + lane;
  const int qend = hb >> 2;
  while (q < qend) {
    T a0 = T(0), a1 = T(0);
    const int qstop = min(qend, q + 256);
    for (; q + 32 < qstop; q += 64) {
      T c0[4], c1[4];
      load4<T>(col + 4 * q, c0);
      load4<T>(col + 4 * (q + 32), c1);
      const double2 *vv0 = reinterpret_cast<const double2 *>(v + 4 * q);
      const double2 *vv1 = reinterpret_cast<const double2 *>(v + 4 * (q + 32));
      const double2 x0 = vv0[0], x1 = vv0[1], y0 = vv1[0], y1 = vv1[1];
      a0 = fma(c0[0], (T)x0.x, a0);
      a0 = fma(c0[1], (T)x0.y, a0);
      a0 = fma(c0[2], (T)x1.x, a0);
      a0 = fma(c0[3], (T)x1.y, a0);
      a1 = fma(c1[0], (T)y0.x, a1);
      a1 = fma(c1[1], (T)y0.y, a1);
      a1 = fma(c1[2], (T)y1.x, a1);
      a1 = fma(c1[3], (T)y1.y, a1);
    }
    for (; q < qstop; q += 32) {
      T c0[4];
      load4<T>(col + 4 * q, c0);
      const double2 *vv0 = reinterpret_cast<const double2 *>(v + 4 * q);
      const double2 x0 = vv0[0], x1 = vv0[1];
      a0 = fma(c0[0], (T)x0.x, a0);
      a0 = fma(c0[1], (T)x0.y, a0);
      a0 = fma(c0[2], (T)x1.x, a0);
      a0 = fma(c0[3], (T)x1.y, a0);
    }
    acc += (double)(a0 + a1);
  }
  for (int i = hb + lane; i < hi; i += 32) acc = fma((double)col[i], v[i], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) w[j] = beta == 0.0 ? alpha * acc : fma(alpha, acc, beta * w[j]);
}

template <class T>
void dotcols(const T *A, int64_t ld, int ncol, int len, int range, const double *v, double *w,
             double alpha, double beta, cudaStream_t st) {
  if (ncol <= 0) return;
  const bool aligned = ((uintptr_t)A % 16 == 0) && ((ld * (int64_t)sizeof(T)) % 16 == 0) &&
                       ((uintptr_t)v % 16 == 0);
  if (aligned)
    k_dotcols_v4<T><<<(ncol + 7) / 8, 256, 0, st>>>(A, ld, ncol, len, range, v, w, alpha, beta);
  else
    k_dotcols<T><<<(ncol + 7) / 8, 256, 0, st>>>(A, ld, ncol, len, range, v, w, alpha, beta);
}

// ---------------------------------------------------------------------------------------------
// Lanczos vector kernels (one CTA; the vectors are short: n <= a few tens of thousands)
// out[0] = sum_i x_i y_i (fixed order: per-thread strided sums, then a tree)
__device__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One three-term step.  w holds op(v_j) (already in place).  s[2j] = alpha_j = <w, v_j>_G with
// Gw given as gw (G = I: gw = w), then w -= alpha_j v_j + beta_{j-1} v_{j-1}.
__global__ void k_lz_alpha(int n, double *w, const double *__restrict__ gvj,
                           const double *__restrict__ vj, const double *__restrict__ vjm1,
                           double *s, int j) {
  __shared__ double red[32];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a = fma(w[i], gvj[i], a);
  a = block_sum(a, red);
  __shared__ double sa;
  if (threadIdx.x == 0) {
    sa = a;
    s[2 * j] = a;
  }
  __syncthreads();
  const double b = j > 0 ? s[2 * j - 1] : 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double x = w[i] - sa * vj[i];
    if (j > 0) x -= b * vjm1[i];
    w[i] = x;
  }
}

// full reorthogonalisation against v_0 .. v_{jcount-1}: h_c = <Qd_c, w>, w -= sum_c h_c Q_c
// (Qd = G Q for the G-inner product, Q itself for the Euclidean one)
__global__ void k_lz_reorth(int n, int jcount, double *w, const double *__restrict__ Qd,
                            const double *__restrict__ Q) {
  __shared__ double red[32];
  __shared__ double h[128];
  for (int c = 0; c < jcount; ++c) {
    double a = 0.0;
    const double *q = Qd + (int64_t)c * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) a = fma(q[i], w[i], a);
    a = block_sum(a, red);
    if (threadIdx.x == 0) h[c] = a;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double x = w[i];
    for (int c = 0; c < jcount; ++c) x -= h[c] * Q[(int64_t)c * n + i];
    w[i] = x;
  }
}

// beta_j = sqrt(<w, w>_G) (gw = G w), s[2j+1] = beta_j, v_{j+1} = w / beta_j and
// G v_{j+1} = gw / beta_j (gvnext may alias nothing else; both 0 if beta_j = 0)
__global__ void k_lz_beta(int n, const double *__restrict__ w, const double *__restrict__ gw,
                          double *vnext, double *gvnext, double *s, int j) {
  __shared__ double red[32];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a = fma(w[i], gw[i], a);
  a = block_sum(a, red);
  __shared__ double sb;
  if (threadIdx.x == 0) {
    sb = sqrt(fmax(a, 0.0));
    s[2 * j + 1] = sb;
  }
  __syncthreads();
  const double inv = sb > 0.0 ? 1.0 / sb : 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    vnext[i] = w[i] * inv;
    if (gvnext) gvnext[i] = gw[i] * inv;
  }
}

// v <- v / sqrt(<v, v>_G), and gv = G v likewise (gv may be v itself)
__global__ void k_lz_normalise(int n, double *v, double *gv) {
  __shared__ double red[32];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a = fma(v[i], gv[i], a);
  a = block_sum(a, red);
  __shared__ double sc;
  if (threadIdx.x == 0) sc = a > 0.0 ? 1.0 / sqrt(a) : 0.0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    v[i] *= sc;
    if (gv != v) gv[i] *= sc;
  }
}

void lz_alpha(int n, double *w, const double *gvj, const double *vj, const double *vjm1,
              double *s, int j, cudaStream_t st) {
  k_lz_alpha<<<1, 1024, 0, st>>>(n, w, gvj, vj, vjm1, s, j);
}
// h_c = <Qd_c, w> (one CTA per c), then w -= sum_c h_c Q_c (grid-stride): the reorthogonalisation
// spread over the SMs
__global__ void k_lz_dots(int n, const double *__restrict__ w, const double *__restrict__ Qd,
                          double *h) {
  __shared__ double red[32];
  const int c = blockIdx.x;
  const double *q = Qd + (int64_t)c * n;
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a = fma(q[i], w[i], a);
  a = block_sum(a, red);
  if (threadIdx.x == 0) h[c] = a;
}
__global__ void k_lz_sub(int n, int jcount, double *w, const double *__restrict__ Q,
                         const double *__restrict__ h) {
  __shared__ double hs[128];
  for (int c = threadIdx.x; c < jcount; c += blockDim.x) hs[c] = h[c];
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double x = w[i];
    for (int c = 0; c < jcount; ++c) x -= hs[c] * Q[(int64_t)c * n + i];
    w[i] = x;
  }
}
void lz_reorth(int n, int jcount, double *w, const double *Qd, const double *Q, double *h,
               cudaStream_t st) {
  k_lz_dots<<<jcount, 512, 0, st>>>(n, w, Qd, h);
  k_lz_sub<<<(n + 255) / 256, 256, 0, st>>>(n, jcount, w, Q, h);
}
void lz_sub(int n, int jcount, double *w, const double *Q, const double *h, cudaStream_t st) {
  k_lz_sub<<<(n + 255) / 256, 256, 0, st>>>(n, jcount, w, Q, h);
}
void lz_beta(int n, const double *w, const double *gw, double *vnext, double *gvnext, double *s,
             int j, cudaStream_t st) {
  k_lz_beta<<<1, 1024, 0, st>>>(n, w, gw, vnext, gvnext, s, j);
}
void lz_normalise(int n, double *v, double *gv, cudaStream_t st) {
  k_lz_normalise<<<1, 1024, 0, st>>>(n, v, gv);
}

// lower triangle of a column-major square copied, the strict upper triangle of dst set to zero
__global__ void k_copy_lower(const double *__restrict__ src, int64_t lds, double *dst, int64_t ldd,
                             int n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    dst[i + (int64_t)j * ldd] = i >= j ? src[i + (int64_t)j * lds] : 0.0;
  }
}
void copy_lower(const double *src, int64_t lds, double *dst, int64_t ldd, int n, cudaStream_t st) {
  if (n <= 0) return;
  const int blocks = (int)std::min<int64_t>(4096, ((int64_t)n * n + 255) / 256);
  k_copy_lower<<<blocks, 256, 0, st>>>(src, lds, dst, ldd, n);
}

// ---------------------------------------------------------------------------------------------
// Dense completion buffers (row-major n x ldw, column of vertex k at colw[k]; the root's
// vertices occupy the first |R| columns)

// W[i][colw[k]] = 1 for the rhs-th unit column k = k0 + rhs of the forest
template <class T>
__global__ void k_unit_cols(T *W, int64_t ldw, const int *__restrict__ colw, int k0, int nk) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < nk) W[(int64_t)(k0 + r) * ldw + colw[k0 + r]] = T(1);
}

// rows of the root, forest columns: W[rbase + i][colw[t]] = W[t][i] for t < nF, i < nR
// (X̂_{R,t} = X̂_{t,R}^T, the symmetry of the completed matrix)
template <class T>
__global__ void k_root_rows_from_cols(T *W, int64_t ldw, const int *__restrict__ colw, int nR,
                                      int nF) {
  __shared__ T tile[32][33];
  const int t0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int t = t0 + r, i = i0 + tx;
    tile[r][tx] = (t < nF && i < nR) ? W[(int64_t)t * ldw + i] : T(0);
  }
  __syncthreads();
  const int rbase = nF;
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + r, t = t0 + tx;
    if (t < nF && i < nR) W[(int64_t)(rbase + i) * ldw + colw[t]] = tile[tx][r];
  }
}

// lower(E) values of a dense completed matrix: outE at every layout entry (row r, column k of
// supernode s, r >= k) = W[r][colw[k]]; root block included (the root occupies columns
// [0, nR) and rows [nF, n))
template <class T>
__global__ void k_extract_dense(DevSym S, const T *__restrict__ W, int64_t ldw,
                                const int *__restrict__ colw, double *outE) {
  const int s = blockIdx.y;
  const int64_t r0 = S.sn_rowptr[s];
  const int nrow = (int)(S.sn_rowptr[s + 1] - r0);
  const int c0 = S.sn_col[s], ncol = S.sn_col[s + 1] - c0;
  const int64_t v0 = S.sn_valptr[s];
  const int64_t cnt = (int64_t)nrow * ncol;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < cnt;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(e % nrow), lc = (int)(e / nrow);
    if (p < lc) continue;
    outE[v0 + e] = (double)W[(int64_t)S.rows[r0 + p] * ldw + colw[c0 + lc]];
  }
}

// V[i][colw[b]] = sum_a W[i][colw[a]] D_ab on the aggregate pattern (V = W D, D symmetric held
// on the layout at the aggregate positions), thread per (row i, column b)
template <class T>
__global__ void k_times_pattern(DevSym S, const double *__restrict__ D, const T *__restrict__ W,
                                T *V, int64_t ldw, const int *__restrict__ colw) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= S.n) return;
  for (int i = blockIdx.y; i < S.n; i += gridDim.y) {
    const T *wr = W + (int64_t)i * ldw;
    T acc = T(0);
    for (int q = S.arow_ptr[b]; q < S.arow_ptr[b + 1]; ++q)
      acc = fma((T)D[S.arow_off[q]], wr[colw[S.arow_col[q]]], acc);
    V[(int64_t)i * ldw + colw[b]] = acc;
  }
}

// M = X̂ D Y^{-1} on the forest's layout entries from the rows of V = X̂ D and of Wy = Y^{-1}:
// Mlow at (r, k) = V[r] . Wy[k], Mup at (r, k) = V[k] . Wy[r] (rows dotted over all columns);
// one CTA per forest supernode, the clique's rows staged in chunks of columns
template <class T>
__global__ void __launch_bounds__(256) k_forest_M(DevSym S, const T *__restrict__ V,
                                                  const T *__restrict__ Wy, int64_t ldw,
                                                  int ncolw, double *Mlow, double *Mup) {
  constexpr int CH = 32, PER = 8, LDS = CH + 1;  // rows padded: threads of a warp take
                                                  // consecutive rows p, so an unpadded stride
                                                  // of 32 would put them in one bank
  extern __shared__ __align__(16) unsigned char smf[];
  const int s = blockIdx.x;
  const int64_t r0 = S.sn_rowptr[s];
  const int nrow = (int)(S.sn_rowptr[s + 1] - r0);
  const int ncol = S.sn_col[s + 1] - S.sn_col[s];
  const int64_t v0 = S.sn_valptr[s];
  T *Vs = reinterpret_cast<T *>(smf);  // [nrow][LDS]
  T *Ys = Vs + nrow * LDS;              // [nrow][LDS]
  int *rw = reinterpret_cast<int *>(Ys + nrow * LDS);
  const int tid = threadIdx.x;
  for (int p = tid; p < nrow; p += blockDim.x) rw[p] = S.rows[r0 + p];
  const int nout = nrow * ncol;
  __syncthreads();
  // outputs in passes of 256 x PER; each thread keeps the lower and upper sums of PER of them
  // sums in T per chunk (FP32 in the mixed form: FP64 arithmetic would run on the slow FP64
  // pipe), carried across chunks in FP64
  for (int pass = 0; pass * 256 * PER < nout; ++pass) {
    double lo[PER], up[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) lo[q] = up[q] = 0.0;
    for (int c0 = 0; c0 < ncolw; c0 += CH) {
      for (int e = tid; e < nrow * CH; e += blockDim.x) {
        const int p = e / CH, c = e % CH;
        const int64_t o = (int64_t)rw[p] * ldw + c0 + c;
        const bool in = c0 + c < ncolw;
        Vs[p * LDS + c] = in ? V[o] : T(0);
        Ys[p * LDS + c] = in ? Wy[o] : T(0);
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int e = pass * 256 * PER + tid + q * 256;
        if (e >= nout) break;
        const int p = e % nrow, lc = e / nrow;
        if (p < lc) continue;
        const T *vp = Vs + p * LDS, *yl = Ys + lc * LDS, *vl = Vs + lc * LDS, *yp = Ys + p * LDS;
        T a = T(0), b = T(0);
#pragma unroll 8
        for (int c = 0; c < CH; ++c) {
          a = fma(vp[c], yl[c], a);
          b = fma(vl[c], yp[c], b);
        }
        lo[q] += (double)a;
        up[q] += (double)b;
      }
      __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = pass * 256 * PER + tid + q * 256;
      if (e >= nout) break;
      const int p = e % nrow, lc = e / nrow;
      if (p < lc) continue;
      Mlow[v0 + e] = lo[q];
      Mup[v0 + e] = up[q];
    }
  }
}

// the root block's Mlow / Mup from the dense product M_RR (column-major, ld nR)
template <class T>
__global__ void k_root_M(const T *__restrict__ M, int nR, double *Mlow, double *Mup) {
  const int64_t cnt = (int64_t)nR * nR;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < cnt;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % nR), j = (int)(e / nR);
    if (i < j) continue;
    Mlow[e] = (double)M[e];
    Mup[e] = (double)M[j + (int64_t)i * nR];
  }
}

// dX on the root block (lower part; the upper part zero): beta mu Y^{-1} - X̄ - sym(M)
__global__ void k_root_dx(int nR, double betamu, const double *__restrict__ X,
                          const double *__restrict__ YinvE, const double *__restrict__ Mlow,
                          const double *__restrict__ Mup, double *dX) {
  const int64_t cnt = (int64_t)nR * nR;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < cnt;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % nR), j = (int)(e / nR);
    double v;
    if (i < j) v = 0.0;
    else if (i == j) v = betamu * YinvE[e] - X[e] - Mlow[e];
    else v = betamu * YinvE[e] - X[e] - 0.5 * (Mlow[e] + Mup[e]);
    dX[e] = v;
  }
}

// Root block of the P-MATRIX: with X̂_FR = -L_FF^{-T} L_RF^T X̂_RR (the completion's forest
// rows of the root columns, X̂^{-1} = L̂ L̂^T), (X̂ U)_RR = X̂_RR U_RR + X̂_RF U_FR
// = X̂_RR (U_RR - L_RF L_FF^{-1} U_F) for any U.  One CTA per tile of 32 root rows x 32 columns:
// a warp takes a root row at a time, lane = column, the row's L_RF entries broadcast; the tile
// is transposed through shared memory.  Column tiles vary slowest across the grid, so the CTAs
// resident together read one 32-column slice of Z (n_F x 32 values), which stays in L2.
template <class T>
__global__ void __launch_bounds__(256) k_root_pull(const int64_t *__restrict__ ptr,
                                                   const int64_t *__restrict__ off,
                                                   const int *__restrict__ frow,
                                                   const T *__restrict__ L,
                                                   const T *__restrict__ U, int64_t ldw, int nF,
                                                   int nR, T *Tt) {
  __shared__ T tile[32][33];
  const int r0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int j = j0 + lane;
  for (int rr = w; rr < 32; rr += 8) {
    const int r = r0 + rr;
    T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
    if (r < nR && j < nR) {
      a0 = U[(int64_t)(nF + r) * ldw + j];
      int64_t e = ptr[r];
      const int64_t e1 = ptr[r + 1];
      for (; e + 4 <= e1; e += 4) {  // four independent chains
        a0 = fma(-L[off[e]], U[(int64_t)frow[e] * ldw + j], a0);
        a1 = fma(-L[off[e + 1]], U[(int64_t)frow[e + 1] * ldw + j], a1);
        a2 = fma(-L[off[e + 2]], U[(int64_t)frow[e + 2] * ldw + j], a2);
        a3 = fma(-L[off[e + 3]], U[(int64_t)frow[e + 3] * ldw + j], a3);
      }
      for (; e < e1; ++e) a0 = fma(-L[off[e]], U[(int64_t)frow[e] * ldw + j], a0);
    }
    tile[rr][lane] = (a0 + a1) + (a2 + a3);
  }
  __syncthreads();
  for (int jj = w; jj < 32; jj += 8) {
    const int jo = j0 + jj, r = r0 + lane;
    if (jo < nR && r < nR) Tt[(int64_t)jo * nR + r] = tile[lane][jj];
  }
}

template <class T>
void launch_root_pull(const int64_t *ptr, const int64_t *off, const int *frow, const T *L,
                      const T *U, int64_t ldw, int nF, int nR, T *Tt, cudaStream_t st) {
  if (nR <= 0) return;
  dim3 grid((nR + 31) / 32, (nR + 31) / 32);
  k_root_pull<T><<<grid, 256, 0, st>>>(ptr, off, frow, L, U, ldw, nF, nR, Tt);
}

// range of the pivots of a Cholesky factor in the layout: out[0] = max_j |L_jj|, out[1] =
// min_j |L_jj| (one CTA; (max/min)^2 is a lower bound on the condition number of L L^T)
__global__ void k_diag_range(DevSym S, const double *__restrict__ L, double *out) {
  __shared__ double smax[32], smin[32];
  double mx = 0.0, mn = 1.0e300;
  for (int j = threadIdx.x; j < S.n; j += blockDim.x) {
    const int t = S.col2sn[j];
    const int64_t nrow = S.sn_rowptr[t + 1] - S.sn_rowptr[t];
    const int lc = j - S.sn_col[t];
    const double v = fabs(L[S.sn_valptr[t] + lc + (int64_t)lc * nrow]);
    mx = fmax(mx, v);
    mn = fmin(mn, v);
  }
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    smax[w] = mx;
    smin[w] = mn;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
      mx = fmax(mx, smax[q]);
      mn = fmin(mn, smin[q]);
    }
    out[0] = mx;
    out[1] = mn;
  }
}

void launch_diag_range(const DevSym &S, const double *L, double *out, cudaStream_t st) {
  k_diag_range<<<1, 1024, 0, st>>>(S, L, out);
}

__global__ void k_cast_f64(const float *__restrict__ a, double *b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}
void cast_f64(const float *a, double *b, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  const int blocks = (int)std::min<int64_t>(4096, (n + 255) / 256);
  k_cast_f64<<<blocks, 256, 0, st>>>(a, b, n);
}

template <class T>
void launch_unit_cols(T *W, int64_t ldw, const int *colw, int k0, int nk, cudaStream_t st) {
  if (nk > 0) k_unit_cols<T><<<(nk + 255) / 256, 256, 0, st>>>(W, ldw, colw, k0, nk);
}
template <class T>
void launch_root_rows_from_cols(T *W, int64_t ldw, const int *colw, int nR, int nF, cudaStream_t st) {
  if (nR <= 0 || nF <= 0) return;
  dim3 grid((nF + 31) / 32, (nR + 31) / 32), blk(32, 8);
  k_root_rows_from_cols<T><<<grid, blk, 0, st>>>(W, ldw, colw, nR, nF);
}
template <class T>
void launch_extract_dense(const DevSym &S, const T *W, int64_t ldw, const int *colw, double *outE,
                          cudaStream_t st) {
  // forest supernodes: one CTA each; the root block: many
  if (S.nforest > 0) k_extract_dense<T><<<dim3(1, S.nforest), 256, 0, st>>>(S, W, ldw, colw, outE);
  if (S.nR > 0) {
    DevSym R = S;
    // the root alone: shift the supernode index by launching with blockIdx.y = 0 on s = ns - 1
    R.sn_rowptr = S.sn_rowptr + (S.ns - 1);
    R.sn_col = S.sn_col + (S.ns - 1);
    R.sn_valptr = S.sn_valptr + (S.ns - 1);
    const int blocks = (int)std::min<int64_t>(4096, ((int64_t)S.nR * S.nR + 255) / 256);
    k_extract_dense<T><<<dim3(blocks, 1), 256, 0, st>>>(R, W, ldw, colw, outE);
  }
}
// V[i][colw[b]] = W[i][colw[b]] d_b for a diagonal D (d_b = D at the diagonal position of b):
// one pass over W
template <class T>
__global__ void k_times_diag(const T *__restrict__ W, T *V, int64_t ldw, const T *__restrict__ dcol,
                             int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    V[e] = W[e] * dcol[e % ldw];
}
// dcol[colw[b]] = D at (b, b) (0 at padding columns)
__global__ void k_diag_to_cols(DevSym S, const double *__restrict__ D, const int *__restrict__ colw,
                               int64_t *diag_off, void *dcol, int fp32) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= S.n) return;
  const int t = S.col2sn[b];
  const int nrow = (int)(S.sn_rowptr[t + 1] - S.sn_rowptr[t]);
  const int lc = b - S.sn_col[t];
  const double v = D[S.sn_valptr[t] + lc + (int64_t)lc * nrow];
  if (fp32) static_cast<float *>(dcol)[colw[b]] = (float)v;
  else static_cast<double *>(dcol)[colw[b]] = v;
  (void)diag_off;
}

template <class T>
void launch_times_diag(const DevSym &S, const double *D, const T *W, T *V, int64_t ldw,
                       const int *colw, T *dcol, cudaStream_t st) {
  cudaMemsetAsync(dcol, 0, ldw * sizeof(T), st);
  k_diag_to_cols<<<(S.n + 255) / 256, 256, 0, st>>>(S, D, colw, nullptr, dcol,
                                                    std::is_same<T, float>::value ? 1 : 0);
  const int64_t total = (int64_t)S.n * ldw;
  const int blocks = (int)std::min<int64_t>(152 * 16, (total + 255) / 256);
  k_times_diag<T><<<blocks, 256, 0, st>>>(W, V, ldw, dcol, total);
}

template <class T>
void launch_times_pattern(const DevSym &S, const double *D, const T *W, T *V, int64_t ldw,
                          const int *colw, cudaStream_t st) {
  dim3 grid((S.n + 127) / 128, std::min(S.n, 65535));
  k_times_pattern<T><<<grid, 128, 0, st>>>(S, D, W, V, ldw, colw);
}
template <class T>
size_t forest_M_smem(const DevSym &S) {
  return (size_t)2 * S.max_nrow * 33 * sizeof(T) + (size_t)S.max_nrow * 4 + 16;
}
template <class T>
void launch_forest_M(const DevSym &S, const T *V, const T *Wy, int64_t ldw, int ncolw,
                     double *Mlow, double *Mup, cudaStream_t st) {
  if (S.nforest <= 0) return;
  const size_t smem = forest_M_smem<T>(S);
  smem_optin((const void *)k_forest_M<T>);
  k_forest_M<T><<<S.nforest, 256, smem, st>>>(S, V, Wy, ldw, ncolw, Mlow, Mup);
}
template <class T>
void launch_root_M(const T *M, int nR, double *Mlow_root, double *Mup_root, cudaStream_t st) {
  if (nR <= 0) return;
  const int blocks = (int)std::min<int64_t>(4096, ((int64_t)nR * nR + 255) / 256);
  k_root_M<T><<<blocks, 256, 0, st>>>(M, nR, Mlow_root, Mup_root);
}
void launch_root_dx(int nR, double betamu, const double *X, const double *YinvE, const double *Mlow,
                    const double *Mup, double *dX, cudaStream_t st) {
  if (nR <= 0) return;
  const int blocks = (int)std::min<int64_t>(4096, ((int64_t)nR * nR + 255) / 256);
  k_root_dx<<<blocks, 256, 0, st>>>(nR, betamu, X, YinvE, Mlow, Mup, dX);
}

template <class T>
__global__ void k_mirror_lower(T *A, int64_t ld, int n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    if (i > j) A[j + (int64_t)i * ld] = A[i + (int64_t)j * ld];
  }
}

template <class T>
void mirror_lower(T *A, int64_t ld, int n, cudaStream_t st) {
  if (n <= 0) return;
  const int blocks = (int)std::min<int64_t>(4096, ((int64_t)n * n + 255) / 256);
  k_mirror_lower<T><<<blocks, 256, 0, st>>>(A, ld, n);
}

// SplitMix64 finaliser of (seed, i): a fixed start vector for the Lanczos iterations
__global__ void k_fill_hash(double *v, int n, unsigned seed) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    unsigned long long z = ((unsigned long long)seed << 32) + (unsigned long long)i + 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    v[i] = (double)(z >> 11) * 0x1.0p-52 - 1.0;
  }
}
void fill_hash(double *v, int n, unsigned seed, cudaStream_t st) {
  if (n > 0) k_fill_hash<<<(n + 255) / 256, 256, 0, st>>>(v, n, seed);
}

__global__ void k_permute_to_cols(const double *__restrict__ src, const int *__restrict__ colw,
                                  double *dst, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) dst[colw[k]] = src[k];
}
void permute_to_cols(const double *src, const int *colw, double *dst, int n, cudaStream_t st) {
  if (n > 0) k_permute_to_cols<<<(n + 255) / 256, 256, 0, st>>>(src, colw, dst, n);
}

#define MCSDP_ROOT_INST(T)                                                                       \
  template void gemm_tn<T>(const GemmArgs<T> &, cudaStream_t, bool);                             \
  template int dense_trtri<T>(const T *, int64_t, const T *, T *, int64_t, int, T *, cudaStream_t); \
  template int dense_lauum<T>(const T *, int64_t, int, T *, int64_t, int64_t, bool, cudaStream_t); \
  template void dotcols<T>(const T *, int64_t, int, int, int, const double *, double *, double,  \
                           double, cudaStream_t);                                                \
  template void launch_unit_cols<T>(T *, int64_t, const int *, int, int, cudaStream_t);          \
  template void launch_root_rows_from_cols<T>(T *, int64_t, const int *, int, int, cudaStream_t); \
  template void launch_extract_dense<T>(const DevSym &, const T *, int64_t, const int *, double *, \
                                        cudaStream_t);                                           \
  template void launch_times_pattern<T>(const DevSym &, const double *, const T *, T *, int64_t,  \
                                        const int *, cudaStream_t);                              \
  template void launch_times_diag<T>(const DevSym &, const double *, const T *, T *, int64_t,     \
                                     const int *, T *, cudaStream_t);                            \
  template void launch_forest_M<T>(const DevSym &, const T *, const T *, int64_t, int, double *,  \
                                   double *, cudaStream_t);                                      \
  template void launch_root_M<T>(const T *, int, double *, double *, cudaStream_t);        \
  template void launch_root_pull<T>(const int64_t *, const int64_t *, const int *, const T *,     \
                                    const T *, int64_t, int, int, T *, cudaStream_t);          \
  template void mirror_lower<T>(T *, int64_t, int, cudaStream_t);
MCSDP_ROOT_INST(double)
MCSDP_ROOT_INST(float)
#undef MCSDP_ROOT_INST
template void copy_square<double, double>(const double *, int64_t, double *, int64_t, int, cudaStream_t);
template void copy_square<double, float>(const double *, int64_t, float *, int64_t, int, cudaStream_t);
template void copy_square<float, double>(const float *, int64_t, double *, int64_t, int, cudaStream_t);
template void symmetrize<double, double>(const double *, int64_t, double *, int64_t, int, cudaStream_t);
template void symmetrize<double, float>(const double *, int64_t, float *, int64_t, int, cudaStream_t);

}  // namespace mcsdp
