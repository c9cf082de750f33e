// FP32 products on the fifth-generation tensor cores (tcgen05, kind::tf32) for the mixed form's
// dense contractions: the trailing updates of the SCM Cholesky (Sec. 3.1, computation type (i),
// the one dense contraction of the method) and of the dense root's products.
//
// An FP32 operand a is carried as two TF32 numbers, a_hi = tf32(a) and a_lo = tf32(a - a_hi)
// (both rounded to nearest, the low 13 mantissa bits zero); a b = a_hi b_hi + a_hi b_lo +
// a_lo b_hi up to a_lo b_lo (relative 2^-22) and the TF32 rounding of the lo parts, so three
// TF32 products with FP32 accumulation in tensor memory give FP32-level accuracy.
//
// C(i, j) = alpha sum_l A(l, i) B(l, j) + beta C(i, j): A and B K-major (row i of the operand is
// K contiguous values), reached through 2-D TMA tensor maps (inner dimension K, outer the rows);
// one CTA per 128 x 128 tile of C, K in blocks of 32 (one 128-byte swizzle atom per row) through a
// three-stage shared-memory ring: warp 0 issues the TMA loads, warp 1 the MMAs (one thread each),
// then all four warps read the accumulator rows from tensor memory (warp w owns lanes 32w..) and
// update C.  Every wait on an mbarrier is bounded: a wait that runs out sets the error word,
// and the CTA drains what it issued before releasing tensor memory.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <algorithm>
#include <mutex>

#include "../../include/mcsdp.h"
#include "internal.h"
#include "tc.h"

namespace mcsdp {

constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 32;
constexpr int TC_STAGES = 3;
constexpr int TC_TILE_BYTES = TC_BM * TC_BK * 4;     // 16 KiB: 128 rows x 128 bytes
constexpr int TC_STAGE_BYTES = 4 * TC_TILE_BYTES;    // A_hi, A_lo, B_hi, B_lo
constexpr int TC_SMEM = TC_STAGES * TC_STAGE_BYTES + 1024 + 256;
constexpr long long TC_WAIT_POLLS = 1ll << 26;       // bounded mbarrier waits (seconds)

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)),
               "r"(bytes)
               : "memory");
}

// waits for the phase with the given parity to complete; false if the poll budget ran out
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity) {
  const uint32_t a = smem_u32(b);
  for (long long it = 0; it < TC_WAIT_POLLS; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (it > 64) __nanosleep(64);
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
      "{%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// shared-memory matrix descriptor: K-major operand tile, 128-byte swizzle (8-row atoms of 1 KiB
// stacked at 1 KiB), start address advanced by 32 bytes per K step of the MMA
__device__ __forceinline__ uint64_t smem_desc_sw128(const void *p) {
  const uint64_t addr = smem_u32(p);
  uint64_t d = 0;
  d |= (addr >> 4) & 0x3FFFull;                 // start address
  d |= (uint64_t)1 << 16;                        // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;              // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                        // descriptor version
  d |= (uint64_t)2 << 61;                        // 128-byte swizzle
  return d;
}

// instruction descriptor of kind::tf32: D F32, A and B TF32, both K-major, M = 128, N = 128
__host__ __device__ constexpr uint32_t tc_idesc() {
  return (1u << 4)                  // D format: F32
         | (2u << 7)                // A format: TF32
         | (2u << 10)               // B format: TF32
         | ((uint32_t)(TC_BN >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
      "l"(adesc), "l"(bdesc), "r"(tc_idesc()), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

struct TcArgs {
  int M, N, K;            // C is M x N; K summed
  int ax, ay, bx, by;     // tensor-map coordinates of A's / B's first element (x = K, y = row)
  float *C;
  int64_t cs_i, cs_j;     // C(i, j) at C[i cs_i + j cs_j]
  float alpha, beta;
  int lower, mirror;      // lower: tiles and entries with i >= j only; mirror: C(j, i) too
  int *err;               // error word (ST_TIMEOUT)
};

__global__ void __launch_bounds__(128, 1)
    k_gemm_3xtf32(const __grid_constant__ CUtensorMap tAh, const __grid_constant__ CUtensorMap tAl,
                  const __grid_constant__ CUtensorMap tBh, const __grid_constant__ CUtensorMap tBl,
                  TcArgs g) {
  extern __shared__ uint8_t tc_raw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t *full = reinterpret_cast<uint64_t *>(sm + TC_STAGES * TC_STAGE_BYTES);
  uint64_t *empty = full + TC_STAGES;
  uint64_t *done = empty + TC_STAGES;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
  int *abort_flag = reinterpret_cast<int *>(tslot + 1);
  const int i0 = blockIdx.x * TC_BM, j0 = blockIdx.y * TC_BN;
  if (g.lower && i0 + TC_BM - 1 < j0) return;  // whole CTA, before any barrier or allocation
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkb = (g.K + TC_BK - 1) / TC_BK;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(TC_BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  int issued = 0;  // producer: K blocks whose loads were issued
  if (warp == 0 && lane == 0) {
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % TC_STAGES;
      const uint32_t ph = (uint32_t)(kb / TC_STAGES) & 1u;
      if (!mbar_wait(empty + s, ph ^ 1u)) {
        atomicOr(g.err, ST_TIMEOUT);
        atomicExch(abort_flag, 1);
        break;
      }
      if (*(volatile int *)abort_flag) break;
      uint8_t *st = sm + s * TC_STAGE_BYTES;
      mbar_expect_tx(full + s, TC_STAGE_BYTES);
      const int kx = kb * TC_BK;
      tma_load_2d(st, &tAh, g.ax + kx, g.ay + i0, full + s);
      tma_load_2d(st + TC_TILE_BYTES, &tAl, g.ax + kx, g.ay + i0, full + s);
      tma_load_2d(st + 2 * TC_TILE_BYTES, &tBh, g.bx + kx, g.by + j0, full + s);
      tma_load_2d(st + 3 * TC_TILE_BYTES, &tBl, g.bx + kx, g.by + j0, full + s);
      issued = kb + 1;
    }
  } else if (warp == 1 && lane == 0) {
    int kb = 0;
    for (; kb < nkb; ++kb) {
      const int s = kb % TC_STAGES;
      const uint32_t ph = (uint32_t)(kb / TC_STAGES) & 1u;
      if (!mbar_wait(full + s, ph)) {
        atomicOr(g.err, ST_TIMEOUT);
        atomicExch(abort_flag, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint8_t *st = sm + s * TC_STAGE_BYTES;
      const uint64_t ah = smem_desc_sw128(st), al = smem_desc_sw128(st + TC_TILE_BYTES);
      const uint64_t bh = smem_desc_sw128(st + 2 * TC_TILE_BYTES);
      const uint64_t bl = smem_desc_sw128(st + 3 * TC_TILE_BYTES);
#pragma unroll
      for (int k = 0; k < TC_BK / 8; ++k) {
        const uint64_t adv = (uint64_t)((k * 32) >> 4);  // 8 TF32 values = 32 bytes along K
        mma_tf32(tmem, ah + adv, bh + adv, (kb | k) != 0);
        mma_tf32(tmem, ah + adv, bl + adv, 1u);
        mma_tf32(tmem, al + adv, bh + adv, 1u);
      }
      mma_commit(empty + s);  // the stage's buffers are free once these MMAs complete
    }
    mma_commit(done);  // every MMA issued so far complete
  }
  // epilogue: the accumulator rows of this warp's 32 lanes
  __syncwarp();
  const bool ok = mbar_wait(done, 0);
  if (!ok) atomicOr(g.err, ST_TIMEOUT);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool skip = !ok || *(volatile int *)abort_flag;
  const int i = i0 + warp * 32 + lane;
  for (int c0 = 0; c0 < TC_BN; c0 += 32) {
    uint32_t v[32];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
        "%30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
          "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
          "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (skip || i >= g.M) continue;
    // the 32 old values first (independent loads in flight), then the updates
    float old[32];
    if (g.beta != 0.f) {
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int j = j0 + c0 + q;
        old[q] = (j < g.N && !(g.lower && i < j))
                     ? __ldcg(g.C + (int64_t)i * g.cs_i + (int64_t)j * g.cs_j) : 0.f;
      }
    }
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      const int j = j0 + c0 + q;
      if (j >= g.N || (g.lower && i < j)) continue;
      const float a = __uint_as_float(v[q]);
      const float r = g.beta == 0.f ? g.alpha * a : fmaf(g.alpha, a, g.beta * old[q]);
      g.C[(int64_t)i * g.cs_i + (int64_t)j * g.cs_j] = r;
      if (g.mirror && i != j) g.C[(int64_t)j * g.cs_i + (int64_t)i * g.cs_j] = r;
    }
  }
  // the producer may have issued loads the MMA side never consumed (abort): wait for them
  if (warp == 0 && lane == 0 && skip) {
    for (int kb = 0; kb < issued; ++kb) {
      const int s = kb % TC_STAGES;
      (void)mbar_wait(full + s, (uint32_t)(kb / TC_STAGES) & 1u);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_BN)
                 : "memory");
}

// hi = tf32(a), lo = tf32(a - hi) (round to nearest), element (r, c) of a rows x cols matrix
// at a[r lda_r + c lda_c] into the K-major pair at hi/lo[c + r ldo] (row r, K index c); with tdst
// the value itself also goes to tdst[c + r tld]
__global__ void k_split_tf32(const float *__restrict__ a, int64_t lda_r, int64_t lda_c, int rows,
                            int cols, float *hi, float *lo, int64_t ldo, float *tdst, int64_t tld) {
  const int64_t cnt = (int64_t)rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < cnt;
       e += (int64_t)gridDim.x * blockDim.x) {
    int c, r;
    if (lda_r == 1) {  // column-major source: consecutive threads take consecutive rows
      r = (int)(e % rows);
      c = (int)(e / rows);
    } else {
      c = (int)(e % cols);
      r = (int)(e / cols);
    }
    const float x = a[r * lda_r + c * lda_c];
    uint32_t h, l;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    const float d = x - __uint_as_float(h);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(d));
    hi[c + r * ldo] = __uint_as_float(h);
    lo[c + r * ldo] = __uint_as_float(l);
    if (tdst) tdst[c + r * tld] = x;
  }
}

// the same for a column-major source (lda_r = 1), through 32 x 32 shared-memory tiles: reads run
// down the source's columns and the K-major writes (and the transposed copy) along the rows, both
// coalesced
__global__ void k_split_tf32_cm(const float *__restrict__ a, int64_t lda_c, int rows, int cols,
                                float *hi, float *lo, int64_t ldo, float *tdst, int64_t tld) {
  __shared__ float t[32][33];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int cc = ty; cc < 32; cc += 8) {
    const int r = r0 + tx, c = c0 + cc;
    t[cc][tx] = (r < rows && c < cols) ? a[r + (int64_t)c * lda_c] : 0.f;
  }
  __syncthreads();
  for (int rr = ty; rr < 32; rr += 8) {
    const int r = r0 + rr, c = c0 + tx;
    if (r >= rows || c >= cols) continue;
    const float x = t[tx][rr];
    uint32_t h, l;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    const float d = x - __uint_as_float(h);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(d));
    hi[c + (int64_t)r * ldo] = __uint_as_float(h);
    lo[c + (int64_t)r * ldo] = __uint_as_float(l);
    if (tdst) tdst[c + (int64_t)r * tld] = x;
  }
}

void split_tf32(const float *a, int64_t lda_r, int64_t lda_c, int rows, int cols, float *hi,
                float *lo, int64_t ldo, float *tdst, int64_t tld, cudaStream_t st) {
  const int64_t cnt = (int64_t)rows * cols;
  if (cnt <= 0) return;
  if (lda_r == 1 && cols <= 32 * 65535) {
    dim3 grid((rows + 31) / 32, (cols + 31) / 32), blk(32, 8);
    k_split_tf32_cm<<<grid, blk, 0, st>>>(a, lda_c, rows, cols, hi, lo, ldo, tdst, tld);
    return;
  }
  const int blocks = (int)std::min<int64_t>(8192, (cnt + 255) / 256);
  k_split_tf32<<<blocks, 256, 0, st>>>(a, lda_r, lda_c, rows, cols, hi, lo, ldo, tdst, tld);
}

namespace {
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}
}  // namespace

// 2-D tensor map of a K-major FP32 operand: rows x kdim values, row r at base + r ld (ld a
// multiple of 4, base 16-byte aligned), boxes of 32 (K) x 128 (rows), 128-byte swizzle, zero fill
// outside [0, kdim) x [0, rows)
bool make_tmap_kmajor(CUtensorMap *map, const float *base, int64_t ld, int64_t kdim, int64_t rows) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn || (ld % 4) != 0 || (reinterpret_cast<uintptr_t>(base) & 15) != 0) return false;
  cuuint64_t dims[2] = {(cuuint64_t)kdim, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)TC_BM};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides,
            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// C = alpha A^T B + beta C through the tensor maps (rows of A: the M index, rows of B: the N
// index; x, y the first element's coordinates)
void gemm_3xtf32(const TcOperand &A, const TcOperand &B, int M, int N, int K, float *C,
                 int64_t cs_i, int64_t cs_j, float alpha, float beta, bool lower, bool mirror,
                 int *err, cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0) return;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_gemm_3xtf32, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
  });
  TcArgs g{};
  g.M = M;
  g.N = N;
  g.K = K;
  g.ax = A.x;
  g.ay = A.y;
  g.bx = B.x;
  g.by = B.y;
  g.C = C;
  g.cs_i = cs_i;
  g.cs_j = cs_j;
  g.alpha = alpha;
  g.beta = beta;
  g.lower = lower ? 1 : 0;
  g.mirror = mirror ? 1 : 0;
  g.err = err;
  dim3 grid((M + TC_BM - 1) / TC_BM, (N + TC_BN - 1) / TC_BN);
  k_gemm_3xtf32<<<grid, 128, TC_SMEM, st>>>(A.hi, A.lo, B.hi, B.lo, g);
}

}  // namespace mcsdp

// ---------------------------------------------------------------------------------------------
// C ABI: the tensor-core FP32 product on its own (for its accuracy test and roofline)
extern "C" mcsdp_status mcsdp_gemm_tc_work_size(int32_t M, int32_t N, int32_t K, size_t *bytes) {
  if (M <= 0 || N <= 0 || K <= 0 || !bytes) return MCSDP_ERR_ARG;
  const int64_t kp = ((int64_t)K + 3) / 4 * 4;
  *bytes = (size_t)(2 * ((int64_t)M + N) * kp * 4) + 1024;
  return MCSDP_OK;
}

extern "C" mcsdp_status mcsdp_gemm_tc(int32_t M, int32_t N, int32_t K, const float *A, int64_t lda,
                                      const float *B, int64_t ldb, float *C, int64_t ldc,
                                      float alpha, float beta, void *work, size_t work_bytes,
                                      void *stream) {
  using namespace mcsdp;
  size_t need = 0;
  if (mcsdp_gemm_tc_work_size(M, N, K, &need) != MCSDP_OK || !A || !B || !C || !work ||
      lda < K || ldb < K || ldc < M || work_bytes < need ||
      (reinterpret_cast<uintptr_t>(work) & 255) != 0)
    return MCSDP_ERR_ARG;
  (void)cudaGetLastError();
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t kp = ((int64_t)K + 3) / 4 * 4;
  float *ah = static_cast<float *>(work), *al = ah + (size_t)M * kp;
  float *bh = al + (size_t)M * kp, *bl = bh + (size_t)N * kp;
  int *err = reinterpret_cast<int *>(bl + (size_t)N * kp);
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return MCSDP_ERR_CUDA;
  split_tf32(A, lda, 1, M, K, ah, al, kp, nullptr, 0, st);
  split_tf32(B, ldb, 1, N, K, bh, bl, kp, nullptr, 0, st);
  TcOperand oa, ob;
  oa.x = oa.y = ob.x = ob.y = 0;
  if (!make_tmap_kmajor(&oa.hi, ah, kp, K, M) || !make_tmap_kmajor(&oa.lo, al, kp, K, M) ||
      !make_tmap_kmajor(&ob.hi, bh, kp, K, N) || !make_tmap_kmajor(&ob.lo, bl, kp, K, N))
    return MCSDP_ERR_CUDA;
  gemm_3xtf32(oa, ob, M, N, K, C, 1, ldc, alpha, beta, false, false, err, st);
  if (cudaGetLastError() != cudaSuccess) return MCSDP_ERR_CUDA;
  int h = 0;
  if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return MCSDP_ERR_CUDA;
  return (h & ST_TIMEOUT) ? MCSDP_ERR_TIMEOUT : MCSDP_OK;
}
