/*
 * mcsdp.h — C ABI of libmcsdp, a single-GPU (sm_103a) implementation of the hot path of the
 * matrix-completion primal-dual interior-point method (MC-PDIPM) of Yamashita & Nakata,
 * "Fast implementation for semidefinite programs with positive matrix completion".
 *
 * Problem (Sec. 1, problems (P) and (D)):
 *     (P) min A_0 . X   s.t.  A_k . X = b_k (k = 1..m),  X psd
 *     (D) max b^T z     s.t.  sum_k A_k z_k + Y = A_0,    Y psd
 * X is kept only on the extended sparsity pattern E (a chordal extension of the aggregate
 * pattern, Sec. 2.1) as X̄; the max-determinant completion X̂ is reached through the factor of
 * its inverse X̂^{-1} = L̂ L̂^T (Algorithm 1, Sec. 3.1) and Y^{-1} through Y = N N^T.
 *
 * Conventions shared by every entry point
 *   - All sizes are in elements; indices are 0-based.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA global memory of the
 *     device the context was created on, valid for the context's stream.
 *   - The caller owns every pointer it passes; the library copies what it keeps and never frees
 *     caller memory.  Every call returns an mcsdp_status and never aborts the process;
 *     mcsdp_last_error() gives a one-line message for the last failing call on a context.
 *   - Work is issued on the stream given to mcsdp_create; calls that return host results
 *     synchronise that stream only (never the whole device).
 *   - "Layout" arrays hold one FP64 value per stored entry of the supernodal factor structure
 *     of E (nnz_layout entries, see mcsdp_sym_info): supernode s is a column-major block of
 *     nrow_s x ncol_s values (rows = the clique C_s in elimination order, columns = S_s);
 *     entries above the diagonal of the leading ncol_s x ncol_s block are unused and zero.
 *     X̄, Y, dX, L̂ and N all use this layout (the memory of L̂ equals that of N, Sec. 3.1).
 *   - Constraint vectors (b, z, dz, g) are in the caller's constraint order.
 *
 * A solve, in order of calls (error checks left out):
 *     mcsdp_problem p = {n, m, 1, b, nnz, mat, row, col, val};   // paper form, A_0 = mat 0
 *     mcsdp_ctx *ctx;  mcsdp_create(&p, NULL, stream, &ctx);      // validation, host analysis
 *     size_t bytes;    mcsdp_workspace_size(ctx, &bytes);
 *     void *ws;        cudaMalloc(&ws, bytes);                     // caller-owned device memory
 *     mcsdp_set_workspace(ctx, ws, bytes);                         // uploads the tables
 *     mcsdp_result r;  mcsdp_solve(ctx, &r);                       // r.pobj, r.dobj, r.gap ...
 *     mcsdp_get_iterate(ctx, Xbar_dev, z_dev, Y_dev);              // the final iterate
 *     mcsdp_destroy(ctx);  cudaFree(ws);
 */
#ifndef MCSDP_H
#define MCSDP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mcsdp_ctx mcsdp_ctx; /* opaque, library-owned */

typedef enum {
  MCSDP_OK = 0,
  MCSDP_ERR_ARG = 1,      /* invalid argument or input data */
  MCSDP_ERR_NOT_PD = 2,   /* a clique block of X̄, Y or the SCM is not positive definite */
  MCSDP_ERR_MAXITER = 3,  /* iteration limit reached before the stopping criterion */
  MCSDP_ERR_STALL = 4,    /* step lengths collapsed */
  MCSDP_ERR_NUMERIC = 5,  /* NaN or Inf met */
  MCSDP_ERR_CUDA = 6,     /* a CUDA call failed (message in mcsdp_last_error) */
  MCSDP_ERR_OOM = 7,      /* workspace too small / allocation failed */
  MCSDP_ERR_TIMEOUT = 8,  /* a bounded device wait gave up */
  MCSDP_ERR_STATE = 9     /* call not valid in the context's state (e.g. no workspace) */
} mcsdp_status;

/* Problem data, host memory, caller-owned.  One symmetric block of order n.
 * form = 0 (SDPA): entries of F_0..F_m with c (length m): the library solves the paper's (P)
 *        with A_0 = -F_0, A_k = F_k, b = c (SDPA's dual is the paper's primal; SDPA's x = -z).
 * form = 1 (paper): mat 0 is A_0 itself and c is b.
 * Entries are the upper triangle (row <= col) of each matrix; mat in [0, m]; duplicates of
 * (mat, row, col) and row > col are rejected with MCSDP_ERR_ARG. */
typedef struct {
  int32_t n, m;
  int32_t form;
  const double *c;   /* length m */
  int64_t nnz;
  const int32_t *mat, *row, *col;
  const double *val;
} mcsdp_problem;

/* Options; pass NULL for defaults.  The paper gives no parameter values ("default parameters",
 * Sec. 4); defaults: beta 0.1, gamma 0.9, gap_tol = feas_tol = 1e-7, max_iter 60.
 * device < 0 builds a host-only context: the symbolic analysis runs and can be exported, every
 * compute call returns MCSDP_ERR_STATE (used to test the host layer without a GPU). */
typedef struct {
  double beta, gamma, gap_tol, feas_tol;
  int32_t max_iter;
  int32_t precision;     /* 0 = FP64.  1 = mixed: the SCM solves and contraction (K3) and the
                            P-MATRIX solves (K6) run in FP32 from FP32 copies of L̂ and N; the
                            SCE B dz = g is solved with an FP32 Cholesky factor of B and FP64
                            iterative refinement against the stored B (for m >= 4096: the factor
                            of the diagonally equilibrated B, and GMRES preconditioned by it); Y's factor, Algorithm 1,
                            the step lengths and the update stay FP64 (with a dense root, see
                            mixed_asm_gap).  The solve promotes to
                            FP64 throughout once the relative gap falls below mixed_gap, the
                            refinement stalls, the FP32 factorisation breaks down or the primal
                            residual grows (m <= 50000). */
  int64_t timeout_cycles;/* bound on any device spin-wait, in SM clock cycles (the SCM
                          * factorisation's task dependencies); <= 0 = library default (2^32).
                          * A wait that runs out aborts the factorisation: the call returns
                          * MCSDP_ERR_TIMEOUT and the context stays usable */
  int32_t device;        /* CUDA device ordinal, or -1 for host-only */
  int32_t verbose;       /* 1 = one log line per iteration on stderr */
  int32_t panel_max;     /* max columns per SCM panel group (<= 96); 0 = default 80 */
  int32_t group_max;     /* max constraints per SCM group (<= 64); 0 = default 64 */
  double panel_budget_mb;/* bound on the SCM panel buffers; 0 = default 1024 MB */
  int32_t profile;       /* 1 = time every kernel class with CUDA events (mcsdp_stats_get) */
  int32_t relax;         /* 1 = relaxed supernode amalgamation (default), 0 = fundamental
                            supernodes only; amalgamation enlarges E with explicit zeros */
  int32_t solve_warps;   /* unused (kept for layout compatibility) */
  double mixed_gap;      /* mixed form: relative gap below which every stage runs in FP64.
                            0 = default: 1e-5 for m < 4096; none for m >= 4096, where the
                            correction is GMRES preconditioned by the FP32 factor and the solve
                            promotes only when it stalls or the FP32 factor breaks down;
                            < 0 = none */
  int32_t root_rows;     /* dense root: cliques with more than this many rows (or more than 96
                            columns) are merged, with all their ancestors, into one root clique R
                            handled by dense kernels; the other cliques keep the small-clique
                            kernels.  0 = default (112, the small-clique kernels' limit),
                            < 0 = never (such problems are then rejected), 1..112 = a lower
                            threshold (smaller problems then also get a dense root) */
  int32_t tensor_cores;  /* mixed form: 1 (default) = the FP32 SCM Cholesky's trailing updates
                            and the dense root's FP32 products on the tensor cores (tcgen05, three
                            TF32 products per FP32 product) for m >= 512; 0 = on the CUDA cores */
  double mixed_asm_gap;  /* mixed form: relative gap below which the SCM and the P-MATRIX are
                            assembled in FP64 while the SCE keeps the FP32 factor and FP64
                            refinement (until promotion).  Above it, with a dense root, the
                            root blocks of Y and X̄ are also factored (and X̄_RR's factor
                            inverted) in FP32.  0 = default: 1e-2 with a dense root, else
                            mixed_gap (1e-5 if that is off) */
  int32_t graph;         /* 1 = after the first iteration, each iteration (the direction, the
                            update with step lengths chosen on the device, and the factors at
                            the new iterate) is captured once into a CUDA graph and replayed: one
                            graph launch and one host synchronisation per iteration instead of
                            about a hundred launches and eight synchronisations; same iterates as
                            0.  2 = that iteration as the body of a WHILE conditional node whose
                            loop test runs on the device (the host loop's tests of failure,
                            convergence and the iteration limit on the new iterate): the rest of
                            the solve is one graph launch and one synchronisation (falls back to
                            1 where the graph cannot be built); same iterates as 0.  FP64 form
                            without a dense root only (else ignored); per-class times (profile)
                            are then not measured.  0 (default) = off */
  int32_t scm_blocks;    /* block-diagonal SCM (the sparse-SCM case of Sec. 3.1: B_pq = 0 when
                            A_p and A_q lie in different connected components of the aggregate
                            pattern, X̂ and Y^{-1} being block-diagonal over them; components are
                            joined through each constraint's support).  0 (default) = when the
                            constraints fall into more than one component, the cross-component
                            blocks of B are neither assembled nor factored: one bordered Cholesky
                            and one backward substitution per diagonal block, in FP64 (the mixed
                            form's FP32 factor then does not apply; its FP32 solves do); 1 = one
                            factorisation of the whole m x m matrix, as for a connected pattern */
} mcsdp_options;

void mcsdp_default_options(mcsdp_options *opt);

/* Validates and copies the problem, runs the host symbolic analysis (aggregate pattern,
 * minimum-degree ordering, elimination tree, fundamental supernodes = cliques C_r with S_r
 * first, running-intersection order; Sec. 2.1 and the CHOLMOD supernode reading of Sec. 3.1)
 * and prepares device-side tables.  cuda_stream is a cudaStream_t (NULL = legacy default). */
mcsdp_status mcsdp_create(const mcsdp_problem *prob, const mcsdp_options *opt, void *cuda_stream,
                          mcsdp_ctx **out);
void mcsdp_destroy(mcsdp_ctx *ctx);
const char *mcsdp_last_error(const mcsdp_ctx *ctx);

/* Device workspace: the library allocates nothing on the device by itself; the caller passes
 * one device buffer of at least mcsdp_workspace_size() bytes (e.g. a torch tensor), 256-byte
 * aligned.  mcsdp_set_workspace uploads the symbolic tables into it; the buffer must stay
 * valid until mcsdp_destroy or the next mcsdp_set_workspace. */
mcsdp_status mcsdp_workspace_size(const mcsdp_ctx *ctx, size_t *bytes);
mcsdp_status mcsdp_set_workspace(mcsdp_ctx *ctx, void *dev_ptr, size_t bytes);

/* Sizes of the symbolic structure. */
typedef struct {
  int32_t n, m, nsuper, ngroup, max_nrow, max_ncol, tree_height;
  int64_t nnz_layout;   /* stored values per layout array */
  int64_t nnz_lower_E;  /* entries of lower(E) including the diagonal */
  int64_t nslot;        /* distinct lower positions of the aggregate pattern */
  int64_t table_bytes;  /* bytes of symbolic tables mcsdp_set_workspace copies host -> device */
  int32_t ncomp;        /* connected components holding constraints (the diagonal blocks of B;
                           internal constraint order keeps each one contiguous) */
  int32_t scm_blocks;   /* 1 = B is assembled and factored block by block (options.scm_blocks) */
} mcsdp_sym_info;
mcsdp_status mcsdp_sym_info_get(const mcsdp_ctx *ctx, mcsdp_sym_info *info);

/* Exports the symbolic structure into caller host arrays (any pointer may be NULL):
 *   perm[n]            new (elimination) index -> caller's row/column index
 *   sn_col[nsuper+1]   first column of each supernode (new indices)
 *   sn_rowptr[nsuper+1], sn_rows[sn_rowptr[nsuper]]  clique C_s rows (new indices, ascending,
 *                      the ncol_s own columns first)
 *   sn_valptr[nsuper+1] offset of each supernode block in a layout array
 *   con_order[m]       internal SCM constraint order -> caller's constraint index */
mcsdp_status mcsdp_sym_export(const mcsdp_ctx *ctx, int32_t *perm, int32_t *sn_col,
                              int64_t *sn_rowptr, int32_t *sn_rows, int64_t *sn_valptr,
                              int32_t *con_order);

/* Full solve (Sec. 2.2 Steps 0-4 with the MC reformulation).  Starts from the iterate set by
 * mcsdp_set_iterate, else from X̄ = I on E and a dual-feasible z0 (z0 = 0 when A_0 is positive
 * definite; for max-cut-shaped problems where every A_k = e_k e_k^T, z0_k = -(sum_j |A_0 kj|)-1);
 * otherwise the caller must set a dual-feasible start.  The final iterate stays on the device
 * (mcsdp_get_iterate). */
typedef struct {
  double pobj, dobj, gap, pinf, dinf, mu;
  int32_t iters, status;
  double seconds;       /* wall time of the loop measured with CUDA events */
  double t_scm, t_chol, t_pmat, t_other; /* per-phase seconds (S-ELEMENTS, S-CHOLESKY, P-MATRIX,
                                            rest), CUDA events */
  int32_t precision;     /* the option the solve ran with */
  int32_t promoted_iter; /* mixed form: first iteration solved with the FP64 factor, -1 if none */
  int32_t refine_steps;  /* mixed form: FP64 refinement steps over the solve (GMRES steps for
                            m >= 4096) */
  int32_t assembly_iter; /* mixed form: first iteration with the SCM and P-MATRIX in FP64, -1 if
                            none */
} mcsdp_result;
mcsdp_status mcsdp_solve(mcsdp_ctx *ctx, mcsdp_result *res);

/* Batched form (not in the paper; small SDPs keep one GPU busy only together): solves count
 * independent problems concurrently, nthreads host threads (0 = min(count, 16)) each taking the
 * next unsolved context; every context runs on its own stream (create each with a distinct
 * stream for the solves to overlap on the device).  The context with the largest workspace is
 * solved first, alone.  results[i] (may be NULL) receives context i's result.  Returns MCSDP_OK
 * when every solve returned MCSDP_OK, else the status of the first (lowest index) that did not. */
mcsdp_status mcsdp_solve_batch(mcsdp_ctx *const *ctxs, int32_t count, int32_t nthreads,
                               mcsdp_result *results);

/* Iterate in device memory: Xbar_layout[nnz_layout] (X̄ on E), z[m]; Y is derived as
 * A_0 - sum z_k A_k.  Any pointer may be NULL (then not copied). */
mcsdp_status mcsdp_set_iterate(mcsdp_ctx *ctx, const double *Xbar_layout_dev, const double *z_dev);
mcsdp_status mcsdp_get_iterate(const mcsdp_ctx *ctx, double *Xbar_layout_dev, double *z_dev,
                               double *Y_layout_dev);

/* SCM assembly at the iterate (X̄ on E, z) given in device memory (eq. newSCM2, Sec. 3.1):
 * K2 (Y = N N^T), K1 (Algorithm 1: L̂ from X̄), K3 (B_ij = A_i . (X̂ A_j Y^{-1})).
 * Writes the lower triangle (i >= j, caller's constraint order) of B into B_dev, column-major
 * with leading dimension ldb >= m; the strict upper triangle is not touched.  With a
 * block-diagonal B (options.scm_blocks) the entries between components are written as zeros
 * (they are neither assembled nor factored).
 * h_dev (may be NULL) receives h_i = A_i . Y^{-1}.  precision 0: the solves and the contraction
 * run in FP64.  precision 1 (the mixed form): they run in FP32 from FP32 copies of L̂ and N (the
 * factors themselves are computed in FP64), and the FP32 sums are stored as FP64 values. */
mcsdp_status mcsdp_scm_assemble(mcsdp_ctx *ctx, const double *Xbar_layout_dev, const double *z_dev,
                                double *B_dev, int64_t ldb, double *h_dev, int32_t precision);

/* One Newton step at the iterate (X̄, z) (Sec. 2.2 eqs. SCE, dX, newdX2, primal_length2):
 * outputs dz[m], dX on E (layout), dY on the layout, the step lengths alpha_p, alpha_d (host) and
 * mu (host).  The iterate itself is not changed. */
mcsdp_status mcsdp_newton_step(mcsdp_ctx *ctx, const double *Xbar_layout_dev, const double *z_dev,
                               double *dz_dev, double *dX_layout_dev, double *dY_layout_dev,
                               double *alpha_p, double *alpha_d, double *mu);

/* Factors at the iterate: L̂ (Algorithm 1) and N (Y = N N^T) in the layout (device). */
mcsdp_status mcsdp_factors(mcsdp_ctx *ctx, const double *Xbar_layout_dev, const double *z_dev,
                           double *Lhat_layout_dev, double *N_layout_dev);

/* Kernel statistics of the context since creation or the last reset: the number of kernel
 * launches the library issued (always counted) and, when options.profile = 1, the device time of
 * each kernel class measured with CUDA events recorded on the context's stream around the
 * launches of that class.  Classes: 0 K2 Y=NN^T, 1 K1 Algorithm 1, 2 SCM panel solves,
 * 3 SCM tile contraction, 4 SCM Cholesky in FP64 (task queue), 5 SCE back substitution,
 * 6 P-MATRIX, 7 primal step length, 8 dual step length (candidate factorisations, or the
 * Lanczos bound with a dense root), 9 other (pattern scatter, scalars, update), 10 P-MATRIX
 * Y^{-1} columns on a side stream (single column block: they run beside the SCM solves; their
 * flops are counted in class 6), 11 the SCM's N solves on a side stream (beside the L̂ solves of
 * class 2; their flops are counted in class 2), 12 the mixed form's FP32 SCM Cholesky (tensor
 * cores for m >= 512; its work is class 4's), 13 the dense root's FP64 P-MATRIX GEMM
 * X̂_RR T (its flops are counted in class 6).  Classes 1, 7, 10 and 11 run on side streams
 * (class 1 beside class 0), so their times overlap the others'. */
#define MCSDP_NCLASS 14
typedef struct {
  int64_t launches;
  int64_t count[16];   /* launches per class */
  double ms[16];       /* device milliseconds per class (profile = 1 only) */
} mcsdp_stats;
mcsdp_status mcsdp_stats_get(const mcsdp_ctx *ctx, mcsdp_stats *st);

/* Algorithmic work of one PDIPM iteration per kernel class (same class numbering as
 * mcsdp_stats): FP64 flops (one multiply-add = 2) that the method needs for the context's
 * structure, and the minimum DRAM bytes (each operand read once, each result written once).
 * For class 8 (dual step) the figures are per candidate factorisation. */
typedef struct {
  double flops[16];
  double bytes[16];
} mcsdp_work;
mcsdp_status mcsdp_work_model(const mcsdp_ctx *ctx, mcsdp_work *w);
mcsdp_status mcsdp_stats_reset(mcsdp_ctx *ctx);

/* Schur complement equation solve that allocates nothing: x = B^{-1} g for a symmetric positive
 * definite B (lower triangle read, column-major, leading dimension ldb >= m; device), g and x
 * device vectors of length m.  The paper has no counterpart: this entry point exists for callers
 * that cannot allocate device memory on their code path, e.g. code whose device memory is owned
 * by another framework's caching allocator that has already reserved the device, or a loop that
 * must not pay for a synchronising allocation.  Its working copy of B and the inverses of the
 * diagonal blocks live in one file-scope device array of the library (about 8.9 MB per GPU that
 * loads the library, held until the process exits), so m <= MCSDP_SCE_NOALLOC_MAX_M; larger m is
 * rejected with MCSDP_ERR_ARG.  B and g are not modified.  Every call looks up the array's device
 * address (cudaGetSymbolAddress; no allocation), so a device reset between calls is harmless; the
 * first call on a device also loads the library's device code and must therefore come before any
 * stream capture.
 * Every call reuses the same array, so calls whose GPU work overlaps (different streams, different
 * host threads) race; serialise them.  Returns MCSDP_ERR_NOT_PD if B is not positive definite.
 * cuda_stream is a cudaStream_t; the call synchronises it before returning. */
#define MCSDP_SCE_NOALLOC_MAX_M 1024
mcsdp_status mcsdp_sce_solve_noalloc(const double *B_dev, int64_t ldb, const double *g_dev,
                                     double *x_dev, int32_t m, void *cuda_stream);

/* The reciprocal that the factorisations' serial pivot loops use instead of a division (the
 * diagonal-block Cholesky of the SCM, Sec. 3.1 type (i), and the supernodal Cholesky of Y, type
 * (ii)): r[i] = 1/d[i] from the PTX approximate FP64 reciprocal (rcp.approx.ftz.f64, relative
 * error about 2^-20) and one third-order series step in FP64, faithfully rounded (error below
 * 0.52 ulp) for positive normal d; outside [2^-1000, 2^1000] and for non-positive or non-finite
 * d it is the IEEE division.  Exposed so its accuracy can be checked
 * against division.  d and r are device arrays of n doubles; asynchronous on cuda_stream
 * (a cudaStream_t).  MCSDP_ERR_ARG for n < 0 or a NULL array with n > 0. */
mcsdp_status mcsdp_pivot_reciprocal(const double *d_dev, double *r_dev, int64_t n,
                                    void *cuda_stream);

/* The ticket order of the FP64 SCM factorisation's task queue (the one persistent launch of
 * Sec. 3.1 type (i)), exposed so the host tests can check it: for an m-column factorisation of a
 * rows x m matrix (rows = m + 1 with the right-hand-side row) on 32 x 32 tiles, *ntask receives
 * the number of tasks and, if tasks is not NULL, tasks[4 t .. 4 t + 3] = (type, i, j, k) of
 * ticket t: 0 POTRF(0), 1 TRSM(i, k), 2 UPD(i, j, k), 3 factor of diagonal tile k, 4 / 5 the
 * j-th four-row piece of TRSM(k, k-1) / UPD(k, k, k-1).  CTAs take tickets in increasing order,
 * so the queue is deadlock-free when every task's dependencies have smaller tickets.  Host only;
 * MCSDP_ERR_ARG for m <= 0, rows < m or ntask NULL. */
mcsdp_status mcsdp_chol_task_order(int32_t m, int32_t rows, int64_t *ntask, int32_t *tasks);

/* The same for the block-diagonal SCM's one-launch factorisation of nblk bordered blocks of mb[b]
 * columns (each with its right-hand-side row): the blocks' tickets interleaved phase by phase
 * (every block's prefix, then every block's iteration 0, ...).  tasks[5 t ..] = (block, type, i,
 * j, k) of ticket t, decoded by the kernel's own lookup; each block's tasks keep the order
 * mcsdp_chol_task_order gives for (mb[b], mb[b] + 1).  tasks NULL: only *ntask.  Host only. */
mcsdp_status mcsdp_chol_block_task_order(int32_t nblk, const int32_t *mb, int64_t *ntask,
                                         int32_t *tasks);

/* The shared-memory layouts (byte offsets) of the staged supernodal level solves that evaluate
 * the columns X̂ e_k and Y^{-1} e_k of Sec. 3.1, exposed so the host tests can check them for every
 * admissible clique size: nc / nr = the level's largest |S_r| / |C_r|, cw / np = the update
 * chunk's source-column / row bounds, with_d = the forward kernel stages the diagonal block,
 * elem_size = 8 (FP64) or 4 (FP32).  fwd[7] = (acc, ds, meta, hdr, buf, bufsz, total) of the
 * forward solve, bwd[6] = (ls, ds, acc, wv, rws, total) of the backward one, *cap (may be NULL)
 * = the largest total a staged launch takes (larger FP64 levels use the unstaged kernels).
 * Host only; MCSDP_ERR_ARG for nc <= 0, nr < nc, cw < 0, np < 0, another elem_size or a NULL
 * fwd / bwd. */
mcsdp_status mcsdp_lsolve_layout(int32_t nc, int32_t nr, int32_t cw, int32_t np, int32_t with_d,
                                 int32_t elem_size, int32_t *fwd, int32_t *bwd, int32_t *cap);

/* The FP32 product that the mixed form's dense contractions run on the tensor cores (the SCM
 * Cholesky's trailing updates, Sec. 3.1 computation type (i), and the dense root's products):
 * C = alpha A^T B + beta C with A (K x M) and B (K x N) column-major (element (l, i) of A at
 * A[l + i lda], lda >= K) and C (M x N) column-major (ldc >= M), all FP32 device arrays.  Each
 * operand is split into two TF32 numbers (hi = tf32(a), lo = tf32(a - hi)) and
 * A^T B ~ hi^T hi + hi^T lo + lo^T hi is formed by tcgen05 MMAs (kind::tf32) with FP32
 * accumulation in tensor memory, operand tiles loaded by TMA: FP32-level accuracy.  work is a
 * caller-owned device buffer of at least mcsdp_gemm_tc_work_size() bytes, 256-byte aligned (the
 * split operands).  Synchronises cuda_stream.  MCSDP_ERR_ARG for bad sizes or buffers,
 * MCSDP_ERR_TIMEOUT if one of the kernel's bounded waits ran out. */
mcsdp_status mcsdp_gemm_tc_work_size(int32_t M, int32_t N, int32_t K, size_t *bytes);
mcsdp_status mcsdp_gemm_tc(int32_t M, int32_t N, int32_t K, const float *A, int64_t lda,
                           const float *B, int64_t ldb, float *C, int64_t ldc, float alpha,
                           float beta, void *work, size_t work_bytes, void *cuda_stream);

/* Differentiation of the solution (not in the paper).  The point differentiated is the
 * central-path point for mu = X̄.Y/n of the context's iterate: the iterate is first re-centred
 * (Newton on z for A(mu Y(z)^{-1}) = b with Y(z) = A_0 - sum z_k A_k, until the residual
 * max|A(X) - b| / max(1, max|b|) is at most 1e-13, or, once three full Newton steps in a row no
 * longer halve it, is at the rounding level of its evaluation, at most 64 eps cond(Y), cond(Y)
 * estimated from below by (max_j N_jj / min_j N_jj)^2 (near the optimum cond(Y) grows like
 * 1/mu, and the point carries that rounding);
 * the context's iterate becomes that point, X̄ = mu Y^{-1} on E).  For the loss
 * l = sum over layout entries gX . X̄ + gz^T z, implicit differentiation of A(X) = b,
 * X = mu Y^{-1} gives, with R = sym(X̂ G Y^{-1}) (G the symmetric matrix of the weights gX),
 * v = B^{-1}(A(R) + gz) (B the SCM at the point), g_{A_0} = sym(X̂ (A^*(v) - G) Y^{-1}):
 *   gb[m]   dl/db (the c vector of the input), = v
 *   gC[n0]  dl/d value of every input entry of matrix 0, in input order
 *   gA[n1]  dl/d value of every input entry of matrices 1..m, in input order (-z_k g_{A_0} -
 *           v_k X̄ at the entry)
 * (an off-diagonal entry stands for both triangles, so its gradient counts twice; form 0 flips
 * the sign for matrix 0).  gX (nnz_layout) and gz (m) may be NULL (zero weights); any output may
 * be NULL.  Device pointers, FP64.  Status MCSDP_ERR_STALL if the centring fails. */
mcsdp_status mcsdp_backward(mcsdp_ctx *ctx, const double *gX_layout_dev, const double *gz_dev,
                            double *gC_dev, double *gb_dev, double *gA_dev);

/* Tile-shape tuner for the batched form (many small SDPs; the paper's FCFS task queue of
 * Algorithm 2 lifted to problems leaves the tile shapes to be chosen per problem size).  The SCM
 * grouping sets the shapes of the level solves' right-hand-side tiles and of the tile
 * contraction: group_max constraints per group, at most panel_max columns per group.
 * mcsdp_tune times `iters` iterations (after one untimed run of the same length) of the problem
 * under each candidate (group_max, panel_max) in {(64, 80), (32, 80), (16, 80), (64, 96),
 * (32, 48)}, skipping candidates the problem's constraints do not fit, and writes the fastest
 * into opt->group_max and opt->panel_max.  The choice is cached process-wide under the key
 * (n, m, largest clique of the default analysis), each rounded up to a power of two: a later
 * problem with the same key takes it without timing (info->cached = 1).  z0_dev: a dual-feasible
 * start (device, m values), or NULL for the library's default start.  ws: device buffer of at
 * least mcsdp_tune_workspace_size bytes, 256-byte aligned; its contents are overwritten.  The
 * other options (precision, graph, ...) are used as given.  MCSDP_ERR_ARG if no candidate
 * runs. */
typedef struct {
  int32_t group_max, panel_max;  /* the choice */
  int32_t cached;                /* 1 = taken from the cache without timing */
  int32_t ncand;                 /* candidates timed (0 when cached) */
  double ms_per_iter[8];         /* per candidate in the order above; < 0 = skipped */
  int64_t key[3];                /* n, m, largest clique, rounded up to powers of two */
} mcsdp_tune_info;
mcsdp_status mcsdp_tune_workspace_size(const mcsdp_problem *prob, const mcsdp_options *opt,
                                       size_t *bytes);
mcsdp_status mcsdp_tune(const mcsdp_problem *prob, mcsdp_options *opt, const double *z0_dev,
                        void *cuda_stream, void *ws, size_t ws_bytes, int32_t iters,
                        mcsdp_tune_info *info);
void mcsdp_tune_cache_clear(void);

#ifdef __cplusplus
}
#endif
#endif /* MCSDP_H */
