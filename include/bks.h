/*
 * bks.h -- C ABI of the GB300 Block Krylov-Schur library.
 *
 * Computes best rank-(r1,r1,r3) approximations of large sparse 3-tensors
 * A (m x m x n) that are symmetric in modes 1 and 2, A(i,j,k) = A(j,i,k)
 * (Definition 2.1 of Eldén & Dehghan, "A Krylov-Schur like method for
 * computing the best rank-(r1,r2,r3) approximation of large and sparse
 * tensors").  The problem (Section 2.4, eqs. (main min) and (max)):
 *
 *     max || A.(U,U,W) ||   subject to  U^T U = I_r1,  W^T W = I_r3,
 *
 * with the optimal core F = A.(U,U,W) (eq. (Rayleigh)).
 *
 * Conventions for every call below
 *   - Return value: BKS_OK (0) or a negative BKS_E* code.  The message of
 *     the last failure on the calling thread is bks_last_error_string().
 *     No C++ exception crosses this boundary.
 *   - Matrices are column-major with an explicit leading dimension
 *     (ld >= rows).  Indices are 0-based.
 *   - Pointers are DEVICE pointers (cudaMalloc'ed or equivalent) unless a
 *     comment says host.  The caller owns every buffer it passes; the
 *     library owns the tensor handle and its device buffers.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are stream-ordered: device results are ready when
 *     the stream reaches the call's end.  Calls that return host-side
 *     values (bks_tensor_info, the solvers' info) synchronise the stream.
 *   - dtype BKS_F64 means double, BKS_F32 means float, for every floating
 *     buffer of the call that the comment calls "dtype-typed".
 *
 * Limits: 2*ceil(log2 m) + ceil(log2 n) <= 64 bits (the ingest sort key),
 * at most 2^31 - 1024 entries after mirroring (input plus mirrors, before
 * duplicates are summed).  The contraction kernels take widths up to 8;
 * wider operands of bks_contract_mode1 / mode3 are cut into chunks of at
 * most 8 columns of X per column of the second operand (one tensor pass
 * each).
 */
#ifndef BKS_GB300_H
#define BKS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define BKS_OK            0
#define BKS_EINVAL       -1  /* bad argument: index out of range, size <= 0, null pointer */
#define BKS_ENOMEM       -2  /* device allocation failed */
#define BKS_ECUDA        -3  /* a CUDA runtime call failed (message has the CUDA error) */
#define BKS_EASYM        -4  /* BKS_VALIDATE_SYMMETRIC: input is not (1,2)-symmetric */
#define BKS_ENOTCONV     -5  /* solver hit max_outer / max_iter; best iterate still written */
#define BKS_EBREAKDOWN   -6  /* a basis block collapsed to zero width where one is required */
#define BKS_ENUMERIC     -7  /* NaN or Inf in ||F|| or in the gradient */
#define BKS_EUNSUPPORTED -8  /* a size beyond the limits above */
#define BKS_ECANCELED    -9  /* the job was cancelled (server) */
#define BKS_EPENDING    -10  /* the job has not finished yet (server poll without wait) */
#define BKS_EBUDGET     -11  /* the job alone needs more device memory than the server's budget */

/* ---- dtypes, flags, options -------------------------------------------- */
#define BKS_F32 1
#define BKS_F64 2

#define BKS_MIRROR             1  /* add (j,i,k,v) for every input entry with i != j */
#define BKS_VALIDATE_SYMMETRIC 2  /* without MIRROR: check A(i,j,k) == A(j,i,k) bitwise */
#define BKS_INPUT_ON_DEVICE    4  /* i, j, k, v are device pointers (default: host) */

#define BKS_PREC_FP64  0  /* contractions in FP64 */
#define BKS_PREC_MIXED 1  /* contractions in FP32 (FP64 orthogonalisation, inner solve, restart) */

#define BKS_VARIANT_BK  0  /* BK schedule, Table 3 */
#define BKS_VARIANT_MIN 1  /* min-BK, Algorithm 4 / Table 1 */
#define BKS_VARIANT_MAX 2  /* max-BK, Table 2 */

#define BKS_INNER_PAPER 0  /* inner solve as Section 6.2: truncated HOSVD + 5 HOOI sweeps,
                              then Newton-Grassmann to the outer stopping criterion */
#define BKS_INNER_FAST  1  /* truncated HOSVD without start sweeps, up to 20 HOOI sweeps, then
                              Newton-Grassmann, to an inexact inner tolerance */

typedef struct bks_tensor bks_tensor;

/* ---- tensor storage (Definition 2.1; Section 4.3 storage reading) -------
 * bks_tensor_create_coo: copy a COO list into a new device-resident
 * (1,2)-symmetric tensor.
 *   m, n      : tensor is m x m x n (m, n >= 1)
 *   nnz       : number of input entries (>= 0)
 *   i, j, k   : int32 indices, host pointers unless BKS_INPUT_ON_DEVICE
 *   v         : values of type vdtype (BKS_F32 or BKS_F64)
 *   flags     : BKS_MIRROR adds the mirror (j,i,k,v) of each off-diagonal
 *               entry.  The stored list is the input in input order, then
 *               the mirrors in input order, stably sorted by (i,j,k);
 *               entries with equal (i,j,k) are summed left to right in
 *               vdtype; exact zeros are kept.  BKS_VALIDATE_SYMMETRIC
 *               (without MIRROR) rejects a summed tensor that is not
 *               bitwise (1,2)-symmetric with BKS_EASYM.
 *   out       : receives the handle (host pointer to a handle)
 * Errors: BKS_EINVAL (index >= m or >= n, m or n < 1, nnz < 0, null
 * pointers), BKS_EUNSUPPORTED (sizes beyond the limits), BKS_EASYM,
 * BKS_ENOMEM, BKS_ECUDA.  On error *out is NULL and nothing leaks. */
int bks_tensor_create_coo(int64_t m, int64_t n, int64_t nnz,
                          const int32_t* i, const int32_t* j, const int32_t* k,
                          const void* v, int vdtype, int flags, void* stream,
                          bks_tensor** out);

/* Free the handle and its device buffers (NULL is a no-op). */
void bks_tensor_destroy(bks_tensor* t);

/* Host outputs (any may be NULL): sizes, stored nonzeros after
 * symmetrisation and ||A||_F^2 (FP64 sum of the stored values squared). */
int bks_tensor_info(const bks_tensor* t, int64_t* m, int64_t* n,
                    int64_t* nnz_stored, double* fro2);

/* Copy the stored tensor in its canonical order (sorted by (i,j,k)) into
 * caller device buffers of nnz_stored entries each; v has the input
 * vdtype.  Used for bit-exact checks of the ingest. */
int bks_tensor_export_coo(const bks_tensor* t, int32_t* i, int32_t* j,
                          int32_t* k, void* v, void* stream);

/* ---- contractions (Section 2.2; Algorithm 3 step (i); Section 4.3.1) ----
 * bks_contract_mode1: out = unfold_1(A.(X,Y)_{2,3}),
 *     out[i + ldo*(a + p*b)] = sum over stored (i,j,k) of v X[j,a] Y[k,b]
 *   X: m x p (ldx), Y: n x q (ldy), out: m x (p*q) (ldo); dtype-typed;
 *   p, q >= 1.  Up to p = 8 one pass over the tensor per group of at most
 *   8 (p <= 4), 5 (p = 5) or 4 (p > 5) columns of Y; above p = 8 one pass
 *   per column of Y and chunk of at most 8 columns of X, each chunk summed
 *   as a p <= 8 call would.  `out` is overwritten (rows without entries
 *   get 0).
 *   dtype BKS_F64 computes in FP64; BKS_F32 computes in FP32 with FP32
 *   accumulation (blocked summation: short sequential runs combined by a
 *   fixed-order tree). Deterministic: the same call gives the same bits. */
int bks_contract_mode1(const bks_tensor* t, const void* X, int64_t ldx, int p,
                       const void* Y, int64_t ldy, int q, void* out,
                       int64_t ldo, int dtype, void* stream);

/* bks_contract_mode1_noalloc: the same result as bks_contract_mode1 (same
 *   arguments, the same code path with the same kernels and summation
 *   order, bitwise the same output) for callers that cannot allocate device
 *   memory -- for example a host framework that has reserved the whole
 *   device for its own memory pool, or code that must not let a library
 *   call cudaMalloc, which can synchronise the device and fail under memory
 *   pressure.  The paper has no counterpart of this call.
 *   Scratch (the packed copies of X and Y and the partial sums of long
 *   rows) lives in a fixed 32 MiB device array inside the library, which
 *   every GPU that loads the library keeps until the process exits.  A call
 *   needs s*(SP*m + SQ*n + PB*QB*nslots) bytes, each of the three pieces
 *   rounded up to 256 bytes, with s = 8 (BKS_F64) or 4 (BKS_F32); PB is the
 *   width bucket of p (1 -> 2; 2, 3, 4, 5 as they are; 6..8 -> 8), QB that
 *   of min(q, 8), or of min(q, 5) when PB = 5 and min(q, 4) when PB = 8; SP,
 *   SQ are the packed row strides (FP32: 2 for width 2, 4 for 3 and 4, 8
 *   for 5 and 8; FP64: the width itself); nslots is the number of pieces into which
 *   rows longer than the work plan's split (512 below 8M stored entries,
 *   1024 below 32M, 2048 from 32M, unless bks_tensor_autotune / set_tiles
 *   chose another) are cut, about nnz / split on power-law tensors.  The
 *   worst case is 64*m + 64*n + 256*nslots bytes in FP64.  A call needing
 *   more than 32 MiB, or with p or q above 8, returns BKS_EUNSUPPORTED
 *   before launching anything.
 *   The call allocates nothing.  Its first call on a device looks up the
 *   array's device address (cudaGetSymbolAddress) with that device current;
 *   make that first call before any stream capture.  All calls share the
 *   one array and every call overwrites what it uses (nothing has to start
 *   at zero), so calls that overlap on the GPU -- on different streams, or
 *   from several host threads -- race; order them on one stream. */
int bks_contract_mode1_noalloc(const bks_tensor* t, const void* X, int64_t ldx,
                               int p, const void* Y, int64_t ldy, int q,
                               void* out, int64_t ldo, int dtype, void* stream);

/* bks_contract_mode3: out = unfold_3(A.(X,X2)_{1,2})
 *   X2 != NULL: out[k + ldo*(a + p*b)] = sum v X[i,a] X2[j,b]; out is
 *     n x (p*q); X2 is m x q (ldx2).
 *   X2 == NULL: the (1,2)-symmetric case X2 = X stored as triunfold_3
 *     (Section 4.3.1): out[k + ldo*(a + b(b+1)/2)] for a <= b; out is
 *     n x p(p+1)/2.
 *   p, q >= 1; above p = 8 the columns are computed as full products of
 *   chunks of at most 8 columns of X with one column of X2 (or of X, a <= b,
 *   in the triangle case), one tensor pass each.  dtype-typed; out
 *   overwritten; deterministic. */
int bks_contract_mode3(const bks_tensor* t, const void* X, int64_t ldx, int p,
                       const void* X2, int64_t ldx2, int q, void* out,
                       int64_t ldo, int dtype, void* stream);

/* bks_core: F = A.(U,U,W) (eq. (Rayleigh); with the Krylov bases it is
 *   C = A.(X,X,Z) of eq. (tkd)).  U: m x r1 (ldu), W: n x r3 (ldw),
 *   F: r1*r1*r3 contiguous, F[a + r1*(b + r1*c)]; dtype-typed; any
 *   r1 <= 128, r3 <= 128.  F is symmetric in (a, b). */
int bks_core(const bks_tensor* t, const void* U, int64_t ldu, int r1,
             const void* W, int64_t ldw, int r3, void* F, int dtype,
             void* stream);

/* ---- solvers (Algorithm 5; Section 6.1) --------------------------------- */
typedef struct {
  int r1, r3;          /* target multilinear rank (r1, r1, r3) */
  int stages;          /* s: BK stages per expansion (paper recommends 2) */
  int block_p;         /* p: leading columns of each ON-block used (paper: 4) */
  double tol;          /* stop when ||grad|| / ||F|| <= tol (Section 6.2) */
  int max_outer;       /* outer-iteration cap (BKS_ENOTCONV past it) */
  int max_inner;       /* inner HOOI sweep cap per outer iteration */
  int variant;         /* BKS_VARIANT_* */
  int precision;       /* BKS_PREC_FP64 or BKS_PREC_MIXED */
  int refine_sweeps;   /* MIXED only: at most this many outer iterations in the refinement
                          form after the FP32 phase */
  uint64_t seed;       /* random start when U0/W0 are NULL */
  double drop_tol;     /* rank-drop threshold of the block QR (relative) */
  double inner_tol;    /* inner stopping tolerance on ||grad_C|| / ||F_C||; <= 0: set by
                          inner_schedule (PAPER: the outer tolerance; FAST: max(tol / 10,
                          ||grad|| / ||F|| / 100) at the current outer point) */
  int tol_scale_free;  /* 0: stop when ||grad|| / ||F|| <= tol (Section 6.2, depends on the
                          scale of A); 1: stop when ||grad|| / ||F||^2 <= tol (invariant
                          under A -> c A) */
  double mixed_tol;    /* MIXED only: the FP32 phase ends when ||grad|| / ||F||^2 <= mixed_tol
                          (<= 0: 1e-4) or when that ratio stops halving for two outer
                          iterations; outer iterations in the refinement form follow until
                          tol (FP64 stage-1 contractions, gradient and stopping test; FP32
                          later Krylov blocks and core C with its first-order blocks
                          replaced by FP64 projections of the stage-1 results) */
  int inner_schedule;  /* BKS_INNER_PAPER (default) or BKS_INNER_FAST: the inner solve of
                          Algorithm 5 step (i).  Both start from the better (larger ||F||) of
                          the truncated HOSVD of C and the current point.  PAPER (Section 6.2)
                          gives the HOSVD start 5 HOOI sweeps, then takes Newton-Grassmann
                          steps (a HOOI sweep where the Hessian is not negative definite or
                          ||F|| would drop) to the outer tolerance; FAST takes up to 20 HOOI
                          sweeps, then Newton-Grassmann steps, to the inexact tolerance above
                          (cheap on well-separated problems, quadratic where HOOI creeps).
                          info.inner_sweeps counts sweeps and Newton steps */
} bks_params;

typedef struct {
  int iters;           /* outer iterations done */
  int converged;       /* 1 if the final gradient test passed */
  double grad_rel;     /* ||grad|| / ||F|| at the returned point */
  double normF;        /* ||F|| at the returned point */
  int k1, k3;          /* basis sizes of the last expansion */
  int inner_sweeps;    /* total inner HOOI sweeps */
  int fp32_iters;      /* MIXED: outer iterations with FP32 contractions */
  double seconds;      /* host wall time of the call */
  double phase_ms[5];  /* device time by phase (CUDA events on the stream): stage 1 with the
                          gradient, rest of the expansion, core C, inner solve, restart */
  double* history;     /* host, optional: 2 doubles (grad_rel, normF) per outer iteration */
  int history_cap;     /* capacity of history in iterations */
  int history_len;     /* filled entries */
  int k2;              /* bks_gen_solve: mode-2 basis size of the last expansion */
} bks_info;

/* Default parameters: r1 = r3 = 2, s = 2, p = 4, tol 1e-10, max_outer 500,
 * max_inner 1000, BK, FP64, refine 1, seed 1, mixed_tol 1e-4, inner schedule
 * BKS_INNER_PAPER, drop_tol 1e-14 (a rank-drop threshold
 * well below the gradient accuracy: near convergence the stage-1 residual
 * columns that carry the gradient are small relative to their raw norms). */
void bks_params_default(bks_params* p);

/* bks_solve: tensor Krylov-Schur (Algorithm 5 with U = V, X = Y).
 *   U0 (m x r1, ld m), W0 (n x r3, ld n): orthonormal start, device FP64,
 *     or NULL for a seeded random start.
 *   U (m x r1, ld m), W (n x r3, ld n), F (r1*r1*r3): device FP64 outputs.
 *   info: host pointer or NULL.
 * Returns BKS_OK, BKS_ENOTCONV (best iterate written), BKS_ENUMERIC,
 * BKS_EBREAKDOWN, BKS_EINVAL, BKS_ENOMEM, BKS_ECUDA.  Synchronises
 * `stream` once per outer iteration to read the convergence test. */
int bks_solve(const bks_tensor* t, const bks_params* prm, const double* U0,
              const double* W0, double* U, double* W, double* F,
              bks_info* info, void* stream);

typedef struct {
  int r1, r3;
  double tol;
  int max_iter;
  int grad_every;      /* gradient test cadence (Section 6.1: every 10) */
  int precision;       /* BKS_PREC_FP64 or BKS_PREC_MIXED: FP32 contractions until the
                          gradient, evaluated from them, has ||grad|| / ||F||^2 <= mixed_tol
                          or stops halving for two evaluations; then FP64 contractions (the
                          gradient is evaluated at the next iteration again) until tol */
  uint64_t seed;
  double mixed_tol;    /* MIXED only (<= 0: 1e-4) */
} hooi_params;

void hooi_params_default(hooi_params* p);

/* hooi_solve: HOOI for (1,2)-symmetric tensors (Section 6.1): U from the
 * r1 leading left singular vectors of unfold_1(A.(U,W)_{2,3}), then W from
 * the r3 leading left singular vectors of unfold_3(A.(U,U)_{1,2}).
 * Same buffers and errors as bks_solve. */
int hooi_solve(const bks_tensor* t, const hooi_params* prm, const double* U0,
               const double* W0, double* U, double* W, double* F,
               bks_info* info, void* stream);

/* ---- work-plan autotuning ------------------------------------------------
 * The contractions process a tensor by rows: rows longer than `split`
 * entries are cut into pieces of at most `split` (their partial sums are
 * added in a fixed order by a second kernel); pieces and rows longer than
 * `tile` entries take one warp each, the others one lane each, 32 to a
 * warp in order of decreasing length (their entries are read from a
 * lane-interleaved copy).  The best sizes depend on how the entries spread
 * over rows.  The default (tile, split) is (32, 512) below 8M stored
 * entries, (64, 1024) below 32M and (128, 2048) from 32M on.
 * bks_tensor_autotune times the mode-1 and triangle mode-3 contractions
 * (FP32, widths 4 x 4) under the plans (tile, split) in {(8,512),
 * (16,512), (64,1024), (128,2048), (32,512)} and keeps the fastest; tile
 * and split (host, nullable) receive the choice.  bks_tensor_set_tiles
 * applies a known choice (1 <= tile <= 128, 128 <= split <= 4096; else
 * BKS_EINVAL).
 * Both synchronise `stream`. */
int bks_tensor_autotune(bks_tensor* t, int* tile, int* split, void* stream);
int bks_tensor_set_tiles(bks_tensor* t, int tile, int split, void* stream);

/* ---- batched solves -------------------------------------------------------
 * bks_batch_solve: njobs independent BKS solves (bks_solve semantics per
 * job) on tensors already stored on the device.  The jobs run on
 * `nstreams` streams at once (one host worker thread per stream), so the
 * kernels of different jobs overlap on the GPU; with
 * BKS_BATCH_AUTOTUNE each tensor first gets the work-tile plan of its size
 * class (log2 of the stored entries), tuned once per class.
 *   T[njobs], P[njobs]: tensors and parameters (host arrays of pointers /
 *     structs).
 *   U0, W0: host arrays of device pointers (or NULL arrays / entries: seeded
 *     random start).  U, W, F: host arrays of device output pointers.
 *   info[njobs] (host, nullable): per-job info; status[njobs] (host,
 *     nullable): per-job return code.
 * Returns BKS_OK when every job returned BKS_OK, else the first failing
 * job's code (the other jobs still ran).  The jobs start after the work
 * queued on the caller's `stream` before the call, and `stream` is made to
 * wait for all jobs. */
#define BKS_BATCH_AUTOTUNE 1
int bks_batch_solve(int njobs, bks_tensor* const* T, const bks_params* P,
                    const double* const* U0, const double* const* W0, double* const* U,
                    double* const* W, double* const* F, bks_info* info, int* status,
                    int nstreams, int flags, void* stream);

/* ---- serving: continuous batching under a device-memory budget -----------
 * A server owns `max_slots` worker threads, each with its own stream.
 * Submitted jobs (host COO + parameters) wait in a FIFO queue; the head job
 * is admitted as soon as a slot is free and its predicted device memory
 * fits into `hbm_budget` minus what the running jobs hold, so jobs that
 * arrive while others run join the GPU as slots and memory free up.  A
 * running job keeps its tensor, Krylov bases and inner-solve state on the
 * device until it completes; results are copied to host memory.
 * Predicted bytes of a job: 96 * nnz + 8 * (m + n) * 168 + 64 MiB (ingest
 * sort buffers, two sorted copies, the interleaved copy of the short rows,
 * bases and workspace).
 * flags: BKS_SERVE_AUTOTUNE tunes the work tiles per size class. */
#define BKS_SERVE_AUTOTUNE 1
typedef struct bks_server bks_server;

/* Create (device = the current device of the calling thread).  Returns
 * NULL on failure (bks_last_error_string). */
bks_server* bks_server_create(size_t hbm_budget, int max_slots, int flags);

/* Submit a job: m, n, nnz, i, j, k, v, vdtype, coo_flags as
 * bks_tensor_create_coo (host pointers; the data are copied), prm its BKS
 * parameters.  *ticket receives the job's ticket.  BKS_EBUDGET if the job
 * alone exceeds the budget; BKS_EINVAL for bad arguments. */
int bks_server_submit(bks_server* srv, int64_t m, int64_t n, int64_t nnz, const int32_t* i,
                      const int32_t* j, const int32_t* k, const void* v, int vdtype,
                      int coo_flags, const bks_params* prm, uint64_t* ticket);

/* Poll a job.  Not finished: BKS_EPENDING (wait = 0) or block until it
 * finishes (wait != 0).  Finished: BKS_OK; *job_status receives the job's
 * own return code (BKS_OK, BKS_ENOTCONV, BKS_ECANCELED, an ingest error
 * ...); U (m x r1), W (n x r3), F (r1 r1 r3) are HOST buffers (nullable)
 * that receive the result; latency_s (nullable) receives completion minus
 * submission time.  The ticket is retired by a successful poll
 * (BKS_EINVAL afterwards). */
int bks_server_poll(bks_server* srv, uint64_t ticket, int wait, double* U, double* W, double* F,
                    bks_info* info, int* job_status, double* latency_s);

/* Cancel a job: a queued job is removed, a running one stops at its next
 * outer iteration; either way it finishes with BKS_ECANCELED. */
int bks_server_cancel(bks_server* srv, uint64_t ticket);

/* Host counters (nullable outputs): jobs queued, running, finished and not
 * yet polled, device bytes currently held by running jobs. */
int bks_server_stats(bks_server* srv, int* queued, int* running, int* finished,
                     size_t* resident_bytes);

/* Cancel what is still queued or running, wait for the workers, free.
 * No other call on the same server may overlap with or follow it. */
void bks_server_destroy(bks_server* srv);

/* Last error message of the calling thread ("" if none). */
const char* bks_last_error_string(void);

/* ---- conditioning diagnostics and slice normalisation (Sections 2.6, 7) ---- */

/* S-values (Section 2.6) at the point (U, U, W) (U m x r1, W n x r3, both
 * orthonormal, device, column-major with leading dimensions ldu, ldw; FP64):
 *   s1[q] = sqrt(lambda_q(<F,F>_{-1})), q < r1, F = A.(U,U,W), and
 *   s1[r1] = sqrt(lambda_max(<F_perp^1, F_perp^1>_{-1})), F_perp^1 =
 *   A.(U_perp,U,W); s3 likewise for mode 3 with F_perp^3 = A.(U,U,W_perp).
 *   (Mode 2 equals mode 1 by the symmetry.)  The gaps of Section 2.6 are
 *   s1[r1-1] - s1[r1] and s3[r3-1] - s3[r3].
 *   s1, s3 : HOST arrays of r1 + 1 and r3 + 1 doubles, descending for q < r.
 * Cost: one mode-1 and one mode-3 FP64 contraction and tall-skinny passes;
 * synchronises the stream.  Errors: BKS_EINVAL (null, r < 1, r >= m or n,
 * r1 or r3 > 8, ld below the rows), BKS_ENOMEM, BKS_ECUDA. */
int bks_s_values(const bks_tensor* t, const double* U, int64_t ldu, int r1,
                 const double* W, int64_t ldw, int r3, double* s1, double* s3,
                 void* stream);

#define BKS_NORM_FRO  0  /* Frobenius norm of each frontal slice A(:,:,k) */
#define BKS_NORM_LMAX 1  /* largest (algebraic) eigenvalue of each slice */

/* Per-slice norms (Section 7): norms[k] for k < n, a DEVICE array of n
 * doubles.  BKS_NORM_FRO: the Frobenius norm (fixed-order FP64 sum).
 * BKS_NORM_LMAX: the largest eigenvalue of the symmetric slice by a batched
 * Lanczos iteration (FP64, no reorthogonalisation, positive seeded start
 * vectors); a slice stops when its estimate moves by at most 1e-13 of
 * itself over 10 steps, at an invariant subspace, or after min(m, 400)
 * steps; an empty slice gets 0.  Work memory: three m x nb FP64 blocks,
 * nb slices at a time, at most 2 GB.  Synchronises the stream.
 * Errors: BKS_EINVAL, BKS_ENOMEM, BKS_ECUDA. */
int bks_slice_norms(const bks_tensor* t, int kind, double* norms, void* stream);

/* A new tensor whose slice k is scales[k] times slice k of t (scales: DEVICE
 * array of n doubles): every stored value times its slice's scale, rounded
 * once to the value dtype; the order of the entries is unchanged.  With
 * scales[k] = 1 / norms[k] from bks_slice_norms this is the slice
 * normalisation of Section 7.  *out receives a handle the caller destroys.
 * Synchronises the stream.  Errors as bks_tensor_create_coo. */
int bks_tensor_scale_slices(const bks_tensor* t, const double* scales, void* stream,
                            bks_tensor** out);

/* Number of CUDA kernels this library has launched since it was loaded
 * (all threads, all devices); a diagnostic counter for benchmarks. */
uint64_t bks_launch_count(void);

/* ---- general (nonsymmetric) l x m x n tensors (Section 5) -----------------
 * The method of Section 5 as the paper states it, before the (1,2)-symmetric
 * specialisation: three bases X (l x k1), Y (m x k2), Z (n x k3) grown by the
 * block-Krylov step of Algorithm 3 in each mode, the G-gradient from the
 * three stage-1 blocks (Proposition 2), the core C = A.(X,Y,Z) (eq. (tkd)),
 * its best rank-(r1,r2,r3) approximation (Algorithm 5 step (i)) and the
 * restart (eq. (tks1)).  FP64 only.  A general handle is refused by the
 * symmetric calls above (BKS_EUNSUPPORTED) and vice versa; destroy it with
 * bks_tensor_destroy; bks_tensor_info reports m, n, nnz and ||A||^2 and
 * bks_tensor_export_coo the sorted entries. */

/* bks_gen_tensor_create_coo: store A (l x m x n) from nnz COO entries.
 *   i < l, j < m, k < n (int32, 0-based); v BKS_F32 or BKS_F64 (vdtype).
 *   Entries are sorted by (i, j, k) (stable) and entries with equal keys
 *   summed left to right in the value dtype; nothing is mirrored.  flags:
 *   BKS_INPUT_ON_DEVICE (i, j, k, v are device pointers) or 0 (host);
 *   BKS_MIRROR / BKS_VALIDATE_SYMMETRIC give BKS_EINVAL.  Errors:
 *   BKS_EINVAL (an index out of range, a dimension < 1, nnz < 0),
 *   BKS_EUNSUPPORTED (a dimension or nnz above int32, l m n above a 64-bit
 *   sort key), BKS_ENOMEM, BKS_ECUDA.  The library owns the handle. */
int bks_gen_tensor_create_coo(int64_t l, int64_t m, int64_t n, int64_t nnz,
                              const int32_t* i, const int32_t* j, const int32_t* k,
                              const void* v, int vdtype, int flags, void* stream,
                              bks_tensor** out);

/* bks_gen_tensor_dims: l, m, n of any handle (l = m for a symmetric one) and
 * general = 1 for a general handle, 0 for a (1,2)-symmetric one.  Host
 * outputs, each nullable. */
int bks_gen_tensor_dims(const bks_tensor* t, int64_t* l, int64_t* m, int64_t* n, int* general);

/* bks_gen_contract: the block contraction of Algorithm 3 step (i) in mode
 * `mode` (Section 2.2), column-major, column a + p*b, out overwritten:
 *   mode 1: out (l x p q)[i, a + p b] = sum v B1[j, a] B2[k, b]; B1 m x p, B2 n x q
 *   mode 2: out (m x p q)[j, a + p b] = sum v B1[i, a] B2[k, b]; B1 l x p, B2 n x q
 *   mode 3: out (n x p q)[k, a + p b] = sum v B1[i, a] B2[j, b]; B1 l x p, B2 m x q
 *   Device pointers of `dtype` (BKS_F32 or BKS_F64), leading dimensions at
 *   least the rows; 1 <= p, q <= 8.  Deterministic (no atomics).  Errors:
 *   BKS_EINVAL, BKS_EUNSUPPORTED (a width above 8, a symmetric handle). */
int bks_gen_contract(const bks_tensor* t, int mode, const void* B1, int64_t ld1, int p,
                     const void* B2, int64_t ld2, int q, void* out, int64_t ldo,
                     int dtype, void* stream);

/* bks_gen_core: C = A.(X,Y,Z) (eq. (tkd)), C[a + k1 (b + k2 c)] (k1 k2 k3
 *   doubles, device); X l x k1 (ldx), Y m x k2 (ldy), Z n x k3 (ldz), FP64
 *   device; 1 <= k1, k2, k3 <= 128. */
int bks_gen_core(const bks_tensor* t, const double* X, int64_t ldx, int k1,
                 const double* Y, int64_t ldy, int k2, const double* Z, int64_t ldz, int k3,
                 double* C, void* stream);

typedef struct {
  int r1, r2, r3;      /* target multilinear rank, each 1..8, pairwise products <= 32 */
  int stages;          /* s: BK stages per expansion */
  int block_p;         /* p: leading columns of each ON-block used (block 0 whole) */
  double tol;          /* stop when ||grad|| / ||F|| <= tol (tol_scale_free: / ||F||^2) */
  int max_outer;       /* outer-iteration cap (BKS_ENOTCONV past it) */
  int max_inner;       /* inner HOOI sweep cap per outer iteration */
  int variant;         /* BKS_VARIANT_BK, _MIN or _MAX, in the general form: stage 1
                          makes U1 from (V0,W0), V1 from (U0,W0), W1 from (U0,V0); BK stage
                          t >= 2 (q = t-1) takes the pairs (0,q), (q,0), ..., (q-1,q), (q,q-1)
                          of the other two modes' blocks in every mode; MIN the pair
                          (t-1, t-1); MAX every unused pair of whole blocks */
  int tol_scale_free;  /* 1: the test is ||grad|| / ||F||^2 <= tol */
  uint64_t seed;       /* random start when a start matrix is NULL */
  double drop_tol;     /* rank-drop threshold of the block QR (relative) */
  double inner_tol;    /* inner tolerance; <= 0: set by inner_schedule */
  int inner_schedule;  /* BKS_INNER_PAPER (default): the HOSVD start gets 5 HOOI sweeps and
                          the sweeps continue to the outer tolerance; BKS_INNER_FAST: no start
                          sweeps and the inexact tolerance max(tol / 10, ||grad|| / ||F|| / 100)
                          at the current outer point (tol in ||grad|| / ||F|| units) */
} bks_gen_params;

/* Defaults: r = (2,2,2), s = 2, p = 4, tol 1e-10, max_outer 500,
 * max_inner 1000, BK, seed 1, drop_tol 1e-14, inner_tol 0,
 * BKS_INNER_PAPER. */
void bks_gen_params_default(bks_gen_params* p);

/* bks_gen_solve: tensor Krylov-Schur for a general tensor (Algorithm 5).
 *   U0 (l x r1), V0 (m x r2), W0 (n x r3): orthonormal device FP64 starts
 *   (ld = rows), each nullable (seeded random start).  Inner solve: the
 *   better of the truncated HOSVD of C after 5 HOOI sweeps and the current
 *   point, then HOOI sweeps (each the leading singular vectors of one
 *   mode's contraction given the other two, so ||F|| never drops) to the
 *   outer tolerance.  Outputs U (l x r1), V (m x r2), W (n x r3), F
 *   (r1 r2 r3, F[a + r1 (b + r2 c)]) on the device; info (host, nullable)
 *   with k1, k2, k3 of the last expansion.  Returns BKS_OK, BKS_ENOTCONV
 *   (the last evaluated point written), BKS_ENUMERIC, BKS_EINVAL,
 *   BKS_EUNSUPPORTED, BKS_ENOMEM, BKS_ECUDA.  Synchronises `stream` once
 *   per outer iteration. */
int bks_gen_solve(const bks_tensor* t, const bks_gen_params* prm, const double* U0,
                  const double* V0, const double* W0, double* U, double* V, double* W,
                  double* F, bks_info* info, void* stream);

typedef struct {
  int r1, r2, r3;      /* target multilinear rank, each 1..8, pairwise products <= 32 */
  double tol;          /* stop when ||grad|| / ||F|| <= tol */
  int max_iter;        /* iteration cap (BKS_ENOTCONV past it) */
  int grad_every;      /* gradient test cadence (Section 6.1: every 10) */
  uint64_t seed;       /* random start when a start matrix is NULL */
} bks_gen_hooi_params;

/* Defaults: r = (2,2,2), tol 1e-10, max_iter 5000, grad_every 10, seed 1. */
void bks_gen_hooi_params_default(bks_gen_hooi_params* p);

/* bks_gen_hooi_solve: HOOI for a general tensor (Section 6.1): U from the
 * r1 leading left singular vectors of unfold_1(A.(V,W)_{2,3}), then V from
 * unfold_2(A.(U,W)_{1,3}) with the new U, then W from unfold_3(A.(U,V)_{1,2})
 * with the new U and V; the G-gradient in global coordinates (three terms)
 * every grad_every iterations at the start of the iteration.  FP64.  Same
 * buffers, info fields and errors as bks_gen_solve (k1, k2, k3 = r). */
int bks_gen_hooi_solve(const bks_tensor* t, const bks_gen_hooi_params* prm, const double* U0,
                       const double* V0, const double* W0, double* U, double* V, double* W,
                       double* F, bks_info* info, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* BKS_GB300_H */
