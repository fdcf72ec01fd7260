// Dense tall-skinny and small-matrix routines of the solvers (FP64 unless a
// template parameter says otherwise).
#pragma once
#include "common.cuh"

namespace bks {

// Workspace for the tall-skinny passes (Gram partials etc.), grown on demand.
struct DenseWork {
  DevBuf gpart;   // double [grid][(K+b) x b] Gram partials
  DevBuf gram;    // double [(K+b) x b]
  DevBuf gram2;   // double [(K+b) x b] (gradient pass)
  DevBuf small;   // double scratch for the small matrices
  DevBuf status;  // int [48]: kept/deferred counts, flags, deferred positions
  DevBuf gtmp;    // double [m x g] gradient pass output
  DevBuf gmat;    // gradient pass small matrices
  DevBuf raw2;    // raw column norms handed to the second level
  int grid = 0;
  int ensure(int K, int b, cudaStream_t s);
};

struct OrthOpts {
  double drop_tol = 0.0;          // rank-drop threshold relative to the raw column norm
  int cap = 1 << 30;              // at most this many new columns
  bool two_level = false;         // defer unresolved columns to a second level (needs B = Q + ldq*K)
  bool fast_first = false;        // first projection round and its Gram in FP32 arithmetic
  const double* raw = nullptr;    // device raw column norms (b) to test drops against, or null
  double* raw_out = nullptr;      // device: receives the raw column norms
  double* grad_out = nullptr;     // device scalar: ||(B - Q H) M||_F^2 (projected block times M)
  const double* grad_mat = nullptr;  // M (b x grad_cols, ld b); null: M = H^T
  int grad_cols = 0;
  double* h_out_early = nullptr;  // device K x b: the projection coefficients H
  int depth = 0;                  // deferral level (internal)
};

// Block Gram-Schmidt + thin QR of B (m x b) against the orthonormal Q
// (m x K) (Algorithm 3 steps (ii)-(iv), Appendix B): on return
// B[:, 0:bo] holds the new orthonormal columns (dropped columns removed).
// Single-level mode also returns H (K x b, ld K) and R (bo x b, ld b) with
// B_in = Q H + B_out R up to the dropped residuals.  With `fast_first` the
// first projection round and the Gram of the first Cholesky QR run in FP32
// arithmetic (for blocks that carry FP32 rounding already); the second
// projection and Cholesky QR stay FP64.
int orth_block(const double* Q, int64_t ldq, int K, double* B, int64_t ldb, int b, int64_t m,
               const OrthOpts& o, double* H, double* R, int* bo_host, DenseWork& ws,
               cudaStream_t s);

// Out (m x bo) = B (m x b) * Mb (b x bo) - Q (m x K) * Mq (K x bo); device
// small matrices (column-major, ld = rows).  Out may alias B or Q columns
// only when every row is read before it is written (tiles are disjoint).
int ts_combine(const double* Q, int64_t ldq, int K, const double* B, int64_t ldb, int b,
               const double* Mq, const double* Mb, int bo, double* Out, int64_t ldo, int64_t m,
               DenseWork& ws, cudaStream_t s);

// Out = B Mb - Q Mq (as ts_combine) and G ((K+bo) x bo) = [Q Out]^T Out.
int ts_combine_gram(const double* Q, int64_t ldq, int K, const double* B, int64_t ldb, int b,
                    const double* Mq, const double* Mb, int bo, double* Out, int64_t ldo,
                    int64_t m, double* G, DenseWork& ws, cudaStream_t s);

// G ((K+b) x b, ld K+b) = [Q B]^T B: rows 0..K-1 hold Q^T B, the rest B^T B.
int ts_gram(const double* Q, int64_t ldq, int K, const double* B, int64_t ldb, int b,
            int64_t m, double* G, DenseWork& ws, cudaStream_t s);

// Column-major -> float copy with a leading dimension
int to_float(const double* X, int64_t ldx, int64_t rows, int cols, float* out, int64_t ldo,
             cudaStream_t s);
int to_double(const float* X, int64_t ldx, int64_t rows, int cols, double* out, int64_t ldo,
              cudaStream_t s);

// r leading left singular vectors of the tall matrix T (m x w): QR by
// orth_block, SVD of the small R by Jacobi, then Out = Qn * Ur.  T is
// overwritten.  Out is m x r (ld ldo).
int top_left_singular(double* T, int64_t ldt, int64_t m, int w, int r, double* Out, int64_t ldo,
                      DenseWork& ws, cudaStream_t s);

// Seeded random start with orthonormal columns (counter-based normal
// variates, then orth_block).
int random_orthonormal(uint64_t seed, uint64_t stream_id, int64_t m, int r, double* Out,
                       DenseWork& ws, cudaStream_t s);

}  // namespace bks
