// Tall-skinny block orthogonalisation (Algorithm 3 steps (ii)-(iv);
// Appendix B: orthogonalise the contraction result in matrix form by a QR)
// and the small dense helpers of the solvers.
//
// orth_block realises "project twice, then thin QR with rank drops" with
// row-streaming passes over the m rows (the only large dimension):
//   P1  G1 = [Q B]^T B                       (round 1 Gram)
//   P2  B1 = B - Q H1,  G2 = [Q B1]^T B1     (projection + round 2 Gram)
//   P3  Bn = (B1 - Q H2) Rk^-1, G3 = [Q Bn]^T Bn   (Cholesky QR with drops)
//   P4  B  = (Bn - Q H3) R3^-1               (second Cholesky QR)
// Every pass reads each row of Q and B once; the (K+b) x b Gram partials
// are reduced in a fixed order, so the result is bitwise reproducible.
#include <algorithm>
#include <type_traits>

#include "dense.cuh"
#include "jacobi.cuh"

namespace bks {

namespace {

constexpr int kRT = 32;           // rows per tile
constexpr int kTSThreads = 256;
constexpr int kMaxK = 160;        // columns of Q
constexpr int kMaxB = 32;         // columns of B and of the output
constexpr int kGramPerThread = (kMaxK + kMaxB) * kMaxB / kTSThreads;  // 24

// Out = B*Mb - Q*Mq for a tile of rows; optional Gram [Q Out]^T Out.
// CU is the arithmetic type of the update, CG that of the Gram (float for
// the fast first round).  The tile is staged in shared memory in the
// arithmetic type when both are the same (one conversion per element
// loaded, none per multiply-add).  CU = float with CG = double (the FP64
// Gram of a block whose input carries FP32 rounding anyway) stages the
// tile twice, in double for the Gram and in float for the update, and the
// coefficients in float, so that no multiply-add converts.
template <typename CU, typename CG>
__global__ void __launch_bounds__(kTSThreads)
k_ts_pass(const double* __restrict__ Q, int64_t ldq, int K, const double* __restrict__ B,
          int64_t ldb, int b, const double* __restrict__ Mq, const double* __restrict__ Mb,
          int bo, int update, double* __restrict__ Out, int64_t ldo, int gram,
          double* __restrict__ gpart, int64_t m) {
  using ST = typename std::conditional<std::is_same<CU, CG>::value, CG, double>::type;
  constexpr bool kDual = !std::is_same<CU, ST>::value;  // update staged apart, in CU
  extern __shared__ double sm_raw[];
  ST* sm = reinterpret_cast<ST*>(sm_raw);
  const int LD = kRT + 1;
  ST* Qs = sm;                             // [K][LD]
  ST* Bs = Qs + (size_t)K * LD;            // [b][LD]
  ST* Os = Bs + (size_t)b * LD;            // [bo][LD]
  ST* Ms = Os + (size_t)kMaxB * LD;        // Mq [K][bo] then Mb [b][bo]
  // the update's operands: the same arrays, or CU copies after Ms (dual)
  CU* Qu = kDual ? reinterpret_cast<CU*>(Ms + (size_t)(K + b) * kMaxB) : reinterpret_cast<CU*>(Qs);
  CU* Bu = kDual ? Qu + (size_t)K * LD : reinterpret_cast<CU*>(Bs);
  CU* Mu = kDual ? Bu + (size_t)b * LD : reinterpret_cast<CU*>(Ms);
  const int tid = threadIdx.x;
  if (update) {
    for (int x = tid; x < K * bo; x += blockDim.x) Mu[x] = (CU)Mq[(x / bo) + (int64_t)K * (x % bo)];
    for (int x = tid; x < b * bo; x += blockDim.x)
      Mu[K * bo + x] = (CU)Mb[(x / bo) + (int64_t)b * (x % bo)];
  }
  const int ocols = update ? bo : b;
  const int gw = K + ocols;  // Gram rows
  CG acc[kGramPerThread];
#pragma unroll
  for (int u = 0; u < kGramPerThread; ++u) acc[u] = CG(0);
  const int64_t ntiles = (m + kRT - 1) / kRT;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * kRT;
    const int rows = (int)((m - r0) < kRT ? (m - r0) : kRT);
    __syncthreads();
    for (int x = tid; x < (K + b) * kRT; x += blockDim.x) {
      const int c = x / kRT, r = x % kRT;
      double val = 0.0;
      if (r < rows) val = c < K ? Q[r0 + r + ldq * c] : B[r0 + r + ldb * (c - K)];
      (c < K ? Qs + (size_t)c * LD : Bs + (size_t)(c - K) * LD)[r] = (ST)val;
      if (kDual && update) (c < K ? Qu + (size_t)c * LD : Bu + (size_t)(c - K) * LD)[r] = (CU)val;
    }
    __syncthreads();
    const ST* O = Bs;
    if (update) {
      for (int x = tid; x < bo * kRT; x += blockDim.x) {
        const int j = x / kRT, r = x % kRT;
        CU sacc = CU(0);
        for (int d = 0; d < b; ++d) sacc += Bu[d * LD + r] * Mu[K * bo + d * bo + j];
        for (int e = 0; e < K; ++e) sacc -= Qu[e * LD + r] * Mu[e * bo + j];
        Os[j * LD + r] = (ST)sacc;
      }
      __syncthreads();
      for (int x = tid; x < bo * kRT; x += blockDim.x) {
        const int j = x / kRT, r = x % kRT;
        if (r < rows) Out[r0 + r + ldo * j] = (double)Os[j * LD + r];
      }
      O = Os;
    }
    if (gram) {
#pragma unroll
      for (int u = 0; u < kGramPerThread; ++u) {
        const int id = tid + u * kTSThreads;
        if (id < gw * ocols) {
          const int i = id % gw, j = id / gw;
          const ST* zi = i < K ? Qs + (size_t)i * LD : O + (size_t)(i - K) * LD;
          const ST* oj = O + (size_t)j * LD;
          CG s = acc[u];
          for (int r = 0; r < rows; ++r) s += (CG)zi[r] * (CG)oj[r];
          acc[u] = s;
        }
      }
    }
  }
  if (gram) {
    double* dst = gpart + (size_t)blockIdx.x * gw * ocols;
#pragma unroll
    for (int u = 0; u < kGramPerThread; ++u) {
      const int id = tid + u * kTSThreads;
      if (id < gw * ocols) dst[id] = (double)acc[u];
    }
  }
}

// G[e] = sum over the per-block partials.  A block of 8 warps takes 32
// consecutive entries: warp w sums the partials p = w, w+8, ... in
// increasing order, then lane-wise the 8 warp sums are added in warp order
// (a fixed order: the result does not depend on the launch).
constexpr int kReduceWarps = 8;
__global__ void __launch_bounds__(32 * kReduceWarps)
k_gram_reduce(const double* __restrict__ gpart, int nparts, int count, double* __restrict__ G) {
  __shared__ double part[kReduceWarps][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + lane;
  double s = 0.0;
  if (e < count)
    for (int p = w; p < nparts; p += kReduceWarps) s += gpart[(size_t)p * count + e];
  part[w][lane] = s;
  __syncthreads();
  if (w == 0 && e < count) {
    double t = part[0][lane];
    for (int q = 1; q < kReduceWarps; ++q) t += part[q][lane];
    G[e] = t;
  }
}

void gram_reduce(const double* gpart, int nparts, int count, double* G, cudaStream_t s) {
  k_gram_reduce<<<std::max(1, (count + 31) / 32), 32 * kReduceWarps, 0, s>>>(gpart, nparts,
                                                                             count, G);
  ::bks::note_launch();
}

// small-matrix scratch layout (doubles), all column-major
struct SmallLayout {
  int K, b;
  size_t H, raw, Mq, Mb, R2, R3, Rinv, kept;
  size_t total;
  __host__ __device__ SmallLayout(int K_, int b_) : K(K_), b(b_) {
    size_t o = 0;
    H = o; o += (size_t)K * b;
    raw = o; o += b;
    Mq = o; o += (size_t)K * b;
    Mb = o; o += (size_t)b * b;
    R2 = o; o += (size_t)b * b;
    R3 = o; o += (size_t)b * b;
    Rinv = o; o += (size_t)b * b;
    kept = o; o += b;
    total = o;
  }
};

// Round 1: H1 = Q^T B, raw column norms, Mq = H1, Mb = I.
__global__ void k_orth_r1(const double* __restrict__ G, int K, int b, double* __restrict__ sm) {
  SmallLayout L(K, b);
  const int gw = K + b;
  for (int x = threadIdx.x; x < K * b; x += blockDim.x) {
    const int i = x % K, j = x / K;
    sm[L.H + x] = G[i + gw * j];
    sm[L.Mq + x] = G[i + gw * j];
  }
  for (int x = threadIdx.x; x < b * b; x += blockDim.x) sm[L.Mb + x] = (x % b == x / b) ? 1.0 : 0.0;
  for (int c = threadIdx.x; c < b; c += blockDim.x) sm[L.raw + c] = sqrt(fmax(G[K + c + gw * c], 0.0));
}

// Round 2: H2 = Q^T B1, S = B1^T B1 - H2^T H2 and a left-to-right Cholesky
// pass.  Column c has the residual d_c after projection on Q and the kept
// columns to its left.  A Gram matrix holds d_c to a few digits only while
// the column is not nearly dependent on those columns, so:
//   sqrt(d_c) > 1e-3 ||(I-QQ^T) b_c||  (resolved): kept if
//       sqrt(d_c) > drop_tol ||b_c|| (the rank-drop rule; the paper gives
//       none), else dropped;
//   otherwise: this column and every column to its right are deferred
//       (two-level mode) to a further pass against [Q, kept columns],
//       where their Gram is formed from re-projected vectors; without
//       two-level mode they are dropped.
// The first column of any pass is always resolved, so every pass decides
// at least one column.  The order of the kept columns is the left-to-right
// order of a column-by-column Gram-Schmidt.
// The output of P3 is [kept columns (Rk^-1 QR) | deferred columns (second
// projection only)]: Mb = [Rk^-1 on kept rows | selection of deferred],
// Mq = [H2[:,kept] Rk^-1 | H2[:,deferred]].
__global__ void k_orth_r2(const double* __restrict__ G, int K, int b, double drop_tol, int cap,
                          int two_level, const double* __restrict__ raw_in,
                          double* __restrict__ sm, int* __restrict__ status) {
  SmallLayout L(K, b);
  const int gw = K + b;
  __shared__ double S[kMaxB * kMaxB];
  __shared__ double R[kMaxB * kMaxB];
  __shared__ int pos[kMaxB];
  __shared__ int dpos[kMaxB];
  __shared__ double Sd[kMaxB];  // the projected diagonal before elimination
  for (int x = threadIdx.x; x < b * b; x += blockDim.x) {
    const int i = x % b, j = x / b;
    double s = G[K + i + gw * j];
    for (int e = 0; e < K; ++e) s -= G[e + gw * i] * G[e + gw * j];
    S[x] = s;
    R[x] = 0.0;
    if (i == j) Sd[i] = s;
  }
  if (raw_in)
    for (int c = threadIdx.x; c < b; c += blockDim.x) sm[L.raw + c] = raw_in[c];
  __syncthreads();
  // Right-looking form of the left-to-right elimination: after column c is
  // kept as the t-th column, every later column c' gets R[t, c'] (one
  // division per column, in parallel) and the trailing Gram entries lose
  // R[t, c'] R[t, c''], in the same order of t as a column-by-column
  // substitution.  Thread 0 only takes the per-column decisions.
  __shared__ int s_nk, s_nd, s_def, s_cls;
  if (threadIdx.x == 0) { s_nk = 0; s_nd = 0; s_def = 0; }
  __syncthreads();
  for (int c = 0; c < b; ++c) {
    if (threadIdx.x == 0) {
      int cls = 0;  // 0 drop, 1 keep, 2 defer
      if (s_def) {
        cls = 2;
      } else {
        const int nk = s_nk;
        const double d = S[c + b * c];  // the trailing diagonal: d_c
        const double raw = sm[L.raw + c];
        const double res = sqrt(fmax(d, 0.0));
        const double proj = sqrt(fmax(Sd[c], 0.0));
        // with no kept column before it at this level, d_c is the Gram
        // diagonal itself and is always resolved (every level decides at
        // least its first column)
        const bool resolved = nk == 0 || res > 1e-3 * proj;
        if (nk < cap && raw > 0.0) {
          if (resolved) cls = res > drop_tol * raw ? 1 : 0;
          else if (two_level) { cls = 2; s_def = 1; }
        }
        if (cls == 1) {
          R[nk + b * c] = res;
          pos[nk] = c;
        }
      }
      if (cls == 2) dpos[s_nd++] = c;
      sm[L.kept + c] = cls;
      s_cls = cls;
    }
    __syncthreads();
    if (s_cls != 1) continue;
    const int t = s_nk;
    const double rcc = R[t + b * c];
    for (int c2 = c + 1 + threadIdx.x; c2 < b; c2 += blockDim.x) R[t + b * c2] = S[c + b * c2] / rcc;
    __syncthreads();
    for (int x = threadIdx.x; x < b * b; x += blockDim.x) {
      const int i = x % b, j = x / b;
      if (i > c && j >= i) S[i + b * j] -= R[t + b * i] * R[t + b * j];
    }
    __syncthreads();
    if (threadIdx.x == 0) s_nk = t + 1;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    // rows of R for deferred columns stay zero, as in the column form
    for (int t = 0; t < s_nd; ++t)
      for (int u = 0; u < s_nk; ++u) R[u + b * dpos[t]] = 0.0;
    status[0] = s_nk;
    status[2] = s_nd;
    for (int t = 0; t < s_nd; ++t) status[8 + t] = dpos[t];
  }
  __syncthreads();
  const int nk = status[0], nd = status[2];
  const int no = nk + nd;
  for (int x = threadIdx.x; x < b * b; x += blockDim.x) sm[L.R2 + x] = ((x % b) < nk) ? R[x] : 0.0;
  for (int x = threadIdx.x; x < K * b; x += blockDim.x) {
    const int i = x % K, j = x / K;
    sm[L.H + x] += G[i + gw * j];
  }
  __syncthreads();
  double* Ri = sm + L.Rinv;  // nk x nk, ld b
  __shared__ double dinv2[kMaxB];
  for (int i = threadIdx.x; i < nk; i += blockDim.x) dinv2[i] = 1.0 / R[i + b * pos[i]];
  __syncthreads();
  for (int j = threadIdx.x; j < nk; j += blockDim.x) {
    for (int i = nk - 1; i >= 0; --i) {
      double v = (i == j) ? 1.0 : 0.0;
      for (int t = i + 1; t <= j; ++t) v -= R[i + b * pos[t]] * Ri[t + b * j];
      Ri[i + b * j] = (i <= j) ? v * dinv2[i] : 0.0;
    }
  }
  __syncthreads();
  // Mb (b x no, ld b)
  for (int x = threadIdx.x; x < b * no; x += blockDim.x) {
    const int c = x % b, j = x / b;
    double v = 0.0;
    if (j < nk) {
      for (int t = 0; t < nk; ++t)
        if (pos[t] == c) v = Ri[t + b * j];
    } else {
      v = (dpos[j - nk] == c) ? 1.0 : 0.0;
    }
    sm[L.Mb + x] = v;
  }
  // Mq (K x no, ld K)
  for (int x = threadIdx.x; x < K * no; x += blockDim.x) {
    const int i = x % K, j = x / K;
    double v = 0.0;
    if (j < nk) {
      for (int t = 0; t <= j; ++t) v += G[i + gw * pos[t]] * Ri[t + b * j];
    } else {
      v = G[i + gw * dpos[j - nk]];
    }
    sm[L.Mq + x] = v;
  }
}

// Gradient pass matrices: gradM (b x g) = (H)^T when `use_h`, else the
// caller's matrix; Mq' = H2 gradM with H2 = Q^T B1 (the second projection).
__global__ void k_grad_prep(const double* __restrict__ G, int K, int b, const double* __restrict__ sm_h,
                            const double* __restrict__ ext, int g, double* __restrict__ gM,
                            double* __restrict__ gQ) {
  const int gw = K + b;
  for (int x = threadIdx.x; x < b * g; x += blockDim.x) {
    const int d = x % b, j = x / b;
    gM[x] = ext ? ext[d + (int64_t)b * j] : sm_h[j + (int64_t)K * d];
  }
  __syncthreads();
  for (int x = threadIdx.x; x < K * g; x += blockDim.x) {
    const int i = x % K, j = x / K;
    double v = 0.0;
    for (int d = 0; d < b; ++d) v += G[i + gw * d] * gM[d + (int64_t)b * j];
    gQ[x] = v;
  }
}

// sum of the diagonal of the output block of a reduced Gram [Q O]^T O
__global__ void k_gram_trace(const double* __restrict__ G, int K, int g, double* __restrict__ out) {
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int j = 0; j < g; ++j) s += G[K + j + (int64_t)(K + g) * j];
    *out = s;
  }
}

// Round 3 on the kept columns (the first nk of the P3 output, which has
// no = nk + nd columns): S3 = R3^T R3; Mb = [R3^-1 | I], Mq = [H3 R3^-1 | 0];
// final H = H + H3 R2 (kept part), R = R3 R2.
__global__ void k_orth_r3(const double* __restrict__ G, int K, int b, double* __restrict__ sm,
                          const int* __restrict__ status, double* __restrict__ Hout,
                          double* __restrict__ Rout, int* __restrict__ flags) {
  SmallLayout L(K, b);
  const int nk = status[0], nd = status[2];
  const int no = nk + nd;
  const int gw = K + no;
  __shared__ double R3[kMaxB * kMaxB];
  __shared__ double Ri[kMaxB * kMaxB];
  // S3 = Bn^T Bn - H3^T H3 on the kept columns (all entries in parallel),
  // then its Cholesky factor on one thread (nk^3/6 operations)
  for (int x = threadIdx.x; x < nk * nk; x += blockDim.x) {
    const int i = x % nk, j = x / nk;
    if (i > j) continue;
    double v = G[K + i + gw * j];
    for (int e = 0; e < K; ++e) v -= G[e + gw * i] * G[e + gw * j];
    Ri[i + kMaxB * j] = v;
  }
  __syncthreads();
  // right-looking Cholesky: one pivot per step, the row and the trailing
  // update in parallel (the same order of subtraction as a column-by-column
  // factorisation)
  for (int c = 0; c < nk; ++c) {
    if (threadIdx.x == 0) {
      double v = Ri[c + kMaxB * c];
      if (!(v > 0.0)) { flags[0] = 1; v = 1e-300; }
      R3[c + kMaxB * c] = sqrt(v);
    }
    __syncthreads();
    const double rcc = R3[c + kMaxB * c];
    for (int c2 = c + 1 + threadIdx.x; c2 < nk; c2 += blockDim.x)
      R3[c + kMaxB * c2] = Ri[c + kMaxB * c2] / rcc;
    __syncthreads();
    for (int x = threadIdx.x; x < nk * nk; x += blockDim.x) {
      const int i = x % nk, j = x / nk;
      if (i > c && j >= i) Ri[i + kMaxB * j] -= R3[c + kMaxB * i] * R3[c + kMaxB * j];
    }
    __syncthreads();
  }
  __shared__ double dinv3[kMaxB];
  for (int x = threadIdx.x; x < nk * nk; x += blockDim.x) {
    const int i = x % nk, j = x / nk;
    if (i > j) R3[i + kMaxB * j] = 0.0;
  }
  for (int i = threadIdx.x; i < nk; i += blockDim.x) dinv3[i] = 1.0 / R3[i + kMaxB * i];
  __syncthreads();
  for (int j = threadIdx.x; j < nk; j += blockDim.x) {
    for (int i = nk - 1; i >= 0; --i) {
      double v = (i == j) ? 1.0 : 0.0;
      for (int t = i + 1; t <= j; ++t) v -= R3[i + kMaxB * t] * Ri[t + kMaxB * j];
      Ri[i + kMaxB * j] = (i <= j) ? v * dinv3[i] : 0.0;
    }
  }
  __syncthreads();
  for (int x = threadIdx.x; x < no * no; x += blockDim.x) {
    const int i = x % no, j = x / no;
    double v;
    if (i < nk && j < nk) v = Ri[i + kMaxB * j];
    else v = (i == j) ? 1.0 : 0.0;
    sm[L.Mb + i + (size_t)no * j] = v;
  }
  for (int x = threadIdx.x; x < K * no; x += blockDim.x) {
    const int i = x % K, j = x / K;
    double v = 0.0;
    if (j < nk)
      for (int t = 0; t <= j; ++t) v += G[i + gw * t] * Ri[t + kMaxB * j];
    sm[L.Mq + x] = v;
  }
  for (int x = threadIdx.x; x < K * b; x += blockDim.x) {
    const int i = x % K, j = x / K;
    double v = sm[L.H + x];
    for (int t = 0; t < nk; ++t) v += G[i + gw * t] * sm[L.R2 + t + (size_t)b * j];
    if (Hout) Hout[x] = v;
  }
  for (int x = threadIdx.x; x < b * b; x += blockDim.x) {
    const int i = x % b, j = x / b;
    double v = 0.0;
    if (i < nk)
      for (int t = i; t < nk; ++t) v += R3[i + kMaxB * t] * sm[L.R2 + t + (size_t)b * j];
    if (Rout) Rout[x] = v;
  }
}

__global__ void k_copy_small(const double* __restrict__ src, double* __restrict__ dst, int n) {
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x)
    dst[x] = src[x];
}

template <typename CU, typename CG>
size_t ts_smem(int K, int b) {
  using ST = typename std::conditional<std::is_same<CU, CG>::value, CG, double>::type;
  const int LD = kRT + 1;
  size_t bytes = sizeof(ST) * ((size_t)(K + b + kMaxB) * LD + (size_t)(K + b) * kMaxB);
  if (!std::is_same<CU, ST>::value)
    bytes += sizeof(CU) * ((size_t)(K + b) * LD + (size_t)(K + b) * kMaxB);
  return bytes;
}

template <typename CU, typename CG>
int launch_ts(const double* Q, int64_t ldq, int K, const double* B, int64_t ldb, int b,
              const double* Mq, const double* Mb, int bo, int update, double* Out, int64_t ldo,
              int gram, double* gpart, int64_t m, int grid, cudaStream_t s) {
  const size_t smem = ts_smem<CU, CG>(K, b);
  // the shared-memory limit is raised once per kernel and device, to the
  // largest tile any call stages (the batch and serving workers launch
  // these kernels from several host threads)
  static PerDeviceOnce once;
  const cudaError_t attr = once.run([] {
    return cudaFuncSetAttribute(k_ts_pass<CU, CG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ts_smem<CU, CG>(kMaxK, kMaxB));
  });
  if (attr != cudaSuccess)
    return fail(BKS_ECUDA, std::string("k_ts_pass shared-memory limit: ") + cudaGetErrorString(attr));
  k_ts_pass<CU, CG><<<grid, kTSThreads, smem, s>>>(Q, ldq, K, B, ldb, b, Mq, Mb, bo, update, Out,
                                                   ldo, gram, gpart, m); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  return BKS_OK;
}

int gram_grid(int64_t m) {
  int64_t tiles = (m + kRT - 1) / kRT;
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, 2LL * num_sms()));
}

}  // namespace

int DenseWork::ensure(int K, int b, cudaStream_t s) {
  const int g = 2 * num_sms();
  const size_t need = (size_t)g * (kMaxK + kMaxB) * kMaxB;
  if (gpart.bytes < need * sizeof(double)) BKS_TRY(gpart.alloc(need * sizeof(double), s));
  if (gram.bytes < (size_t)(kMaxK + kMaxB) * kMaxB * sizeof(double))
    BKS_TRY(gram.alloc((size_t)(kMaxK + kMaxB) * kMaxB * sizeof(double), s));
  SmallLayout L(kMaxK, kMaxB);
  if (small.bytes < L.total * sizeof(double)) BKS_TRY(small.alloc(L.total * sizeof(double), s));
  if (status.bytes < 48 * sizeof(int)) BKS_TRY(status.alloc(48 * sizeof(int), s));
  if (gram2.bytes < (size_t)(kMaxK + kMaxB) * kMaxB * sizeof(double))
    BKS_TRY(gram2.alloc((size_t)(kMaxK + kMaxB) * kMaxB * sizeof(double), s));
  grid = g;
  (void)K; (void)b;
  return BKS_OK;
}

int orth_block(const double* Q, int64_t ldq, int K, double* B, int64_t ldb, int b, int64_t m,
               const OrthOpts& o, double* H, double* R, int* bo_host, DenseWork& ws,
               cudaStream_t s) {
  if (b <= 0) {
    *bo_host = 0;
    return BKS_OK;
  }
  if (K > kMaxK || b > kMaxB)
    return fail(BKS_EUNSUPPORTED, "block orthogonalisation: basis above 160 or block above 32 columns");
  if (o.two_level && B != Q + ldq * K)
    return fail(BKS_EINVAL, "two-level orthogonalisation needs B to follow Q in one array");
  BKS_TRY(ws.ensure(K, b, s));
  const int grid = gram_grid(m);
  double* sm = ws.small.as<double>();
  SmallLayout L(K, b);
  int* st = ws.status.as<int>();
  BKS_CUDA_TRY(cudaMemsetAsync(st, 0, 48 * sizeof(int), s));
  const int gw = K + b;
  auto reduce = [&](int count) {
    gram_reduce(ws.gpart.as<double>(), grid, count, ws.gram.as<double>(), s);
  };
  // P1: Gram of [Q B]^T B (first projection coefficients)
  if (o.fast_first)
    BKS_TRY((launch_ts<float, float>(Q, ldq, K, B, ldb, b, nullptr, nullptr, b, 0, nullptr, 0, 1,
                                    ws.gpart.as<double>(), m, grid, s)));
  else
    BKS_TRY((launch_ts<double, double>(Q, ldq, K, B, ldb, b, nullptr, nullptr, b, 0, nullptr, 0, 1,
                                      ws.gpart.as<double>(), m, grid, s)));
  reduce(gw * b);
  k_orth_r1<<<1, 256, 0, s>>>(ws.gram.as<double>(), K, b, sm); ::bks::note_launch();
  // P2: B1 = B - Q H1 (in place) and the Gram of [Q B1]^T B1 (FP32 with
  // fast_first: the input block then carries FP32 rounding anyway, the
  // first Cholesky from it only has to leave a well-conditioned block for
  // the FP64 round P3/P4, and the deferral test res > 1e-3 proj needs a
  // few digits of res only)
  if (o.fast_first)
    BKS_TRY((launch_ts<float, float>(Q, ldq, K, B, ldb, b, sm + L.Mq, sm + L.Mb, b, 1, B, ldb, 1,
                                     ws.gpart.as<double>(), m, grid, s)));
  else
    BKS_TRY((launch_ts<double, double>(Q, ldq, K, B, ldb, b, sm + L.Mq, sm + L.Mb, b, 1, B, ldb, 1,
                                      ws.gpart.as<double>(), m, grid, s)));
  reduce(gw * b);
  k_orth_r2<<<1, 256, 0, s>>>(ws.gram.as<double>(), K, b, o.drop_tol, o.cap, o.two_level ? 1 : 0,
                              o.raw, sm, st); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  if (o.raw_out) {
    k_copy_small<<<1, 32, 0, s>>>(sm + L.raw, o.raw_out, b); ::bks::note_launch();
  }
  // optional gradient pass: || (B1 - Q H2) gradM ||_F^2
  if (o.grad_out) {
    const int g = o.grad_cols;
    if (ws.gtmp.bytes < sizeof(double) * (size_t)m * g) BKS_TRY(ws.gtmp.alloc(sizeof(double) * m * g, s));
    if (ws.gmat.bytes < sizeof(double) * (size_t)(kMaxB + kMaxK) * kMaxB)
      BKS_TRY(ws.gmat.alloc(sizeof(double) * (kMaxB + kMaxK) * kMaxB, s));
    double* gM = ws.gmat.as<double>();
    double* gQ = gM + (size_t)b * g;
    k_grad_prep<<<1, 256, 0, s>>>(ws.gram.as<double>(), K, b, sm + L.H, o.grad_mat, g, gM, gQ); ::bks::note_launch();
    BKS_TRY((launch_ts<double, double>(Q, ldq, K, B, ldb, b, gQ, gM, g, 1, ws.gtmp.as<double>(), m, 1,
                                      ws.gpart.as<double>(), m, grid, s)));
    gram_reduce(ws.gpart.as<double>(), grid, (K + g) * g, ws.gram2.as<double>(), s);
    k_gram_trace<<<1, 32, 0, s>>>(ws.gram2.as<double>(), K, g, o.grad_out); ::bks::note_launch();
    BKS_CUDA_TRY(cudaGetLastError());
  }
  if (o.h_out_early) {
    k_copy_small<<<1, 256, 0, s>>>(sm + L.H, o.h_out_early, K * b); ::bks::note_launch();
  }
  int hst[40];
  BKS_CUDA_TRY(cudaMemcpyAsync(hst, st, 40 * sizeof(int), cudaMemcpyDeviceToHost, s));
  BKS_CUDA_TRY(cudaStreamSynchronize(s));
  const int nk = hst[0], nd = hst[2], no = nk + nd;
  if (no == 0) {
    *bo_host = 0;
    if (H) {
      k_copy_small<<<1, 256, 0, s>>>(sm + L.H, H, K * b); ::bks::note_launch();
      BKS_CUDA_TRY(cudaGetLastError());
    }
    return BKS_OK;
  }
  // P3: [Bn | D] = B1 Mb - Q Mq (no columns, in place) and its Gram in
  // FP64 (with fast_first the update in FP32: B1 carries FP32 rounding
  // already, and P4 takes Bn to FP64 orthogonality from this FP64 Gram)
  const int gw3 = K + no;
  if (o.fast_first)
    BKS_TRY((launch_ts<float, double>(Q, ldq, K, B, ldb, b, sm + L.Mq, sm + L.Mb, no, 1, B, ldb, 1,
                                      ws.gpart.as<double>(), m, grid, s)));
  else
    BKS_TRY((launch_ts<double, double>(Q, ldq, K, B, ldb, b, sm + L.Mq, sm + L.Mb, no, 1, B, ldb, 1,
                                      ws.gpart.as<double>(), m, grid, s)));
  reduce(gw3 * no);
  k_orth_r3<<<1, 256, 0, s>>>(ws.gram.as<double>(), K, b, sm, st, H, R, st + 1); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  // P4: kept columns <- Bn R3^-1 - Q H3 R3^-1; deferred columns unchanged
  BKS_TRY((launch_ts<double, double>(Q, ldq, K, B, ldb, no, sm + L.Mq, sm + L.Mb, no, 1, B, ldb, 0,
                                    nullptr, m, grid, s)));
  int bo = nk;
  if (nd > 0) {
    // second level: the deferred columns against [Q, kept columns]
    if (ws.raw2.bytes < sizeof(double) * kMaxB) BKS_TRY(ws.raw2.alloc(sizeof(double) * kMaxB, s));
    std::vector<double> rawh(b);
    BKS_CUDA_TRY(cudaMemcpyAsync(rawh.data(), sm + L.raw, sizeof(double) * b, cudaMemcpyDeviceToHost, s));
    BKS_CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<double> rawd(nd);
    for (int t = 0; t < nd; ++t) rawd[t] = rawh[hst[8 + t]];
    BKS_CUDA_TRY(cudaMemcpyAsync(ws.raw2.p, rawd.data(), sizeof(double) * nd, cudaMemcpyHostToDevice, s));
    BKS_CUDA_TRY(cudaStreamSynchronize(s));
    OrthOpts o2;
    o2.drop_tol = o.drop_tol;
    o2.cap = o.cap - nk;
    o2.two_level = nd > 1;  // the suffix's first column is always decided
    o2.depth = o.depth + 1;
    if (o2.depth > kMaxB + 1) return fail(BKS_EBREAKDOWN, "block QR: deferral did not terminate");
    o2.fast_first = false;
    o2.raw = ws.raw2.as<double>();
    int bo2 = 0;
    BKS_TRY(orth_block(Q, ldq, K + nk, B + ldb * nk, ldb, nd, m, o2, nullptr, nullptr, &bo2, ws, s));
    bo += bo2;
  }
  *bo_host = bo;
  return BKS_OK;
}

int ts_combine(const double* Q, int64_t ldq, int K, const double* B, int64_t ldb, int b,
               const double* Mq, const double* Mb, int bo, double* Out, int64_t ldo, int64_t m,
               DenseWork& ws, cudaStream_t s) {
  if (K > kMaxK || b > kMaxB || bo > kMaxB)
    return fail(BKS_EUNSUPPORTED, "tall-skinny combine: sizes above 160/32/32");
  BKS_TRY(ws.ensure(K, b, s));
  return launch_ts<double, double>(Q, ldq, K, B, ldb, b, Mq, Mb, bo, 1, Out, ldo, 0, nullptr, m,
                                   gram_grid(m), s);
}

int ts_gram(const double* Q, int64_t ldq, int K, const double* B, int64_t ldb, int b,
            int64_t m, double* G, DenseWork& ws, cudaStream_t s) {
  if (K > kMaxK || b > kMaxB) return fail(BKS_EUNSUPPORTED, "tall-skinny Gram: sizes above 160/32");
  BKS_TRY(ws.ensure(K, b, s));
  const int grid = gram_grid(m);
  BKS_TRY((launch_ts<double, double>(Q, ldq, K, B, ldb, b, nullptr, nullptr, b, 0, nullptr, 0, 1,
                                     ws.gpart.as<double>(), m, grid, s)));
  gram_reduce(ws.gpart.as<double>(), grid, (K + b) * b, G, s);
  BKS_CUDA_TRY(cudaGetLastError());
  return BKS_OK;
}

int ts_combine_gram(const double* Q, int64_t ldq, int K, const double* B, int64_t ldb, int b,
                    const double* Mq, const double* Mb, int bo, double* Out, int64_t ldo,
                    int64_t m, double* G, DenseWork& ws, cudaStream_t s) {
  if (K > kMaxK || b > kMaxB || bo > kMaxB)
    return fail(BKS_EUNSUPPORTED, "tall-skinny combine: sizes above 160/32/32");
  BKS_TRY(ws.ensure(K, b, s));
  const int grid = gram_grid(m);
  BKS_TRY((launch_ts<double, double>(Q, ldq, K, B, ldb, b, Mq, Mb, bo, 1, Out, ldo, 1,
                                     ws.gpart.as<double>(), m, grid, s)));
  gram_reduce(ws.gpart.as<double>(), grid, (K + bo) * bo, G, s);
  BKS_CUDA_TRY(cudaGetLastError());
  return BKS_OK;
}

namespace {
template <typename A, typename Bt>
__global__ void k_cast2d(const A* __restrict__ X, int64_t ldx, int64_t rows, int cols,
                         Bt* __restrict__ out, int64_t ldo) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < rows * cols;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t % rows, c = t / rows;
    out[r + ldo * c] = (Bt)X[r + ldx * c];
  }
}
inline int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)num_sms() * 32));
}

// left singular vectors of the small R (bo x w): eigenvectors of R R^T
__global__ void k_small_left(const double* __restrict__ R, int ldr, int bo, int w, int r,
                             double* __restrict__ Ur) {
  __shared__ double A[kMaxB * kMaxB];
  __shared__ double V[kMaxB * kMaxB];
  __shared__ double red[64];
  __shared__ double cs[4 * kMaxB + 64];
  __shared__ int idx[kMaxB];
  for (int x = threadIdx.x; x < bo * bo; x += blockDim.x) {
    const int i = x % bo, j = x / bo;
    double v = 0.0;
    for (int t = 0; t < w; ++t) v += R[i + (int64_t)ldr * t] * R[j + (int64_t)ldr * t];
    A[i * bo + j] = v;
  }
  __syncthreads();
  block_jacobi_eig<double>(A, V, bo, 0.0, 40, red, cs);
  top_diag<double>(A, bo, r, idx);
  for (int x = threadIdx.x; x < bo * r; x += blockDim.x) {
    const int i = x % bo, t = x / bo;
    Ur[i + (int64_t)bo * t] = V[i * bo + idx[t]];
  }
}

__device__ __forceinline__ uint64_t splitmix(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// N(0,1) variates by Box-Muller on counter-hashed uniforms
__global__ void k_randn(uint64_t seed, uint64_t sid, int64_t count, double* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x) {
    uint64_t h1 = splitmix(seed ^ splitmix(sid * 0x100000001B3ull + 2 * (uint64_t)t));
    uint64_t h2 = splitmix(h1 + 0x632BE59BD9B4E019ull);
    double u1 = ((h1 >> 11) + 1) * (1.0 / 9007199254740993.0);
    double u2 = (h2 >> 11) * (1.0 / 9007199254740992.0);
    out[t] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
  }
}
}  // namespace

int to_float(const double* X, int64_t ldx, int64_t rows, int cols, float* out, int64_t ldo,
             cudaStream_t s) {
  if (rows * cols == 0) return BKS_OK;
  k_cast2d<double, float><<<grid_for(rows * cols), 256, 0, s>>>(X, ldx, rows, cols, out, ldo); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  return BKS_OK;
}
int to_double(const float* X, int64_t ldx, int64_t rows, int cols, double* out, int64_t ldo,
              cudaStream_t s) {
  if (rows * cols == 0) return BKS_OK;
  k_cast2d<float, double><<<grid_for(rows * cols), 256, 0, s>>>(X, ldx, rows, cols, out, ldo); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  return BKS_OK;
}

int top_left_singular(double* T, int64_t ldt, int64_t m, int w, int r, double* Out, int64_t ldo,
                      DenseWork& ws, cudaStream_t s) {
  DevBuf Rb, Ur;
  BKS_TRY(Rb.alloc(sizeof(double) * w * w, s));
  int bo = 0;
  OrthOpts o;
  o.drop_tol = 0.0;
  o.cap = w;
  BKS_TRY(orth_block(nullptr, m, 0, T, ldt, w, m, o, nullptr, Rb.as<double>(), &bo, ws, s));
  if (bo < r) return fail(BKS_EBREAKDOWN, "contraction has rank below the target rank");
  BKS_TRY(Ur.alloc(sizeof(double) * bo * r, s));
  k_small_left<<<1, 256, 0, s>>>(Rb.as<double>(), w, bo, w, r, Ur.as<double>()); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  // Out = Qn * Ur  (Qn = T[:, 0:bo])
  return ts_combine(nullptr, m, 0, T, ldt, bo, nullptr, Ur.as<double>(), r, Out, ldo, m, ws, s);
}

int random_orthonormal(uint64_t seed, uint64_t sid, int64_t m, int r, double* Out, DenseWork& ws,
                       cudaStream_t s) {
  k_randn<<<grid_for(m * r), 256, 0, s>>>(seed, sid, m * r, Out); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  DevBuf Rb;
  BKS_TRY(Rb.alloc(sizeof(double) * r * r, s));
  int bo = 0;
  OrthOpts o;
  o.drop_tol = 0.0;
  o.cap = r;
  BKS_TRY(orth_block(nullptr, m, 0, Out, m, r, m, o, nullptr, Rb.as<double>(), &bo, ws, s));
  if (bo < r) return fail(BKS_EBREAKDOWN, "random start lost rank");
  return BKS_OK;
}

}  // namespace bks
