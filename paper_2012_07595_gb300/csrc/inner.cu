// Inner problem of the tensor Krylov-Schur method (Algorithm 5 step (i)):
// the best rank-(r1,r1,r3) approximation of the dense (1,2)-symmetric core
// C = A.(X,X,Z) (k1 x k1 x k3), solved by one cooperative grid kernel.
//
// Section 6.2 starts from the truncated HOSVD of C, runs 5 HOOI sweeps and
// then Newton-Grassmann.  This library's reading: the truncated HOSVD start
// and the current point (Uh = [I;0], Wh = [I;0]) are compared by ||F||; the
// better one continues with symmetric HOOI sweeps until its G-gradient is
// below tol * ||F|| or max_inner sweeps are done.
//
// The HOSVD start only seeds the iteration, so its two Gram matrices and
// their eigenvectors are computed in FP32 (k_hosvd); the sweeps, the
// gradient and every result are FP64.
#include <algorithm>
#include <cmath>

#include <cooperative_groups.h>

#include "common.cuh"
#include "jacobi.cuh"
#include "newton.cuh"

namespace bks {

namespace {

constexpr int kInnerThreads = 512;
constexpr int kMaxR = 8;                 // r1, r3 <= 8
constexpr int kMaxW = kMaxR * kMaxR;     // r1^2 <= 64
constexpr int kMaxW1 = 32;               // r1*r3 <= 32

inline int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)num_sms() * 32));
}

// G1 = unfold1(C) unfold1(C)^T (k1 x k1), G3 = unfold3(C) unfold3(C)^T
// (k3 x k3), in FP32, split over blocks along the summed index; partials
// are summed in a fixed order by k_hosvd.
__global__ void k_hosvd_grams(const double* __restrict__ C, int k1, int k3,
                              float* __restrict__ part1, float* __restrict__ part3) {
  // block b sums slices c in [c0, c1) for G1, and rows a-pairs for G3
  const int nb = gridDim.x;
  const int tid = threadIdx.x;
  // G1 part: sum over (b, c) with c in this block's range
  const int c0 = (int)((int64_t)k3 * blockIdx.x / nb), c1 = (int)((int64_t)k3 * (blockIdx.x + 1) / nb);
  for (int x = tid; x < k1 * k1; x += blockDim.x) {
    const int a = x % k1, a2 = x / k1;
    float s = 0.f;
    for (int c = c0; c < c1; ++c)
      for (int b = 0; b < k1; ++b)
        s += (float)C[a + (int64_t)k1 * (b + (int64_t)k1 * c)] *
             (float)C[a2 + (int64_t)k1 * (b + (int64_t)k1 * c)];
    part1[(int64_t)blockIdx.x * k1 * k1 + x] = s;
  }
  // G3 part: sum over pairs (a, b) with b in this block's range
  const int b0 = (int)((int64_t)k1 * blockIdx.x / nb), b1 = (int)((int64_t)k1 * (blockIdx.x + 1) / nb);
  for (int x = tid; x < k3 * k3; x += blockDim.x) {
    const int c = x % k3, c2 = x / k3;
    float s = 0.f;
    for (int b = b0; b < b1; ++b)
      for (int a = 0; a < k1; ++a)
        s += (float)C[a + (int64_t)k1 * (b + (int64_t)k1 * c)] *
             (float)C[a + (int64_t)k1 * (b + (int64_t)k1 * c2)];
    part3[(int64_t)blockIdx.x * k3 * k3 + x] = s;
  }
}

// Eigenvectors of the two Grams (FP32 Jacobi), r leading ones -> FP64.
__global__ void __launch_bounds__(kInnerThreads)
k_hosvd(const float* __restrict__ part1, const float* __restrict__ part3, int nparts, int k1,
        int k3, int r1, int r3, double* __restrict__ Uh, double* __restrict__ Wh) {
  extern __shared__ float shf[];
  const int nmax = max(k1, k3);
  float* A = shf;
  float* V = A + nmax * nmax;
  float* red = V + nmax * nmax;
  float* cs = red + 64;
  __shared__ int idx[kMaxR];
  {
    const int pass = blockIdx.x;  // block 0: the mode-1 Gram, block 1: the mode-3 Gram
    const int n = pass == 0 ? k1 : k3;
    const int r = pass == 0 ? r1 : r3;
    const float* part = pass == 0 ? part1 : part3;
    for (int x = threadIdx.x; x < n * n; x += blockDim.x) {
      float s = 0.f;
      for (int p = 0; p < nparts; ++p) s += part[(int64_t)p * n * n + x];
      A[x] = s;
    }
    __syncthreads();
    // a start only: a relative threshold of 1e-4 and at most 6 sweeps
    block_jacobi_eig<float>(A, V, n, 1e-4f, 6, red, cs);
    top_diag<float>(A, n, r, idx);
    double* out = pass == 0 ? Uh : Wh;
    for (int x = threadIdx.x; x < n * r; x += blockDim.x) {
      const int i = x % n, t = x / n;
      out[x] = (double)V[i * n + idx[t]];
    }
    __syncthreads();
  }
}

// ---- FP64 symmetric HOOI on the core --------------------------------------
struct InnerShared {
  double Uh[128 * kMaxR];
  double Wh[128 * kMaxR];
  double T1[128 * kMaxW1];   // k1 x (r1 r3), column b + r1 c
  double T3[128 * kMaxW];    // k3 x r1^2,    column a + r1 b
  double G[kMaxW * kMaxW];   // small Gram
  double V[kMaxW * kMaxW];
  float Gf[kMaxW * kMaxW];   // FP32 copy for the first eigen-decomposition
  float Vf[kMaxW * kMaxW];
  double lam[kMaxW];
  double F1[kMaxR * kMaxW];
  double F3[kMaxR * kMaxW];
  double FF1[kMaxR * kMaxR];
  double FF3[kMaxR * kMaxR];
  double red[64];
  double cs[4 * kMaxW];  // >= 4 * 32 + 64 doubles
  int idx[kMaxW];
};

// Block-wide sums of three values, returned to thread 0 (other threads get
// partial values): a shuffle tree in each warp, then a shuffle tree over
// the warps' sums in warp 0 (a fixed order).  Every thread must call.
__device__ void block_sum3(double& a, double& b, double& c) {
  __shared__ double part[3][32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    part[0][wid] = a;
    part[1][wid] = b;
    part[2][wid] = c;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = (int)(blockDim.x >> 5);
    a = lane < nw ? part[0][lane] : 0.0;
    b = lane < nw ? part[1][lane] : 0.0;
    c = lane < nw ? part[2][lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
      c += __shfl_down_sync(0xffffffffu, c, o);
    }
  }
  __syncthreads();
}

// Block-wide maxima of three values, returned to thread 0 (the same tree
// as block_sum3).  Every thread must call.
__device__ void block_max3(double& a, double& b, double& c) {
  __shared__ double part[3][32];
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_down_sync(0xffffffffu, a, o));
    b = fmax(b, __shfl_down_sync(0xffffffffu, b, o));
    c = fmax(c, __shfl_down_sync(0xffffffffu, c, o));
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    part[0][wid] = a;
    part[1][wid] = b;
    part[2][wid] = c;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = (int)(blockDim.x >> 5);
    a = lane < nw ? part[0][lane] : 0.0;
    b = lane < nw ? part[1][lane] : 0.0;
    c = lane < nw ? part[2][lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      a = fmax(a, __shfl_down_sync(0xffffffffu, a, o));
      b = fmax(b, __shfl_down_sync(0xffffffffu, b, o));
      c = fmax(c, __shfl_down_sync(0xffffffffu, c, o));
    }
  }
  __syncthreads();
}

// Modified Gram-Schmidt, twice, on the columns of Out (n x r, shared
// memory; n <= 128, r <= 8), FP64; every thread of the block calls.
__device__ void block_mgs2(double* Out, int n, int r, double* red) {
  for (int rep = 0; rep < 2; ++rep) {
    for (int t = 0; t < r; ++t) {
      for (int u = 0; u < t; ++u) {
        double d = 0.0;
        if (threadIdx.x < 32) {
          for (int i = threadIdx.x; i < n; i += 32) d = fma(Out[i + n * u], Out[i + n * t], d);
          for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
          if (threadIdx.x == 0) red[0] = d;
        }
        __syncthreads();
        d = red[0];
        for (int i = threadIdx.x; i < n; i += blockDim.x) Out[i + n * t] -= d * Out[i + n * u];
        __syncthreads();
      }
      double d = 0.0;
      if (threadIdx.x < 32) {
        for (int i = threadIdx.x; i < n; i += 32) d = fma(Out[i + n * t], Out[i + n * t], d);
        for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
        if (threadIdx.x == 0) red[0] = d;
      }
      __syncthreads();
      const double inv = nr_rsqrt(red[0]);
      for (int i = threadIdx.x; i < n; i += blockDim.x) Out[i + n * t] *= inv;
      __syncthreads();
    }
  }
}

// One Cholesky QR pass on the nearly orthonormal columns of Out (n x r,
// shared, r <= 8): Gram Out^T Out, its Cholesky factor R on one thread,
// Out <- Out R^-1 row by row.  Falls back to two MGS passes when the Gram
// is not numerically positive definite.  W: 2 r^2 doubles of shared scratch.
__device__ void block_cholqr(double* Out, int n, int r, double* W, double* red) {
  double* G = W;          // r x r Gram, then R (upper), column-major
  double* Ri = W + r * r; // R^-1
  for (int x = threadIdx.x; x < r * r; x += blockDim.x) {
    const int i = x % r, j = x / r;
    if (i > j) continue;
    double s = 0.0;
    for (int t = 0; t < n; ++t) s = fma(Out[t + n * i], Out[t + n * j], s);
    G[x] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    bool ok = true;
    for (int j = 0; j < r && ok; ++j) {
      for (int i = 0; i <= j; ++i) {
        double v = G[i + r * j];
        for (int t = 0; t < i; ++t) v -= G[t + r * i] * G[t + r * j];
        if (i == j) {
          if (!(v > 1e-8 * G[j + r * j] + 1e-300)) { ok = false; break; }
          G[j + r * j] = sqrt(v);
        } else {
          G[i + r * j] = v / G[i + r * i];
        }
      }
    }
    if (ok) {
      for (int j = 0; j < r; ++j)
        for (int i = j; i >= 0; --i) {
          double v = (i == j) ? 1.0 : 0.0;
          for (int t = i + 1; t <= j; ++t) v -= G[i + r * t] * Ri[t + r * j];
          Ri[i + r * j] = v / G[i + r * i];
        }
    }
    red[0] = ok ? 1.0 : 0.0;
  }
  __syncthreads();
  if (red[0] == 0.0) {
    block_mgs2(Out, n, r, red);
    return;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double row[kMaxR], o[kMaxR];
    for (int t = 0; t < r; ++t) row[t] = Out[i + n * t];
    for (int j = 0; j < r; ++j) {
      double v = 0.0;
      for (int t = 0; t <= j; ++t) v = fma(row[t], Ri[t + r * j], v);
      o[j] = v;
    }
    for (int j = 0; j < r; ++j) Out[i + n * j] = o[j];
  }
  __syncthreads();
}

// Eigen-decomposition of the small symmetric G (w x w, FP64, shared):
// cyclic Jacobi in FP32 on a rounded copy (to its rounding floor), then
// steps of the iterative
// refinement of Ogita & Aishima (Japan J. Indust. Appl. Math. 35, 2018) in
// FP64.  With X the current eigenvector matrix, R = I - X^T X,
// S = X^T G X, lambda_i = s_ii / (1 - r_ii), the correction X <- X (I + E)
// has e_ii = r_ii / 2 and, for eigenvalues farther apart than
// delta = 2 (||offdiag S|| + ||lambda|| ||R||), e_ij = (s_ij + lambda_j r_ij) /
// (lambda_j - lambda_i); closer pairs get r_ij / 2 (they are a cluster and
// only their joint span is determined).  Each step squares the relative
// error; the steps stop after one whose largest correction to the r
// leading vectors (the r largest eigenvalues, ties to the lower index) is
// below 1e-8 (at most four), which takes those FP32 vectors to FP64
// accuracy.  The trailing vectors are not used: with (nearly) repeated
// small eigenvalues they need not settle, and the test ignores them.  Only
// FP64 matrix products remain, which keeps the FP64 instruction count (a
// slow pipe on this GPU) small.  On return S.V holds X (row-major,
// V[i*w + j] = component i of vector j) and S.lam the eigenvalues.
// P, R, E: w x w FP64 scratch (global).  Every thread of the block calls.
__device__ __forceinline__ int desc_rank(const double* lam, int w, int j) {
  int k = 0;
  for (int l = 0; l < w; ++l) k += (lam[l] > lam[j]) || (lam[l] == lam[j] && l < j);
  return k;
}

__device__ void block_eig_refined(int w, int r, InnerShared& S, double* P, double* R, double* E) {
  for (int x = threadIdx.x; x < w * w; x += blockDim.x) S.Gf[x] = (float)S.G[x];
  __syncthreads();
  // FP32 cyclic Jacobi to its rounding floor (every thread of the block takes part)
  block_jacobi_eig<float>(S.Gf, S.Vf, w, 0.f, 40, reinterpret_cast<float*>(S.red),
                          reinterpret_cast<float*>(S.cs));
  for (int x = threadIdx.x; x < w * w; x += blockDim.x) S.V[x] = (double)S.Vf[x];
  __syncthreads();
  double* X = S.V;
  for (int step = 0; step < 4; ++step) {
    for (int x = threadIdx.x; x < w * w; x += blockDim.x) {
      const int i = x / w, j = x % w;
      double pg = 0.0, rr = 0.0;
      for (int l = 0; l < w; ++l) {
        pg = fma(S.G[i * w + l], X[l * w + j], pg);
        rr = fma(X[l * w + i], X[l * w + j], rr);
      }
      P[x] = pg;                      // G X
      R[x] = (i == j ? 1.0 : 0.0) - rr;  // I - X^T X
    }
    __syncthreads();
    double off = 0.0, rn = 0.0, ln = 0.0;
    for (int x = threadIdx.x; x < w * w; x += blockDim.x) {
      const int i = x / w, j = x % w;
      double sv = 0.0;
      for (int l = 0; l < w; ++l) sv = fma(X[l * w + i], P[l * w + j], sv);
      E[x] = sv;                      // S = X^T G X (held in E for now)
      if (i != j) off = fma(sv, sv, off);
      rn = fma(R[x], R[x], rn);
      if (i == j) {
        const double lv = sv / (1.0 - R[x]);
        S.lam[i] = lv;
        ln = fma(lv, lv, ln);
      }
    }
    block_sum3(off, rn, ln);
    if (threadIdx.x == 0) S.red[0] = 2.0 * (sqrt(off) + sqrt(ln) * sqrt(rn));
    __syncthreads();
    const double delta = S.red[0];
    // E <- correction (in place: entry x reads only S(x) = E[x], R and lam)
    double emax = 0.0;
    for (int x = threadIdx.x; x < w * w; x += blockDim.x) {
      const int i = x / w, j = x % w;
      double e;
      if (i == j) {
        e = 0.5 * R[x];
      } else {
        const double gap = S.lam[j] - S.lam[i];
        e = fabs(gap) > delta ? (E[x] + S.lam[j] * R[x]) / gap : 0.5 * R[x];
      }
      E[x] = e;
      if (desc_rank(S.lam, w, j) < r) emax = fmax(emax, fabs(e));
    }
    double d1 = 0.0, d2 = 0.0;
    block_max3(emax, d1, d2);
    if (threadIdx.x == 0) S.red[1] = emax;
    __syncthreads();
    // X <- X + X E (into P, then back)
    for (int x = threadIdx.x; x < w * w; x += blockDim.x) {
      const int i = x / w, j = x % w;
      double v = X[x];
      for (int l = 0; l < w; ++l) v = fma(X[i * w + l], E[l * w + j], v);
      P[x] = v;
    }
    __syncthreads();
    for (int x = threadIdx.x; x < w * w; x += blockDim.x) X[x] = P[x];
    __syncthreads();
    // the error left after a step is about the square of its correction
    if (S.red[1] < 1e-8) break;
  }
}

// r leading left singular vectors of T (n x w, ld n) into Out (n x r):
// eigenvectors of T^T T (block_eig_refined), Out = T v / sigma, then one
// Cholesky QR pass.  P, R, E: w x w FP64 scratch.
__device__ void inner_topsvd(const double* T, int n, int w, int r, InnerShared& S, double* Out,
                             double* P, double* R, double* E) {
  for (int x = threadIdx.x; x < w * w; x += blockDim.x) {
    const int i = x % w, j = x / w;
    double s = 0.0;
    for (int t = 0; t < n; ++t) s = fma(T[t + n * i], T[t + n * j], s);
    S.G[i * w + j] = s;
  }
  __syncthreads();
  block_eig_refined(w, r, S, P, R, E);
  // the r largest eigenvalues (descending) on the diagonal of S.G
  for (int i = threadIdx.x; i < w; i += blockDim.x) S.G[i * w + i] = S.lam[i];
  __syncthreads();
  top_diag<double>(S.G, w, r, S.idx);
  // Out = T v_t / sqrt(lambda_t): orthonormal up to the eigenvectors' error
  for (int x = threadIdx.x; x < n * r; x += blockDim.x) {
    const int i = x % n, t = x / n;
    double s = 0.0;
    for (int j = 0; j < w; ++j) s = fma(T[i + n * j], S.V[j * w + S.idx[t]], s);
    const double lt = S.lam[S.idx[t]];
    Out[i + n * t] = lt > 0.0 ? s * nr_rsqrt(lt) : s;
  }
  __syncthreads();
  block_cholqr(Out, n, r, S.G, S.red);
}

// G-gradient of the inner problem at (Uh, Wh) from T1 (at Uh, Wh) and T3
// (at Uh): ||grad||^2 = 2 ||(I - Uh Uh^T) T1 F1^T||^2 + ||(I - Wh Wh^T) T3 F3^T||^2.
__device__ void inner_grad(int k1, int k3, int r1, int r3, InnerShared& S, double* gout,
                           double* fout) {
  const int w1 = r1 * r3, w3 = r1 * r1;
  // F1 = Uh^T T1 (r1 x w1), F3 = Wh^T T3 (r3 x w3)
  for (int x = threadIdx.x; x < r1 * w1 + r3 * w3; x += blockDim.x) {
    if (x < r1 * w1) {
      const int a = x % r1, j = x / r1;
      double s = 0.0;
      for (int i = 0; i < k1; ++i) s = fma(S.Uh[i + k1 * a], S.T1[i + k1 * j], s);
      S.F1[x] = s;
    } else {
      const int y = x - r1 * w1;
      const int c = y % r3, j = y / r3;
      double s = 0.0;
      for (int i = 0; i < k3; ++i) s = fma(S.Wh[i + k3 * c], S.T3[i + k3 * j], s);
      S.F3[y] = s;
    }
  }
  __syncthreads();
  // FF1 = F1 F1^T, FF3 = F3 F3^T
  for (int x = threadIdx.x; x < r1 * r1 + r3 * r3; x += blockDim.x) {
    if (x < r1 * r1) {
      const int a = x % r1, b = x / r1;
      double s = 0.0;
      for (int j = 0; j < w1; ++j) s = fma(S.F1[a + r1 * j], S.F1[b + r1 * j], s);
      S.FF1[x] = s;
    } else {
      const int y = x - r1 * r1;
      const int c = y % r3, e = y / r3;
      double s = 0.0;
      for (int j = 0; j < w3; ++j) s = fma(S.F3[c + r3 * j], S.F3[e + r3 * j], s);
      S.FF3[y] = s;
    }
  }
  __syncthreads();
  double g1 = 0.0, g3 = 0.0, nf = 0.0;
  // mode 1: (T1 F1^T - Uh FF1) (k1 x r1)
  for (int x = threadIdx.x; x < k1 * r1; x += blockDim.x) {
    const int i = x % k1, a = x / k1;
    double d = 0.0;
    for (int j = 0; j < w1; ++j) d = fma(S.T1[i + k1 * j], S.F1[a + r1 * j], d);
    for (int b = 0; b < r1; ++b) d = fma(-S.Uh[i + k1 * b], S.FF1[b + r1 * a], d);
    g1 = fma(d, d, g1);
  }
  // mode 3: (T3 F3^T - Wh FF3) (k3 x r3)
  for (int x = threadIdx.x; x < k3 * r3; x += blockDim.x) {
    const int i = x % k3, c = x / k3;
    double d = 0.0;
    for (int j = 0; j < w3; ++j) d = fma(S.T3[i + k3 * j], S.F3[c + r3 * j], d);
    for (int e = 0; e < r3; ++e) d = fma(-S.Wh[i + k3 * e], S.FF3[e + r3 * c], d);
    g3 = fma(d, d, g3);
  }
  for (int x = threadIdx.x; x < r1 * w1; x += blockDim.x) nf = fma(S.F1[x], S.F1[x], nf);
  block_sum3(g1, g3, nf);
  if (threadIdx.x == 0) {
    *gout = sqrt(2.0 * g1 + g3);
    *fout = sqrt(nf);
  }
  __syncthreads();
}


// ---- cooperative multi-block HOOI on the core ------------------------------
// The FP64 contractions of a sweep (C x_3 Wh^T, C x_1 Uh^T and their second
// factors) are spread over every block of the grid; the small steps (the
// gradient, the r leading singular vectors, the convergence decision) run
// on block 0.  grid.sync() separates the phases; every block reads the
// decision after the same barrier, so all blocks take the same path.
namespace cg = cooperative_groups;

struct CoopArgs {
  const double* C;
  int k1, k3, r1, r3;
  double tol;
  int max_inner, init_sweeps;
  const double* Uh0;  // HOSVD candidate
  const double* Wh0;
  double* Ug;         // current iterate k1 x r1
  double* Wg;         // current iterate k3 x r3
  double* Ub;         // saved candidate
  double* Wb;
  double* D;          // k1 x k1 x r3
  double* E;          // r1 x k1 x k3
  double* T1;         // k1 x r1 r3
  double* T3;         // k3 x r1^2
  double* ctl;        // [0] grad [1] normF [2] stop flag
  double* P;          // three w x w FP64 scratch matrices of the eigensolver
  double* R;
  double* E2;
  double* Uh_out;
  double* Wh_out;
  double* negU;
  double* negW;
  double* info;
  int from_current;   // 1: continue from (Ug, Wg) as given (no start candidates)
};

__device__ __forceinline__ int64_t gtid() { return blockIdx.x * (int64_t)blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gsize() { return (int64_t)gridDim.x * blockDim.x; }

// D[x + k1^2 t] = sum_c C[x + k1^2 c] Wh[c, t]
__device__ void coop_D(const CoopArgs& a) {
  const int64_t kk = (int64_t)a.k1 * a.k1;
  for (int64_t o = gtid(); o < kk * a.r3; o += gsize()) {
    const int64_t x = o % kk;
    const int t = (int)(o / kk);
    double s = 0.0;
    for (int c = 0; c < a.k3; ++c) s = fma(a.C[x + kk * c], a.Wg[c + a.k3 * t], s);
    a.D[o] = s;
  }
}
// T1[a + k1 (b' + r1 c')] = sum_b D[a + k1 (b + k1 c')] Uh[b, b']
__device__ void coop_T1(const CoopArgs& a) {
  const int64_t n = (int64_t)a.k1 * a.r1 * a.r3;
  for (int64_t o = gtid(); o < n; o += gsize()) {
    const int i = (int)(o % a.k1);
    const int j = (int)(o / a.k1);
    const int bp = j % a.r1, cp = j / a.r1;
    double s = 0.0;
    for (int b = 0; b < a.k1; ++b)
      s = fma(a.D[i + (int64_t)a.k1 * (b + (int64_t)a.k1 * cp)], a.Ug[b + a.k1 * bp], s);
    a.T1[o] = s;
  }
}
// E[t + r1 (b + k1 c)] = sum_a Uh[a, t] C[b + k1 (a + k1 c)]  (C symmetric in a, b)
__device__ void coop_E(const CoopArgs& a) {
  const int64_t bc = (int64_t)a.k1 * a.k3;
  for (int64_t o = gtid(); o < bc * a.r1; o += gsize()) {
    const int64_t x = o % bc;
    const int t = (int)(o / bc);
    const int b = (int)(x % a.k1);
    const int64_t c = x / a.k1;
    double s = 0.0;
    for (int i = 0; i < a.k1; ++i)
      s = fma(a.Ug[i + a.k1 * t], a.C[b + (int64_t)a.k1 * (i + (int64_t)a.k1 * c)], s);
    a.E[t + (int64_t)a.r1 * x] = s;
  }
}
// T3[c + k3 (a' + r1 b')] = sum_b E[a' + r1 (b + k1 c)] Uh[b, b']
__device__ void coop_T3(const CoopArgs& a) {
  const int64_t n = (int64_t)a.k3 * a.r1 * a.r1;
  for (int64_t o = gtid(); o < n; o += gsize()) {
    const int c = (int)(o % a.k3);
    const int j = (int)(o / a.k3);
    const int ap = j % a.r1, bp = j / a.r1;
    double s = 0.0;
    for (int b = 0; b < a.k1; ++b)
      s = fma(a.E[ap + (int64_t)a.r1 * (b + (int64_t)a.k1 * c)], a.Ug[b + a.k1 * bp], s);
    a.T3[o] = s;
  }
}

__device__ void block_copy(const double* src, double* dst, int n) {
  for (int x = threadIdx.x; x < n; x += blockDim.x) dst[x] = src[x];
}

// T3 = unfold_3(C.(Uh,Uh)_{1,2}) (n x r1^2, column a + r1 b) has equal
// columns (a, b) and (b, a), C being symmetric in its first two modes, so
// T3 T3^T = T' T'^T with the r1(r1+1)/2 columns t_aa and (t_ab + t_ba)/sqrt(2),
// a < b (column b(b+1)/2 + a): the same left singular vectors and values
// from a smaller Gram without the r1(r1-1)/2 zero eigenvalues.  In place,
// one row per thread.  Returns the new column count; when r exceeds
// r1(r1+1)/2, T3 is left as it is and r1^2 is returned.
__device__ int fold_sym_columns(double* T, int n, int r1, int r) {
  const int wf = r1 * (r1 + 1) / 2;
  if (wf < r) return r1 * r1;
  constexpr double kInvSqrt2 = 0.70710678118654752440;
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    double row[kMaxW];
    for (int j = 0; j < r1 * r1; ++j) row[j] = T[c + (int64_t)n * j];
    int o = 0;
    for (int b = 0; b < r1; ++b)
      for (int a = 0; a <= b; ++a, ++o)
        T[c + (int64_t)n * o] =
            a == b ? row[a + r1 * b] : (row[a + r1 * b] + row[b + r1 * a]) * kInvSqrt2;
  }
  __syncthreads();
  return wf;
}

// HOOI sweeps from (Ug, Wg); returns the number of sweeps; ctl[0..1] hold
// the gradient and ||F|| at the returned point.
__device__ int coop_sweeps(const CoopArgs& a, int max_sweeps, double tol, InnerShared& S,
                           cg::grid_group& grid) {
  coop_E(a);
  grid.sync();
  coop_T3(a);
  grid.sync();
  int done = 0;
  for (;;) {
    coop_D(a);
    grid.sync();
    coop_T1(a);
    grid.sync();
    if (blockIdx.x == 0) {
      block_copy(a.Ug, S.Uh, a.k1 * a.r1);
      block_copy(a.Wg, S.Wh, a.k3 * a.r3);
      block_copy(a.T1, S.T1, a.k1 * a.r1 * a.r3);
      block_copy(a.T3, S.T3, a.k3 * a.r1 * a.r1);
      __syncthreads();
      inner_grad(a.k1, a.k3, a.r1, a.r3, S, &a.ctl[0], &a.ctl[1]);
      const double g = a.ctl[0], nf = a.ctl[1];
      const bool stop = done >= max_sweeps || g <= tol * nf;
      if (!stop) {
        inner_topsvd(S.T1, a.k1, a.r1 * a.r3, a.r1, S, S.Uh, a.P, a.R, a.E2);
        block_copy(S.Uh, a.Ug, a.k1 * a.r1);
      }
      if (threadIdx.x == 0) a.ctl[2] = stop ? 1.0 : 0.0;
      __threadfence();
    }
    grid.sync();
    if (a.ctl[2] != 0.0) break;
    coop_E(a);
    grid.sync();
    coop_T3(a);
    grid.sync();
    if (blockIdx.x == 0) {
      block_copy(a.T3, S.T3, a.k3 * a.r1 * a.r1);
      __syncthreads();
      const int w3 = fold_sym_columns(S.T3, a.k3, a.r1, a.r3);
      inner_topsvd(S.T3, a.k3, w3, a.r3, S, S.Wh, a.P, a.R, a.E2);
      block_copy(S.Wh, a.Wg, a.k3 * a.r3);
      __threadfence();
    }
    grid.sync();
    ++done;
  }
  return done;
}

__global__ void __launch_bounds__(kInnerThreads) k_inner_coop(CoopArgs a) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ double shd[];
  InnerShared& S = *reinterpret_cast<InnerShared*>(shd);
  const int nu = a.k1 * a.r1, nw = a.k3 * a.r3;
  bool hosvd_won = false;
  if (!a.from_current) {  // uniform over the grid (a kernel argument)
  // candidate 1: truncated HOSVD (+ init sweeps).  Its FP32 eigenvectors
  // are orthonormalised in FP64 first: ||F|| is compared between points of
  // the Stiefel manifolds, and a start whose columns are longer than one
  // would win the comparison by its length.
  if (blockIdx.x == 0) {
    block_copy(a.Uh0, S.Uh, nu);
    block_copy(a.Wh0, S.Wh, nw);
    __syncthreads();
    block_mgs2(S.Uh, a.k1, a.r1, S.red);
    block_mgs2(S.Wh, a.k3, a.r3, S.red);
    block_copy(S.Uh, a.Ug, nu);
    block_copy(S.Wh, a.Wg, nw);
    __threadfence();
  }
  grid.sync();
  coop_sweeps(a, a.init_sweeps, 0.0, S, grid);
  const double nf_a = a.ctl[1];
  for (int64_t x = gtid(); x < nu; x += gsize()) a.Ub[x] = a.Ug[x];
  for (int64_t x = gtid(); x < nw; x += gsize()) a.Wb[x] = a.Wg[x];
  grid.sync();
  // candidate 2: the current point [I; 0], evaluated without sweeps
  for (int64_t x = gtid(); x < nu; x += gsize()) a.Ug[x] = (x % a.k1 == x / a.k1) ? 1.0 : 0.0;
  for (int64_t x = gtid(); x < nw; x += gsize()) a.Wg[x] = (x % a.k3 == x / a.k3) ? 1.0 : 0.0;
  grid.sync();
  coop_sweeps(a, 0, 0.0, S, grid);
  const double nf_b = a.ctl[1];
  hosvd_won = nf_a >= nf_b;
  grid.sync();
  if (hosvd_won) {
    for (int64_t x = gtid(); x < nu; x += gsize()) a.Ug[x] = a.Ub[x];
    for (int64_t x = gtid(); x < nw; x += gsize()) a.Wg[x] = a.Wb[x];
  }
  grid.sync();
  }
  // HOOI sweeps to the tolerance (none with max_inner = 0: the contractions
  // and the gradient at the current point are still formed)
  const int done = coop_sweeps(a, a.max_inner, a.tol, S, grid);
  if (blockIdx.x == 0) {
    for (int x = threadIdx.x; x < nu; x += blockDim.x) {
      a.Uh_out[x] = a.Ug[x];
      a.negU[x] = -a.Ug[x];
    }
    for (int x = threadIdx.x; x < nw; x += blockDim.x) {
      a.Wh_out[x] = a.Wg[x];
      a.negW[x] = -a.Wg[x];
    }
    if (threadIdx.x == 0) {
      a.info[0] = a.ctl[0];
      a.info[1] = a.ctl[1];
      a.info[2] = done + (hosvd_won ? a.init_sweeps : 0);
      a.info[3] = hosvd_won ? 1.0 : 0.0;
    }
  }
}

// ---- general core (Section 5): three factors -------------------------------
// C is k1 x k2 x k3 without symmetry.  A sweep updates Uh from
// T1 = unfold_1(C.(Vh,Wh)_{2,3}), then Vh from T2 = unfold_2(C.(Uh,Wh)_{1,3})
// with the new Uh, then Wh from T3 = unfold_3(C.(Uh,Vh)_{1,2}) with the new
// Uh and Vh; each update is the r leading left singular vectors, which
// maximises ||F|| over that factor, so ||F|| never drops.
struct GenArgs {
  const double* C;
  int k1, k2, k3, r1, r2, r3;
  double tol;
  int max_inner, init_sweeps;
  const double* Uh0;  // HOSVD candidate
  const double* Vh0;
  const double* Wh0;
  double* Ug;         // current factors
  double* Vg;
  double* Wg;
  double* Ub;         // saved candidate
  double* Vb;
  double* Wb;
  double* D;          // k1 k2 x r3: C x_3 Wh^T
  double* E;          // r1 x k2 x k3: C x_1 Uh^T
  double* T1;         // k1 x r2 r3, column b' + r2 c'
  double* T2;         // k2 x r1 r3, column a' + r1 c'
  double* T3;         // k3 x r1 r2, column a' + r1 b'
  double* ctl;        // [0] grad [1] normF [2] stop flag
  double* P;
  double* R;
  double* E2;
  double* negU;
  double* negV;
  double* negW;
  double* info;
};

// D[x + k1 k2 t] = sum_c C[x + k1 k2 c] Wh[c, t]
__device__ void gen_D(const GenArgs& a) {
  const int64_t kk = (int64_t)a.k1 * a.k2;
  for (int64_t o = gtid(); o < kk * a.r3; o += gsize()) {
    const int64_t x = o % kk;
    const int t = (int)(o / kk);
    double s = 0.0;
    for (int c = 0; c < a.k3; ++c) s = fma(a.C[x + kk * c], a.Wg[c + a.k3 * t], s);
    a.D[o] = s;
  }
}
// T1[i + k1 (b' + r2 c')] = sum_b D[i + k1 (b + k2 c')] Vh[b, b']
__device__ void gen_T1(const GenArgs& a) {
  const int64_t n = (int64_t)a.k1 * a.r2 * a.r3;
  for (int64_t o = gtid(); o < n; o += gsize()) {
    const int i = (int)(o % a.k1);
    const int j = (int)(o / a.k1);
    const int bp = j % a.r2, cp = j / a.r2;
    double s = 0.0;
    for (int b = 0; b < a.k2; ++b)
      s = fma(a.D[i + (int64_t)a.k1 * (b + (int64_t)a.k2 * cp)], a.Vg[b + a.k2 * bp], s);
    a.T1[o] = s;
  }
}
// T2[b + k2 (a' + r1 c')] = sum_a D[a + k1 (b + k2 c')] Uh[a, a']
__device__ void gen_T2(const GenArgs& a) {
  const int64_t n = (int64_t)a.k2 * a.r1 * a.r3;
  for (int64_t o = gtid(); o < n; o += gsize()) {
    const int b = (int)(o % a.k2);
    const int j = (int)(o / a.k2);
    const int ap = j % a.r1, cp = j / a.r1;
    const double* d = a.D + (int64_t)a.k1 * (b + (int64_t)a.k2 * cp);
    double s = 0.0;
    for (int i = 0; i < a.k1; ++i) s = fma(d[i], a.Ug[i + a.k1 * ap], s);
    a.T2[o] = s;
  }
}
// E[t + r1 (b + k2 c)] = sum_i Uh[i, t] C[i + k1 (b + k2 c)]
__device__ void gen_E(const GenArgs& a) {
  const int64_t bc = (int64_t)a.k2 * a.k3;
  for (int64_t o = gtid(); o < bc * a.r1; o += gsize()) {
    const int64_t x = o % bc;
    const int t = (int)(o / bc);
    const double* col = a.C + (int64_t)a.k1 * x;
    double s = 0.0;
    for (int i = 0; i < a.k1; ++i) s = fma(a.Ug[i + a.k1 * t], col[i], s);
    a.E[t + (int64_t)a.r1 * x] = s;
  }
}
// T3[c + k3 (a' + r1 b')] = sum_b E[a' + r1 (b + k2 c)] Vh[b, b']
__device__ void gen_T3(const GenArgs& a) {
  const int64_t n = (int64_t)a.k3 * a.r1 * a.r2;
  for (int64_t o = gtid(); o < n; o += gsize()) {
    const int c = (int)(o % a.k3);
    const int j = (int)(o / a.k3);
    const int ap = j % a.r1, bp = j / a.r1;
    double s = 0.0;
    for (int b = 0; b < a.k2; ++b)
      s = fma(a.E[ap + (int64_t)a.r1 * (b + (int64_t)a.k2 * c)], a.Vg[b + a.k2 * bp], s);
    a.T3[o] = s;
  }
}

// One mode's part of the G-gradient at the current point: with F = Q^T T
// (r x w), adds ||T F^T - Q (F F^T)||^2 of this thread's rows to g and,
// for mode 1, ||F||^2 of its entries to nf.  Q (k x r) and T (k x w) in
// global memory; F and F F^T in S.F1, S.FF1.  Every thread calls.
__device__ void gen_mode_grad(const double* Q, const double* T, int k, int r, int w,
                              InnerShared& S, bool first, double& g, double& nf) {
  for (int x = threadIdx.x; x < r * w; x += blockDim.x) {
    const int aa = x % r, j = x / r;
    double s = 0.0;
    for (int i = 0; i < k; ++i) s = fma(Q[i + k * aa], T[i + k * j], s);
    S.F1[x] = s;
  }
  __syncthreads();
  for (int x = threadIdx.x; x < r * r; x += blockDim.x) {
    const int aa = x % r, bb = x / r;
    double s = 0.0;
    for (int j = 0; j < w; ++j) s = fma(S.F1[aa + r * j], S.F1[bb + r * j], s);
    S.FF1[x] = s;
  }
  __syncthreads();
  for (int x = threadIdx.x; x < k * r; x += blockDim.x) {
    const int i = x % k, aa = x / k;
    double d = 0.0;
    for (int j = 0; j < w; ++j) d = fma(T[i + k * j], S.F1[aa + r * j], d);
    for (int bb = 0; bb < r; ++bb) d = fma(-Q[i + k * bb], S.FF1[bb + r * aa], d);
    g = fma(d, d, g);
  }
  if (first)
    for (int x = threadIdx.x; x < r * w; x += blockDim.x) nf = fma(S.F1[x], S.F1[x], nf);
  __syncthreads();
}

// ||grad||, ||F|| at (Ug, Vg, Wg) from T1, T2, T3 there, to ctl[0..1]
// (block 0 only).
__device__ void gen_grad(const GenArgs& a, InnerShared& S) {
  double g = 0.0, nf = 0.0, z = 0.0;
  gen_mode_grad(a.Ug, a.T1, a.k1, a.r1, a.r2 * a.r3, S, true, g, nf);
  gen_mode_grad(a.Vg, a.T2, a.k2, a.r2, a.r1 * a.r3, S, false, g, nf);
  gen_mode_grad(a.Wg, a.T3, a.k3, a.r3, a.r1 * a.r2, S, false, g, nf);
  block_sum3(g, nf, z);
  if (threadIdx.x == 0) {
    a.ctl[0] = sqrt(g);
    a.ctl[1] = sqrt(nf);
  }
  __syncthreads();
}

// new factor (k x r) into the global `dst`: the r leading left singular
// vectors of T (k x w); block 0 only
__device__ void gen_update(const GenArgs& a, const double* T, int k, int w, int r, double* dst,
                           InnerShared& S) {
  inner_topsvd(T, k, w, r, S, S.Uh, a.P, a.R, a.E2);
  block_copy(S.Uh, dst, k * r);
  __threadfence();
}

// General HOOI sweeps from (Ug, Vg, Wg); returns the sweeps done; ctl[0..1]
// hold the gradient and ||F|| at the returned point.
__device__ int gen_sweeps(const GenArgs& a, int max_sweeps, double tol, InnerShared& S,
                          cg::grid_group& grid) {
  gen_E(a);
  grid.sync();
  gen_T3(a);
  grid.sync();
  int done = 0;
  for (;;) {
    gen_D(a);
    grid.sync();
    gen_T1(a);
    gen_T2(a);
    grid.sync();
    if (blockIdx.x == 0) {
      gen_grad(a, S);
      const double g = a.ctl[0], nf = a.ctl[1];
      const bool stop = done >= max_sweeps || g <= tol * nf;
      if (!stop) gen_update(a, a.T1, a.k1, a.r2 * a.r3, a.r1, a.Ug, S);
      if (threadIdx.x == 0) a.ctl[2] = stop ? 1.0 : 0.0;
      __threadfence();
    }
    grid.sync();
    if (a.ctl[2] != 0.0) break;
    gen_T2(a);
    grid.sync();
    if (blockIdx.x == 0) gen_update(a, a.T2, a.k2, a.r1 * a.r3, a.r2, a.Vg, S);
    grid.sync();
    gen_E(a);
    grid.sync();
    gen_T3(a);
    grid.sync();
    if (blockIdx.x == 0) gen_update(a, a.T3, a.k3, a.r1 * a.r2, a.r3, a.Wg, S);
    grid.sync();
    ++done;
  }
  return done;
}

__global__ void __launch_bounds__(kInnerThreads) k_inner_gen(GenArgs a) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ double shd[];
  InnerShared& S = *reinterpret_cast<InnerShared*>(shd);
  const int nu = a.k1 * a.r1, nv = a.k2 * a.r2, nw = a.k3 * a.r3;
  // candidate 1: truncated HOSVD (FP32 eigenvectors orthonormalised in
  // FP64 first) + init sweeps
  if (blockIdx.x == 0) {
    const double* src[3] = {a.Uh0, a.Vh0, a.Wh0};
    double* dst[3] = {a.Ug, a.Vg, a.Wg};
    const int kk[3] = {a.k1, a.k2, a.k3}, rr[3] = {a.r1, a.r2, a.r3};
    for (int md = 0; md < 3; ++md) {
      block_copy(src[md], S.Uh, kk[md] * rr[md]);
      __syncthreads();
      block_mgs2(S.Uh, kk[md], rr[md], S.red);
      block_copy(S.Uh, dst[md], kk[md] * rr[md]);
      __syncthreads();
    }
    __threadfence();
  }
  grid.sync();
  gen_sweeps(a, a.init_sweeps, 0.0, S, grid);
  const double nf_a = a.ctl[1];
  for (int64_t x = gtid(); x < nu; x += gsize()) a.Ub[x] = a.Ug[x];
  for (int64_t x = gtid(); x < nv; x += gsize()) a.Vb[x] = a.Vg[x];
  for (int64_t x = gtid(); x < nw; x += gsize()) a.Wb[x] = a.Wg[x];
  grid.sync();
  // candidate 2: the current point [I; 0], evaluated without sweeps
  for (int64_t x = gtid(); x < nu; x += gsize()) a.Ug[x] = (x % a.k1 == x / a.k1) ? 1.0 : 0.0;
  for (int64_t x = gtid(); x < nv; x += gsize()) a.Vg[x] = (x % a.k2 == x / a.k2) ? 1.0 : 0.0;
  for (int64_t x = gtid(); x < nw; x += gsize()) a.Wg[x] = (x % a.k3 == x / a.k3) ? 1.0 : 0.0;
  grid.sync();
  gen_sweeps(a, 0, 0.0, S, grid);
  const double nf_b = a.ctl[1];
  const bool hosvd_won = nf_a >= nf_b;
  grid.sync();
  if (hosvd_won) {
    for (int64_t x = gtid(); x < nu; x += gsize()) a.Ug[x] = a.Ub[x];
    for (int64_t x = gtid(); x < nv; x += gsize()) a.Vg[x] = a.Vb[x];
    for (int64_t x = gtid(); x < nw; x += gsize()) a.Wg[x] = a.Wb[x];
  }
  grid.sync();
  const int done = gen_sweeps(a, a.max_inner, a.tol, S, grid);
  if (blockIdx.x == 0) {
    for (int x = threadIdx.x; x < nu; x += blockDim.x) a.negU[x] = -a.Ug[x];
    for (int x = threadIdx.x; x < nv; x += blockDim.x) a.negV[x] = -a.Vg[x];
    for (int x = threadIdx.x; x < nw; x += blockDim.x) a.negW[x] = -a.Wg[x];
    if (threadIdx.x == 0) {
      a.info[0] = a.ctl[0];
      a.info[1] = a.ctl[1];
      a.info[2] = done + (hosvd_won ? a.init_sweeps : 0);
      a.info[3] = hosvd_won ? 1.0 : 0.0;
    }
  }
}

// Partial Grams of the unfoldings of the general core in FP32: part[md]
// (nparts x k_md x k_md) with block b of grid row md summing its share of
// the other two indices (o = the column of unfold_md, first index fastest).
__global__ void k_gen_grams(const double* __restrict__ C, int k1, int k2, int k3,
                            float* __restrict__ p1, float* __restrict__ p2,
                            float* __restrict__ p3) {
  const int md = blockIdx.y;
  const int n = md == 0 ? k1 : (md == 1 ? k2 : k3);
  const int64_t ncol = (int64_t)k1 * k2 * k3 / n;
  float* part = md == 0 ? p1 : (md == 1 ? p2 : p3);
  const int nb = gridDim.x;
  const int64_t o0 = ncol * blockIdx.x / nb, o1 = ncol * (blockIdx.x + 1) / nb;
  for (int x = threadIdx.x; x < n * n; x += blockDim.x) {
    const int u = x % n, w = x / n;
    float s = 0.f;
    for (int64_t o = o0; o < o1; ++o) {
      int64_t eu, ew;
      if (md == 0) {
        eu = u + (int64_t)k1 * o;
        ew = w + (int64_t)k1 * o;
      } else if (md == 1) {
        const int64_t aa = o % k1, cc = o / k1;
        eu = aa + (int64_t)k1 * (u + (int64_t)k2 * cc);
        ew = aa + (int64_t)k1 * (w + (int64_t)k2 * cc);
      } else {
        eu = o + (int64_t)k1 * k2 * u;
        ew = o + (int64_t)k1 * k2 * w;
      }
      s += (float)C[eu] * (float)C[ew];
    }
    part[(int64_t)blockIdx.x * n * n + x] = s;
  }
}

}  // namespace

struct InnerWork {
  DevBuf part1, part3, Uh0, Wh0, D, E, Ug, Wg, Ub, Wb, Uo, Wo, T1, T3, ctl, K;
  int coop_grid = 0;
  NewtonWork ng;
  double host_info[4] = {0, 0, 0, 0};
  int host_flag = 0;
};

// Inner solve: C (k1 x k1 x k3, FP64, device) -> Uh (k1 x r1), Wh (k3 x r3),
// their negatives (for the restart combine) and info[4] = {grad, ||F||,
// sweeps (HOOI sweeps plus Newton steps), hosvd_won} on the device.  The
// start is the better of the truncated HOSVD (after init_sweeps HOOI
// sweeps) and the current point; then HOOI sweeps towards the tolerance,
// at most newton_after of them when newton_after >= 0, after which
// Newton-Grassmann steps (newton.cu) continue to the tolerance, a HOOI
// sweep wherever a step is refused; newton_after < 0: HOOI sweeps only.
// At most max_inner sweeps and steps.
int inner_solve(const double* C, int k1, int k3, int r1, int r3, double tol, int max_inner,
                int init_sweeps, int newton_after, double* Uh, double* Wh, double* negU,
                double* negW, double* info, cudaStream_t s) {
  if (k1 > 128 || k3 > 128) return fail(BKS_EUNSUPPORTED, "inner solve: k1, k3 must be <= 128");
  if (r1 > kMaxR || r3 > kMaxR) return fail(BKS_EUNSUPPORTED, "inner solve: r1, r3 must be <= 8");
  // workspace of the calling thread on the current device
  static thread_local InnerWork ws_by_dev[kMaxDevices];
  const int dev = current_device();
  if (dev < 0) return fail(BKS_EUNSUPPORTED, "inner solve: device index above 63");
  InnerWork& w = ws_by_dev[dev];
  const int nparts = std::min(64, std::max(k1, k3));
  const size_t p1 = sizeof(float) * (size_t)nparts * k1 * k1, p3 = sizeof(float) * (size_t)nparts * k3 * k3;
  if (w.part1.bytes < p1) BKS_TRY(w.part1.alloc(p1, s));
  if (w.part3.bytes < p3) BKS_TRY(w.part3.alloc(p3, s));
  if (w.Uh0.bytes < sizeof(double) * 128 * kMaxR) BKS_TRY(w.Uh0.alloc(sizeof(double) * 128 * kMaxR, s));
  if (w.Wh0.bytes < sizeof(double) * 128 * kMaxR) BKS_TRY(w.Wh0.alloc(sizeof(double) * 128 * kMaxR, s));
  const size_t dsz = sizeof(double) * (size_t)k1 * k1 * kMaxR;
  if (w.D.bytes < dsz) BKS_TRY(w.D.alloc(dsz, s));
  const size_t esz = sizeof(double) * (size_t)kMaxR * k1 * k3;
  if (w.E.bytes < esz) BKS_TRY(w.E.alloc(esz, s));
  w.part1.persist(); w.part3.persist(); w.Uh0.persist(); w.Wh0.persist(); w.D.persist(); w.E.persist();
  k_hosvd_grams<<<nparts, 256, 0, s>>>(C, k1, k3, w.part1.as<float>(), w.part3.as<float>()); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  const int nmax = std::max(k1, k3);
  // A, V (nmax^2 each), red (64), cs (the one-warp Jacobi needs 128)
  const size_t hs = sizeof(float) * (2 * (size_t)nmax * nmax + 64 + std::max<size_t>(128, 4 * (size_t)nmax));
  // raised once per device, to the size at k1 = 128
  static PerDeviceOnce once;
  const cudaError_t attr = once.run([] {
    return cudaFuncSetAttribute(k_hosvd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(float) * (2 * 128 * 128 + 64 + 4 * 128)));
  });
  if (attr != cudaSuccess)
    return fail(BKS_ECUDA, std::string("k_hosvd shared-memory limit: ") + cudaGetErrorString(attr));
  k_hosvd<<<2, kInnerThreads, hs, s>>>(w.part1.as<float>(), w.part3.as<float>(), nparts, k1, k3,
                                       r1, r3, w.Uh0.as<double>(), w.Wh0.as<double>()); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  const size_t mat = sizeof(double) * 128 * kMaxR;
  for (DevBuf* b : {&w.Ug, &w.Wg, &w.Ub, &w.Wb, &w.Uo, &w.Wo})
    if (b->bytes < mat) { BKS_TRY(b->alloc(mat, s)); b->persist(); }
  const size_t tsz = sizeof(double) * 128 * kMaxW;
  for (DevBuf* b : {&w.T1, &w.T3})
    if (b->bytes < tsz) { BKS_TRY(b->alloc(tsz, s)); b->persist(); }
  if (w.ctl.bytes < sizeof(double) * 8) { BKS_TRY(w.ctl.alloc(sizeof(double) * 8, s)); w.ctl.persist(); }
  if (w.K.bytes < sizeof(double) * 3 * kMaxW * kMaxW) {
    BKS_TRY(w.K.alloc(sizeof(double) * 3 * kMaxW * kMaxW, s));
    w.K.persist();
  }
  if (w.coop_grid == 0) {
    int per_sm = 0;
    BKS_CUDA_TRY(cudaFuncSetAttribute(k_inner_coop, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sizeof(InnerShared)));
    BKS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_inner_coop,
                                                               kInnerThreads, sizeof(InnerShared)));
    if (per_sm < 1) return fail(BKS_ECUDA, "inner solve: cooperative kernel does not fit on an SM");
    w.coop_grid = std::min(64, per_sm * num_sms());
  }
  // blocks in proportion to the largest contraction phase (512 outputs per
  // block), so that small cores leave the GPU to concurrent jobs
  const int64_t work = std::max<int64_t>((int64_t)k1 * k1 * r3, (int64_t)k1 * k3 * r1);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(w.coop_grid, (work + 511) / 512));
  CoopArgs a;
  const bool newton = newton_after >= 0;
  a.C = C; a.k1 = k1; a.k3 = k3; a.r1 = r1; a.r3 = r3; a.tol = tol;
  a.max_inner = newton ? std::min(max_inner, newton_after) : max_inner;
  a.init_sweeps = std::max(0, init_sweeps); a.Uh0 = w.Uh0.as<double>(); a.Wh0 = w.Wh0.as<double>();
  a.Ug = w.Ug.as<double>(); a.Wg = w.Wg.as<double>(); a.Ub = w.Ub.as<double>();
  a.Wb = w.Wb.as<double>(); a.D = w.D.as<double>(); a.E = w.E.as<double>();
  a.T1 = w.T1.as<double>(); a.T3 = w.T3.as<double>(); a.ctl = w.ctl.as<double>();
  a.P = w.K.as<double>(); a.R = a.P + kMaxW * kMaxW; a.E2 = a.R + kMaxW * kMaxW;
  a.Uh_out = Uh; a.Wh_out = Wh; a.negU = negU; a.negW = negW; a.info = info;
  a.from_current = 0;
  auto launch = [&]() -> int {
    void* kargs[] = {&a};
    BKS_CUDA_TRY(cudaLaunchCooperativeKernel((void*)k_inner_coop, dim3(grid),
                                             dim3(kInnerThreads), kargs, sizeof(InnerShared), s));
    ::bks::note_launch();
    return BKS_OK;
  };
  // the start (truncated HOSVD with its start sweeps, or the current point)
  // and, without Newton, the HOOI sweeps to the tolerance
  BKS_TRY(launch());
  if (!newton) return BKS_OK;
  // Newton-Grassmann continuation: a step is taken when -H is positive
  // definite and ||F|| does not drop, else one HOOI sweep from the point
  auto read_state = [&](bool with_flag) -> int {
    BKS_CUDA_TRY(cudaMemcpyAsync(w.host_info, info, sizeof(w.host_info), cudaMemcpyDeviceToHost, s));
    if (with_flag)
      BKS_CUDA_TRY(cudaMemcpyAsync(&w.host_flag, w.ng.flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    BKS_CUDA_TRY(cudaStreamSynchronize(s));
    return BKS_OK;
  };
  BKS_TRY(w.ng.ensure(k1, k3, r1, r3, s));
  BKS_TRY(read_state(false));
  double g = w.host_info[0], nf = w.host_info[1];
  const double start_sweeps = w.host_info[2], hosvd_won = w.host_info[3];
  int steps = 0, sweeps = (int)start_sweeps - (hosvd_won != 0.0 ? a.init_sweeps : 0);
  const int64_t nu = (int64_t)k1 * r1, nw = (int64_t)k3 * r3;
  a.from_current = 1;
  while (std::isfinite(g) && g > tol * nf && steps + sweeps < max_inner) {
    BKS_TRY(newton_step(w.D.as<double>(), w.T1.as<double>(), w.E.as<double>(), w.T3.as<double>(),
                        w.Ug.as<double>(), w.Wg.as<double>(), k1, k3, r1, r3, w.Ub.as<double>(),
                        w.Wb.as<double>(), w.ng, s));
    // keep the point, move to the step and evaluate it there
    BKS_CUDA_TRY(cudaMemcpyAsync(w.Uo.p, w.Ug.p, sizeof(double) * nu, cudaMemcpyDeviceToDevice, s));
    BKS_CUDA_TRY(cudaMemcpyAsync(w.Wo.p, w.Wg.p, sizeof(double) * nw, cudaMemcpyDeviceToDevice, s));
    BKS_CUDA_TRY(cudaMemcpyAsync(w.Ug.p, w.Ub.p, sizeof(double) * nu, cudaMemcpyDeviceToDevice, s));
    BKS_CUDA_TRY(cudaMemcpyAsync(w.Wg.p, w.Wb.p, sizeof(double) * nw, cudaMemcpyDeviceToDevice, s));
    a.max_inner = 0;
    a.tol = 0.0;
    BKS_TRY(launch());
    BKS_TRY(read_state(true));
    const double gn = w.host_info[0], nfn = w.host_info[1];
    if (w.host_flag == 0 && std::isfinite(gn) && nfn >= nf * (1.0 - 1e-14)) {
      g = gn;
      nf = nfn;
      ++steps;
      continue;
    }
    // refused: back to the point, one HOOI sweep
    BKS_CUDA_TRY(cudaMemcpyAsync(w.Ug.p, w.Uo.p, sizeof(double) * nu, cudaMemcpyDeviceToDevice, s));
    BKS_CUDA_TRY(cudaMemcpyAsync(w.Wg.p, w.Wo.p, sizeof(double) * nw, cudaMemcpyDeviceToDevice, s));
    a.max_inner = 1;
    BKS_TRY(launch());
    BKS_TRY(read_state(false));
    g = w.host_info[0];
    nf = w.host_info[1];
    ++sweeps;
  }
  // info[2]: the HOOI sweeps (start and refused steps) plus the Newton steps
  w.host_info[0] = g;
  w.host_info[1] = nf;
  w.host_info[2] = (hosvd_won != 0.0 ? a.init_sweeps : 0) + sweeps + steps;
  w.host_info[3] = hosvd_won;
  BKS_CUDA_TRY(cudaMemcpyAsync(info, w.host_info, sizeof(w.host_info), cudaMemcpyHostToDevice, s));
  BKS_CUDA_TRY(cudaStreamSynchronize(s));
  return BKS_OK;
}


struct GenInnerWork {
  DevBuf p1, p2, p3, Uh0, Vh0, Wh0, scratch, Ug, Vg, Wg, Ub, Vb, Wb, D, E, T1, T2, T3, ctl, K;
  int coop_grid = 0;
};

// General inner solve (Algorithm 5 step (i) for a k1 x k2 x k3 core): the
// better (larger ||F||) of the truncated HOSVD after init_sweeps HOOI
// sweeps and the current point, then HOOI sweeps until ||grad|| <= tol
// ||F|| or max_inner sweeps.  Writes -Uh, -Vh, -Wh (for the restart
// combine) and info[4] = {grad, ||F||, sweeps, hosvd_won} on the device.
int gen_inner_solve(const double* C, int k1, int k2, int k3, int r1, int r2, int r3, double tol,
                    int max_inner, int init_sweeps, double* negU, double* negV, double* negW,
                    double* info, cudaStream_t s) {
  if (k1 > 128 || k2 > 128 || k3 > 128)
    return fail(BKS_EUNSUPPORTED, "inner solve: k1, k2, k3 must be <= 128");
  if (r1 > kMaxR || r2 > kMaxR || r3 > kMaxR || r1 * r2 > kMaxW || r1 * r3 > kMaxW ||
      r2 * r3 > kMaxW)
    return fail(BKS_EUNSUPPORTED, "inner solve: ranks must be <= 8");
  if (r1 > k1 || r2 > k2 || r3 > k3) return fail(BKS_EINVAL, "inner solve: rank above the basis size");
  static thread_local GenInnerWork ws_by_dev[kMaxDevices];
  const int dev = current_device();
  if (dev < 0) return fail(BKS_EUNSUPPORTED, "inner solve: device index above 63");
  GenInnerWork& w = ws_by_dev[dev];
  auto grow = [&](DevBuf& b, size_t bytes) -> int {
    if (b.bytes < bytes) {
      BKS_TRY(b.alloc(bytes, s));
      b.persist();
    }
    return BKS_OK;
  };
  const int kmax = std::max(k1, std::max(k2, k3));
  const int nparts = std::min(64, kmax);
  BKS_TRY(grow(w.p1, sizeof(float) * (size_t)nparts * k1 * k1));
  BKS_TRY(grow(w.p2, sizeof(float) * (size_t)nparts * k2 * k2));
  BKS_TRY(grow(w.p3, sizeof(float) * (size_t)nparts * k3 * k3));
  const size_t mat = sizeof(double) * 128 * kMaxR;
  for (DevBuf* b : {&w.Uh0, &w.Vh0, &w.Wh0, &w.scratch, &w.Ug, &w.Vg, &w.Wg, &w.Ub, &w.Vb, &w.Wb})
    BKS_TRY(grow(*b, mat));
  BKS_TRY(grow(w.D, sizeof(double) * (size_t)k1 * k2 * r3));
  BKS_TRY(grow(w.E, sizeof(double) * (size_t)r1 * k2 * k3));
  const size_t tsz = sizeof(double) * 128 * kMaxW;
  for (DevBuf* b : {&w.T1, &w.T2, &w.T3}) BKS_TRY(grow(*b, tsz));
  BKS_TRY(grow(w.ctl, sizeof(double) * 8));
  BKS_TRY(grow(w.K, sizeof(double) * 3 * kMaxW * kMaxW));
  k_gen_grams<<<dim3(nparts, 3), 256, 0, s>>>(C, k1, k2, k3, w.p1.as<float>(), w.p2.as<float>(),
                                              w.p3.as<float>()); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  static PerDeviceOnce once;
  const cudaError_t attr = once.run([] {
    return cudaFuncSetAttribute(k_hosvd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(float) * (2 * 128 * 128 + 64 + 4 * 128)));
  });
  if (attr != cudaSuccess)
    return fail(BKS_ECUDA, std::string("k_hosvd shared-memory limit: ") + cudaGetErrorString(attr));
  auto hs = [](int nmax) {
    return sizeof(float) * (2 * (size_t)nmax * nmax + 64 + std::max<size_t>(128, 4 * (size_t)nmax));
  };
  // modes 1 and 2 in one launch (block 0, block 1), mode 3 in a second
  k_hosvd<<<2, kInnerThreads, hs(std::max(k1, k2)), s>>>(w.p1.as<float>(), w.p2.as<float>(), nparts,
                                                        k1, k2, r1, r2, w.Uh0.as<double>(),
                                                        w.Vh0.as<double>()); ::bks::note_launch();
  k_hosvd<<<2, kInnerThreads, hs(k3), s>>>(w.p3.as<float>(), w.p3.as<float>(), nparts, k3, k3, r3,
                                           r3, w.Wh0.as<double>(), w.scratch.as<double>()); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  if (w.coop_grid == 0) {
    int per_sm = 0;
    BKS_CUDA_TRY(cudaFuncSetAttribute(k_inner_gen, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sizeof(InnerShared)));
    BKS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_inner_gen,
                                                               kInnerThreads, sizeof(InnerShared)));
    if (per_sm < 1) return fail(BKS_ECUDA, "inner solve: cooperative kernel does not fit on an SM");
    w.coop_grid = std::min(64, per_sm * num_sms());
  }
  const int64_t work = std::max<int64_t>((int64_t)k1 * k2 * r3, (int64_t)r1 * k2 * k3);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(w.coop_grid, (work + 511) / 512));
  GenArgs a;
  a.C = C; a.k1 = k1; a.k2 = k2; a.k3 = k3; a.r1 = r1; a.r2 = r2; a.r3 = r3;
  a.tol = tol; a.max_inner = max_inner; a.init_sweeps = std::max(0, init_sweeps);
  a.Uh0 = w.Uh0.as<double>(); a.Vh0 = w.Vh0.as<double>(); a.Wh0 = w.Wh0.as<double>();
  a.Ug = w.Ug.as<double>(); a.Vg = w.Vg.as<double>(); a.Wg = w.Wg.as<double>();
  a.Ub = w.Ub.as<double>(); a.Vb = w.Vb.as<double>(); a.Wb = w.Wb.as<double>();
  a.D = w.D.as<double>(); a.E = w.E.as<double>();
  a.T1 = w.T1.as<double>(); a.T2 = w.T2.as<double>(); a.T3 = w.T3.as<double>();
  a.ctl = w.ctl.as<double>();
  a.P = w.K.as<double>(); a.R = a.P + kMaxW * kMaxW; a.E2 = a.R + kMaxW * kMaxW;
  a.negU = negU; a.negV = negV; a.negW = negW; a.info = info;
  void* kargs[] = {&a};
  BKS_CUDA_TRY(cudaLaunchCooperativeKernel((void*)k_inner_gen, dim3(grid), dim3(kInnerThreads),
                                           kargs, sizeof(InnerShared), s));
  ::bks::note_launch();
  return BKS_OK;
}

}  // namespace bks
