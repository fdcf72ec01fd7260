// Newton-Grassmann steps for the inner problem of the tensor Krylov-Schur
// method (Algorithm 5 step (i); Section 6.2 names the method, which the
// paper does not state).  This library's step for the (1,2)-symmetric
// problem max ||C.(U,U,W)|| over orthonormal U (k1 x r1), W (k3 x r3):
// in the local coordinates U(X) = (U + Up X)(I + X^T X)^(-1/2), W(Y) =
// (W + Wp Y)(I + Y^T Y)^(-1/2), with [U Up], [W Wp] orthogonal, the
// second-order expansion of g = 1/2 ||C.(U(X),U(X),W(Y))||^2 at X = Y = 0
// has the gradient
//   gX[s,a] = 2 sum_{bc} F0[a,b,c] B1[s,b,c],   gY[t,c] = sum_{ab} F0[a,b,c] B3[a,b,t]
// and the Hessian (x = (s,a) index s + d1 a, y = (t,c) index t + d3 c)
//   Hxx = 2 d_aa' S[s,s'] + 2 sum_c B1[s,a',c] B1[s',a,c] + 2 sum_c F0[a,a',c] B11[s,s',c]
//         - 2 d_ss' M1[a,a']
//   Hxy = 2 sum_b B1[s,b,c] B3[a,b,t] + 2 sum_b F0[a,b,c] B13[s,b,t]
//   Hyy = d_cc' S3[t,t'] - d_tt' M3[c,c']
// where F0 = C.(U,U,W), B1 = C.(Up,U,W), B11 = C.(Up,Up,W), B3 = C.(U,U,Wp),
// B13 = C.(Up,U,Wp), S = unfold_1(B1) unfold_1(B1)^T, S3 = unfold_3(B3)
// unfold_3(B3)^T, M1 = unfold_1(F0) unfold_1(F0)^T, M3 = unfold_3(F0)
// unfold_3(F0)^T.  The step solves (-H) z = grad (a maximum has -H positive
// definite); the new point is the orthonormalised (U + Up X, W + Wp Y).
//
// The blocks are formed from the contractions the cooperative inner kernel
// leaves at the current point: D = C x_3 W^T (k1 x k1 x r3), T1 = unfold_1
// C.(., U, W) (k1 x r1 r3), E = C x_1 U^T (r1 x k1 x k3), T3 = unfold_3
// C.(U, U, .) (k3 x r1^2).  The linear system is factored in FP32
// (Cholesky; a non-positive pivot marks -H as not definite) and the
// solution refined twice with FP64 residuals.
#include <algorithm>

#include "common.cuh"
#include "dense.cuh"
#include "newton.cuh"

namespace bks {

namespace {

inline int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)num_sms() * 16));
}

__device__ __forceinline__ int64_t gid() { return blockIdx.x * (int64_t)blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

// Block 0: Up (k1 x (k1 - r1)) completing Ug; block 1: Wp completing Wg.
// Householder QR of the r columns (reflectors kept in shared memory), then
// Q e_j = H_0 H_1 ... H_{r-1} e_j for j = r .. k-1, one column per thread.
__global__ void k_ng_complement(const double* __restrict__ Ug, int k1, int r1,
                                const double* __restrict__ Wg, int k3, int r3,
                                double* __restrict__ Up, double* __restrict__ Wp) {
  __shared__ double A[kNgMaxK * kNgMaxR];
  __shared__ double V[kNgMaxK * kNgMaxR];
  __shared__ double red[32];
  const double* Q = blockIdx.x == 0 ? Ug : Wg;
  const int k = blockIdx.x == 0 ? k1 : k3, r = blockIdx.x == 0 ? r1 : r3;
  double* out = blockIdx.x == 0 ? Up : Wp;
  for (int x = threadIdx.x; x < k * r; x += blockDim.x) {
    A[x] = Q[x];
    V[x] = 0.0;
  }
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    // x = A[j:, j]; v = x - alpha e_1 with alpha = -sign(x_j) ||x||; v /= ||v||
    if (threadIdx.x < 32) {
      double s = 0.0;
      for (int i = j + threadIdx.x; i < k; i += 32) s = fma(A[i + k * j], A[i + k * j], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (threadIdx.x == 0) red[0] = s;
    }
    __syncthreads();
    const double nx = sqrt(red[0]);
    const double xj = A[j + k * j];
    const double alpha = xj >= 0.0 ? -nx : nx;
    for (int i = j + threadIdx.x; i < k; i += blockDim.x)
      V[i + k * j] = A[i + k * j] - (i == j ? alpha : 0.0);
    __syncthreads();
    if (threadIdx.x < 32) {
      double s = 0.0;
      for (int i = j + threadIdx.x; i < k; i += 32) s = fma(V[i + k * j], V[i + k * j], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (threadIdx.x == 0) red[1] = s;
    }
    __syncthreads();
    const double inv = red[1] > 0.0 ? 1.0 / sqrt(red[1]) : 0.0;
    for (int i = j + threadIdx.x; i < k; i += blockDim.x) V[i + k * j] *= inv;
    __syncthreads();
    // A[j:, j+1:] -= 2 v (v^T A[j:, j+1:]), one column per thread
    for (int c = j + 1 + threadIdx.x; c < r; c += blockDim.x) {
      double d = 0.0;
      for (int i = j; i < k; ++i) d = fma(V[i + k * j], A[i + k * c], d);
      for (int i = j; i < k; ++i) A[i + k * c] -= 2.0 * d * V[i + k * j];
    }
    __syncthreads();
  }
  // complement columns: x = e_{r + c}, apply H_{r-1}, ..., H_0 (the product
  // H_0 ... H_{r-1} applied to e)
  for (int c = threadIdx.x; c < k - r; c += blockDim.x) {
    double* x = out + (int64_t)k * c;
    for (int i = 0; i < k; ++i) x[i] = (i == r + c) ? 1.0 : 0.0;
    for (int j = r - 1; j >= 0; --j) {
      double d = 0.0;
      for (int i = j; i < k; ++i) d = fma(V[i + k * j], x[i], d);
      for (int i = j; i < k; ++i) x[i] -= 2.0 * d * V[i + k * j];
    }
  }
}

struct NgDims {
  int k1, k3, r1, r3, d1, d3, N;
};

// First-level blocks (one output per thread, grid-stride over their union).
__global__ void k_ng_blocks1(NgDims z, const double* __restrict__ Ug, const double* __restrict__ Up,
                             const double* __restrict__ Wp, const double* __restrict__ D,
                             const double* __restrict__ T1, const double* __restrict__ E,
                             const double* __restrict__ T3, double* __restrict__ F0,
                             double* __restrict__ B1, double* __restrict__ DUp,
                             double* __restrict__ B3, double* __restrict__ G) {
  const int k1 = z.k1, k3 = z.k3, r1 = z.r1, r3 = z.r3, d1 = z.d1, d3 = z.d3;
  const int64_t nF0 = (int64_t)r1 * r1 * r3, nB1 = (int64_t)d1 * r1 * r3,
                nDU = (int64_t)k1 * d1 * r3, nB3 = (int64_t)r1 * r1 * d3,
                nG = (int64_t)r1 * k1 * d3;
  const int64_t tot = nF0 + nB1 + nDU + nB3 + nG;
  for (int64_t o = gid(); o < tot; o += gstride()) {
    int64_t x = o;
    if (x < nF0) {
      // F0[a + r1 (b + r1 c)] = sum_i Ug[i, a] T1[i + k1 (b + r1 c)]
      const int a = (int)(x % r1), bc = (int)(x / r1);
      double s = 0.0;
      for (int i = 0; i < k1; ++i) s = fma(Ug[i + k1 * a], T1[i + (int64_t)k1 * bc], s);
      F0[x] = s;
      continue;
    }
    x -= nF0;
    if (x < nB1) {
      // B1[s + d1 (b + r1 c)] = sum_i Up[i, s] T1[i + k1 (b + r1 c)]
      const int sI = (int)(x % d1), bc = (int)(x / d1);
      double s = 0.0;
      for (int i = 0; i < k1; ++i) s = fma(Up[i + (int64_t)k1 * sI], T1[i + (int64_t)k1 * bc], s);
      B1[x] = s;
      continue;
    }
    x -= nB1;
    if (x < nDU) {
      // DUp[i + k1 (p + d1 t)] = sum_b D[i + k1 (b + k1 t)] Up[b, p]
      const int i = (int)(x % k1);
      const int64_t pt = x / k1;
      const int p = (int)(pt % d1), t = (int)(pt / d1);
      double s = 0.0;
      for (int b = 0; b < k1; ++b)
        s = fma(D[i + (int64_t)k1 * (b + (int64_t)k1 * t)], Up[b + (int64_t)k1 * p], s);
      DUp[x] = s;
      continue;
    }
    x -= nDU;
    if (x < nB3) {
      // B3[a + r1 (b + r1 t)] = sum_c T3[c + k3 (a + r1 b)] Wp[c, t]
      const int ab = (int)(x % (r1 * r1)), t = (int)(x / (r1 * r1));
      double s = 0.0;
      for (int c = 0; c < k3; ++c) s = fma(T3[c + (int64_t)k3 * ab], Wp[c + (int64_t)k3 * t], s);
      B3[x] = s;
      continue;
    }
    x -= nB3;
    {
      // G[b + r1 (i + k1 t)] = sum_c E[b + r1 (i + k1 c)] Wp[c, t]
      const int bi = (int)(x % ((int64_t)r1 * k1)), t = (int)(x / ((int64_t)r1 * k1));
      double s = 0.0;
      for (int c = 0; c < k3; ++c)
        s = fma(E[bi + (int64_t)r1 * k1 * c], Wp[c + (int64_t)k3 * t], s);
      G[x] = s;
    }
  }
}

// Second-level blocks, the small Grams and the gradient.
__global__ void k_ng_blocks2(NgDims z, const double* __restrict__ Up,
                             const double* __restrict__ F0, const double* __restrict__ B1,
                             const double* __restrict__ DUp, const double* __restrict__ B3,
                             const double* __restrict__ G, double* __restrict__ B11,
                             double* __restrict__ B13, double* __restrict__ S,
                             double* __restrict__ S3, double* __restrict__ M1,
                             double* __restrict__ M3, double* __restrict__ grad) {
  const int k1 = z.k1, r1 = z.r1, r3 = z.r3, d1 = z.d1, d3 = z.d3;
  const int64_t n11 = (int64_t)d1 * d1 * r3, n13 = (int64_t)d1 * r1 * d3, nS = (int64_t)d1 * d1,
                nS3 = (int64_t)d3 * d3, nM1 = (int64_t)r1 * r1, nM3 = (int64_t)r3 * r3,
                ngX = (int64_t)d1 * r1, ngY = (int64_t)d3 * r3;
  const int64_t tot = n11 + n13 + nS + nS3 + nM1 + nM3 + ngX + ngY;
  for (int64_t o = gid(); o < tot; o += gstride()) {
    int64_t x = o;
    if (x < n11) {
      // B11[s + d1 (p + d1 t)] = sum_i Up[i, s] DUp[i + k1 (p + d1 t)]
      const int sI = (int)(x % d1);
      const int64_t pt = x / d1;
      double s = 0.0;
      for (int i = 0; i < k1; ++i) s = fma(Up[i + (int64_t)k1 * sI], DUp[i + (int64_t)k1 * pt], s);
      B11[x] = s;
      continue;
    }
    x -= n11;
    if (x < n13) {
      // B13[s + d1 (b + r1 t)] = sum_i Up[i, s] G[b + r1 (i + k1 t)]
      const int sI = (int)(x % d1);
      const int bt = (int)(x / d1);
      const int b = bt % r1, t = bt / r1;
      double s = 0.0;
      for (int i = 0; i < k1; ++i)
        s = fma(Up[i + (int64_t)k1 * sI], G[b + (int64_t)r1 * (i + (int64_t)k1 * t)], s);
      B13[x] = s;
      continue;
    }
    x -= n13;
    if (x < nS) {
      // S[s + d1 p] = sum_{bc} B1[s, b, c] B1[p, b, c]
      const int sI = (int)(x % d1), p = (int)(x / d1);
      double s = 0.0;
      for (int bc = 0; bc < r1 * r3; ++bc)
        s = fma(B1[sI + (int64_t)d1 * bc], B1[p + (int64_t)d1 * bc], s);
      S[x] = s;
      continue;
    }
    x -= nS;
    if (x < nS3) {
      // S3[t + d3 u] = sum_{ab} B3[a, b, t] B3[a, b, u]
      const int t = (int)(x % d3), u = (int)(x / d3);
      double s = 0.0;
      for (int ab = 0; ab < r1 * r1; ++ab)
        s = fma(B3[ab + (int64_t)r1 * r1 * t], B3[ab + (int64_t)r1 * r1 * u], s);
      S3[x] = s;
      continue;
    }
    x -= nS3;
    if (x < nM1) {
      // M1[a + r1 A] = sum_{bc} F0[a, b, c] F0[A, b, c]
      const int a = (int)(x % r1), A = (int)(x / r1);
      double s = 0.0;
      for (int bc = 0; bc < r1 * r3; ++bc) s = fma(F0[a + r1 * bc], F0[A + r1 * bc], s);
      M1[x] = s;
      continue;
    }
    x -= nM1;
    if (x < nM3) {
      // M3[c + r3 C] = sum_{ab} F0[a, b, c] F0[a, b, C]
      const int c = (int)(x % r3), C = (int)(x / r3);
      double s = 0.0;
      for (int ab = 0; ab < r1 * r1; ++ab) s = fma(F0[ab + r1 * r1 * c], F0[ab + r1 * r1 * C], s);
      M3[x] = s;
      continue;
    }
    x -= nM3;
    if (x < ngX) {
      // gX[s + d1 a] = 2 sum_{bc} F0[a, b, c] B1[s, b, c]
      const int sI = (int)(x % d1), a = (int)(x / d1);
      double s = 0.0;
      for (int bc = 0; bc < r1 * r3; ++bc) s = fma(F0[a + r1 * bc], B1[sI + (int64_t)d1 * bc], s);
      grad[x] = 2.0 * s;
      continue;
    }
    x -= ngX;
    {
      // gY[t + d3 c] = sum_{ab} F0[a, b, c] B3[a, b, t]
      const int t = (int)(x % d3), c = (int)(x / d3);
      double s = 0.0;
      for (int ab = 0; ab < r1 * r1; ++ab)
        s = fma(F0[ab + r1 * r1 * c], B3[ab + (int64_t)r1 * r1 * t], s);
      grad[ngX + x] = s;
    }
  }
}

// A = -H (N x N, column-major, FP64) and its FP32 copy.
__global__ void k_ng_hessian(NgDims z, const double* __restrict__ F0, const double* __restrict__ B1,
                             const double* __restrict__ B11, const double* __restrict__ B3,
                             const double* __restrict__ B13, const double* __restrict__ S,
                             const double* __restrict__ S3, const double* __restrict__ M1,
                             const double* __restrict__ M3, double* __restrict__ A,
                             float* __restrict__ A32) {
  const int r1 = z.r1, r3 = z.r3, d1 = z.d1, d3 = z.d3, N = z.N;
  const int nx = d1 * r1;
  for (int64_t o = gid(); o < (int64_t)N * N; o += gstride()) {
    const int i = (int)(o % N), j = (int)(o / N);
    double h = 0.0;
    if (i < nx && j < nx) {
      const int s = i % d1, a = i / d1, p = j % d1, a2 = j / d1;
      if (a == a2) h += 2.0 * S[s + d1 * p];
      if (s == p) h -= 2.0 * M1[a + r1 * a2];
      for (int c = 0; c < r3; ++c) {
        h += 2.0 * B1[s + d1 * (a2 + r1 * c)] * B1[p + d1 * (a + r1 * c)];
        h += 2.0 * F0[a + r1 * (a2 + r1 * c)] * B11[s + d1 * (p + (int64_t)d1 * c)];
      }
    } else if (i >= nx && j >= nx) {
      const int t = (i - nx) % d3, c = (i - nx) / d3, u = (j - nx) % d3, c2 = (j - nx) / d3;
      if (c == c2) h += S3[t + d3 * u];
      if (t == u) h -= M3[c + r3 * c2];
    } else {
      // Hxy with x = (s, a) and y = (t, c)
      const int xi = i < nx ? i : j, yi = (i < nx ? j : i) - nx;
      const int s = xi % d1, a = xi / d1, t = yi % d3, c = yi / d3;
      for (int b = 0; b < r1; ++b) {
        h += 2.0 * B1[s + d1 * (b + r1 * c)] * B3[a + r1 * (b + r1 * t)];
        h += 2.0 * F0[a + r1 * (b + r1 * c)] * B13[s + d1 * (b + r1 * t)];
      }
    }
    A[o] = -h;
    A32[o] = (float)(-h);
  }
}

// (-H) z = grad: FP32 Cholesky of A32 (in shared memory, column-major
// lower triangle, when N <= kNgSmemN; else in place in global memory),
// FP32 substitutions, two FP64 residual corrections.  flag[0] = 1 when a
// pivot is not positive (-H not positive definite).  One block.
__global__ void __launch_bounds__(1024)
k_ng_solve(int N, const double* __restrict__ A, float* __restrict__ A32g,
           const double* __restrict__ grad, double* __restrict__ zout, float* __restrict__ w32,
           double* __restrict__ res, int* __restrict__ flag) {
  extern __shared__ float shL[];
  const bool in_smem = N <= kNgSmemN;
  float* L = in_smem ? shL : A32g;
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  if (in_smem)
    for (int64_t x = threadIdx.x; x < (int64_t)N * N; x += blockDim.x) L[x] = A32g[x];
  __syncthreads();
  // right-looking Cholesky, lower triangle
  for (int j = 0; j < N; ++j) {
    const float d = L[j + (int64_t)N * j];
    if (!(d > 0.0f)) {
      if (threadIdx.x == 0) bad = 1;
      __syncthreads();
      break;
    }
    const float ljj = sqrtf(d);
    const float inv = 1.0f / ljj;
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < N; i += blockDim.x) L[i + (int64_t)N * j] *= inv;
    if (threadIdx.x == 0) L[j + (int64_t)N * j] = ljj;
    __syncthreads();
    const int m = N - j - 1;
    for (int64_t x = threadIdx.x; x < (int64_t)m * m; x += blockDim.x) {
      const int ii = (int)(x % m), kk = (int)(x / m);
      if (ii < kk) continue;
      const int i = j + 1 + ii, c = j + 1 + kk;
      L[i + (int64_t)N * c] -= L[i + (int64_t)N * j] * L[c + (int64_t)N * j];
    }
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0) flag[0] = 1;
    return;
  }
  // z = 0; res = grad; then three rounds: w = L^-T L^-1 res (FP32), z += w,
  // res = grad - A z (FP64)
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    zout[i] = 0.0;
    res[i] = grad[i];
  }
  __syncthreads();
  for (int round = 0; round < 3; ++round) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) w32[i] = (float)res[i];
    __syncthreads();
    // forward: L w = res (column-oriented)
    for (int j = 0; j < N; ++j) {
      if (threadIdx.x == 0) w32[j] /= L[j + (int64_t)N * j];
      __syncthreads();
      const float wj = w32[j];
      for (int i = j + 1 + threadIdx.x; i < N; i += blockDim.x) w32[i] -= L[i + (int64_t)N * j] * wj;
      __syncthreads();
    }
    // backward: L^T w = w (row j of L^T is column j of L)
    for (int j = N - 1; j >= 0; --j) {
      if (threadIdx.x < 32) {
        float s = 0.0f;
        for (int i = j + 1 + threadIdx.x; i < N; i += 32) s = fmaf(L[i + (int64_t)N * j], w32[i], s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) w32[j] = (w32[j] - s) / L[j + (int64_t)N * j];
      }
      __syncthreads();
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) zout[i] += (double)w32[i];
    __syncthreads();
    if (round == 2) break;
    // res = grad - A z, FP64, one row per thread
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      double s = grad[i];
      for (int c = 0; c < N; ++c) s = fma(-A[i + (int64_t)N * c], zout[c], s);
      res[i] = s;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) flag[0] = 0;
}

// Un = orthonormalised (Ug + Up X), Wn = orthonormalised (Wg + Wp Y)
// (two passes of modified Gram-Schmidt); block 0: U, block 1: W.
__global__ void k_ng_update(NgDims z, const double* __restrict__ Ug, const double* __restrict__ Up,
                            const double* __restrict__ Wg, const double* __restrict__ Wp,
                            const double* __restrict__ zv, double* __restrict__ Un,
                            double* __restrict__ Wn) {
  __shared__ double M[kNgMaxK * kNgMaxR];
  __shared__ double red[2];
  const bool isU = blockIdx.x == 0;
  const int k = isU ? z.k1 : z.k3, r = isU ? z.r1 : z.r3, d = isU ? z.d1 : z.d3;
  const double* Q = isU ? Ug : Wg;
  const double* P = isU ? Up : Wp;
  const double* X = isU ? zv : zv + (int64_t)z.d1 * z.r1;
  double* out = isU ? Un : Wn;
  for (int x = threadIdx.x; x < k * r; x += blockDim.x) {
    const int i = x % k, a = x / k;
    double s = Q[x];
    for (int t = 0; t < d; ++t) s = fma(P[i + (int64_t)k * t], X[t + d * a], s);
    M[x] = s;
  }
  __syncthreads();
  for (int rep = 0; rep < 2; ++rep)
    for (int t = 0; t < r; ++t) {
      for (int u = 0; u <= t; ++u) {
        if (threadIdx.x < 32) {
          double s = 0.0;
          for (int i = threadIdx.x; i < k; i += 32) s = fma(M[i + k * u], M[i + k * t], s);
          for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
          if (threadIdx.x == 0) red[0] = s;
        }
        __syncthreads();
        const double dd = red[0];
        if (u < t) {
          for (int i = threadIdx.x; i < k; i += blockDim.x) M[i + k * t] -= dd * M[i + k * u];
        } else {
          const double inv = dd > 0.0 ? 1.0 / sqrt(dd) : 0.0;
          for (int i = threadIdx.x; i < k; i += blockDim.x) M[i + k * t] *= inv;
        }
        __syncthreads();
      }
    }
  for (int x = threadIdx.x; x < k * r; x += blockDim.x) out[x] = M[x];
}

}  // namespace

int NewtonWork::ensure(int k1, int k3, int r1, int r3, cudaStream_t s) {
  const int d1 = k1 - r1, d3 = k3 - r3;
  const int64_t N = (int64_t)d1 * r1 + (int64_t)d3 * r3;
  auto grow = [&](DevBuf& b, size_t bytes) -> int {
    if (b.bytes < bytes) {
      BKS_TRY(b.alloc(bytes, s));
      b.persist();
    }
    return BKS_OK;
  };
  BKS_TRY(grow(Up, sizeof(double) * (size_t)k1 * std::max(d1, 1)));
  BKS_TRY(grow(Wp, sizeof(double) * (size_t)k3 * std::max(d3, 1)));
  BKS_TRY(grow(F0, sizeof(double) * (size_t)r1 * r1 * r3));
  BKS_TRY(grow(B1, sizeof(double) * (size_t)std::max(d1, 1) * r1 * r3));
  BKS_TRY(grow(DUp, sizeof(double) * (size_t)k1 * std::max(d1, 1) * r3));
  BKS_TRY(grow(B3, sizeof(double) * (size_t)r1 * r1 * std::max(d3, 1)));
  BKS_TRY(grow(G, sizeof(double) * (size_t)r1 * k1 * std::max(d3, 1)));
  BKS_TRY(grow(B11, sizeof(double) * (size_t)std::max(d1, 1) * std::max(d1, 1) * r3));
  BKS_TRY(grow(B13, sizeof(double) * (size_t)std::max(d1, 1) * r1 * std::max(d3, 1)));
  BKS_TRY(grow(S, sizeof(double) * (size_t)std::max(d1, 1) * std::max(d1, 1)));
  BKS_TRY(grow(S3, sizeof(double) * (size_t)std::max(d3, 1) * std::max(d3, 1)));
  BKS_TRY(grow(M1, sizeof(double) * (size_t)r1 * r1));
  BKS_TRY(grow(M3, sizeof(double) * (size_t)r3 * r3));
  BKS_TRY(grow(grad, sizeof(double) * (size_t)std::max<int64_t>(N, 1)));
  BKS_TRY(grow(z, sizeof(double) * (size_t)std::max<int64_t>(N, 1)));
  BKS_TRY(grow(res, sizeof(double) * (size_t)std::max<int64_t>(N, 1)));
  BKS_TRY(grow(w32, sizeof(float) * (size_t)std::max<int64_t>(N, 1)));
  BKS_TRY(grow(A, sizeof(double) * (size_t)std::max<int64_t>(N * N, 1)));
  BKS_TRY(grow(A32, sizeof(float) * (size_t)std::max<int64_t>(N * N, 1)));
  BKS_TRY(grow(flag, sizeof(int) * 4));
  return BKS_OK;
}

int newton_step(const double* D, const double* T1, const double* E, const double* T3,
                const double* Ug, const double* Wg, int k1, int k3, int r1, int r3,
                double* Un, double* Wn, NewtonWork& w, cudaStream_t s) {
  if (k1 > kNgMaxK || k3 > kNgMaxK || r1 > kNgMaxR || r3 > kNgMaxR || r1 > k1 || r3 > k3)
    return fail(BKS_EUNSUPPORTED, "Newton step: sizes beyond the limits");
  NgDims z{k1, k3, r1, r3, k1 - r1, k3 - r3, (k1 - r1) * r1 + (k3 - r3) * r3};
  BKS_TRY(w.ensure(k1, k3, r1, r3, s));
  if (k1 == r1 && k3 == r3) {
    // no tangent directions: the point is the only one (the gradient is zero)
    BKS_CUDA_TRY(cudaMemsetAsync(w.flag.p, 0xff, sizeof(int), s));
    return BKS_OK;
  }

  k_ng_complement<<<2, 256, 0, s>>>(Ug, k1, r1, Wg, k3, r3, w.Up.as<double>(), w.Wp.as<double>());
  ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  const int64_t n1 = (int64_t)r1 * r1 * r3 + (int64_t)z.d1 * r1 * r3 + (int64_t)k1 * z.d1 * r3 +
                     (int64_t)r1 * r1 * z.d3 + (int64_t)r1 * k1 * z.d3;
  k_ng_blocks1<<<grid_for(n1), 256, 0, s>>>(z, Ug, w.Up.as<double>(), w.Wp.as<double>(), D, T1, E,
                                            T3, w.F0.as<double>(), w.B1.as<double>(),
                                            w.DUp.as<double>(), w.B3.as<double>(),
                                            w.G.as<double>());
  ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  const int64_t n2 = (int64_t)z.d1 * z.d1 * r3 + (int64_t)z.d1 * r1 * z.d3 +
                     (int64_t)z.d1 * z.d1 + (int64_t)z.d3 * z.d3 + r1 * r1 + r3 * r3 +
                     (int64_t)z.d1 * r1 + (int64_t)z.d3 * r3;
  k_ng_blocks2<<<grid_for(n2), 256, 0, s>>>(z, w.Up.as<double>(), w.F0.as<double>(),
                                            w.B1.as<double>(), w.DUp.as<double>(),
                                            w.B3.as<double>(), w.G.as<double>(),
                                            w.B11.as<double>(), w.B13.as<double>(),
                                            w.S.as<double>(), w.S3.as<double>(),
                                            w.M1.as<double>(), w.M3.as<double>(),
                                            w.grad.as<double>());
  ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  k_ng_hessian<<<grid_for((int64_t)z.N * z.N), 256, 0, s>>>(
      z, w.F0.as<double>(), w.B1.as<double>(), w.B11.as<double>(), w.B3.as<double>(),
      w.B13.as<double>(), w.S.as<double>(), w.S3.as<double>(), w.M1.as<double>(),
      w.M3.as<double>(), w.A.as<double>(), w.A32.as<float>());
  ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  // the FP32 factor lives in shared memory when it fits
  static PerDeviceOnce once;
  const cudaError_t attr = once.run([] {
    return cudaFuncSetAttribute(k_ng_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(float) * kNgSmemN * kNgSmemN));
  });
  if (attr != cudaSuccess)
    return fail(BKS_ECUDA, std::string("k_ng_solve shared-memory limit: ") + cudaGetErrorString(attr));
  const size_t smem = z.N <= kNgSmemN ? sizeof(float) * (size_t)z.N * z.N : 0;
  k_ng_solve<<<1, 1024, smem, s>>>(z.N, w.A.as<double>(), w.A32.as<float>(), w.grad.as<double>(),
                                   w.z.as<double>(), w.w32.as<float>(), w.res.as<double>(),
                                   w.flag.as<int>());
  ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  k_ng_update<<<2, 256, 0, s>>>(z, Ug, w.Up.as<double>(), Wg, w.Wp.as<double>(), w.z.as<double>(),
                                Un, Wn);
  ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  return BKS_OK;
}

}  // namespace bks
