// Block-parallel cyclic Jacobi eigensolvers for small symmetric matrices
// held in shared memory (Golub & Van Loan, Section 8.5: two-sided Jacobi
// with a round-robin ordering, so the n/2 rotations of one step touch
// disjoint row/column pairs and run concurrently).
#pragma once
#include "common.cuh"

namespace bks {

// A: n x n symmetric positive semidefinite (ld = n) in shared memory,
// overwritten by a nearly diagonal matrix; V: n x n in shared memory,
// receives the eigenvectors (columns).  Every thread of the block must call.
// `red` is 64 elements of shared scratch, `cs` 4*64.  Threshold Jacobi: a
// pair is rotated only while |a_pq| > tol sqrt(a_pp a_qq) and |a_pq| >
// f trace(A), tol = the unit roundoff unless a larger tol is given and
// f = 1e-2 tol in FP64, 4 units of roundoff in FP32; the sweeps stop after
// a sweep without rotations.
// For FP64 the rotation angle is computed in FP32 from FP64 differences and
// the pair (c, s) is then normalised in FP64, so every rotation is
// orthogonal to FP64 precision while costing few FP64 instructions (the
// angle's accuracy only sets how fast a_pq goes to zero).  In FP32 the
// angle is exact to working precision and the rotated a_pq is set to zero
// (the rounding residue would otherwise keep the threshold test from ever
// passing when the diagonal entries differ by orders of magnitude).
// Returns the number of sweeps.
template <typename T>
__device__ int block_jacobi_eig(T* A, T* V, int n, T tol, int max_sweeps, T* red, T* cs) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int x = tid; x < n * n; x += nt) V[x] = (x % n == x / n) ? T(1) : T(0);
  if (tid == 0) {
    T tr = 0;
    for (int k = 0; k < n; ++k) tr += fabs(A[k * n + k]);
    red[0] = tr;
  }
  __syncthreads();
  if (n <= 1) return 0;
  const T ulp = sizeof(T) == 4 ? T(1.1920929e-7) : T(2.220446049250313e-16);
  const T eps = tol > ulp ? tol : ulp;
  const T eps2 = eps * eps;
  // absolute floor: in FP32 entries below a few units of roundoff of the
  // trace are rounding noise of the other rotations
  const T fl = sizeof(T) == 4 ? T(4) * ulp : T(1e-2) * eps;
  const T floor2 = (fl * red[0]) * (fl * red[0]);
  const int N = (n + 1) & ~1;  // even number of players (one dummy if n is odd)
  const int half = N / 2;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    int rotated = 0;
    for (int step = 0; step < N - 1; ++step) {
      for (int pi = tid; pi < half; pi += nt) {
        int a = (pi == 0) ? N - 1 : (pi + step) % (N - 1);
        int b = (pi == 0) ? step % (N - 1) : (N - 1 - pi + step) % (N - 1);
        int p = min(a, b), q = max(a, b);
        T c = 1, s = 0;
        int act = 0;
        if (q < n) {
          const T apq = A[p * n + q];
          const T app = A[p * n + p], aqq = A[q * n + q];
          if (apq * apq > eps2 * fabs(app * aqq) && apq * apq > floor2) {
            act = 1;
            const float fd = (float)(aqq - app), fa = (float)apq;
            const float theta = 0.5f * fd / fa;
            float tf;
            if (fabsf(theta) > 1e7f) tf = 0.5f / theta;
            else tf = (theta >= 0.f ? 1.f : -1.f) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
            const float cf = rsqrtf(tf * tf + 1.f);
            c = (T)cf;
            s = (T)(tf * cf);
            if (sizeof(T) == 8) {
              // exact normalisation in FP64: (c, s) / sqrt(c^2 + s^2), Newton rsqrt
              const T nn = c * c + s * s;
              T y = T(1) - T(0.5) * (nn - T(1));  // nn = 1 + O(1e-7): one Newton step from 1
              y = y * (T(1.5) - T(0.5) * nn * y * y);
              c *= y;
              s *= y;
            }
          }
        }
        cs[4 * pi + 0] = c;
        cs[4 * pi + 1] = s;
        reinterpret_cast<int*>(cs + 4 * pi + 2)[0] = p;
        reinterpret_cast<int*>(cs + 4 * pi + 3)[0] = act ? q : -1;
        rotated |= act;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int x = tid; x < half * n; x += nt) {
        int pi = x / n, k = x % n;
        int p = reinterpret_cast<int*>(cs + 4 * pi + 2)[0], q = reinterpret_cast<int*>(cs + 4 * pi + 3)[0];
        if (q < 0) continue;
        T c = cs[4 * pi], s = cs[4 * pi + 1];
        T akp = A[k * n + p], akq = A[k * n + q];
        A[k * n + p] = c * akp - s * akq;
        A[k * n + q] = s * akp + c * akq;
        T vkp = V[k * n + p], vkq = V[k * n + q];
        V[k * n + p] = c * vkp - s * vkq;
        V[k * n + q] = s * vkp + c * vkq;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int x = tid; x < half * n; x += nt) {
        int pi = x / n, k = x % n;
        int p = reinterpret_cast<int*>(cs + 4 * pi + 2)[0], q = reinterpret_cast<int*>(cs + 4 * pi + 3)[0];
        if (q < 0) continue;
        T c = cs[4 * pi], s = cs[4 * pi + 1];
        T apk = A[p * n + k], aqk = A[q * n + k];
        A[p * n + k] = (sizeof(T) == 4 && k == q) ? T(0) : c * apk - s * aqk;
        A[q * n + k] = (sizeof(T) == 4 && k == p) ? T(0) : s * apk + c * aqk;
      }
      __syncthreads();
    }
    if (!__syncthreads_or(rotated)) break;
  }
  return sweep;
}

// Indices of the r largest diagonal entries of A (descending), written to
// idx[0..r) by thread 0 (selection; n is small).
template <typename T>
__device__ void top_diag(const T* A, int n, int r, int* idx) {
  if (threadIdx.x == 0) {
    for (int t = 0; t < r; ++t) {
      int best = -1;
      for (int x = 0; x < n; ++x) {
        bool used = false;
        for (int u = 0; u < t; ++u) used |= idx[u] == x;
        if (used) continue;
        if (best < 0 || A[x * n + x] > A[best * n + best]) best = x;
      }
      idx[t] = best;
    }
  }
  __syncthreads();
}

}  // namespace bks

namespace bks {

// FP64 reciprocal and reciprocal square root by Newton's method from a
// single-precision first guess (x_{k+1} = x_k (2 - a x_k) and
// y_{k+1} = y_k (3 - a y_k^2) / 2; each step doubles the correct digits:
// 24 -> 48 -> 96 bits).  Used where the FP64 divide and square root, long
// instruction sequences on this GPU, sit on the critical path of a
// one-warp loop.  Arguments outside single-precision range fall back to
// the FP64 operators.
__device__ __forceinline__ double nr_rcp(double a) {
  const double aa = fabs(a);
  if (!(aa > 1e-30 && aa < 1e30)) return 1.0 / a;
  double x = (double)(1.0f / (float)a);
  x = x * (2.0 - a * x);
  x = x * (2.0 - a * x);
  return x;
}
__device__ __forceinline__ double nr_rsqrt(double a) {
  if (!(a > 1e-30 && a < 1e30)) return 1.0 / sqrt(a);
  double y = (double)rsqrtf((float)a);
  y = y * (1.5 - 0.5 * a * y * y);
  y = y * (1.5 - 0.5 * a * y * y);
  return y;
}

// One-warp Jacobi for a small symmetric positive semidefinite matrix A
// (n x n, n <= 64, shared memory) with the round-robin ordering: in each of
// the N-1 steps of a sweep (N = n rounded up to even) the N/2 disjoint
// pairs are rotated at once, lane t computing the rotation of pair t.  A
// pair is rotated only while |a_pq| > eps sqrt(a_pp a_qq) and |a_pq| >
// 1e-2 eps trace(A) (threshold Jacobi, Golub & Van Loan, Section 8.5); the
// sweeps stop when a sweep rotates nothing.  V receives the eigenvectors
// (columns).  cs is shared scratch of 128 elements of T.  Only the calling
// warp may touch A, V, cs.  Used in single precision, where the rotations
// run at the full instruction rate; the inner solve then refines the
// vectors to FP64 accuracy.
__device__ __forceinline__ float rcp_t(float a) { return 1.0f / a; }
__device__ __forceinline__ double rcp_t(double a) { return nr_rcp(a); }
__device__ __forceinline__ float rsqrt_t(float a) { return rsqrtf(a); }
__device__ __forceinline__ double rsqrt_t(double a) { return nr_rsqrt(a); }

template <typename T>
__device__ inline int warp_jacobi_eig(T* A, T* V, int n, int max_sweeps, T* cs) {
  const int lane = threadIdx.x & 31;
  for (int x = lane; x < n * n; x += 32) V[x] = (x % n == x / n) ? T(1) : T(0);
  __syncwarp();
  if (n <= 1) return 0;
  const T eps = sizeof(T) == 4 ? T(1.1920929e-7) : T(2.220446049250313e-16);
  const T eps2 = eps * eps;
  const int N = (n + 1) & ~1;
  const int half = N / 2;
  int* ci = reinterpret_cast<int*>(cs + 64);
  T tr = 0;
  for (int k = 0; k < n; ++k) tr += fabs(A[k * n + k]);
  const T floor2 = (T(1e-2) * eps * tr) * (T(1e-2) * eps * tr);
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    bool rotated = false;
    for (int step = 0; step < N - 1; ++step) {
      bool mine = false;
      if (lane < half) {
        const int a = (lane == 0) ? N - 1 : (lane + step) % (N - 1);
        const int b = (lane == 0) ? step % (N - 1) : (N - 1 - lane + step) % (N - 1);
        const int p = min(a, b), q = max(a, b);
        T c = 1, s = 0;
        if (q < n) {
          const T apq = A[p * n + q];
          const T app = A[p * n + p], aqq = A[q * n + q];
          if (apq * apq > eps2 * fabs(app * aqq) && apq * apq > floor2) {
            mine = true;
            const T theta = (aqq - app) * T(0.5) * rcp_t(apq);
            T t;
            if (fabs(theta) > T(1e7)) {
              t = T(0.5) * rcp_t(theta);
            } else {
              const T r = theta * theta + T(1);
              t = (theta >= 0 ? T(1) : T(-1)) * rcp_t(fabs(theta) + r * rsqrt_t(r));
            }
            c = rsqrt_t(t * t + T(1));
            s = t * c;
          }
        }
        cs[2 * lane] = c;
        cs[2 * lane + 1] = s;
        ci[2 * lane] = p;
        ci[2 * lane + 1] = (q < n && mine) ? q : -1;
      }
      rotated |= __any_sync(0xffffffffu, mine);
      __syncwarp();
      for (int x = lane; x < half * n; x += 32) {  // A <- A J, V <- V J
        const int pi = x / n, k = x % n;
        const int q = ci[2 * pi + 1];
        if (q < 0) continue;
        const int p = ci[2 * pi];
        const T c = cs[2 * pi], s = cs[2 * pi + 1];
        const T akp = A[k * n + p], akq = A[k * n + q];
        A[k * n + p] = c * akp - s * akq;
        A[k * n + q] = s * akp + c * akq;
        const T vkp = V[k * n + p], vkq = V[k * n + q];
        V[k * n + p] = c * vkp - s * vkq;
        V[k * n + q] = s * vkp + c * vkq;
      }
      __syncwarp();
      for (int x = lane; x < half * n; x += 32) {  // A <- J^T A
        const int pi = x / n, k = x % n;
        const int q = ci[2 * pi + 1];
        if (q < 0) continue;
        const int p = ci[2 * pi];
        const T c = cs[2 * pi], s = cs[2 * pi + 1];
        const T apk = A[p * n + k], aqk = A[q * n + k];
        A[p * n + k] = c * apk - s * aqk;
        A[q * n + k] = s * apk + c * aqk;
      }
      __syncwarp();
    }
    if (!rotated) break;
  }
  return sweep;
}

}  // namespace bks
