// Block-parallel cyclic Jacobi eigensolver for small symmetric matrices held
// in shared memory (Golub & Van Loan, Section 8.5: two-sided Jacobi with a
// round-robin ordering, so the n/2 rotations of one step touch disjoint
// row/column pairs and run concurrently).
#pragma once
#include "common.cuh"

namespace bks {

// A: n x n symmetric (ld = n) in shared memory, overwritten by a nearly
// diagonal matrix; V: n x n in shared memory, receives the eigenvectors
// (columns).  Every thread of the block must call.  `red` is 64 elements
// of shared scratch.  Returns the number of sweeps.
template <typename T>
__device__ int block_jacobi_eig(T* A, T* V, int n, T tol, int max_sweeps, T* red, T* cs) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int x = tid; x < n * n; x += nt) V[x] = (x % n == x / n) ? T(1) : T(0);
  __syncthreads();
  if (n <= 1) return 0;
  const int N = (n + 1) & ~1;  // even number of players (one dummy if n is odd)
  const int half = N / 2;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    // convergence: off-diagonal mass vs total
    T off = 0, tot = 0;
    for (int x = tid; x < n * n; x += nt) {
      T a = A[x];
      tot += a * a;
      if (x % n != x / n) off += a * a;
    }
    // block reduce (two values)
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_down_sync(0xffffffffu, off, o);
      tot += __shfl_down_sync(0xffffffffu, tot, o);
    }
    if ((tid & 31) == 0) { red[tid >> 5] = off; red[32 + (tid >> 5)] = tot; }
    __syncthreads();
    if (tid == 0) {
      T o2 = 0, t2 = 0;
      for (int w = 0; w < (nt + 31) / 32; ++w) { o2 += red[w]; t2 += red[32 + w]; }
      red[0] = o2;
      red[32] = t2;
    }
    __syncthreads();
    const bool done = !(red[0] > tol * tol * red[32]);
    __syncthreads();
    if (done) break;
    for (int step = 0; step < N - 1; ++step) {
      // rotation parameters, one thread per pair
      for (int pi = tid; pi < half; pi += nt) {
        int a = (pi == 0) ? N - 1 : (pi + step) % (N - 1);
        int b = (N - 1 - pi + step) % (N - 1);
        if (pi == 0) a = N - 1, b = step % (N - 1);
        int p = min(a, b), q = max(a, b);
        T c = 1, s = 0;
        if (q < n) {
          T apq = A[p * n + q];
          if (apq != T(0)) {
            T app = A[p * n + p], aqq = A[q * n + q];
            T theta = (aqq - app) / (T(2) * apq);
            T t = (theta >= 0 ? T(1) : T(-1)) / (fabs(theta) + sqrt(theta * theta + T(1)));
            c = T(1) / sqrt(t * t + T(1));
            s = t * c;
          }
        }
        cs[4 * pi + 0] = c;
        cs[4 * pi + 1] = s;
        reinterpret_cast<int*>(cs + 4 * pi + 2)[0] = p;
        reinterpret_cast<int*>(cs + 4 * pi + 3)[0] = q;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int x = tid; x < half * n; x += nt) {
        int pi = x / n, k = x % n;
        int p = reinterpret_cast<int*>(cs + 4 * pi + 2)[0], q = reinterpret_cast<int*>(cs + 4 * pi + 3)[0];
        if (q >= n) continue;
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
        if (q >= n) continue;
        T c = cs[4 * pi], s = cs[4 * pi + 1];
        T apk = A[p * n + k], aqk = A[q * n + k];
        A[p * n + k] = c * apk - s * aqk;
        A[q * n + k] = s * apk + c * aqk;
      }
      __syncthreads();
    }
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
