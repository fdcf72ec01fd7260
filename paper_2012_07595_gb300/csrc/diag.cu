// Conditioning diagnostics and slice normalisations.
//
// * S-values and gaps (Section 2.6) at a point (U, U, W): s_i^(k) =
//   sqrt(lambda_i(<F,F>_{-k})) for i <= r_k, and s_{r_k+1}^(k) =
//   sqrt(lambda_max(<F_perp^k, F_perp^k>_{-k})) with F_perp^1 =
//   A.(U_perp, U, W) and F_perp^3 = A.(U, U, W_perp) (Section 2.5).  Since
//   unfold_1(F_perp^1) = U_perp^T T1 with T1 = unfold_1(A.(I, U, W)),
//   lambda_max is ||(I - U U^T) T1||_2^2: one mode-1 and one mode-3
//   contraction, two projections each (classical Gram-Schmidt twice) and
//   the eigenvalues of small Grams.
// * Per-slice norms of the frontal slices A(:,:,k) (symmetric m x m
//   matrices): the Frobenius norm, or the largest eigenvalue by a batched
//   Lanczos iteration over all slices at once (Section 7 scales adjacency
//   slices to largest eigenvalue 1, or to Frobenius norm 1).
// * A new tensor with its slices scaled.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "dense.cuh"

namespace bks {

namespace {

// ---- host: small symmetric eigenproblems ----------------------------------
// Eigenvalues of the n x n symmetric A (column-major), descending, by the
// cyclic Jacobi method (Golub & Van Loan, Section 8.5): sweeps of plane
// rotations that zero a_pq, until the off-diagonal mass is below 1e-30 of
// the total.
std::vector<double> sym_eigvals(std::vector<double> A, int n) {
  auto at = [&](int r, int c) -> double& { return A[(size_t)r + (size_t)n * c]; };
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int c = 0; c < n; ++c)
      for (int r = 0; r < n; ++r) {
        tot += at(r, c) * at(r, c);
        if (r != c) off += at(r, c) * at(r, c);
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = at(p, q);
        if (apq == 0.0) continue;
        const double theta = (at(q, q) - at(p, p)) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double akp = at(k, p), akq = at(k, q);
          at(k, p) = c * akp - s * akq;
          at(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double apk = at(p, k), aqk = at(q, k);
          at(p, k) = c * apk - s * aqk;
          at(q, k) = s * apk + c * aqk;
        }
      }
  }
  std::vector<double> ev(n);
  for (int i = 0; i < n; ++i) ev[i] = at(i, i);
  std::sort(ev.begin(), ev.end(), [](double x, double y) { return x > y; });
  return ev;
}

// Number of eigenvalues below x of the symmetric tridiagonal matrix with
// diagonal a[0..j) and off-diagonal b[0..j-1), from the signs of the LDL^T
// pivots of T - x I (Sturm sequence, Golub & Van Loan, Section 8.4).
int sturm_below(const double* a, const double* b, int j, double x) {
  int count = 0;
  double d = 1.0;
  for (int i = 0; i < j; ++i) {
    const double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
    d = a[i] - x - (i > 0 ? bb / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) ++count;
  }
  return count;
}

// Largest eigenvalue of that tridiagonal matrix by bisection between the
// Gershgorin bounds, to a relative width of 1e-15.
double tridiag_max_eig(const double* a, const double* b, int j) {
  double lo = 0.0, hi = 0.0;
  for (int i = 0; i < j; ++i) {
    const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < j ? std::fabs(b[i]) : 0.0);
    lo = i == 0 ? a[i] - r : std::min(lo, a[i] - r);
    hi = i == 0 ? a[i] + r : std::max(hi, a[i] + r);
  }
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(std::fabs(lo), std::fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_below(a, b, j, mid) == j) hi = mid;  // every eigenvalue is below mid
    else lo = mid;
  }
  return hi;
}

// ---- device kernels ----------------------------------------------------------
constexpr int kRed = 256;  // threads of the per-column reductions

// Fixed-order block sum of x over the block's threads (result in thread 0).
__device__ __forceinline__ double block_sum(double x, double* sh) {
  sh[threadIdx.x] = x;
  __syncthreads();
  for (int o = kRed / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// out[k] = sqrt(sum of the squared values of slice k) over the rows of the
// mode-3 copy; one block per slice, fixed order.
template <typename V>
__global__ void k_slice_fro(const int32_t* __restrict__ ptr, const V* __restrict__ v, int64_t n,
                            double* __restrict__ out) {
  __shared__ double sh[kRed];
  for (int64_t k = blockIdx.x; k < n; k += gridDim.x) {
    double acc = 0.0;
    for (int32_t e = ptr[k] + threadIdx.x; e < ptr[k + 1]; e += blockDim.x) {
      const double x = (double)v[e];
      acc += x * x;
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) out[k] = sqrt(s);
  }
}

// slice of every entry of the mode-3 copy
__global__ void k_slice_of(const int32_t* __restrict__ ptr, int64_t n, int32_t* __restrict__ kk) {
  for (int64_t k = blockIdx.x; k < n; k += gridDim.x)
    for (int32_t e = ptr[k] + threadIdx.x; e < ptr[k + 1]; e += blockDim.x) kk[e] = (int32_t)k;
}

// 1 where a run of equal (slice, row) starts
__global__ void k_seg_flags(const int32_t* __restrict__ kk, const int32_t* __restrict__ ii,
                            int64_t nnz, int32_t* __restrict__ f) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    f[e] = (e == 0 || kk[e] != kk[e - 1] || ii[e] != ii[e - 1]) ? 1 : 0;
}

__global__ void k_seg_starts(const int32_t* __restrict__ f, const int32_t* __restrict__ pos,
                             int64_t nnz, int32_t* __restrict__ start) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    if (f[e]) start[pos[e]] = (int32_t)e;
}

// first[k] = index of the first run of slice k (the runs that start before
// its first entry), nseg past the last entry
__global__ void k_first_run(const int32_t* __restrict__ ptr, const int32_t* __restrict__ pos,
                            int64_t n, int64_t nnz, int32_t nseg, int32_t* __restrict__ first) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= n;
       k += (int64_t)gridDim.x * blockDim.x)
    first[k] = ptr[k] < nnz ? pos[ptr[k]] : nseg;
}

// y[i + m (k - k0)] = sum over the run's entries of v x[j + m (k - k0)], one
// thread per run of equal (k, i) (the runs s0 .. s1 - 1 of the slices
// k0 .. k0 + nb - 1; run s covers entries seg[s] .. seg[s + 1] - 1), the
// entries in stored order.  Y is zero where no run writes.
template <typename V>
__global__ void k_slice_spmv(const int32_t* __restrict__ seg, int32_t s0, int32_t s1,
                             const int32_t* __restrict__ kk, const int32_t* __restrict__ ii,
                             const int32_t* __restrict__ jj, const V* __restrict__ v, int64_t m,
                             int32_t k0, const double* __restrict__ X, double* __restrict__ Y) {
  for (int64_t s = s0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < s1;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e0 = seg[s], e1 = seg[s + 1];
    const int64_t col = (int64_t)m * (kk[e0] - k0);
    double acc = 0.0;
    for (int32_t e = e0; e < e1; ++e) acc += (double)v[e] * X[jj[e] + col];
    Y[ii[e0] + col] = acc;
  }
}

// Seeded positive start vectors (so that they meet the Perron vector of a
// nonnegative slice), one column per slice: 1 + u/2, u in [0, 1) from a
// counter hash of (row, slice).
__global__ void k_lanczos_start(double* __restrict__ X, int64_t m, int nb, int32_t k0) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m * nb;
       t += (int64_t)gridDim.x * blockDim.x) {
    uint64_t h = (uint64_t)(t % m) * 0x9E3779B97F4A7C15ull + (uint64_t)(k0 + t / m) * 0xD1B54A32D192ED03ull;
    h ^= h >> 31; h *= 0x94D049BB133111EBull; h ^= h >> 29;
    X[t] = 1.0 + 0.5 * (double)(h >> 11) * (1.0 / 9007199254740992.0);
  }
}

// out[c] = x_c . y_c, one block per column, fixed order
__global__ void k_col_dot(const double* __restrict__ X, const double* __restrict__ Y, int64_t m,
                          int nb, double* __restrict__ out) {
  __shared__ double sh[kRed];
  for (int c = blockIdx.x; c < nb; c += gridDim.x) {
    double acc = 0.0;
    for (int64_t r = threadIdx.x; r < m; r += blockDim.x) acc += X[r + m * c] * Y[r + m * c];
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) out[c] = s;
  }
}

// y_c -= alpha_c x_c + beta_c xp_c (beta null: 0), out[c] = ||y_c||
__global__ void k_lanczos_update(double* __restrict__ Y, const double* __restrict__ X,
                                 const double* __restrict__ Xp, const double* __restrict__ alpha,
                                 const double* __restrict__ beta, int64_t m, int nb,
                                 double* __restrict__ out) {
  __shared__ double sh[kRed];
  for (int c = blockIdx.x; c < nb; c += gridDim.x) {
    const double a = alpha[c], b = beta ? beta[c] : 0.0;
    double acc = 0.0;
    for (int64_t r = threadIdx.x; r < m; r += blockDim.x) {
      const int64_t t = r + m * c;
      const double y = Y[t] - a * X[t] - b * Xp[t];
      Y[t] = y;
      acc += y * y;
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) out[c] = sqrt(s);
  }
}

// y_c /= nrm_c where nrm_c > eps_c, else y_c = 0 (an invariant subspace was
// found: the column stays zero)
__global__ void k_col_scale(double* __restrict__ Y, int64_t m, int nb,
                            const double* __restrict__ nrm, const double* __restrict__ eps) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m * nb;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t / m);
    Y[t] = nrm[c] > eps[c] ? Y[t] / nrm[c] : 0.0;
  }
}

template <typename V>
__global__ void k_scale_values(V* __restrict__ v, const int32_t* __restrict__ kk, int64_t nnz,
                               const double* __restrict__ scale) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    v[e] = (V)((double)v[e] * scale[kk[e]]);
}

inline int blocks_for(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 16));
}

template <typename V>
int slice_fro(const bks_tensor* t, double* out, cudaStream_t s) {
  const Part& Q = t->m3;
  k_slice_fro<V><<<(int)std::min<int64_t>(t->n, 65535), kRed, 0, s>>>(
      Q.ptr.as<int32_t>(), Q.v.as<V>(), t->n, out);
  ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  return BKS_OK;
}

// Largest eigenvalue of every slice by Lanczos (no reorthogonalisation: the
// largest Ritz value converges to the largest eigenvalue and never exceeds
// it), slices in batches whose three m x nb work vectors take at most 2 GB.
// A slice stops at convergence (its estimate moved by at most 1e-13 of
// itself over the last 10 steps), at an invariant subspace (the new
// vector's norm below 1e-13 of the slice's Frobenius norm: the estimate is
// then exact), or after min(m, 400) steps.
template <typename V>
int slice_lmax(const bks_tensor* t, double* out, cudaStream_t s) {
  const Part& Q = t->m3;
  const int64_t m = t->m, n = t->n, nnz = t->nnz;
  BKS_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double) * n, s));
  if (nnz == 0) return BKS_OK;
  DevBuf fro, kk, flags, pos, tot, seg;
  BKS_TRY(fro.alloc(sizeof(double) * n, s));
  BKS_TRY(slice_fro<V>(t, fro.as<double>(), s));
  BKS_TRY(kk.alloc(sizeof(int32_t) * nnz, s));
  BKS_TRY(flags.alloc(sizeof(int32_t) * nnz, s));
  BKS_TRY(pos.alloc(sizeof(int32_t) * nnz, s));
  BKS_TRY(tot.alloc(sizeof(int32_t), s));
  k_slice_of<<<(int)std::min<int64_t>(n, 65535), 256, 0, s>>>(Q.ptr.as<int32_t>(), n, kk.as<int32_t>());
  ::bks::note_launch();
  k_seg_flags<<<blocks_for(nnz), 256, 0, s>>>(kk.as<int32_t>(), Q.c0.as<int32_t>(), nnz,
                                               flags.as<int32_t>());
  ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  BKS_TRY(exclusive_scan_i32(flags.as<int32_t>(), pos.as<int32_t>(), nnz, tot.as<int32_t>(), s));
  int32_t nseg = 0;
  BKS_CUDA_TRY(cudaMemcpyAsync(&nseg, tot.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  std::vector<int32_t> hpos;
  BKS_CUDA_TRY(cudaStreamSynchronize(s));
  BKS_TRY(seg.alloc(sizeof(int32_t) * ((size_t)nseg + 1), s));
  k_seg_starts<<<blocks_for(nnz), 256, 0, s>>>(flags.as<int32_t>(), pos.as<int32_t>(), nnz,
                                                seg.as<int32_t>());
  ::bks::note_launch();
  const int32_t nnz32 = (int32_t)nnz;
  BKS_CUDA_TRY(cudaMemcpyAsync(seg.as<int32_t>() + nseg, &nnz32, sizeof(int32_t),
                               cudaMemcpyHostToDevice, s));
  // first run of every slice: the number of runs that start before it
  hpos.resize(n + 1);
  {
    DevBuf first;
    BKS_TRY(first.alloc(sizeof(int32_t) * (n + 1), s));
    k_first_run<<<blocks_for(n + 1), 256, 0, s>>>(Q.ptr.as<int32_t>(), pos.as<int32_t>(), n,
                                                  nnz, nseg, first.as<int32_t>());
    ::bks::note_launch();
    BKS_CUDA_TRY(cudaMemcpyAsync(hpos.data(), first.p, sizeof(int32_t) * (n + 1),
                                 cudaMemcpyDeviceToHost, s));
    BKS_CUDA_TRY(cudaStreamSynchronize(s));
  }
  std::vector<double> hfro(n);
  BKS_CUDA_TRY(cudaMemcpyAsync(hfro.data(), fro.p, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  BKS_CUDA_TRY(cudaStreamSynchronize(s));
  const int64_t nb_max = std::max<int64_t>(1, std::min<int64_t>(n, ((int64_t)1 << 31) / (24 * m)));
  const int maxit = (int)std::min<int64_t>(m, 400);
  DevBuf bx, by, bp, alpha, beta, eps;
  BKS_TRY(bx.alloc(sizeof(double) * m * nb_max, s));
  BKS_TRY(by.alloc(sizeof(double) * m * nb_max, s));
  BKS_TRY(bp.alloc(sizeof(double) * m * nb_max, s));
  BKS_TRY(alpha.alloc(sizeof(double) * (size_t)maxit * nb_max, s));
  BKS_TRY(beta.alloc(sizeof(double) * (size_t)maxit * nb_max, s));
  BKS_TRY(eps.alloc(sizeof(double) * nb_max, s));
  std::vector<double> hout(n, 0.0), ha, hb, heps(nb_max);
  for (int64_t k0 = 0; k0 < n; k0 += nb_max) {
    const int nb = (int)std::min<int64_t>(nb_max, n - k0);
    if (hpos[k0 + nb] == hpos[k0]) continue;  // every slice of the batch is empty
    for (int c = 0; c < nb; ++c) heps[c] = 1e-13 * hfro[k0 + c];
    BKS_CUDA_TRY(cudaMemcpyAsync(eps.p, heps.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, s));
    double *X = bx.as<double>(), *Y = by.as<double>(), *Xp = bp.as<double>();
    const int g = blocks_for(m * nb);
    const int gc = std::min(nb, 65535);
    k_lanczos_start<<<g, 256, 0, s>>>(X, m, nb, (int32_t)k0);
    ::bks::note_launch();
    // normalise the start (beta row 0 holds zeros: alpha = 0 and eps = 0;
    // alpha row 0 receives the norms)
    BKS_CUDA_TRY(cudaMemsetAsync(Xp, 0, sizeof(double) * m * nb, s));
    BKS_CUDA_TRY(cudaMemsetAsync(beta.p, 0, sizeof(double) * nb, s));
    k_lanczos_update<<<gc, kRed, 0, s>>>(X, Xp, Xp, beta.as<double>(), nullptr, m, nb,
                                         alpha.as<double>());
    ::bks::note_launch();
    k_col_scale<<<g, 256, 0, s>>>(X, m, nb, alpha.as<double>(), beta.as<double>());
    ::bks::note_launch();
    std::vector<double> lam(nb, 0.0);
    std::vector<char> done(nb, 0);
    for (int c = 0; c < nb; ++c) done[c] = hpos[k0 + c + 1] == hpos[k0 + c];  // empty slice
    int j = 0;
    while (j < maxit) {
      BKS_CUDA_TRY(cudaMemsetAsync(Y, 0, sizeof(double) * m * nb, s));
      const int32_t s0 = hpos[k0], s1 = hpos[k0 + nb];
      k_slice_spmv<V><<<blocks_for(s1 - s0), 256, 0, s>>>(
          seg.as<int32_t>(), s0, s1, kk.as<int32_t>(), Q.c0.as<int32_t>(), Q.c1.as<int32_t>(),
          Q.v.as<V>(), m, (int32_t)k0, X, Y);
      ::bks::note_launch();
      double* a_j = alpha.as<double>() + (size_t)j * nb;
      double* b_j = beta.as<double>() + (size_t)j * nb;
      k_col_dot<<<gc, kRed, 0, s>>>(X, Y, m, nb, a_j);
      ::bks::note_launch();
      k_lanczos_update<<<gc, kRed, 0, s>>>(Y, X, Xp, a_j, j > 0 ? b_j - nb : nullptr, m, nb, b_j);
      ::bks::note_launch();
      k_col_scale<<<g, 256, 0, s>>>(Y, m, nb, b_j, eps.as<double>());
      ::bks::note_launch();
      BKS_CUDA_TRY(cudaGetLastError());
      std::swap(Xp, X);  // previous <- current
      std::swap(X, Y);   // current <- new; Y takes the old previous (overwritten next step)
      ++j;
      if (j % 10 != 0 && j != maxit) continue;
      ha.resize((size_t)j * nb);
      hb.resize((size_t)j * nb);
      BKS_CUDA_TRY(cudaMemcpyAsync(ha.data(), alpha.p, sizeof(double) * j * nb, cudaMemcpyDeviceToHost, s));
      BKS_CUDA_TRY(cudaMemcpyAsync(hb.data(), beta.p, sizeof(double) * j * nb, cudaMemcpyDeviceToHost, s));
      BKS_CUDA_TRY(cudaStreamSynchronize(s));
      bool all = true;
      std::vector<double> a(j), b(j);
      for (int c = 0; c < nb; ++c) {
        if (done[c]) continue;
        int len = 0;
        bool stop = false;
        for (int q = 0; q < j; ++q) {
          a[q] = ha[(size_t)q * nb + c];
          b[q] = hb[(size_t)q * nb + c];
          ++len;
          if (b[q] <= heps[c]) { stop = true; break; }
        }
        const double l = tridiag_max_eig(a.data(), b.data(), len);
        if (stop || std::fabs(l - lam[c]) <= 1e-13 * std::fabs(l) || j == maxit) done[c] = 1;
        lam[c] = l;
        all = all && done[c];
      }
      if (all) break;
    }
    for (int c = 0; c < nb; ++c) hout[k0 + c] = lam[c];
  }
  BKS_CUDA_TRY(cudaMemcpyAsync(out, hout.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
  BKS_CUDA_TRY(cudaStreamSynchronize(s));
  return BKS_OK;
}

template <typename V>
int scale_values(V* v, const int32_t* kk, int64_t nnz, const double* scales, cudaStream_t s) {
  k_scale_values<V><<<blocks_for(nnz), 256, 0, s>>>(v, kk, nnz, scales);
  ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  return BKS_OK;
}

// Gram P^T P (cols x cols, ld cols) of a tall m x cols block in chunks of at
// most 32 columns (the tall-skinny Gram takes at most 32 right-hand columns).
int full_gram(const double* P, int64_t ldp, int cols, int64_t m, double* G, DenseWork& ws,
              DevBuf& tmp, cudaStream_t s) {
  BKS_TRY(tmp.alloc(sizeof(double) * (size_t)(cols + 32) * 32, s));
  for (int c0 = 0; c0 < cols; c0 += 32) {
    const int b = std::min(32, cols - c0);
    // rows 0..cols-1 of the result: P^T P[:, c0:c0+b]
    BKS_TRY(ts_gram(P, ldp, cols, P + ldp * c0, ldp, b, m, tmp.as<double>(), ws, s));
    BKS_CUDA_TRY(cudaMemcpy2DAsync(G + (size_t)cols * c0, sizeof(double) * cols, tmp.p,
                                   sizeof(double) * (cols + b), sizeof(double) * cols, b,
                                   cudaMemcpyDeviceToDevice, s));
  }
  return BKS_OK;
}

// P <- (I - U U^T) P twice (classical Gram-Schmidt against the orthonormal
// U, repeated for accuracy), in column chunks of at most 32.
int project_out(const double* U, int64_t ldu, int r, double* P, int64_t ldp, int cols, int64_t m,
                DenseWork& ws, DevBuf& tmp, cudaStream_t s) {
  std::vector<double> eye(32 * 32, 0.0);
  for (int q = 0; q < 32; ++q) eye[q + 32 * q] = 1.0;
  DevBuf I, H;
  BKS_TRY(I.alloc(sizeof(double) * 32 * 32, s));
  BKS_TRY(H.alloc(sizeof(double) * (size_t)r * 32, s));
  BKS_TRY(tmp.alloc(sizeof(double) * (size_t)(r + 32) * 32, s));
  BKS_CUDA_TRY(cudaMemcpyAsync(I.p, eye.data(), sizeof(double) * 32 * 32, cudaMemcpyHostToDevice, s));
  for (int round = 0; round < 2; ++round)
    for (int c0 = 0; c0 < cols; c0 += 32) {
      const int b = std::min(32, cols - c0);
      double* Pc = P + ldp * c0;
      BKS_TRY(ts_gram(U, ldu, r, Pc, ldp, b, m, tmp.as<double>(), ws, s));
      // H (r x b) = rows 0..r-1 of the Gram
      BKS_CUDA_TRY(cudaMemcpy2DAsync(H.p, sizeof(double) * r, tmp.p, sizeof(double) * (r + b),
                                     sizeof(double) * r, b, cudaMemcpyDeviceToDevice, s));
      // identity with leading dimension b: the first b x b block of a 32 x 32
      // identity read with ld 32 is not it, so build I_b with ld b
      std::vector<double> eb((size_t)b * b, 0.0);
      for (int q = 0; q < b; ++q) eb[q + (size_t)b * q] = 1.0;
      BKS_CUDA_TRY(cudaMemcpyAsync(I.p, eb.data(), sizeof(double) * b * b, cudaMemcpyHostToDevice, s));
      BKS_CUDA_TRY(cudaStreamSynchronize(s));  // eb is a host temporary
      BKS_TRY(ts_combine(U, ldu, r, Pc, ldp, b, H.as<double>(), I.as<double>(), b, Pc, ldp, m, ws, s));
    }
  return BKS_OK;
}

}  // namespace

int s_values_impl(const bks_tensor* t, const double* U, int64_t ldu, int r1, const double* W,
                  int64_t ldw, int r3, double* s1, double* s3, cudaStream_t s) {
  const int64_t m = t->m, n = t->n;
  const int w1 = r1 * r3, w3 = r1 * r1;
  DevBuf T1, T3, G, tmp;
  DenseWork ws;
  BKS_TRY(T1.alloc(sizeof(double) * m * w1, s));
  BKS_TRY(T3.alloc(sizeof(double) * n * w3, s));
  BKS_TRY(contract_mode1_x(t, U, ldu, r1, W, ldw, r3, T1.as<double>(), m, false, s));
  BKS_TRY(contract_mode3_x(t, U, ldu, r1, U, ldu, r1, T3.as<double>(), n, false, s));
  // F: unfold_1(F) = U^T T1 (r1 x r1 r3)
  BKS_TRY(G.alloc(sizeof(double) * (size_t)(r1 + 32) * 64, s));
  std::vector<double> F((size_t)r1 * w1);
  for (int c0 = 0; c0 < w1; c0 += 32) {
    const int b = std::min(32, w1 - c0);
    BKS_TRY(ts_gram(U, ldu, r1, T1.as<double>() + m * c0, m, b, m, G.as<double>(), ws, s));
    BKS_CUDA_TRY(cudaMemcpy2DAsync(F.data() + (size_t)r1 * c0, sizeof(double) * r1, G.p,
                                   sizeof(double) * (r1 + b), sizeof(double) * r1, b,
                                   cudaMemcpyDeviceToHost, s));
  }
  BKS_CUDA_TRY(cudaStreamSynchronize(s));
  // S-values of F from the Grams of its mode-1 and mode-3 unfoldings
  std::vector<double> G1((size_t)r1 * r1, 0.0), G3((size_t)r3 * r3, 0.0);
  auto f = [&](int a, int b, int c) { return F[(size_t)a + (size_t)r1 * (b + (size_t)r1 * c)]; };
  for (int a = 0; a < r1; ++a)
    for (int a2 = 0; a2 < r1; ++a2) {
      double acc = 0.0;
      for (int c = 0; c < r3; ++c)
        for (int b = 0; b < r1; ++b) acc += f(a, b, c) * f(a2, b, c);
      G1[a + (size_t)r1 * a2] = acc;
    }
  for (int c = 0; c < r3; ++c)
    for (int c2 = 0; c2 < r3; ++c2) {
      double acc = 0.0;
      for (int b = 0; b < r1; ++b)
        for (int a = 0; a < r1; ++a) acc += f(a, b, c) * f(a, b, c2);
      G3[c + (size_t)r3 * c2] = acc;
    }
  const std::vector<double> e1 = sym_eigvals(G1, r1), e3 = sym_eigvals(G3, r3);
  for (int q = 0; q < r1; ++q) s1[q] = std::sqrt(std::max(e1[q], 0.0));
  for (int q = 0; q < r3; ++q) s3[q] = std::sqrt(std::max(e3[q], 0.0));
  // the (r+1)-st: the largest singular value of the projected contractions
  BKS_TRY(project_out(U, ldu, r1, T1.as<double>(), m, w1, m, ws, tmp, s));
  BKS_TRY(project_out(W, ldw, r3, T3.as<double>(), n, w3, n, ws, tmp, s));
  DevBuf PG;
  BKS_TRY(PG.alloc(sizeof(double) * (size_t)std::max(w1 * w1, w3 * w3), s));
  std::vector<double> h1((size_t)w1 * w1), h3((size_t)w3 * w3);
  BKS_TRY(full_gram(T1.as<double>(), m, w1, m, PG.as<double>(), ws, tmp, s));
  BKS_CUDA_TRY(cudaMemcpyAsync(h1.data(), PG.p, sizeof(double) * w1 * w1, cudaMemcpyDeviceToHost, s));
  BKS_CUDA_TRY(cudaStreamSynchronize(s));
  BKS_TRY(full_gram(T3.as<double>(), n, w3, n, PG.as<double>(), ws, tmp, s));
  BKS_CUDA_TRY(cudaMemcpyAsync(h3.data(), PG.p, sizeof(double) * w3 * w3, cudaMemcpyDeviceToHost, s));
  BKS_CUDA_TRY(cudaStreamSynchronize(s));
  s1[r1] = std::sqrt(std::max(sym_eigvals(h1, w1)[0], 0.0));
  s3[r3] = std::sqrt(std::max(sym_eigvals(h3, w3)[0], 0.0));
  return BKS_OK;
}

}  // namespace bks

using namespace bks;

extern "C" int bks_s_values(const bks_tensor* t, const double* U, int64_t ldu, int r1,
                            const double* W, int64_t ldw, int r3, double* s1, double* s3,
                            void* stream) {
  if (!t || !U || !W || !s1 || !s3) return fail(BKS_EINVAL, "null argument");
  BKS_TRY(require_symmetric(t));
  if (r1 < 1 || r3 < 1 || r1 > 8 || r3 > 8 || r1 >= t->m || r3 >= t->n)
    return fail(BKS_EINVAL, "need 1 <= r1 < m, 1 <= r3 < n and r1, r3 <= 8");
  if (ldu < t->m || ldw < t->n) return fail(BKS_EINVAL, "leading dimension below the rows");
  return s_values_impl(t, U, ldu, r1, W, ldw, r3, s1, s3, (cudaStream_t)stream);
}

extern "C" int bks_slice_norms(const bks_tensor* t, int kind, double* norms, void* stream) {
  if (!t || !norms) return fail(BKS_EINVAL, "null argument");
  BKS_TRY(require_symmetric(t));
  cudaStream_t s = (cudaStream_t)stream;
  const bool f64 = t->vdtype == BKS_F64;
  if (kind == BKS_NORM_FRO)
    return f64 ? slice_fro<double>(t, norms, s) : slice_fro<float>(t, norms, s);
  if (kind == BKS_NORM_LMAX)
    return f64 ? slice_lmax<double>(t, norms, s) : slice_lmax<float>(t, norms, s);
  return fail(BKS_EINVAL, "kind must be BKS_NORM_FRO or BKS_NORM_LMAX");
}

extern "C" int bks_tensor_scale_slices(const bks_tensor* t, const double* scales, void* stream,
                                       bks_tensor** out) {
  if (!out) return fail(BKS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!t || !scales) return fail(BKS_EINVAL, "null argument");
  BKS_TRY(require_symmetric(t));
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t nnz = t->nnz;
  const size_t vs = t->vdtype == BKS_F64 ? 8 : 4;
  DevBuf i, j, k, v;
  BKS_TRY(i.alloc(4 * std::max<int64_t>(nnz, 1), s));
  BKS_TRY(j.alloc(4 * std::max<int64_t>(nnz, 1), s));
  BKS_TRY(k.alloc(4 * std::max<int64_t>(nnz, 1), s));
  BKS_TRY(v.alloc(vs * std::max<int64_t>(nnz, 1), s));
  BKS_TRY(bks_tensor_export_coo(t, i.as<int32_t>(), j.as<int32_t>(), k.as<int32_t>(), v.p, stream));
  if (nnz > 0) {
    if (t->vdtype == BKS_F64) BKS_TRY(scale_values<double>(v.as<double>(), k.as<int32_t>(), nnz, scales, s));
    else BKS_TRY(scale_values<float>(v.as<float>(), k.as<int32_t>(), nnz, scales, s));
  }
  // the canonical list has no duplicates and holds both halves: stored as is
  return bks_tensor_create_coo(t->m, t->n, nnz, i.as<int32_t>(), j.as<int32_t>(), k.as<int32_t>(),
                               v.p, t->vdtype, BKS_INPUT_ON_DEVICE, stream, out);
}
