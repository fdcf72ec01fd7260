// Sparse tensor x dense block contractions (Section 2.2; Algorithm 3 step
// (i); Section 4.3.1) and the cores F = A.(U,U,W), C = A.(X,X,Z)
// (eq. (Rayleigh), eq. (tkd)): the front end (operand packing, column
// chunks, cores); the tile kernels are in contract_tile_impl.cuh.
//
// Layout.  The stored tensor has two sorted copies: rows i (entries sorted
// by (j, k) inside a row) for the mode-1 contraction, and rows k (sorted by
// (i, j)) for the mode-3 contraction and the cores.  A contraction writes
// one output row per tensor row, so the work is a segmented reduction over
// the entries of each row:
//
//   out_row[a + p*b] = sum over the row's entries e of v_e * A[ia_e, a] * B[ib_e, b]
//
// with (A, ia, B, ib) = (X, j, Y, k) for mode 1 and (X, i, X2, j) for mode 3.
// Sorting a mode-1 row by j puts the entries that gather the same X row
// next to each other (a long row of a power-law tensor meets each frequent
// j under many k), so that the lanes of one step share cache lines; Y has
// only n rows and is read from shared memory.
//
// Kernel design (work plan in common.cuh): rows longer than `split` are cut
// into pieces whose partial sums a second kernel adds in a fixed order.
// Rows and pieces longer than `tile` entries take one warp each: the lanes
// stride over the entries (coalesced index and value loads, the next group
// loaded while the current one's gathers are in flight) and the lane sums
// are combined by a recursive-halving shuffle reduction.  Shorter rows take
// one lane each, 32 to a warp in order of decreasing length, and are summed
// in registers; their entries are read from a lane-interleaved copy (entry
// t of lane l at base + 32 t + l), so that the warp's loads of one step are
// coalesced as well.  Each warp or lane reads its item (first entry, end,
// output row, partial slot) with one 16-byte load.  No atomics: the result
// is bitwise reproducible.  The dense operands are gathered from row-major
// copies padded to PB (QB) columns (2, 4 or 8; 3 stays 3 in FP64, whose
// kernels are bound by the FP64 pipe), built by a pack kernel, so one entry
// costs one 8-64 byte gather per operand.
#include <algorithm>

#include "contract_tile.cuh"

namespace bks {

namespace {

// ---- pack a column-major m x p block into row-major m x PB (zero padded)
// Rows whose packed width is a multiple of 16 bytes (and a 16-byte aligned
// destination) are written with 16-byte stores.
template <typename IT, typename T>
__device__ __forceinline__ void pack_row(const IT* __restrict__ X, int64_t ldx, int64_t r, int p,
                                         int PB, T* __restrict__ out, bool vec) {
  constexpr int V = (int)(16 / sizeof(T));
  if (vec) {
    for (int a0 = 0; a0 < PB; a0 += V) {
      union { T v[V]; uint4 q; } u;
#pragma unroll
      for (int t = 0; t < V; ++t) u.v[t] = a0 + t < p ? (T)X[r + ldx * (a0 + t)] : T(0);
      reinterpret_cast<uint4*>(out + r * PB + a0)[0] = u.q;
    }
  } else {
    for (int a = 0; a < PB; ++a) out[r * PB + a] = a < p ? (T)X[r + ldx * a] : T(0);
  }
}
template <typename T>
__device__ __forceinline__ bool vec_ok(int PB, const T* out) {
  return (PB % (int)(16 / sizeof(T))) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0;
}

template <typename IT, typename T>
__global__ void k_pack(const IT* __restrict__ X, int64_t ldx, int64_t rows, int p, int PB,
                       T* __restrict__ out) {
  const bool vec = vec_ok(PB, out);
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x)
    pack_row(X, ldx, r, p, PB, out, vec);
}

// Both operands of a contraction in one launch: rows [0, rows1) of the
// first, then the rows of the second.
template <typename IT, typename T>
__global__ void k_pack2(const IT* __restrict__ X, int64_t ldx, int64_t rows1, int p, int PB,
                        T* __restrict__ out1, const IT* __restrict__ Y, int64_t ldy,
                        int64_t rows2, int q, int QB, T* __restrict__ out2) {
  const bool vec1 = vec_ok(PB, out1), vec2 = vec_ok(QB, out2);
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows1 + rows2;
       r += (int64_t)gridDim.x * blockDim.x) {
    if (r < rows1) pack_row(X, ldx, r, p, PB, out1, vec1);
    else pack_row(Y, ldy, r - rows1, q, QB, out2, vec2);
  }
}

template <typename T>
__device__ __forceinline__ void load4(const T* __restrict__ p, T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    float4 q = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else {
    double2 a = __ldg(reinterpret_cast<const double2*>(p));
    double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
}

// Width buckets of the kernels: 1 -> 2, 2..5 as they are, 6..8 -> 8.  The
// kernels multiply only the bucket width (3 x 4 is 12 products per entry,
// 5 x 5 is 25), whatever the row stride.
inline int bucket(int x) { return x <= 2 ? 2 : (x <= 5 ? x : 8); }
template <typename T> int bucket_t(int x) { return bucket(x); }
// Columns of the second operand per kernel call: the accumulators of one
// output row (PB x QB) stay at most 32.
inline int qchunk_of(int PB) { return PB <= 4 ? 8 : (PB == 5 ? 5 : 4); }

template <typename T, typename IT>
int pack_into(const IT* X, int64_t ldx, int64_t rows, int p, int PB, T* dst, cudaStream_t s) {
  k_pack<IT, T><<<grid_for(rows), 256, 0, s>>>(X, ldx, rows, p, PB, dst); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  return BKS_OK;
}

template <typename T, typename IT>
int pack(const IT* X, int64_t ldx, int64_t rows, int p, int PB, DevBuf& buf, cudaStream_t s) {
  BKS_TRY(buf.alloc(sizeof(T) * (size_t)rows * PB, s));
  return pack_into<T, IT>(X, ldx, rows, p, PB, buf.as<T>(), s);
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Temporaries of one mode-1 contraction: the packed operands and the
// partial sums of cut rows.  Taken from a fixed region when `fixed` is
// given (the allocation-free entry point), else allocated on the stream.
struct Mode1Scratch {
  unsigned char* fixed = nullptr;
  size_t fixed_bytes = 0;
};

// Bytes of the temporaries of a mode-1 contraction with widths p x q in
// arithmetic type T (each piece 256-byte aligned): packed X (m x PB),
// packed Y (n x QB, reused by every chunk of Y columns) and the partial
// sums (nslots x PB*QB).
template <typename T>
size_t mode1_scratch_bytes(const bks_tensor* t, int p, int q);

template <typename T, typename IT, typename OT>
int mode1_typed(const bks_tensor* t, const IT* X, int64_t ldx, int p, const IT* Y, int64_t ldy,
                int q, OT* out, int64_t ldo, cudaStream_t s, const Mode1Scratch* fx = nullptr) {
  const int PB = bucket_t<T>(p);
  // keep PB*QB <= 32: the Y columns in chunks of at most qchunk_of(PB)
  const int qchunk = qchunk_of(PB);
  const int QBmax = bucket_t<T>(std::min(qchunk, q));
  const size_t xb = align256(sizeof(T) * (size_t)t->m * row_stride<T>(PB));
  const size_t yb = align256(sizeof(T) * (size_t)t->n * row_stride<T>(QBmax));
  const size_t pb = align256(sizeof(T) * (size_t)t->m1.nslots * PB * QBmax);
  DevBuf own;
  unsigned char* base = nullptr;
  if (fx) {
    if (xb + yb + pb > fx->fixed_bytes)
      return fail(BKS_EUNSUPPORTED, "mode-1 contraction needs " + std::to_string(xb + yb + pb) +
                                        " bytes of scratch, above the fixed " +
                                        std::to_string(fx->fixed_bytes) + " bytes");
    base = fx->fixed;
  } else {
    BKS_TRY(own.alloc(xb + yb + pb, s));
    base = static_cast<unsigned char*>(own.p);
  }
  T* Xp = reinterpret_cast<T*>(base);
  T* Yp = reinterpret_cast<T*>(base + xb);
  T* part = t->m1.nslots > 0 ? reinterpret_cast<T*>(base + xb + yb) : nullptr;
  if (q <= qchunk) {  // one chunk of Y columns: both packs in one launch
    k_pack2<IT, T><<<grid_for(t->m + t->n), 256, 0, s>>>(X, ldx, t->m, p, row_stride<T>(PB), Xp,
                                                         Y, ldy, t->n, q,
                                                         row_stride<T>(QBmax), Yp); ::bks::note_launch();
    BKS_CUDA_TRY(cudaGetLastError());
  } else {
    BKS_TRY((pack_into<T, IT>(X, ldx, t->m, p, row_stride<T>(PB), Xp, s)));
  }
  for (int q0 = 0; q0 < q; q0 += qchunk) {
    const int qq = std::min(qchunk, q - q0);
    const int QB = bucket_t<T>(qq);
    // stream order: the previous chunk's kernels have read Yp and the
    // partial sums before this pack overwrites them
    if (q > qchunk)
      BKS_TRY((pack_into<T, IT>(Y + ldy * q0, ldy, t->n, qq, row_stride<T>(QB), Yp, s)));
    // columns a + p*(q0 + b) of the full output start at column p*q0
    BKS_TRY((dispatch<T, OT>(t->m1, t->vdtype, t->m1.c1.as<int32_t>(), t->m1.c0.as<int32_t>(),
                             Xp, PB, Yp, QB, t->n, false, p, qq, out + ldo * (p * q0), ldo, s,
                             part)));
  }
  return BKS_OK;
}

template <typename T>
size_t mode1_scratch_bytes(const bks_tensor* t, int p, int q) {
  const int PB = bucket_t<T>(p);
  const int QBmax = bucket_t<T>(std::min(qchunk_of(PB), q));
  return align256(sizeof(T) * (size_t)t->m * row_stride<T>(PB)) +
         align256(sizeof(T) * (size_t)t->n * row_stride<T>(QBmax)) +
         align256(sizeof(T) * (size_t)t->m1.nslots * PB * QBmax);
}

template <typename T, typename IT, typename OT>
int mode3_typed(const bks_tensor* t, const IT* X, int64_t ldx, int p, const IT* X2, int64_t ldx2,
                int q, OT* out, int64_t ldo, cudaStream_t s) {
  const int PB = bucket_t<T>(p);
  DevBuf Xp;
  const int qchunk = qchunk_of(PB);
  if (X2 && q <= qchunk) {  // one chunk of X2 columns: both packs in one launch
    const int QB = bucket_t<T>(q);
    const size_t xb = align256(sizeof(T) * (size_t)t->m * row_stride<T>(PB));
    BKS_TRY(Xp.alloc(xb + sizeof(T) * (size_t)t->m * row_stride<T>(QB), s));
    T* X2p = reinterpret_cast<T*>(static_cast<unsigned char*>(Xp.p) + xb);
    k_pack2<IT, T><<<grid_for(2 * t->m), 256, 0, s>>>(X, ldx, t->m, p, row_stride<T>(PB),
                                                      Xp.as<T>(), X2, ldx2, t->m, q,
                                                      row_stride<T>(QB), X2p); ::bks::note_launch();
    BKS_CUDA_TRY(cudaGetLastError());
    return dispatch<T, OT>(t->m3, t->vdtype, t->m3.c0.as<int32_t>(), t->m3.c1.as<int32_t>(),
                           Xp.as<T>(), PB, X2p, QB, t->m, false, p, q, out, ldo, s);
  }
  BKS_TRY((pack<T, IT>(X, ldx, t->m, p, row_stride<T>(PB), Xp, s)));
  if (!X2)
    return dispatch<T, OT>(t->m3, t->vdtype, t->m3.c0.as<int32_t>(), t->m3.c1.as<int32_t>(),
                           Xp.as<T>(), PB, Xp.as<T>(), PB, t->m, true, p, p, out, ldo, s);
  for (int q0 = 0; q0 < q; q0 += qchunk) {
    const int qq = std::min(qchunk, q - q0);
    const int QB = bucket_t<T>(qq);
    DevBuf X2p;
    BKS_TRY((pack<T, IT>(X2 + ldx2 * q0, ldx2, t->m, qq, row_stride<T>(QB), X2p, s)));
    BKS_TRY((dispatch<T, OT>(t->m3, t->vdtype, t->m3.c0.as<int32_t>(), t->m3.c1.as<int32_t>(),
                             Xp.as<T>(), PB, X2p.as<T>(), QB, t->m, false, p, qq,
                             out + ldo * (p * q0), ldo, s)));
  }
  return BKS_OK;
}

// ---- cores ----------------------------------------------------------------
// Small rank (r1 <= 8): F[a,b,c] = sum_k W[k,c] T[k, tri(a,b)] with T the
// triangle mode-3 contraction A.(U,U)_{1,2}.  Blocks of kTriThreads threads
// (the size of the shared reduction array).
constexpr int kTriThreads = 256;
template <typename T, typename IT, typename OT>
__global__ void __launch_bounds__(kTriThreads) k_core_from_tri(const T* __restrict__ Tm, int64_t n, int r1, const IT* __restrict__ W,
                                int64_t ldw, int r3, OT* __restrict__ F) {
  const int ntri = r1 * (r1 + 1) / 2;
  for (int o = blockIdx.x; o < ntri * r3; o += gridDim.x) {
    const int tcol = o % ntri, c = o / ntri;
    __shared__ T sh[kTriThreads];
    T acc = T(0);
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) acc += (T)W[k + ldw * c] * Tm[k + n * tcol];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      int b = 0;
      while ((b + 1) * (b + 2) / 2 <= tcol) ++b;
      const int a = tcol - b * (b + 1) / 2;
      F[a + r1 * (b + r1 * c)] = (OT)sh[0];
      F[b + r1 * (a + r1 * c)] = (OT)sh[0];
    }
    __syncthreads();
  }
}

// Large rank (the Krylov core C = A.(X,X,Z), k1 up to 128): per chunk of
// one slice k, M = sum_e v_e X[i_e,:]^T X[j_e,:] accumulated in registers
// as 4x4 tiles of the upper block triangle; chunk partials are combined
// with Z in a second kernel, C[a,b,c] = sum_k Z[k,c] sum_{chunks of k} M.
//
// A block stages a batch of entries (v X[i,:] and X[j,:], 16-byte vector
// gathers of the packed rows) in shared memory.  When the triangle has
// fewer tiles than the block has threads, the threads form `ngroups`
// groups that take the batch's entries round-robin (entry e to group
// e mod ngroups), each with its own tile accumulators; the groups' sums
// are added in group order at the end, so the result is deterministic.
constexpr int kCoreThreads = 256;

// 16-byte shared-memory vector access (4 floats, or 4 doubles as two
// 16-byte halves); p is 16-byte aligned
template <typename T>
__device__ __forceinline__ void store4_shared(T* p, const T (&x)[4]) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
  } else {
    reinterpret_cast<double2*>(p)[0] = make_double2(x[0], x[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(x[2], x[3]);
  }
}
template <typename T>
__device__ __forceinline__ void load4_shared(const T* p, T (&x)[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    x[0] = q.x; x[1] = q.y; x[2] = q.z; x[3] = q.w;
  } else {
    const double2 q0 = reinterpret_cast<const double2*>(p)[0];
    const double2 q1 = reinterpret_cast<const double2*>(p)[1];
    x[0] = q0.x; x[1] = q0.y; x[2] = q1.x; x[3] = q1.y;
  }
}

template <typename T, int TPT>
__global__ void __launch_bounds__(kCoreThreads)
k_core_chunks(const int32_t* __restrict__ chunk_run, const int32_t* __restrict__ run_start,
              const int32_t* __restrict__ ii, const int32_t* __restrict__ jj,
              const T* __restrict__ vals, const T* __restrict__ Xp, int K, int KP, int batch,
              int ngroups, T* __restrict__ Mpart) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* As = reinterpret_cast<T*>(smem_raw);          // [batch][KP]
  T* Bs = As + (size_t)batch * KP;                  // [batch][KP]
  const int ch = blockIdx.x;
  const int lo = chunk_run[ch], hi = chunk_run[ch + 1];  // the chunk's runs
  const int nt = KP / 4;                            // tiles per side
  const int ntiles = nt * (nt + 1) / 2;
  const int slots = kCoreThreads / ngroups;         // threads per group
  const int g = threadIdx.x / slots, ts = threadIdx.x % slots;
  const bool active = g < ngroups;
  int ta[TPT], tb[TPT];
#pragma unroll
  for (int u = 0; u < TPT; ++u) {
    const int id = ts + u * slots;
    ta[u] = -1; tb[u] = -1;
    if (active && id < ntiles) {
      int b = 0;
      while ((b + 1) * (b + 2) / 2 <= id) ++b;
      ta[u] = id - b * (b + 1) / 2;
      tb[u] = b;
    }
  }
  T acc[TPT][4][4];
#pragma unroll
  for (int u = 0; u < TPT; ++u)
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[u][x][y] = T(0);
  for (int base = lo; base < hi; base += batch) {
    const int cnt = min(batch, hi - base);
    __syncthreads();
    // run r of the batch: As[r] = X[i_r, :], Bs[r] = sum over the run's
    // entries (in order) of v_e X[j_e, :]
    for (int t = threadIdx.x; t < cnt * nt; t += kCoreThreads) {
      const int e = t / nt, q = t % nt;
      const int e0 = run_start[base + e], e1 = run_start[base + e + 1];
      T xa[4], xb[4] = {T(0), T(0), T(0), T(0)};
      load4(Xp + (int64_t)ii[e0] * KP + 4 * q, xa);
      int idx = e0;
      for (; idx + 1 < e1; idx += 2) {  // two gathers in flight
        T y0[4], y1[4];
        const T v0 = vals[idx], v1 = vals[idx + 1];
        load4(Xp + (int64_t)jj[idx] * KP + 4 * q, y0);
        load4(Xp + (int64_t)jj[idx + 1] * KP + 4 * q, y1);
#pragma unroll
        for (int x = 0; x < 4; ++x) xb[x] = fma(v1, y1[x], fma(v0, y0[x], xb[x]));
      }
      if (idx < e1) {
        T y0[4];
        const T v0 = vals[idx];
        load4(Xp + (int64_t)jj[idx] * KP + 4 * q, y0);
#pragma unroll
        for (int x = 0; x < 4; ++x) xb[x] = fma(v0, y0[x], xb[x]);
      }
      store4_shared(As + e * KP + 4 * q, xa);
      store4_shared(Bs + e * KP + 4 * q, xb);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
      if (ta[u] < 0) continue;
      for (int e = g; e < cnt; e += ngroups) {
        T xa[4], xb[4];
        load4_shared(As + e * KP + ta[u] * 4, xa);
        load4_shared(Bs + e * KP + tb[u] * 4, xb);
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[u][x][y] = fma(xa[x], xb[y], acc[u][x][y]);
      }
    }
  }
  T* dst = Mpart + (int64_t)ch * K * K;
  if (ngroups == 1) {
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
      if (ta[u] < 0) continue;
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          const int a = ta[u] * 4 + x, b = tb[u] * 4 + y;
          if (a < K && b < K && a <= b) dst[a + (int64_t)K * b] = acc[u][x][y];
        }
    }
    return;
  }
  // ngroups > 1 (then TPT == 1): group sums in group order through shared
  // memory ([ngroups][ntiles][16], reusing the staging area)
  __syncthreads();
  T* red = As;
  if (ta[0] >= 0) {
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) red[((size_t)g * ntiles + ts) * 16 + 4 * x + y] = acc[0][x][y];
  }
  __syncthreads();
  for (int o = threadIdx.x; o < ntiles * 16; o += kCoreThreads) {
    const int id = o / 16, xy = o % 16;
    T sum = red[(size_t)id * 16 + xy];
    for (int q = 1; q < ngroups; ++q) sum += red[((size_t)q * ntiles + id) * 16 + xy];
    int b = 0;
    while ((b + 1) * (b + 2) / 2 <= id) ++b;
    const int a = (id - b * (b + 1) / 2) * 4 + xy / 4, bb = b * 4 + xy % 4;
    if (a < K && bb < K && a <= bb) dst[a + (int64_t)K * bb] = sum;
  }
}

// S[sl, t] = sum over the chunks of non-empty slice sl (in chunk order) of
// M_chunk[a, b], t = a + b(b+1)/2 (a <= b).
template <typename T>
__global__ void k_core_slice_sum(const T* __restrict__ Mpart, const int32_t* __restrict__ sl_first,
                                 int nsl, int K, T* __restrict__ S) {
  const int ntri = K * (K + 1) / 2;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < (int64_t)nsl * ntri;
       o += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(o % ntri), sl = (int)(o / ntri);
    int b = 0;
    while ((b + 1) * (b + 2) / 2 <= t) ++b;
    const int a = t - b * (b + 1) / 2;
    T sum = T(0);
    for (int ch = sl_first[sl]; ch < sl_first[sl + 1]; ++ch)
      sum += Mpart[(int64_t)ch * K * K + a + (int64_t)K * b];
    S[o] = sum;
  }
}

// C[a,b,c] = C[b,a,c] = sum over non-empty slices (in order) of Z[k,c] S[sl, t].
template <typename T, typename IT, typename OT>
__global__ void k_core_combine(const T* __restrict__ S, const int32_t* __restrict__ sl_k, int nsl,
                               int K, const IT* __restrict__ Z, int64_t ldz, int r3,
                               OT* __restrict__ C) {
  const int ntri = K * (K + 1) / 2;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < (int64_t)ntri * r3;
       o += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(o % ntri), c = (int)(o / ntri);
    int b = 0;
    while ((b + 1) * (b + 2) / 2 <= t) ++b;
    const int a = t - b * (b + 1) / 2;
    T acc = T(0);
    for (int sl = 0; sl < nsl; ++sl)
      acc = fma((T)Z[sl_k[sl] + ldz * c], S[(int64_t)sl * ntri + t], acc);
    C[a + (int64_t)K * (b + (int64_t)K * c)] = (OT)acc;
    C[b + (int64_t)K * (a + (int64_t)K * c)] = (OT)acc;
  }
}

template <typename T, typename IT, typename OT>
int core_typed(const bks_tensor* t, const IT* U, int64_t ldu, int r1, const IT* W, int64_t ldw,
               int r3, OT* F, cudaStream_t s) {
  if (r1 <= 8) {
    const int ntri = r1 * (r1 + 1) / 2;
    DevBuf Tm;
    BKS_TRY(Tm.alloc(sizeof(T) * (size_t)t->n * ntri, s));
    BKS_TRY((mode3_typed<T, IT, T>(t, U, ldu, r1, nullptr, 0, r1, Tm.as<T>(), t->n, s)));
    k_core_from_tri<T, IT, OT><<<std::min(ntri * r3, 1024), kTriThreads, 0, s>>>(Tm.as<T>(), t->n, r1, W,
                                                                         ldw, r3, F); ::bks::note_launch();
    BKS_CUDA_TRY(cudaGetLastError());
    return BKS_OK;
  }
  if (r1 > 128) return fail(BKS_EUNSUPPORTED, "core rank above 128");
  const int KP = (r1 + 3) / 4 * 4;
  const Part& P = t->m3;
  const CorePlan& cp = t->cp;
  const int nch = cp.nch;
  if (nch == 0) {
    BKS_CUDA_TRY(cudaMemsetAsync(F, 0, sizeof(OT) * (size_t)r1 * r1 * r3, s));
    return BKS_OK;
  }
  DevBuf Xp, Mp, Sl;
  BKS_TRY((pack<T, IT>(U, ldu, t->m, r1, KP, Xp, s)));
  BKS_TRY(Mp.alloc(sizeof(T) * (size_t)nch * r1 * r1, s));
  // thread groups over the batch's entries when the triangle has fewer
  // tiles than the block has threads
  const int nt = KP / 4, ntiles = nt * (nt + 1) / 2;
  const int ngroups = ntiles <= kCoreThreads ? std::min(32, kCoreThreads / ntiles) : 1;
  const bool big = ntiles > kCoreThreads;  // k1 > 88: three tiles per thread
  int batch = (int)std::min<size_t>(64, (64 * 1024) / (2 * sizeof(T) * (size_t)KP));
  batch = std::max(batch, 8);
  const size_t smem = std::max(sizeof(T) * 2 * (size_t)batch * KP,
                               sizeof(T) * (size_t)ngroups * ntiles * 16);
  auto kern = big ? k_core_chunks<T, 3> : k_core_chunks<T, 1>;
  // The shared-memory limit is raised once per kernel and device to the
  // largest size any call asks for (k1 <= 128: 64 KB of staged rows, or 528
  // tiles of 16 accumulators), so that calls from several host threads
  // never lower it under one another.
  constexpr size_t kSmemMax = std::max<size_t>(64 * 1024, sizeof(T) * 16 * (32 * 33 / 2));
  static PerDeviceOnce once;
  const cudaError_t attr = once.run([] {
    cudaError_t e = cudaFuncSetAttribute(k_core_chunks<T, 1>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_core_chunks<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kSmemMax);
  });
  if (attr != cudaSuccess)
    return fail(BKS_ECUDA, "k_core_chunks shared-memory limit not accepted");
  if (smem > kSmemMax) return fail(BKS_EUNSUPPORTED, "core: shared-memory tile above its limit");
  kern<<<nch, kCoreThreads, smem, s>>>(cp.chunk_run.as<int32_t>(), cp.run_start.as<int32_t>(),
                                       P.c0.as<int32_t>(), P.c1.as<int32_t>(),
                                       values_of<T>(P, t->vdtype), Xp.as<T>(), r1, KP, batch,
                                       ngroups, Mp.as<T>()); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  const int64_t ntri = (int64_t)r1 * (r1 + 1) / 2;
  BKS_TRY(Sl.alloc(sizeof(T) * (size_t)cp.nsl * ntri, s));
  k_core_slice_sum<T><<<grid_for(cp.nsl * ntri), 256, 0, s>>>(Mp.as<T>(), cp.sl_first.as<int32_t>(),
                                                             cp.nsl, r1, Sl.as<T>()); ::bks::note_launch();
  k_core_combine<T, IT, OT><<<grid_for(ntri * r3), 256, 0, s>>>(Sl.as<T>(), cp.sl_k.as<int32_t>(),
                                                                cp.nsl, r1, W, ldw, r3, F); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  return BKS_OK;
}

// ---- general (nonsymmetric) tensors, Section 5 ----------------------------
// Mode md in {1, 2, 3}: out_row[a + p b] = sum v B1[ia, a] B2[ib, b] over the
// rows of the md-th sorted copy, with (copy, ia, ib, B1 rows, B2 rows) =
// (m1, j, k, m, n), (m2, i, k, l, n), (m3, i, j, l, m).
template <typename T, typename IT, typename OT>
int gen_contract_typed(const bks_tensor* t, int md, const IT* B1, int64_t ld1, int p,
                       const IT* B2, int64_t ld2, int q, OT* out, int64_t ldo, cudaStream_t s) {
  const Part& P = md == 1 ? t->m1 : (md == 2 ? t->m2 : t->m3);
  const int32_t* ia = md == 3 ? P.c0.as<int32_t>() : P.c1.as<int32_t>();
  const int32_t* ib = md == 3 ? P.c1.as<int32_t>() : P.c0.as<int32_t>();
  const int64_t rows1 = md == 1 ? t->m : t->l;
  const int64_t rows2 = md == 3 ? t->m : t->n;
  const int PB = bucket_t<T>(p);
  DevBuf Ap;
  const int qchunk = qchunk_of(PB);
  if (q <= qchunk) {  // one chunk of B2 columns: both packs in one launch
    const int QB = bucket_t<T>(q);
    const size_t ab = align256(sizeof(T) * (size_t)rows1 * row_stride<T>(PB));
    BKS_TRY(Ap.alloc(ab + sizeof(T) * (size_t)rows2 * row_stride<T>(QB), s));
    T* Bp = reinterpret_cast<T*>(static_cast<unsigned char*>(Ap.p) + ab);
    k_pack2<IT, T><<<grid_for(rows1 + rows2), 256, 0, s>>>(B1, ld1, rows1, p, row_stride<T>(PB),
                                                           Ap.as<T>(), B2, ld2, rows2, q,
                                                           row_stride<T>(QB), Bp); ::bks::note_launch();
    BKS_CUDA_TRY(cudaGetLastError());
    return dispatch<T, OT>(P, t->vdtype, ia, ib, Ap.as<T>(), PB, Bp, QB, rows2, false, p, q, out,
                           ldo, s);
  }
  BKS_TRY((pack<T, IT>(B1, ld1, rows1, p, row_stride<T>(PB), Ap, s)));
  for (int q0 = 0; q0 < q; q0 += qchunk) {
    const int qq = std::min(qchunk, q - q0);
    const int QB = bucket_t<T>(qq);
    DevBuf Bp;
    BKS_TRY((pack<T, IT>(B2 + ld2 * q0, ld2, rows2, qq, row_stride<T>(QB), Bp, s)));
    BKS_TRY((dispatch<T, OT>(P, t->vdtype, ia, ib, Ap.as<T>(), PB, Bp.as<T>(), QB, rows2, false,
                             p, qq, out + ldo * (p * q0), ldo, s)));
  }
  return BKS_OK;
}

// General core C = A.(X,Y,Z) (eq. (tkd)), k1, k2 <= 128: per chunk of one
// slice k of the mode-3 copy, M = sum over runs of equal (k, i) of
// X[i,:]^T (sum over the run of v Y[j,:]), all 4x4 tiles of the k1 x k2
// rectangle in registers (TPT tiles per thread); then C[a,b,c] =
// sum_k Z[k,c] sum_{chunks of k} M[a,b].  Groups of threads take a batch's
// runs round-robin when the rectangle has fewer tiles than the block has
// threads; their sums are added in group order.
template <typename T, int TPT>
__global__ void __launch_bounds__(kCoreThreads)
k_gcore_chunks(const int32_t* __restrict__ chunk_run, const int32_t* __restrict__ run_start,
               const int32_t* __restrict__ ii, const int32_t* __restrict__ jj,
               const T* __restrict__ vals, const T* __restrict__ Xp, int K1, int KP1,
               const T* __restrict__ Yp, int K2, int KP2, int batch, int ngroups,
               T* __restrict__ Mpart) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* As = reinterpret_cast<T*>(smem_raw);          // [batch][KP1]
  T* Bs = As + (size_t)batch * KP1;                 // [batch][KP2]
  const int ch = blockIdx.x;
  const int lo = chunk_run[ch], hi = chunk_run[ch + 1];
  const int nt1 = KP1 / 4, nt2 = KP2 / 4, ntiles = nt1 * nt2;
  const int slots = kCoreThreads / ngroups;
  const int g = threadIdx.x / slots, ts = threadIdx.x % slots;
  const bool active = g < ngroups;
  int ta[TPT], tb[TPT];
#pragma unroll
  for (int u = 0; u < TPT; ++u) {
    const int id = ts + u * slots;
    ta[u] = -1; tb[u] = -1;
    if (active && id < ntiles) { ta[u] = id % nt1; tb[u] = id / nt1; }
  }
  T acc[TPT][4][4];
#pragma unroll
  for (int u = 0; u < TPT; ++u)
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[u][x][y] = T(0);
  for (int base = lo; base < hi; base += batch) {
    const int cnt = min(batch, hi - base);
    __syncthreads();
    // run r of the batch: As[r] = X[i_r, :], Bs[r] = sum over the run's
    // entries (in order) of v_e Y[j_e, :]
    for (int t = threadIdx.x; t < cnt * nt1; t += kCoreThreads) {
      const int e = t / nt1, q = t % nt1;
      T xa[4];
      load4(Xp + (int64_t)ii[run_start[base + e]] * KP1 + 4 * q, xa);
      store4_shared(As + e * KP1 + 4 * q, xa);
    }
    for (int t = threadIdx.x; t < cnt * nt2; t += kCoreThreads) {
      const int e = t / nt2, q = t % nt2;
      const int e0 = run_start[base + e], e1 = run_start[base + e + 1];
      T xb[4] = {T(0), T(0), T(0), T(0)};
      for (int idx = e0; idx < e1; ++idx) {
        T y0[4];
        const T v0 = vals[idx];
        load4(Yp + (int64_t)jj[idx] * KP2 + 4 * q, y0);
#pragma unroll
        for (int x = 0; x < 4; ++x) xb[x] = fma(v0, y0[x], xb[x]);
      }
      store4_shared(Bs + e * KP2 + 4 * q, xb);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
      if (ta[u] < 0) continue;
      for (int e = g; e < cnt; e += ngroups) {
        T xa[4], xb[4];
        load4_shared(As + e * KP1 + ta[u] * 4, xa);
        load4_shared(Bs + e * KP2 + tb[u] * 4, xb);
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[u][x][y] = fma(xa[x], xb[y], acc[u][x][y]);
      }
    }
  }
  T* dst = Mpart + (int64_t)ch * K1 * K2;
  if (ngroups == 1) {
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
      if (ta[u] < 0) continue;
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          const int a = ta[u] * 4 + x, b = tb[u] * 4 + y;
          if (a < K1 && b < K2) dst[a + (int64_t)K1 * b] = acc[u][x][y];
        }
    }
    return;
  }
  // ngroups > 1 (then TPT == 1): group sums in group order through shared
  // memory ([ngroups][ntiles][16], reusing the staging area)
  __syncthreads();
  T* red = As;
  if (ta[0] >= 0) {
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) red[((size_t)g * ntiles + ts) * 16 + 4 * x + y] = acc[0][x][y];
  }
  __syncthreads();
  for (int o = threadIdx.x; o < ntiles * 16; o += kCoreThreads) {
    const int id = o / 16, xy = o % 16;
    T sum = red[(size_t)id * 16 + xy];
    for (int q = 1; q < ngroups; ++q) sum += red[((size_t)q * ntiles + id) * 16 + xy];
    const int a = (id % nt1) * 4 + xy / 4, b = (id / nt1) * 4 + xy % 4;
    if (a < K1 && b < K2) dst[a + (int64_t)K1 * b] = sum;
  }
}

// S[sl, x] = sum over the chunks of non-empty slice sl (in chunk order) of
// M_chunk[x], x = a + K1 b.
template <typename T>
__global__ void k_gcore_slice_sum(const T* __restrict__ Mpart, const int32_t* __restrict__ sl_first,
                                  int nsl, int64_t kk, T* __restrict__ S) {
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < (int64_t)nsl * kk;
       o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = o % kk;
    const int sl = (int)(o / kk);
    T sum = T(0);
    for (int ch = sl_first[sl]; ch < sl_first[sl + 1]; ++ch) sum += Mpart[(int64_t)ch * kk + x];
    S[o] = sum;
  }
}

// C[x + kk c] = sum over non-empty slices (in order) of Z[k,c] S[sl, x].
template <typename T>
__global__ void k_gcore_combine(const T* __restrict__ S, const int32_t* __restrict__ sl_k, int nsl,
                                int64_t kk, const double* __restrict__ Z, int64_t ldz, int k3,
                                double* __restrict__ C) {
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < kk * k3;
       o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = o % kk;
    const int c = (int)(o / kk);
    T acc = T(0);
    for (int sl = 0; sl < nsl; ++sl) acc = fma((T)Z[sl_k[sl] + ldz * c], S[(int64_t)sl * kk + x], acc);
    C[o] = (double)acc;
  }
}

int gen_core_fp64(const bks_tensor* t, const double* X, int64_t ldx, int k1, const double* Y,
                  int64_t ldy, int k2, const double* Z, int64_t ldz, int k3, double* C,
                  cudaStream_t s) {
  using T = double;
  const CorePlan& cp = t->cp;
  const int64_t kk = (int64_t)k1 * k2;
  if (cp.nch == 0 || kk * k3 == 0) {
    if (kk * k3 > 0) BKS_CUDA_TRY(cudaMemsetAsync(C, 0, sizeof(double) * (size_t)kk * k3, s));
    return BKS_OK;
  }
  const int KP1 = (k1 + 3) / 4 * 4, KP2 = (k2 + 3) / 4 * 4;
  const int nt1 = KP1 / 4, nt2 = KP2 / 4, ntiles = nt1 * nt2;
  const int tpt = ntiles <= kCoreThreads ? 1 : (ntiles <= 2 * kCoreThreads ? 2 : 4);
  const int ngroups = ntiles <= kCoreThreads ? std::min(32, kCoreThreads / ntiles) : 1;
  int batch = (int)std::min<size_t>(64, (64 * 1024) / (sizeof(T) * (size_t)(KP1 + KP2)));
  batch = std::max(batch, 8);
  // the group reduction reuses the staging area when there are groups
  const size_t smem = std::max(sizeof(T) * (size_t)batch * (KP1 + KP2),
                               ngroups > 1 ? sizeof(T) * (size_t)ngroups * ntiles * 16 : 0);
  constexpr size_t kSmemMax = 64 * 1024;
  static PerDeviceOnce once;
  const cudaError_t attr = once.run([] {
    cudaError_t e = cudaFuncSetAttribute(k_gcore_chunks<T, 1>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_gcore_chunks<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kSmemMax);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_gcore_chunks<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kSmemMax);
    return e;
  });
  if (attr != cudaSuccess) return fail(BKS_ECUDA, "k_gcore_chunks shared-memory limit not accepted");
  if (smem > kSmemMax) return fail(BKS_EUNSUPPORTED, "general core: shared-memory tile above its limit");
  DevBuf Xp, Yp, Mp, Sl;
  BKS_TRY((pack<T, double>(X, ldx, t->l, k1, KP1, Xp, s)));
  BKS_TRY((pack<T, double>(Y, ldy, t->m, k2, KP2, Yp, s)));
  BKS_TRY(Mp.alloc(sizeof(T) * (size_t)cp.nch * kk, s));
  const Part& P = t->m3;
  auto kern = tpt == 1 ? k_gcore_chunks<T, 1> : (tpt == 2 ? k_gcore_chunks<T, 2> : k_gcore_chunks<T, 4>);
  kern<<<cp.nch, kCoreThreads, smem, s>>>(cp.chunk_run.as<int32_t>(), cp.run_start.as<int32_t>(),
                                          P.c0.as<int32_t>(), P.c1.as<int32_t>(),
                                          values_of<T>(P, t->vdtype), Xp.as<T>(), k1, KP1,
                                          Yp.as<T>(), k2, KP2, batch, ngroups, Mp.as<T>()); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  BKS_TRY(Sl.alloc(sizeof(T) * (size_t)cp.nsl * kk, s));
  k_gcore_slice_sum<T><<<grid_for(cp.nsl * kk), 256, 0, s>>>(Mp.as<T>(), cp.sl_first.as<int32_t>(),
                                                            cp.nsl, kk, Sl.as<T>()); ::bks::note_launch();
  k_gcore_combine<T><<<grid_for(kk * k3), 256, 0, s>>>(Sl.as<T>(), cp.sl_k.as<int32_t>(), cp.nsl,
                                                       kk, Z, ldz, k3, C); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  return BKS_OK;
}

// ---- run plan of the core ---------------------------------------------------
// Runs: maximal ranges of equal (slice, i) of the mode-3 copy, cut at chunk
// starts and after every kRunCap entries.
constexpr int kRunCap = 32;

// f[e] = 1 where i changes; chunk starts are set by k_mark_starts
__global__ void k_run_flags(const int32_t* __restrict__ ii, int64_t nnz, int32_t* __restrict__ f) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    f[e] = (e == 0 || ii[e] != ii[e - 1]) ? 1 : 0;
}
__global__ void k_mark_starts(const int32_t* __restrict__ lo, int nch, int32_t* __restrict__ f) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nch; c += gridDim.x * blockDim.x)
    f[lo[c]] = 1;
}
__global__ void k_run_scatter(const int32_t* __restrict__ f, const int32_t* __restrict__ id,
                              int64_t nnz, int32_t* __restrict__ start) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    if (f[e]) start[id[e]] = (int32_t)e;
}
// f2[e] = 1 where a run of f starts or kRunCap entries of it have passed
__global__ void k_run_cap(const int32_t* __restrict__ f, const int32_t* __restrict__ id,
                          const int32_t* __restrict__ start, int64_t nnz, int32_t* __restrict__ f2) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t run = id[e] - 1 + f[e];
    f2[e] = (f[e] || (e - start[run]) % kRunCap == 0) ? 1 : 0;
  }
}
__global__ void k_chunk_runs(const int32_t* __restrict__ lo, int nch, const int32_t* __restrict__ id,
                             int32_t nruns, int32_t* __restrict__ chunk_run) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= nch; c += gridDim.x * blockDim.x)
    chunk_run[c] = c < nch ? id[lo[c]] : nruns;
}

}  // namespace

// Core chunk plan (see CorePlan): host loop over the slices of the mode-3
// copy, uploaded once.
int build_core_plan(const Part& m3, int64_t n, int64_t nnz, CorePlan& cp, cudaStream_t s) {
  // about 16 chunks per SM: several waves of blocks, so that uneven
  // chunk times even out across the SMs
  const int64_t target = std::max<int64_t>(256, nnz / (16LL * num_sms()) + 1);
  std::vector<int32_t> lo, hi, slk, slf;
  for (int64_t k = 0; k < n; ++k) {
    const int32_t a = m3.host_ptr[k], b = m3.host_ptr[k + 1];
    if (b <= a) continue;
    slk.push_back((int32_t)k);
    slf.push_back((int32_t)lo.size());
    for (int64_t x = a; x < b; x += target) {
      lo.push_back((int32_t)x);
      hi.push_back((int32_t)std::min<int64_t>(b, x + target));
    }
  }
  slf.push_back((int32_t)lo.size());
  cp.nch = (int32_t)lo.size();
  cp.nsl = (int32_t)slk.size();
  if (cp.nch == 0) return BKS_OK;
  BKS_TRY(cp.lo.alloc(4 * lo.size(), s));
  BKS_TRY(cp.hi.alloc(4 * hi.size(), s));
  BKS_TRY(cp.sl_k.alloc(4 * slk.size(), s));
  BKS_TRY(cp.sl_first.alloc(4 * slf.size(), s));
  BKS_CUDA_TRY(cudaMemcpyAsync(cp.lo.p, lo.data(), 4 * lo.size(), cudaMemcpyHostToDevice, s));
  BKS_CUDA_TRY(cudaMemcpyAsync(cp.hi.p, hi.data(), 4 * hi.size(), cudaMemcpyHostToDevice, s));
  BKS_CUDA_TRY(cudaMemcpyAsync(cp.sl_k.p, slk.data(), 4 * slk.size(), cudaMemcpyHostToDevice, s));
  BKS_CUDA_TRY(cudaMemcpyAsync(cp.sl_first.p, slf.data(), 4 * slf.size(), cudaMemcpyHostToDevice, s));
  // the host vectors are read by the async copies: wait before they go
  BKS_CUDA_TRY(cudaStreamSynchronize(s));
  // runs of equal (slice, i), cut at chunk starts and every kRunCap entries
  {
    DevBuf f1, id1, st1, f2, id2, tot;
    BKS_TRY(f1.alloc(4 * nnz, s));
    BKS_TRY(id1.alloc(4 * nnz, s));
    BKS_TRY(st1.alloc(4 * nnz, s));
    BKS_TRY(f2.alloc(4 * nnz, s));
    BKS_TRY(id2.alloc(4 * nnz, s));
    BKS_TRY(tot.alloc(4, s));
    const int g = grid_for(nnz);
    k_run_flags<<<g, 256, 0, s>>>(m3.c0.as<int32_t>(), nnz, f1.as<int32_t>()); ::bks::note_launch();
    k_mark_starts<<<grid_for(cp.nch), 256, 0, s>>>(cp.lo.as<int32_t>(), cp.nch, f1.as<int32_t>()); ::bks::note_launch();
    BKS_TRY(exclusive_scan_i32(f1.as<int32_t>(), id1.as<int32_t>(), nnz, tot.as<int32_t>(), s));
    k_run_scatter<<<g, 256, 0, s>>>(f1.as<int32_t>(), id1.as<int32_t>(), nnz, st1.as<int32_t>()); ::bks::note_launch();
    k_run_cap<<<g, 256, 0, s>>>(f1.as<int32_t>(), id1.as<int32_t>(), st1.as<int32_t>(), nnz,
                                f2.as<int32_t>()); ::bks::note_launch();
    BKS_TRY(exclusive_scan_i32(f2.as<int32_t>(), id2.as<int32_t>(), nnz, tot.as<int32_t>(), s));
    int32_t nruns = 0;
    BKS_CUDA_TRY(cudaMemcpyAsync(&nruns, tot.p, 4, cudaMemcpyDeviceToHost, s));
    BKS_CUDA_TRY(cudaStreamSynchronize(s));
    cp.nruns = nruns;
    BKS_TRY(cp.run_start.alloc(4 * ((size_t)nruns + 1), s));
    BKS_TRY(cp.chunk_run.alloc(4 * ((size_t)cp.nch + 1), s));
    k_run_scatter<<<g, 256, 0, s>>>(f2.as<int32_t>(), id2.as<int32_t>(), nnz,
                                    cp.run_start.as<int32_t>()); ::bks::note_launch();
    const int32_t end = (int32_t)nnz;
    BKS_CUDA_TRY(cudaMemcpyAsync(cp.run_start.as<int32_t>() + nruns, &end, 4,
                                 cudaMemcpyHostToDevice, s));
    k_chunk_runs<<<grid_for(cp.nch + 1), 256, 0, s>>>(cp.lo.as<int32_t>(), cp.nch, id2.as<int32_t>(),
                                                      nruns, cp.chunk_run.as<int32_t>()); ::bks::note_launch();
    BKS_CUDA_TRY(cudaGetLastError());
    BKS_CUDA_TRY(cudaStreamSynchronize(s));  // `end` is a host temporary
  }
  return BKS_OK;
}

// First operands wider than the largest kernel bucket (8 columns): for each
// column b of the second operand, the first operand in chunks of at most 8
// columns [a0, a0 + pp).  Output columns a + p*b, a in the chunk, are then
// the columns of a pp x 1 product written from column a0 + p*b on (mode 1
// and full mode 3), or from a0 + b(b+1)/2 on with the chunks cut at b
// (triangle: a <= b).  One tensor pass per chunk and column: a completeness
// path for wide operands, not the solvers' path.
constexpr int kWideChunk = 8;

template <typename T>
int mode1_wide(const bks_tensor* t, const T* X, int64_t ldx, int p, const T* Y, int64_t ldy,
               int q, T* out, int64_t ldo, cudaStream_t s) {
  for (int b = 0; b < q; ++b)
    for (int a0 = 0; a0 < p; a0 += kWideChunk) {
      const int pp = std::min(kWideChunk, p - a0);
      BKS_TRY((mode1_typed<T, T, T>(t, X + ldx * a0, ldx, pp, Y + ldy * b, ldy, 1,
                                    out + ldo * (a0 + (int64_t)p * b), ldo, s)));
    }
  return BKS_OK;
}

template <typename T>
int mode3_wide(const bks_tensor* t, const T* X, int64_t ldx, int p, const T* X2, int64_t ldx2,
               int q, T* out, int64_t ldo, cudaStream_t s) {
  const bool tri = X2 == nullptr;
  const int nb = tri ? p : q;
  for (int b = 0; b < nb; ++b) {
    const int alim = tri ? b + 1 : p;
    const int64_t col0 = tri ? (int64_t)b * (b + 1) / 2 : (int64_t)p * b;
    const T* xb = tri ? X + ldx * b : X2 + ldx2 * b;
    const int64_t ldb = tri ? ldx : ldx2;
    for (int a0 = 0; a0 < alim; a0 += kWideChunk) {
      const int pp = std::min(kWideChunk, alim - a0);
      BKS_TRY((mode3_typed<T, T, T>(t, X + ldx * a0, ldx, pp, xb, ldb, 1,
                                    out + ldo * (col0 + a0), ldo, s)));
    }
  }
  return BKS_OK;
}

int contract_mode1(const bks_tensor* t, const void* X, int64_t ldx, int p, const void* Y,
                   int64_t ldy, int q, void* out, int64_t ldo, int dtype, cudaStream_t s) {
  if (p > kWideChunk) {
    if (dtype == BKS_F64)
      return mode1_wide<double>(t, (const double*)X, ldx, p, (const double*)Y, ldy, q,
                                (double*)out, ldo, s);
    return mode1_wide<float>(t, (const float*)X, ldx, p, (const float*)Y, ldy, q, (float*)out,
                             ldo, s);
  }
  if (dtype == BKS_F64)
    return mode1_typed<double, double, double>(t, (const double*)X, ldx, p, (const double*)Y, ldy,
                                               q, (double*)out, ldo, s);
  return mode1_typed<float, float, float>(t, (const float*)X, ldx, p, (const float*)Y, ldy, q,
                                          (float*)out, ldo, s);
}

int contract_mode3(const bks_tensor* t, const void* X, int64_t ldx, int p, const void* X2,
                   int64_t ldx2, int q, void* out, int64_t ldo, int dtype, cudaStream_t s) {
  if (p > kWideChunk) {
    if (dtype == BKS_F64)
      return mode3_wide<double>(t, (const double*)X, ldx, p, (const double*)X2, ldx2, q,
                                (double*)out, ldo, s);
    return mode3_wide<float>(t, (const float*)X, ldx, p, (const float*)X2, ldx2, q, (float*)out,
                             ldo, s);
  }
  if (dtype == BKS_F64)
    return mode3_typed<double, double, double>(t, (const double*)X, ldx, p, (const double*)X2,
                                               ldx2, q, (double*)out, ldo, s);
  return mode3_typed<float, float, float>(t, (const float*)X, ldx, p, (const float*)X2, ldx2, q,
                                          (float*)out, ldo, s);
}

int contract_core(const bks_tensor* t, const void* U, int64_t ldu, int r1, const void* W,
                  int64_t ldw, int r3, void* F, int dtype, cudaStream_t s) {
  if (dtype == BKS_F64)
    return core_typed<double, double, double>(t, (const double*)U, ldu, r1, (const double*)W, ldw,
                                              r3, (double*)F, s);
  return core_typed<float, float, float>(t, (const float*)U, ldu, r1, (const float*)W, ldw, r3,
                                         (float*)F, s);
}

// FP64 operands and results; fp32 = true computes in FP32 (the mixed form)
int contract_mode1_x(const bks_tensor* t, const double* X, int64_t ldx, int p, const double* Y,
                     int64_t ldy, int q, double* out, int64_t ldo, bool fp32, cudaStream_t s) {
  if (fp32) return mode1_typed<float, double, double>(t, X, ldx, p, Y, ldy, q, out, ldo, s);
  return mode1_typed<double, double, double>(t, X, ldx, p, Y, ldy, q, out, ldo, s);
}
int contract_mode3_x(const bks_tensor* t, const double* X, int64_t ldx, int p, const double* X2,
                     int64_t ldx2, int q, double* out, int64_t ldo, bool fp32, cudaStream_t s) {
  if (fp32) return mode3_typed<float, double, double>(t, X, ldx, p, X2, ldx2, q, out, ldo, s);
  return mode3_typed<double, double, double>(t, X, ldx, p, X2, ldx2, q, out, ldo, s);
}
int contract_core_x(const bks_tensor* t, const double* U, int64_t ldu, int r1, const double* W,
                    int64_t ldw, int r3, double* F, bool fp32, cudaStream_t s) {
  if (fp32) return core_typed<float, double, double>(t, U, ldu, r1, W, ldw, r3, F, s);
  return core_typed<double, double, double>(t, U, ldu, r1, W, ldw, r3, F, s);
}

int gen_contract_x(const bks_tensor* t, int md, const double* B1, int64_t ld1, int p,
                   const double* B2, int64_t ld2, int q, double* out, int64_t ldo, cudaStream_t s) {
  return gen_contract_typed<double, double, double>(t, md, B1, ld1, p, B2, ld2, q, out, ldo, s);
}
int gen_core_x(const bks_tensor* t, const double* X, int64_t ldx, int k1, const double* Y,
               int64_t ldy, int k2, const double* Z, int64_t ldz, int k3, double* C,
               cudaStream_t s) {
  return gen_core_fp64(t, X, ldx, k1, Y, ldy, k2, Z, ldz, k3, C, s);
}

}  // namespace bks

using namespace bks;

static int check_common(const bks_tensor* t, const void* X, int64_t ldx, int p, int dtype,
                        int64_t rows) {
  if (!t) return fail(BKS_EINVAL, "null tensor");
  if (!X) return fail(BKS_EINVAL, "null operand");
  if (dtype != BKS_F32 && dtype != BKS_F64) return fail(BKS_EINVAL, "dtype must be BKS_F32 or BKS_F64");
  if (ldx < rows) return fail(BKS_EINVAL, "leading dimension smaller than the row count");
  if (p < 1) return fail(BKS_EINVAL, "width must be >= 1");
  return BKS_OK;
}

extern "C" int bks_contract_mode1(const bks_tensor* t, const void* X, int64_t ldx, int p,
                                  const void* Y, int64_t ldy, int q, void* out, int64_t ldo,
                                  int dtype, void* stream) {
  BKS_TRY(require_symmetric(t));
  BKS_TRY(check_common(t, X, ldx, p, dtype, t ? t->m : 0));
  BKS_TRY(check_common(t, Y, ldy, q, dtype, t->n));
  if (!out || ldo < t->m) return fail(BKS_EINVAL, "bad output");
  return contract_mode1(t, X, ldx, p, Y, ldy, q, out, ldo, dtype, (cudaStream_t)stream);
}

extern "C" int bks_contract_mode3(const bks_tensor* t, const void* X, int64_t ldx, int p,
                                  const void* X2, int64_t ldx2, int q, void* out, int64_t ldo,
                                  int dtype, void* stream) {
  BKS_TRY(require_symmetric(t));
  BKS_TRY(check_common(t, X, ldx, p, dtype, t ? t->m : 0));
  if (X2) BKS_TRY(check_common(t, X2, ldx2, q, dtype, t->m));
  if (!out || ldo < t->n) return fail(BKS_EINVAL, "bad output");
  return contract_mode3(t, X, ldx, p, X2, ldx2, q, out, ldo, dtype, (cudaStream_t)stream);
}

extern "C" int bks_core(const bks_tensor* t, const void* U, int64_t ldu, int r1, const void* W,
                        int64_t ldw, int r3, void* F, int dtype, void* stream) {
  BKS_TRY(require_symmetric(t));
  BKS_TRY(check_common(t, U, ldu, r1, dtype, t ? t->m : 0));
  BKS_TRY(check_common(t, W, ldw, r3, dtype, t->n));
  if (!F) return fail(BKS_EINVAL, "null F");
  if (r1 > 128 || r3 > 128) return fail(BKS_EUNSUPPORTED, "core ranks must be <= 128");
  return contract_core(t, U, ldu, r1, W, ldw, r3, F, dtype, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// Mode-1 contraction without device allocation.
//
// Some callers cannot allocate device memory: a host framework that has
// reserved the whole device for its own memory pool, or code that must not
// let a library call cudaMalloc (which can synchronise the device and fail
// under memory pressure).  This variant keeps the contraction's scratch --
// the packed row-major copies of X and Y and the partial sums of long rows --
// in one file-scope device array of fixed size instead of allocating it.
// ---------------------------------------------------------------------------
namespace bks {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
unsigned char* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device with that device current (host code only sees a stand-in
// symbol, not a device address).
int noalloc_scratch(unsigned char** out) {
  const int dev = current_device();
  if (dev < 0) return fail(BKS_EUNSUPPORTED, "no current device, or a device index above 63");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    BKS_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return BKS_OK;
}

// The allocating path's own code with its temporaries in the fixed array:
// the same buckets, kernels and summation order, hence the same bits.
template <typename T>
int mode1_noalloc_typed(const bks_tensor* t, const T* X, int64_t ldx, int p, const T* Y,
                        int64_t ldy, int q, T* out, int64_t ldo, cudaStream_t s) {
  const size_t need = mode1_scratch_bytes<T>(t, p, q);
  if (need > kNoAllocScratchBytes)
    return fail(BKS_EUNSUPPORTED,
                "bks_contract_mode1_noalloc: needs " + std::to_string(need) +
                    " bytes of scratch, above the fixed " +
                    std::to_string(kNoAllocScratchBytes) + " bytes");
  Mode1Scratch fx;
  BKS_TRY(noalloc_scratch(&fx.fixed));
  fx.fixed_bytes = kNoAllocScratchBytes;
  return mode1_typed<T, T, T>(t, X, ldx, p, Y, ldy, q, out, ldo, s, &fx);
}

}  // namespace
}  // namespace bks

extern "C" int bks_contract_mode1_noalloc(const bks_tensor* t, const void* X, int64_t ldx,
                                          int p, const void* Y, int64_t ldy, int q, void* out,
                                          int64_t ldo, int dtype, void* stream) {
  BKS_TRY(require_symmetric(t));
  BKS_TRY(check_common(t, X, ldx, p, dtype, t ? t->m : 0));
  BKS_TRY(check_common(t, Y, ldy, q, dtype, t->n));
  if (!out || ldo < t->m) return fail(BKS_EINVAL, "bad output");
  if (p > 8 || q > 8) return fail(BKS_EUNSUPPORTED, "mode-1 widths p, q must be <= 8");
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == BKS_F64)
    return mode1_noalloc_typed<double>(t, (const double*)X, ldx, p, (const double*)Y, ldy, q,
                                       (double*)out, ldo, s);
  return mode1_noalloc_typed<float>(t, (const float*)X, ldx, p, (const float*)Y, ldy, q,
                                    (float*)out, ldo, s);
}

extern "C" int bks_gen_contract(const bks_tensor* t, int mode, const void* B1, int64_t ld1, int p,
                                const void* B2, int64_t ld2, int q, void* out, int64_t ldo,
                                int dtype, void* stream) {
  if (!t) return fail(BKS_EINVAL, "null tensor");
  BKS_TRY(require_general(t));
  if (mode < 1 || mode > 3) return fail(BKS_EINVAL, "mode must be 1, 2 or 3");
  const int64_t rows1 = mode == 1 ? t->m : t->l;
  const int64_t rows2 = mode == 3 ? t->m : t->n;
  const int64_t rows_out = mode == 1 ? t->l : (mode == 2 ? t->m : t->n);
  BKS_TRY(check_common(t, B1, ld1, p, dtype, rows1));
  BKS_TRY(check_common(t, B2, ld2, q, dtype, rows2));
  if (!out || ldo < rows_out) return fail(BKS_EINVAL, "bad output");
  if (p > 8 || q > 8) return fail(BKS_EUNSUPPORTED, "widths p, q must be <= 8");
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == BKS_F64)
    return gen_contract_typed<double, double, double>(t, mode, (const double*)B1, ld1, p,
                                                      (const double*)B2, ld2, q, (double*)out,
                                                      ldo, s);
  return gen_contract_typed<float, float, float>(t, mode, (const float*)B1, ld1, p,
                                                 (const float*)B2, ld2, q, (float*)out, ldo, s);
}

extern "C" int bks_gen_core(const bks_tensor* t, const double* X, int64_t ldx, int k1,
                            const double* Y, int64_t ldy, int k2, const double* Z, int64_t ldz,
                            int k3, double* C, void* stream) {
  if (!t) return fail(BKS_EINVAL, "null tensor");
  BKS_TRY(require_general(t));
  BKS_TRY(check_common(t, X, ldx, k1, BKS_F64, t->l));
  BKS_TRY(check_common(t, Y, ldy, k2, BKS_F64, t->m));
  BKS_TRY(check_common(t, Z, ldz, k3, BKS_F64, t->n));
  if (!C) return fail(BKS_EINVAL, "null C");
  if (k1 > 128 || k2 > 128 || k3 > 128) return fail(BKS_EUNSUPPORTED, "core ranks must be <= 128");
  return gen_core_fp64(t, X, ldx, k1, Y, ldy, k2, Z, ldz, k3, C, (cudaStream_t)stream);
}
