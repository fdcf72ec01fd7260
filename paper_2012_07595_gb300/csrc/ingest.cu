// Tensor ingest (Definition 2.1): validate, mirror, stable sort by (i,j,k),
// sum duplicates left to right in the value dtype, build the sorted copies
// (rows i for the mode-1 contraction, rows k for mode 3 and the cores, and
// for a general l x m x n tensor rows j for mode 2) with their work-tile
// plans.  Runs once per tensor.
#include <algorithm>
#include <cstring>
#include <atomic>
#include <mutex>

#include "common.cuh"

namespace bks {

static thread_local std::string g_err;
static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void set_error(const std::string& msg) { g_err = msg; }
int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

namespace {

__global__ void k_validate(const int32_t* i, const int32_t* j, const int32_t* k, int64_t nnz,
                           int64_t l, int64_t m, int64_t n, int* bad) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (i[e] < 0 || i[e] >= l || j[e] < 0 || j[e] >= m || k[e] < 0 || k[e] >= n) atomicOr(bad, 1);
  }
}

__global__ void k_offdiag_flags(const int32_t* i, const int32_t* j, int64_t nnz, int32_t* f) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    f[e] = i[e] != j[e] ? 1 : 0;
}

// Expanded list: entries 0..nnz-1 are the input, nnz+t is the mirror of the
// t-th off-diagonal input entry.  Key = (i << (bj+bk)) | (j << bk) | k.
__global__ void k_build_keys(const int32_t* i, const int32_t* j, const int32_t* k, int64_t nnz,
                             const int32_t* offpos, int mirror, int bj, int bk, uint64_t* keys,
                             uint32_t* pay, uint32_t* mirror_src) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    uint64_t a = (uint64_t)i[e], b = (uint64_t)j[e], c = (uint64_t)k[e];
    keys[e] = (a << (bj + bk)) | (b << bk) | c;
    pay[e] = (uint32_t)e;
    if (mirror && a != b) {
      int64_t slot = nnz + offpos[e];
      keys[slot] = (b << (bj + bk)) | (a << bk) | c;
      pay[slot] = (uint32_t)slot;
      mirror_src[offpos[e]] = (uint32_t)e;
    }
  }
}

__global__ void k_head_flags(const uint64_t* keys, int64_t N, int32_t* f) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x)
    f[t] = (t == 0 || keys[t] != keys[t - 1]) ? 1 : 0;
}

__global__ void k_seg_starts(const int32_t* f, const int32_t* pos, int64_t N, int32_t* starts) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x)
    if (f[t]) starts[pos[t]] = (int32_t)t;
}

// One thread per run of equal keys: sum the values left to right in V.
// Long runs (the heaviest duplicated keys of a power-law input) load eight
// values ahead of their additions; the order of the additions is the same.
template <typename V>
__device__ __forceinline__ V run_value(const uint32_t* pay, int64_t t, const V* vin,
                                       const uint32_t* mirror_src, int64_t nnz_in) {
  const uint32_t p = pay[t];
  return (p < (uint64_t)nnz_in) ? vin[p] : vin[mirror_src[p - nnz_in]];
}
template <typename V>
__global__ void k_sum_runs(const uint64_t* keys, const uint32_t* pay, const int32_t* starts,
                           int64_t nseg, int64_t N, const V* vin, const uint32_t* mirror_src,
                           int64_t nnz_in, int bj, int bk, int32_t* row, int32_t* kk,
                           int32_t* jj, V* vout) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < nseg;
       u += (int64_t)gridDim.x * blockDim.x) {
    int64_t s = starts[u];
    int64_t e = (u + 1 < nseg) ? starts[u + 1] : N;
    V acc = run_value(pay, s, vin, mirror_src, nnz_in);  // the first value as it is
    int64_t t = s + 1;
    for (; t + 8 <= e; t += 8) {
      V x[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) x[q] = run_value(pay, t + q, vin, mirror_src, nnz_in);
#pragma unroll
      for (int q = 0; q < 8; ++q) acc = add_rn(acc, x[q]);
    }
    for (; t < e; ++t) acc = add_rn(acc, run_value(pay, t, vin, mirror_src, nnz_in));
    uint64_t key = keys[s];
    row[u] = (int32_t)(key >> (bj + bk));
    jj[u] = (int32_t)((key >> bk) & ((1ull << bj) - 1ull));
    kk[u] = (int32_t)(key & ((1ull << bk) - 1ull));
    vout[u] = acc;
  }
}

// ptr[r] = first position whose row is >= r (rows sorted ascending)
__global__ void k_row_ptr(const int32_t* row, int64_t nnz, int64_t rows, int32_t* ptr) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t <= nnz;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = (t == 0) ? 0 : (int64_t)row[t - 1] + 1;
    int64_t hi = (t == nnz) ? rows : (int64_t)row[t];
    for (int64_t r = lo; r <= hi && r <= rows; ++r) ptr[r] = (int32_t)t;
  }
}

template <typename V>
__global__ void k_check_symmetric(const int32_t* ptr, const int32_t* kk, const int32_t* jj,
                                  const V* v, int64_t m, int* bad) {
  // entry (i, j, k) at row i; find (j, i, k) in row j by binary search on (j, k)
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int32_t e = ptr[i]; e < ptr[i + 1]; ++e) {
      int32_t j = jj[e], k = kk[e];
      int32_t lo = ptr[j], hi = ptr[j + 1];
      while (lo < hi) {
        int32_t mid = (lo + hi) >> 1;
        bool less = jj[mid] < (int32_t)i || (jj[mid] == (int32_t)i && kk[mid] < k);
        if (less) lo = mid + 1; else hi = mid;
      }
      bool ok = lo < ptr[j + 1] && kk[lo] == k && jj[lo] == (int32_t)i;
      if (ok) {
        V a = v[e], b = v[lo];
        ok = same_bits(a, b);
      }
      if (!ok) atomicOr(bad, 1);
    }
  }
}

template <typename A, typename B>
__global__ void k_convert(const A* in, B* out, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    out[t] = (B)in[t];
}

// ||A||^2 in FP64: fixed partition over 1024 blocks, then one block in order.
template <typename V>
__global__ void k_sumsq_partial(const V* v, int64_t n, double* part) {
  __shared__ double sh[256];
  double s = 0.0;
  int64_t per = (n + gridDim.x - 1) / gridDim.x;
  int64_t lo = per * blockIdx.x, hi = min(n, lo + per);
  for (int64_t t = lo + threadIdx.x; t < hi; t += blockDim.x) {
    double x = (double)v[t];
    s = fma(x, x, s);
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}
__global__ void k_sum_partials(const double* part, int np, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int t = 0; t < np; ++t) s += part[t];
    *out = s;
  }
}

// mode-3 copy: key (k << (bi+bj)) | (i << bj) | j
__global__ void k_keys_mode3(const int32_t* row, const int32_t* kk, const int32_t* jj,
                             int64_t nnz, int bi, int bj, uint64_t* keys, uint32_t* pay) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz;
       t += (int64_t)gridDim.x * blockDim.x) {
    keys[t] = ((uint64_t)kk[t] << (bi + bj)) | ((uint64_t)row[t] << bj) | (uint64_t)jj[t];
    pay[t] = (uint32_t)t;
  }
}
template <typename V>
__global__ void k_gather_mode3(const uint64_t* keys, const uint32_t* pay, int64_t nnz, int bi,
                               int bj, const V* vsrc, int32_t* krow, int32_t* ii, int32_t* jj,
                               V* v) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz;
       t += (int64_t)gridDim.x * blockDim.x) {
    uint64_t key = keys[t];
    krow[t] = (int32_t)(key >> (bi + bj));
    ii[t] = (int32_t)((key >> bj) & ((1ull << bi) - 1ull));
    jj[t] = (int32_t)(key & ((1ull << bj) - 1ull));
    v[t] = vsrc[pay[t]];
  }
}

// mode-2 copy of a general tensor: key (j << (bi+bk)) | (i << bk) | k
__global__ void k_keys_mode2(const int32_t* row, const int32_t* kk, const int32_t* jj,
                             int64_t nnz, int bi, int bk, uint64_t* keys, uint32_t* pay) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz;
       t += (int64_t)gridDim.x * blockDim.x) {
    keys[t] = ((uint64_t)jj[t] << (bi + bk)) | ((uint64_t)row[t] << bk) | (uint64_t)kk[t];
    pay[t] = (uint32_t)t;
  }
}
template <typename V>
__global__ void k_gather_mode2(const uint64_t* keys, const uint32_t* pay, int64_t nnz, int bi,
                               int bk, const V* vsrc, int32_t* jrow, int32_t* ii, int32_t* kk,
                               V* v) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz;
       t += (int64_t)gridDim.x * blockDim.x) {
    uint64_t key = keys[t];
    jrow[t] = (int32_t)(key >> (bi + bk));
    ii[t] = (int32_t)((key >> bk) & ((1ull << bi) - 1ull));
    kk[t] = (int32_t)(key & ((1ull << bk) - 1ull));
    v[t] = vsrc[pay[t]];
  }
}

// ---- tile plan ------------------------------------------------------------
__global__ void k_vcount(const int32_t* ptr, int64_t rows, int split, int32_t* nvr,
                         int32_t* nslot, int32_t* issplit, int32_t* isempty) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x) {
    int32_t len = ptr[r + 1] - ptr[r];
    int32_t c = (len + split - 1) / split;
    nvr[r] = c;
    nslot[r] = c > 1 ? c : 0;
    issplit[r] = c > 1 ? 1 : 0;
    isempty[r] = c == 0 ? 1 : 0;
  }
}
__global__ void k_empty_list(const int32_t* isempty, const int32_t* pos, int64_t rows,
                             int32_t* out) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x)
    if (isempty[r]) out[pos[r]] = (int32_t)r;
}
__global__ void k_vfill(const int32_t* ptr, int64_t rows, int split, const int32_t* vbase,
                        const int32_t* nvr, const int32_t* slotbase, const int32_t* splitpos,
                        int32_t* vptr, int32_t* vrow, int32_t* vslot, int32_t* split_row,
                        int32_t* split_first) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x) {
    int32_t c = nvr[r];
    for (int32_t t = 0; t < c; ++t) {
      int32_t v = vbase[r] + t;
      vptr[v] = ptr[r] + t * split;
      vrow[v] = (int32_t)r;
      vslot[v] = c > 1 ? slotbase[r] + t : -1;
    }
    if (c > 1) {
      split_row[splitpos[r]] = (int32_t)r;
      split_first[splitpos[r]] = slotbase[r];
    }
  }
}

// Work classes of the virtual rows: length > tile -> one warp each
// (isvec), else one lane each; the short ones get the sort key tile - len so
// that a stable sort orders them by decreasing length.
__global__ void k_vclass(const int32_t* vptr, int32_t nv, int tile, int32_t* isvec,
                         int32_t* isshort) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t len = vptr[v + 1] - vptr[v];
    isvec[v] = len > tile ? 1 : 0;
    isshort[v] = len > tile ? 0 : 1;
  }
}
__global__ void k_vsplit_lists(const int32_t* vptr, int32_t nv, int tile, const int32_t* isvec,
                               const int32_t* vecpos, const int32_t* shortpos, int32_t* vorder,
                               uint64_t* skeys, uint32_t* svals) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
       v += (int64_t)gridDim.x * blockDim.x) {
    if (isvec[v]) {
      vorder[vecpos[v]] = (int32_t)v;
    } else {
      const int32_t len = vptr[v + 1] - vptr[v];
      skeys[shortpos[v]] = (uint64_t)(tile - len);
      svals[shortpos[v]] = (uint32_t)v;
    }
  }
}
__global__ void k_copy_u32(const uint32_t* in, int64_t n, int32_t* out) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n;
       x += (int64_t)gridDim.x * blockDim.x)
    out[x] = (int32_t)in[x];
}

// The kernel's per-item record in processing order: first entry, end,
// output row, partial slot (one 16-byte load instead of two dependent ones)
// 32 x the length of the first (longest) short row of each group of 32
__global__ void k_sell_len(const int4* items, int32_t nshort, int32_t ngroups, int64_t* glen) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ngroups;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int4 it = items[g * 32];
    glen[g] = 32 * (int64_t)(it.y - it.x);
  }
}
// Copy the short rows' entries into the lane-interleaved layout and point
// their work items at it (each thread rewrites only its own item).
__global__ void k_sell_fill(int4* items, int32_t nshort, const int64_t* gbase,
                            const int32_t* c0, const int32_t* c1, const float* vf,
                            const double* vd, int32_t* sc0, int32_t* sc1, float* svf,
                            double* svd) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < nshort;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int4 it = items[x];
    const int64_t base = gbase[x / 32] + (x % 32);
    const int len = it.y - it.x;
    for (int t = 0; t < len; ++t) {
      const int64_t d = base + 32 * (int64_t)t;
      sc0[d] = c0[it.x + t];
      sc1[d] = c1[it.x + t];
      svf[d] = vf[it.x + t];
      svd[d] = vd[it.x + t];
    }
    items[x] = make_int4((int32_t)base, (int32_t)(base + 32 * (int64_t)len), it.z, it.w);
  }
}

__global__ void k_vitems(const int32_t* vorder, int32_t nv, const int32_t* vptr,
                         const int32_t* vrow, const int32_t* vslot, int4* items) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < nv;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = vorder[x];
    items[x] = make_int4(vptr[v], vptr[v + 1], vrow[v], vslot[v]);
  }
}

__global__ void k_expand_rows(const int32_t* ptr, int64_t rows, int32_t* out) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x)
    for (int32_t e = ptr[r]; e < ptr[r + 1]; ++e) out[e] = (int32_t)r;
}

inline int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)num_sms() * 32));
}

int bits_for(int64_t x) {  // bits needed for values 0..x-1 (at least 1)
  int b = 1;
  while (b < 63 && (1ll << b) < x) ++b;
  return b;
}

int read_i32(const int32_t* dptr, int32_t* host, cudaStream_t s) {
  BKS_CUDA_TRY(cudaMemcpyAsync(host, dptr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  BKS_CUDA_TRY(cudaStreamSynchronize(s));
  return BKS_OK;
}

template <typename V>
int ingest_typed(bks_tensor* T, const int32_t* di, const int32_t* dj, const int32_t* dk,
                 const V* dv, int64_t nnz, int flags, cudaStream_t s) {
  const int64_t l = T->l, m = T->m, n = T->n;
  const bool mirror = !T->general && (flags & BKS_MIRROR);
  const int bi = bits_for(l), bj = bits_for(m), bk = bits_for(n);
  if (bi + bj + bk > 64) return fail(BKS_EUNSUPPORTED, "dimensions too large for a 64-bit sort key");
  // mirror positions
  DevBuf offf, offpos, mirror_src;
  int32_t noff = 0;
  BKS_TRY(offpos.alloc(sizeof(int32_t) * std::max<int64_t>(nnz, 1), s));
  if (mirror && nnz > 0) {
    BKS_TRY(offf.alloc(sizeof(int32_t) * nnz, s));
    DevBuf tot;
    BKS_TRY(tot.alloc(sizeof(int32_t), s));
    k_offdiag_flags<<<grid_for(nnz), 256, 0, s>>>(di, dj, nnz, offf.as<int32_t>()); ::bks::note_launch();
    BKS_TRY(exclusive_scan_i32(offf.as<int32_t>(), offpos.as<int32_t>(), nnz, tot.as<int32_t>(), s));
    BKS_TRY(read_i32(tot.as<int32_t>(), &noff, s));
  }
  const int64_t N = nnz + noff;
  // int32 entry positions, with room for the kernels' look-ahead past a row's end
  if (N > (1ll << 31) - 1024)
    return fail(BKS_EUNSUPPORTED, "more than 2^31 - 1024 expanded entries");
  DevBuf keys, pay;
  BKS_TRY(keys.alloc(sizeof(uint64_t) * std::max<int64_t>(N, 1), s));
  BKS_TRY(pay.alloc(sizeof(uint32_t) * std::max<int64_t>(N, 1), s));
  BKS_TRY(mirror_src.alloc(sizeof(uint32_t) * std::max<int32_t>(noff, 1), s));
  if (nnz > 0)
    k_build_keys<<<grid_for(nnz), 256, 0, s>>>(di, dj, dk, nnz, offpos.as<int32_t>(), mirror ? 1 : 0,
                                               bj, bk, keys.as<uint64_t>(), pay.as<uint32_t>(),
                                               mirror_src.as<uint32_t>()); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  BKS_TRY(radix_sort_pairs(keys.as<uint64_t>(), pay.as<uint32_t>(), N, bi + bk + bj, s));
  // runs of equal keys
  int32_t nseg = 0;
  DevBuf head, hpos, starts, row;
  if (N > 0) {
    BKS_TRY(head.alloc(sizeof(int32_t) * N, s));
    BKS_TRY(hpos.alloc(sizeof(int32_t) * N, s));
    DevBuf tot;
    BKS_TRY(tot.alloc(sizeof(int32_t), s));
    k_head_flags<<<grid_for(N), 256, 0, s>>>(keys.as<uint64_t>(), N, head.as<int32_t>()); ::bks::note_launch();
    BKS_TRY(exclusive_scan_i32(head.as<int32_t>(), hpos.as<int32_t>(), N, tot.as<int32_t>(), s));
    BKS_TRY(read_i32(tot.as<int32_t>(), &nseg, s));
    BKS_TRY(starts.alloc(sizeof(int32_t) * nseg, s));
    k_seg_starts<<<grid_for(N), 256, 0, s>>>(head.as<int32_t>(), hpos.as<int32_t>(), N,
                                              starts.as<int32_t>()); ::bks::note_launch();
    BKS_CUDA_TRY(cudaGetLastError());
  }
  T->nnz = nseg;
  Part& P = T->m1;
  P.rows = l;
  const int64_t S = std::max<int64_t>(nseg, 1);
  BKS_TRY(row.alloc(sizeof(int32_t) * S, s));
  BKS_TRY(P.c0.alloc(sizeof(int32_t) * S, s));
  BKS_TRY(P.c1.alloc(sizeof(int32_t) * S, s));
  BKS_TRY(P.v.alloc(sizeof(V) * S, s));
  if (nseg > 0)
    k_sum_runs<V><<<grid_for(nseg), 256, 0, s>>>(keys.as<uint64_t>(), pay.as<uint32_t>(),
                                                 starts.as<int32_t>(), nseg, N, dv,
                                                 mirror_src.as<uint32_t>(), nnz, bj, bk,
                                                 row.as<int32_t>(), P.c0.as<int32_t>(),
                                                 P.c1.as<int32_t>(), P.v.as<V>()); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  head.release(); hpos.release(); starts.release(); offf.release(); offpos.release();
  BKS_TRY(P.ptr.alloc(sizeof(int32_t) * (l + 1), s));
  k_row_ptr<<<grid_for(nseg + 1), 256, 0, s>>>(row.as<int32_t>(), nseg, l, P.ptr.as<int32_t>()); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  if (!T->general && !mirror && (flags & BKS_VALIDATE_SYMMETRIC)) {
    DevBuf bad;
    BKS_TRY(bad.alloc(sizeof(int), s));
    BKS_CUDA_TRY(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
    k_check_symmetric<V><<<grid_for(m), 256, 0, s>>>(P.ptr.as<int32_t>(), P.c0.as<int32_t>(),
                                                     P.c1.as<int32_t>(), P.v.as<V>(), m,
                                                     bad.as<int>()); ::bks::note_launch();
    int hb = 0;
    BKS_CUDA_TRY(cudaMemcpyAsync(&hb, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    BKS_CUDA_TRY(cudaStreamSynchronize(s));
    if (hb) return fail(BKS_EASYM, "input is not (1,2)-symmetric");
  }
  // value copies in the other precision
  if (sizeof(V) == 8) {
    BKS_TRY(P.v32.alloc(sizeof(float) * S, s));
    k_convert<double, float><<<grid_for(nseg), 256, 0, s>>>((const double*)P.v.p, P.v32.as<float>(), nseg); ::bks::note_launch();
  } else {
    BKS_TRY(P.v64.alloc(sizeof(double) * S, s));
    k_convert<float, double><<<grid_for(nseg), 256, 0, s>>>((const float*)P.v.p, P.v64.as<double>(), nseg); ::bks::note_launch();
  }
  BKS_CUDA_TRY(cudaGetLastError());
  // ||A||^2
  {
    DevBuf part, out;
    BKS_TRY(part.alloc(sizeof(double) * 1024, s));
    BKS_TRY(out.alloc(sizeof(double), s));
    k_sumsq_partial<V><<<1024, 256, 0, s>>>(P.v.as<V>(), nseg, part.as<double>()); ::bks::note_launch();
    k_sum_partials<<<1, 32, 0, s>>>(part.as<double>(), 1024, out.as<double>()); ::bks::note_launch();
    BKS_CUDA_TRY(cudaMemcpyAsync(&T->fro2, out.p, sizeof(double), cudaMemcpyDeviceToHost, s));
    BKS_CUDA_TRY(cudaStreamSynchronize(s));
  }
  // mode-3 copy sorted by (k, i, j)
  Part& Q = T->m3;
  Q.rows = n;
  BKS_TRY(Q.c0.alloc(sizeof(int32_t) * S, s));
  BKS_TRY(Q.c1.alloc(sizeof(int32_t) * S, s));
  BKS_TRY(Q.v.alloc(sizeof(V) * S, s));
  {
    DevBuf krow;
    BKS_TRY(krow.alloc(sizeof(int32_t) * S, s));
    if (nseg > 0) {
      k_keys_mode3<<<grid_for(nseg), 256, 0, s>>>(row.as<int32_t>(), P.c0.as<int32_t>(),
                                                  P.c1.as<int32_t>(), nseg, bi, bj,
                                                  keys.as<uint64_t>(), pay.as<uint32_t>()); ::bks::note_launch();
      BKS_CUDA_TRY(cudaGetLastError());
      BKS_TRY(radix_sort_pairs(keys.as<uint64_t>(), pay.as<uint32_t>(), nseg, bk + bi + bj, s));
      k_gather_mode3<V><<<grid_for(nseg), 256, 0, s>>>(keys.as<uint64_t>(), pay.as<uint32_t>(),
                                                       nseg, bi, bj, P.v.as<V>(),
                                                       krow.as<int32_t>(), Q.c0.as<int32_t>(),
                                                       Q.c1.as<int32_t>(), Q.v.as<V>()); ::bks::note_launch();
      BKS_CUDA_TRY(cudaGetLastError());
    }
    BKS_TRY(Q.ptr.alloc(sizeof(int32_t) * (n + 1), s));
    k_row_ptr<<<grid_for(nseg + 1), 256, 0, s>>>(krow.as<int32_t>(), nseg, n, Q.ptr.as<int32_t>()); ::bks::note_launch();
    BKS_CUDA_TRY(cudaGetLastError());
  }
  if (sizeof(V) == 8) {
    BKS_TRY(Q.v32.alloc(sizeof(float) * S, s));
    k_convert<double, float><<<grid_for(nseg), 256, 0, s>>>((const double*)Q.v.p, Q.v32.as<float>(), nseg); ::bks::note_launch();
  } else {
    BKS_TRY(Q.v64.alloc(sizeof(double) * S, s));
    k_convert<float, double><<<grid_for(nseg), 256, 0, s>>>((const float*)Q.v.p, Q.v64.as<double>(), nseg); ::bks::note_launch();
  }
  BKS_CUDA_TRY(cudaGetLastError());
  if (T->general) {
    // mode-2 copy sorted by (j, i, k)
    Part& R = T->m2;
    R.rows = m;
    BKS_TRY(R.c0.alloc(sizeof(int32_t) * S, s));
    BKS_TRY(R.c1.alloc(sizeof(int32_t) * S, s));
    BKS_TRY(R.v.alloc(sizeof(V) * S, s));
    DevBuf jrow;
    BKS_TRY(jrow.alloc(sizeof(int32_t) * S, s));
    if (nseg > 0) {
      k_keys_mode2<<<grid_for(nseg), 256, 0, s>>>(row.as<int32_t>(), P.c0.as<int32_t>(),
                                                  P.c1.as<int32_t>(), nseg, bi, bk,
                                                  keys.as<uint64_t>(), pay.as<uint32_t>()); ::bks::note_launch();
      BKS_CUDA_TRY(cudaGetLastError());
      BKS_TRY(radix_sort_pairs(keys.as<uint64_t>(), pay.as<uint32_t>(), nseg, bj + bi + bk, s));
      k_gather_mode2<V><<<grid_for(nseg), 256, 0, s>>>(keys.as<uint64_t>(), pay.as<uint32_t>(),
                                                       nseg, bi, bk, P.v.as<V>(),
                                                       jrow.as<int32_t>(), R.c1.as<int32_t>(),
                                                       R.c0.as<int32_t>(), R.v.as<V>()); ::bks::note_launch();
      BKS_CUDA_TRY(cudaGetLastError());
    }
    BKS_TRY(R.ptr.alloc(sizeof(int32_t) * (m + 1), s));
    k_row_ptr<<<grid_for(nseg + 1), 256, 0, s>>>(jrow.as<int32_t>(), nseg, m, R.ptr.as<int32_t>()); ::bks::note_launch();
    BKS_CUDA_TRY(cudaGetLastError());
    if (sizeof(V) == 8) {
      BKS_TRY(R.v32.alloc(sizeof(float) * S, s));
      k_convert<double, float><<<grid_for(nseg), 256, 0, s>>>((const double*)R.v.p, R.v32.as<float>(), nseg); ::bks::note_launch();
    } else {
      BKS_TRY(R.v64.alloc(sizeof(double) * S, s));
      k_convert<float, double><<<grid_for(nseg), 256, 0, s>>>((const float*)R.v.p, R.v64.as<double>(), nseg); ::bks::note_launch();
    }
    BKS_CUDA_TRY(cudaGetLastError());
  }
  {
    int tile = kTile, split = kSplit;
    default_plan(nseg, &tile, &split);
    T->m1.tile = T->m2.tile = T->m3.tile = tile;
    T->m1.split = T->m2.split = T->m3.split = split;
  }
  BKS_TRY(build_tile_plan(T->m1, nseg, s));
  if (T->general) BKS_TRY(build_tile_plan(T->m2, nseg, s));
  BKS_TRY(build_tile_plan(T->m3, nseg, s));
  Q.host_ptr.resize(n + 1);
  BKS_CUDA_TRY(cudaMemcpyAsync(Q.host_ptr.data(), Q.ptr.p, sizeof(int32_t) * (n + 1),
                               cudaMemcpyDeviceToHost, s));
  BKS_CUDA_TRY(cudaStreamSynchronize(s));
  BKS_TRY(build_core_plan(Q, n, nseg, T->cp, s));
  P.persist();
  Q.persist();
  if (T->general) T->m2.persist();
  T->cp.persist();
  return BKS_OK;
}

}  // namespace

namespace {

// The lane-interleaved copy of the short rows (see Part).
int build_sell(Part& P, cudaStream_t s) {
  const int32_t ng = (P.nshortv + 31) / 32;
  DevBuf glen, gbase, tot;
  BKS_TRY(glen.alloc(sizeof(int64_t) * ng, s));
  BKS_TRY(gbase.alloc(sizeof(int64_t) * ng, s));
  BKS_TRY(tot.alloc(sizeof(int64_t), s));
  int4* items = P.vitems.as<int4>() + P.nvec;
  k_sell_len<<<grid_for(ng), 256, 0, s>>>(items, P.nshortv, ng, glen.as<int64_t>()); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  BKS_TRY(exclusive_scan_i64(glen.as<int64_t>(), gbase.as<int64_t>(), ng, tot.as<int64_t>(), s));
  int64_t nsell = 0;
  BKS_CUDA_TRY(cudaMemcpyAsync(&nsell, tot.p, sizeof(nsell), cudaMemcpyDeviceToHost, s));
  BKS_CUDA_TRY(cudaStreamSynchronize(s));
  if (nsell > ((int64_t)1 << 31) - 1024)
    return fail(BKS_EUNSUPPORTED, "interleaved short-row copy exceeds int32 positions");
  P.nsell = nsell;
  BKS_TRY(P.sc0.alloc(sizeof(int32_t) * std::max<int64_t>(nsell, 1), s));
  BKS_TRY(P.sc1.alloc(sizeof(int32_t) * std::max<int64_t>(nsell, 1), s));
  BKS_TRY(P.sv32.alloc(sizeof(float) * std::max<int64_t>(nsell, 1), s));
  BKS_TRY(P.sv64.alloc(sizeof(double) * std::max<int64_t>(nsell, 1), s));
  // values in both arithmetic types: the input dtype's array and its converted copy
  const float* vf = P.v32.p ? P.v32.as<float>() : P.v.as<float>();
  const double* vd = P.v64.p ? P.v64.as<double>() : P.v.as<double>();
  k_sell_fill<<<grid_for(P.nshortv), 256, 0, s>>>(items, P.nshortv, gbase.as<int64_t>(),
                                                  P.c0.as<int32_t>(), P.c1.as<int32_t>(), vf, vd,
                                                  P.sc0.as<int32_t>(), P.sc1.as<int32_t>(),
                                                  P.sv32.as<float>(), P.sv64.as<double>()); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  return BKS_OK;
}

}  // namespace

int build_tile_plan(Part& P, int64_t nnz, cudaStream_t s) {
  const int64_t R = P.rows;
  DevBuf nvr, nslot, issplit, vbase, slotbase, splitpos, tot, isempty, emptypos;
  BKS_TRY(isempty.alloc(sizeof(int32_t) * R, s));
  BKS_TRY(emptypos.alloc(sizeof(int32_t) * R, s));
  BKS_TRY(nvr.alloc(sizeof(int32_t) * R, s));
  BKS_TRY(nslot.alloc(sizeof(int32_t) * R, s));
  BKS_TRY(issplit.alloc(sizeof(int32_t) * R, s));
  BKS_TRY(vbase.alloc(sizeof(int32_t) * R, s));
  BKS_TRY(slotbase.alloc(sizeof(int32_t) * R, s));
  BKS_TRY(splitpos.alloc(sizeof(int32_t) * R, s));
  BKS_TRY(tot.alloc(sizeof(int32_t) * 4, s));
  k_vcount<<<grid_for(R), 256, 0, s>>>(P.ptr.as<int32_t>(), R, P.split, nvr.as<int32_t>(),
                                       nslot.as<int32_t>(), issplit.as<int32_t>(),
                                       isempty.as<int32_t>()); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  BKS_TRY(exclusive_scan_i32(nvr.as<int32_t>(), vbase.as<int32_t>(), R, tot.as<int32_t>(), s));
  BKS_TRY(exclusive_scan_i32(nslot.as<int32_t>(), slotbase.as<int32_t>(), R, tot.as<int32_t>() + 1, s));
  BKS_TRY(exclusive_scan_i32(issplit.as<int32_t>(), splitpos.as<int32_t>(), R, tot.as<int32_t>() + 2, s));
  BKS_TRY(exclusive_scan_i32(isempty.as<int32_t>(), emptypos.as<int32_t>(), R, tot.as<int32_t>() + 3, s));
  int32_t h[4];
  BKS_CUDA_TRY(cudaMemcpyAsync(h, tot.p, sizeof(h), cudaMemcpyDeviceToHost, s));
  BKS_CUDA_TRY(cudaStreamSynchronize(s));
  P.nv = h[0];
  P.nslots = h[1];
  P.nsplit = h[2];
  P.nempty = h[3];
  BKS_TRY(P.empty_rows.alloc(sizeof(int32_t) * std::max(P.nempty, 1), s));
  k_empty_list<<<grid_for(R), 256, 0, s>>>(isempty.as<int32_t>(), emptypos.as<int32_t>(), R,
                                           P.empty_rows.as<int32_t>()); ::bks::note_launch();
  BKS_TRY(P.vptr.alloc(sizeof(int32_t) * (P.nv + 1), s));
  BKS_TRY(P.vrow.alloc(sizeof(int32_t) * std::max(P.nv, 1), s));
  BKS_TRY(P.vslot.alloc(sizeof(int32_t) * std::max(P.nv, 1), s));
  BKS_TRY(P.split_row.alloc(sizeof(int32_t) * std::max(P.nsplit, 1), s));
  BKS_TRY(P.split_first.alloc(sizeof(int32_t) * (P.nsplit + 1), s));
  k_vfill<<<grid_for(R), 256, 0, s>>>(P.ptr.as<int32_t>(), R, P.split, vbase.as<int32_t>(),
                                      nvr.as<int32_t>(), slotbase.as<int32_t>(),
                                      splitpos.as<int32_t>(), P.vptr.as<int32_t>(),
                                      P.vrow.as<int32_t>(), P.vslot.as<int32_t>(),
                                      P.split_row.as<int32_t>(), P.split_first.as<int32_t>()); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  int32_t nn = (int32_t)nnz;
  BKS_CUDA_TRY(cudaMemcpyAsync(P.vptr.as<int32_t>() + P.nv, &nn, sizeof(int32_t),
                               cudaMemcpyHostToDevice, s));
  int32_t ns = P.nslots;
  BKS_CUDA_TRY(cudaMemcpyAsync(P.split_first.as<int32_t>() + P.nsplit, &ns, sizeof(int32_t),
                               cudaMemcpyHostToDevice, s));
  // classes and the processing order of the virtual rows
  if (P.nv > 0) {
    DevBuf isvec, isshort, vecpos, shortpos, skeys, svals, tot2;
    BKS_TRY(isvec.alloc(sizeof(int32_t) * P.nv, s));
    BKS_TRY(isshort.alloc(sizeof(int32_t) * P.nv, s));
    BKS_TRY(vecpos.alloc(sizeof(int32_t) * P.nv, s));
    BKS_TRY(shortpos.alloc(sizeof(int32_t) * P.nv, s));
    BKS_TRY(tot2.alloc(sizeof(int32_t) * 2, s));
    k_vclass<<<grid_for(P.nv), 256, 0, s>>>(P.vptr.as<int32_t>(), P.nv, P.tile,
                                            isvec.as<int32_t>(), isshort.as<int32_t>()); ::bks::note_launch();
    BKS_CUDA_TRY(cudaGetLastError());
    BKS_TRY(exclusive_scan_i32(isvec.as<int32_t>(), vecpos.as<int32_t>(), P.nv, tot2.as<int32_t>(), s));
    BKS_TRY(exclusive_scan_i32(isshort.as<int32_t>(), shortpos.as<int32_t>(), P.nv,
                               tot2.as<int32_t>() + 1, s));
    int32_t h2[2];
    BKS_CUDA_TRY(cudaMemcpyAsync(h2, tot2.p, sizeof(h2), cudaMemcpyDeviceToHost, s));
    BKS_CUDA_TRY(cudaStreamSynchronize(s));
    P.nvec = h2[0];
    P.nshortv = h2[1];
    BKS_TRY(P.vorder.alloc(sizeof(int32_t) * P.nv, s));
    BKS_TRY(skeys.alloc(sizeof(uint64_t) * std::max(P.nshortv, 1), s));
    BKS_TRY(svals.alloc(sizeof(uint32_t) * std::max(P.nshortv, 1), s));
    k_vsplit_lists<<<grid_for(P.nv), 256, 0, s>>>(P.vptr.as<int32_t>(), P.nv, P.tile,
                                                  isvec.as<int32_t>(), vecpos.as<int32_t>(),
                                                  shortpos.as<int32_t>(), P.vorder.as<int32_t>(),
                                                  skeys.as<uint64_t>(), svals.as<uint32_t>()); ::bks::note_launch();
    BKS_CUDA_TRY(cudaGetLastError());
    if (P.nshortv > 0) {
      BKS_TRY(radix_sort_pairs(skeys.as<uint64_t>(), svals.as<uint32_t>(), P.nshortv,
                               bits_for(P.tile + 1), s));
      k_copy_u32<<<grid_for(P.nshortv), 256, 0, s>>>(svals.as<uint32_t>(), P.nshortv,
                                                      P.vorder.as<int32_t>() + P.nvec); ::bks::note_launch();
      BKS_CUDA_TRY(cudaGetLastError());
    }
    BKS_TRY(P.vitems.alloc(sizeof(int4) * P.nv, s));
    k_vitems<<<grid_for(P.nv), 256, 0, s>>>(P.vorder.as<int32_t>(), P.nv, P.vptr.as<int32_t>(),
                                            P.vrow.as<int32_t>(), P.vslot.as<int32_t>(),
                                            P.vitems.as<int4>()); ::bks::note_launch();
    BKS_CUDA_TRY(cudaGetLastError());
    if (P.nshortv > 0) BKS_TRY(build_sell(P, s));
  } else {
    P.nvec = P.nshortv = 0;
  }
  BKS_CUDA_TRY(cudaStreamSynchronize(s));  // host copies above read stack values
  P.persist();
  return BKS_OK;
}

}  // namespace bks

using namespace bks;

namespace bks {
namespace {
int create_impl(int64_t l, int64_t m, int64_t n, int64_t nnz, const int32_t* i, const int32_t* j,
                const int32_t* k, const void* v, int vdtype, int flags, bool general, void* stream,
                bks_tensor** out) {
  if (!out) return fail(BKS_EINVAL, "out is NULL");
  *out = nullptr;
  if (l < 1 || m < 1 || n < 1 || nnz < 0) return fail(BKS_EINVAL, "need dimensions >= 1, nnz >= 0");
  if (l >= (1ll << 31) || m >= (1ll << 31) || n >= (1ll << 31))
    return fail(BKS_EUNSUPPORTED, "dimensions must fit int32");
  if (nnz > 0 && (!i || !j || !k || !v)) return fail(BKS_EINVAL, "null index or value pointer");
  if (vdtype != BKS_F32 && vdtype != BKS_F64) return fail(BKS_EINVAL, "vdtype must be BKS_F32 or BKS_F64");
  if (general && (flags & (BKS_MIRROR | BKS_VALIDATE_SYMMETRIC)))
    return fail(BKS_EINVAL, "BKS_MIRROR and BKS_VALIDATE_SYMMETRIC apply to symmetric tensors only");
  if ((flags & BKS_MIRROR) && (flags & BKS_VALIDATE_SYMMETRIC))
    return fail(BKS_EINVAL, "BKS_VALIDATE_SYMMETRIC applies to input without BKS_MIRROR");
  if (nnz >= (1ll << 31)) return fail(BKS_EUNSUPPORTED, "nnz must fit int32");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t vs = vdtype == BKS_F64 ? 8 : 4;
  auto* T = new bks_tensor();
  T->l = l;
  T->m = m;
  T->n = n;
  T->vdtype = vdtype;
  T->general = general ? 1 : 0;
  int rc = BKS_OK;
  {
    DevBuf hi, hj, hk, hv;
    const int32_t *di = i, *dj = j, *dk = k;
    const void* dv = v;
    if (!(flags & BKS_INPUT_ON_DEVICE) && nnz > 0) {
      rc = hi.alloc(4 * nnz, s);
      if (rc == BKS_OK) rc = hj.alloc(4 * nnz, s);
      if (rc == BKS_OK) rc = hk.alloc(4 * nnz, s);
      if (rc == BKS_OK) rc = hv.alloc(vs * nnz, s);
      if (rc == BKS_OK) {
        cudaError_t e = cudaMemcpyAsync(hi.p, i, 4 * nnz, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hj.p, j, 4 * nnz, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hk.p, k, 4 * nnz, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hv.p, v, vs * nnz, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) rc = fail(BKS_ECUDA, std::string("copy input: ") + cudaGetErrorString(e));
      }
      di = hi.as<int32_t>(); dj = hj.as<int32_t>(); dk = hk.as<int32_t>(); dv = hv.p;
    }
    if (rc == BKS_OK && nnz > 0) {
      DevBuf bad;
      rc = bad.alloc(sizeof(int), s);
      if (rc == BKS_OK) {
        int hb = 0;
        cudaMemsetAsync(bad.p, 0, sizeof(int), s);
        k_validate<<<grid_for(nnz), 256, 0, s>>>(di, dj, dk, nnz, l, m, n, bad.as<int>()); ::bks::note_launch();
        cudaError_t e = cudaMemcpyAsync(&hb, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = fail(BKS_ECUDA, std::string("validate: ") + cudaGetErrorString(e));
        else if (hb) rc = fail(BKS_EINVAL, general ? "index out of range (i >= l, j >= m, k >= n or negative)"
                                                   : "index out of range (i, j >= m or k >= n or negative)");
      }
    }
    if (rc == BKS_OK) {
      if (vdtype == BKS_F64)
        rc = ingest_typed<double>(T, di, dj, dk, (const double*)dv, nnz, flags, s);
      else
        rc = ingest_typed<float>(T, di, dj, dk, (const float*)dv, nnz, flags, s);
    }
    cudaStreamSynchronize(s);
  }
  if (rc != BKS_OK) {
    delete T;
    return rc;
  }
  *out = T;
  return BKS_OK;
}
}  // namespace
}  // namespace bks

extern "C" int bks_tensor_create_coo(int64_t m, int64_t n, int64_t nnz, const int32_t* i,
                                     const int32_t* j, const int32_t* k, const void* v,
                                     int vdtype, int flags, void* stream, bks_tensor** out) {
  return create_impl(m, m, n, nnz, i, j, k, v, vdtype, flags, false, stream, out);
}

extern "C" int bks_gen_tensor_create_coo(int64_t l, int64_t m, int64_t n, int64_t nnz,
                                         const int32_t* i, const int32_t* j, const int32_t* k,
                                         const void* v, int vdtype, int flags, void* stream,
                                         bks_tensor** out) {
  return create_impl(l, m, n, nnz, i, j, k, v, vdtype, flags, true, stream, out);
}

extern "C" void bks_tensor_destroy(bks_tensor* t) {
  if (!t) return;
  cudaDeviceSynchronize();
  delete t;
}

extern "C" int bks_gen_tensor_dims(const bks_tensor* t, int64_t* l, int64_t* m, int64_t* n,
                                   int* general) {
  if (!t) return fail(BKS_EINVAL, "null tensor");
  if (l) *l = t->l;
  if (m) *m = t->m;
  if (n) *n = t->n;
  if (general) *general = t->general;
  return BKS_OK;
}

extern "C" int bks_tensor_info(const bks_tensor* t, int64_t* m, int64_t* n, int64_t* nnz,
                               double* fro2) {
  if (!t) return fail(BKS_EINVAL, "null tensor");
  if (m) *m = t->m;
  if (n) *n = t->n;
  if (nnz) *nnz = t->nnz;
  if (fro2) *fro2 = t->fro2;
  return BKS_OK;
}

extern "C" int bks_tensor_export_coo(const bks_tensor* t, int32_t* i, int32_t* j, int32_t* k,
                                     void* v, void* stream) {
  if (!t) return fail(BKS_EINVAL, "null tensor");
  if (t->nnz == 0) return BKS_OK;
  if (!i || !j || !k || !v) return fail(BKS_EINVAL, "null output pointer");
  cudaStream_t s = (cudaStream_t)stream;
  const Part& P = t->m1;
  k_expand_rows<<<grid_for(P.rows), 256, 0, s>>>(P.ptr.as<int32_t>(), P.rows, i); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  BKS_CUDA_TRY(cudaMemcpyAsync(j, P.c1.p, 4 * t->nnz, cudaMemcpyDeviceToDevice, s));
  BKS_CUDA_TRY(cudaMemcpyAsync(k, P.c0.p, 4 * t->nnz, cudaMemcpyDeviceToDevice, s));
  BKS_CUDA_TRY(cudaMemcpyAsync(v, P.v.p, (t->vdtype == BKS_F64 ? 8 : 4) * t->nnz,
                               cudaMemcpyDeviceToDevice, s));
  return BKS_OK;
}

extern "C" const char* bks_last_error_string(void) { return g_err.c_str(); }

extern "C" uint64_t bks_launch_count(void) { return g_launches.load(); }
