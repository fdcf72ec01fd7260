// Device-wide exclusive scans and a stable LSD radix sort of (key, payload)
// pairs.  Both are used once per tensor by the ingest step (the sort key is
// the packed (i, k, j) or (k, i, j) index; stability keeps equal keys in
// their input order, which fixes the order in which duplicates are summed).
#include "common.cuh"

namespace bks {

namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ T block_exclusive_scan(T x, T* warp_tot, T* block_total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    T w = lane < nw ? warp_tot[lane] : T(0);
    T winc = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, winc, o);
      if (lane >= o) winc += y;
    }
    if (lane < nw) warp_tot[lane] = winc - w;
    if (lane == nw - 1) *block_total = winc;
  }
  __syncthreads();
  T r = warp_tot[warp] + inc - x;
  __syncthreads();
  return r;
}

template <typename T>
__global__ void scan_block_sums(const T* in, int64_t n, T* sums) {
  __shared__ T wt[32];
  __shared__ T tot;
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  T s = 0;
#pragma unroll
  for (int t = 0; t < kScanItems; ++t)
    if (base + t < n) s += in[base + t];
  block_exclusive_scan<T>(s, wt, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <typename T>
__global__ void scan_block_apply(const T* in, T* out, int64_t n, const T* offs,
                                 T* total) {
  __shared__ T wt[32];
  __shared__ T tot;
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  T v[kScanItems];
  T s = 0;
#pragma unroll
  for (int t = 0; t < kScanItems; ++t) {
    v[t] = (base + t < n) ? in[base + t] : T(0);
    s += v[t];
  }
  T ex = block_exclusive_scan<T>(s, wt, &tot);
  T run = ex + (offs ? offs[blockIdx.x] : T(0));
#pragma unroll
  for (int t = 0; t < kScanItems; ++t) {
    if (base + t < n) out[base + t] = run;
    run += v[t];
  }
  if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1)
    *total = run;
}

template <typename T>
int exclusive_scan(const T* in, T* out, int64_t n, T* total, cudaStream_t s) {
  if (n <= 0) {
    if (total) BKS_CUDA_TRY(cudaMemsetAsync(total, 0, sizeof(T), s));
    return BKS_OK;
  }
  int64_t blocks = (n + kScanTile - 1) / kScanTile;
  if (blocks == 1) {
    scan_block_apply<T><<<1, kScanThreads, 0, s>>>(in, out, n, nullptr, total); ::bks::note_launch();
    BKS_CUDA_TRY(cudaGetLastError());
    return BKS_OK;
  }
  DevBuf sums;
  BKS_TRY(sums.alloc(sizeof(T) * blocks, s));
  scan_block_sums<T><<<(unsigned)blocks, kScanThreads, 0, s>>>(in, n, sums.as<T>()); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  BKS_TRY(exclusive_scan<T>(sums.as<T>(), sums.as<T>(), blocks, nullptr, s));
  scan_block_apply<T><<<(unsigned)blocks, kScanThreads, 0, s>>>(in, out, n, sums.as<T>(), total); ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  return BKS_OK;
}

// ---- radix sort --------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortTile = kSortThreads * kSortItems;

__global__ void radix_hist(const uint64_t* keys, int64_t n, int shift, int32_t* counts,
                           int ntiles) {
  __shared__ int32_t h[256];
  for (int d = threadIdx.x; d < 256; d += blockDim.x) h[d] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int t = threadIdx.x; t < kSortTile; t += blockDim.x) {
    int64_t idx = base + t;
    if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += blockDim.x)
    counts[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

// Stable scatter: within a tile, warp w owns items [w*32*kSortItems, ...),
// processed in rounds of 32 consecutive items; an item's rank among equal
// digits is (items of that digit in earlier warps) + (in earlier rounds of
// its warp) + (in lower lanes of its round).
__global__ void radix_scatter(const uint64_t* kin, const uint32_t* vin, uint64_t* kout,
                              uint32_t* vout, int64_t n, int shift,
                              const int32_t* offs, int ntiles) {
  __shared__ int32_t wh[kSortWarps][257];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int x = threadIdx.x; x < kSortWarps * 257; x += blockDim.x) (&wh[0][0])[x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)warp * 32 * kSortItems;
  const unsigned lt = (1u << lane) - 1u;
  uint64_t key[kSortItems];
  uint32_t val[kSortItems];
  int rank[kSortItems];
  int dig[kSortItems];
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    int64_t idx = base + r * 32 + lane;
    bool ok = idx < n;
    key[r] = ok ? kin[idx] : 0ull;
    val[r] = ok ? vin[idx] : 0u;
    int d = ok ? (int)((key[r] >> shift) & 255u) : 256;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    int before = wh[warp][d];
    __syncwarp();
    rank[r] = before + __popc(peers & lt);
    if ((peers & lt) == 0) wh[warp][d] = before + __popc(peers);
    __syncwarp();
    dig[r] = d;
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += blockDim.x) {
    int run = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
      int c = wh[w][d];
      wh[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    if (dig[r] < 256) {
      int64_t pos = (int64_t)offs[(int64_t)dig[r] * ntiles + blockIdx.x] + wh[warp][dig[r]] + rank[r];
      kout[pos] = key[r];
      vout[pos] = val[r];
    }
  }
}

}  // namespace

int exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t count, int32_t* total,
                       cudaStream_t s) {
  return exclusive_scan<int32_t>(in, out, count, total, s);
}
int exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t count, int64_t* total,
                       cudaStream_t s) {
  return exclusive_scan<int64_t>(in, out, count, total, s);
}

int radix_sort_pairs(uint64_t* keys, uint32_t* vals, int64_t n, int bits, cudaStream_t s) {
  if (n <= 1 || bits <= 0) return BKS_OK;
  const int ntiles = (int)((n + kSortTile - 1) / kSortTile);
  if ((int64_t)ntiles * 256 >= (int64_t)1 << 31)
    return fail(BKS_EUNSUPPORTED, "radix sort: too many items");
  DevBuf k2, v2, counts;
  BKS_TRY(k2.alloc(sizeof(uint64_t) * n, s));
  BKS_TRY(v2.alloc(sizeof(uint32_t) * n, s));
  BKS_TRY(counts.alloc(sizeof(int32_t) * 256 * (size_t)ntiles, s));
  uint64_t *ka = keys, *kb = k2.as<uint64_t>();
  uint32_t *va = vals, *vb = v2.as<uint32_t>();
  int passes = 0;
  for (int shift = 0; shift < bits; shift += 8, ++passes) {
    radix_hist<<<ntiles, kSortThreads, 0, s>>>(ka, n, shift, counts.as<int32_t>(), ntiles); ::bks::note_launch();
    BKS_CUDA_TRY(cudaGetLastError());
    BKS_TRY(exclusive_scan_i32(counts.as<int32_t>(), counts.as<int32_t>(), 256LL * ntiles,
                               nullptr, s));
    radix_scatter<<<ntiles, kSortThreads, 0, s>>>(ka, va, kb, vb, n, shift,
                                                  counts.as<int32_t>(), ntiles); ::bks::note_launch();
    BKS_CUDA_TRY(cudaGetLastError());
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != keys) {
    BKS_CUDA_TRY(cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
    BKS_CUDA_TRY(cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
  }
  return BKS_OK;
}

}  // namespace bks
