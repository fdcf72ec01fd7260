// Shared internals of the GB300 BKS library: error state, device buffers,
// the stored-tensor layout and the launch helpers used by every .cu file.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/bks.h"

namespace bks {

// ---- launch accounting (bks_launch_count) --------------------------------
void note_launch();

// ---- error handling (thread-local message, status codes of bks.h) -------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);

struct Status {
  int code = BKS_OK;
  std::string msg;
};

#define BKS_CUDA_TRY(expr)                                                   \
  do {                                                                       \
    cudaError_t e_ = (expr);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      return ::bks::fail(e_ == cudaErrorMemoryAllocation ? BKS_ENOMEM        \
                                                         : BKS_ECUDA,        \
                         std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    }                                                                        \
  } while (0)

#define BKS_TRY(expr)            \
  do {                           \
    int r_ = (expr);             \
    if (r_ != BKS_OK) return r_; \
  } while (0)

// ---- device memory owned by the library ----------------------------------
// Allocations go through cudaMallocAsync on the call's stream so that
// temporaries are stream-ordered.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t s = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept { *this = std::move(o); }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p; bytes = o.bytes; s = o.s;
      o.p = nullptr; o.bytes = 0;
    }
    return *this;
  }
  ~DevBuf() { release(); }
  int alloc(size_t nbytes, cudaStream_t stream) {
    release();
    s = stream;
    bytes = nbytes;
    if (nbytes == 0) return BKS_OK;
    BKS_CUDA_TRY(cudaMallocAsync(&p, nbytes, stream));
    return BKS_OK;
  }
  void release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    bytes = 0;
  }
  // long-lived buffers are freed on the legacy stream (the allocating
  // stream may be gone by then)
  void persist() { s = nullptr; }
  template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
};

// ---- stored tensor layout -------------------------------------------------
// Work plan of the sparse contractions.  A row longer than `split` entries
// is cut into "virtual rows" of at most `split` entries (their sums go to
// per-piece partials that a second kernel adds in a fixed order).  Virtual
// rows of at most `tile` entries ("short") are processed one per lane, 32
// to a warp, in order of decreasing length so that the lanes of a warp run
// loops of nearly equal trip count; longer ones are processed one per warp
// with the lanes striding over the entries.  The sizes are per tensor
// (defaults below; bks_tensor_autotune picks them by timing).
constexpr int kTile = 32;
constexpr int kSplit = 512;
// Default plan by size (measured on GB300 Zipf tensors, FP32 mode-1 calls
// at 5.0M, 11.8M and 48.5M stored entries): (32, 512) below 8M stored
// entries, (64, 1024) below 32M, (128, 2048) from 32M on.
inline void default_plan(int64_t nnz, int* tile, int* split) {
  if (nnz >= ((int64_t)32 << 20)) {
    *tile = 128;
    *split = 2048;
  } else if (nnz >= ((int64_t)8 << 20)) {
    *tile = 64;
    *split = 1024;
  } else {
    *tile = kTile;
    *split = kSplit;
  }
}
constexpr int kMaxTile = 128;
constexpr int kMinSplit = 128;
constexpr int kMaxSplit = 4096;

struct Part {
  // one sorted copy of the stored entries, CSR over `rows`
  int64_t rows = 0;
  DevBuf ptr;      // int32 [rows+1]
  DevBuf c0;       // int32 [nnz]: mode-1 copy -> k, mode-3 copy -> i
  DevBuf c1;       // int32 [nnz]: j
  DevBuf v;        // [nnz] in the input value dtype
  DevBuf v32;      // float [nnz] when the input dtype is double
  DevBuf v64;      // double [nnz] when the input dtype is float
  // tile plan
  int tile = kTile, split = kSplit;
  int32_t nv = 0, nslots = 0, nsplit = 0;
  int32_t nvec = 0, nshortv = 0;  // virtual rows taken one per warp / one per lane
  DevBuf vptr;        // int32 [nv+1]   first entry of each virtual row
  DevBuf vrow;        // int32 [nv]     row of each virtual row
  DevBuf vslot;       // int32 [nv]     partial-sum slot, -1 if the row is not cut
  DevBuf vorder;      // int32 [nv]: the nvec warp rows, then the short rows by decreasing length
  DevBuf vitems;      // int4 [nv]: per vorder position (first entry, end, row, slot);
                      // for the short rows, first and end in the interleaved copy below
  // Lane-interleaved copy of the short virtual rows' entries: the short
  // rows are taken 32 at a time in vorder order (group g, lane l), and
  // entry t of a row sits at sell_base[g] + 32 t + l, so that the 32 lanes'
  // loads of one step are consecutive.  Positions past a row's end are
  // padding and never read.
  int64_t nsell = 0;
  DevBuf sc0, sc1;    // int32 [nsell]: c0, c1 of the entries
  DevBuf sv32;        // float [nsell]
  DevBuf sv64;        // double [nsell]
  DevBuf split_row;   // int32 [nsplit]   rows that were cut
  DevBuf split_first; // int32 [nsplit+1] their first slot (slots are consecutive)
  int32_t nempty = 0;
  DevBuf empty_rows;  // int32 [nempty] rows without entries (their output is zero)
  std::vector<int32_t> host_ptr;  // host copy of ptr (kept for the mode-3 copy only)
  void persist() {
    for (DevBuf* b : {&ptr, &c0, &c1, &v, &v32, &v64, &vptr, &vrow, &vslot, &vorder, &vitems,
                      &sc0, &sc1, &sv32, &sv64, &split_row, &split_first, &empty_rows})
      b->persist();
  }
};

// Chunks of the mode-3 copy for the large-rank cores: every slice k is cut
// into pieces of about nnz / (16 SMs) entries; the chunks of a slice are
// consecutive.  Built once per tensor at ingest.
struct CorePlan {
  int32_t nch = 0, nsl = 0;
  DevBuf lo, hi;      // int32 [nch]: entry range of each chunk
  DevBuf sl_k;        // int32 [nsl]: slice index k of each non-empty slice
  DevBuf sl_first;    // int32 [nsl+1]: first chunk of each non-empty slice
  // runs: maximal ranges of entries with equal (k, i), cut at chunk starts
  // and every 32 entries; the core sums v X[j, :] over a run before its
  // outer product with X[i, :]
  int32_t nruns = 0;
  DevBuf run_start;   // int32 [nruns+1]: first entry of each run (nnz at the end)
  DevBuf chunk_run;   // int32 [nch+1]: first run of each chunk
  void persist() {
    for (DevBuf* b : {&lo, &hi, &sl_k, &sl_first, &run_start, &chunk_run}) b->persist();
  }
};

int build_core_plan(const Part& m3, int64_t n, int64_t nnz, CorePlan& cp, cudaStream_t s);

}  // namespace bks

// A stored tensor.  (1,2)-symmetric (general == 0): l = m, two sorted
// copies.  General l x m x n (general == 1, Section 5): a third copy for
// the mode-2 contraction.
struct bks_tensor {
  int64_t l = 0, m = 0, n = 0, nnz = 0;
  int vdtype = BKS_F64;
  int general = 0;
  double fro2 = 0.0;
  bks::Part m1;   // sorted by (i, j, k): rows i, c0 = k, c1 = j
  bks::Part m2;   // general only, sorted by (j, i, k): rows j, c0 = k, c1 = i
  bks::Part m3;   // sorted by (k, i, j): rows k, c0 = i, c1 = j
  bks::CorePlan cp;
};

namespace bks {
// Entry points of the (1,2)-symmetric method refuse a general tensor and
// the general ones a symmetric tensor.
inline int require_symmetric(const bks_tensor* t) {
  if (t && t->general)
    return fail(BKS_EUNSUPPORTED, "a general (l x m x n) tensor: use the bks_gen_* calls");
  return BKS_OK;
}
inline int require_general(const bks_tensor* t) {
  if (t && !t->general)
    return fail(BKS_EUNSUPPORTED, "a (1,2)-symmetric tensor: use the symmetric calls");
  return BKS_OK;
}
}  // namespace bks

namespace bks {

// exact IEEE adds (no contraction into FMA) and bitwise equality
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ bool same_bits(float a, float b) {
  return __float_as_uint(a) == __float_as_uint(b);
}
__device__ __forceinline__ bool same_bits(double a, double b) {
  return __double_as_longlong(a) == __double_as_longlong(b);
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
// ---- per-device state -------------------------------------------------------
// Calls may come from any host thread with any current device; what is
// cached per process (SM counts, raised shared-memory limits, workspaces)
// is therefore kept per device index.
constexpr int kMaxDevices = 64;

// The calling thread's current device, or -1 when it cannot be used as an
// index into the per-device caches.
inline int current_device() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return -1;
  return dev;
}

// SM count of the current device (queried once per device).
inline int num_sms() {
  static std::atomic<int> cache[kMaxDevices];
  const int dev = current_device();
  int n = dev >= 0 ? cache[dev].load(std::memory_order_relaxed) : 0;
  if (n > 0) return n;
  int d = 0;
  cudaGetDevice(&d);
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || n <= 0) n = 1;
  if (dev >= 0) cache[dev].store(n, std::memory_order_relaxed);
  return n;
}

// Runs an initialisation (a cudaFuncSetAttribute, say) once per device, the
// first time a thread with that device current asks, and returns its
// result on every later call for that device.  Thread-safe.
class PerDeviceOnce {
 public:
  template <typename F>
  cudaError_t run(F&& init) {
    const int dev = current_device();
    if (dev < 0) return init();
    std::lock_guard<std::mutex> lock(mu_);
    if (!done_[dev]) {
      err_[dev] = init();
      done_[dev] = true;
    }
    return err_[dev];
  }

 private:
  std::mutex mu_;
  bool done_[kMaxDevices] = {};
  cudaError_t err_[kMaxDevices] = {};
};

// ---- scans (scan.cu) ------------------------------------------------------
// out[i] = sum_{t<i} in[i]; out may alias in; total (device) optional.
int exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t count,
                       int32_t* total_dev, cudaStream_t s);
int exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t count,
                       int64_t* total_dev, cudaStream_t s);
// stable LSD radix sort of (key, payload) by the low `bits` bits of key
int radix_sort_pairs(uint64_t* keys, uint32_t* vals, int64_t count, int bits,
                     cudaStream_t s);

// ---- tile plans (ingest.cu) -----------------------------------------------
int build_tile_plan(Part& P, int64_t nnz, cudaStream_t s);

// ---- contractions (contract.cu) ------------------------------------------
// Row-major padded "gather" copies of the dense operands are built inside.
int contract_mode1(const bks_tensor* t, const void* X, int64_t ldx, int p,
                   const void* Y, int64_t ldy, int q, void* out, int64_t ldo,
                   int dtype, cudaStream_t s);
int contract_mode3(const bks_tensor* t, const void* X, int64_t ldx, int p,
                   const void* X2, int64_t ldx2, int q, void* out, int64_t ldo,
                   int dtype, cudaStream_t s);
int contract_core(const bks_tensor* t, const void* U, int64_t ldu, int r1,
                  const void* W, int64_t ldw, int r3, void* F, int dtype,
                  cudaStream_t s);
// FP64 operands/results; fp32 selects FP32 arithmetic (the mixed form)
int contract_mode1_x(const bks_tensor* t, const double* X, int64_t ldx, int p, const double* Y,
                     int64_t ldy, int q, double* out, int64_t ldo, bool fp32, cudaStream_t s);
int contract_mode3_x(const bks_tensor* t, const double* X, int64_t ldx, int p, const double* X2,
                     int64_t ldx2, int q, double* out, int64_t ldo, bool fp32, cudaStream_t s);
int contract_core_x(const bks_tensor* t, const double* U, int64_t ldu, int r1, const double* W,
                    int64_t ldw, int r3, double* F, bool fp32, cudaStream_t s);
// general tensors (Section 5): mode md in {1, 2, 3} with the other two
// modes' operands; the core C = A.(X,Y,Z) (k1, k2 <= 128), FP64
int gen_contract_x(const bks_tensor* t, int md, const double* B1, int64_t ld1, int p,
                   const double* B2, int64_t ld2, int q, double* out, int64_t ldo, cudaStream_t s);
int gen_core_x(const bks_tensor* t, const double* X, int64_t ldx, int k1, const double* Y,
               int64_t ldy, int k2, const double* Z, int64_t ldz, int k3, double* C,
               cudaStream_t s);
// inner solve (inner.cu)
int inner_solve(const double* C, int k1, int k3, int r1, int r3, double tol, int max_inner,
                int init_sweeps, int newton_after, double* Uh, double* Wh, double* negU, double* negW, double* info,
                cudaStream_t s);
// general core (k1 x k2 x k3): HOSVD start vs the current point, then HOOI
// sweeps; negated factors and info[4] = {grad, ||F||, sweeps, hosvd_won}
int gen_inner_solve(const double* C, int k1, int k2, int k3, int r1, int r2, int r3, double tol,
                    int max_inner, int init_sweeps, double* negU, double* negV, double* negW,
                    double* info, cudaStream_t s);

}  // namespace bks
