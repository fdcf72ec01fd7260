// Tile kernels of the sparse contractions (Section 2.2; Algorithm 3 step
// (i); Section 4.3.1): the row-class kernel k_contract, the piece reduction
// and the zero rows, and dispatch() over the width buckets.  Included only
// by the per-type instantiation files.
#pragma once
#include "contract_tile.cuh"

namespace bks {

namespace {

// The first N values of a packed row (stride RowStride<T, N>) from global
// memory through the read-only path, with an L2 eviction-priority policy
// (pol): one 32-byte load for 8-float rows (sm_100 and later), 16-byte
// loads when rows are 16-byte aligned (the unused tail of the last vector
// is padding of the row), else 8-byte loads for FP32, else scalar.
__device__ __forceinline__ void ldg32_hint(const float* p, float (&v)[8], uint64_t pol) {
  asm("ld.global.nc.L2::cache_hint.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8], %9;"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]),
        "=f"(v[7])
      : "l"(p), "l"(pol));
}
__device__ __forceinline__ uint4 ldg16_hint(const void* p, uint64_t pol) {
  uint4 r;
  asm("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
      : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
      : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ uint2 ldg8_hint(const void* p, uint64_t pol) {
  uint2 r;
  asm("ld.global.nc.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;" : "=r"(r.x), "=r"(r.y) : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ float ldg_hint(const float* p, uint64_t pol) {
  float r;
  asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(r) : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ double ldg_hint(const double* p, uint64_t pol) {
  double r;
  asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(r) : "l"(p), "l"(pol));
  return r;
}

template <typename T, int N>
__device__ __forceinline__ void load_row(const T* __restrict__ base, T (&x)[N], uint64_t pol) {
  constexpr int S = RowStride<T, N>::v;
  if constexpr (sizeof(T) == 4 && S == 8) {
    float v[8];
    ldg32_hint(reinterpret_cast<const float*>(base), v, pol);
#pragma unroll
    for (int u = 0; u < N; ++u) x[u] = v[u];
  } else if constexpr ((sizeof(T) * S) % 16 == 0) {
    constexpr int V = (int)(16 / sizeof(T));
    constexpr int NV = (N + V - 1) / V;  // NV V <= S: S is a multiple of V and S >= N
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      const uint4 q = ldg16_hint(reinterpret_cast<const uint4*>(base) + t, pol);
      const T* qq = reinterpret_cast<const T*>(&q);
#pragma unroll
      for (int u = 0; u < V; ++u)
        if (t * V + u < N) x[t * V + u] = qq[u];
    }
  } else if constexpr (sizeof(T) == 4 && S % 2 == 0) {
#pragma unroll
    for (int t = 0; t < N / 2; ++t) {
      const uint2 q = ldg8_hint(reinterpret_cast<const uint2*>(base) + t, pol);
      x[2 * t] = __uint_as_float(q.x);
      x[2 * t + 1] = __uint_as_float(q.y);
    }
  } else {
#pragma unroll
    for (int t = 0; t < N; ++t) x[t] = ldg_hint(base + t, pol);
  }
}

// The first N values of a packed row held in shared memory.
template <typename T, int N>
__device__ __forceinline__ void load_row_smem(const T* base, T (&x)[N]) {
  constexpr int S = RowStride<T, N>::v;
  if constexpr ((sizeof(T) * S) % 16 == 0) {
    constexpr int V = (int)(16 / sizeof(T));
    constexpr int NV = (N + V - 1) / V;
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      const float4 q = reinterpret_cast<const float4*>(base)[t];
      const T* qq = reinterpret_cast<const T*>(&q);
#pragma unroll
      for (int u = 0; u < V; ++u)
        if (t * V + u < N) x[t * V + u] = qq[u];
    }
  } else {
#pragma unroll
    for (int t = 0; t < N; ++t) x[t] = base[t];
  }
}

// accumulator shape: TRI -> upper triangle of PB x PB, else PB x QB
template <int PB, int QB, bool TRI>
struct Shape {
  static constexpr int W = TRI ? PB * (PB + 1) / 2 : PB * QB;
};

template <typename T, int PB, int QB, bool TRI>
__device__ __forceinline__ void accumulate(T (&acc)[Shape<PB, QB, TRI>::W], T v,
                                           const T (&xa)[PB], const T (&xb)[TRI ? PB : QB]) {
  T va[PB];
#pragma unroll
  for (int a = 0; a < PB; ++a) va[a] = v * xa[a];
  if constexpr (TRI) {
#pragma unroll
    for (int b = 0; b < PB; ++b)
#pragma unroll
      for (int a = 0; a <= b; ++a) acc[a + b * (b + 1) / 2] = fma(va[a], xb[b], acc[a + b * (b + 1) / 2]);
  } else {
#pragma unroll
    for (int b = 0; b < QB; ++b)
#pragma unroll
      for (int a = 0; a < PB; ++a) acc[a + PB * b] = fma(va[a], xb[b], acc[a + PB * b]);
  }
}

struct TileArgs {
  const int4* items;      // per work item (vorder order): first entry, end, row, slot
  const int32_t* vorder;  // the nvec warp rows, then the short rows by decreasing length
  const int32_t* vptr;
  const int32_t* vrow;
  const int32_t* vslot;
  int32_t nvec, nshortv;
  const int32_t* ia;   // index into operand A per entry
  const int32_t* ib;   // index into operand B per entry
  const int32_t* sia;  // the same for the lane-interleaved copy of the short rows
  const int32_t* sib;
  int32_t nbs;         // rows of operand B held in shared memory (0: gathered from global)
  const int32_t* empty_rows;  // rows without entries: their wcols output columns are zeroed
  int32_t nempty, wcols;
};

template <typename T, typename OT, int PB, int QB, bool TRI>
__device__ __forceinline__ void flush_row(int64_t row, int slot,
                                          const T (&acc)[Shape<PB, QB, TRI>::W], int p, int q,
                                          OT* __restrict__ out, int64_t ldo,
                                          T* __restrict__ partial) {
  constexpr int W = Shape<PB, QB, TRI>::W;
  if (slot >= 0) {
    T* dst = partial + (int64_t)slot * W;
#pragma unroll
    for (int c = 0; c < W; ++c) dst[c] = acc[c];
    return;
  }
  if constexpr (TRI) {
#pragma unroll
    for (int b = 0; b < PB; ++b)
#pragma unroll
      for (int a = 0; a <= b; ++a)
        if (b < p) out[row + ldo * (a + b * (b + 1) / 2)] = (OT)acc[a + b * (b + 1) / 2];
  } else {
#pragma unroll
    for (int b = 0; b < QB; ++b)
#pragma unroll
      for (int a = 0; a < PB; ++a)
        if (a < p && b < q) out[row + ldo * (a + p * b)] = (OT)acc[a + PB * b];
  }
}

constexpr int next_pow2(int x) { return x <= 1 ? 1 : 2 * next_pow2((x + 1) / 2); }

// One level of a recursive-halving sum over the lanes: each lane holds N
// values; the lanes with bit `o` set keep the upper half and receive it
// from the partner lane (lane ^ o), the others keep the lower half, so that
// every lane ends with N/2 sums.  With N = 1 the value is added as it is.
template <typename T, int N>
__device__ __forceinline__ void halve(T* a, int lane, int o) {
  if constexpr (N >= 2) {
    constexpr int H = N / 2;
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int c = 0; c < H; ++c) {
      const T send = upper ? a[c] : a[H + c];
      const T keep = upper ? a[H + c] : a[c];
      a[c] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  } else {
    a[0] += __shfl_xor_sync(0xffffffffu, a[0], o);
  }
}

// Warp sum of acc[W] (five halving levels, a fixed order), written to the
// virtual row's output row or partial slot by the lanes that hold each sum.
template <typename T, typename OT, int PB, int QB, bool TRI>
__device__ __forceinline__ void warp_reduce_flush(int64_t row, int slot,
                                                  const T (&acc)[Shape<PB, QB, TRI>::W], int p,
                                                  int q, OT* __restrict__ out, int64_t ldo,
                                                  T* __restrict__ partial, int lane) {
  constexpr int W = Shape<PB, QB, TRI>::W;
  constexpr int W2 = next_pow2(W);
  T a[W2];
#pragma unroll
  for (int c = 0; c < W2; ++c) a[c] = c < W ? acc[c] : T(0);
  halve<T, W2>(a, lane, 16);
  halve<T, (W2 / 2 > 1 ? W2 / 2 : 1)>(a, lane, 8);
  halve<T, (W2 / 4 > 1 ? W2 / 4 : 1)>(a, lane, 4);
  halve<T, (W2 / 8 > 1 ? W2 / 8 : 1)>(a, lane, 2);
  halve<T, (W2 / 16 > 1 ? W2 / 16 : 1)>(a, lane, 1);
  // index of a[0] in this lane, and whether this lane is the first of the
  // lanes that hold the same sums
  int base = 0;
  bool writer = true;
  {
    int n = W2;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      if (n >= 2) {
        n >>= 1;
        if (lane & o) base += n;
      } else if (lane & o) {
        writer = false;
      }
    }
  }
  if (!writer) return;
  constexpr int R = W2 / 32 > 1 ? W2 / 32 : 1;
#pragma unroll
  for (int c = 0; c < R; ++c) {
    const int idx = base + c;
    if (idx >= W) continue;
    if (slot >= 0) {
      partial[(int64_t)slot * W + idx] = a[c];
      continue;
    }
    if constexpr (TRI) {
      int b = 0;
      while ((b + 1) * (b + 2) / 2 <= idx) ++b;
      if (b < p) out[row + ldo * idx] = (OT)a[c];
    } else {
      const int aa = idx % PB, bb = idx / PB;
      if (aa < p && bb < q) out[row + ldo * (aa + p * bb)] = (OT)a[c];
    }
  }
}

// ---- the tile kernel --------------------------------------------------------
constexpr int kTileWarps = 8;                    // warps per block
constexpr size_t kBSmemMax = 32 * 1024;          // operand B staged in shared memory up to this

// L2 policies: lines read once (the entry streams) leave first; lines
// gathered again and again (the packed operands) stay longest.
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// Stream loads: read once, not kept in L1, first out of L2.
__device__ __forceinline__ int ldg_stream(const int32_t* p, uint64_t pol) {
  int r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(r) : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ float ldg_stream(const float* p, uint64_t pol) {
  float r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(r) : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ double ldg_stream(const double* p, uint64_t pol) {
  double r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(r) : "l"(p), "l"(pol));
  return r;
}

// One entry pair of gathers: operand A's row from global memory (kept in
// L2), operand B's from shared memory (BSM) or global memory.
template <typename T, int PB, int QB, bool TRI, bool BSM>
__device__ __forceinline__ void gather_pair(const T* __restrict__ Ap, const T* __restrict__ Bp,
                                            const T* Bs, int ia, int ib, uint64_t pol,
                                            T (&xa)[PB], T (&xb)[TRI ? PB : QB]) {
  constexpr int NB = TRI ? PB : QB;
  load_row<T, PB>(Ap + (int64_t)ia * RowStride<T, PB>::v, xa, pol);
  if constexpr (BSM)
    load_row_smem<T, NB>(Bs + (int64_t)ib * RowStride<T, NB>::v, xb);
  else
    load_row<T, NB>(Bp + (int64_t)ib * RowStride<T, NB>::v, xb, pol);
}

// Blocks per SM the tile kernel is compiled for: its live values are
// about the accumulators, four entries' gathered rows and 32 others.
template <typename T, int PB, int QB, bool TRI, bool BSM>
struct RegBlocks {
  static constexpr int NB = TRI ? PB : QB;
  static constexpr int live = (int)(sizeof(T) / 4) *
                                  (Shape<PB, QB, TRI>::W + 4 * (PB + (BSM ? 0 : NB))) + 32;
  static constexpr int regs = (live + 7) / 8 * 8;
  static constexpr int by_regs = 65536 / (kTileWarps * 32 * regs);
  static constexpr int v0 = by_regs < 1 ? 1 : (by_regs > 8 ? 8 : by_regs);
  // The FP32 3-column triangle with operand B gathered spills 40 bytes at
  // four blocks (64 registers); at three blocks it ran 4% (5.0M entries)
  // and 12% (48.5M entries) faster on GB300.  One block fewer lost 1-8% on
  // every other measured shape (mode 1, 3 x 3 to 5 x 5, FP32 and FP64).
  static constexpr bool spills = sizeof(T) == 4 && TRI && !BSM && PB == 3;
  static constexpr int v = spills && v0 > 1 ? v0 - 1 : v0;
};

// Mode-1 / mode-3 contraction over the work plan (see common.cuh).  The
// warp items are the nvec long virtual rows (one warp each) followed by the
// groups of 32 short rows (one lane each, in order of decreasing length); a
// persistent grid takes them round robin (warp w: items w, w + nwarps, ...).
// Long rows: the lanes stride over the entries, loading the next group of
// four entries' indices and values while the current group's gathers are in
// flight, and the lane sums are combined by warp_reduce_flush.  Short rows:
// each lane sums its row from the lane-interleaved copy (coalesced loads)
// and writes it.  Operand B (the mode-1 Y, n rows) is read from shared
// memory when it fits (BSM).  The entry streams are loaded with an
// evict-first L2 policy and the gathered rows with evict-last, so that the
// packed operands stay in L2.  No atomics: every sum has a fixed order.
template <typename T, typename OT, int PB, int QB, bool TRI, bool BSM>
__global__ void __launch_bounds__(kTileWarps * 32, (RegBlocks<T, PB, QB, TRI, BSM>::v))
k_contract(TileArgs ta, const T* __restrict__ vals, const T* __restrict__ svals,
           const T* __restrict__ Ap, const T* __restrict__ Bp, int p, int q,
           OT* __restrict__ out, int64_t ldo, T* __restrict__ partial) {
  constexpr int W = Shape<PB, QB, TRI>::W;
  constexpr int NB = TRI ? PB : QB;
  extern __shared__ __align__(128) unsigned char tile_smem[];
  T* Bs = reinterpret_cast<T*>(tile_smem);
  if constexpr (BSM) {
    const int64_t cnt = (int64_t)ta.nbs * RowStride<T, NB>::v;
    for (int64_t x = threadIdx.x; x < cnt; x += blockDim.x) Bs[x] = Bp[x];
    __syncthreads();
  }
  // rows without entries get zeros, spread over the whole grid before the
  // items (these scattered stores overlap the items' loads)
  {
    const int64_t tot = (int64_t)ta.nempty * ta.wcols;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
         t += (int64_t)gridDim.x * blockDim.x) {
      const int r = (int)(t % ta.nempty), c = (int)(t / ta.nempty);
      out[ta.empty_rows[r] + ldo * c] = OT(0);
    }
  }
  const int lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * kTileWarps;
  const int total = ta.nvec + (ta.nshortv + 31) / 32;
  const uint64_t once = policy_evict_first(), keep = policy_evict_last();
  for (int u = blockIdx.x * kTileWarps + (threadIdx.x >> 5); u < total; u += nwarps) {
    T acc[W];
#pragma unroll
    for (int c = 0; c < W; ++c) acc[c] = T(0);
    if (u < ta.nvec) {
      const int4 it = __ldg(ta.items + u);
      const int e = it.y;
      int x = it.x + lane;
      int iav[4], ibv[4];
      T v[4];
      if (x + 96 < e) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          iav[k] = ldg_stream(ta.ia + x + 32 * k, once);
          ibv[k] = ldg_stream(ta.ib + x + 32 * k, once);
          v[k] = ldg_stream(vals + x + 32 * k, once);
        }
      }
      while (x + 96 < e) {
        T xa[4][PB], xb[4][NB];
#pragma unroll
        for (int k = 0; k < 4; ++k)
          gather_pair<T, PB, QB, TRI, BSM>(Ap, Bp, Bs, iav[k], ibv[k], keep, xa[k], xb[k]);
        T vc[4] = {v[0], v[1], v[2], v[3]};
        x += 128;
        if (x + 96 < e) {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            iav[k] = ldg_stream(ta.ia + x + 32 * k, once);
            ibv[k] = ldg_stream(ta.ib + x + 32 * k, once);
            v[k] = ldg_stream(vals + x + 32 * k, once);
          }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) accumulate<T, PB, QB, TRI>(acc, vc[k], xa[k], xb[k]);
      }
      for (; x < e; x += 32) {
        T xa[PB], xb[NB];
        gather_pair<T, PB, QB, TRI, BSM>(Ap, Bp, Bs, ldg_stream(ta.ia + x, once),
                                         ldg_stream(ta.ib + x, once), keep, xa, xb);
        accumulate<T, PB, QB, TRI>(acc, ldg_stream(vals + x, once), xa, xb);
      }
      warp_reduce_flush<T, OT, PB, QB, TRI>(it.z, it.w, acc, p, q, out, ldo, partial, lane);
      continue;
    }
    const int sidx = (u - ta.nvec) * 32 + lane;
    if (sidx >= ta.nshortv) continue;
    // the row's entries in the lane-interleaved copy: it.x, it.x + 32, ... < it.y
    const int4 it = __ldg(ta.items + ta.nvec + sidx);
    const int e = it.y;
    int x = it.x;
    for (; x + 96 < e; x += 128) {
      int iav[4], ibv[4];
      T v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        iav[k] = ldg_stream(ta.sia + x + 32 * k, once);
        ibv[k] = ldg_stream(ta.sib + x + 32 * k, once);
        v[k] = ldg_stream(svals + x + 32 * k, once);
      }
      T xa[4][PB], xb[4][NB];
#pragma unroll
      for (int k = 0; k < 4; ++k)
        gather_pair<T, PB, QB, TRI, BSM>(Ap, Bp, Bs, iav[k], ibv[k], keep, xa[k], xb[k]);
#pragma unroll
      for (int k = 0; k < 4; ++k) accumulate<T, PB, QB, TRI>(acc, v[k], xa[k], xb[k]);
    }
    for (; x < e; x += 32) {
      T xa[PB], xb[NB];
      gather_pair<T, PB, QB, TRI, BSM>(Ap, Bp, Bs, ldg_stream(ta.sia + x, once),
                                       ldg_stream(ta.sib + x, once), keep, xa, xb);
      accumulate<T, PB, QB, TRI>(acc, ldg_stream(svals + x, once), xa, xb);
    }
    flush_row<T, OT, PB, QB, TRI>(it.z, it.w, acc, p, q, out, ldo, partial);
  }
}


// number of warps of a plan
inline int plan_warps(const Part& P) { return P.nvec + (P.nshortv + 31) / 32; }


// s + y into the unevaluated sum s + c, the rounding error of s + y going
// to c (TwoSum, Knuth's error-free transformation: exact in IEEE
// arithmetic, no FMA contraction involved).
template <typename T>
__device__ __forceinline__ void two_sum_acc(T& s, T& c, T y) {
  const T t = s + y;
  const T bp = t - s;
  c += (s - (t - bp)) + (y - bp);
  s = t;
}

// Rows cut into pieces: add the pieces' partial sums in a fixed order, with
// TwoSum compensation at both levels (pieces into 256 / W group sums, the
// group sums into one), so that the error of a cut row does not grow with
// its number of pieces.
template <typename T, typename OT, int PB, int QB, bool TRI>
__global__ void k_split_reduce(const int32_t* __restrict__ split_row,
                               const int32_t* __restrict__ split_first, int nsplit,
                               const T* __restrict__ partial, int p, int q, OT* __restrict__ out,
                               int64_t ldo) {
  constexpr int W = Shape<PB, QB, TRI>::W;
  static_assert(W <= 256, "one output column per thread of the 256-thread block");
  __shared__ T sh[256], shc[256];
  const int s = blockIdx.x;
  if (s >= nsplit) return;
  const int f0 = split_first[s], f1 = split_first[s + 1];
  const int groups = 256 / W;
  const int c = threadIdx.x % W, g = threadIdx.x / W;
  T acc = T(0), cmp = T(0);
  if (g < groups) {
    // four loads issued before their four additions (the same order of
    // additions as one piece at a time)
    int f = f0 + g;
    for (; f + 3 * groups < f1; f += 4 * groups) {
      const T y0 = partial[(int64_t)f * W + c];
      const T y1 = partial[(int64_t)(f + groups) * W + c];
      const T y2 = partial[(int64_t)(f + 2 * groups) * W + c];
      const T y3 = partial[(int64_t)(f + 3 * groups) * W + c];
      two_sum_acc(acc, cmp, y0);
      two_sum_acc(acc, cmp, y1);
      two_sum_acc(acc, cmp, y2);
      two_sum_acc(acc, cmp, y3);
    }
    for (; f < f1; f += groups) two_sum_acc(acc, cmp, partial[(int64_t)f * W + c]);
  }
  sh[threadIdx.x] = acc;
  shc[threadIdx.x] = cmp;
  __syncthreads();
  if (threadIdx.x < W) {
    T tot = T(0), tc = T(0);
    for (int t = 0; t < groups; ++t) {
      tc += shc[t * W + threadIdx.x];
      two_sum_acc(tot, tc, sh[t * W + threadIdx.x]);
    }
    const int64_t row = split_row[s];
    int col = -1;
    if constexpr (TRI) {
      int b = 0;
      while ((b + 1) * (b + 2) / 2 <= c) ++b;
      if (b < p) col = c;
    } else {
      int a = c % PB, b = c / PB;
      if (a < p && b < q) col = a + p * b;
    }
    if (col >= 0) out[row + ldo * col] = (OT)(tot + tc);
  }
}

template <typename T>
__global__ void k_zero_rows(const int32_t* __restrict__ rows, int nrows, int w,
                            T* __restrict__ out, int64_t ldo) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)nrows * w;
       t += (int64_t)gridDim.x * blockDim.x) {
    int r = (int)(t % nrows), c = (int)(t / nrows);
    out[rows[r] + ldo * c] = T(0);
  }
}

// The tile kernel on a persistent grid: as many blocks as fit on the GPU
// at this shared-memory size (operand B), at most one warp per item.
template <typename T, typename OT, int PB, int QB, bool TRI, bool BSM>
int launch_tiles(const TileArgs& ta, int items, size_t smem, const T* vals, const T* svals,
                 const T* Ap, const T* Bp, int p, int q, OT* out, int64_t ldo, T* part,
                 cudaStream_t s) {
  static PerDeviceOnce once;
  const cudaError_t attr = once.run([] {
    return cudaFuncSetAttribute(k_contract<T, OT, PB, QB, TRI, BSM>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBSmemMax);
  });
  if (attr != cudaSuccess)
    return fail(BKS_ECUDA, std::string("k_contract shared-memory limit: ") +
                               cudaGetErrorString(attr));
  // resident blocks per SM, cached per device for the last shared-memory size
  static std::atomic<int64_t> occ[kMaxDevices];
  const int dev = current_device();
  const int64_t key = (int64_t)(smem + 1) << 8;
  int64_t hit = dev >= 0 ? occ[dev].load(std::memory_order_relaxed) : 0;
  int per_sm = (hit & ~int64_t(255)) == key ? (int)(hit & 255) : 0;
  if (per_sm == 0) {
    BKS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, k_contract<T, OT, PB, QB, TRI, BSM>, kTileWarps * 32, smem));
    if (dev >= 0 && per_sm > 0 && per_sm < 256)
      occ[dev].store(key | per_sm, std::memory_order_relaxed);
  }
  const int64_t fit = (int64_t)std::max(1, per_sm) * num_sms();
  const int blocks = (int)std::max<int64_t>(
      1, std::min<int64_t>(fit, ((int64_t)items + kTileWarps - 1) / kTileWarps));
  k_contract<T, OT, PB, QB, TRI, BSM><<<blocks, kTileWarps * 32, smem, s>>>(
      ta, vals, svals, Ap, Bp, p, q, out, ldo, part);
  ::bks::note_launch();
  BKS_CUDA_TRY(cudaGetLastError());
  return BKS_OK;
}

// One launch pair (tile kernel + piece reduction) for fixed buckets.  The
// partial sums of cut rows go to `part` (nslots x W values) when the caller
// provides it, else to a stream-ordered allocation.
template <typename T, typename OT, int PB, int QB, bool TRI>
int launch_contract(const Part& P, int vdtype, const int32_t* ia, const int32_t* ib,
                    const T* Ap, const T* Bp, int64_t brows, int p, int q, OT* out, int64_t ldo,
                    T* part, cudaStream_t s) {
  constexpr int W = Shape<PB, QB, TRI>::W;
  constexpr int NB = TRI ? PB : QB;
  const size_t bbytes = sizeof(T) * (size_t)brows * row_stride<T>(NB);
  const int nbs = bbytes <= kBSmemMax ? (int)brows : 0;
  const size_t smem = nbs > 0 ? bbytes : 0;
  const int w = TRI ? p * (p + 1) / 2 : p * q;
  // The tile kernel zeroes the rows without entries when its grid is large
  // enough for them: at most 64 stores per thread of the smallest grid it
  // can get (one block per 8 items, at most one block per SM).  A tensor
  // with few entries and many empty rows gets the separate zero kernel,
  // sized by its own work.
  const int64_t min_blocks =
      std::min<int64_t>(((int64_t)plan_warps(P) + kTileWarps - 1) / kTileWarps, num_sms());
  const bool fused_zero =
      P.nv > 0 && (int64_t)P.nempty * w <= 64 * (int64_t)kTileWarps * 32 * min_blocks;
  TileArgs ta{P.vitems.as<int4>(), P.vorder.as<int32_t>(), P.vptr.as<int32_t>(),
              P.vrow.as<int32_t>(), P.vslot.as<int32_t>(), P.nvec, P.nshortv, ia, ib,
              sell_of(P, ia), sell_of(P, ib), nbs, P.empty_rows.as<int32_t>(),
              fused_zero ? P.nempty : 0, w};
  DevBuf partial;
  if (P.nslots > 0 && !part) {
    BKS_TRY(partial.alloc(sizeof(T) * (size_t)P.nslots * W, s));
    part = partial.as<T>();
  }
  if (P.nv > 0) {
    // persistent grid: as many blocks as fit on the GPU, at most one warp per item
    const int items = plan_warps(P);
    if (nbs > 0)
      BKS_TRY((launch_tiles<T, OT, PB, QB, TRI, true>(ta, items, smem, values_of<T>(P, vdtype),
                                                      sell_values_of<T>(P), Ap, Bp, p, q, out,
                                                      ldo, part, s)));
    else
      BKS_TRY((launch_tiles<T, OT, PB, QB, TRI, false>(ta, items, smem, values_of<T>(P, vdtype),
                                                       sell_values_of<T>(P), Ap, Bp, p, q, out,
                                                       ldo, part, s)));
  }
  if (P.nsplit > 0) {
    k_split_reduce<T, OT, PB, QB, TRI><<<P.nsplit, 256, 0, s>>>(
        P.split_row.as<int32_t>(), P.split_first.as<int32_t>(), P.nsplit, part, p, q,
        out, ldo); ::bks::note_launch();
    BKS_CUDA_TRY(cudaGetLastError());
  }
  if (P.nempty > 0 && !fused_zero) {
    k_zero_rows<OT><<<grid_for((int64_t)P.nempty * w), 256, 0, s>>>(P.empty_rows.as<int32_t>(),
                                                                    P.nempty, w, out, ldo); ::bks::note_launch();
    BKS_CUDA_TRY(cudaGetLastError());
  }
  return BKS_OK;
}

}  // namespace

template <typename T, typename OT>
int dispatch(const Part& P, int vdtype, const int32_t* ia, const int32_t* ib, const T* Ap,
             int PB, const T* Bp, int QB, int64_t brows, bool tri, int p, int q, OT* out,
             int64_t ldo, cudaStream_t s, T* part) {
#define BKS_CASE(pb, qb)                                                                      \
  if (!tri && PB == pb && QB == qb)                                                           \
    return launch_contract<T, OT, pb, qb, false>(P, vdtype, ia, ib, Ap, Bp, brows, p, q, out,  \
                                                 ldo, part, s);
  BKS_CASE(2, 2) BKS_CASE(2, 3) BKS_CASE(2, 4) BKS_CASE(2, 5) BKS_CASE(2, 8)
  BKS_CASE(3, 2) BKS_CASE(3, 3) BKS_CASE(3, 4) BKS_CASE(3, 5) BKS_CASE(3, 8)
  BKS_CASE(4, 2) BKS_CASE(4, 3) BKS_CASE(4, 4) BKS_CASE(4, 5) BKS_CASE(4, 8)
  BKS_CASE(5, 2) BKS_CASE(5, 3) BKS_CASE(5, 4) BKS_CASE(5, 5)
  BKS_CASE(8, 2) BKS_CASE(8, 3) BKS_CASE(8, 4)
#undef BKS_CASE
#define BKS_TRI(pb)                                                                           \
  if (tri && PB == pb)                                                                        \
    return launch_contract<T, OT, pb, pb, true>(P, vdtype, ia, ib, Ap, Bp, brows, p, p, out,    \
                                                ldo, part, s);
  BKS_TRI(2) BKS_TRI(3) BKS_TRI(4) BKS_TRI(5) BKS_TRI(8)
#undef BKS_TRI
  return fail(BKS_EUNSUPPORTED, "contraction bucket not instantiated");
}

}  // namespace bks
