// Declarations shared by the contraction front end (contract.cu) and the
// tile kernels (contract_tile_impl.cuh, instantiated per arithmetic type in
// contract_tile_f32.cu, contract_tile_f32d.cu and contract_tile_f64.cu, so
// that the three compile in parallel).
#pragma once
#include <algorithm>

#include "common.cuh"

namespace bks {

namespace {

// Row stride of a packed operand of (bucket) width N: FP32 rows are padded
// to 2, 4 or 8 values so that a row is one or two aligned vector loads (a
// 3-wide row is one float4, a 5-wide row one float4 and one float); FP64
// rows keep 3 and 5 values (those kernels are bound by the FP64 pipe, not
// by loads).
template <typename T, int N>
struct RowStride {
  static constexpr int v = sizeof(T) == 4 ? (N <= 2 ? 2 : N <= 4 ? 4 : 8) : N;
};
template <typename T> inline int row_stride(int N) {
  return sizeof(T) == 4 ? (N <= 2 ? 2 : N <= 4 ? 4 : 8) : N;
}

inline int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)num_sms() * 32));
}


template <typename T> const T* values_of(const Part& P, int vdtype);
template <typename T> const T* sell_values_of(const Part& P);
template <> const float* sell_values_of<float>(const Part& P) { return P.sv32.as<float>(); }
template <> const double* sell_values_of<double>(const Part& P) { return P.sv64.as<double>(); }
// the interleaved copy of the index array `a` (c0 or c1 of P)
inline const int32_t* sell_of(const Part& P, const int32_t* a) {
  return a == P.c0.as<int32_t>() ? P.sc0.as<int32_t>() : P.sc1.as<int32_t>();
}
template <> const float* values_of<float>(const Part& P, int vdtype) {
  return vdtype == BKS_F32 ? P.v.as<float>() : P.v32.as<float>();
}
template <> const double* values_of<double>(const Part& P, int vdtype) {
  return vdtype == BKS_F64 ? P.v.as<double>() : P.v64.as<double>();
}

}  // namespace

// One contraction over a work plan (see contract_tile_impl.cuh): operand A
// (packed, width bucket PB) gathered by ia, operand B (packed, bucket QB,
// brows rows) by ib; tri: the upper triangle of A^T A per row.  Partial
// sums of cut rows go to `part` when given, else to a stream allocation.
template <typename T, typename OT>
int dispatch(const Part& P, int vdtype, const int32_t* ia, const int32_t* ib, const T* Ap,
             int PB, const T* Bp, int QB, int64_t brows, bool tri, int p, int q, OT* out,
             int64_t ldo, cudaStream_t s, T* part = nullptr);

}  // namespace bks
