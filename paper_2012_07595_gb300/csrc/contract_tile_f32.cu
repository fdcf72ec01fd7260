// Contraction tile kernels: FP32 arithmetic, FP32 output.
#include "contract_tile_impl.cuh"

namespace bks {
template int dispatch<float, float>(const Part&, int, const int32_t*, const int32_t*, const float*,
                                 int, const float*, int, int64_t, bool, int, int, float*, int64_t,
                                 cudaStream_t, float*);
}  // namespace bks
