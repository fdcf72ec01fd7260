// Contraction tile kernels: FP32 arithmetic, FP64 output.
#include "contract_tile_impl.cuh"

namespace bks {
template int dispatch<float, double>(const Part&, int, const int32_t*, const int32_t*, const float*,
                                 int, const float*, int, int64_t, bool, int, int, double*, int64_t,
                                 cudaStream_t, float*);
}  // namespace bks
