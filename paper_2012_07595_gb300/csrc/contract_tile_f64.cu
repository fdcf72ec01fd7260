// Contraction tile kernels: FP64 arithmetic, FP64 output.
#include "contract_tile_impl.cuh"

namespace bks {
template int dispatch<double, double>(const Part&, int, const int32_t*, const int32_t*, const double*,
                                 int, const double*, int, int64_t, bool, int, int, double*, int64_t,
                                 cudaStream_t, double*);
}  // namespace bks
