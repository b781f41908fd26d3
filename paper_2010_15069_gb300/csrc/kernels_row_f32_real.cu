// Real-time row-pass kernels instantiated for float (complex64).
#include "launch_row.cuh"

namespace spgpe {
SPGPE_INSTANTIATE_ROW_SHAPE(float)
SPGPE_INSTANTIATE_ROW_FLAG(float, kRealFirst)
SPGPE_INSTANTIATE_ROW_FLAG(float, kRealMid)
SPGPE_INSTANTIATE_ROW_FLAG(float, kRealLast)
}  // namespace spgpe
