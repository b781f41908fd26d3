// Real-time row-pass kernels instantiated for double (complex128).
#include "launch_row.cuh"

namespace spgpe {
SPGPE_INSTANTIATE_ROW_SHAPE(double)
SPGPE_INSTANTIATE_ROW_FLAG(double, kRealFirst)
SPGPE_INSTANTIATE_ROW_FLAG(double, kRealMid)
SPGPE_INSTANTIATE_ROW_FLAG(double, kRealLast)
}  // namespace spgpe
