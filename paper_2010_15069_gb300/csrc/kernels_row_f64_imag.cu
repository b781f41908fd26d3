// Imaginary-time row-pass kernels instantiated for double (complex128): opening,
// pass B and the final rescale.
#include "launch_row.cuh"

namespace spgpe {
SPGPE_INSTANTIATE_ROW_FLAG(double, kImagFirst)
SPGPE_INSTANTIATE_ROW_FLAG(double, kImagB)
SPGPE_INSTANTIATE_ROW_FLAG(double, kImagScale)
}  // namespace spgpe
