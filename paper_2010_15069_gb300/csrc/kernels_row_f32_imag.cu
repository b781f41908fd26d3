// Imaginary-time row-pass kernels instantiated for float (complex64): opening,
// pass B and the final rescale.
#include "launch_row.cuh"

namespace spgpe {
SPGPE_INSTANTIATE_ROW_FLAG(float, kImagFirst)
SPGPE_INSTANTIATE_ROW_FLAG(float, kImagB)
SPGPE_INSTANTIATE_ROW_FLAG(float, kImagScale)
}  // namespace spgpe
