// Imaginary-time row-pass kernels with atom-number partials instantiated for
// float (complex64): pass A and the lagged pass.
#include "launch_row.cuh"

namespace spgpe {
SPGPE_INSTANTIATE_ROW_FLAG(float, kImagA)
SPGPE_INSTANTIATE_ROW_FLAG(float, kImagLag)
}  // namespace spgpe
