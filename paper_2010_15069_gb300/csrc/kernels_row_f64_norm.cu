// Imaginary-time row-pass kernels with atom-number partials instantiated for
// double (complex128): pass A and the lagged pass.
#include "launch_row.cuh"

namespace spgpe {
SPGPE_INSTANTIATE_ROW_FLAG(double, kImagA)
SPGPE_INSTANTIATE_ROW_FLAG(double, kImagLag)
}  // namespace spgpe
