// Row-pass kernels instantiated for float (complex64).
#include "launch_row.cuh"

namespace spgpe {
SPGPE_INSTANTIATE_ROW(float)
}  // namespace spgpe
