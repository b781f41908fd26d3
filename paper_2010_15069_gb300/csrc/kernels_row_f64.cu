// Row-pass kernels instantiated for double (complex128).
#include "launch_row.cuh"

namespace spgpe {
SPGPE_INSTANTIATE_ROW(double)
}  // namespace spgpe
