// Column-pass, energy and reduction kernels instantiated for float (complex64).
#include "launch_col.cuh"

namespace spgpe {
SPGPE_INSTANTIATE_COL(float)
}  // namespace spgpe
