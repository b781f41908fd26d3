// Column-pass, energy and reduction kernels instantiated for double (complex128).
#include "launch_col.cuh"

namespace spgpe {
SPGPE_INSTANTIATE_COL(double)
}  // namespace spgpe
