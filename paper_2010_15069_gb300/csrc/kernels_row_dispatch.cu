// Dispatch of the row pass on its flag combination; the kernels themselves
// are instantiated per flag group in the kernels_row_*.cu units.
#include "internal.h"

namespace spgpe {

template <class T> cudaError_t launch_row(int flags, RowArgs a, cudaStream_t st) {
  switch (flags) {
    case kRealFirst: return launch_row_f<T, kRealFirst>(a, st);
    case kRealMid: return launch_row_f<T, kRealMid>(a, st);
    case kRealLast: return launch_row_f<T, kRealLast>(a, st);
    case kImagFirst: return launch_row_f<T, kImagFirst>(a, st);
    case kImagB: return launch_row_f<T, kImagB>(a, st);
    case kImagA: return launch_row_f<T, kImagA>(a, st);
    case kImagScale: return launch_row_f<T, kImagScale>(a, st);
    case kImagLag: return launch_row_f<T, kImagLag>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

template <class T> cudaError_t launch_row_p(int flags, RowArgs a, cudaStream_t st, int sms) {
  switch (flags) {
    case kRealFirst: return launch_row_pf<T, kRealFirst>(a, st, sms);
    case kRealMid: return launch_row_pf<T, kRealMid>(a, st, sms);
    case kRealLast: return launch_row_pf<T, kRealLast>(a, st, sms);
    case kImagFirst: return launch_row_pf<T, kImagFirst>(a, st, sms);
    case kImagB: return launch_row_pf<T, kImagB>(a, st, sms);
    case kImagA: return launch_row_pf<T, kImagA>(a, st, sms);
    case kImagScale: return launch_row_pf<T, kImagScale>(a, st, sms);
    case kImagLag: return launch_row_pf<T, kImagLag>(a, st, sms);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_row<float>(int, RowArgs, cudaStream_t);
template cudaError_t launch_row<double>(int, RowArgs, cudaStream_t);
template cudaError_t launch_row_p<float>(int, RowArgs, cudaStream_t, int);
template cudaError_t launch_row_p<double>(int, RowArgs, cudaStream_t, int);

}  // namespace spgpe
