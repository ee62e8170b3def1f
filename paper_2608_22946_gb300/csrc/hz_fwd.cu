// Explicit instantiations of the forward stencil (hz_fwd.cuh), split by
// (precision, mode) so that the build compiles the parts in parallel: this
// file is compiled once per part with -DHZ_FWD_PART=0..5.
#include "hz_fwd_launch.cuh"

#ifndef HZ_FWD_PART
#error "compile with -DHZ_FWD_PART=<0..5>"
#endif

namespace hz {

#define HZ_FWD_INST(R, MODE)                                                     \
  template void launch_fwd<R, MODE>(const StencilCall<R>&, int, cudaStream_t); \
  template void fwd_init_attrs<R, MODE>();

#if HZ_FWD_PART == 0
HZ_FWD_INST(float, M_APPLY)
#elif HZ_FWD_PART == 1
HZ_FWD_INST(float, M_RESID)
#elif HZ_FWD_PART == 2
HZ_FWD_INST(float, M_J2)
#elif HZ_FWD_PART == 3
HZ_FWD_INST(float, M_JSWEEP)
#elif HZ_FWD_PART == 4
HZ_FWD_INST(double, M_APPLY)
HZ_FWD_INST(double, M_RESID)
HZ_FWD_INST(double, M_J2)
HZ_FWD_INST(double, M_JSWEEP)
#elif HZ_FWD_PART == 5
HZ_FWD_INST(float, M_AWIN)
HZ_FWD_INST(double, M_AWIN)
#endif

#undef HZ_FWD_INST

}  // namespace hz
