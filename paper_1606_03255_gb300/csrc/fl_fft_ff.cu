// fl_fft_ff.cu -- the four-step FFT passes of the band grids in float pairs
// (the FP64-accuracy form FL_FP64_FF: the forward transform, and the
// adjoint's sign -1 transform of the spread grids), compiled as their own
// translation unit.
#include "fl_fft.cuh"

namespace fl {

template cudaError_t launch_pass1<ff, 1, 0, false>(FL_P1_SIG(ff));
template cudaError_t launch_pass2<ff, 1>(FL_P2_SIG(ff));
template cudaError_t launch_pass1<ff, -1, 1, false>(FL_P1_SIG(ff));
template cudaError_t launch_pass2<ff, -1>(FL_P2_SIG(ff));

}  // namespace fl
