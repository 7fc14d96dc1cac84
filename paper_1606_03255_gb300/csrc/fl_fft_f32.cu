// fl_fft_f32.cu -- the four-step FFT passes of the band grids in float
// (instantiations of fl_fft.cuh, compiled as their own translation unit).
#include "fl_fft.cuh"

namespace fl {

template cudaError_t launch_pass1<float, 1, 0, false>(FL_P1_SIG(float));
template cudaError_t launch_pass1<float, 1, 0, true>(FL_P1_SIG(float));
template cudaError_t launch_pass1<float, -1, 1, false>(FL_P1_SIG(float));
template cudaError_t launch_pass1<float, 1, 1, false>(FL_P1_SIG(float));
template cudaError_t launch_pass2<float, 1>(FL_P2_SIG(float));
template cudaError_t launch_pass2<float, -1>(FL_P2_SIG(float));

}  // namespace fl
