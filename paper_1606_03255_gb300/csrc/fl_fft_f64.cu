// fl_fft_f64.cu -- the four-step FFT passes of the band grids in double
// (instantiations of fl_fft.cuh, compiled as their own translation unit).
#include "fl_fft.cuh"

namespace fl {

template cudaError_t launch_pass1<double, 1, 0, false>(FL_P1_SIG(double));
template cudaError_t launch_pass1<double, 1, 0, true>(FL_P1_SIG(double));
template cudaError_t launch_pass1<double, -1, 1, false>(FL_P1_SIG(double));
template cudaError_t launch_pass1<double, 1, 1, false>(FL_P1_SIG(double));
template cudaError_t launch_pass2<double, 1>(FL_P2_SIG(double));
template cudaError_t launch_pass2<double, -1>(FL_P2_SIG(double));

}  // namespace fl
