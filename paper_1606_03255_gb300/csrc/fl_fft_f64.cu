// fl_fft_f64.cu -- the four-step FFT passes of the band grids in double
// (instantiations of fl_fft.cuh, compiled as their own translation unit).
#include "fl_fft.cuh"

namespace fl {

template cudaError_t launch_pass1<double, 1, 0, false>(const BandDev&, int, int, int, int,
                                                  const C_t<double>*, const double*, const C_t<double>*,
                                                  C_t<double>*, cudaStream_t);
template cudaError_t launch_pass1<double, 1, 0, true>(const BandDev&, int, int, int, int,
                                                 const C_t<double>*, const double*, const C_t<double>*,
                                                 C_t<double>*, cudaStream_t);
template cudaError_t launch_pass1<double, -1, 1, false>(const BandDev&, int, int, int, int,
                                                   const C_t<double>*, const double*, const C_t<double>*,
                                                   C_t<double>*, cudaStream_t);
template cudaError_t launch_pass2<double, 1>(const BandDev&, int, int, int, int, const C_t<double>*,
                                        C_t<double>*, cudaStream_t);
template cudaError_t launch_pass2<double, -1>(const BandDev&, int, int, int, int, const C_t<double>*,
                                         C_t<double>*, cudaStream_t);

}  // namespace fl
