// fl_fft_f32.cu -- the four-step FFT passes of the band grids in float
// (instantiations of fl_fft.cuh, compiled as their own translation unit).
#include "fl_fft.cuh"

namespace fl {

template cudaError_t launch_pass1<float, 1, 0, false>(const BandDev&, int, int, int, int,
                                                  const C_t<float>*, const float*, const C_t<float>*,
                                                  C_t<float>*, cudaStream_t);
template cudaError_t launch_pass1<float, 1, 0, true>(const BandDev&, int, int, int, int,
                                                 const C_t<float>*, const float*, const C_t<float>*,
                                                 C_t<float>*, cudaStream_t);
template cudaError_t launch_pass1<float, -1, 1, false>(const BandDev&, int, int, int, int,
                                                   const C_t<float>*, const float*, const C_t<float>*,
                                                   C_t<float>*, cudaStream_t);
template cudaError_t launch_pass2<float, 1>(const BandDev&, int, int, int, int, const C_t<float>*,
                                        C_t<float>*, cudaStream_t);
template cudaError_t launch_pass2<float, -1>(const BandDev&, int, int, int, int, const C_t<float>*,
                                         C_t<float>*, cudaStream_t);

}  // namespace fl
