// fl_small_fft.cu -- the FFTs of the band grids of at most 4096 points (one CTA
// per work item; fl_fft.cuh), instantiated in their own translation unit.
#include "fl_fft.cuh"

namespace fl {

#define FL_SMALL_INST(T)                                                        \
    template cudaError_t launch_small_fft<T, 1, 0, false>(FL_SMALL_SIG(T));     \
    template cudaError_t launch_small_fft<T, 1, 0, true>(FL_SMALL_SIG(T));      \
    template cudaError_t launch_small_fft<T, -1, 1, false>(FL_SMALL_SIG(T));    \
    template cudaError_t launch_small_fft<T, 1, 1, false>(FL_SMALL_SIG(T));
FL_SMALL_INST(float)
FL_SMALL_INST(double)
#undef FL_SMALL_INST
template cudaError_t launch_small_fft<ff, 1, 0, false>(FL_SMALL_SIG(ff));
template cudaError_t launch_small_fft<ff, -1, 1, false>(FL_SMALL_SIG(ff));

}  // namespace fl
