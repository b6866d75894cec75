// Forward kernel instantiations: FitzHugh-Nagumo network, OU, GBM and the
// linear ODE, double.
#include "em_forward_impl.cuh"

namespace sdeb {

cudaError_t launch_forward_other_f64(const ForwardArgs &a, Layout l, cudaStream_t s) {
    switch (a.model) {
    case kFhnNet:
        return a.milstein ? dispatch_default_layouts<FhnMilsteinLane, double>(a, l, s)
                          : dispatch_default_layouts<FhnEmLane, double>(a, l, s);
    case kOu: return dispatch_default_layouts<OuLane, double>(a, l, s);
    case kGbm:
        return a.milstein ? dispatch_default_layouts<GbmMilsteinLane, double>(a, l, s)
                          : dispatch_default_layouts<GbmLane, double>(a, l, s);
    case kLinearOde: return dispatch_default_layouts<LinearLane, double>(a, l, s);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace sdeb
