// Forward kernel instantiations: FitzHugh-Nagumo network, OU, GBM and the
// linear ODE, float.
#include "em_forward_impl.cuh"

namespace sdeb {

cudaError_t launch_forward_other_f32(const ForwardArgs &a, Layout l, cudaStream_t s) {
    switch (a.model) {
    case kFhnNet:
        return a.milstein ? dispatch_default_layouts<FhnMilsteinLane, float>(a, l, s)
                          : dispatch_default_layouts<FhnEmLane, float>(a, l, s);
    case kOu: return dispatch_default_layouts<OuLane, float>(a, l, s);
    case kGbm:
        return a.milstein ? dispatch_default_layouts<GbmMilsteinLane, float>(a, l, s)
                          : dispatch_default_layouts<GbmLane, float>(a, l, s);
    case kLinearOde: return dispatch_default_layouts<LinearLane, float>(a, l, s);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace sdeb
