// Forward kernel instantiations of the classical fourth-order Runge-Kutta
// step on the drift alone (the ODE path), every model, float.
#include "em_forward_impl.cuh"

namespace sdeb {

cudaError_t launch_forward_rk4_f32(const ForwardArgs &a, Layout l, cudaStream_t s) {
    switch (a.model) {
    case kKuramoto: return dispatch_rk4_layouts<KuramotoScalarLane, float>(a, l, s);
    case kKuramotoPaper: return dispatch_rk4_layouts<KuramotoPaperLane, float>(a, l, s);
    case kFhnNet: return dispatch_rk4_layouts<FhnEmLane, float>(a, l, s);
    case kOu: return dispatch_rk4_layouts<OuLane, float>(a, l, s);
    case kGbm: return dispatch_rk4_layouts<GbmLane, float>(a, l, s);
    case kLinearOde: return dispatch_rk4_layouts<LinearLane, float>(a, l, s);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace sdeb
