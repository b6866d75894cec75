// Forward kernel instantiations of the classical fourth-order Runge-Kutta
// step on the drift alone (the ODE path), every model, double.
#include "em_forward_impl.cuh"

namespace sdeb {

cudaError_t launch_forward_rk4_f64(const ForwardArgs &a, Layout l, cudaStream_t s) {
    switch (a.model) {
    case kKuramoto: return dispatch_rk4_layouts<KuramotoScalarLane, double>(a, l, s);
    case kKuramotoPaper: return dispatch_rk4_layouts<KuramotoPaperLane, double>(a, l, s);
    case kFhnNet: return dispatch_rk4_layouts<FhnEmLane, double>(a, l, s);
    case kOu: return dispatch_rk4_layouts<OuLane, double>(a, l, s);
    case kGbm: return dispatch_rk4_layouts<GbmLane, double>(a, l, s);
    case kLinearOde: return dispatch_rk4_layouts<LinearLane, double>(a, l, s);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace sdeb
