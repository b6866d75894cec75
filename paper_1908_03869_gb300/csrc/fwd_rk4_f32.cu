// Forward kernel instantiations of the classical fourth-order Runge-Kutta
// step on the drift alone (the ODE path), every model, float.
#include "em_forward_impl.cuh"

namespace sdeb {

cudaError_t launch_forward_rk4_f32(const ForwardArgs &a, Layout l, cudaStream_t s) {
    switch (a.model) {
    case kKuramoto: return dispatch_ode_layouts<KuramotoScalarLane, float, kSchemeRk4>(a, l, s);
    case kKuramotoPaper: return dispatch_ode_layouts<KuramotoPaperLane, float, kSchemeRk4>(a, l, s);
    case kFhnNet: return dispatch_ode_layouts<FhnEmLane, float, kSchemeRk4>(a, l, s);
    case kOu: return dispatch_ode_layouts<OuLane, float, kSchemeRk4>(a, l, s);
    case kGbm: return dispatch_ode_layouts<GbmLane, float, kSchemeRk4>(a, l, s);
    case kLinearOde: return dispatch_ode_layouts<LinearLane, float, kSchemeRk4>(a, l, s);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace sdeb
