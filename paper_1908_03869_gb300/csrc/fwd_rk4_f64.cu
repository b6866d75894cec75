// Forward kernel instantiations of the classical fourth-order Runge-Kutta
// step on the drift alone (the ODE path), every model, double.
#include "em_forward_impl.cuh"

namespace sdeb {

cudaError_t launch_forward_rk4_f64(const ForwardArgs &a, Layout l, cudaStream_t s) {
    switch (a.model) {
    case kKuramoto: return dispatch_ode_layouts<KuramotoScalarLane, double, kSchemeRk4>(a, l, s);
    case kKuramotoPaper: return dispatch_ode_layouts<KuramotoPaperLane, double, kSchemeRk4>(a, l, s);
    case kFhnNet: return dispatch_ode_layouts<FhnEmLane, double, kSchemeRk4>(a, l, s);
    case kOu: return dispatch_ode_layouts<OuLane, double, kSchemeRk4>(a, l, s);
    case kGbm: return dispatch_ode_layouts<GbmLane, double, kSchemeRk4>(a, l, s);
    case kLinearOde: return dispatch_ode_layouts<LinearLane, double, kSchemeRk4>(a, l, s);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace sdeb
