// Forward kernel instantiations of the implicit Euler and implicit midpoint
// steps on the drift alone (the ODE path, theta chosen at run time), every
// model, double.
#include "em_forward_impl.cuh"

namespace sdeb {

cudaError_t launch_forward_implicit_f64(const ForwardArgs &a, Layout l, cudaStream_t s) {
    switch (a.model) {
    case kKuramoto: return dispatch_ode_layouts<KuramotoScalarLane, double, kSchemeImplicit>(a, l, s);
    case kKuramotoPaper: return dispatch_ode_layouts<KuramotoPaperLane, double, kSchemeImplicit>(a, l, s);
    case kFhnNet: return dispatch_ode_layouts<FhnEmLane, double, kSchemeImplicit>(a, l, s);
    case kOu: return dispatch_ode_layouts<OuLane, double, kSchemeImplicit>(a, l, s);
    case kGbm: return dispatch_ode_layouts<GbmLane, double, kSchemeImplicit>(a, l, s);
    case kLinearOde: return dispatch_ode_layouts<LinearLane, double, kSchemeImplicit>(a, l, s);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace sdeb
