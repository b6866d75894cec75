// Forward kernel instantiations of the implicit Euler and implicit midpoint
// steps on the drift alone (the ODE path, theta chosen at run time), every
// model, float.
#include "em_forward_impl.cuh"

namespace sdeb {

cudaError_t launch_forward_implicit_f32(const ForwardArgs &a, Layout l, cudaStream_t s) {
    switch (a.model) {
    case kKuramoto: return dispatch_ode_layouts<KuramotoScalarLane, float, kSchemeImplicit>(a, l, s);
    case kKuramotoPaper: return dispatch_ode_layouts<KuramotoPaperLane, float, kSchemeImplicit>(a, l, s);
    case kFhnNet: return dispatch_ode_layouts<FhnEmLane, float, kSchemeImplicit>(a, l, s);
    case kOu: return dispatch_ode_layouts<OuLane, float, kSchemeImplicit>(a, l, s);
    case kGbm: return dispatch_ode_layouts<GbmLane, float, kSchemeImplicit>(a, l, s);
    case kLinearOde: return dispatch_ode_layouts<LinearLane, float, kSchemeImplicit>(a, l, s);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace sdeb
