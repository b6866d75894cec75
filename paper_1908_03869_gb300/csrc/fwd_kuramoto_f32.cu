// Forward kernel instantiations: Kuramoto models, float.
#include "em_forward_impl.cuh"

namespace sdeb {

cudaError_t launch_forward_kuramoto_f32(const ForwardArgs &a, Layout l, cudaStream_t s) {
    if (a.model == kKuramoto) return dispatch_tuning_layouts<KuramotoScalarLane, float>(a, l, s);
    if (a.model == kKuramotoPaper) return dispatch_default_layouts<KuramotoPaperLane, float>(a, l, s);
    return cudaErrorNotSupported;
}

}  // namespace sdeb
