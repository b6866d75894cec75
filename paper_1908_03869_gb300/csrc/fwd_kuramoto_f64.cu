// Forward kernel instantiations: Kuramoto models, double.
#include "em_forward_impl.cuh"

namespace sdeb {

cudaError_t launch_forward_kuramoto_f64(const ForwardArgs &a, Layout l, cudaStream_t s) {
    if (a.model == kKuramoto) return dispatch_tuning_layouts<KuramotoScalarLane, double>(a, l, s);
    if (a.model == kKuramotoPaper) return dispatch_default_layouts<KuramotoPaperLane, double>(a, l, s);
    return cudaErrorNotSupported;
}

}  // namespace sdeb
