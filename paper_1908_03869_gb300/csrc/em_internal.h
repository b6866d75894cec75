// Internal launch descriptors shared by the C-ABI layer and the kernel
// translation units.  Host-only declarations; no device code.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "em_device.cuh"

namespace sdeb {

enum ModelId : int32_t {
    kKuramoto = 1,
    kKuramotoPaper = 2,
    kFhnNet = 3,
    kOu = 4,
    kGbm = 5,
    kLinearOde = 6,
};

struct Layout {
    int G;  // lanes per orbit
    int P;  // units per lane
};

// Arguments of one forward launch (one precision; pointers are typed void*
// here and cast in the kernel translation unit).
struct ForwardArgs {
    int32_t model;
    int32_t n;        // state components per orbit
    int32_t units;    // Wiener channels / coupling units per orbit
    int64_t orbits;
    const void *params;
    int64_t param_stride;  // d, or 0 when every orbit shares one vector
    void *x;               // [orbits][n] state, updated in place
    float *comp;           // [orbits][n] Kahan compensation (FP32 only)
    void *frames;          // [F][orbits][n] or nullptr
    int64_t nframes;
    float *ckpt_comp;      // [C+1][orbits][n] compensation at checkpoints (FP32)
    void *ckpt;            // [C+1][orbits][n] state at checkpoints, or nullptr
    uint32_t ckpt_every;
    uint32_t k_begin, k_end, stride;
    uint32_t orbit_offset;
    double dt;
    uint8_t *flags;  // [orbits]
    PhiloxKeys keys;
};

// Returns cudaSuccess or the launch error; cudaErrorNotSupported when the
// (model, precision, layout) combination has no instantiation.
cudaError_t launch_forward_kuramoto_f32(const ForwardArgs &a, Layout l, cudaStream_t s);
cudaError_t launch_forward_kuramoto_f64(const ForwardArgs &a, Layout l, cudaStream_t s);
cudaError_t launch_forward_other_f32(const ForwardArgs &a, Layout l, cudaStream_t s);
cudaError_t launch_forward_other_f64(const ForwardArgs &a, Layout l, cudaStream_t s);

// Arguments of the discrete-adjoint launch (Kuramoto models).
struct AdjointArgs {
    int32_t model;
    int32_t n, units, d;
    int64_t orbits;
    const void *params;
    int64_t param_stride;
    const void *ckpt;          // [C+1][orbits][n], checkpoint c = state at step c*ckpt_every
    const float *ckpt_comp;    // FP32 compensation at the checkpoints
    uint32_t ckpt_every, steps;
    uint32_t orbit_offset;
    double dt;
    void *seg;                 // [ckpt_every][orbits][2n] replayed phases and normals (scratch)
    const void *dL_dxK;        // [orbits][n]
    void *dL_dp;               // [orbits][d]
    void *dL_dx0;              // [orbits][n] or nullptr
    PhiloxKeys keys;
};

cudaError_t launch_adjoint(const AdjointArgs &a, Layout l, bool fp64, cudaStream_t s);
// out[q] = sum over orbits of in[o][q], in a fixed order (deterministic).
cudaError_t launch_sum_over_orbits(const void *in, int64_t orbits, int32_t d, bool fp64, void *out,
                                   cudaStream_t s);

// Default layout for a number of units (smallest lane group holding them).
inline bool default_layout(int units, Layout &l) {
    if (units <= 1) l = {1, 1};
    else if (units <= 2) l = {1, 2};
    else if (units <= 4) l = {1, 4};
    else if (units <= 8) l = {1, 8};
    else if (units <= 16) l = {2, 8};
    else if (units <= 32) l = {4, 8};
    else if (units <= 64) l = {8, 8};
    else if (units <= 128) l = {16, 8};
    else if (units <= 256) l = {32, 8};
    else return false;
    return true;
}

// Auxiliary kernels (aux_kernels.cu).
cudaError_t launch_philox_fill(uint64_t seed, uint32_t k0, int64_t nk, uint32_t b0, int64_t nb,
                               uint32_t o0, int64_t no, uint32_t stream_id, uint32_t *out,
                               cudaStream_t s);
cudaError_t launch_normals_fill(uint64_t seed, uint32_t k0, int64_t nk, uint32_t o0, int64_t no,
                                int32_t m, bool fp64, void *out, cudaStream_t s);
cudaError_t launch_order_param(const void *theta, int64_t orbits, int32_t n, bool fp64, void *r,
                               void *dr, cudaStream_t s);

}  // namespace sdeb
