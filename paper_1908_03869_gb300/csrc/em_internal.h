// Internal launch descriptors shared by the C-ABI layer and the kernel
// translation units.  Host-only declarations; no device code.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "em_device.cuh"
#include "sdeb.h"

namespace sdeb {

// The step-scheme flags of sdeb_problem.flags; at most one may be set.
constexpr uint32_t kImplicitFlags = SDEB_FLAG_IMPLICIT_EULER | SDEB_FLAG_IMPLICIT_MIDPOINT;
constexpr uint32_t kSchemeFlags = SDEB_FLAG_MILSTEIN | SDEB_FLAG_RK4 | kImplicitFlags;
inline bool scheme_flags_valid(uint32_t flags) {
    const uint32_t f = flags & kSchemeFlags;
    return (f & (f - 1u)) == 0u;
}
// ForwardArgs::implicit of the flags: 1 implicit Euler, 2 implicit midpoint, 0 neither.
inline int32_t implicit_kind(uint32_t flags) {
    return (flags & SDEB_FLAG_IMPLICIT_EULER) ? 1 : (flags & SDEB_FLAG_IMPLICIT_MIDPOINT) ? 2 : 0;
}

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
    int32_t milstein;  // 1: Milstein step (models with multiplicative noise), 0: Euler-Maruyama
    int32_t rk4;       // 1: fourth-order Runge-Kutta on the drift alone (launch_forward_rk4_*)
    int32_t implicit;  // 1: implicit Euler, 2: implicit midpoint on the drift alone (launch_forward_implicit_*)
    int32_t final_value;  // 1: leave the state's value x - c in x at k_end (no later resume)
    int64_t nckpt;         // checkpoints in ckpt
    unsigned long long *check;  // bounds-check status word (checked build), or null
};

// The checked build's device status word on the current device (null in the
// unchecked build, which compiles no checks).  checked.cu.
unsigned long long *check_word();

// True when the forward kernel of a problem keeps its FP32 phase states with
// the compensation folded in every kCompPeriod steps: x alone is then not the
// state's value between periods (sdeb_read_final returns x - c).
inline bool delayed_compensation(int32_t model, int32_t precision, uint32_t flags) {
    return precision == SDEB_FP32_KAHAN && (model == kKuramoto || model == kKuramotoPaper) &&
           !(flags & (SDEB_FLAG_RK4 | SDEB_FLAG_IMPLICIT_EULER | SDEB_FLAG_IMPLICIT_MIDPOINT));
}
// dst[i] = x[i] - comp[i] (FP32), count elements, on the stream (aux_kernels.cu).
cudaError_t launch_state_value(const float *x, const float *comp, int64_t count, float *dst, cudaStream_t s);

// Returns cudaSuccess or the launch error; cudaErrorNotSupported when the
// (model, precision, layout) combination has no instantiation.
cudaError_t launch_forward_kuramoto_f32(const ForwardArgs &a, Layout l, cudaStream_t s);
cudaError_t launch_forward_kuramoto_f64(const ForwardArgs &a, Layout l, cudaStream_t s);
cudaError_t launch_forward_other_f32(const ForwardArgs &a, Layout l, cudaStream_t s);
cudaError_t launch_forward_other_f64(const ForwardArgs &a, Layout l, cudaStream_t s);
cudaError_t launch_forward_rk4_f32(const ForwardArgs &a, Layout l, cudaStream_t s);
cudaError_t launch_forward_rk4_f64(const ForwardArgs &a, Layout l, cudaStream_t s);
cudaError_t launch_forward_implicit_f32(const ForwardArgs &a, Layout l, cudaStream_t s);
cudaError_t launch_forward_implicit_f64(const ForwardArgs &a, Layout l, cudaStream_t s);

// The forward launch of a problem: Runge-Kutta, implicit, phase models or the others.
inline cudaError_t launch_forward_any(const ForwardArgs &a, Layout l, bool fp64, cudaStream_t s) {
    if (a.rk4) return fp64 ? launch_forward_rk4_f64(a, l, s) : launch_forward_rk4_f32(a, l, s);
    if (a.implicit) return fp64 ? launch_forward_implicit_f64(a, l, s) : launch_forward_implicit_f32(a, l, s);
    const bool phase = a.model == kKuramoto || a.model == kKuramotoPaper;
    if (phase) return fp64 ? launch_forward_kuramoto_f64(a, l, s) : launch_forward_kuramoto_f32(a, l, s);
    return fp64 ? launch_forward_other_f64(a, l, s) : launch_forward_other_f32(a, l, s);
}

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
    int64_t nckpt;             // checkpoints in ckpt
    unsigned long long *check; // bounds-check status word (checked build), or null
    int32_t records;           // SDEB_RECORDS_*: where the replay keeps a segment's records
};

cudaError_t launch_adjoint(const AdjointArgs &a, Layout l, bool fp64, cudaStream_t s);
// out[q] = sum over orbits of in[o][q], in a fixed order (deterministic).
cudaError_t launch_sum_over_orbits(const void *in, int64_t orbits, int32_t d, bool fp64, void *out,
                                   cudaStream_t s);

// ---- Batched heterogeneous instances ------------------------------------
// Every problem of a batch is an "instance" with its own n, steps, dt,
// stride, orbits and buffers (concatenated); an "item" is one orbit of one
// instance.  The persistent kernel's blocks (four warps) pull tasks from a
// queue sorted longest-first: one item on all 128 lanes of the block, two
// items on 64 lanes each (sums exchanged through shared memory), or four
// warps.  A packed warp holds several items side by side, each on
// ceil(units / P) consecutive lanes (P = 8 or 4 units per lane), items of
// similar step counts; an item's coupling sums are a segmented scan over
// its own lanes.  A single-warp item (at most 64 units, 2 per lane) has the
// warp to itself and sums with one redux.  Long items get fewer units per
// lane (teams, single-warp items), so the longest sequential chains are
// spread over more lanes.
struct BatchInstance {
    int32_t n, units, d;
    int32_t param_stride;          // d, or 0 when the instance shares one parameter vector
    uint32_t steps, stride, orbit_offset, has_frames;
    int64_t orbits;
    int64_t x_off, p_off, f_off;   // element offsets into the concatenated buffers
    int64_t o_off;                 // offset of the instance's first orbit among all items (flags)
    double dt;
};

struct BatchItem {
    int32_t instance;
    int32_t orbit;                 // orbit within the instance
};

struct BatchWarpTask {
    int16_t p;                     // units per lane: 8 or 4 (packed), 2 (one item alone on the warp)
    int16_t count;                 // items in the warp, in lane order; 0 = idle warp
    int32_t first;                 // first item index
    uint32_t kmax;                 // largest step count among the warp's items
};

enum : int32_t { kBatchWarps = 0, kBatchTeam128 = 1, kBatchTeam64 = 2 };

struct BatchTask {
    int32_t kind;                  // kBatchWarps, kBatchTeam128 or kBatchTeam64
    int32_t team_p;                // units per lane of team items (2 or 4)
    int32_t item[2];               // team items (item[1] < 0: none)
    BatchWarpTask warp[4];
};

constexpr int kBatchBlock = 128;   // threads per block of the batch kernel

struct BatchArgs {
    const BatchInstance *inst;
    const BatchItem *items;
    const BatchTask *tasks;
    int32_t ntasks;
    int *head;                     // queue position, zeroed before each launch
    const void *params;
    void *x;
    float *comp;
    void *frames;                  // nullptr: no frames (tuning runs)
    uint8_t *flags;
    PhiloxKeys keys;
    // extents for the checked build's bounds checks
    int32_t ninst;
    int64_t nitems, state_elems, frame_elems, param_elems;
    unsigned long long *check;
};

cudaError_t launch_batch(const BatchArgs &a, int grid, bool fp64, cudaStream_t s);
// Blocks of the batch kernel resident per SM (occupancy of its launch bounds).
int batch_blocks_per_sm(bool fp64);

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

// ---- Ensemble moments of stored frames (moments.cu) ------------------------
// Orbits per chunk of the FP64 moment accumulation: fixed, so a frame's bits
// do not depend on the frame range of a call.
constexpr int64_t kMomChunk = 4096;

struct FrameMomentsPlan {
    int chunks = 1;               // ceil(orbits / kMomChunk)
    int64_t frames_per_pass = 1;  // frames whose partials fit the scratch at once
    size_t partial_bytes = 0;     // scratch for one pass's partials
    size_t out_bytes = 0;         // one pass's results ([frames][n][2] + [frames][2] doubles)
};
FrameMomentsPlan frame_moments_plan(int64_t orbits, int n, int64_t count);
// Moments of frames [f0, f0 + count) (count <= plan.frames_per_pass) of a
// [F][orbits][n] frame buffer: state_out [count][n][2] = (mean, variance) of
// every component over the orbits, r_out [count][2] = (mean, variance) of
// the order parameter of Eq. 7; either may be nullptr.  partial: device
// scratch of plan.partial_bytes.
cudaError_t launch_frame_moments_pass(const void *frames, bool fp64, int64_t orbits, int n, int64_t f0,
                                      int64_t count, int64_t nframes, const FrameMomentsPlan &plan, void *partial,
                                      double *state_out, double *r_out, cudaStream_t s);

// Auxiliary kernels (aux_kernels.cu).
cudaError_t launch_philox_fill(uint64_t seed, uint32_t k0, int64_t nk, uint32_t b0, int64_t nb,
                               uint32_t o0, int64_t no, uint32_t stream_id, uint32_t *out,
                               cudaStream_t s);
cudaError_t launch_normals_fill(uint64_t seed, uint32_t k0, int64_t nk, uint32_t o0, int64_t no,
                                int32_t m, bool fp64, void *out, cudaStream_t s);
cudaError_t launch_order_param(const void *theta, int64_t orbits, int32_t n, bool fp64, void *r,
                               void *dr, cudaStream_t s);

}  // namespace sdeb
