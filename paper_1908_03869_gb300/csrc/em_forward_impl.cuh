// Forward Euler-Maruyama kernel (Eq. 2) for the lane-group layout, with the
// Philox draw, Box-Muller, drift, diffusion, compensated update and strided
// output fused into one pass over the horizon.  Included by the translation
// units that instantiate it for a set of models, precisions and layouts.
#pragma once

#include <type_traits>

#include "em_internal.h"
#include "em_models.cuh"

namespace sdeb {

constexpr int kForwardBlock = 128;

// Loads / stores of a lane's units: component c of unit j is row[c*units + j].
// Full, 16-byte aligned runs use 16-byte vector accesses.
template <typename Real, int U, int P>
__device__ __forceinline__ void load_units(const Real *row, int units, int u0, Real (&v)[U][P]) {
    constexpr int kVec = 16 / sizeof(Real);
#pragma unroll
    for (int c = 0; c < U; ++c) {
        const Real *src = row + (int64_t)c * units + u0;
        if (P % kVec == 0 && u0 + P <= units && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
#pragma unroll
            for (int i = 0; i < P; i += kVec) {
                if (sizeof(Real) == 4) {
                    float4 q = *reinterpret_cast<const float4 *>(src + i);
                    v[c][i] = q.x; v[c][i + 1] = q.y; v[c][i + 2] = q.z; v[c][i + 3] = q.w;
                } else {
                    double2 q = *reinterpret_cast<const double2 *>(src + i);
                    v[c][i] = q.x; v[c][i + 1] = q.y;
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < P; ++i) v[c][i] = (u0 + i < units) ? src[i] : Real(0);
        }
    }
}

template <typename Real, int U, int P>
__device__ __forceinline__ void store_units(Real *row, int units, int u0, const Real (&v)[U][P]) {
    constexpr int kVec = 16 / sizeof(Real);
#pragma unroll
    for (int c = 0; c < U; ++c) {
        Real *dst = row + (int64_t)c * units + u0;
        if (P % kVec == 0 && u0 + P <= units && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
#pragma unroll
            for (int i = 0; i < P; i += kVec) {
                if (sizeof(Real) == 4) {
                    *reinterpret_cast<float4 *>(dst + i) =
                        make_float4(v[c][i], v[c][i + 1], v[c][i + 2], v[c][i + 3]);
                } else {
                    *reinterpret_cast<double2 *>(dst + i) = make_double2(v[c][i], v[c][i + 1]);
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < P; ++i)
                if (u0 + i < units) dst[i] = v[c][i];
        }
    }
}

// Coupling-sum reducers.  WarpGroupSum<G>: butterfly over the G lanes of an
// orbit inside one warp.  TeamSum<NW>: an orbit spread over the NW warps of
// the whole thread block -- warp butterflies, then the NW partial sums
// exchanged through shared memory (double-buffered, one barrier per call) and
// added in warp order, so every lane gets bit-identical totals.
template <int G>
struct WarpGroupSum {
    template <typename Real, int NR>
    __device__ __forceinline__ void operator()(Real (&r)[NR]) const {
#pragma unroll
        for (int q = 0; q < NR; ++q) r[q] = group_sum<G>(r[q]);
    }
};

template <int NW, typename Real>
struct TeamSum {
    Real *buf;  // shared memory, [2][NW][NRMAX]
    int flip;
    static constexpr int NRMAX = 2;
    template <int NR>
    __device__ __forceinline__ void operator()(Real (&r)[NR]) {
        static_assert(NR <= NRMAX, "TeamSum holds at most NRMAX sums");
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        Real *slot = buf + flip * NW * NRMAX;
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            r[q] = group_sum<32>(r[q]);
            if (lane == 0) slot[warp * NRMAX + q] = r[q];
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            Real t = slot[q];
#pragma unroll
            for (int w = 1; w < NW; ++w) t += slot[w * NRMAX + q];
            r[q] = t;
        }
        flip ^= 1;
    }
};

// The lane's fixed Philox words: round 1 of the noise counters (k, block,
// orbit, 0) of its blocks without k, formed once per launch.
template <int P>
struct NoiseLane {
    static constexpr int NB = P < 4 ? 1 : P / 4;
    PhiloxRound1 r1[NB];
    __device__ __forceinline__ NoiseLane(uint32_t orbit, int u0, const PhiloxKeys &keys) {
#pragma unroll
        for (int blk = 0; blk < NB; ++blk) r1[blk] = philox_round1_fixed((uint32_t)(u0 >> 2) + blk, orbit, keys);
    }
};

// Normal pairs of a step in polar form: the lane's P normals are
// N_i = amp[pair(i)] * trig[i], pair(i) = i / 2 (one pair when P < 4).  Per
// noise block one Philox call (counter (k, block, orbit, 0)) and two
// Box-Muller pairs.  A lane holding 1 or 2 units draws the block that
// contains them and transforms only the word pair that holds them (several
// lanes of a group draw the same block).
template <int P>
constexpr int kNoisePairs = P < 4 ? 1 : P / 2;

template <int P>
__device__ __forceinline__ constexpr int noise_pair(int i) { return P < 4 ? 0 : i / 2; }

template <typename Real, int P>
__device__ __forceinline__ void draw_noise(Real (&amp)[kNoisePairs<P>], Real (&trig)[P], uint32_t k, int u0,
                                           const NoiseLane<P> &nl, const PhiloxKeys &keys) {
    if constexpr (P < 4) {
        const U32x4 w = philox4x32_10_fixed(k, nl.r1[0], keys);
        const bool high = (u0 & 2) != 0;
        Real c, s;
        box_muller_polar<Real>(high ? w.z : w.x, high ? w.w : w.y, amp[0], c, s);
        trig[0] = (P == 1 && (u0 & 1)) ? s : c;
        if constexpr (P == 2) trig[1] = s;
    } else {
#pragma unroll
        for (int blk = 0; blk < P / 4; ++blk) {
            const U32x4 w = philox4x32_10_fixed(k, nl.r1[blk], keys);
            box_muller_polar<Real>(w.x, w.y, amp[2 * blk], trig[4 * blk], trig[4 * blk + 1]);
            box_muller_polar<Real>(w.z, w.w, amp[2 * blk + 1], trig[4 * blk + 2], trig[4 * blk + 3]);
        }
    }
}

// One step of Eq. 2 for the lane's units: the normals (they do not depend on
// the state, so they are drawn first and their latency overlaps the coupling
// sums), the coupling sums over the orbit's lanes (RED), and the compensated
// update of every unit.  Every unit's increment reads only the old state
// (synchronous update).  A model with one additive noise strength for all
// its units (kSplitNoise) takes each normal as amplitude times sine or
// cosine, scaled once per pair, so the normal's product folds into the
// increment's last fused multiply-add.  With RECORD the step's phases,
// normals and coupling sums go to rec (the adjoint's replay).
// What the adjoint's replay keeps of a step (phase models): the reduced
// phase and the normal of each unit, and the orbit's coupling sums C, S.
template <typename Real, int P>
struct StepRecord {
    Real phase[P];
    Real z[P];
    Real sums[2];
};

// The step of Eq. 2 given its normals in polar form (em_step draws them).
template <class M, typename Real, int P, bool RECORD = false, class RED>
__device__ __forceinline__ void em_step_noise(M &model, Real (&x)[M::U][P], Real (&cp)[M::U][P],
                                              Real (&amp)[kNoisePairs<P>], const Real (&trig)[P], int u0, int units,
                                              RED &reduce, StepRecord<Real, P> *rec = nullptr) {
    constexpr int NRA = M::NR > 0 ? M::NR : 1;
    Real red[NRA];
    model.prepare(x, cp, u0, units, red);
    if constexpr (M::NR > 0) reduce(red);
    if constexpr (RECORD) {
        rec->sums[0] = red[0];
        rec->sums[1] = red[1];
#pragma unroll
        for (int i = 0; i < P; ++i) rec->phase[i] = model.rph[i];
    }
    if constexpr (M::kSplitNoise) {
        Real amp_s[kNoisePairs<P>];
#pragma unroll
        for (int j = 0; j < kNoisePairs<P>; ++j) amp_s[j] = model.noise_scaled(amp[j]);  // includes bm_amp_unit
#pragma unroll
        for (int i = 0; i < P; ++i) {
            Real inc[M::U];
            model.incr_split(i, red, amp_s[noise_pair<P>(i)], trig[i], inc);
#pragma unroll
            for (int c = 0; c < M::U; ++c) {
                if constexpr (M::kDelayedComp) accumulate_delayed(x[c][i], cp[c][i], inc[c]);
                else accumulate(x[c][i], cp[c][i], inc[c]);
            }
            if constexpr (RECORD) rec->z[i] = mul_r(mul_r(amp[noise_pair<P>(i)], bm_amp_unit<Real>()), trig[i]);
        }
    } else {
#pragma unroll
        for (int j = 0; j < kNoisePairs<P>; ++j) amp[j] = mul_r(amp[j], bm_amp_unit<Real>());
#pragma unroll
        for (int i = 0; i < P; ++i) {
            const Real z = mul_r(amp[noise_pair<P>(i)], trig[i]);
            Real inc[M::U];
            model.incr(i, x, red, z, inc);
#pragma unroll
            for (int c = 0; c < M::U; ++c) {
                if constexpr (M::kDelayedComp) accumulate_delayed(x[c][i], cp[c][i], inc[c]);
                else accumulate(x[c][i], cp[c][i], inc[c]);
            }
            if constexpr (RECORD) rec->z[i] = z;
        }
    }
}

template <class M, typename Real, int P, bool RECORD = false, class RED>
__device__ __forceinline__ void em_step(M &model, Real (&x)[M::U][P], Real (&cp)[M::U][P], uint32_t k,
                                        const NoiseLane<P> &nl, int u0, int units, const PhiloxKeys &keys,
                                        RED &reduce, StepRecord<Real, P> *rec = nullptr) {
    static_assert(P == 1 || P == 2 || P % 4 == 0, "a lane holds 1, 2 or a multiple of 4 units");
    Real amp[kNoisePairs<P>], trig[P];
    if constexpr (M::kNoise) {
        draw_noise<Real, P>(amp, trig, k, u0, nl, keys);
    } else {
#pragma unroll
        for (int j = 0; j < kNoisePairs<P>; ++j) amp[j] = Real(0);
#pragma unroll
        for (int i = 0; i < P; ++i) trig[i] = Real(0);
    }
    em_step_noise<M, Real, P, RECORD>(model, x, cp, amp, trig, u0, units, reduce, rec);
}

// The step for a lane of 2 units whose Philox word pair (wa, wb) is given
// (a pair of lanes sharing a noise block can split the block's two Philox
// calls of two steps between them).
template <class M, typename Real, class RED>
__device__ __forceinline__ void em_step_words(M &model, Real (&x)[M::U][2], Real (&cp)[M::U][2], uint32_t wa,
                                              uint32_t wb, int u0, int units, RED &reduce) {
    Real amp[1], trig[2];
    box_muller_polar<Real>(wa, wb, amp[0], trig[0], trig[1]);
    em_step_noise<M, Real, 2>(model, x, cp, amp, trig, u0, units, reduce);
}

// End of a compensation period (models with kDelayedComp): every unit's
// compensation folded into its state.
template <int U, int P>
__device__ __forceinline__ void renormalize_units(float (&x)[U][P], float (&cp)[U][P]) {
#pragma unroll
    for (int c = 0; c < U; ++c)
#pragma unroll
        for (int i = 0; i < P; ++i) renormalize(x[c][i], cp[c][i]);
}
template <int U, int P>
__device__ __forceinline__ void renormalize_units(double (&)[U][P], double (&)[U][P]) {}

// The units' values x - c (what a frame or a final state holds).
template <typename Real, int U, int P>
__device__ __forceinline__ void unit_values(const Real (&x)[U][P], const Real (&cp)[U][P], Real (&v)[U][P]) {
#pragma unroll
    for (int c = 0; c < U; ++c)
#pragma unroll
        for (int i = 0; i < P; ++i) v[c][i] = state_value(x[c][i], cp[c][i]);
}

// One stage of the classical fourth-order Runge-Kutta step (below): the
// coupling sums at the stage state `at`, then per unit the
// model's drift increment h f(at); acc += weight h f(at), and
// y = base + frac_next h f(at) is the next stage's state (y may be `at`:
// each unit is read before it is overwritten, the sums were taken first).
template <class M, typename Real, int P, class RED>
__device__ __forceinline__ void rk4_stage(M &model, const Real (&at)[M::U][P], const Real (&base)[M::U][P],
                                          int u0, int units, RED &reduce, Real (&acc)[M::U][P], Real (&y)[M::U][P],
                                          Real weight, Real frac_next) {
    constexpr int NRA = M::NR > 0 ? M::NR : 1;
    Real red[NRA];
    model.prepare_stage(at, u0, units, red);
    if constexpr (M::NR > 0) reduce(red);
#pragma unroll
    for (int i = 0; i < P; ++i) {
        Real inc[M::U];
        model.drift_incr(i, at, red, inc);
#pragma unroll
        for (int c = 0; c < M::U; ++c) {
            acc[c][i] = fma_r(weight, inc[c], acc[c][i]);
            y[c][i] = fma_r(frac_next, inc[c], base[c][i]);
        }
    }
}

// One step of the classical fourth-order Runge-Kutta method on the drift
// alone (the ODE path; the paper lists Runge-Kutta among its ODE
// integrators, Sec. 1.5): stages at x, x + k1/2, x + k2/2, x + k3 with
// k = h f, and (k1 + 2 k2 + 2 k3 + k4) / 6 goes through the same compensated
// accumulation as an Euler-Maruyama increment.  No noise is drawn.  The
// stage states are built on the model's stage base (for the phase models
// the compensated phase reduced to [-pi, pi], so a stage phase carries the
// rounding of a number below pi rather than of the unreduced phase).
template <class M, typename Real, int P, class RED>
__device__ __forceinline__ void rk4_step(M &model, Real (&x)[M::U][P], Real (&cp)[M::U][P], int u0, int units,
                                         RED &reduce) {
    Real acc[M::U][P], y[M::U][P], base[M::U][P];
#pragma unroll
    for (int c = 0; c < M::U; ++c)
#pragma unroll
        for (int i = 0; i < P; ++i) acc[c][i] = Real(0);
    model.stage_base(x, cp, base);
    rk4_stage<M, Real, P>(model, base, base, u0, units, reduce, acc, y, Real(1), Real(0.5));
    rk4_stage<M, Real, P>(model, y, base, u0, units, reduce, acc, y, Real(2), Real(0.5));
    rk4_stage<M, Real, P>(model, y, base, u0, units, reduce, acc, y, Real(2), Real(1));
    rk4_stage<M, Real, P>(model, y, base, u0, units, reduce, acc, y, Real(1), Real(0));
#pragma unroll
    for (int i = 0; i < P; ++i)
#pragma unroll
        for (int c = 0; c < M::U; ++c) accumulate(x[c][i], cp[c][i], mul_r(acc[c][i], Real(1) / Real(6)));
}

// Newton iterations per implicit step (a fixed count, from the old state).
constexpr int kNewtonIters = 4;

// One step of an implicit ODE scheme on the drift alone (the paper lists
// implicit Euler and implicit midpoint among its ODE integrators, Sec. 1.5):
// the increment d solves d = h f(x + theta d) -- theta = 1 implicit Euler,
// 1/2 implicit midpoint -- by kNewtonIters Newton iterations from d = 0:
// at z = x + theta d the residual r = h f(z) - d (the model's drift
// increment), then d += (I - theta h J(z))^-1 r, the solve done by the
// model in closed form for its Jacobian's structure.  d then goes through
// the compensated accumulation.  No noise is drawn.  z is built on the
// model's stage base, as the Runge-Kutta stages are.
template <class M, typename Real, int P, class RED>
__device__ __forceinline__ void implicit_step(M &model, Real (&x)[M::U][P], Real (&cp)[M::U][P], int u0, int units,
                                              RED &reduce, Real theta) {
    constexpr int NRA = M::NR > 0 ? M::NR : 1;
    Real base[M::U][P], d[M::U][P], z[M::U][P];
    model.stage_base(x, cp, base);
#pragma unroll
    for (int c = 0; c < M::U; ++c)
#pragma unroll
        for (int i = 0; i < P; ++i) d[c][i] = Real(0);
#pragma unroll 1
    for (int it = 0; it < kNewtonIters; ++it) {
#pragma unroll
        for (int c = 0; c < M::U; ++c)
#pragma unroll
            for (int i = 0; i < P; ++i) z[c][i] = fma_r(theta, d[c][i], base[c][i]);
        Real red[NRA];
        model.prepare_stage(z, u0, units, red);
        if constexpr (M::NR > 0) reduce(red);
        Real r[M::U][P];
#pragma unroll
        for (int i = 0; i < P; ++i) {
            Real inc[M::U];
            model.drift_incr(i, z, red, inc);
#pragma unroll
            for (int c = 0; c < M::U; ++c) r[c][i] = inc[c] - d[c][i];
        }
        model.newton_solve(z, red, r, theta, u0, units, reduce);
#pragma unroll
        for (int c = 0; c < M::U; ++c)
#pragma unroll
            for (int i = 0; i < P; ++i) d[c][i] += r[c][i];
    }
#pragma unroll
    for (int i = 0; i < P; ++i)
#pragma unroll
        for (int c = 0; c < M::U; ++c) accumulate(x[c][i], cp[c][i], d[c][i]);
}

// Step schemes of the forward kernel.
enum : int { kSchemeEm = 0, kSchemeRk4 = 1, kSchemeImplicit = 2 };

// Blocks per SM the forward kernel's registers are capped for (0: the
// compiler's choice); see em_forward_kernel_capped.
template <class M, typename Real, int G, int P, int SCHEME>
constexpr int kForwardMinBlocks =
    !(std::is_same<Real, float>::value && G > 1 && M::U == 1 && P <= 8) ? 0
    : SCHEME == kSchemeEm ? (P <= 4 ? 7 : 5)
    : SCHEME == kSchemeImplicit ? 5
    : 0;

template <class M, typename Real, int G, int P, int SCHEME>
__device__ __forceinline__ void em_forward_body(const ForwardArgs &a) {
    constexpr int U = M::U;
    constexpr bool kKahan = std::is_same<Real, float>::value;
    static_assert(P == 1 || P == 2 || P % 4 == 0, "a lane holds 1, 2 or a multiple of 4 units");
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t orbit = tid / G;
    const int lig = (int)(tid & (G - 1));
    const bool active = orbit < a.orbits;
    const int64_t o = active ? orbit : a.orbits - 1;
    const int u0 = lig * P;
    const int units = a.units;
    const int64_t n = a.n;
    // o is clamped into [0, orbits) (lanes past the last orbit repeat it and
    // store nothing): the check records a launch whose orbit count is wrong
    (void)SDEB_CHECK(a.check, o >= 0 && o < a.orbits, kChkForwardState, o);

    M model;
    model.load(static_cast<const Real *>(a.params) + o * a.param_stride, u0, units, (Real)a.dt,
               (Real)sqrt(a.dt));

    Real *xrow = static_cast<Real *>(a.x) + o * n;
    Real x[U][P], cp[U][P];
    load_units<Real, U, P>(xrow, units, u0, x);
    if constexpr (kKahan) {
        load_units<float, U, P>(a.comp + o * n, units, u0, cp);
    } else {
#pragma unroll
        for (int c = 0; c < U; ++c)
#pragma unroll
            for (int i = 0; i < P; ++i) cp[c][i] = Real(0);
    }

    const uint32_t gorb = a.orbit_offset + (uint32_t)o;
    Real *frames = static_cast<Real *>(a.frames);
    Real *ckpt = static_cast<Real *>(a.ckpt);
    uint32_t to_frame = a.stride - (a.k_begin % a.stride);
    uint32_t to_ckpt = a.ckpt_every ? a.ckpt_every - (a.k_begin % a.ckpt_every) : 0u;

    WarpGroupSum<G> reduce;
    const NoiseLane<P> noise(gorb, u0, a.keys);
    // Steps run in runs that end at the next frame, checkpoint or k_end (and,
    // with the periodic compensation, at the next multiple of kCompPeriod),
    // so the step loop itself carries no per-step bookkeeping.  FP32 unrolls
    // two steps (more independent work between the SFU waits); FP64 keeps
    // one, its registers are already near the limit.
    constexpr bool kDelayed = SCHEME == kSchemeEm && M::kDelayedComp;
    constexpr uint32_t kRunShort = 8;
    static_assert(kCompPeriod % kRunShort == 0, "a compensation period is whole chunks");
    constexpr bool kChunkRuns = kForwardMinBlocks<M, Real, G, P, SCHEME> == 0;
    constexpr int kRunUnroll = kKahan ? 2 : 1;
    uint32_t k = a.k_begin;
    while (k < a.k_end) {
        uint64_t k_stop = a.k_end;
        if (frames != nullptr) k_stop = min(k_stop, (uint64_t)k + to_frame);
        if (ckpt != nullptr) k_stop = min(k_stop, (uint64_t)k + to_ckpt);
        if constexpr (kDelayed) k_stop = min(k_stop, (uint64_t)((k | (kCompPeriod - 1u)) + 1u));
        const uint32_t run = (uint32_t)(k_stop - k);
        bool fixed = false;  // the run went through a loop of fixed trip count
        if constexpr (kDelayed && kChunkRuns) {
            // whole 8-step chunks (a compensation period is two): kernels
            // without a register cap
            if (run % kRunShort == 0) {
                for (uint32_t s0 = 0; s0 < run; s0 += kRunShort) {
#pragma unroll 2
                    for (uint32_t s = 0; s < kRunShort; ++s)
                        em_step<M, Real, P>(model, x, cp, k + s0 + s, noise, u0, units, a.keys, reduce);
                }
                fixed = true;
            }
        } else if constexpr (kDelayed) {
            // a whole compensation period, or the stretch between
            // checkpoints kept every kRunShort steps: capped kernels keep
            // the loop without an outer level (no spills within the cap)
            if (run == kCompPeriod) {
#pragma unroll 2
                for (uint32_t s = 0; s < kCompPeriod; ++s)
                    em_step<M, Real, P>(model, x, cp, k + s, noise, u0, units, a.keys, reduce);
                fixed = true;
            } else if (run == kRunShort) {
#pragma unroll 2
                for (uint32_t s = 0; s < kRunShort; ++s)
                    em_step<M, Real, P>(model, x, cp, k + s, noise, u0, units, a.keys, reduce);
                fixed = true;
            }
        }
        if (!fixed) {
#pragma unroll kRunUnroll
            for (uint32_t s = 0; s < run; ++s) {
                if constexpr (SCHEME == kSchemeRk4)
                    rk4_step<M, Real, P>(model, x, cp, u0, units, reduce);
                else if constexpr (SCHEME == kSchemeImplicit)
                    implicit_step<M, Real, P>(model, x, cp, u0, units, reduce, a.implicit == 1 ? Real(1) : Real(0.5));
                else
                    em_step<M, Real, P>(model, x, cp, k + s, noise, u0, units, a.keys, reduce);
            }
        }
        k += run;
        if constexpr (kDelayed) {
            if ((k & (kCompPeriod - 1u)) == 0) renormalize_units(x, cp);
        }
        if (frames != nullptr && (to_frame -= run) == 0) {
            to_frame = a.stride;
            const int64_t f = (int64_t)(k / a.stride);
            if (active && SDEB_CHECK(a.check, f < a.nframes, kChkForwardFrame, f)) {
                if constexpr (kDelayed) {
                    Real v[U][P];
                    unit_values(x, cp, v);
                    store_units<Real, U, P>(frames + (f * a.orbits + o) * n, units, u0, v);
                } else {
                    store_units<Real, U, P>(frames + (f * a.orbits + o) * n, units, u0, x);
                }
            }
        }
        if (ckpt != nullptr && (to_ckpt -= run) == 0) {
            to_ckpt = a.ckpt_every;
            const int64_t c = (int64_t)(k / a.ckpt_every);
            if (active && SDEB_CHECK(a.check, c < a.nckpt, kChkForwardCkpt, c)) {
                store_units<Real, U, P>(ckpt + (c * a.orbits + o) * n, units, u0, x);
                if constexpr (kKahan)
                    store_units<float, U, P>(a.ckpt_comp + (c * a.orbits + o) * n, units, u0, cp);
            }
        }
    }

    // final state, compensation and the non-finite flag (a state stored for
    // resuming keeps its pair (x, c); final_value stores the value x - c)
    if constexpr (kDelayed) {
        if (a.final_value) {
            Real v[U][P];
            unit_values(x, cp, v);
#pragma unroll
            for (int c = 0; c < U; ++c)
#pragma unroll
                for (int i = 0; i < P; ++i) {
                    x[c][i] = v[c][i];
                    cp[c][i] = Real(0);
                }
        }
    }
    bool bad = false;
#pragma unroll
    for (int c = 0; c < U; ++c)
#pragma unroll
        for (int i = 0; i < P; ++i)
            if (u0 + i < units && !isfinite(state_value(x[c][i], cp[c][i]))) bad = true;
    const unsigned ballot = __ballot_sync(0xffffffffu, bad);
    const int lane = threadIdx.x & 31;
    unsigned group_bits;
    if constexpr (G == 32) {
        group_bits = ballot;
    } else {
        group_bits = (ballot >> (lane & ~(G - 1))) & ((1u << G) - 1u);
    }
    if (active) {
        store_units<Real, U, P>(xrow, units, u0, x);
        if constexpr (kKahan) store_units<float, U, P>(a.comp + o * n, units, u0, cp);
        if (lig == 0) a.flags[o] = group_bits ? 1u : 0u;
    }
}

template <class M, typename Real, int G, int P, int SCHEME>
__global__ void __launch_bounds__(kForwardBlock) em_forward_kernel(const ForwardArgs a) {
    em_forward_body<M, Real, G, P, SCHEME>(a);
}

// The same kernel with registers capped so that MINB blocks fit per SM,
// for FP32 one-component models on multi-lane layouts: 4 units per lane fit
// 72 registers (seven blocks), 8 units 96 registers (five blocks) without
// spilling; both ran faster than at the compiler's choice (96 and 128
// registers: five and four blocks).  The implicit schemes take five blocks
// (a few spilled words, 1 % faster than four); Runge-Kutta fits 96
// registers by itself.  The single-lane layouts keep the compiler's choice.
template <class M, typename Real, int G, int P, int SCHEME, int MINB>
__global__ void __launch_bounds__(kForwardBlock, MINB) em_forward_kernel_capped(const ForwardArgs a) {
    em_forward_body<M, Real, G, P, SCHEME>(a);
}

// SCHEME: kSchemeEm (Euler-Maruyama, or Milstein chosen by the model
// functor), or an ODE-path scheme (kSchemeRk4, kSchemeImplicit).
template <template <typename, int> class MF, typename Real, int G, int P, int SCHEME = kSchemeEm>
cudaError_t launch_forward_layout(const ForwardArgs &a, cudaStream_t s) {
    using M = MF<Real, P>;
    const int64_t threads = a.orbits * G;
    const int64_t grid = (threads + kForwardBlock - 1) / kForwardBlock;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    constexpr int minb = kForwardMinBlocks<M, Real, G, P, SCHEME>;
    if constexpr (minb > 0)
        em_forward_kernel_capped<M, Real, G, P, SCHEME, minb><<<(unsigned)grid, kForwardBlock, 0, s>>>(a);
    else
        em_forward_kernel<M, Real, G, P, SCHEME><<<(unsigned)grid, kForwardBlock, 0, s>>>(a);
    return cudaGetLastError();
}

#define SDEB_FORWARD_LAYOUT(G_, P_) \
    if (l.G == (G_) && l.P == (P_)) return launch_forward_layout<MF, Real, G_, P_>(a, s);
#define SDEB_FORWARD_LAYOUT_ODE(G_, P_) \
    if (l.G == (G_) && l.P == (P_)) return launch_forward_layout<MF, Real, G_, P_, SCHEME>(a, s);

// The layouts default_layout() can return.
template <template <typename, int> class MF, typename Real>
cudaError_t dispatch_default_layouts(const ForwardArgs &a, Layout l, cudaStream_t s) {
    SDEB_FORWARD_LAYOUT(1, 1)
    SDEB_FORWARD_LAYOUT(1, 2)
    SDEB_FORWARD_LAYOUT(1, 4)
    SDEB_FORWARD_LAYOUT(1, 8)
    SDEB_FORWARD_LAYOUT(2, 8)
    SDEB_FORWARD_LAYOUT(4, 8)
    SDEB_FORWARD_LAYOUT(8, 8)
    SDEB_FORWARD_LAYOUT(16, 8)
    SDEB_FORWARD_LAYOUT(32, 8)
    return cudaErrorNotSupported;
}

// The ODE-path instantiations (SCHEME), for the layouts default_layout() can return.
template <template <typename, int> class MF, typename Real, int SCHEME>
cudaError_t dispatch_ode_layouts(const ForwardArgs &a, Layout l, cudaStream_t s) {
    SDEB_FORWARD_LAYOUT_ODE(1, 1)
    SDEB_FORWARD_LAYOUT_ODE(1, 2)
    SDEB_FORWARD_LAYOUT_ODE(1, 4)
    SDEB_FORWARD_LAYOUT_ODE(1, 8)
    SDEB_FORWARD_LAYOUT_ODE(2, 8)
    SDEB_FORWARD_LAYOUT_ODE(4, 8)
    SDEB_FORWARD_LAYOUT_ODE(8, 8)
    SDEB_FORWARD_LAYOUT_ODE(16, 8)
    SDEB_FORWARD_LAYOUT_ODE(32, 8)
    return cudaErrorNotSupported;
}

// Extra layouts tried by the layout tuner for the phase models.
template <template <typename, int> class MF, typename Real>
cudaError_t dispatch_tuning_layouts(const ForwardArgs &a, Layout l, cudaStream_t s) {
    SDEB_FORWARD_LAYOUT(2, 4)
    SDEB_FORWARD_LAYOUT(4, 4)
    SDEB_FORWARD_LAYOUT(8, 4)
    SDEB_FORWARD_LAYOUT(16, 4)
    SDEB_FORWARD_LAYOUT(32, 4)
    SDEB_FORWARD_LAYOUT(4, 16)
    SDEB_FORWARD_LAYOUT(8, 16)
    return dispatch_default_layouts<MF, Real>(a, l, s);
}

template <typename Real, int P>
using KuramotoScalarLane = KuramotoLane<Real, P, false>;
template <typename Real, int P>
using KuramotoPaperLane = KuramotoLane<Real, P, true>;
template <typename Real, int P>
using FhnEmLane = FhnLane<Real, P, false>;
template <typename Real, int P>
using FhnMilsteinLane = FhnLane<Real, P, true>;
template <typename Real, int P>
using OuLane = ScalarLane<Real, P, 0>;
template <typename Real, int P>
using GbmLane = ScalarLane<Real, P, 1>;
template <typename Real, int P>
using GbmMilsteinLane = ScalarLane<Real, P, 1, true>;
template <typename Real, int P>
using LinearLane = ScalarLane<Real, P, 2>;

}  // namespace sdeb
