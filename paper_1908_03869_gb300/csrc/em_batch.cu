// Persistent kernel for batches of heterogeneous instances (different n,
// steps, dt, stride, orbits): the many parameter combinations of the paper's
// optimisation use (Sec. 1.2) in one launch, scheduled longest-first so the
// instances with the longest sequential chains start at once.  Work sizing
// replaces the hand-tuned work-group sizes of the paper's Table 4.
//
// Each item (one orbit of one instance) runs Eq. 2 with the step code of the
// forward kernel (em_step); its coupling sums run over its own lanes only,
// in an order fixed by its layout, so an item's results do not depend on
// the other items or on the schedule beyond its (lanes, units per lane).
// No block ever waits on another: the only shared state is the queue head,
// advanced with atomicAdd.
#include "em_forward_impl.cuh"

namespace sdeb {

namespace {

// Reducers whose FP32 sums are 32-bit fixed point (multiples of 2^-22) mark
// themselves with kScaled22: they take partial sums already scaled by 2^22
// and return the integer totals unscaled, and the item's model carries the
// two powers of two instead (its unit weights times 2^22, its (K/n) dt times
// 2^-22).  Scaling by a power of two commutes with every rounding here (no
// value comes near the subnormal range unless (K/n) dt is below 2^-104), so
// the partials, totals and drift products are the same bits as with the
// scalings in the reducer, two multiplies fewer per sum and step.
template <class R, class = void>
struct Scaled22 : std::false_type {};
template <class R>
struct Scaled22<R, std::void_t<decltype(R::kScaled22)>> : std::bool_constant<R::kScaled22> {};

template <typename Real, int P>
__device__ __forceinline__ void flag_nonfinite(uint8_t *flag, const Real (&x)[1][P], int u0, int units) {
    bool bad = false;
#pragma unroll
    for (int i = 0; i < P; ++i)
        if (u0 + i < units && !isfinite(x[0][i])) bad = true;
    if (bad) *flag = 1;  // flags start at 0; several lanes may write the same 1
}

// Integrates one item on the calling lanes: `lane` is the lane's index in the
// item's lane group, the group sums with `reduce`.  Steps 0..kmax-1 are taken
// (the group's shuffles or barriers need every lane), the item's own state is
// stored, framed and flagged only while k < its step count (`live`).
template <typename Real, int P, class RED, bool SHARE_PHILOX = false>
__device__ __forceinline__ void run_item(const BatchArgs &a, const BatchItem it, bool has, int lane, uint32_t kmax,
                                         RED &reduce) {
    static_assert(!SHARE_PHILOX || P == 2, "Philox sharing pairs lanes of two units");
    using M = KuramotoLane<Real, P, false>;
    constexpr bool kKahan = std::is_same<Real, float>::value;
    const BatchInstance in = a.inst[it.instance];
    const int u0 = lane * P;
    const int units = in.units;
    const int64_t n = in.n;
    // the item's rows lie inside the concatenated buffers; its lane offset inside the item
    (void)SDEB_CHECK(a.check, !has || (it.orbit >= 0 && it.orbit < in.orbits), kChkBatchInstance, it.orbit);
    (void)SDEB_CHECK(a.check, !has || in.x_off + ((int64_t)it.orbit + 1) * n <= a.state_elems, kChkBatchState,
                     in.x_off + (int64_t)it.orbit * n);
    (void)SDEB_CHECK(a.check, !has || in.p_off + (int64_t)it.orbit * in.param_stride + in.d <= a.param_elems,
                     kChkBatchParams, in.p_off + (int64_t)it.orbit * in.param_stride);
    (void)SDEB_CHECK(a.check, !has || in.o_off + it.orbit < a.nitems, kChkBatchFlags, in.o_off + it.orbit);
    (void)SDEB_CHECK(a.check, u0 >= 0 && u0 < 256, kChkBatchLane, u0);
    M model;
    model.load(static_cast<const Real *>(a.params) + in.p_off + (int64_t)it.orbit * in.param_stride, u0, units,
               (Real)in.dt, (Real)sqrt(in.dt));
    if constexpr (Scaled22<RED>::value) {
#pragma unroll
        for (int i = 0; i < P; ++i) model.live[i] *= 0x1p22f;
        model.kn_dt *= 0x1p-22f;
    }
    Real *xrow = static_cast<Real *>(a.x) + in.x_off + (int64_t)it.orbit * n;
    float *crow = kKahan ? a.comp + in.x_off + (int64_t)it.orbit * n : nullptr;
    Real x[1][P], cp[1][P];
    load_units<Real, 1, P>(xrow, units, u0, x);
    if constexpr (kKahan) {
        load_units<float, 1, P>(crow, units, u0, cp);
    } else {
#pragma unroll
        for (int i = 0; i < P; ++i) cp[0][i] = Real(0);
    }
    Real *frames = a.frames != nullptr && in.has_frames ? static_cast<Real *>(a.frames) + in.f_off : nullptr;
    if (has && frames != nullptr) store_units<Real, 1, P>(frames + (int64_t)it.orbit * n, units, u0, x);
    const uint32_t gorb = in.orbit_offset + (uint32_t)it.orbit;
    const NoiseLane<P> noise(gorb, u0, a.keys);
    const uint32_t steps = in.steps;
    uint32_t to_frame = in.stride;
    // Steps run in runs that end at the next event (a frame or the end) of
    // any item of the warp, or at the end of a compensation period, so the
    // step loop carries no per-step checks; the run length is the warp's
    // minimum, the same in every warp of a team.  A whole period runs as a
    // loop of fixed trip count (one step per iteration: two would spill
    // within the kernel's 96 registers).
    uint32_t k = 0;
    while (k < kmax) {
        const bool live = has && k < steps;
        uint32_t mine = kmax - k;
        if (live) mine = min(mine, min(to_frame, steps - k));
        if constexpr (M::kDelayedComp) mine = min(mine, ((k | (kCompPeriod - 1u)) + 1u) - k);
        const uint32_t run = __reduce_min_sync(0xffffffffu, mine);
        if constexpr (SHARE_PHILOX) {
            // Lanes 2b and 2b + 1 (units 4b.. and 4b + 2..) use the two
            // halves of noise block b: over a pair of steps each lane draws
            // the block for one of the steps (the even lane step k, the odd
            // lane step k + 1) and hands its partner the half the partner
            // uses, so a block costs one Philox call per step instead of two.
            const bool odd = (lane & 1) != 0;
            uint32_t s = 0;
#pragma unroll 1
            for (; s + 2 <= run; s += 2) {
                const U32x4 w = philox4x32_10_fixed(k + s + (odd ? 1u : 0u), noise.r1[0], a.keys);
                const uint32_t r0 = __shfl_xor_sync(0xffffffffu, odd ? w.x : w.z, 1);
                const uint32_t r1 = __shfl_xor_sync(0xffffffffu, odd ? w.y : w.w, 1);
                em_step_words<M, Real>(model, x, cp, odd ? r0 : w.x, odd ? r1 : w.y, u0, units, reduce);
                em_step_words<M, Real>(model, x, cp, odd ? w.z : r0, odd ? w.w : r1, u0, units, reduce);
            }
            if (s < run) em_step<M, Real, P>(model, x, cp, k + s, noise, u0, units, a.keys, reduce);
        } else if (M::kDelayedComp && run == kCompPeriod) {
#pragma unroll 1
            for (uint32_t s = 0; s < kCompPeriod; ++s)
                em_step<M, Real, P>(model, x, cp, k + s, noise, u0, units, a.keys, reduce);
        } else {
#pragma unroll 1
            for (uint32_t s = 0; s < run; ++s)
                em_step<M, Real, P>(model, x, cp, k + s, noise, u0, units, a.keys, reduce);
        }
        if constexpr (M::kDelayedComp) {
            if (((k + run) & (kCompPeriod - 1u)) == 0) renormalize_units(x, cp);
        }
        k += run;
        if (live) {
            Real v[1][P];
            unit_values(x, cp, v);   // the state's value (x - c)
            to_frame -= run;
            if (to_frame == 0) {
                to_frame = in.stride;
                const int64_t frow = in.f_off + ((int64_t)(k / in.stride) * in.orbits + it.orbit) * n;
                if (frames != nullptr && SDEB_CHECK(a.check, frow + n <= a.frame_elems, kChkBatchFrame, frow))
                    store_units<Real, 1, P>(frames + ((int64_t)(k / in.stride) * in.orbits + it.orbit) * n, units, u0,
                                            v);
            }
            if (k == steps) {
                store_units<Real, 1, P>(xrow, units, u0, v);
                flag_nonfinite<Real, P>(a.flags + in.o_off + it.orbit, v, u0, units);
            }
        }
    }
}

// Sums over one item's lanes [s, e) of a packed warp: an inclusive scan by
// shfl_up -- at level q a lane adds the partial of the lane 2^q below while
// that lane is in the segment, so after level q lane L holds the sum over
// [max(L - 2^(q+1) + 1, s), L] -- then lane e - 1's total is broadcast.  The
// addition tree depends only on L - s: an item's sums, and so its orbit,
// are the same bits wherever it sits in the warp.  Levels past the warp's
// longest segment add nothing and are skipped (the count is warp-uniform).
struct SegmentSum {
    int last;       // e - 1
    int levels;     // ceil(log2(longest segment of the warp))
    unsigned take;  // bit q: L - 2^q >= s
    template <typename Real, int NR>
    __device__ __forceinline__ void operator()(Real (&r)[NR]) const {
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            if (q >= levels) break;
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                const Real t = __shfl_up_sync(0xffffffffu, r[j], 1u << q);
                if (take & (1u << q)) r[j] += t;
            }
        }
#pragma unroll
        for (int j = 0; j < NR; ++j) r[j] = __shfl_sync(0xffffffffu, r[j], last);
    }
};

// A packed warp: the task's items lie side by side in lane order, item j on
// ceil(units_j / P) lanes.  Lanes past the last item idle through the steps
// on a one-lane segment of their own (the scans need every lane).
template <typename Real, int P>
__device__ __forceinline__ void run_packed_warp(const BatchArgs &a, const BatchWarpTask &t) {
    const int lane = threadIdx.x & 31;
    int start = 0, mine = -1, s = lane, e = lane + 1, longest = 1;
    if (!SDEB_CHECK(a.check, t.first >= 0 && t.first + t.count <= a.nitems, kChkBatchItem, t.first)) return;
    for (int j = 0; j < t.count; ++j) {
        const int32_t ins = a.items[t.first + j].instance;
        if (!SDEB_CHECK(a.check, ins >= 0 && ins < a.ninst, kChkBatchInstance, ins)) return;
        const int len = (a.inst[ins].units + P - 1) / P;
        if (lane >= start && lane < start + len) {
            mine = j;
            s = start;
            e = start + len;
        }
        longest = max(longest, len);
        start += len;
    }
    // the item's segment [s, e) lies inside the warp (the packing keeps it within 32 lanes)
    if (!SDEB_CHECK(a.check, s >= 0 && e <= 32 && s < e, kChkBatchLane, (int64_t)s * 64 + e)) return;
    SegmentSum reduce;
    reduce.last = e - 1;
    reduce.levels = 32 - __clz(longest - 1);
    reduce.take = 0;
#pragma unroll
    for (int q = 0; q < 5; ++q)
        if (lane - (1 << q) >= s) reduce.take |= 1u << q;
    const bool has = mine >= 0;
    run_item<Real, P>(a, a.items[t.first + (has ? mine : 0)], has, lane - s, t.kmax, reduce);
}

// One item alone on a warp, 2 units per lane: the coupling sums over the
// whole warp, FP64 by butterfly (the same bits in every lane), FP32 in the
// 32-bit fixed point of the teams' sums (multiples of 2^-22) added by one
// redux.sync, so an item's FP32 sums are the bits a one-warp team would
// form.  No shared memory and no barrier.
template <typename Real>
struct SoloWarpSum {
    template <int NR>
    __device__ __forceinline__ void operator()(Real (&r)[NR]) const {
#pragma unroll
        for (int q = 0; q < NR; ++q) r[q] = group_sum<32>(r[q]);
    }
};

template <>
struct SoloWarpSum<float> {
    static constexpr bool kScaled22 = true;   // partials arrive times 2^22, totals leave unscaled
    template <int NR>
    __device__ __forceinline__ void operator()(float (&r)[NR]) const {
#pragma unroll
        for (int q = 0; q < NR; ++q) r[q] = __int2float_rn(__reduce_add_sync(0xffffffffu, __float2int_rn(r[q])));
    }
};

// A single-warp item (a warp task with p == 2 and one item): lanes 2b and
// 2b + 1 share noise block b as a team's lane pairs do; lanes past the
// item's ceil(n / 2) hold no units and add zeros.
template <typename Real>
__device__ __forceinline__ void run_solo_warp(const BatchArgs &a, const BatchWarpTask &t) {
    if (!SDEB_CHECK(a.check, t.count == 1 && t.first >= 0 && t.first < a.nitems, kChkBatchItem, t.first)) return;
    const BatchItem it = a.items[t.first];
    if (!SDEB_CHECK(a.check, it.instance >= 0 && it.instance < a.ninst, kChkBatchInstance, it.instance)) return;
    if (!SDEB_CHECK(a.check, a.inst[it.instance].units <= 64, kChkBatchLane, a.inst[it.instance].units)) return;
    SoloWarpSum<Real> reduce;
    run_item<Real, 2, SoloWarpSum<Real>, true>(a, it, true, (int)(threadIdx.x & 31), a.inst[it.instance].steps,
                                               reduce);
}

// Team of NW warps on one item; BAR = 0 is the whole block's barrier,
// otherwise named barrier BAR for the team's 32 * NW threads.
template <int NW, int BAR, typename Real>
struct NamedTeamSum {
    Real *buf;   // [2][NW][2] in shared memory
    int flip;
    int warp0;
    template <int NR>
    __device__ __forceinline__ void operator()(Real (&r)[NR]) {
        static_assert(NR <= 2, "two sums at most");
        const int warp = (threadIdx.x >> 5) - warp0, lane = threadIdx.x & 31;
        Real *slot = buf + flip * NW * 2;
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            r[q] = group_sum<32>(r[q]);
            if (lane == 0) slot[warp * 2 + q] = r[q];
        }
        if constexpr (BAR == 0) {
            __syncthreads();
        } else {
            asm volatile("bar.sync %0, %1;" ::"n"(BAR), "n"(NW * 32) : "memory");
        }
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            Real t = slot[q];
#pragma unroll
            for (int w = 1; w < NW; ++w) t += slot[w * 2 + q];
            r[q] = t;
        }
        flip ^= 1;
    }
};

// FP32: the team's sums in 32-bit fixed point, multiples of 2^-22 (a sum
// over at most 256 units of terms in [-1, 1] stays below 2^30): each lane's
// partial rounded once, added across the warp by one redux.sync and across
// the team's warps through shared memory.  Integer addition is exact, so the
// totals are the same bits in every lane and in any order, and the rounding
// (at most 2^-23 per lane) is of the order of the FP32 butterfly's.
// With two sums the warp's pair goes to shared memory as one 8-byte store
// and the team's slots come back as 16-byte loads (the slots are 16-byte
// aligned).  The partials arrive scaled by 2^22 (kScaled22).
template <int NW, int BAR>
struct NamedTeamSum<NW, BAR, float> {
    static constexpr bool kScaled22 = true;
    float *buf;  // [2][NW][2] words in shared memory, used as int; 16-byte aligned
    int flip;
    int warp0;
    template <int NR>
    __device__ __forceinline__ void operator()(float (&r)[NR]) {
        static_assert(NR <= 2, "two sums at most");
        constexpr bool kVec = NR == 2 && (NW == 2 || NW == 4);
        const int warp = (threadIdx.x >> 5) - warp0, lane = threadIdx.x & 31;
        int *slot = reinterpret_cast<int *>(buf) + flip * NW * 2;
        int ws[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) ws[q] = __reduce_add_sync(0xffffffffu, __float2int_rn(r[q]));
        if (lane == 0) {
            if constexpr (kVec) {
                *reinterpret_cast<int2 *>(slot + warp * 2) = make_int2(ws[0], ws[NR - 1]);
            } else {
#pragma unroll
                for (int q = 0; q < NR; ++q) slot[warp * 2 + q] = ws[q];
            }
        }
        if constexpr (BAR == 0) {
            __syncthreads();
        } else {
            asm volatile("bar.sync %0, %1;" ::"n"(BAR), "n"(NW * 32) : "memory");
        }
        if constexpr (kVec) {
            const int4 u = reinterpret_cast<const int4 *>(slot)[0];
            int t0 = u.x + u.z, t1 = u.y + u.w;
            if constexpr (NW == 4) {
                const int4 v = reinterpret_cast<const int4 *>(slot)[1];
                t0 += v.x + v.z;
                t1 += v.y + v.w;
            }
            r[0] = __int2float_rn(t0);
            r[NR - 1] = __int2float_rn(t1);
        } else {
#pragma unroll
            for (int q = 0; q < NR; ++q) {
                int t = slot[q];
#pragma unroll
                for (int w = 1; w < NW; ++w) t += slot[w * 2 + q];
                r[q] = __int2float_rn(t);
            }
        }
        flip ^= 1;
    }
};

template <typename Real, int NW, int P, int BAR>
__device__ __forceinline__ void run_team(const BatchArgs &a, int32_t item, Real *buf, int warp0) {
    NamedTeamSum<NW, BAR, Real> reduce{buf, 0, warp0};
    // a task's item index comes from the host's table: every thread of the team checks the same value
    if (!SDEB_CHECK(a.check, item >= 0 && item < a.nitems, kChkBatchItem, item)) return;
    const BatchItem it = a.items[item];
    if (!SDEB_CHECK(a.check, it.instance >= 0 && it.instance < a.ninst, kChkBatchInstance, it.instance)) return;
    const uint32_t steps = a.inst[it.instance].steps;
    run_item<Real, P, NamedTeamSum<NW, BAR, Real>, P == 2>(a, it, true, (int)threadIdx.x - warp0 * 32, steps,
                                                           reduce);
}

// Registers capped for five resident blocks per SM (96 per thread, a few
// spilled words): 8 % faster on the 4096-instance workload than the
// compiler's 119 at four blocks, whichever residency the tuner then picks.
template <typename Real>
__global__ void __launch_bounds__(kBatchBlock, 5) em_batch_kernel(const BatchArgs a) {
    __shared__ int s_task;
    __shared__ __align__(16) Real s_red[2][2 * 4 * 2];
    for (;;) {
        if (threadIdx.x == 0) s_task = atomicAdd(a.head, 1);
        __syncthreads();
        const int t = s_task;
        __syncthreads();
        if (t >= a.ntasks) return;
        const BatchTask &task = a.tasks[t];  // read in place: the warp index is not a constant
        const int warp = threadIdx.x >> 5;
        if (task.kind == kBatchWarps) {
            const BatchWarpTask wt = task.warp[warp];
            switch (wt.count > 0 ? wt.p : 0) {
            case 8: run_packed_warp<Real, 8>(a, wt); break;
            case 4: run_packed_warp<Real, 4>(a, wt); break;
            case 2: run_solo_warp<Real>(a, wt); break;
            default: break;
            }
        } else if (task.kind == kBatchTeam128) {
            run_team<Real, 4, 2, 0>(a, task.item[0], s_red[0], 0);
        } else {
            const int half = warp >> 1;
            const int32_t item = task.item[half];
            if (item >= 0) {
                if (half == 0) {
                    if (task.team_p == 2) run_team<Real, 2, 2, 1>(a, item, s_red[0], 0);
                    else run_team<Real, 2, 4, 1>(a, item, s_red[0], 0);
                } else {
                    if (task.team_p == 2) run_team<Real, 2, 2, 2>(a, item, s_red[1], 2);
                    else run_team<Real, 2, 4, 2>(a, item, s_red[1], 2);
                }
            }
        }
    }
}

}  // namespace

cudaError_t launch_batch(const BatchArgs &a, int grid, bool fp64, cudaStream_t s) {
    if (a.ntasks == 0) return cudaSuccess;
    if (grid < 1) grid = 1;
    if (fp64)
        em_batch_kernel<double><<<grid, kBatchBlock, 0, s>>>(a);
    else
        em_batch_kernel<float><<<grid, kBatchBlock, 0, s>>>(a);
    return cudaGetLastError();
}

int batch_blocks_per_sm(bool fp64) {
    int blocks = 0;
    cudaError_t e = fp64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, em_batch_kernel<double>, kBatchBlock, 0)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, em_batch_kernel<float>, kBatchBlock, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return blocks > 0 ? blocks : 1;
}

}  // namespace sdeb
