// Discrete adjoint of the Euler-Maruyama recursion (Eq. 2) for the Kuramoto
// models of Eq. 5/6, giving pathwise gradients of a loss L(X^K) with respect
// to the parameters and the initial state (the parameter-optimisation use of
// Sec. 1.2; the adjoint itself is not in the paper).
//
// For theta^{k+1}_i = theta^k_i + dt [omega_i + (K/n) sum_j sin(theta^k_j - theta^k_i)]
//                     + g_i sqrt(dt) N^k_i
// and lambda^k = dL/dtheta^k:
//   lambda^k_l = lambda^{k+1}_l + (K dt / n) [cos x_l A + sin x_l B
//                                             - lambda^{k+1}_l (cos x_l C + sin x_l S)]
// with A = sum_i lambda^{k+1}_i cos x_i, B = sum_i lambda^{k+1}_i sin x_i,
// C = sum_j cos x_j, S = sum_j sin x_j at x = theta^k (the pairwise sums
// sum_i lambda_i cos(x_i - x_l) and sum_j cos(x_j - x_l) rewritten exactly);
//   dL/dK      += (dt / n) sum_i lambda^{k+1}_i (S cos x_i - C sin x_i) = (dt / n) (S A - C B),
//   dL/domega_i += dt lambda^{k+1}_i,
//   dL/dg      += sqrt(dt) sum_i lambda^{k+1}_i N^k_i   (g = sigma, or p_i per unit),
// and dL/dtheta^0 = lambda^0.
//
// States are recomputed segment by segment from the checkpoints the forward
// pass stored every ckpt_every steps, with the same step code (bit-identical
// trajectory).  The forward pass stores no noise: the replay regenerates the
// Philox normals of each step (they drive the recomputed states) and keeps
// them, with the sine and cosine of each unit's phase and the orbit's
// coupling sums C and S, for the reverse sweep of the same segment: in the
// shared memory of the thread (segments short enough to fit), or in a global
// segment buffer with the reduced phase (FP32: x - c folded into [-pi, pi])
// in place of sine and cosine, which the sweep then takes again.
#include <type_traits>

#include "em_forward_impl.cuh"

namespace sdeb {

namespace {

// Step step_off's record of orbit o from the global segment buffer.
template <typename Real, int P>
__device__ __forceinline__ void load_record(const Real *seg, const Real *seg_sums, uint32_t step_off, int64_t orbits,
                                            int64_t o, int64_t n, int units, int u0, Real (&r)[1][P],
                                            Real (&z)[1][P], Real &C, Real &S) {
    const int64_t rowi = (int64_t)step_off * orbits + o;
    const Real *row = seg + rowi * (2 * n);
    load_units<Real, 1, P>(row, units, u0, r);
    load_units<Real, 1, P>(row + n, units, u0, z);
    C = seg_sums[2 * rowi];
    S = seg_sums[2 * rowi + 1];
}

// A vector of V Reals, aligned to its size (one 8- or 16-byte shared-memory
// access).
template <typename Real, int V>
struct alignas(V * sizeof(Real)) RVec {
    Real v[V];
};

// The records a thread keeps per step when the segment's records sit in
// shared memory: sine, cosine and normal of each unit in vectors of V Reals
// (V = P up to 16 bytes), and the orbit's C, S as one pair.
template <typename Real, int P>
struct SmemRec {
    static constexpr int V = P * (int)sizeof(Real) < 16 ? P : 16 / (int)sizeof(Real);
    static constexpr int NV = 3 * P / V;  // vectors per step: sines, cosines, normals
    using Vec = RVec<Real, V>;
    using Pair = RVec<Real, 2>;
    static constexpr int64_t kStepBytes = (int64_t)NV * sizeof(Vec) + (int64_t)sizeof(Pair);
};

// SMEM: the replay keeps the segment's records in shared memory (dynamic:
// ckpt_every steps x SmemRec::kStepBytes per thread).  The vectors of step s
// come first, vector v of thread t at index (s * NV + v) * blockDim + t, then
// the pairs, step s of thread t at s * blockDim + t: consecutive threads
// access consecutive addresses.  The sweep reads back the sine and cosine
// the replay's drift took instead of taking them again.  Otherwise the
// records go through the global segment buffer.
template <bool PAPER, typename Real, int G, int P, bool SMEM>
__global__ void __launch_bounds__(kForwardBlock) em_adjoint_kernel(const AdjointArgs a) {
    using M = KuramotoLane<Real, P, PAPER>;
    static_assert(P == 1 || P == 2 || P % 4 == 0, "a lane holds 1, 2 or a multiple of 4 units");
    extern __shared__ __align__(16) unsigned char adj_smem[];
    using SR = SmemRec<Real, P>;
    constexpr int V = SR::V, NV = SR::NV;
    typename SR::Vec *const vrec = reinterpret_cast<typename SR::Vec *>(adj_smem) + threadIdx.x;
    typename SR::Pair *const prec =
        reinterpret_cast<typename SR::Pair *>(adj_smem + (size_t)a.ckpt_every * NV * kForwardBlock *
                                                             sizeof(typename SR::Vec)) + threadIdx.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t orbit = tid / G;
    const int lig = (int)(tid & (G - 1));
    const bool active = orbit < a.orbits;
    const int64_t o = active ? orbit : a.orbits - 1;
    const int u0 = lig * P;
    const int units = a.units;
    const int64_t n = a.n;
    const Real dt = (Real)a.dt;
    const Real sqdt = (Real)sqrt(a.dt);
    const Real *prow = static_cast<const Real *>(a.params) + o * a.param_stride;

    M model;
    model.load(prow, u0, units, dt, sqdt);
    const Real kdt_n = mul_r(model.kn, dt);
    Real kdt_n_live[P];  // (K/n) dt for the orbit's units, 0 for padding
#pragma unroll
    for (int i = 0; i < P; ++i) kdt_n_live[i] = kdt_n * model.live[i];
    const uint32_t gorb = a.orbit_offset + (uint32_t)o;

    Real lam[1][P];
    load_units<Real, 1, P>(static_cast<const Real *>(a.dL_dxK) + o * n, units, u0, lam);
    Real g_omega[P], g_noise[PAPER ? P : 1];
#pragma unroll
    for (int i = 0; i < P; ++i) g_omega[i] = Real(0);
#pragma unroll
    for (int i = 0; i < (PAPER ? P : 1); ++i) g_noise[i] = Real(0);
    Real g_k = Real(0);

    const Real *ckpt = static_cast<const Real *>(a.ckpt);
    Real *seg = static_cast<Real *>(a.seg);
    // after the [ckpt_every][orbits][2n] phase and normal rows: [ckpt_every][orbits][2] sums
    Real *seg_sums = seg + (int64_t)a.ckpt_every * a.orbits * (2 * n);
    WarpGroupSum<G> reduce;
    const NoiseLane<P> noise(gorb, u0, a.keys);
    const int64_t nseg = ((int64_t)a.steps + a.ckpt_every - 1) / a.ckpt_every;

    // Checkpoint c's state (and FP32 compensation) into (cx, ccp).
    auto load_ckpt = [&](int64_t c, Real (&cx)[1][P], Real (&ccp)[1][P]) {
        if (SDEB_CHECK(a.check, c < a.nckpt, kChkAdjointCkpt, c)) {
            load_units<Real, 1, P>(ckpt + (c * a.orbits + o) * n, units, u0, cx);
        } else {
#pragma unroll
            for (int i = 0; i < P; ++i) cx[0][i] = Real(0);
        }
        if constexpr (std::is_same<Real, float>::value) {
            if (c < a.nckpt) {
                load_units<float, 1, P>(a.ckpt_comp + (c * a.orbits + o) * n, units, u0, ccp);
            } else {
#pragma unroll
                for (int i = 0; i < P; ++i) ccp[0][i] = 0.0f;
            }
        } else {
#pragma unroll
            for (int i = 0; i < P; ++i) ccp[0][i] = Real(0);
        }
    };
    // FP32: the next segment's checkpoint is loaded one segment ahead, so
    // its memory latency passes under the current segment instead of
    // stalling every warp at the segment's start (FP64 has no registers to
    // spare and loads at the start).
    constexpr bool kPrefetch = sizeof(Real) == 4;
    Real xn[1][P], cpn[1][P];
    if constexpr (kPrefetch) load_ckpt(nseg - 1, xn, cpn);

    for (int64_t c = nseg - 1; c >= 0; --c) {
        const uint32_t k0 = (uint32_t)(c * a.ckpt_every);
        const uint32_t k1 = (uint32_t)((int64_t)k0 + a.ckpt_every < (int64_t)a.steps ? k0 + a.ckpt_every : a.steps);
        // ---- replay the segment from its checkpoint --------------------------
        Real x[1][P], cp[1][P];
        if constexpr (kPrefetch) {
#pragma unroll
            for (int i = 0; i < P; ++i) {
                x[0][i] = xn[0][i];
                cp[0][i] = cpn[0][i];
            }
            if (c > 0) load_ckpt(c - 1, xn, cpn);
        } else {
            load_ckpt(c, x, cp);
        }
        // FP32 replays two steps per iteration, as the forward does (more
        // independent work between the special-function unit's waits)
        constexpr int kReplayUnroll = sizeof(Real) == 4 ? 2 : 1;
#pragma unroll kReplayUnroll
        for (uint32_t k = k0; k < k1; ++k) {
            StepRecord<Real, P> rec;
            em_step<M, Real, P, true>(model, x, cp, k, noise, u0, units, a.keys, reduce, &rec);
            if constexpr (M::kDelayedComp) {
                if (((k + 1u) & (kCompPeriod - 1u)) == 0) renormalize_units(x, cp);
            }
            if constexpr (SMEM) {
                if (SDEB_CHECK(a.check, k - k0 < a.ckpt_every, kChkAdjointSeg, k - k0)) {
                    typename SR::Vec *row = vrec + (int)(k - k0) * NV * kForwardBlock;
#pragma unroll
                    for (int v = 0; v < P / V; ++v) {
                        typename SR::Vec vs, vc, vz;
#pragma unroll
                        for (int j = 0; j < V; ++j) {
                            vs.v[j] = model.sn[v * V + j];
                            vc.v[j] = model.cs[v * V + j];
                            vz.v[j] = rec.z[v * V + j];
                        }
                        row[v * kForwardBlock] = vs;
                        row[(P / V + v) * kForwardBlock] = vc;
                        row[(2 * P / V + v) * kForwardBlock] = vz;
                    }
                    prec[(int)(k - k0) * kForwardBlock] = typename SR::Pair{{rec.sums[0], rec.sums[1]}};
                }
            } else if (active && SDEB_CHECK(a.check, k - k0 < a.ckpt_every, kChkAdjointSeg, k - k0)) {
                const int64_t rowi = (int64_t)(k - k0) * a.orbits + o;
                Real *row = seg + rowi * (2 * n);
                store_units<Real, 1, P>(row, units, u0, *reinterpret_cast<const Real(*)[1][P]>(&rec.phase));
                store_units<Real, 1, P>(row + n, units, u0, *reinterpret_cast<const Real(*)[1][P]>(&rec.z));
                if (lig == 0) {
                    seg_sums[2 * rowi] = rec.sums[0];
                    seg_sums[2 * rowi + 1] = rec.sums[1];
                }
            }
        }
        // ---- reverse sweep ---------------------------------------------------
        // (global records: the next row, step k - 1, is loaded while step k
        // is processed)
        Real rn[1][P], zn[1][P], Cn = Real(0), Sn = Real(0);
        (void)SDEB_CHECK(a.check, k1 > k0 && k1 - 1 - k0 < a.ckpt_every, kChkAdjointSeg, k1 - k0);
        if constexpr (!SMEM) load_record(seg, seg_sums, k1 - 1 - k0, a.orbits, o, n, units, u0, rn, zn, Cn, Sn);
        for (uint32_t kk = k1; kk > k0; --kk) {
            const uint32_t k = kk - 1;
            // Padding units: their lambda stays 0 (it starts at 0 and its
            // update is scaled by live), so they add nothing to A, B or the
            // gradients; C and S are the replay's, padding already excluded.
            Real sn[P], cs[P], z[P], C, S;
            if constexpr (SMEM) {
                const typename SR::Vec *row = vrec + (int)(k - k0) * NV * kForwardBlock;
#pragma unroll
                for (int v = 0; v < P / V; ++v) {
                    const typename SR::Vec vs = row[v * kForwardBlock], vc = row[(P / V + v) * kForwardBlock],
                                           vz = row[(2 * P / V + v) * kForwardBlock];
#pragma unroll
                    for (int j = 0; j < V; ++j) {
                        sn[v * V + j] = vs.v[j];
                        cs[v * V + j] = vc.v[j];
                        z[v * V + j] = vz.v[j];
                    }
                }
                const typename SR::Pair cs2 = prec[(int)(k - k0) * kForwardBlock];
                C = cs2.v[0];
                S = cs2.v[1];
            } else {
                Real r[P];
#pragma unroll
                for (int i = 0; i < P; ++i) {
                    r[i] = rn[0][i];
                    z[i] = zn[0][i];
                }
                C = Cn;
                S = Sn;
                if (k > k0) load_record(seg, seg_sums, k - 1 - k0, a.orbits, o, n, units, u0, rn, zn, Cn, Sn);
#pragma unroll
                for (int i = 0; i < P; ++i) sincos_reduced(r[i], sn[i], cs[i]);
            }
            Real A = 0, B = 0;
#pragma unroll
            for (int i = 0; i < P; ++i) {
                A = fma_r(lam[0][i], cs[i], A);
                B = fma_r(lam[0][i], sn[i], B);
            }
            A = group_sum<G>(A);
            B = group_sum<G>(B);
            // parameter gradients use lambda^{k+1}:
            // sum_i lambda_i (S cos x_i - C sin x_i) = S A - C B, the same in every lane of the group
            g_k = fma_r(S, A, fma_r(-C, B, g_k));
#pragma unroll
            for (int i = 0; i < P; ++i) {
                const Real l = lam[0][i];
                g_omega[i] += l;
                g_noise[PAPER ? i : 0] = fma_r(l, z[i], g_noise[PAPER ? i : 0]);
                // lambda^k: cos x_l (A - lambda_l C) + sin x_l (B - lambda_l S)
                const Real jac = fma_r(cs[i], fma_r(-l, C, A), mul_r(sn[i], fma_r(-l, S, B)));
                lam[0][i] = fma_r(kdt_n_live[i], jac, l);
            }
        }
    }

    // per-orbit gradients: p = (K, sigma, omega_1..omega_n) or (K, omega, p_1..p_n)
    if (!PAPER) g_noise[0] = group_sum<G>(g_noise[0]);
    if (active && SDEB_CHECK(a.check, o < a.orbits, kChkAdjointOut, o)) {
        Real *gp = static_cast<Real *>(a.dL_dp) + o * a.d;
        if (lig == 0) {
            gp[0] = g_k * (dt / (Real)units);
            if (!PAPER) gp[1] = g_noise[0] * sqdt;
        }
#pragma unroll
        for (int i = 0; i < P; ++i) {
            const int j = u0 + i;
            if (j < units) {
                gp[(PAPER ? 1 : 2) + j] = g_omega[i] * dt;
                if (PAPER) gp[1 + units + j] = g_noise[PAPER ? i : 0] * sqdt;
            }
        }
        if (a.dL_dx0 != nullptr) store_units<Real, 1, P>(static_cast<Real *>(a.dL_dx0) + o * n, units, u0, lam);
    }
}

// Segment records in shared memory while they take at most this much per
// block (two blocks of 128 threads per SM still fit), else in global memory.
constexpr int64_t kAdjointSmemMax = 112 * 1024;

template <bool PAPER, typename Real, int G, int P>
cudaError_t launch_adjoint_layout(const AdjointArgs &a, cudaStream_t s) {
    const int64_t grid = (a.orbits * G + kForwardBlock - 1) / kForwardBlock;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const int64_t smem = (int64_t)a.ckpt_every * SmemRec<Real, P>::kStepBytes * kForwardBlock;
    const bool fits = smem <= kAdjointSmemMax;
    if (a.records == SDEB_RECORDS_SHARED && !fits) return cudaErrorNotSupported;
    if (fits && a.records != SDEB_RECORDS_GLOBAL) {
        cudaError_t e = cudaFuncSetAttribute(em_adjoint_kernel<PAPER, Real, G, P, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        em_adjoint_kernel<PAPER, Real, G, P, true><<<(unsigned)grid, kForwardBlock, (size_t)smem, s>>>(a);
    } else {
        em_adjoint_kernel<PAPER, Real, G, P, false><<<(unsigned)grid, kForwardBlock, 0, s>>>(a);
    }
    return cudaGetLastError();
}

#define SDEB_ADJOINT_LAYOUT(G_, P_) \
    if (l.G == (G_) && l.P == (P_)) return launch_adjoint_layout<PAPER, Real, G_, P_>(a, s);

template <bool PAPER, typename Real>
cudaError_t dispatch_adjoint(const AdjointArgs &a, Layout l, cudaStream_t s) {
    SDEB_ADJOINT_LAYOUT(1, 1)
    SDEB_ADJOINT_LAYOUT(1, 2)
    SDEB_ADJOINT_LAYOUT(1, 4)
    SDEB_ADJOINT_LAYOUT(1, 8)
    SDEB_ADJOINT_LAYOUT(2, 8)
    SDEB_ADJOINT_LAYOUT(4, 8)
    SDEB_ADJOINT_LAYOUT(8, 8)
    SDEB_ADJOINT_LAYOUT(16, 8)
    SDEB_ADJOINT_LAYOUT(32, 8)
    SDEB_ADJOINT_LAYOUT(2, 4)
    SDEB_ADJOINT_LAYOUT(4, 4)
    SDEB_ADJOINT_LAYOUT(8, 4)
    SDEB_ADJOINT_LAYOUT(16, 4)
    SDEB_ADJOINT_LAYOUT(32, 4)
    SDEB_ADJOINT_LAYOUT(4, 16)
    SDEB_ADJOINT_LAYOUT(8, 16)
    return cudaErrorNotSupported;
}

// out[q] = sum_o in[o][q]: one block per parameter, a fixed-order strided
// sum per thread in FP64, then a fixed-shape tree over the block.
template <typename Real>
__global__ void sum_over_orbits_kernel(const Real *in, int64_t orbits, int32_t d, Real *out) {
    __shared__ double part[256];
    const int q = blockIdx.x;
    double acc = 0.0;
    for (int64_t o = threadIdx.x; o < orbits; o += blockDim.x) acc += (double)in[o * d + q];
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = (Real)part[0];
}

}  // namespace

cudaError_t launch_adjoint(const AdjointArgs &a, Layout l, bool fp64, cudaStream_t s) {
    if (a.model == kKuramoto)
        return fp64 ? dispatch_adjoint<false, double>(a, l, s) : dispatch_adjoint<false, float>(a, l, s);
    if (a.model == kKuramotoPaper)
        return fp64 ? dispatch_adjoint<true, double>(a, l, s) : dispatch_adjoint<true, float>(a, l, s);
    return cudaErrorNotSupported;
}

cudaError_t launch_sum_over_orbits(const void *in, int64_t orbits, int32_t d, bool fp64, void *out,
                                   cudaStream_t s) {
    if (d <= 0) return cudaSuccess;
    if (fp64)
        sum_over_orbits_kernel<double><<<d, 256, 0, s>>>(static_cast<const double *>(in), orbits, d,
                                                          static_cast<double *>(out));
    else
        sum_over_orbits_kernel<float><<<d, 256, 0, s>>>(static_cast<const float *>(in), orbits, d,
                                                         static_cast<float *>(out));
    return cudaGetLastError();
}

}  // namespace sdeb
