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
//   dL/dK      += (dt / n) sum_i lambda^{k+1}_i (S cos x_i - C sin x_i),
//   dL/domega_i += dt lambda^{k+1}_i,
//   dL/dg      += sqrt(dt) sum_i lambda^{k+1}_i N^k_i   (g = sigma, or p_i per unit),
// and dL/dtheta^0 = lambda^0.
//
// States are recomputed segment by segment from the checkpoints the forward
// pass stored every ckpt_every steps, with the same step code (bit-identical
// trajectory).  The forward pass stores no noise: the replay regenerates the
// Philox normals of each step (they drive the recomputed states), and keeps
// them, with the step's reduced phase (FP32: x - c folded into [-pi, pi])
// and the orbit's coupling sums C and S, in a segment buffer that the
// reverse sweep of the same segment reads back (the sweep takes sin and cos
// of the phase again, but not C and S).
#include <type_traits>

#include "em_forward_impl.cuh"

namespace sdeb {

namespace {

template <bool PAPER, typename Real, int G, int P>
__global__ void __launch_bounds__(kForwardBlock) em_adjoint_kernel(const AdjointArgs a) {
    using M = KuramotoLane<Real, P, PAPER>;
    static_assert(P == 1 || P == 2 || P % 4 == 0, "a lane holds 1, 2 or a multiple of 4 units");
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

    for (int64_t c = nseg - 1; c >= 0; --c) {
        const uint32_t k0 = (uint32_t)(c * a.ckpt_every);
        const uint32_t k1 = (uint32_t)((int64_t)k0 + a.ckpt_every < (int64_t)a.steps ? k0 + a.ckpt_every : a.steps);
        // ---- replay the segment from its checkpoint --------------------------
        Real x[1][P], cp[1][P];
        if (SDEB_CHECK(a.check, c < a.nckpt, kChkAdjointCkpt, c)) {
            load_units<Real, 1, P>(ckpt + (c * a.orbits + o) * n, units, u0, x);
        } else {
#pragma unroll
            for (int i = 0; i < P; ++i) x[0][i] = Real(0);
        }
        if constexpr (std::is_same<Real, float>::value) {
            if (c < a.nckpt) {
                load_units<float, 1, P>(a.ckpt_comp + (c * a.orbits + o) * n, units, u0, cp);
            } else {
#pragma unroll
                for (int i = 0; i < P; ++i) cp[0][i] = 0.0f;
            }
        } else {
#pragma unroll
            for (int i = 0; i < P; ++i) cp[0][i] = Real(0);
        }
        for (uint32_t k = k0; k < k1; ++k) {
            StepRecord<Real, P> rec;
            em_step<M, Real, P, true>(model, x, cp, k, noise, u0, units, a.keys, reduce, &rec);
            if constexpr (M::kDelayedComp) {
                if (((k + 1u) & (kCompPeriod - 1u)) == 0) renormalize_units(x, cp);
            }
            if (active && SDEB_CHECK(a.check, k - k0 < a.ckpt_every, kChkAdjointSeg, k - k0)) {
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
        // the next row (step k - 1) is loaded while step k is processed
        Real rn[1][P], zn[1][P], Cn, Sn;
        (void)SDEB_CHECK(a.check, k1 > k0 && k1 - 1 - k0 < a.ckpt_every, kChkAdjointSeg, k1 - k0);
        {
            const int64_t rowi = (int64_t)(k1 - 1 - k0) * a.orbits + o;
            const Real *row = seg + rowi * (2 * n);
            load_units<Real, 1, P>(row, units, u0, rn);
            load_units<Real, 1, P>(row + n, units, u0, zn);
            Cn = seg_sums[2 * rowi];
            Sn = seg_sums[2 * rowi + 1];
        }
        for (uint32_t kk = k1; kk > k0; --kk) {
            const uint32_t k = kk - 1;
            Real r[1][P], z[1][P];
#pragma unroll
            for (int i = 0; i < P; ++i) {
                r[0][i] = rn[0][i];
                z[0][i] = zn[0][i];
            }
            const Real C = Cn, S = Sn;
            if (k > k0) {
                const int64_t rowi = (int64_t)(k - 1 - k0) * a.orbits + o;
                const Real *row = seg + rowi * (2 * n);
                load_units<Real, 1, P>(row, units, u0, rn);
                load_units<Real, 1, P>(row + n, units, u0, zn);
                Cn = seg_sums[2 * rowi];
                Sn = seg_sums[2 * rowi + 1];
            }
            // Padding units: their lambda stays 0 (it starts at 0 and its
            // update is scaled by live), so they add nothing to A, B or the
            // gradients; C and S are the replay's, padding already excluded.
            Real sn[P], cs[P];
            Real A = 0, B = 0;
#pragma unroll
            for (int i = 0; i < P; ++i) {
                sincos_reduced(r[0][i], sn[i], cs[i]);
                A = fma_r(lam[0][i], cs[i], A);
                B = fma_r(lam[0][i], sn[i], B);
            }
            A = group_sum<G>(A);
            B = group_sum<G>(B);
#pragma unroll
            for (int i = 0; i < P; ++i) {
                const Real l = lam[0][i];
                // parameter gradients use lambda^{k+1}
                g_k = fma_r(l, fma_r(S, cs[i], -mul_r(C, sn[i])), g_k);
                g_omega[i] += l;
                g_noise[PAPER ? i : 0] = fma_r(l, z[0][i], g_noise[PAPER ? i : 0]);
                // lambda^k
                const Real jac = fma_r(cs[i], A, mul_r(sn[i], B)) - l * fma_r(cs[i], C, mul_r(sn[i], S));
                lam[0][i] = fma_r(kdt_n_live[i], jac, l);
            }
        }
    }

    // per-orbit gradients: p = (K, sigma, omega_1..omega_n) or (K, omega, p_1..p_n)
    g_k = group_sum<G>(g_k);
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

template <bool PAPER, typename Real, int G, int P>
cudaError_t launch_adjoint_layout(const AdjointArgs &a, cudaStream_t s) {
    const int64_t grid = (a.orbits * G + kForwardBlock - 1) / kForwardBlock;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    em_adjoint_kernel<PAPER, Real, G, P><<<(unsigned)grid, kForwardBlock, 0, s>>>(a);
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
