// Drift / diffusion functors of Eq. 1 for the lane-group layout.
//
// An orbit is integrated by G consecutive lanes; lane g owns the P "units"
// u0 = g P .. u0 + P - 1.  A unit is one Wiener channel with its U state
// components (U = 1 for the phase / scalar models, U = 2 for a
// FitzHugh-Nagumo unit (v, w)).  Units at or past `units` are padding: they
// hold zeros, add nothing to the coupling sums and are never stored.
//
// Each functor provides
//   load(p, u0, units, dt, sqdt)      parameters of the orbit into registers
//   prepare(x, cp, u0, units, red)    per-lane partial coupling sums (and any
//                                     per-unit value reused by incr); cp is
//                                     the Kahan compensation (zero in FP64)
//   prepare_stage(z, u0, units, red)  prepare for a stage state of the ODE
//                                     schemes, built on stage_base (no
//                                     compensation word; a phase within a
//                                     step of [-pi, pi] is not reduced again)
//   incr(i, x, red, N, inc)           the Eq. 2 increment f dt + g sqrt(dt) N
//                                     of unit i's components, after red has
//                                     been summed over the G lanes.
//   drift_incr(i, x, red, inc)        f dt alone (the ODE schemes' stages)
//   newton_solve(z, red, r, theta,    r <- (I - theta dt J(z))^-1 r for the
//                u0, units, reduce)   implicit ODE schemes, J the drift's
//                                     Jacobian, after prepare(z) and the sums
//                                     red; padding units do not enter its
//                                     sums.
// State component c of unit j lives at x[c * units + j] in the orbit's row.
#pragma once

#include "em_device.cuh"

namespace sdeb {

// Kuramoto, Eq. 5/6, drift in its mean-field form: with C = sum_j cos x_j and
// S = sum_j sin x_j, sum_j sin(x_j - x_i) = S cos x_i - C sin x_i.
// PAPER = false: p = (K, sigma, omega_1..omega_n); true: p = (K, omega, p_1..p_n).
template <typename Real, int P, bool PAPER>
struct KuramotoLane {
    static constexpr int U = 1;
    static constexpr int NR = 2;
    static constexpr bool kNoise = true;
    static constexpr bool kSplitNoise = !PAPER;  // one noise strength for every unit
    // FP32: compensation folded into x every kCompPeriod steps (the phase
    // the drift reads is x - c, formed anyway by the phase reduction)
    static constexpr bool kDelayedComp = sizeof(Real) == 4;
    Real omega_dt[P];         // omega_i dt
    Real live[P];             // 1 for the orbit's units, 0 for padding
    Real gsq[PAPER ? P : 1];  // noise strength times sqrt(dt)
    Real gsq_bm;              // g sqrt(dt) times the factor box_muller_polar leaves out
    Real kn;                  // K / n
    Real kn_dt;               // (K / n) dt
    Real sn[P], cs[P];

    __device__ __forceinline__ void load(const Real *p, int u0, int units, Real dt, Real sqdt) {
        kn = p[0] / (Real)units;
        kn_dt = mul_r(kn, dt);
        if (!PAPER) {
            gsq[0] = p[1] * sqdt;
            gsq_bm = mul_r(gsq[0], bm_amp_unit<Real>());
        }
#pragma unroll
        for (int i = 0; i < P; ++i) {
            int j = u0 + i;
            bool ok = j < units;
            omega_dt[i] = ok ? mul_r(p[(PAPER ? 1 : 2) + j], dt) : Real(0);
            live[i] = ok ? Real(1) : Real(0);
            if (PAPER) gsq[i] = ok ? p[1 + units + j] * sqdt : Real(0);
        }
    }

    // Base of the ODE schemes' stage states: the compensated phase reduced
    // to [-pi, pi] (sin and cos are 2 pi periodic; the stages see the phase
    // with the rounding of a number below pi).
    __device__ __forceinline__ void stage_base(const Real (&x)[U][P], const Real (&cp)[U][P],
                                               Real (&base)[U][P]) const {
#pragma unroll
        for (int i = 0; i < P; ++i) base[0][i] = reduce_phase(x[0][i], cp[0][i]);
    }

    // Padding units enter the sums with weight 0: fma(1, v, s) == s + v.
    // rph: the phases x - c reduced to [-pi, pi] (FP32) that sin and cos were
    // taken of, kept for the adjoint's replay record.
    Real rph[P];

    __device__ __forceinline__ void prepare(const Real (&x)[U][P], const Real (&cp)[U][P], int, int,
                                            Real (&red)[NR]) {
        Real C = 0, S = 0;
#pragma unroll
        for (int i = 0; i < P; ++i) {
            rph[i] = reduce_phase(x[0][i], cp[0][i]);
            sincos_reduced(rph[i], sn[i], cs[i]);
            C = fma_r(live[i], cs[i], C);
            S = fma_r(live[i], sn[i], S);
        }
        red[0] = C;
        red[1] = S;
    }

    __device__ __forceinline__ void prepare_stage(const Real (&z)[U][P], int, int, Real (&red)[NR]) {
        Real C = 0, S = 0;
#pragma unroll
        for (int i = 0; i < P; ++i) {
            sincos_reduced(z[0][i], sn[i], cs[i]);
            C = fma_r(live[i], cs[i], C);
            S = fma_r(live[i], sn[i], S);
        }
        red[0] = C;
        red[1] = S;
    }

    // f dt = (K/n) dt (S cos x_i - C sin x_i) + omega_i dt, with (K/n) dt S
    // and (K/n) dt C formed once per step (the same products for every unit).
    __device__ __forceinline__ Real drift_dt(int i, const Real (&red)[NR]) const {
        const Real kS = mul_r(kn_dt, red[1]), kC = mul_r(kn_dt, red[0]);
        return fma_r(kS, cs[i], fma_r(-kC, sn[i], omega_dt[i]));
    }

    // f dt + g sqrt(dt) N
    __device__ __forceinline__ void incr(int i, const Real (&x)[U][P], const Real (&red)[NR], Real N,
                                         Real (&inc)[U]) const {
        (void)x;
        const Real kS = mul_r(kn_dt, red[1]), kC = mul_r(kn_dt, red[0]);
        inc[0] = fma_r(kS, cs[i], fma_r(-kC, sn[i], fma_r(gsq[PAPER ? i : 0], N, omega_dt[i])));
    }

    // The scalar noise strength g sqrt(dt) times a Box-Muller amplitude (and
    // the factor the polar form leaves out), once per pair; the increment is
    // then f dt + (g sqrt(dt) amp) trig.
    __device__ __forceinline__ Real noise_scaled(Real amp) const { return mul_r(gsq_bm, amp); }

    __device__ __forceinline__ void incr_split(int i, const Real (&red)[NR], Real amp_scaled, Real trig,
                                               Real (&inc)[U]) const {
        inc[0] = fma_r(amp_scaled, trig, drift_dt(i, red));
    }

    __device__ __forceinline__ void drift_incr(int i, const Real (&)[U][P], const Real (&red)[NR],
                                               Real (&inc)[U]) const {
        inc[0] = drift_dt(i, red);
    }

    // With c_i = cos z_i, s_i = sin z_i the drift's Jacobian is
    // (K/n) (c c^T + s s^T) - diag((K/n) (C c_i + S s_i)), so
    // I - theta dt J = D - beta U U^T with U = [c s], beta = theta (K/n) dt,
    // D = diag(1 + beta (C c_i + S s_i)): solved by the Woodbury identity,
    // w = D^-1 r, m = U^T D^-1 U and q = U^T w summed over the orbit's units,
    // r <- w + beta D^-1 U (I - beta m)^-1 q.  m22 = sum s^2 / a is taken as
    // sum 1 / a - m11 (c^2 + s^2 = 1).  D is nonsingular while theta K dt < 1.
    // Padding units get a zero correction.
    template <class RED>
    __device__ __forceinline__ void newton_solve(const Real (&)[U][P], const Real (&red)[NR], Real (&r)[U][P],
                                                 Real theta, int, int, RED &reduce) const {
        const Real C = red[0], S = red[1], beta = theta * kn_dt;
        Real inv_a[P], m[2] = {Real(0), Real(0)}, q[2] = {Real(0), Real(0)}, ia[1] = {Real(0)};
#pragma unroll
        for (int i = 0; i < P; ++i) {
            inv_a[i] = live[i] * recip_fast(fma_r(beta, fma_r(C, cs[i], mul_r(S, sn[i])), Real(1)));
            const Real w = r[0][i] * inv_a[i];
            const Real tc = cs[i] * inv_a[i];
            r[0][i] = w;
            m[0] = fma_r(cs[i], tc, m[0]);
            m[1] = fma_r(sn[i], tc, m[1]);
            ia[0] += inv_a[i];
            q[0] = fma_r(cs[i], w, q[0]);
            q[1] = fma_r(sn[i], w, q[1]);
        }
        reduce(m);
        reduce(q);
        reduce(ia);
        const Real e11 = Real(1) - beta * m[0], e22 = Real(1) - beta * (ia[0] - m[0]), e12 = -beta * m[1];
        const Real b_det = beta * recip_fast(e11 * e22 - e12 * e12);
        const Real z1 = (e22 * q[0] - e12 * q[1]) * b_det, z2 = (e11 * q[1] - e12 * q[0]) * b_det;
#pragma unroll
        for (int i = 0; i < P; ++i) r[0][i] = fma_r(inv_a[i], fma_r(cs[i], z1, sn[i] * z2), r[0][i]);
    }
};

// Milstein correction for diagonal noise whose channel drives one component
// with g = s x (multiplicative): 1/2 g g' (dW^2 - dt) = 1/2 (s sqrt(dt))^2 x (N^2 - 1).
// (The Milstein scheme, named by the paper as the next integrator in
// Sec. 2.1 and Sec. 3; Kloeden and Platen's form for diagonal noise.)
template <typename Real>
__device__ __forceinline__ Real milstein_multiplicative(Real half_gsq2, Real x, Real N) {
    return half_gsq2 * x * (N * N - Real(1));
}

// FitzHugh-Nagumo network: unit j has v_j = x[j], w_j = x[units + j];
// p = (a, b, eps, I, c, sigma); multiplicative noise sigma v_j dW_j on v only.
// MIL: Milstein step (adds 1/2 g g' (dW^2 - dt) to v) instead of Euler-Maruyama.
template <typename Real, int P, bool MIL>
struct FhnLane {
    static constexpr int U = 2;
    static constexpr int NR = 1;
    static constexpr bool kNoise = true;
    static constexpr bool kSplitNoise = false;
    static constexpr bool kDelayedComp = false;
    Real a, b, eps, I, c, gsq, dt, inv_units;
    Real half_gsq2;  // (sigma sqrt(dt))^2 / 2, the Milstein coefficient

    // Base of the ODE schemes' stage states: the state itself.
    __device__ __forceinline__ void stage_base(const Real (&x)[U][P], const Real (&)[U][P],
                                               Real (&base)[U][P]) const {
#pragma unroll
        for (int c = 0; c < U; ++c)
#pragma unroll
            for (int i = 0; i < P; ++i) base[c][i] = x[c][i];
    }

    __device__ __forceinline__ void load(const Real *p, int, int units, Real dt_, Real sqdt) {
        a = p[0];
        b = p[1];
        eps = p[2];
        I = p[3];
        c = p[4];
        gsq = p[5] * sqdt;
        dt = dt_;
        inv_units = Real(1) / (Real)units;
        half_gsq2 = Real(0.5) * gsq * gsq;
    }

    __device__ __forceinline__ void prepare(const Real (&x)[U][P], const Real (&)[U][P], int u0, int units,
                                            Real (&red)[NR]) {
        Real sv = 0;
#pragma unroll
        for (int i = 0; i < P; ++i)
            if (u0 + i < units) sv += x[0][i];
        red[0] = sv;
    }

    __device__ __forceinline__ void prepare_stage(const Real (&z)[U][P], int u0, int units, Real (&red)[NR]) {
        prepare(z, z, u0, units, red);
    }

    __device__ __forceinline__ void incr(int i, const Real (&x)[U][P], const Real (&red)[NR], Real N,
                                         Real (&inc)[U]) const {
        Real v = x[0][i], w = x[1][i];
        Real mean_v = red[0] * inv_units;
        Real fv = v - v * v * v * Real(1.0 / 3.0) - w + I + c * mean_v - c * v;
        Real fw = eps * (v + a - b * w);
        inc[0] = fv * dt + gsq * v * N;
        if constexpr (MIL) inc[0] += milstein_multiplicative(half_gsq2, v, N);
        inc[1] = fw * dt;
    }

    __device__ __forceinline__ void drift_incr(int i, const Real (&x)[U][P], const Real (&red)[NR],
                                               Real (&inc)[U]) const {
        Real v = x[0][i], w = x[1][i];
        Real mean_v = red[0] * inv_units;
        inc[0] = (v - v * v * v * Real(1.0 / 3.0) - w + I + c * mean_v - c * v) * dt;
        inc[1] = eps * (v + a - b * w) * dt;
    }

    // I - theta dt J is block diagonal, E_i = [[1 - th (1 - v_i^2 - c), th],
    // [-th eps, 1 + th eps b]] with th = theta dt, minus the mean-field
    // coupling's rank-1 term gamma e e^T (e: 1 on every v, gamma = th c / u):
    // by Sherman-Morrison, p = E^-1 r and q = E^-1 e unit by unit, P and Q
    // the sums of their v parts over the orbit's units,
    // r <- p + gamma P / (1 - gamma Q) q.
    template <class RED>
    __device__ __forceinline__ void newton_solve(const Real (&z)[U][P], const Real (&)[NR], Real (&r)[U][P],
                                                 Real theta, int u0, int units, RED &reduce) const {
        const Real th = theta * dt, gamma = th * c * inv_units;
        const Real e12 = th, e21 = -th * eps, e22 = Real(1) + th * eps * b;
        Real qv[P], qw[P], sums[2] = {Real(0), Real(0)};
#pragma unroll
        for (int i = 0; i < P; ++i) {
            const Real v = z[0][i];
            const Real e11 = Real(1) - th * (Real(1) - v * v - c);
            const Real inv_det = Real(1) / (e11 * e22 - e12 * e21);
            const Real pv = (e22 * r[0][i] - e12 * r[1][i]) * inv_det;
            const Real pw = (e11 * r[1][i] - e21 * r[0][i]) * inv_det;
            r[0][i] = pv;
            r[1][i] = pw;
            qv[i] = e22 * inv_det;
            qw[i] = -e21 * inv_det;
            if (u0 + i < units) {
                sums[0] += pv;
                sums[1] += qv[i];
            }
        }
        reduce(sums);
        const Real coef = gamma * sums[0] / (Real(1) - gamma * sums[1]);
#pragma unroll
        for (int i = 0; i < P; ++i) {
            r[0][i] = fma_r(coef, qv[i], r[0][i]);
            r[1][i] = fma_r(coef, qw[i], r[1][i]);
        }
    }
};

// Ornstein-Uhlenbeck (KIND 0), geometric Brownian motion (KIND 1) and the
// linear ODE (KIND 2, no noise): componentwise, no coupling.  MIL: Milstein
// step; only GBM's multiplicative noise has a correction (OU's noise is
// additive, where Milstein equals Euler-Maruyama).
template <typename Real, int P, int KIND, bool MIL = false>
struct ScalarLane {
    static constexpr int U = 1;
    static constexpr int NR = 0;
    static constexpr bool kNoise = KIND != 2;
    static constexpr bool kSplitNoise = false;
    static constexpr bool kDelayedComp = false;
    Real rate, gsq, dt, half_gsq2;

    // Base of the ODE schemes' stage states: the state itself.
    __device__ __forceinline__ void stage_base(const Real (&x)[U][P], const Real (&)[U][P],
                                               Real (&base)[U][P]) const {
#pragma unroll
        for (int i = 0; i < P; ++i) base[0][i] = x[0][i];
    }

    __device__ __forceinline__ void load(const Real *p, int, int, Real dt_, Real sqdt) {
        rate = p[0];
        gsq = KIND == 2 ? Real(0) : p[1] * sqdt;
        dt = dt_;
        half_gsq2 = Real(0.5) * gsq * gsq;
    }

    __device__ __forceinline__ void prepare(const Real (&)[U][P], const Real (&)[U][P], int, int,
                                            Real (&)[NR > 0 ? NR : 1]) {}
    __device__ __forceinline__ void prepare_stage(const Real (&)[U][P], int, int, Real (&)[NR > 0 ? NR : 1]) {}

    __device__ __forceinline__ void incr(int i, const Real (&x)[U][P], const Real (&)[NR > 0 ? NR : 1],
                                         Real N, Real (&inc)[U]) const {
        Real xi = x[0][i];
        if (KIND == 0) inc[0] = -rate * xi * dt + gsq * N;
        if (KIND == 1) {
            inc[0] = rate * xi * dt + gsq * xi * N;
            if constexpr (MIL) inc[0] += milstein_multiplicative(half_gsq2, xi, N);
        }
        if (KIND == 2) inc[0] = -rate * xi * dt;
    }

    __device__ __forceinline__ void drift_incr(int i, const Real (&x)[U][P], const Real (&)[NR > 0 ? NR : 1],
                                               Real (&inc)[U]) const {
        inc[0] = (KIND == 1 ? rate : -rate) * x[0][i] * dt;
    }

    // The drift is lambda x (lambda = rate for GBM, -rate otherwise):
    // I - theta dt J = 1 - theta dt lambda.
    template <class RED>
    __device__ __forceinline__ void newton_solve(const Real (&)[U][P], const Real (&)[NR > 0 ? NR : 1],
                                                 Real (&r)[U][P], Real theta, int, int, RED &) const {
        const Real lambda = KIND == 1 ? rate : -rate;
        const Real inv = Real(1) / (Real(1) - theta * dt * lambda);
#pragma unroll
        for (int i = 0; i < P; ++i) r[0][i] *= inv;
    }
};

}  // namespace sdeb
