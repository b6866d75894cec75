// The kernel of a user-defined model, compiled at run time by NVRTC (the GPU
// counterpart of the paper's run-time assembly of the OpenCL source from
// the user's model functions, Sec. 2.1.3 and Table 1).  The source is this
// file after em_device.cuh, rtc_args.h and the user's code; the host
// defines SDEB_REAL (float or double), SDEB_N, SDEB_M, SDEB_D (states, Wiener
// channels, parameters) and SDEB_RK4 (1: the ODE path).  The user's code
// provides, for one orbit,
//   __device__ void sdeb_drift(double t, const sdeb_real *x, const sdeb_real *p, sdeb_real *f);
//   __device__ void sdeb_diffusion(double t, const sdeb_real *x, const sdeb_real *p, sdeb_real *g);
// with f[SDEB_N] and g[SDEB_N * SDEB_M] (row-major, g[i * SDEB_M + j]); or, if
// the user's code defines SDEB_DIAGONAL_NOISE, g[SDEB_M] with channel j
// driving state component j alone (g[j] = g_jj), the O(n) form.
//
// One thread integrates one orbit: Eq. 2 with the dense diffusion,
// X_i += f_i dt + sum_j g_ij sqrt(dt) N_j, f and g at the old state and
// t_k = t0 + k dt, the normals N_j from the same Philox counters and
// Box-Muller as the built-in models (block j / 4 of step k and the global
// orbit), FP32 with a Kahan word per state component; or, with SDEB_RK4,
// the classical fourth-order Runge-Kutta step on the drift alone.

namespace sdeb {

__device__ __forceinline__ void rtc_accumulate(float &x, float &c, float inc) { accumulate(x, c, inc); }
__device__ __forceinline__ void rtc_accumulate(double &x, double &, double inc) { x = __dadd_rn(x, inc); }

extern "C" __global__ void sdeb_user_kernel(const UserArgs a) {
    const long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= a.orbits) return;  // no cross-thread exchange: finished threads leave
    constexpr bool kKahan = sizeof(sdeb_real) == 4;
    const sdeb_real *p = static_cast<const sdeb_real *>(a.params) + o * a.param_stride;
    sdeb_real *xrow = static_cast<sdeb_real *>(a.x) + o * SDEB_N;
    sdeb_real x[SDEB_N], c[SDEB_N], f[SDEB_N];
#pragma unroll
    for (int i = 0; i < SDEB_N; ++i) {
        x[i] = xrow[i];
        c[i] = kKahan ? (sdeb_real)a.comp[o * SDEB_N + i] : sdeb_real(0);
    }
    const sdeb_real dt = (sdeb_real)a.dt;
    const sdeb_real sqdt = (sdeb_real)sqrt(a.dt);
    const uint32_t gorb = a.orbit_offset + (uint32_t)o;
    sdeb_real *frames = static_cast<sdeb_real *>(a.frames);
    for (uint32_t k = a.k_begin; k < a.k_end; ++k) {
        const double t = a.t0 + (double)k * a.dt;
#if SDEB_RK4
        sdeb_real acc[SDEB_N], y[SDEB_N];
        sdeb_drift(t, x, p, f);
        for (int i = 0; i < SDEB_N; ++i) {
            acc[i] = f[i];
            y[i] = x[i] + sdeb_real(0.5) * dt * f[i];
        }
        sdeb_drift(t + 0.5 * a.dt, y, p, f);
        for (int i = 0; i < SDEB_N; ++i) {
            acc[i] += sdeb_real(2) * f[i];
            y[i] = x[i] + sdeb_real(0.5) * dt * f[i];
        }
        sdeb_drift(t + 0.5 * a.dt, y, p, f);
        for (int i = 0; i < SDEB_N; ++i) {
            acc[i] += sdeb_real(2) * f[i];
            y[i] = x[i] + dt * f[i];
        }
        sdeb_drift(t + a.dt, y, p, f);
        for (int i = 0; i < SDEB_N; ++i) rtc_accumulate(x[i], c[i], dt * (acc[i] + f[i]) / sdeb_real(6));
#else
        sdeb_drift(t, x, p, f);
#if SDEB_M > 0
#ifdef SDEB_DIAGONAL_NOISE
        sdeb_real g[SDEB_M];
#else
        sdeb_real g[SDEB_N * SDEB_M];
#endif
        sdeb_real z[(SDEB_M + 3) / 4 * 4];
        sdeb_diffusion(t, x, p, g);
#pragma unroll
        for (int b = 0; b < (SDEB_M + 3) / 4; ++b) {
            const U32x4 w = philox4x32_10(k, (uint32_t)b, gorb, 0u, a.keys);
            box_muller<sdeb_real>(w.x, w.y, z[4 * b], z[4 * b + 1]);
            box_muller<sdeb_real>(w.z, w.w, z[4 * b + 2], z[4 * b + 3]);
        }
#endif
#pragma unroll
        for (int i = 0; i < SDEB_N; ++i) {
            sdeb_real noise = 0;
#if SDEB_M > 0
#ifdef SDEB_DIAGONAL_NOISE
            if (i < SDEB_M) noise = g[i] * sqdt * z[i];
#else
#pragma unroll
            for (int j = 0; j < SDEB_M; ++j) noise += g[i * SDEB_M + j] * sqdt * z[j];
#endif
#endif
            rtc_accumulate(x[i], c[i], f[i] * dt + noise);
        }
#endif
        if (frames != nullptr && (k + 1) % a.stride == 0 &&
            SDEB_CHECK(a.check, (long long)((k + 1) / a.stride) < a.nframes, kChkUserFrame, (k + 1) / a.stride)) {
            sdeb_real *fr = frames + ((long long)((k + 1) / a.stride) * a.orbits + o) * SDEB_N;
#pragma unroll
            for (int i = 0; i < SDEB_N; ++i) fr[i] = x[i];
        }
    }
    bool bad = false;
#pragma unroll
    for (int i = 0; i < SDEB_N; ++i) {
        xrow[i] = x[i];
        if (kKahan) a.comp[o * SDEB_N + i] = (float)c[i];
        bad = bad || !isfinite(x[i]);
    }
    a.flags[o] = bad ? 1 : 0;
}

}  // namespace sdeb
