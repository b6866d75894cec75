// Particle swarm search over model parameters (sdeb_swarm_*, declared in
// include/sdeb.h): the population-based parameter optimisation the paper
// builds the integrator for (Sec. 1.2).  Three small kernels around the
// integration of a generation, all on the caller's stream:
//   expand   particles -> the per-orbit parameter rows the integrator reads
//   fitness  the order parameter of Eq. 7 of every realisation, averaged per
//            particle, squared distance to the target (one warp a particle)
//   update   personal bests, the global best, velocities and positions of the
//            inertia-weight swarm (one block: the global best is a reduction
//            over all particles between the two element-wise phases)
#include <cmath>
#include <cstdint>
#include <cstdio>

#include "em_internal.h"

namespace sdeb {
void record_error(const char *msg);  // sdeb_last_error(NULL) text (sdeb_api.cu)
}

namespace {

using namespace sdeb;

struct DimColumns {
    int32_t col[SDEB_SWARM_MAX_DIMS];  // parameter column of each searched dimension
};

struct UpdateArgs {
    double *x, *v, *pbest, *pbest_fit;
    const double *fit;
    int32_t *gbest;
    int64_t particles;
    int32_t dims;
    double lo[SDEB_SWARM_MAX_DIMS], hi[SDEB_SWARM_MAX_DIMS], vmax[SDEB_SWARM_MAX_DIMS];
    double w, c1, c2;
    PhiloxKeys keys;
    uint32_t generation;
};

constexpr int kUpdateBlock = 1024;
constexpr int kFitnessBlock = 256;

sdeb_status fail(sdeb_status s, const char *fmt, long long a = 0, long long b = 0) {
    char buf[256];
    snprintf(buf, sizeof buf, fmt, a, b);
    record_error(buf);
    return s;
}

sdeb_status launched(const char *what) {
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return SDEB_OK;
    char buf[256];
    snprintf(buf, sizeof buf, "%s launch failed: %s", what, cudaGetErrorString(e));
    record_error(buf);
    return SDEB_ECUDA;
}

unsigned grid_for(int64_t work, int block) {
    int64_t g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 152 * 32) g = 152 * 32;  // grid-stride loops
    return (unsigned)g;
}

template <typename Real>
__global__ void swarm_expand_kernel(const double *x, int64_t particles, int32_t dims, DimColumns cols,
                                    const Real *base, int32_t d, int32_t realisations, Real *out) {
    const int64_t total = particles * realisations * d;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = (int32_t)(t % d);
        const int64_t i = t / ((int64_t)d * realisations);
        Real val = base[c];
        for (int32_t j = 0; j < dims; ++j)
            if (cols.col[j] == c) val = (Real)x[i * dims + j];
        out[t] = val;
    }
}

// One warp per particle: lane l takes realisations l, l + 32, ...; r of a
// realisation as Eq. 7 (sums of cos and sin in column order, divided by n);
// the lanes' partial sums are then added by a butterfly, a fixed order.
template <typename Real>
__global__ void __launch_bounds__(kFitnessBlock) swarm_fitness_kernel(const Real *theta, int64_t particles,
                                                                      int32_t realisations, int32_t n,
                                                                      double r_target, double *fit) {
    const int64_t warps = (int64_t)gridDim.x * (kFitnessBlock / 32);
    const int lane = threadIdx.x & 31;
    for (int64_t i = (int64_t)blockIdx.x * (kFitnessBlock / 32) + (threadIdx.x >> 5); i < particles; i += warps) {
        double acc = 0.0;
        for (int32_t q = lane; q < realisations; q += 32) {
            const Real *th = theta + (i * realisations + q) * (int64_t)n;
            double C = 0.0, S = 0.0;
            for (int32_t j = 0; j < n; ++j) {
                double s, c;
                sincos((double)th[j], &s, &c);
                C += c;
                S += s;
            }
            C /= n;
            S /= n;
            acc += sqrt(C * C + S * S);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            const double dev = acc / realisations - r_target;
            fit[i] = dev * dev;
        }
    }
}

__global__ void __launch_bounds__(kUpdateBlock) swarm_update_kernel(const UpdateArgs a) {
    __shared__ double s_val[kUpdateBlock];
    __shared__ int64_t s_idx[kUpdateBlock];
    const int64_t P = a.particles;
    const int D = a.dims;
    // 1. personal bests (a NaN fitness compares false and never improves)
    for (int64_t i = threadIdx.x; i < P; i += kUpdateBlock) {
        const double f = a.fit[i];
        if (f < a.pbest_fit[i]) {
            a.pbest_fit[i] = f;
            for (int j = 0; j < D; ++j) a.pbest[i * D + j] = a.x[i * D + j];
        }
    }
    __syncthreads();
    // 2. global best: the least personal best, the lowest index among equals
    double best = INFINITY;
    int64_t idx = INT64_MAX;
    for (int64_t i = threadIdx.x; i < P; i += kUpdateBlock) {
        const double f = a.pbest_fit[i];
        if (f < best || (f == best && i < idx)) {
            best = f;
            idx = i;
        }
    }
    s_val[threadIdx.x] = best;
    s_idx[threadIdx.x] = idx;
    __syncthreads();
    for (int half = kUpdateBlock / 2; half > 0; half >>= 1) {
        if ((int)threadIdx.x < half) {
            const double fo = s_val[threadIdx.x + half];
            const int64_t io = s_idx[threadIdx.x + half];
            if (fo < s_val[threadIdx.x] || (fo == s_val[threadIdx.x] && io < s_idx[threadIdx.x])) {
                s_val[threadIdx.x] = fo;
                s_idx[threadIdx.x] = io;
            }
        }
        __syncthreads();
    }
    const int64_t b = s_idx[0] == INT64_MAX ? 0 : s_idx[0];
    if (threadIdx.x == 0) *a.gbest = (int32_t)b;
    // 3. velocities and positions, each operation rounded on its own
    for (int64_t t = threadIdx.x; t < P * D; t += kUpdateBlock) {
        const int64_t i = t / D;
        const int j = (int)(t % D);
        const U32x4 wd = philox4x32_10(a.generation, (uint32_t)j, (uint32_t)i, 2u, a.keys);
        const double r1 = uniform_f64(wd.x), r2 = uniform_f64(wd.y);
        const double xi = a.x[t];
        const double inertia = __dmul_rn(a.w, a.v[t]);
        const double cog = __dmul_rn(__dmul_rn(a.c1, r1), __dsub_rn(a.pbest[t], xi));
        const double soc = __dmul_rn(__dmul_rn(a.c2, r2), __dsub_rn(a.pbest[b * D + j], xi));
        double vn = __dadd_rn(__dadd_rn(inertia, cog), soc);
        vn = vn < -a.vmax[j] ? -a.vmax[j] : vn;
        vn = vn > a.vmax[j] ? a.vmax[j] : vn;
        double xn = __dadd_rn(xi, vn);
        xn = xn < a.lo[j] ? a.lo[j] : xn;
        xn = xn > a.hi[j] ? a.hi[j] : xn;
        a.v[t] = vn;
        a.x[t] = xn;
    }
}

cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

}  // namespace

extern "C" sdeb_status sdeb_swarm_expand(const double *x, int64_t particles, int32_t dims_count, const int32_t *dims,
                                         const void *base, int32_t d, int32_t realisations, int32_t precision,
                                         void *params_out, void *stream) {
    if (!x || !dims || !base || !params_out)
        return fail(SDEB_EINVAL, "x, dims, base and params_out must not be NULL");
    if (particles < 1 || realisations < 1 || d < 1)
        return fail(SDEB_EINVAL, "particles, realisations and d must be positive");
    if (dims_count < 1 || dims_count > SDEB_SWARM_MAX_DIMS)
        return fail(SDEB_EINVAL, "dims_count must be in [1, %lld]", SDEB_SWARM_MAX_DIMS);
    if (precision != SDEB_FP32_KAHAN && precision != SDEB_FP64) return fail(SDEB_EINVAL, "unknown precision");
    DimColumns cols{};
    for (int32_t j = 0; j < dims_count; ++j) {
        if (dims[j] < 0 || dims[j] >= d) return fail(SDEB_EINVAL, "dims[%lld] = %lld is not a column", j, dims[j]);
        for (int32_t k = 0; k < j; ++k)
            if (dims[k] == dims[j]) return fail(SDEB_EINVAL, "column %lld searched twice", dims[j]);
        cols.col[j] = dims[j];
    }
    const int64_t total = particles * realisations * d;
    const unsigned grid = grid_for(total, 256);
    if (precision == SDEB_FP64)
        swarm_expand_kernel<double><<<grid, 256, 0, as_stream(stream)>>>(
            x, particles, dims_count, cols, static_cast<const double *>(base), d, realisations,
            static_cast<double *>(params_out));
    else
        swarm_expand_kernel<float><<<grid, 256, 0, as_stream(stream)>>>(
            x, particles, dims_count, cols, static_cast<const float *>(base), d, realisations,
            static_cast<float *>(params_out));
    return launched("sdeb_swarm_expand");
}

extern "C" sdeb_status sdeb_swarm_fitness(const void *theta, int64_t particles, int32_t realisations, int32_t n,
                                          int32_t precision, double r_target, double *fit, void *stream) {
    if (!theta || !fit) return fail(SDEB_EINVAL, "theta and fit must not be NULL");
    if (particles < 1 || realisations < 1 || n < 1)
        return fail(SDEB_EINVAL, "particles, realisations and n must be positive");
    if (precision != SDEB_FP32_KAHAN && precision != SDEB_FP64) return fail(SDEB_EINVAL, "unknown precision");
    const unsigned grid = grid_for(particles * 32, kFitnessBlock);
    if (precision == SDEB_FP64)
        swarm_fitness_kernel<double><<<grid, kFitnessBlock, 0, as_stream(stream)>>>(
            static_cast<const double *>(theta), particles, realisations, n, r_target, fit);
    else
        swarm_fitness_kernel<float><<<grid, kFitnessBlock, 0, as_stream(stream)>>>(
            static_cast<const float *>(theta), particles, realisations, n, r_target, fit);
    return launched("sdeb_swarm_fitness");
}

extern "C" sdeb_status sdeb_swarm_update(double *x, double *v, double *pbest, double *pbest_fit, const double *fit,
                                         int64_t particles, int32_t dims_count, const double *lo, const double *hi,
                                         double w, double c1, double c2, uint64_t seed, uint32_t generation,
                                         int32_t *gbest, void *stream) {
    if (!x || !v || !pbest || !pbest_fit || !fit || !lo || !hi || !gbest)
        return fail(SDEB_EINVAL, "swarm arrays and bounds must not be NULL");
    if (particles < 1 || particles > (1LL << 24)) return fail(SDEB_EINVAL, "particles must be in [1, 2^24]");
    if (dims_count < 1 || dims_count > SDEB_SWARM_MAX_DIMS)
        return fail(SDEB_EINVAL, "dims_count must be in [1, %lld]", SDEB_SWARM_MAX_DIMS);
    UpdateArgs a{};
    for (int32_t j = 0; j < dims_count; ++j) {
        if (!(lo[j] <= hi[j])) return fail(SDEB_EINVAL, "lo[%lld] > hi[%lld] (or NaN)", j, j);
        a.lo[j] = lo[j];
        a.hi[j] = hi[j];
        a.vmax[j] = hi[j] - lo[j];
    }
    a.x = x;
    a.v = v;
    a.pbest = pbest;
    a.pbest_fit = pbest_fit;
    a.fit = fit;
    a.gbest = gbest;
    a.particles = particles;
    a.dims = dims_count;
    a.w = w;
    a.c1 = c1;
    a.c2 = c2;
    a.keys = philox_key_schedule(seed);
    a.generation = generation;
    swarm_update_kernel<<<1, kUpdateBlock, 0, as_stream(stream)>>>(a);
    return launched("sdeb_swarm_update");
}
