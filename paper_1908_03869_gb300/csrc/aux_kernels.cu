// Stand-alone kernels of the path, used for parity checks and by the loss:
//   philox_fill   raw Philox4x32-10 words in the Wiener counter layout (Sec. 2.1.2)
//   normals_fill  the Eq. 3 normals of whole steps, exactly as the integrator draws them
//   order_param   Eq. 7, r = |(1/n) sum_j exp(i theta_j)| and dr/dtheta
#include "em_internal.h"

namespace sdeb {

namespace {

__global__ void philox_fill_kernel(PhiloxKeys keys, uint32_t k0, int64_t nk, uint32_t b0, int64_t nb,
                                   uint32_t o0, int64_t no, uint32_t stream_id, uint4 *out) {
    const int64_t total = nk * nb * no;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = t % no;
        const int64_t b = (t / no) % nb;
        const int64_t k = t / (no * nb);
        U32x4 w = philox4x32_10(k0 + (uint32_t)k, b0 + (uint32_t)b, o0 + (uint32_t)o, stream_id, keys);
        out[t] = make_uint4(w.x, w.y, w.z, w.w);
    }
}

template <typename Real>
__global__ void normals_fill_kernel(PhiloxKeys keys, uint32_t k0, int64_t nk, uint32_t o0, int64_t no,
                                    int32_t m, Real *out) {
    const int32_t nblk = (m + 3) / 4;
    const int64_t total = nk * no * nblk;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t b = (int32_t)(t % nblk);
        const int64_t o = (t / nblk) % no;
        const int64_t k = t / (nblk * no);
        U32x4 w = philox4x32_10(k0 + (uint32_t)k, (uint32_t)b, o0 + (uint32_t)o, 0u, keys);
        Real z[4];
        box_muller<Real>(w.x, w.y, z[0], z[1]);
        box_muller<Real>(w.z, w.w, z[2], z[3]);
        Real *dst = out + (k * no + o) * m + 4 * b;
        for (int q = 0; q < 4 && 4 * b + q < m; ++q) dst[q] = z[q];
    }
}

template <typename Real>
__global__ void order_param_kernel(const Real *theta, int64_t orbits, int32_t n, Real *r, Real *dr) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < orbits;
         o += (int64_t)gridDim.x * blockDim.x) {
        const Real *th = theta + o * n;
        Real C = 0, S = 0;
        for (int j = 0; j < n; ++j) {
            Real s, c;
            sincos_phase(th[j], s, c);
            C += c;
            S += s;
        }
        const Real inv_n = Real(1) / (Real)n;
        C *= inv_n;
        S *= inv_n;
        const Real rr = sqrt(C * C + S * S);
        r[o] = rr;
        if (dr != nullptr) {
            const Real scale = rr > Real(0) ? inv_n / rr : Real(0);
            for (int l = 0; l < n; ++l) {
                Real s, c;
                sincos_phase(th[l], s, c);
                dr[o * n + l] = (S * c - C * s) * scale;
            }
        }
    }
}

__global__ void state_value_kernel(const float *x, const float *comp, int64_t count, float *dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = state_value(x[i], comp[i]);
}

unsigned grid_for(int64_t work, int block) {
    int64_t g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 152 * 64) g = 152 * 64;  // grid-stride loops: a few waves over 152 SMs
    return (unsigned)g;
}

}  // namespace

cudaError_t launch_philox_fill(uint64_t seed, uint32_t k0, int64_t nk, uint32_t b0, int64_t nb,
                               uint32_t o0, int64_t no, uint32_t stream_id, uint32_t *out,
                               cudaStream_t s) {
    const int64_t total = nk * nb * no;
    if (total == 0) return cudaSuccess;
    philox_fill_kernel<<<grid_for(total, 256), 256, 0, s>>>(philox_key_schedule(seed), k0, nk, b0, nb,
                                                            o0, no, stream_id,
                                                            reinterpret_cast<uint4 *>(out));
    return cudaGetLastError();
}

cudaError_t launch_normals_fill(uint64_t seed, uint32_t k0, int64_t nk, uint32_t o0, int64_t no,
                                int32_t m, bool fp64, void *out, cudaStream_t s) {
    const int64_t total = nk * no * ((m + 3) / 4);
    if (total == 0) return cudaSuccess;
    const PhiloxKeys keys = philox_key_schedule(seed);
    if (fp64)
        normals_fill_kernel<double><<<grid_for(total, 256), 256, 0, s>>>(keys, k0, nk, o0, no, m,
                                                                        static_cast<double *>(out));
    else
        normals_fill_kernel<float><<<grid_for(total, 256), 256, 0, s>>>(keys, k0, nk, o0, no, m,
                                                                       static_cast<float *>(out));
    return cudaGetLastError();
}

cudaError_t launch_state_value(const float *x, const float *comp, int64_t count, float *dst, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    state_value_kernel<<<grid_for(count, 256), 256, 0, s>>>(x, comp, count, dst);
    return cudaGetLastError();
}

cudaError_t launch_order_param(const void *theta, int64_t orbits, int32_t n, bool fp64, void *r,
                               void *dr, cudaStream_t s) {
    if (orbits == 0) return cudaSuccess;
    if (fp64)
        order_param_kernel<double><<<grid_for(orbits, 128), 128, 0, s>>>(
            static_cast<const double *>(theta), orbits, n, static_cast<double *>(r),
            static_cast<double *>(dr));
    else
        order_param_kernel<float><<<grid_for(orbits, 128), 128, 0, s>>>(
            static_cast<const float *>(theta), orbits, n, static_cast<float *>(r),
            static_cast<float *>(dr));
    return cudaGetLastError();
}

}  // namespace sdeb
