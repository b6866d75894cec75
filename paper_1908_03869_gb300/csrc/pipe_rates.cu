// sdeb_pipe_rate: the issue rate of one arithmetic pipe of this GPU, in
// results per SM per clock, measured by a kernel (no counterpart in the
// paper: the peaks the benchmark divides by).
//
// One block of 1024 threads per SM (its dynamic shared memory is sized so a
// second block cannot fit), each thread running 8 independent chains of
// `iters` dependent operations of the pipe; the block's SM-clock cycles
// between two block barriers (clock64) divide the block's 8192 * iters
// operations.  A rate per clock does not depend on the clock the GPU runs at;
// the benchmark multiplies it by the SM count and the SM clock it samples.
// The chains keep their values bounded (sine of a sine, square roots towards
// 1, the base-2 logarithm of 1 + |x|, contracting fused multiply-adds) and
// one conditional store keeps them live.
#include <algorithm>
#include <vector>

#include "em_internal.h"

namespace sdeb {
void record_error(const char *msg);  // sdeb_last_error(NULL) text (sdeb_api.cu)
}

namespace {

using namespace sdeb;

constexpr int kPipeThreads = 1024;
constexpr int kChains = 8;

template <int PIPE>
__device__ __forceinline__ float op_f32(float x) {
    float r;
    if constexpr (PIPE == 0) {
        asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    } else if constexpr (PIPE == 1) {
        asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        r = fabsf(r) + 1.0f;
    } else if constexpr (PIPE == 2) {
        asm volatile("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    } else {
        r = __fmaf_rn(x, 0.999999f, 1e-7f);
    }
    return r;
}

template <int PIPE>
__global__ void __launch_bounds__(kPipeThreads) pipe_kernel(int iters, long long *cycles, float *sink) {
    extern __shared__ unsigned char pad[];  // occupancy control only
    const float base = 1.0f + 1e-3f * (float)(threadIdx.x & 63);
    long long t0 = 0, t1 = 0;
    float acc = 0.0f;
    if constexpr (PIPE == 3) {
        double a[kChains];
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = (double)base + j;
        __syncthreads();
        t0 = clock64();
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < kChains; ++j) a[j] = __fma_rn(a[j], 0.999999999, 1e-9);
        }
        __syncthreads();
        t1 = clock64();
#pragma unroll
        for (int j = 0; j < kChains; ++j) acc += (float)a[j];
    } else {
        float a[kChains];
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = base + 0.1f * j;
        __syncthreads();
        t0 = clock64();
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < kChains; ++j) a[j] = op_f32<PIPE>(a[j]);
        }
        __syncthreads();
        t1 = clock64();
#pragma unroll
        for (int j = 0; j < kChains; ++j) acc += a[j];
    }
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
    if (acc == 12345.678f) sink[blockIdx.x] = acc + (float)pad[0];
}

template <int PIPE>
cudaError_t run_pipe(int grid, int iters, size_t smem, long long *cycles, float *sink, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(pipe_kernel<PIPE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    pipe_kernel<PIPE><<<grid, kPipeThreads, smem, s>>>(iters, cycles, sink);
    return cudaGetLastError();
}

}  // namespace

extern "C" sdeb_status sdeb_pipe_rate(int32_t pipe, int32_t iters, double *ops_per_clk_per_sm, void *stream) {
    if (!ops_per_clk_per_sm || pipe < 0 || pipe > 4 || iters < 1 || iters > (1 << 24)) {
        record_error("sdeb_pipe_rate: pipe in [0, 4], iters in [1, 2^24] and an output pointer required");
        return SDEB_EINVAL;
    }
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0, smem_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e != cudaSuccess || sms < 1) {
        cudaGetLastError();
        record_error("sdeb_pipe_rate: device query failed");
        return SDEB_ECUDA;
    }
    // more than half of the SM's shared memory: one block per SM
    const size_t smem = (size_t)smem_sm / 2 + 1024;
    long long *d_cycles = nullptr;
    float *d_sink = nullptr;
    e = cudaMallocAsync(&d_cycles, sizeof(long long) * sms, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_sink, sizeof(float) * sms, s);
    if (e == cudaSuccess) {
        // pipe 4 is the FP32 fused multiply-add: op_f32's last branch
        switch (pipe) {
        case 0: e = run_pipe<0>(sms, iters, smem, d_cycles, d_sink, s); break;
        case 1: e = run_pipe<1>(sms, iters, smem, d_cycles, d_sink, s); break;
        case 2: e = run_pipe<2>(sms, iters, smem, d_cycles, d_sink, s); break;
        case 3: e = run_pipe<3>(sms, iters, smem, d_cycles, d_sink, s); break;
        default: e = run_pipe<4>(sms, iters, smem, d_cycles, d_sink, s); break;
        }
    }
    std::vector<long long> cyc((size_t)sms);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cyc.data(), d_cycles, sizeof(long long) * sms, cudaMemcpyDeviceToHost, s);
    if (d_cycles) cudaFreeAsync(d_cycles, s);
    if (d_sink) cudaFreeAsync(d_sink, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        record_error("sdeb_pipe_rate: kernel failed");
        return SDEB_ECUDA;
    }
    std::sort(cyc.begin(), cyc.end());
    const double median = (double)cyc[cyc.size() / 2];
    if (!(median > 0.0)) {
        record_error("sdeb_pipe_rate: no cycles measured");
        return SDEB_ECUDA;
    }
    *ops_per_clk_per_sm = (double)kPipeThreads * kChains * (double)iters / median;
    return SDEB_OK;
}
