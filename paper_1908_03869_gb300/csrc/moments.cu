// Ensemble moments of the stored frames, accumulated in FP64 on the GPU.
//
// The paper's accuracy experiment (Sec. 2.3) reports, over realisations, the
// mean and the standard deviation of the Kuramoto order parameter r(t) of
// Eq. 7; an SDE user generally wants the mean and variance over orbits of
// every state component at every output time.  Both are computed here from
// the frames in HBM, whatever the context precision, with FP64 accumulators
// and in a fixed order (the same bits on every call):
//
//   1. a block takes one frame and one chunk of kMomChunk orbits; each thread
//      accumulates its share of one state component (or, for r, one orbit
//      after another) as shifted sums in FP64 -- shift K = the first value
//      it reads, s1 = sum (x - K), s2 = sum (x - K)^2, so mean = K + s1 / c
//      and M2 = s2 - s1^2 / c without cancellation against a large mean;
//   2. the threads' (count, mean, M2) triples of a component are combined
//      in thread order with the pairwise update of Chan, Golub and LeVeque
//      (1979): mean_ab = mean_a + d n_b / n, M2_ab = M2_a + M2_b +
//      d^2 n_a n_b / n, d = mean_b - mean_a;
//   3. a second kernel combines the chunks of a frame in chunk order and
//      writes (mean, M2 / count): the mean and the population variance.
//
// The chunk size is fixed, so a frame's result does not depend on which
// frame range a call asks for.  Reading every frame element once is the HBM
// cost (the forward kernel that wrote them runs ~100x longer).
#include <algorithm>

#include "em_internal.h"

namespace sdeb {

namespace {

constexpr int kMomBlock = 256;

struct Acc {
    double cnt, mean, m2;
};

__device__ __forceinline__ void chan_merge(Acc &a, const Acc &b) {
    if (b.cnt == 0.0) return;
    if (a.cnt == 0.0) {
        a = b;
        return;
    }
    const double n = a.cnt + b.cnt;
    const double d = b.mean - a.mean;
    a.mean = fma(d, b.cnt / n, a.mean);
    a.m2 = a.m2 + b.m2 + d * d * (a.cnt * b.cnt / n);
    a.cnt = n;
}

__device__ __forceinline__ Acc acc_from_shifted(double cnt, double K, double s1, double s2) {
    Acc a{0.0, 0.0, 0.0};
    if (cnt > 0.0) {
        a.cnt = cnt;
        a.mean = K + s1 / cnt;
        a.m2 = fmax(s2 - s1 * (s1 / cnt), 0.0);
    }
    return a;
}

// Per (frame, chunk) block: the moments of every state component over the
// chunk's orbits.  Components cb .. cb + ncomp - 1 are taken 256 at a time;
// thread t reads component comp = t mod ncomp of the orbits row, row + R,
// ... (R = 256 / ncomp rows), so consecutive threads read consecutive
// addresses.
template <typename Real>
__global__ void __launch_bounds__(kMomBlock) state_moments_partial(const Real *frames, int64_t orbits, int n,
                                                                   int64_t f0, int64_t nframes, int C, Acc *part,
                                                                   unsigned long long *check) {
    __shared__ Acc sh[kMomBlock];
    const int c = (int)(blockIdx.x % (unsigned)C);
    const int64_t fr = blockIdx.x / (unsigned)C;
    if (!SDEB_CHECK(check, f0 + fr < nframes, kChkMomentFrame, f0 + fr)) return;  // uniform over the block
    const int64_t o0 = (int64_t)c * kMomChunk;
    const int64_t o1 = min(orbits, o0 + kMomChunk);
    const Real *base = frames + (f0 + fr) * orbits * (int64_t)n;
    const int t = threadIdx.x;
    for (int cb = 0; cb < n; cb += kMomBlock) {
        const int ncomp = min(n - cb, kMomBlock);
        const int R = kMomBlock / ncomp;
        const int row = t / ncomp, comp = cb + (t - row * ncomp);
        double K = 0.0, s1 = 0.0, s2 = 0.0, cnt = 0.0;
        if (row < R) {
            int64_t o = o0 + row;
            if (o < o1) K = (double)base[o * n + comp];
            for (; o < o1; o += R) {
                const double d = (double)base[o * n + comp] - K;
                s1 += d;
                s2 = fma(d, d, s2);
                cnt += 1.0;
            }
        }
        sh[t] = acc_from_shifted(cnt, K, s1, s2);
        __syncthreads();
        if (t < ncomp) {
            Acc m = sh[t];
            for (int r = 1; r < R; ++r) chan_merge(m, sh[r * ncomp + t]);
            part[(fr * C + c) * (int64_t)n + cb + t] = m;
        }
        __syncthreads();
    }
}

// Per (frame, chunk) block: the moments of the order parameter of Eq. 7,
// r = |(1/n) sum_j exp(i theta_j)|, over the chunk's orbits.  A group of G
// lanes (G a power of two, G >= n up to 32) takes one orbit at a time: each
// lane sums cos and sin of components lig, lig + G, ... in the frame's
// precision (FP32: the phase reduced to [-pi, pi] and the special-function
// unit; FP64: CUDA's double sincos), the group adds them by a butterfly, and
// the group's first lane forms r in FP64 and accumulates it.  Every group
// runs the same number of iterations, so the shuffles always have the whole
// warp.
template <typename Real, int G>
__global__ void __launch_bounds__(kMomBlock) r_moments_partial(const Real *frames, int64_t orbits, int n,
                                                               int64_t f0, int64_t nframes, int C, Acc *part,
                                                               unsigned long long *check) {
    constexpr int kGroups = kMomBlock / G;
    __shared__ Acc sh[kGroups];
    const int c = (int)(blockIdx.x % (unsigned)C);
    const int64_t fr = blockIdx.x / (unsigned)C;
    if (!SDEB_CHECK(check, f0 + fr < nframes, kChkMomentFrame, f0 + fr)) return;  // uniform over the block
    const int64_t o0 = (int64_t)c * kMomChunk;
    const int64_t o1 = min(orbits, o0 + kMomChunk);
    const Real *base = frames + (f0 + fr) * orbits * (int64_t)n;
    const int g = threadIdx.x / G, lig = threadIdx.x & (G - 1);
    const int64_t iters = (o1 - o0 + kGroups - 1) / kGroups;
    const double inv_n = 1.0 / (double)n;
    double K = 0.0, s1 = 0.0, s2 = 0.0, cnt = 0.0;
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t o = o0 + g + it * kGroups;
        const bool valid = o < o1;
        Real Cs = Real(0), Ss = Real(0);
        if (valid) {
            const Real *row = base + o * n;
            for (int j = lig; j < n; j += G) {
                Real s, co;
                sincos_phase(row[j], s, co);
                Cs += co;
                Ss += s;
            }
        }
#pragma unroll
        for (int off = 1; off < G; off <<= 1) {
            Cs += __shfl_xor_sync(0xffffffffu, Cs, off);
            Ss += __shfl_xor_sync(0xffffffffu, Ss, off);
        }
        if (valid && lig == 0) {
            const double Cd = (double)Cs, Sd = (double)Ss;
            const double r = sqrt(fma(Cd, Cd, Sd * Sd)) * inv_n;
            if (cnt == 0.0) K = r;
            const double d = r - K;
            s1 += d;
            s2 = fma(d, d, s2);
            cnt += 1.0;
        }
    }
    if (lig == 0) sh[g] = acc_from_shifted(cnt, K, s1, s2);
    __syncthreads();
    if (threadIdx.x == 0) {
        Acc m = sh[0];
        for (int q = 1; q < kGroups; ++q) chan_merge(m, sh[q]);
        part[fr * C + c] = m;
    }
}

// out[i][0..1] = (mean, population variance) of the chunks of item i (an
// item is a (frame, component) pair or a frame), merged in chunk order.
__global__ void merge_chunks(const Acc *part, int64_t items, int per_frame, int C, double *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < items;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t fr = i / per_frame;
        const int q = (int)(i - fr * per_frame);
        Acc m = part[(fr * C) * per_frame + q];
        for (int c = 1; c < C; ++c) chan_merge(m, part[(fr * C + c) * per_frame + q]);
        out[2 * i] = m.mean;
        out[2 * i + 1] = m.cnt > 0.0 ? m.m2 / m.cnt : 0.0;
    }
}

template <typename Real>
cudaError_t launch_r_partial(const Real *frames, int64_t orbits, int n, int64_t f0, int64_t nframes, int C,
                             int64_t blocks, Acc *part, cudaStream_t s) {
    unsigned long long *ck = check_word();
    if (n <= 1) r_moments_partial<Real, 1><<<(unsigned)blocks, kMomBlock, 0, s>>>(frames, orbits, n, f0, nframes, C, part, ck);
    else if (n <= 2) r_moments_partial<Real, 2><<<(unsigned)blocks, kMomBlock, 0, s>>>(frames, orbits, n, f0, nframes, C, part, ck);
    else if (n <= 4) r_moments_partial<Real, 4><<<(unsigned)blocks, kMomBlock, 0, s>>>(frames, orbits, n, f0, nframes, C, part, ck);
    else if (n <= 8) r_moments_partial<Real, 8><<<(unsigned)blocks, kMomBlock, 0, s>>>(frames, orbits, n, f0, nframes, C, part, ck);
    else if (n <= 16) r_moments_partial<Real, 16><<<(unsigned)blocks, kMomBlock, 0, s>>>(frames, orbits, n, f0, nframes, C, part, ck);
    else r_moments_partial<Real, 32><<<(unsigned)blocks, kMomBlock, 0, s>>>(frames, orbits, n, f0, nframes, C, part, ck);
    return cudaGetLastError();
}

unsigned merge_grid(int64_t items) {
    int64_t g = (items + 255) / 256;
    return (unsigned)(g < 1 ? 1 : (g > 152 * 32 ? 152 * 32 : g));
}

}  // namespace

FrameMomentsPlan frame_moments_plan(int64_t orbits, int n, int64_t count) {
    FrameMomentsPlan p;
    p.chunks = (int)((orbits + kMomChunk - 1) / kMomChunk);
    // frames per pass: partials of at most ~64 MiB and at most 2^31 - 1 blocks
    const int64_t per_frame = (int64_t)p.chunks * (n + 1) * (int64_t)sizeof(Acc);
    int64_t fb = std::max<int64_t>(1, (64ll << 20) / per_frame);
    fb = std::min<int64_t>(fb, 0x7fffffffLL / p.chunks);
    p.frames_per_pass = std::max<int64_t>(1, std::min<int64_t>(fb, count));
    p.partial_bytes = (size_t)(p.frames_per_pass * per_frame);
    p.out_bytes = (size_t)p.frames_per_pass * (n + 1) * 2 * sizeof(double);
    return p;
}

cudaError_t launch_frame_moments_pass(const void *frames, bool fp64, int64_t orbits, int n, int64_t f0,
                                      int64_t count, int64_t nframes, const FrameMomentsPlan &plan, void *partial,
                                      double *state_out, double *r_out, cudaStream_t s) {
    unsigned long long *ck = check_word();
    if (count <= 0) return cudaSuccess;
    const int C = plan.chunks;
    const int64_t blocks = (int64_t)C * count;
    Acc *part_state = static_cast<Acc *>(partial);
    Acc *part_r = part_state + count * C * (int64_t)n;
    cudaError_t e = cudaSuccess;
    if (state_out != nullptr) {
        if (fp64)
            state_moments_partial<double><<<(unsigned)blocks, kMomBlock, 0, s>>>(
                static_cast<const double *>(frames), orbits, n, f0, nframes, C, part_state, ck);
        else
            state_moments_partial<float><<<(unsigned)blocks, kMomBlock, 0, s>>>(
                static_cast<const float *>(frames), orbits, n, f0, nframes, C, part_state, ck);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        merge_chunks<<<merge_grid(count * n), 256, 0, s>>>(part_state, count * n, n, C, state_out);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (r_out != nullptr) {
        e = fp64 ? launch_r_partial<double>(static_cast<const double *>(frames), orbits, n, f0, nframes, C, blocks,
                                            part_r, s)
                 : launch_r_partial<float>(static_cast<const float *>(frames), orbits, n, f0, nframes, C, blocks,
                                           part_r, s);
        if (e != cudaSuccess) return e;
        merge_chunks<<<merge_grid(count), 256, 0, s>>>(part_r, count, 1, C, r_out);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace sdeb
