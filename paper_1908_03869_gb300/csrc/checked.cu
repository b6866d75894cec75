// The checked build's device status word and its host calls
// (sdeb_check_status, sdeb_check_selftest).  In the unchecked build the
// kernels compile no checks, check_word() is null and both calls return
// SDEB_EUNSUPPORTED without touching the GPU.
#include "em_internal.h"
#include "sdeb.h"

namespace sdeb {
void record_error(const char *msg);  // sdeb_last_error(NULL) text (sdeb_api.cu)
}

namespace {

#ifdef SDEB_CHECKED
__device__ unsigned long long g_check_word;

// Records a violation at site kChkSelftest with index 12345 through the same
// path as a failed check; touches no memory besides the status word.
__global__ void check_selftest_kernel(unsigned long long *word) {
    if (threadIdx.x == 0 && blockIdx.x == 0) (void)SDEB_CHECK(word, false, sdeb::kChkSelftest, 12345);
}
#endif

}  // namespace

namespace sdeb {

unsigned long long *check_word() {
#ifdef SDEB_CHECKED
    // looked up on every launch, with the launching device current (no cache
    // that a replaced context could leave stale)
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_check_word) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return static_cast<unsigned long long *>(p);
#else
    return nullptr;
#endif
}

}  // namespace sdeb

extern "C" sdeb_status sdeb_check_status(uint64_t *word) {
    if (!word) {
        sdeb::record_error("sdeb_check_status: word is NULL");
        return SDEB_EINVAL;
    }
    *word = 0;
#ifdef SDEB_CHECKED
    unsigned long long w = 0, zero = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&w, g_check_word, sizeof w);
    if (e == cudaSuccess && w != 0) e = cudaMemcpyToSymbol(g_check_word, &zero, sizeof zero);
    if (e != cudaSuccess) {
        cudaGetLastError();
        sdeb::record_error("sdeb_check_status: reading the status word failed");
        return SDEB_ECUDA;
    }
    *word = w;
    if (w != 0) {
        sdeb::record_error("bounds check failed (site << 48 | index in the status word)");
        return SDEB_EBOUNDS;
    }
    return SDEB_OK;
#else
    sdeb::record_error("not a checked build (libsdeb_checked.so has the bounds checks)");
    return SDEB_EUNSUPPORTED;
#endif
}

extern "C" sdeb_status sdeb_check_selftest(void *stream) {
#ifdef SDEB_CHECKED
    unsigned long long *w = sdeb::check_word();
    if (!w) {
        sdeb::record_error("sdeb_check_selftest: no status word");
        return SDEB_ECUDA;
    }
    check_selftest_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(w);
    if (cudaGetLastError() != cudaSuccess) {
        sdeb::record_error("sdeb_check_selftest: launch failed");
        return SDEB_ECUDA;
    }
    return SDEB_OK;
#else
    (void)stream;
    sdeb::record_error("not a checked build (libsdeb_checked.so has the bounds checks)");
    return SDEB_EUNSUPPORTED;
#endif
}
