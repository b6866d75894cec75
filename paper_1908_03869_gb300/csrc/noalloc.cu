// sdeb_integrate_noalloc: the forward integration for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA graph is
// being captured, allocators with a fixed arena they manage themselves,
// embedded or real-time hosts that forbid allocation after start-up, and
// plugins whose host application owns every device allocation.  The context
// API (sdeb_create) allocates its state, compensation, frame and flag
// buffers, so those callers cannot use it.  This entry point takes every
// input and output from the caller and keeps the only scratch the forward
// kernel needs -- the Kahan compensation word of every FP32 state component
// and the per-orbit status byte -- in a fixed array in the library's own
// device memory.
//
// The scratch is a file-scope __device__ array of kScratchBytes bytes.  Every
// GPU that loads the library holds it until the process exits.  Host code
// cannot use the array's name as a device address (on the host that name
// is only a stand-in), so the first call on each device, with that device
// current, looks the address up with cudaGetSymbolAddress and caches it
// together with the identity of the CUDA context it belongs to.  A later
// call in another context of that device (the primary context released and
// created again, or cudaDeviceReset) finds the identity changed and looks
// the address up again, so a stale address is never handed to a kernel.
// The call that does a look-up should come before any stream capture
// starts: the first call on a device, and the first after its context was
// replaced.  Every call shares the array and it keeps the last call's
// contents: each call clears the part that must start at zero, and calls
// whose work overlaps on the GPU race on it.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "em_internal.h"
#include "sdeb.h"

namespace sdeb {
void record_error(const char *msg);  // sdeb_last_error(NULL) text (sdeb_api.cu)
}

namespace {

using namespace sdeb;

// Maximum problem size of the allocation-free path.
constexpr int64_t kMaxStates = SDEB_NOALLOC_MAX_STATES;   // orbits * n
constexpr int64_t kMaxOrbits = SDEB_NOALLOC_MAX_ORBITS;
constexpr size_t kCompBytes = (size_t)kMaxStates * sizeof(float);
constexpr size_t kScratchBytes = kCompBytes + (size_t)kMaxOrbits;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct ScratchCache {
    unsigned char *ptr;       // device address of g_noalloc_scratch
    unsigned long long ctx;   // identity (cuCtxGetId) of the context it was looked up in
};
ScratchCache g_scratch[kMaxDevices] = {};

// Driver entry points, resolved through the runtime (the library does not
// link the driver library itself).
typedef int (*CtxGetCurrentFn)(void **ctx);
typedef int (*CtxGetIdFn)(void *ctx, unsigned long long *id);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
bool g_driver_resolved = false;

bool resolve_driver_entry_points() {
    if (g_driver_resolved) return g_ctx_get_current != nullptr && g_ctx_get_id != nullptr;
    g_driver_resolved = true;
    void *f1 = nullptr, *f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess) {
        cudaGetLastError();
        return false;
    }
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f2);
    return true;
}

// Identity of the CUDA context current on this thread (0: none current).
bool current_context_id(unsigned long long *id) {
    void *ctx = nullptr;
    if (g_ctx_get_current(&ctx) != 0) return false;
    *id = 0;
    if (ctx == nullptr) return true;
    return g_ctx_get_id(ctx, id) == 0;
}

sdeb_status fail(sdeb_status s, const char *fmt, long long a = 0, long long b = 0) {
    char buf[256];
    snprintf(buf, sizeof buf, fmt, a, b);
    record_error(buf);
    return s;
}

// Device address of the scratch array in the current device's current
// context: the cached one while the context is the one it was looked up in,
// else a fresh look-up.
sdeb_status scratch_address(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(SDEB_ECUDA, "cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices) return fail(SDEB_EUNSUPPORTED, "device index %lld out of range", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!resolve_driver_entry_points()) return fail(SDEB_ECUDA, "driver context queries unavailable");
    unsigned long long ctx = 0;
    if (!current_context_id(&ctx)) return fail(SDEB_ECUDA, "cannot identify the current CUDA context");
    if (ctx == 0 || g_scratch[dev].ptr == nullptr || g_scratch[dev].ctx != ctx) {
        // The runtime makes the device's primary context current here when
        // none was (a fresh thread or process).
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            g_scratch[dev] = ScratchCache{};
            return fail(SDEB_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
        }
        if (!current_context_id(&ctx) || ctx == 0) {
            g_scratch[dev] = ScratchCache{};
            return fail(SDEB_ECUDA, "no CUDA context current after the scratch look-up");
        }
        g_scratch[dev] = ScratchCache{static_cast<unsigned char *>(p), ctx};
    }
    *out = g_scratch[dev].ptr;
    return SDEB_OK;
}

bool shape_ok(const sdeb_problem *pb, int32_t &units) {
    int32_t m, d;
    switch (pb->model) {
    case SDEB_KURAMOTO: m = pb->n; d = pb->n + 2; units = pb->n; break;
    case SDEB_KURAMOTO_PAPER: m = pb->n; d = 2 * pb->n + 1; units = pb->n; break;
    case SDEB_FHN_NET:
        if (pb->n % 2) return false;
        m = pb->n / 2; d = 6; units = pb->n / 2; break;
    case SDEB_OU:
    case SDEB_GBM: m = pb->n; d = 2; units = pb->n; break;
    case SDEB_LINEAR_ODE: m = 0; d = 1; units = pb->n; break;
    default: return false;
    }
    return pb->m == m && pb->d == d;
}

}  // namespace

extern "C" sdeb_status sdeb_integrate_noalloc(const sdeb_problem *pb, const void *params, const void *x0,
                                              void *x_final, void *frames, void *stream) {
    if (!pb || !params || !x0 || !x_final) return fail(SDEB_EINVAL, "pb, params, x0 and x_final must not be NULL");
    int32_t units = 0;
    if (pb->n <= 0 || !shape_ok(pb, units)) return fail(SDEB_EINVAL, "model / n / m / d inconsistent");
    if (pb->orbits <= 0 || !(pb->dt > 0.0) || !std::isfinite(pb->dt) || !std::isfinite(pb->t0) ||
        pb->steps < 0 || pb->steps > 0xffffffffLL || pb->stride < 1 || pb->stride > 0xffffffffLL ||
        (pb->precision != SDEB_FP32_KAHAN && pb->precision != SDEB_FP64) || pb->reserved != 0 ||
        (pb->flags & ~(uint32_t)(SDEB_FLAG_SHARED_PARAMS | SDEB_FLAG_NO_FRAMES | kSchemeFlags)) ||
        !scheme_flags_valid(pb->flags) || pb->orbit_offset < 0 ||
        pb->orbit_offset + pb->orbits > 0x100000000LL)
        return fail(SDEB_EINVAL, "problem fields out of range");
    if (pb->ckpt_every != 0) return fail(SDEB_EUNSUPPORTED, "checkpoints need the context API");
    if (pb->orbits > kMaxOrbits || pb->orbits * (int64_t)pb->n > kMaxStates)
        return fail(SDEB_EINVAL, "orbits=%lld states=%lld exceed the allocation-free limits", (long long)pb->orbits,
                    (long long)(pb->orbits * (int64_t)pb->n));
    Layout layout;
    if (!default_layout(units, layout)) return fail(SDEB_EUNSUPPORTED, "more than 256 units per orbit");

    unsigned char *scratch = nullptr;
    sdeb_status st = scratch_address(&scratch);
    if (st != SDEB_OK) return st;

    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool fp64 = pb->precision == SDEB_FP64;
    const size_t elem = fp64 ? 8 : 4;
    const size_t state_bytes = (size_t)pb->orbits * pb->n * elem;
    const bool want_frames = frames != nullptr && !(pb->flags & SDEB_FLAG_NO_FRAMES);
    float *comp = reinterpret_cast<float *>(scratch);
    uint8_t *flags = scratch + kCompBytes;

    cudaError_t e = cudaMemcpyAsync(x_final, x0, state_bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && !fp64) e = cudaMemsetAsync(comp, 0, (size_t)pb->orbits * pb->n * sizeof(float), s);
    if (e == cudaSuccess && want_frames) e = cudaMemcpyAsync(frames, x0, state_bytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SDEB_ECUDA, "stream-ordered copy failed");
    }
    if (pb->steps == 0) return SDEB_OK;

    ForwardArgs a{};
    a.model = pb->model;
    a.n = pb->n;
    a.units = units;
    a.orbits = pb->orbits;
    a.params = params;
    a.param_stride = (pb->flags & SDEB_FLAG_SHARED_PARAMS) ? 0 : pb->d;
    a.x = x_final;
    a.comp = fp64 ? nullptr : comp;
    a.frames = want_frames ? frames : nullptr;
    a.nframes = want_frames ? pb->steps / pb->stride + 1 : 0;
    a.ckpt = nullptr;
    a.ckpt_comp = nullptr;
    a.ckpt_every = 0;
    a.k_begin = 0;
    a.k_end = (uint32_t)pb->steps;
    a.stride = (uint32_t)pb->stride;
    a.orbit_offset = (uint32_t)pb->orbit_offset;
    a.dt = pb->dt;
    a.flags = flags;
    a.keys = philox_key_schedule(pb->seed);
    a.nckpt = 0;
    a.check = check_word();
    a.milstein = (pb->flags & SDEB_FLAG_MILSTEIN) ? 1 : 0;
    a.rk4 = (pb->flags & SDEB_FLAG_RK4) ? 1 : 0;
    a.implicit = implicit_kind(pb->flags);
    a.final_value = 1;   // no resume on this path: x_final gets the state's value
    e = launch_forward_any(a, layout, fp64, s);
    if (e == cudaErrorNotSupported) return fail(SDEB_EUNSUPPORTED, "no kernel for this model and layout");
    if (e != cudaSuccess) return fail(SDEB_ECUDA, "forward kernel launch failed");
    return SDEB_OK;
}
