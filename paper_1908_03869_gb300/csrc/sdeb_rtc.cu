// Run-time compilation of user-defined models: the library's step kernel
// (rtc_kernel.cuh, on top of em_device.cuh) and the caller's drift and
// diffusion are compiled together by NVRTC for the current GPU, loaded as a
// CUDA library and launched through the runtime API.  NVRTC is opened on
// first use, so the library itself does not depend on it.
#include <dlfcn.h>
#include <nvrtc.h>

#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "sdeb_rtc.h"

namespace sdeb {

namespace {

// The device sources, embedded at build time from csrc/ (generated file).
#include "sdeb_rtc_sources.inc"

struct Nvrtc {
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
    decltype(&nvrtcGetErrorString) error_string = nullptr;
    bool ok = false;
};

const Nvrtc &nvrtc() {
    static Nvrtc api;
    static std::once_flag once;
    std::call_once(once, [] {
        const char *names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                               "/usr/local/cuda/lib64/libnvrtc.so"};
        void *h = nullptr;
        for (const char *n : names)
            if ((h = dlopen(n, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
        if (!h) return;
        api.create = reinterpret_cast<decltype(api.create)>(dlsym(h, "nvrtcCreateProgram"));
        api.compile = reinterpret_cast<decltype(api.compile)>(dlsym(h, "nvrtcCompileProgram"));
        api.log_size = reinterpret_cast<decltype(api.log_size)>(dlsym(h, "nvrtcGetProgramLogSize"));
        api.log = reinterpret_cast<decltype(api.log)>(dlsym(h, "nvrtcGetProgramLog"));
        api.cubin_size = reinterpret_cast<decltype(api.cubin_size)>(dlsym(h, "nvrtcGetCUBINSize"));
        api.cubin = reinterpret_cast<decltype(api.cubin)>(dlsym(h, "nvrtcGetCUBIN"));
        api.destroy = reinterpret_cast<decltype(api.destroy)>(dlsym(h, "nvrtcDestroyProgram"));
        api.error_string = reinterpret_cast<decltype(api.error_string)>(dlsym(h, "nvrtcGetErrorString"));
        api.ok = api.create && api.compile && api.log_size && api.log && api.cubin_size && api.cubin &&
                 api.destroy && api.error_string;
    });
    return api;
}

std::string assemble(const sdeb_problem &pb, const char *user_source) {
    char prelude[256];
    std::snprintf(prelude, sizeof prelude,
                  "#define SDEB_REAL %s\n#define SDEB_N %d\n#define SDEB_M %d\n#define SDEB_D %d\n#define SDEB_RK4 %d\n",
                  pb.precision == SDEB_FP64 ? "double" : "float", pb.n, pb.m, pb.d,
                  (pb.flags & SDEB_FLAG_RK4) ? 1 : 0);
    std::string src = prelude;
    src += kRtcCheck;
    src += "\n";
    src += kRtcEmDevice;
    src += "\n";
    src += kRtcArgs;
    src += "\ntypedef SDEB_REAL sdeb_real;\n#line 1 \"user_model\"\n";
    src += user_source;
    src += "\n#line 1 \"sdeb_step_kernel\"\n";
    src += kRtcKernel;
    return src;
}

}  // namespace

struct RtcModule {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kernel = nullptr;
};

sdeb_status rtc_build(const sdeb_problem &pb, const char *user_source, RtcModule **out, std::string &log) {
    *out = nullptr;
    const Nvrtc &api = nvrtc();
    if (!api.ok) {
        log = "the run-time compiler library libnvrtc could not be loaded";
        return SDEB_EUNSUPPORTED;
    }
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
        cudaGetLastError();
        major = 10;  // no device: compile for sm_103a (the library's target) so the source is still checked
        minor = 3;
    }
    char arch[64];
    std::snprintf(arch, sizeof arch, "--gpu-architecture=sm_%d%da", major, minor);
    const std::string src = assemble(pb, user_source);
    nvrtcProgram prog = nullptr;
    if (api.create(&prog, src.c_str(), "sdeb_user_model.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
        log = "nvrtcCreateProgram failed";
        return SDEB_EINVAL;
    }
#ifdef SDEB_CHECKED
    const char *opts[] = {arch, "-std=c++17", "-default-device", "-DSDEB_RTC=1", "-DSDEB_CHECKED=1"};
#else
    const char *opts[] = {arch, "-std=c++17", "-default-device", "-DSDEB_RTC=1"};
#endif
    const nvrtcResult rc = api.compile(prog, 4, opts);
    size_t ls = 0;
    api.log_size(prog, &ls);
    log.assign(ls > 1 ? ls - 1 : 0, '\0');
    if (ls > 1) api.log(prog, &log[0]);
    if (rc != NVRTC_SUCCESS) {
        log = std::string(api.error_string(rc)) + "\n" + log;
        api.destroy(&prog);
        return SDEB_EINVAL;
    }
    size_t cs = 0;
    api.cubin_size(prog, &cs);
    std::vector<char> cubin(cs);
    api.cubin(prog, cubin.data());
    api.destroy(&prog);
    RtcModule *m = new RtcModule;
    cudaError_t e = cudaLibraryLoadData(&m->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&m->kernel, m->lib, "sdeb_user_kernel");
    if (e != cudaSuccess) {
        cudaGetLastError();
        log = std::string("loading the compiled kernel failed: ") + cudaGetErrorString(e);
        if (m->lib) cudaLibraryUnload(m->lib);
        delete m;
        return SDEB_ECUDA;
    }
    *out = m;
    return SDEB_OK;
}

cudaError_t rtc_launch(const RtcModule *m, const UserArgs &a, cudaStream_t s) {
    const int block = 128;
    const long long grid = (a.orbits + block - 1) / block;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    UserArgs copy = a;
    void *args[] = {&copy};
    return cudaLaunchKernel(reinterpret_cast<const void *>(m->kernel), dim3((unsigned)grid), dim3(block), args, 0,
                            s);
}

void rtc_release(RtcModule *m) {
    if (!m) return;
    if (m->lib) cudaLibraryUnload(m->lib);
    delete m;
}

}  // namespace sdeb
