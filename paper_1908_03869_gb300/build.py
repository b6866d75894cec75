"""Build the CUDA library libsdeb.so in-tree (paper_1908_03869_gb300/_build/).

Each translation unit under csrc/ is compiled for sm_103a only
(-gencode arch=compute_103a,code=sm_103a), in parallel, then linked into one
shared library with the CUDA runtime linked statically.  No cmake, no
architecture flags for the host compiler (the same command builds on x86_64
and aarch64 hosts).
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_NAME = "libsdeb.so"
LIB_PATH = os.path.join(BUILD_DIR, LIB_NAME)
# The bounds-checked build: the same sources compiled with SDEB_CHECKED.
CHECKED_BUILD_DIR = os.path.join(HERE, "_build_checked")
CHECKED_LIB_PATH = os.path.join(CHECKED_BUILD_DIR, "libsdeb_checked.so")

GEN_DIR = os.path.join(BUILD_DIR, "gen")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
              "-I" + INCLUDE, "-I" + CSRC, "-I" + GEN_DIR]

# Device sources compiled again at run time for user-defined models (NVRTC):
# embedded into the library as string constants, one per file.
RTC_EMBED = [("kRtcCheck", "check.cuh"), ("kRtcEmDevice", "em_device.cuh"), ("kRtcArgs", "rtc_args.h"),
             ("kRtcKernel", "rtc_kernel.cuh")]
RTC_INC = os.path.join(GEN_DIR, "sdeb_rtc_sources.inc")


def generate_rtc_sources():
    parts = ["// Generated by build.py from csrc/: the device sources of the run-time compiled kernel.\n"]
    for name, fname in RTC_EMBED:
        with open(os.path.join(CSRC, fname)) as f:
            text = f.read()
        if ")SDEBRTC" in text:
            raise RuntimeError("%s contains the raw-string delimiter" % fname)
        parts.append('static const char %s[] = R"SDEBRTC(%s)SDEBRTC";\n' % (name, text))
    content = "".join(parts)
    os.makedirs(GEN_DIR, exist_ok=True)
    if os.path.exists(RTC_INC):
        with open(RTC_INC) as f:
            if f.read() == content:
                return
    with open(RTC_INC, "w") as f:
        f.write(content)


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return hs + [os.path.join(INCLUDE, "sdeb.h")]


def needs_build(checked=False):
    lib = CHECKED_LIB_PATH if checked else LIB_PATH
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in sources() + headers() + [os.path.abspath(__file__)])


def _compile(src, verbose_ptxas=False, checked=False):
    obj = os.path.join(CHECKED_BUILD_DIR if checked else BUILD_DIR, os.path.basename(src)[:-3] + ".o")
    cmd = [_nvcc()] + ARCH + NVCC_FLAGS + (["-DSDEB_CHECKED=1"] if checked else []) + ["-c", src, "-o", obj]
    if verbose_ptxas:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s" % (src, r.stderr))
    return obj, r.stderr


def build(force=False, verbose_ptxas=False, jobs=None, checked=False):
    """Build libsdeb.so, or with checked=True the bounds-checked
    libsdeb_checked.so (every kernel compiled with SDEB_CHECKED)."""
    lib = CHECKED_LIB_PATH if checked else LIB_PATH
    if not force and not needs_build(checked):
        return lib
    os.makedirs(CHECKED_BUILD_DIR if checked else BUILD_DIR, exist_ok=True)
    os.makedirs(GEN_DIR, exist_ok=True)
    generate_rtc_sources()
    srcs = sources()
    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    with concurrent.futures.ThreadPoolExecutor(max_workers=jobs) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose_ptxas, checked), srcs))
    if verbose_ptxas:
        for _, log in results:
            sys.stderr.write(log)
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [_nvcc()] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results] + ["-cudart", "static", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stderr)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv, checked="--checked" in sys.argv))
