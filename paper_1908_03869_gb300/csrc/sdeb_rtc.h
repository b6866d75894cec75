// Run-time compilation of user-defined models (host side).
#pragma once

#include <string>

#include "em_internal.h"
#include "rtc_args.h"
#include "sdeb.h"

namespace sdeb {

struct RtcModule;

// Compiles the step kernel of a user-defined model with NVRTC for the
// current device (n, m, d, precision and the Runge-Kutta flag from pb) and
// loads it.  On failure returns SDEB_EINVAL (the source does not compile;
// `log` holds the compiler's messages), SDEB_EUNSUPPORTED (libnvrtc cannot
// be loaded) or SDEB_ECUDA (the kernel cannot be loaded on the device).
sdeb_status rtc_build(const sdeb_problem &pb, const char *user_source, RtcModule **out, std::string &log);

// Launches the compiled kernel: one thread per orbit.
cudaError_t rtc_launch(const RtcModule *m, const UserArgs &a, cudaStream_t s);

void rtc_release(RtcModule *m);

}  // namespace sdeb
