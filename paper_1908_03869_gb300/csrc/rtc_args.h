// Launch arguments of the run-time compiled kernel of a user-defined model.
// Plain data with fixed-width fields: the host code and the NVRTC-compiled
// kernel include this same header, so both see one layout.
#pragma once

namespace sdeb {

struct UserArgs {
    const void *params;   // [orbits][d], or [d] when param_stride == 0
    long long param_stride;
    void *x;              // [orbits][n], updated in place
    float *comp;          // [orbits][n] Kahan compensation (FP32), or null
    void *frames;         // [F][orbits][n], or null
    long long orbits;
    double t0, dt;
    unsigned int k_begin, k_end, stride, orbit_offset;
    unsigned char *flags; // [orbits], bit 0 = non-finite
    PhiloxKeys keys;
    long long nframes;    // frames in frames
    unsigned long long *check;  // bounds-check status word (checked build), or null
};

}  // namespace sdeb
