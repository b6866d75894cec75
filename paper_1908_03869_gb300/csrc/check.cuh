// Bounds checks of the checked build (compiled with SDEB_CHECKED; the
// library is then libsdeb_checked.so).  At the places where a kernel forms a
// row or table index from run-time data -- an orbit's state row, a frame or
// checkpoint index, an adjoint segment row, a batch's task, item and
// instance tables, its packed-warp lane offsets, a user model's frame index,
// a moment reduction's frame -- the index is compared with the extent of the
// buffer it addresses.  A failed check records (site << 48 | index) in one
// device status word (the first failure wins) and the access is skipped; no
// trap, no fault.  The host reads and clears the word with
// sdeb_check_status.  Without SDEB_CHECKED every check is the constant true
// and costs nothing.
#pragma once

namespace sdeb {

enum CheckSite : unsigned {
    kChkForwardState = 1,
    kChkForwardFrame = 2,
    kChkForwardCkpt = 3,
    kChkAdjointCkpt = 4,
    kChkAdjointSeg = 5,
    kChkAdjointOut = 6,
    kChkBatchItem = 7,
    kChkBatchInstance = 8,
    kChkBatchState = 9,
    kChkBatchFrame = 10,
    kChkBatchParams = 11,
    kChkBatchFlags = 12,
    kChkBatchLane = 13,
    kChkUserFrame = 14,
    kChkMomentFrame = 15,
    kChkSelftest = 0xFFFF
};

#ifdef SDEB_CHECKED
__device__ __forceinline__ bool sdeb_check(unsigned long long *word, bool ok, unsigned site, long long index) {
    if (!ok && word != nullptr)
        atomicCAS(word, 0ull, ((unsigned long long)site << 48) | ((unsigned long long)index & 0xFFFFFFFFFFFFull));
    return ok;
}
#define SDEB_CHECK(word, cond, site, index) ::sdeb::sdeb_check((word), (cond), (site), (long long)(index))
#else
#define SDEB_CHECK(word, cond, site, index) true
#endif

}  // namespace sdeb
