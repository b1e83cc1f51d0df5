// Bounds checks of the kernels' hand-computed indices, compiled in only with
// -DAFD_CHECK (a debug build of the library; the release build has none).
//
// A check that fails skips the access (the caller guards it) and records, in
// the context's device check block (words kCheckCount.. of the error word
// array), the number of violations, the first violation's code and index.
// Nothing traps or asserts: the kernel keeps running and the host reads the
// record with afd_check_violations().
#pragma once

#include <cstdint>

namespace afd {

// Offsets (in ints) of the check record inside the context's error block.
constexpr int kCheckCount = 8;   // violations so far
constexpr int kCheckCode = 9;    // code of the first one
constexpr int kCheckIndex = 10;  // its index (low 32 bits)

// Check codes: which access was out of range.
enum CheckCode : int {
    kChkStreamSlot = 101,   // streaming kernel: shared-memory slot read
    kChkStreamStore = 102,  // streaming kernel: global store
    kChkStreamTile = 103,   // streaming kernel: tile / chunk decode
    kChkTbSmem = 111,       // temporally blocked kernel: shared-memory stage access
    kChkTbStore = 112,      // temporally blocked kernel: global store
    kChkSmoothSmem = 121,   // smoothing: shared-memory access
    kChkSmoothStore = 122,  // smoothing: global store
    kChkSmoothWeight = 123, // smoothing: weight index
};

#ifdef AFD_CHECK
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

// true if lo <= i < hi; otherwise records a violation (checked build) and
// returns false.  In the release build it is always true and costs nothing.
__device__ __forceinline__ bool check_range(int *block, int64_t i, int64_t lo, int64_t hi,
                                            int code)
{
    if constexpr (!kChecked) {
        return true;
    } else {
        if (i >= lo && i < hi)
            return true;
        if (block) {
            if (atomicAdd(&block[kCheckCount], 1) == 0) {
                block[kCheckCode] = code;
                block[kCheckIndex] = static_cast<int>(i);
            }
        }
        return false;
    }
}

}  // namespace afd
