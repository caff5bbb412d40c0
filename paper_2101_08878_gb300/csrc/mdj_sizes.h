// Size gates of the library's host code that a CPU test can check on its own
// (plain C++, no CUDA headers).
#pragma once

#include <stdint.h>

namespace mdj {

// Output positions of a compaction over m candidate rows come from an
// exclusive scan of m + 1 keep flags; its last entry (the kept total) must
// fit the position type, so 32-bit positions serve only while m + 1 <= 2^32 - 1.
inline constexpr bool compaction_needs_u64_positions(uint64_t m) { return m + 1 > 0xFFFFFFFFull; }

}  // namespace mdj
