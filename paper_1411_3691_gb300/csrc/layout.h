// layout.h -- y-cache layout ranges of the forward launch (plain C++, shared by the plan
// tables and the kernel arguments).
#pragma once

#include <stdint.h>

#include "../../include/mhc.h"

namespace mhc {

constexpr int kMaxFwdRanges = 4;  // launches of fwd_kernel per forward pass, at most

// Work positions [first, first + count) of the family order, whose families all use the
// y-cache layout (yoff, slots): per flavour n slots for rank 1, r n + 1 for rank r >= 2.
struct FwdRange {
  int64_t first, count;
  int slots, yoff[MHC_FMAX];
};

}  // namespace mhc
