// sf_seqdag.h -- host-side eligibility of the S = 1 dependency-graph path (sf_seqdag.cu).
#pragma once

#include "sf_internal.h"

namespace sfk {

// The graph path sorts every row by Fat counter (bucket x z + slot) with one spare key value, so
// besides w >= kDagMinW it needs w * z < 2^32.
inline bool dag_eligible(uint32_t w, uint32_t z) { return w >= kDagMinW && (uint64_t)w * z < (1ull << 32); }

}  // namespace sfk
