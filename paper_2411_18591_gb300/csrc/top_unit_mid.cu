// Engines for half-lengths 256 and 512 (padded sizes 512 and 1024).
#include "top_unit.cuh"

namespace top {
using Eng256 = Engine<256, 16, 16, 16>;
using Eng512 = Engine<512, 16, 16, 32>;
}  // namespace top

#define LIST(X) X(Eng256) X(Eng512)
TOP_DEFINE_UNIT(mid, LIST)
TOP_DEFINE_CZT(mid, LIST)
