// Engine for half-length 1024 (padded size 2048): 32 x 32, one warp per line.
#include "top_unit.cuh"

namespace top {
using Eng1024 = Engine<1024, 32, 32, 32>;
}  // namespace top

#define LIST(X) X(Eng1024)
TOP_DEFINE_UNIT(m1024, LIST)
TOP_DEFINE_CZT(m1024, LIST)
