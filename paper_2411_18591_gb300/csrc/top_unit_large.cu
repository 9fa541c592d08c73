// Engines for half-lengths 2048 and 4096 (padded sizes 4096 and 8192).
#include "top_unit.cuh"

namespace top {
using Eng2048 = Engine<2048, 64, 16, 16, 8>;
using Eng4096 = Engine<4096, 128, 16, 16, 16>;
}  // namespace top

#define LIST(X) X(Eng2048) X(Eng4096)
TOP_DEFINE_UNIT(large, LIST)
TOP_DEFINE_CZT(large, LIST)
#define SPLIT_LIST(X) X(Eng4096)
TOP_DEFINE_CZT_SPLIT(large, SPLIT_LIST)
