// Engines for half-lengths 16 .. 128 (padded sizes 32 .. 256).
#include "top_unit.cuh"

namespace top {
using Eng16 = Engine<16, 4, 4, 4>;
using Eng32 = Engine<32, 4, 4, 8>;
using Eng64 = Engine<64, 8, 8, 8>;
using Eng128 = Engine<128, 8, 8, 16>;
}  // namespace top

#define LIST(X) X(Eng16) X(Eng32) X(Eng64) X(Eng128)
TOP_DEFINE_UNIT(small, LIST)
TOP_DEFINE_CZT(small, LIST)
