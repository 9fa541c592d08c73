// Mixed-radix engines (factors 2, 3, 5) for half-lengths 250, 500, 768 and 1000
// (padded sizes 500, 1000, 1536 and 2000). Line groups of 25 or 50 threads do not
// tile a warp, so their exchanges synchronise the whole block; three stages of radix 10
// (two exchanges a transform) measured faster than the four-stage 4 x 5 x 5 (x 5 or 10)
// plans (1000-point propagation 102 -> 88 us per field before the register caps).
#include "top_unit.cuh"

namespace top {
using Eng250 = Engine<250, 25, 5, 5, 10>;
using Eng500 = Engine<500, 25, 5, 10, 10>;
using Eng768 = Engine<768, 32, 12, 8, 8>;
using Eng1000 = Engine<1000, 50, 10, 10, 10>;
}  // namespace top

#define LIST(X) X(Eng250) X(Eng500) X(Eng768) X(Eng1000)
TOP_DEFINE_UNIT(mixed, LIST)
