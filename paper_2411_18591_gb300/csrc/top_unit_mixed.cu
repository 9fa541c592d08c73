// Mixed-radix engines (factors 2, 3, 5) for half-lengths 250, 500, 768 and 1000
// (padded sizes 500, 1000, 1536 and 2000). Line groups of 25 or 50 threads do not
// tile a warp, so their exchanges synchronise the whole block; three stages of radix 10
// (two exchanges a transform) measured faster than the four-stage 4 x 5 x 5 (x 5 or 10)
// plans (1000-point propagation 102 -> 88 us per field before the register caps). The 500-point
// plan takes 50 threads a line (10 samples a thread: 19.8 -> 17.5 us per propagation); 100 threads
// a line measured slower for the 1000-point one (65.8 -> 81.6 us).
#include "top_unit.cuh"

namespace top {
using Eng250 = Engine<250, 25, 5, 5, 10>;
#ifndef TOP_G500
#define TOP_G500 50
#endif
using Eng500 = Engine<500, TOP_G500, 5, 10, 10>;
using Eng768 = Engine<768, 32, 12, 8, 8>;
#ifndef TOP_G1000
#define TOP_G1000 50
#endif
using Eng1000 = Engine<1000, TOP_G1000, 10, 10, 10>;
}  // namespace top

#define LIST(X) X(Eng250) X(Eng500) X(Eng768) X(Eng1000)
TOP_DEFINE_UNIT(mixed, LIST)
