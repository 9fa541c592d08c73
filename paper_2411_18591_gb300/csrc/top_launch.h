// Kernel launch and dynamic shared-memory spellings used by every unit.
#pragma once

#ifndef TOP_LAUNCH
#define TOP_LAUNCH(kernel, grid, block, smem, stream, ...) kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__)
#endif

#ifndef TOP_DYN_SMEM
#define TOP_DYN_SMEM(T, name) extern __shared__ T name[]
#endif
