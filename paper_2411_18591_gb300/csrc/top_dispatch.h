// Registry of the instantiated FFT engines (one translation unit per group so the
// build compiles them in parallel).
#pragma once

#include <cuda_runtime.h>

#include "top_internal.h"

namespace top {

struct EngineInfo {
  int M;      // line length handled (half of an even padded size)
  int G;      // threads per line
  int NS;     // number of radix stages
  int R[4];   // radices
  int tw_size;
  int rows;         // rows per block of the row passes
  size_t row_smem;  // shared memory of a row block before any staged planes
};

// PASS_ROWS_CHAIN: the inverse row pass of one propagation fused with the forward row pass of
// the next (the second parameter block).
enum PassKind : int { PASS_ROWS_FWD = 0, PASS_COLS = 1, PASS_ROWS_INV = 2, PASS_ROWS_CHAIN = 3 };

#define TOP_DECLARE_UNIT(name)                                                                        \
  bool engine_info_##name(int M, EngineInfo* info);                                                   \
  cudaError_t launch_pass_##name(int kind, int M, const PassParams& p, const PassParams* next, cudaStream_t s, \
                                 bool* found);

TOP_DECLARE_UNIT(small)
TOP_DECLARE_UNIT(mid)
TOP_DECLARE_UNIT(m1024)
TOP_DECLARE_UNIT(large)
TOP_DECLARE_UNIT(mixed)

#undef TOP_DECLARE_UNIT

// Bluestein line transforms (CztParams) on the power-of-two engines of a unit.
cudaError_t launch_czt_small(int M, const CztParams& p, cudaStream_t s, bool* found);
cudaError_t launch_czt_mid(int M, const CztParams& p, cudaStream_t s, bool* found);
cudaError_t launch_czt_m1024(int M, const CztParams& p, cudaStream_t s, bool* found);
cudaError_t launch_czt_large(int M, const CztParams& p, cudaStream_t s, bool* found);
// The same as two halves on the 4096-point engine (convolution length 8192).
cudaError_t launch_czt_split_large(int M, const CztParams& p, cudaStream_t s, bool* found);

}  // namespace top
