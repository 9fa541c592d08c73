// Helpers that expand an engine list into the registry functions of one unit.
#pragma once

#include "top_czt.cuh"
#include "top_dispatch.h"
#include "top_passes.cuh"

namespace top {

template <class EN>
inline void fill_engine_info(EngineInfo* info) {
  info->M = EN::M;
  info->G = EN::G;
  info->NS = EN::NS;
  for (int s = 0; s < 4; ++s) info->R[s] = s < EN::NS ? EN::radix(s) : 1;
  info->tw_size = EN::TW_SIZE;
  info->rows = RowShape<EN>::ROWS;
  info->row_smem = RowShape<EN>::SMEM;
}

template <class EN>
inline cudaError_t launch_pass_of(int kind, const PassParams& p, const PassParams* next, cudaStream_t s) {
  if (kind == PASS_ROWS_FWD) return launch_rows_fwd<EN>(p, s);
  if (kind == PASS_COLS) return launch_cols<EN>(p, s);
  if (kind == PASS_ROWS_CHAIN) return next ? launch_rows_chain<EN>(p, *next, s) : cudaErrorInvalidValue;
  return launch_rows_inv<EN>(p, s);
}

}  // namespace top

#define TOP_INFO_CASE(EN) \
  case EN::M:             \
    fill_engine_info<EN>(info); \
    return true;
#define TOP_LAUNCH_CASE(EN) \
  case EN::M:               \
    *found = true;          \
    return launch_pass_of<EN>(kind, p, next, s);

#define TOP_DEFINE_UNIT(name, LIST)                                                                 \
  namespace top {                                                                                   \
  bool engine_info_##name(int M, EngineInfo* info) {                                                \
    switch (M) { LIST(TOP_INFO_CASE) default: return false; }                                       \
  }                                                                                                 \
  cudaError_t launch_pass_##name(int kind, int M, const PassParams& p, const PassParams* next, cudaStream_t s, \
                                 bool* found) {                                                     \
    *found = false;                                                                                 \
    switch (M) { LIST(TOP_LAUNCH_CASE) default: return cudaSuccess; }                               \
  }                                                                                                 \
  }

#define TOP_CZT_CASE(EN) \
  case EN::M:            \
    *found = true;       \
    return launch_czt<EN>(p, s);

// Bluestein line transforms on the unit's (power-of-two) engines.
#define TOP_DEFINE_CZT(name, LIST)                                                                 \
  namespace top {                                                                                  \
  cudaError_t launch_czt_##name(int M, const CztParams& p, cudaStream_t s, bool* found) {          \
    *found = false;                                                                                \
    switch (M) { LIST(TOP_CZT_CASE) default: return cudaSuccess; }                                 \
  }                                                                                                \
  }

#define TOP_CZT_SPLIT_CASE(EN) \
  case EN::M:                  \
    *found = true;             \
    return launch_czt_split<EN>(p, s);

// Bluestein line transforms as two halves on the unit's engines of half the convolution length.
#define TOP_DEFINE_CZT_SPLIT(name, LIST)                                                           \
  namespace top {                                                                                  \
  cudaError_t launch_czt_split_##name(int M, const CztParams& p, cudaStream_t s, bool* found) {    \
    *found = false;                                                                                \
    switch (M) { LIST(TOP_CZT_SPLIT_CASE) default: return cudaSuccess; }                           \
  }                                                                                                \
  }
