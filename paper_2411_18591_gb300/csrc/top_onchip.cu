// Whole propagations of 64 x 64 fields at padding 2 (128 x 128 transforms, Eq. 4 with H of Eq. 5)
// in one kernel, every intermediate in shared memory: one block of 128 threads per field, the
// fields of a launch taken in turn by a grid of two blocks per SM.
//
// A field crosses HBM twice (read once, written once: 16 n^2 bytes) instead of the 80 n^2 of the
// three passes, and each half line is one thread's 64-point DFT in registers (no exchanges):
//   1. rows:    thread (r, y) folds row y into half r (even or odd frequencies, the odd half
//               carrying exp(-2 pi i p / 128)), transforms it and stores its bins in a tile
//               [kpos][y] (kpos = r M + k holds kx = 2 k + r);
//   2. columns: thread (r, column) folds the column from the tile, transforms it, multiplies by
//               H / (Py Px) (conjugated for the adjoint) from the quadrant table staged in shared
//               memory, inverse transforms; the two halves combine through the tile into the
//               cropped column;
//   3. rows:    thread (r, y) inverse transforms the bins of row y; the halves combine into the
//               cropped row, staged for a coalesced store.
// The fold, the transfer-function entries and the combines follow the three-pass kernels; the
// line transforms are the natural-order composite DFTs of top_engine.cuh, so results agree with
// the three passes to rounding, not bit for bit.
#include "top_aux.h"
#include "top_passes.cuh"

namespace top {

namespace {

constexpr int kN = 64;                   // field side
constexpr int kM = 64;                   // half of the padded side
constexpr int kP = 2 * kM;               // padded side
constexpr int kLT = kN + 1;              // tile stride (float2): [kpos][y] and the [y][x] staging
constexpr int kHS = kM + 2;              // quadrant-table row (the FieldSet::hq layout)
constexpr int kLH = kHS + 1;             // staged row stride: consecutive |kx| 6 banks apart
constexpr int kHRows = kP / 2 + 1;       // |kx| = 0 .. 64
constexpr int kThreads = 128;
constexpr int kTile = kP * kLT;          // float2
constexpr size_t kSmem = sizeof(float2) * (size_t(kTile) + size_t(kHRows) * kLH);
static_assert(2 * kN * kLT <= kTile, "two [y][x] staging planes fit the tile");

// v[pos] * exp(DIR 2 pi i pos / 128) for every slot, the constants folded at compile time.
template <int DIR, int... I>
__device__ __forceinline__ void half_twiddles(float2 (&v)[kM], std::integer_sequence<int, I...>) {
  ((v[I] = tw_const<DIR, long(I), long(kP)>(v[I])), ...);
}
// The fold's odd-half twiddle: slots below M/2 hold the copy at p = pos + M, whose factor is
// exp(-2 pi i (pos + M) / 128) = -exp(-2 pi i pos / 128).
template <int... I>
__device__ __forceinline__ void fold_twiddles(float2 (&v)[kM], std::integer_sequence<int, I...>) {
  ((v[I] = tw_const<-1, long(I < kM / 2 ? I + kM : I), long(kP)>(v[I])), ...);
}

__global__ void __launch_bounds__(kThreads, 2) k_onchip64(const __grid_constant__ PassParams p) {
  TOP_DYN_SMEM(float2, smem);
  float2* tile = smem;           // [kpos][y] bins, or two [y][x] planes
  float2* hs = smem + kTile;     // staged quadrant rows [|kx|][kLH]
  const int tid = threadIdx.x;
  const int r = tid >> 6;        // half: warps 0-1 even, 2-3 odd
  const int c = tid & 63;        // row y (phases 1, 3) or column slot (phase 2)
  const float2* staged = nullptr;  // the quadrant table in shared memory
  float2 v[kM];

  for (int f = blockIdx.x; f < p.nfields; f += gridDim.x) {
    // ---- stage the field rows [y][x] (stride kLT) and, when the set changes, its quadrant rows
    const float2* src = field_in(p, f);
#pragma unroll 4
    for (int i = tid; i < kN * kN; i += kThreads) top_cp_async8(tile + (i >> 6) * kLT + (i & 63), src + i);
    const float2* hq = p.hq_list ? p.hq_list[f] : p.sets[p.set_of[f]].hq;
    if (hq != staged) {
      for (int i = tid; i < kHRows * kHS; i += kThreads) {
        const int row = i / kHS, e = i - row * kHS;
        top_cp_async8(hs + row * kLH + e, hq + i);
      }
      staged = hq;
    }
    top_cp_async_wait_all();
    __syncthreads();

    // ---- 1. rows: fold (X2: slot pos holds sample pos +/- M/2), forward DFT, bins to the tile
    {
      const float2* row = tile + c * kLT;
#pragma unroll
      for (int pos = 0; pos < kM; ++pos) v[pos] = row[pos < kM / 2 ? pos + kM / 2 : pos - kM / 2];
      if (r) fold_twiddles(v, std::make_integer_sequence<int, kM>{});
      dft<kM, 1, -1>(v);
      __syncthreads();  // every row is read before the bins overwrite it
#pragma unroll
      for (int k = 0; k < kM; ++k) tile[(r * kM + k) * kLT + c] = v[k];
      __syncthreads();
    }

    // ---- 2. columns, in two rounds of 64 (consecutive lanes take consecutive |kx|)
#pragma unroll 1
    for (int it = 0; it < 2; ++it) {
      const int kxi = it * kM + c;                        // index of kx in [0, P)
      const int kpos = (kxi & 1) ? kM + (kxi >> 1) : (kxi >> 1);
      const int akx = kxi <= kP / 2 ? kxi : kP - kxi;     // |kx|
      float2* col = tile + kpos * kLT;
#pragma unroll
      for (int pos = 0; pos < kM; ++pos) v[pos] = col[pos < kM / 2 ? pos + kM / 2 : pos - kM / 2];
      if (r) fold_twiddles(v, std::make_integer_sequence<int, kM>{});
      dft<kM, 1, -1>(v);
      // bin k holds ky index 2k + r: entry k of the half's part below the middle, M - r - k above
      const float2* part = hs + akx * kLH + r * (kM / 2 + 1);
      if (p.adjoint) {
#pragma unroll
        for (int k = 0; k < kM; ++k) v[k] = c_mulc(v[k], part[k < kM / 2 ? k : kM - r - k]);
      } else {
#pragma unroll
        for (int k = 0; k < kM; ++k) v[k] = c_mul(v[k], part[k < kM / 2 ? k : kM - r - k]);
      }
      dft<kM, 1, +1>(v);
      if (r) half_twiddles<+1>(v, std::make_integer_sequence<int, kM>{});  // O' = exp(2 pi i pos / P) O
      __syncthreads();  // both halves have read the column
      // the column's sample y = pos + M/2 is E[pos] - O'[pos] (pos < M/2), y = pos - M/2 is
      // E[pos] + O'[pos] (pos >= M/2): the odd half leaves O' below M/2, the even half E above
#pragma unroll
      for (int k = 0; k < kM / 2; ++k) col[k + (r ? 0 : kM / 2)] = r ? v[k] : v[k + kM / 2];
      __syncthreads();
      float2 o[kM / 2];
#pragma unroll
      for (int k = 0; k < kM / 2; ++k) {
        o[k] = r ? c_add(col[k + kM / 2], v[k + kM / 2])   // y = k
                 : c_sub(v[k], col[k]);                   // y = k + M/2
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < kM / 2; ++k) col[k + (r ? 0 : kM / 2)] = o[k];
    }
    __syncthreads();

    // ---- 3. rows: inverse DFT of the bins of row y, halves combined into the cropped row
    {
#pragma unroll
      for (int k = 0; k < kM; ++k) v[k] = tile[(r * kM + k) * kLT + c];
      dft<kM, 1, +1>(v);
      if (r) half_twiddles<+1>(v, std::make_integer_sequence<int, kM>{});
      __syncthreads();  // every bin is read: the tile becomes two [y][x] planes
      float2* s1 = tile + c * kLT;            // exchange plane
      float2* s2 = tile + (kN + c) * kLT;     // output plane
#pragma unroll
      for (int k = 0; k < kM / 2; ++k) s1[k + (r ? 0 : kM / 2)] = r ? v[k] : v[k + kM / 2];
      __syncthreads();
      // x = pos - M/2 (pos >= M/2): E[pos] + O'[pos]; x = pos + M/2 (pos < M/2): E[pos] - O'[pos]
#pragma unroll
      for (int k = 0; k < kM / 2; ++k) {
        if (r) s2[k] = c_add(s1[k + kM / 2], v[k + kM / 2]);
        else s2[k + kM / 2] = c_sub(v[k], s1[k]);
      }
      __syncthreads();
      float2* dst = field_out(p, f);
#pragma unroll 4
      for (int i = tid; i < kN * kN; i += kThreads) dst[i] = tile[(kN + (i >> 6)) * kLT + (i & 63)];
    }
  }
}

}  // namespace

bool onchip_supported(const PassParams& p) {
  return p.Py == kP && p.Px == kP && p.ny == kN && p.nx == kN && p.src_kind == SRC_FIELD && p.msrc.flags == 0 &&
         p.epi_kind == EPI_FIELD && p.mepi.flags == 0 && p.in_repeat >= 1 && !p.spec_in && !p.spec_out && !p.hq_out;
}

cudaError_t launch_onchip(const PassParams& p, cudaStream_t s) {
  // SM count of the current device (the grid is two blocks per SM)
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_onchip64, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSmem));
  if (e != cudaSuccess) return e;
  const int grid = p.nfields < 2 * sms ? p.nfields : 2 * sms;
  if (grid <= 0) return cudaSuccess;
  TOP_LAUNCH(k_onchip64, grid, kThreads, kSmem, s, p);
  return cudaGetLastError();
}

}  // namespace top
