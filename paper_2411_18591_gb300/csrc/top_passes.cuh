// The three passes of one batched propagation, Eq. 4 with H_z of Eq. 5:
//
//   R1  rows:    modulate (Eq. 1), zero-pad along x, forward DFT along x,
//                store transposed:  ws[field][kx][y]
//   C   columns: zero-pad along y, forward DFT along y, multiply by H(kx, ky) / (Py Px)
//                (a float64-built table), inverse DFT along y, crop:  ws[field][kx][y] in place
//   R2  rows:    inverse DFT along x, crop, epilogue (modulation, |psi|^2,
//                incoherent sums of Eq. 14, or modulation gradients)
//
// Each padded line of even length P = 2M is handled as its two interleaved
// halves (even and odd frequencies), transformed by two thread groups side by
// side. With a field of n <= P samples at offset o, the even half is the M-point
// DFT of the folded sequence v[q] = sum_{p = q mod M} x[p - o] and the odd half
// that of sum_{p = q mod M} x[p - o] exp(-2 pi i p / P). Zero samples of the
// padding are never loaded or transformed, and the inverse only produces the
// cropped window: x[p] = E[p mod M] + exp(2 pi i p / P) O[p mod M].
//
// Layout of the workspace between passes: for each field, Px frequency lines of
// ny samples, line kpos = r Mx + k holding frequency kx = 2 k + r, stored in
// blocks of four lines: sample (kpos, y) at ((kpos / 4) ny + y) 4 + kpos % 4.
// Four consecutive lanes of a two-stage FFT hold four consecutive lines, so the
// row passes move whole 32-byte sectors straight between registers and memory,
// and the column pass reads pairs of lines as one 16-byte stream.
#pragma once

#include <type_traits>
#include <utility>

#include "top_engine.cuh"
#include "top_internal.h"
#include "top_launch.h"

namespace top {

// Threads per block of the row passes (a block holds TOP_ROW_THREADS / G rows).
#ifndef TOP_ROW_THREADS
#define TOP_ROW_THREADS 64
#endif
// Whether two-stage plans move their row bins directly between registers and the workspace.
#ifndef TOP_ROW_DIRECT
#define TOP_ROW_DIRECT 1
#endif

// Workspace index of sample (kpos, y) in the four-line block layout.
__device__ __forceinline__ long long ws_index(int kpos, int y, int ny) {
  return ((long long)(kpos >> 2) * ny + y) * 4 + (kpos & 3);
}

// A two-stage plan holds one radix-RL butterfly per thread (E == RL): lane t of half r holds the
// bins kbase(t) + e M/RL, and with M/RL a multiple of 4 their workspace samples in row y sit at
// ws_index(r M + kbase(t), y) + e (M/RL) ny. Returns that first sample; the step is (M/RL) ny.
template <class EN>
__device__ __forceinline__ long long direct_base(int r, int t, int y, int ny) {
  static_assert(EN::E == EN::RL && (EN::M / EN::RL) % 4 == 0, "direct bins need one butterfly a thread");
  return ws_index(r * EN::M + EN::kbase(t), y, ny);
}

// Blocks per SM of the column pass of two-stage plans with blocks of 128 threads or fewer.
#ifndef TOP_COL_MINB_SMALL
#define TOP_COL_MINB_SMALL 5
#endif

// Registers a thread of the blocks whose line groups do not tile a warp (the mixed-radix plans of
// 25 and 50 threads a line) are held to, per pass kind: left to itself the compiler took 160-210
// and one to three blocks per SM for twenty samples a thread (measured on the 1000-point plan:
// column pass 52.0 -> 38.5 us per field at 96, inverse rows 25.8 -> 17.7 at 128).
#ifndef TOP_GROUP_REGS_COLS
#define TOP_GROUP_REGS_COLS 96
#endif
#ifndef TOP_GROUP_REGS_ROWS
#define TOP_GROUP_REGS_ROWS 128
#endif
// Blocks per SM that hold a block of `threads` to at most `regs` registers a thread.
__host__ __device__ constexpr int blocks_for_regs(int threads, int regs) {
  return 65536 / (((threads + 31) / 32) * 32 * regs) > 0 ? 65536 / (((threads + 31) / 32) * 32 * regs) : 1;
}

// Rows per block of the row passes; two thread groups (the two halves) per row. Two-stage plans
// move their bins directly between registers and the workspace (DIRECT); deeper plans stage them
// through a shared tile [2M][LD].
template <class EN>
struct RowShape {
  static constexpr int ROWS = (TOP_ROW_THREADS / EN::G) >= 1 ? (TOP_ROW_THREADS / EN::G) : 1;
  static constexpr int GROUPS = 2 * ROWS;
  static constexpr int THREADS = GROUPS * EN::G;
  static constexpr bool DIRECT = TOP_ROW_DIRECT && EN::NS == 2;
  // tile [2M][LD], bin k of a row at tslot(k) * LD + row: an odd stride keeps the column writes
  // free of bank conflicts; plans whose lanes hold bins 16 apart pad the bin index instead
  static constexpr int LD = EN::BIN_PAD ? (ROWS % 2 ? ROWS : ROWS + 1) : ROWS + 1;
  __host__ __device__ __forceinline__ static constexpr int tslot(int k) { return EN::bin_slot(k); }
  static constexpr int TILE = DIRECT ? 0 : tslot(2 * EN::M) * LD;
  static constexpr int XCH = GROUPS * EN::BUF;
  static constexpr int ROWBUF = ROWS * 2 * EN::M;  // input rows (n <= P = 2M) or E/O halves of the inverse
  static constexpr int MAX2 = TILE > XCH ? TILE : XCH;
  static constexpr size_t SMEM = sizeof(float2) * (MAX2 > ROWBUF ? MAX2 : ROWBUF);
  // the inverse pass keeps 128 registers a thread (four 128-thread blocks per SM, two of 256);
  // the forward pass of 256-thread blocks too (smaller blocks stay below 128 unbounded)
  static constexpr int MINB_INV = THREADS % 128 == 0 ? 512 / THREADS : blocks_for_regs(THREADS, TOP_GROUP_REGS_ROWS);
  static constexpr bool FWD_B2 = THREADS == 256;
  // R1 stages the planes its source needs besides the field rows after SMEM (at most five floats
  // per sample: intensity gradient, phase, amplitude, complex mask)
  static constexpr size_t SMEM_SRC_MAX = SMEM + sizeof(float) * 5 * ROWS * 2 * EN::M < 227 * 1024
                                             ? SMEM + sizeof(float) * 5 * ROWS * 2 * EN::M
                                             : 227 * 1024;
  // R2 stages its epilogue planes (accumulators, masks, the saved modulation input) after SMEM
  static constexpr size_t SMEM_EPI_MAX = SMEM + sizeof(float) * 10 * ROWS * 2 * EN::M < 227 * 1024
                                             ? SMEM + sizeof(float) * 10 * ROWS * 2 * EN::M
                                             : 227 * 1024;
  static_assert(SMEM % 16 == 0, "staged planes start on a 16-byte boundary");
  static_assert(SMEM >= 3 * sizeof(double) * THREADS, "room for the overlap reduction");
  static_assert(THREADS <= 1024, "row block too large");
  static_assert(EN::G <= 32 || EN::G % 32 != 0 || THREADS / EN::G <= 15, "one named barrier id per group");
  static_assert(EN::M % 2 == 0, "the four-line workspace blocks need P = 2M to be a multiple of 4");
};

// Columns per block of the column pass (even; a multiple of four from four up); two thread groups
// (the two halves) per column. The columns' samples are de-interleaved from the four-line blocks
// into contiguous lines [COLS][LS] of shared memory (after the fold a line serves as its even
// half's exchange buffer, then carries the column's output), followed by one exchange buffer per
// odd half, which finally carries that half's output.
#ifndef TOP_COL_MIN
#define TOP_COL_MIN 4
#endif
template <class EN>
struct ColShape {
  static constexpr int C0 = (64 / EN::G) & ~1;
  // whole four-line blocks where the block stays at 256 threads or below, else pairs
  static constexpr int COLS = C0 >= 4 ? C0 : ((TOP_COL_MIN > 2 && EN::G <= 32) ? 4 : 2);
  static constexpr int CB = COLS >= 4 ? 4 : 2;  // lines moved together: one block of four, or a pair
  static constexpr int GROUPS = 2 * COLS;
  static constexpr int THREADS = GROUPS * EN::G;
  // two-stage power-of-two plans fit five blocks per SM (96 registers) without real spills; other
  // blocks of whole 128-thread multiples keep 128 registers a thread (at least two blocks of 256)
  static constexpr int MINB = (EN::NS == 2 && (EN::G & (EN::G - 1)) == 0 && THREADS <= 128) ? TOP_COL_MINB_SMALL
                              : (THREADS % 128 == 0 && THREADS <= 256) ? 512 / THREADS
                              : THREADS % 32 != 0 ? blocks_for_regs(THREADS, TOP_GROUP_REGS_COLS) : 1;
  // line stride: room for the column and an exchange buffer, and LS = 16 / CB (mod 16) so that the
  // CB lines of a copy instruction fall on distinct banks
  __host__ __device__ static constexpr int line_stride(int ny) {
    const int l = ny > EN::BUF ? ny : EN::BUF;
    return l + ((16 / CB - l) % 16 + 16) % 16;
  }
  // Two-stage plans without bin padding read their H entries straight from the table (L1/L2; a
  // warp's loads for one slot are consecutive): measured faster than staging the rows (1024-point
  // plan 15.9 -> 15.1 us per field); the deeper plans stage them (2048-point 108 against 130 us).
  static constexpr bool TWO_STAGE_GLOBAL_H = EN::NS == 2 && !EN::BIN_PAD;
  // With padding exactly 2 (ny = M) the transfer-function rows of the block's columns (HS entries
  // each) are staged in shared memory too, where that keeps two blocks per SM (or where the
  // registers hold one block per SM anyway); otherwise the rows are read from global memory.
  // Entry i of a staged row sits at bin_slot(i) (rows HSS apart).
  static constexpr int HS = EN::M + 2;
  static constexpr int HSS = (EN::bin_slot(HS - 1) + 2) & ~1;
  static constexpr size_t H_BUDGET = 65536 / (THREADS * 128) >= 2 ? 110 * 1024 : 220 * 1024;
  template <bool X2>
  static constexpr bool stage_h() {
    return X2 && !TWO_STAGE_GLOBAL_H && sizeof(float2) * COLS * (line_stride(EN::M) + EN::BUF + HSS) <= H_BUDGET;
  }
  template <bool X2>
  static size_t smem(int ny) {
    return sizeof(float2) * (size_t(COLS) * (line_stride(ny) + EN::BUF) + (stage_h<X2>() ? COLS * HSS : 0));
  }
  static constexpr size_t SMEM_MAX =
      sizeof(float2) * COLS * ((2 * EN::M > EN::BUF ? 2 * EN::M : EN::BUF) + 16 + EN::BUF > line_stride(EN::M) + EN::BUF + HSS
                                   ? (2 * EN::M > EN::BUF ? 2 * EN::M : EN::BUF) + 16 + EN::BUF
                                   : line_stride(EN::M) + EN::BUF + HSS);
  static_assert(COLS % CB == 0, "columns come in whole copy units");
  static_assert(!EN::BIN_PAD || EN::bin_slot(EN::M / 2) < EN::BUF, "a half's row part fits its exchange buffer");
  static_assert(EN::G <= 32 || EN::G % 32 != 0 || THREADS / EN::G + COLS <= 15,
                "group barrier ids (15 down) clear of the column barrier ids (1 up)");
  static_assert(SMEM_MAX <= 227 * 1024, "column block above the shared-memory limit");
};

// Group index and lane of a thread (masks when G is a power of two, so lane ranges are known).
template <int G>
__device__ __forceinline__ void group_lane(int tid, int& grp, int& t) {
  if constexpr ((G & (G - 1)) == 0) {
    grp = tid / G;
    t = tid & (G - 1);
  } else {
    grp = tid / G;
    t = tid - grp * G;
  }
}

__device__ __forceinline__ float2 ldg2(const float2* p) { return __ldg(p); }

// Calls f(std::integral_constant<int, e>) for every register slot e, so slot positions are constants.
template <class F, int... Es>
__device__ __forceinline__ void for_slots(F&& f, std::integer_sequence<int, Es...>) {
  (f(std::integral_constant<int, Es>{}), ...);
}

// exp(-2 pi i pos / 2M) for the stage-0 position pos = t + G q + SP0 j of slot e, as the lane's
// exp(-2 pi i t / 2M) times a compile-time constant.
template <class EN, int e>
__device__ __forceinline__ float2 slot_split_twiddle(float2 wt) {
  constexpr int R0 = EN::radix(0), SP0 = EN::span(0);
  return tw_const<-1, long(EN::G * (e / R0) + SP0 * (e % R0)), long(2 * EN::M)>(wt);
}

// exp(i a) for a float32 phase: two-constant Cody-Waite reduction of a to [-pi, pi]
// (2 pi = 6.28125 + 1.9353071795864769e-3, the first part exact in a few bits) and the
// fast sin/cos there; large arguments take the library path.
__device__ __forceinline__ float2 cis(float a) {
  float s, c;
  if (fabsf(a) < 1.0e5f) {
    const float n = rintf(a * 0.15915494309189535f);
    float r = fmaf(-n, 6.28125f, a);
    r = fmaf(-n, 1.9353071795864769e-3f, r);
    __sincosf(r, &s, &c);
  } else {
    sincosf(a, &s, &c);
  }
  return make_float2(c, s);
}

// M(x, y) of Eq. 1 for field f at sample (y, x)
__device__ __forceinline__ float2 mod_value(const ModDev& m, uint32_t flags, int conj, const float2* lx,
                                            const float2* ly, int f, int y, int x, int nx) {
  if (flags & TOP_MOD_CIRC) {
    const int2 rg = __ldg(m.circ + y);
    if (x < rg.x || x > rg.y) return make_float2(0.f, 0.f);
  }
  float2 r = make_float2(1.f, 0.f);
  const long long idx = (long long)f * m.stride + (long long)y * nx + x;
  if (flags & TOP_MOD_COMPLEX) r = ldg2(m.cmask + idx);
  if (flags & TOP_MOD_AMPLITUDE) r = c_scale(r, __ldg(m.amp + idx));
  if (flags & TOP_MOD_PHASE) r = c_mul(r, cis(__ldg(m.phase + idx)));
  if (flags & TOP_MOD_LENS) r = c_mul(r, c_mul(ldg2(lx + x), ldg2(ly + y)));
  return conj ? c_conj(r) : r;
}

// Source field f of R1 and output field f of R2 (per-field pointers for ragged batches).
__device__ __forceinline__ const float2* field_in(const PassParams& p, int f) {
  return p.in_list ? p.in_list[f] : p.in + (long long)(f / p.in_repeat) * p.in_stride;
}
__device__ __forceinline__ float2* field_out(const PassParams& p, int f) {
  return p.out_list ? p.out_list[f] : p.out + (long long)f * p.out_stride;
}

__device__ __forceinline__ float2 load_src(const PassParams& p, const FieldSet& fs, int f, int y, int x) {
  const long long idx = (long long)y * p.nx + x;
  float2 s;
  if (p.src_kind == SRC_FIELD) {
    s = ldg2(field_in(p, f) + idx);
  } else {
    const float gi = __ldg(p.gI + (long long)(f / p.src_group) * p.gI_stride + idx);
    const float w = p.weights ? __ldg(p.weights + f) : 1.f;
    s = c_scale(ldg2(p.psi + (long long)f * p.psi_stride + idx), 2.f * w * gi);
  }
  if (p.msrc.flags) s = c_mul(s, mod_value(p.msrc, p.msrc.flags, p.msrc.conj, fs.src_lx, fs.src_ly, f, y, x, p.nx));
  return s;
}

// Whether R1 copies its source rows (and planes) into shared memory with asynchronous 16-byte
// copies: every row start must be 16-byte aligned and the planes must fit.
template <class EN>
__host__ __device__ inline bool src_staged(const PassParams& p) {
  const size_t extra = src_plane_floats(p, RowShape<EN>::ROWS);
  if (extra == 0) return p.nx % 2 == 0;
  return p.nx % 4 == 0 && RowShape<EN>::SMEM + sizeof(float) * extra <= RowShape<EN>::SMEM_SRC_MAX;
}

// Slots of half r folded from a line of n samples at offset o, sample x at line[x * LS] (the odd
// half carries exp(-2 pi i p / 2M); the copy at p + M picks up the opposite sign). X2: n = M and
// o = M/2 (padding exactly 2), where every slot has one source, (pos + M/2) mod M, lying in the
// upper copy when pos < M/2.
template <class EN, bool X2, int LS>
__device__ __forceinline__ void fold(float2 (&v)[EN::E], const float2* line, int n, int o, int r,
                                     const float2* __restrict__ wp, int t) {
  constexpr int M = EN::M;
#pragma unroll
  for (int e = 0; e < EN::E; ++e) {
    const int pos = EN::in_pos(t, e);
    if constexpr (X2) {
      const bool upper = pos < M / 2;
      v[e] = line[(upper ? pos + M / 2 : pos - M / 2) * LS];
    } else {
      const int x0 = pos - o, x1 = pos + M - o;
      const float2 a0 = (x0 >= 0 && x0 < n) ? line[x0 * LS] : make_float2(0.f, 0.f);
      const float2 a1 = (x1 >= 0 && x1 < n) ? line[x1 * LS] : make_float2(0.f, 0.f);
      v[e] = r ? c_mul(c_sub(a0, a1), ldg2(wp + pos)) : c_add(a0, a1);
    }
  }
  if constexpr (X2) {
    if (r) {
      const float2 wt = ldg2(wp + t);
      for_slots(
          [&](auto ec) {
            constexpr int e = decltype(ec)::value;
            const float2 w = slot_split_twiddle<EN, e>(wt);
            v[e] = c_mul(v[e], EN::in_pos(t, e) < M / 2 ? c_neg(w) : w);
          },
          std::make_integer_sequence<int, EN::E>{});
    }
  }
}

// ----------------------------------------------------------------------------- R1

// Planes of an R1 source staged in shared memory (null when not needed).
struct SrcPlanes {
  const float* gi;
  const float* ph;
  const float* am;
  const float2* cm;
};

// Issue the 16-byte async copies of the planes the source of field f needs (rows y0 .. y0 +
// nrows - 1) into `planes` (src_plane_floats(p, ROWS) floats).
template <class EX>
__device__ __forceinline__ SrcPlanes stage_src_planes(const PassParams& p, int f, int y0, int nrows, float* planes) {
  using SH = RowShape<EX>;
  constexpr int ROWS = SH::ROWS, NT = SH::THREADS;
  const int nx = p.nx, plane = ROWS * nx;
  const ModDev& m = p.msrc;
  const long long row0 = (long long)y0 * nx;
  auto stage = [&](const float* from, int floats_per_sample) {
    float* dst = planes;
    planes += plane * floats_per_sample;
    const float4* s4 = reinterpret_cast<const float4*>(from);
    float4* d4 = reinterpret_cast<float4*>(dst);
    const int n4 = nrows * nx * floats_per_sample / 4;
    for (int i = threadIdx.x; i < n4; i += NT) top_cp_async16(d4 + i, s4 + i);
    return dst;
  };
  const long long midx = (long long)f * m.stride + row0;
  SrcPlanes sp{};
  if (p.src_kind == SRC_INTENSITY) sp.gi = stage(p.gI + (long long)(f / p.src_group) * p.gI_stride + row0, 1);
  if (m.flags & TOP_MOD_PHASE) sp.ph = stage(m.phase + midx, 1);
  if (m.flags & TOP_MOD_AMPLITUDE) sp.am = stage(m.amp + midx, 1);
  if (m.flags & TOP_MOD_COMPLEX)
    sp.cm = reinterpret_cast<const float2*>(stage(reinterpret_cast<const float*>(m.cmask + midx), 2));
  return sp;
}

// The source arithmetic in place on rows [ROWS][nx] of shared memory: 2 w g_I psi for the
// intensity backward, times the source modulation M (Eq. 1).
template <class EX>
__device__ __forceinline__ void modulate_src_rows(const PassParams& p, const FieldSet& fs, int f, int y0, int nrows,
                                                  float2* rows, const SrcPlanes& sp) {
  constexpr int NT = RowShape<EX>::THREADS;
  const int nx = p.nx;
  const ModDev& m = p.msrc;
  const bool inten = p.src_kind == SRC_INTENSITY;
  const float w2 = inten ? 2.f * (p.weights ? __ldg(p.weights + f) : 1.f) : 1.f;
  for (int rr = 0; rr < nrows; ++rr) {
    const int y = y0 + rr;
    const int2 rg = (m.flags & TOP_MOD_CIRC) ? __ldg(m.circ + y) : make_int2(0, nx - 1);
    const float2 ly = (m.flags & TOP_MOD_LENS) ? ldg2(fs.src_ly + y) : make_float2(1.f, 0.f);
    for (int x = threadIdx.x; x < nx; x += NT) {
      const int i = rr * nx + x;
      float2 s = rows[i];
      if (inten) s = c_scale(s, w2 * sp.gi[i]);
      if (m.flags) {
        float2 mv = make_float2(1.f, 0.f);
        if (m.flags & TOP_MOD_COMPLEX) mv = sp.cm[i];
        if (m.flags & TOP_MOD_AMPLITUDE) mv = c_scale(mv, sp.am[i]);
        if (m.flags & TOP_MOD_PHASE) mv = c_mul(mv, cis(sp.ph[i]));
        if (m.flags & TOP_MOD_LENS) mv = c_mul(mv, c_mul(ldg2(fs.src_lx + x), ly));
        if (x < rg.x || x > rg.y) mv = make_float2(0.f, 0.f);
        s = c_mul(s, m.conj ? c_conj(mv) : mv);
      }
      rows[i] = s;
    }
  }
}

// Fold, forward-transform and store the bins of rows [ROWS][nx] (shared memory; they may alias
// the exchange buffers at `smem`, which are written only after a block barrier).
template <class EX, bool X2>
__device__ __forceinline__ void forward_rows(const PassParams& p, int f, int y0, int nrows, const float2* rows,
                                             float2* smem, int grp, int t) {
  using SH = RowShape<EX>;
  constexpr int E = EX::E, M = EX::M, ROWS = SH::ROWS, LD = SH::LD, NT = SH::THREADS;
  const int row = grp >> 1, r = grp & 1;
  const int nx = p.nx, ny = p.ny;
  float2 v[E];
  fold<EX, X2, 1>(v, rows + row * nx, nx, p.ox, r, p.wpx, t);
  __syncthreads();  // the rows may alias the exchange buffers
  EX::fwd(v, smem + grp * EX::BUF, t, p.twx);
  float2* ws = p.ws + (long long)f * p.ws_stride;
  if constexpr (SH::DIRECT) {
    // bins straight to the workspace: four consecutive lanes fill one 32-byte sector
    if (row < nrows) {
      float2* wp = ws + direct_base<EX>(r, t, y0 + row, ny);
      const int step = (M / EX::RL) * ny;
#pragma unroll
      for (int e = 0; e < E; ++e) wp[e * step] = v[e];
    }
  } else {
    __syncthreads();  // the exchange buffers alias the tile
#pragma unroll
    for (int e = 0; e < E; ++e) smem[SH::tslot(r * M + EX::bin(t, e)) * LD + row] = v[e];
    __syncthreads();
    // the tile, ROWS rows x 4 lines per block, to the workspace in address order
    for (int i = threadIdx.x; i < 2 * M * ROWS; i += NT) {
      const int c = i & 3, q = i >> 2;
      const int yo = q % ROWS, blk = q / ROWS;
      if (yo < nrows) ws[((long long)blk * ny + y0 + yo) * 4 + c] = smem[SH::tslot(4 * blk + c) * LD + yo];
    }
  }
}

template <class EX, bool X2>
__device__ __forceinline__ void rows_fwd(const PassParams& p) {
  using SH = RowShape<EX>;
  constexpr int ROWS = SH::ROWS, NT = SH::THREADS;
  TOP_DYN_SMEM(float2, smem);
  int grp, t;
  group_lane<EX::G>(threadIdx.x, grp, t);
  const int y0 = blockIdx.x * ROWS;
  const int nrows = min(ROWS, p.ny - y0);
  const int f = blockIdx.y;
  const FieldSet& fs = p.sets[p.set_of[f]];
  const int nx = p.nx;

  // modulated input rows -> shared [ROWS][nx]
  if (src_staged<EX>(p)) {
    // the field rows and the planes the source needs, each one contiguous block copied as
    // 16-byte pieces, then the source arithmetic in place
    const bool inten = p.src_kind == SRC_INTENSITY;
    const long long row0 = (long long)y0 * nx;
    const float2* src = inten ? p.psi + (long long)f * p.psi_stride + row0
                              : field_in(p, f) + row0;
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(smem);
    const int n4 = nrows * nx / 2, all4 = ROWS * nx / 2;
    for (int i = threadIdx.x; i < all4; i += NT) {
      if (i < n4) top_cp_async16(d4 + i, s4 + i);
      else d4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const SrcPlanes sp = stage_src_planes<EX>(p, f, y0, nrows, reinterpret_cast<float*>(smem + SH::SMEM / sizeof(float2)));
    top_cp_async_wait_all();
    if (inten || p.msrc.flags) {
      __syncthreads();
      modulate_src_rows<EX>(p, fs, f, y0, nrows, smem, sp);
    }
  } else {
#pragma unroll 2
    for (int rr = 0; rr < ROWS; ++rr) {
      for (int x = threadIdx.x; x < nx; x += NT)
        smem[rr * nx + x] = rr < nrows ? load_src(p, fs, f, y0 + rr, x) : make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
  forward_rows<EX, X2>(p, f, y0, nrows, smem, smem, grp, t);
}

// R1. Blocks of 128 threads or fewer take the compiler's own register choice (below 128); an
// explicit bound of two 256-thread blocks per SM is a separate kernel.
template <class EX, bool X2>
__global__ void __launch_bounds__(RowShape<EX>::THREADS) k_rows_fwd(const __grid_constant__ PassParams p) {
  rows_fwd<EX, X2>(p);
}
template <class EX, bool X2>
__global__ void __launch_bounds__(RowShape<EX>::THREADS, 2) k_rows_fwd_b2(const __grid_constant__ PassParams p) {
  rows_fwd<EX, X2>(p);
}

// ----------------------------------------------------------------------------- C

// Multiply the bins of half r of column kx by H(kx, ky) / (Py Px), conjugated for the adjoint,
// from the quadrant row of |kx| (shared or global memory): bin k of the half holds ky = 2k + r,
// whose |signed ky| is 2k + r below the middle and Py - 2k - r above it, so the even half reads
// entries k or M - k of the row's even part and the odd half entries k or M - 1 - k of its odd part.
// A row in shared memory holds entry i at bin_slot(i).
// With HALF the shared row holds only this half's part (entry j at bin_slot(j)).
template <class EY, bool SHARED, bool HALF = false>
__device__ __forceinline__ void apply_transfer(float2 (&v)[EY::E], const float2* row, int r, bool adjoint, int t) {
  constexpr int M = EY::M;
  const float sg = adjoint ? -1.f : 1.f;
  const int part = HALF ? 0 : r * (M / 2 + 1);
  const int mirror = M - r;
  // eight loads at a time: the compiler barrier keeps it from hoisting all E loads at once
  constexpr int CH = EY::E % 8 == 0 ? 8 : EY::E;
#pragma unroll
  for (int e0 = 0; e0 < EY::E; e0 += CH) {
#pragma unroll
    for (int e = e0; e < e0 + CH; ++e) {
      const int k = EY::bin(t, e);
      const int j = k < M / 2 ? k : mirror - k;
      float2 h = SHARED ? row[EY::bin_slot(part + j)] : ldg2(row + part + j);
      h.y *= sg;
      v[e] = c_mul(v[e], h);
    }
    asm volatile("" ::: "memory");
  }
}

// apply_transfer for two-stage plans with one butterfly a thread, from a row in shared memory: slot e
// holds bin kbase(t) + e M/RL, below M/2 exactly for e < RL/2, so the mirror choice is fixed per slot.
template <class EY>
__device__ __forceinline__ void apply_transfer_direct(float2 (&v)[EY::E], const float2* row, int r, bool adjoint,
                                                      int t) {
  constexpr int M = EY::M, S = M / EY::RL;
  const float2* part = row + r * (M / 2 + 1);
  const int kb = EY::kbase(t);
  const float2* up = part + kb;             // entry k = kb + e S for e < RL/2
  const float2* down = part + (M - r - kb);  // entry M - r - k for e >= RL/2
  if (adjoint) {
#pragma unroll
    for (int e = 0; e < EY::E; ++e) v[e] = c_mulc(v[e], e < EY::RL / 2 ? up[e * S] : down[-e * S]);
  } else {
#pragma unroll
    for (int e = 0; e < EY::E; ++e) v[e] = c_mul(v[e], e < EY::RL / 2 ? up[e * S] : down[-e * S]);
  }
}

// Workspace index of copy j of the CB columns from kpos0 (sample j / CB of column kpos0 + j % CB):
// a four-line block is one contiguous stretch; a pair covers half of each of its 32-byte rows.
template <int CB>
__device__ __forceinline__ long long col_src(int j, int kpos0, int ny) {
  if constexpr (CB == 4) {
    return (long long)kpos0 * ny + j;
  } else {
    return ws_index(kpos0 + (j & 1), j >> 1, ny);
  }
}

// Barrier of the two thread groups of column cl only (the steps between the column loads and the
// final stores touch the column's own line and exchange buffers): one warp, a named barrier of
// the column's warps, or the whole block where neither fits.
template <class EY, int COLS>
__device__ __forceinline__ void column_sync(int cl) {
  constexpr int T2 = 2 * EY::G;
  if constexpr (T2 == 32) {
    __syncwarp();
  } else if constexpr (T2 % 32 == 0 && COLS < 16) {
    top_named_barrier(1 + cl, T2);
  } else {
    __syncthreads();
  }
}

template <class EY, bool X2>
__global__ void __launch_bounds__(ColShape<EY>::THREADS, ColShape<EY>::MINB) k_cols(const __grid_constant__ PassParams p) {
  using SH = ColShape<EY>;
  constexpr int G = EY::G, E = EY::E, M = EY::M, COLS = SH::COLS, CB = SH::CB, NT = SH::THREADS;
  TOP_DYN_SMEM(float2, smem);
  int grp, t;
  group_lane<G>(threadIdx.x, grp, t);
  const int cl = grp >> 1, r = grp & 1;
  const int ny = p.ny;
  const int LS = SH::line_stride(ny);
  const int kpos0 = blockIdx.x * COLS;
  const int ncols = min(COLS, p.Px - kpos0);  // a multiple of CB
  const int f = blockIdx.y;
  const FieldSet& fs = p.sets[p.set_of[f]];
  const float2* hq = p.hq_list ? p.hq_list[f] : fs.hq;
  float2* line = smem + cl * LS;                            // [COLS][LS]
  float2* obuf = smem + COLS * LS + cl * EY::BUF;           // the odd half's exchange buffer and output
  float2* xbuf = r ? obuf : line;
  float2* hrows = smem + COLS * (LS + EY::BUF);             // [COLS][HSS] transfer-function rows
  float2* ws = p.ws + (long long)f * p.ws_stride;
  auto abs_kx = [&](int c) {  // |signed kx| of the block's column c (the last column repeats past the end)
    const int kp = min(kpos0 + c, p.Px - 1);
    const int rx = kp >= p.Mx ? 1 : 0;
    const int kx = 2 * (kp - rx * p.Mx) + rx;
    return kx <= p.Px / 2 ? kx : p.Px - kx;
  };

  // the columns of the block one wave of resident blocks later go to L2 while this one works
  if (threadIdx.x == 0 && p.l2_ahead > 0 && !p.spec_in) {
    const long long nb = (long long)gridDim.x * gridDim.y;
    const long long lb = (long long)blockIdx.y * gridDim.x + blockIdx.x + p.l2_ahead;
    if (lb < nb) {
      const int kp = int(lb % gridDim.x) * COLS;
      const int k0 = kp & ~3, k1 = min((kp + COLS + 3) & ~3, p.Px);
      top_prefetch_l2(p.ws + (lb / gridDim.x) * p.ws_stride + (long long)k0 * ny, unsigned(k1 - k0) * ny * 8u);
    }
  }
  // (A) de-interleave each unit of CB columns into contiguous lines: copy j of a unit holds
  // sample j / CB of its line j % CB (not needed when the column starts from a stored spectrum)
  if (!p.spec_in) {
    if constexpr (X2 && CB == 4 && COLS == 4 && (4 * M) % NT == 0) {
      // one four-line block of M samples a line, contiguous: thread i copies samples i + NT k
      const float2* src = ws + (long long)kpos0 * M + threadIdx.x;
      float2* dst = smem + (threadIdx.x & 3) * LS + (threadIdx.x >> 2);
#pragma unroll
      for (int k = 0; k < 4 * M / NT; ++k) top_cp_async8(dst + k * (NT / 4), src + k * NT);
    } else {
      for (int u = 0; u < ncols; u += CB) {
        for (int j = threadIdx.x; j < CB * ny; j += NT)
          top_cp_async8(smem + (u + j % CB) * LS + j / CB, ws + col_src<CB>(j, kpos0 + u, ny));
      }
    }
  }
  top_cp_async_commit();
  if constexpr (SH::template stage_h<X2>()) {
    // the column's own two groups copy its transfer-function row as a second group of copies,
    // waited for only where it is applied: the copy overlaps the forward transform
    if (!p.spec_out && !p.hq_out) {
      const int ct = threadIdx.x - cl * 2 * G;  // thread of the column's 2G
      const float2* hsrc = hq + (long long)abs_kx(cl) * SH::HS;
      float2* hdst = hrows + cl * SH::HSS;
      if constexpr (EY::BIN_PAD) {
        for (int q = ct; q < SH::HS; q += 2 * G) top_cp_async8(hdst + EY::bin_slot(q), hsrc + q);
      } else {
        for (int q = ct; q < SH::HS / 2; q += 2 * G) top_cp_async16(hdst + 2 * q, hsrc + 2 * q);  // 16-byte units
      }
    }
  }
  top_cp_async_commit();
  top_cp_async_wait_group<1>();  // this thread's column copies
  __syncthreads();

  float2 v[E];
  // spectrum slot of this thread's column and half (spec_in / spec_out)
  const long long spec_at = ((long long)min(kpos0 + cl, p.Px - 1) * 2 + r) * M + t;
  if (p.spec_in) {
    const float2* sp = p.spec_in + (long long)(f / p.in_repeat) * p.Px * (2 * M) + spec_at;
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = ldg2(sp + e * G);
  } else {
    fold<EY, X2, 1>(v, line, ny, p.oy, r, p.wpy, t);
    column_sync<EY, COLS>(cl);  // the column's line becomes its even half's exchange buffer
    EY::fwd(v, xbuf, t, p.twy);
  }
  if (p.spec_out) {
    // forward transform only: the spectrum, for the fields that share this source
    if (kpos0 + cl < p.Px) {
      float2* sp = p.spec_out + (long long)f * p.Px * (2 * M) + spec_at;
#pragma unroll
      for (int e = 0; e < E; ++e) sp[e * G] = v[e];
    }
    return;
  }
  if (p.hq_out) {
    // forward transform only (a transfer-function table from sampled kernels): half r holds
    // ky = 2k + r, kept where |ky| <= Py/2, i.e. k <= M/2 (even) and k < M/2 (odd), plus the
    // zero that pads each row
    if (kpos0 + cl < p.Px) {
      const int kp = kpos0 + cl;
      const int rx = kp >= p.Mx ? 1 : 0;
      const int kx = 2 * (kp - rx * p.Mx) + rx;
      if (kx <= p.Px / 2) {
        float2* row = p.hq_out + (long long)kx * (M + 2);
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int k = EY::bin(t, e);
          if (r == 0) {
            if (k <= M / 2) row[k] = c_scale(v[e], p.hq_scale);
          } else if (k < M / 2) {
            row[M / 2 + 1 + k] = c_scale(v[e], p.hq_scale);
          } else if (k == M / 2) {
            row[M + 1] = make_float2(0.f, 0.f);
          }
        }
      }
    }
    return;
  }
  if constexpr (SH::template stage_h<X2>()) {
    top_cp_async_wait_all();
    column_sync<EY, COLS>(cl);  // the column's transfer-function row is in place
    if constexpr (EY::NS == 2 && EY::E == EY::RL && !EY::BIN_PAD) {
      apply_transfer_direct<EY>(v, hrows + cl * SH::HSS, r, p.adjoint, t);
    } else {
      apply_transfer<EY, true>(v, hrows + cl * SH::HSS, r, p.adjoint, t);
    }
  } else if constexpr (EY::BIN_PAD) {
    // lanes hold bins 16 apart: the half's part of the row goes, read in order, into the half's
    // own exchange buffer (free between the transforms) and is applied from there
    const float2* part = hq + (long long)abs_kx(cl) * SH::HS + r * (M / 2 + 1);
    EY::sync_group();  // every lane is past its last read of the forward transform's exchanges
    for (int i = t; i < M / 2 + 1; i += G) xbuf[EY::bin_slot(i)] = ldg2(part + i);
    EY::sync_group();
    apply_transfer<EY, true, true>(v, xbuf, r, p.adjoint, t);
  } else {
    apply_transfer<EY, false>(v, hq + (long long)abs_kx(cl) * SH::HS, r, p.adjoint, t);
  }
  EY::inv(v, xbuf, t, p.twy);
  if constexpr (X2 && CB == 4 && COLS == 4 && (4 * M) % NT == 0 && EY::NS == 2 && EY::E == EY::RL &&
                EY::radix(0) % 2 == 0) {
    // Balanced combine: with slot k of the half below M/2 at position lo(k) and its partner at
    // lo(k) + M/2, the column's sample y = pos +/- M/2 is E[pos] -/+ O'[pos]. The even warp sends
    // E above M/2 through its own line, the odd warp O' below M/2 through its buffer; the even
    // warp then writes the samples y >= M/2 (its slots below M/2) into the odd buffer's upper half,
    // the odd warp the samples y < M/2 into the line's lower half.
    constexpr int R0 = EY::radix(0), HM = M / 2, H = E / 2;
    auto lo = [](int k) { return (k / (R0 / 2)) * R0 + k % (R0 / 2); };
    EY::sync_group();  // every lane is past the last reads of its exchange buffer
    if (r) {
      const float2 wt = ldg2(p.wpy + t);
      for_slots(
          [&](auto ec) {
            constexpr int e = decltype(ec)::value;
            v[e] = c_mulc(v[e], slot_split_twiddle<EY, e>(wt));  // O' = exp(2 pi i pos / P) O
          },
          std::make_integer_sequence<int, E>{});
#pragma unroll
      for (int k = 0; k < H; ++k) obuf[EY::in_pos(t, lo(k))] = v[lo(k)];
    } else {
#pragma unroll
      for (int k = 0; k < H; ++k) line[EY::in_pos(t, lo(k)) + HM] = v[lo(k) + R0 / 2];
    }
    column_sync<EY, COLS>(cl);
    if (r) {
#pragma unroll
      for (int k = 0; k < H; ++k) {
        const int pos = EY::in_pos(t, lo(k));
        line[pos] = c_add(line[pos + HM], v[lo(k) + R0 / 2]);  // y = pos: E[pos + M/2] + O'[pos + M/2]
      }
    } else {
#pragma unroll
      for (int k = 0; k < H; ++k) {
        const int pos = EY::in_pos(t, lo(k));
        obuf[pos + HM] = c_sub(v[lo(k)], obuf[pos]);  // y = pos + M/2: E[pos] - O'[pos]
      }
    }
    __syncthreads();
    // (B) the samples y < M/2 from the lines, y >= M/2 from the odd buffers, interleaved as in (A)
    {
      float2* dst = ws + (long long)kpos0 * M + threadIdx.x;
      const int c = threadIdx.x & 3, y0 = threadIdx.x >> 2;
      const float2* lo_src = smem + c * LS + y0;
      const float2* hi_src = smem + COLS * LS + c * EY::BUF + y0;
#pragma unroll
      constexpr int YS = NT / 4;  // rows per step
      static_assert(HM % YS == 0, "a step's rows lie on one side of M/2");
      for (int k = 0; k < 4 * M / NT; ++k) dst[k * NT] = (k * YS < HM) ? lo_src[k * YS] : hi_src[k * YS];
    }
    return;
  }
  EY::sync_group();  // every lane is past the last reads of its exchange buffer
  if (r) {
    if constexpr (X2) {
      const float2 wt = ldg2(p.wpy + t);
      for_slots(
          [&](auto ec) {
            constexpr int e = decltype(ec)::value;
            obuf[EY::in_pos(t, e)] = c_mulc(v[e], slot_split_twiddle<EY, e>(wt));  // exp(2 pi i pos / P) O[pos]
          },
          std::make_integer_sequence<int, E>{});
    } else {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int pos = EY::in_pos(t, e);
        obuf[pos] = c_mulc(v[e], ldg2(p.wpy + pos));  // exp(2 pi i pos / P) O[pos]
      }
    }
  }
  column_sync<EY, COLS>(cl);  // the odd half's output is in its buffer
  if (!r) {
    // combine the halves into the column's line
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int pos = EY::in_pos(t, e);
      const float2 o = obuf[pos];
      if constexpr (X2) {
        if (pos < M / 2) line[pos + M / 2] = c_sub(v[e], o);
        else line[pos - M / 2] = c_add(v[e], o);
      } else {
        const int y0 = pos - p.oy, y1 = pos + M - p.oy;
        if (y0 >= 0 && y0 < ny) line[y0] = c_add(v[e], o);
        if (y1 >= 0 && y1 < ny) line[y1] = c_sub(v[e], o);
      }
    }
  }
  __syncthreads();
  // (B) interleave back in the copy order of (A)
  for (int u = 0; u < ncols; u += CB) {
    for (int j = threadIdx.x; j < CB * ny; j += NT) ws[col_src<CB>(j, kpos0 + u, ny)] = smem[(u + j % CB) * LS + j / CB];
  }
}

// ----------------------------------------------------------------------------- R2

// Per-thread float64 sums of the overlap epilogue: psi conj(phi) and |psi|^2.
struct OvAcc {
  double re, im, pw;
};

__device__ __forceinline__ void overlap_add(OvAcc& acc, float2 val, float2 phi) {
  const double vx = val.x, vy = val.y, px = phi.x, py = phi.y;
  acc.re = fma(vx, px, fma(vy, py, acc.re));
  acc.im = fma(vy, px, fma(-vx, py, acc.im));
  acc.pw = fma(vx, vx, fma(vy, vy, acc.pw));
}

// Rows of the R2 epilogue held in shared memory ([ROWS][nx] each, sample i = rr nx + x): the
// accumulators of a group (intensity, modulation-gradient partials), written back once after the
// group's last field, and the planes the epilogue reads (mask factors, the saved modulation input).
struct EpiPlanes {
  float* acc_i;
  float* acc_ph;
  float* acc_am;
  float2* acc_cm;
  const float* ph;
  const float* am;
  const float2* cm;
  const float2* xs;
};

// Floats per sample of the staged epilogue planes.
__host__ __device__ inline int epi_plane_floats(const PassParams& p) {
  int n = 0;
  const uint32_t fl = p.mepi.flags;
  if (p.epi_kind == EPI_INTENSITY) n += 1;
  if (p.epi_kind == EPI_MODGRAD) {
    if (p.part_phase) n += 1;
    if (p.part_amp) n += 1;
    if (p.part_mask) n += 2;
    if (p.part_phase || p.part_amp || p.part_mask) n += 2;  // saved input
  }
  if (fl & TOP_MOD_PHASE) n += 1;
  if (fl & TOP_MOD_AMPLITUDE) n += 1;
  if (fl & TOP_MOD_COMPLEX) n += 2;
  return n;
}

// Whether R2 stages its epilogue planes: there is something to stage, rows are 16-byte units
// and the planes fit.
template <class EN>
__host__ __device__ inline bool epi_staged(const PassParams& p) {
  const int n = epi_plane_floats(p);
  return n > 0 && p.nx % 4 == 0 &&
         RowShape<EN>::SMEM + sizeof(float) * size_t(n) * RowShape<EN>::ROWS * p.nx <= RowShape<EN>::SMEM_EPI_MAX;
}

// M(x, y) of Eq. 1 from staged planes (sample i of the block) with the aperture range rg of the row
__device__ __forceinline__ float2 mod_value_planes(const EpiPlanes& e, uint32_t flags, int conj, const float2* lx,
                                                   float2 ly, int2 rg, int i, int x) {
  float2 r = make_float2(1.f, 0.f);
  if (flags & TOP_MOD_COMPLEX) r = e.cm[i];
  if (flags & TOP_MOD_AMPLITUDE) r = c_scale(r, e.am[i]);
  if (flags & TOP_MOD_PHASE) r = c_mul(r, cis(e.ph[i]));
  if (flags & TOP_MOD_LENS) r = c_mul(r, c_mul(ldg2(lx + x), ly));
  if ((flags & TOP_MOD_CIRC) && (x < rg.x || x > rg.y)) r = make_float2(0.f, 0.f);
  return conj ? c_conj(r) : r;
}

// Epilogue of one output sample val = psi(y, x) of field f in group g, from staged planes.
template <int KIND>
__device__ __forceinline__ void epilogue_planes(const PassParams& p, const FieldSet& fs, const EpiPlanes& e, int f,
                                                bool first, int y, int x, int i, float2 ly, int2 rg, float2 val,
                                                OvAcc& acc) {
  const long long idx = (long long)y * p.nx + x;
  const ModDev& m = p.mepi;
  if constexpr (KIND == EPI_OVERLAP) {
    if (m.flags) val = c_mul(val, mod_value_planes(e, m.flags, m.conj, fs.epi_lx, ly, rg, i, x));
    if (p.out) p.out[(long long)f * p.out_stride + idx] = val;
    overlap_add(acc, val, ldg2(p.target + (long long)f * p.target_stride + idx));
  } else if constexpr (KIND == EPI_FIELD) {
    if (m.flags) val = c_mul(val, mod_value_planes(e, m.flags, m.conj, fs.epi_lx, ly, rg, i, x));
    field_out(p, f)[idx] = val;
  } else if constexpr (KIND == EPI_INTENSITY) {
    if (m.flags) val = c_mul(val, mod_value_planes(e, m.flags, m.conj, fs.epi_lx, ly, rg, i, x));
    if (p.out) p.out[(long long)f * p.out_stride + idx] = val;
    const float w = p.weights ? __ldg(p.weights + f) : 1.f;
    const float v = w * fmaf(val.x, val.x, val.y * val.y);
    e.acc_i[i] = first ? v : e.acc_i[i] + v;
  } else {
    const float2 mv = mod_value_planes(e, m.flags, 0, fs.epi_lx, ly, rg, i, x);
    if (p.out) p.out[(long long)f * p.out_stride + idx] = c_mulc(val, mv);
    if (e.xs) {
      const float2 xs = e.xs[i];
      if (e.acc_ph) {
        const float2 ys = c_mul(mv, xs);
        e.acc_ph[i] += fmaf(val.y, ys.x, -val.x * ys.y);
      }
      if (e.acc_am) {
        const float2 mna = mod_value_planes(e, m.flags & ~TOP_MOD_AMPLITUDE, 0, fs.epi_lx, ly, rg, i, x);
        const float2 d = c_mul(mna, xs);
        e.acc_am[i] += fmaf(val.x, d.x, val.y * d.y);
      }
      if (e.acc_cm) {
        const float2 mnc = mod_value_planes(e, m.flags & ~TOP_MOD_COMPLEX, 0, fs.epi_lx, ly, rg, i, x);
        e.acc_cm[i] = c_add(e.acc_cm[i], c_mulc(val, c_mul(mnc, xs)));
      }
    }
  }
}

// Epilogue of one output sample val = psi(y, x) of field f in group g.
template <int KIND>
__device__ __forceinline__ void epilogue(const PassParams& p, const FieldSet& fs, int f, int g, bool first, int y,
                                         int x, float2 val, OvAcc& acc) {
  const long long idx = (long long)y * p.nx + x;
  if constexpr (KIND == EPI_OVERLAP) {
    if (p.mepi.flags) val = c_mul(val, mod_value(p.mepi, p.mepi.flags, p.mepi.conj, fs.epi_lx, fs.epi_ly, f, y, x, p.nx));
    if (p.out) p.out[(long long)f * p.out_stride + idx] = val;
    overlap_add(acc, val, ldg2(p.target + (long long)f * p.target_stride + idx));
  } else if constexpr (KIND == EPI_FIELD) {
    if (p.mepi.flags) val = c_mul(val, mod_value(p.mepi, p.mepi.flags, p.mepi.conj, fs.epi_lx, fs.epi_ly, f, y, x, p.nx));
    field_out(p, f)[idx] = val;
  } else if constexpr (KIND == EPI_INTENSITY) {
    if (p.mepi.flags) val = c_mul(val, mod_value(p.mepi, p.mepi.flags, p.mepi.conj, fs.epi_lx, fs.epi_ly, f, y, x, p.nx));
    if (p.out) p.out[(long long)f * p.out_stride + idx] = val;
    const float w = p.weights ? __ldg(p.weights + f) : 1.f;
    const float i = w * fmaf(val.x, val.x, val.y * val.y);
    float* dst = p.outf + (long long)g * p.outf_stride + idx;
    *dst = first ? i : *dst + i;
  } else {  // EPI_MODGRAD: val = dL/dy with y = M x (M without conjugation)
    const ModDev& m = p.mepi;
    const float2 mv = mod_value(m, m.flags, 0, fs.epi_lx, fs.epi_ly, f, y, x, p.nx);
    if (p.out) p.out[(long long)f * p.out_stride + idx] = c_mulc(val, mv);  // conj(M) dL/dy
    if (p.part_phase || p.part_amp || p.part_mask) {
      const float2 xs = ldg2(p.xs + (long long)f * p.xs_stride + idx);
      const long long pidx = (long long)g * p.part_stride + idx;
      const bool fresh = first && !p.part_accumulate;
      if (p.part_phase) {
        const float2 ys = c_mul(mv, xs);
        const float gp = fmaf(val.y, ys.x, -val.x * ys.y);  // Im(val conj(y))
        p.part_phase[pidx] = fresh ? gp : p.part_phase[pidx] + gp;
      }
      if (p.part_amp) {
        // dM/dA = M without its amplitude factor
        const float2 mna = mod_value(m, m.flags & ~TOP_MOD_AMPLITUDE, 0, fs.epi_lx, fs.epi_ly, f, y, x, p.nx);
        const float2 d = c_mul(mna, xs);
        const float ga = fmaf(val.x, d.x, val.y * d.y);  // Re(conj(val) d)
        p.part_amp[pidx] = fresh ? ga : p.part_amp[pidx] + ga;
      }
      if (p.part_mask) {
        const float2 mnc = mod_value(m, m.flags & ~TOP_MOD_COMPLEX, 0, fs.epi_lx, fs.epi_ly, f, y, x, p.nx);
        const float2 gm = c_mulc(val, c_mul(mnc, xs));  // val conj(M_rest x)
        p.part_mask[pidx] = fresh ? gm : c_add(p.part_mask[pidx], gm);
      }
    }
  }
}

// Combine the two inverse halves of each row in shared memory ([r][ROWS][M], natural order; the
// odd half already carries exp(2 pi i pos / P)) over the cropped window and hand every output
// sample to the epilogue (one cooperative loop; with padding exactly 2 its trip count is fixed).
template <class EX, bool X2, int KIND>
__device__ __forceinline__ void combine_rows(const PassParams& p, const FieldSet& fs, const float2* smem, int f, int g,
                                             bool first, int y0, int nrows, const EpiPlanes* ep, OvAcc& acc) {
  using SH = RowShape<EX>;
  constexpr int M = EX::M, ROWS = SH::ROWS, NT = SH::THREADS;
  if (ep) {
    const ModDev& m = p.mepi;
    for (int rr = 0; rr < nrows; ++rr) {
      const int y = y0 + rr;
      const int2 rg = (m.flags & TOP_MOD_CIRC) ? __ldg(m.circ + y) : make_int2(0, p.nx - 1);
      const float2 ly = (m.flags & TOP_MOD_LENS) ? ldg2(fs.epi_ly + y) : make_float2(1.f, 0.f);
      if constexpr (X2 && (M / 2) % NT == 0) {
        // nx = M: the lower half of the row combines e + o from slots M/2 on, the upper half e - o
        // from slot 0 on, a fixed number of samples a thread in each
        const float2* ev = smem + rr * M;
        const float2* od = smem + (ROWS + rr) * M;
#pragma unroll 4
        for (int i = 0; i < M / 2 / NT; ++i) {
          const int x = threadIdx.x + i * NT;
          epilogue_planes<KIND>(p, fs, *ep, f, first, y, x, rr * M + x, ly, rg,
                                c_add(ev[x + M / 2], od[x + M / 2]), acc);
        }
#pragma unroll 4
        for (int i = 0; i < M / 2 / NT; ++i) {
          const int x = M / 2 + threadIdx.x + i * NT;
          epilogue_planes<KIND>(p, fs, *ep, f, first, y, x, rr * M + x, ly, rg,
                                c_sub(ev[x - M / 2], od[x - M / 2]), acc);
        }
        continue;
      }
      for (int x = threadIdx.x; x < p.nx; x += NT) {
        int pos;
        bool upper;
        if constexpr (X2) {
          upper = x >= M / 2;
          pos = upper ? x - M / 2 : x + M / 2;
        } else {
          const int pp = x + p.ox;
          upper = pp >= M;
          pos = upper ? pp - M : pp;
        }
        const float2 o = smem[(ROWS + rr) * M + pos];
        const float2 ev = smem[rr * M + pos];
        epilogue_planes<KIND>(p, fs, *ep, f, first, y, x, rr * p.nx + x, ly, rg, upper ? c_sub(ev, o) : c_add(ev, o),
                              acc);
      }
    }
    return;
  }
  auto one = [&](int rr, int x) {
    int pos;
    bool upper;
    if constexpr (X2) {
      upper = x >= M / 2;
      pos = upper ? x - M / 2 : x + M / 2;
    } else {
      const int pp = x + p.ox;
      upper = pp >= M;
      pos = upper ? pp - M : pp;
    }
    const float2 o = smem[(ROWS + rr) * M + pos];
    const float2 ev = smem[rr * M + pos];
    epilogue<KIND>(p, fs, f, g, first, y0 + rr, x, upper ? c_sub(ev, o) : c_add(ev, o), acc);
  };
  if constexpr (X2 && M % NT == 0) {
    for (int rr = 0; rr < nrows; ++rr) {
#pragma unroll 4
      for (int i = 0; i < M / NT; ++i) one(rr, threadIdx.x + i * NT);
    }
  } else {
    for (int rr = 0; rr < nrows; ++rr)
      for (int x = threadIdx.x; x < p.nx; x += NT) one(rr, x);
  }
}

// Bins of this thread's half row (row y0 + row of field f) straight from the workspace into
// registers (two-stage plans): four consecutive lanes read one 32-byte sector.
template <class EX>
__device__ __forceinline__ void load_bins(const PassParams& p, int f, int y0, int nrows, int grp, int t,
                                          float2 (&v)[EX::E]) {
  constexpr int E = EX::E, M = EX::M;
  const int row = grp >> 1, r = grp & 1;
  if (row < nrows) {
    const float2* wp = p.ws + (long long)f * p.ws_stride + direct_base<EX>(r, t, y0 + row, p.ny);
    const int step = (M / EX::RL) * p.ny;
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = wp[e * step];
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = make_float2(0.f, 0.f);
  }
}

// Inverse-transform the bins in v and leave both halves in natural order in shared memory
// [r][ROWS][M] at `smem`, the odd one times exp(2 pi i pos / P). Ends before the barrier that makes
// the halves visible.
template <class EX, bool X2>
__device__ __forceinline__ void inverse_halves(const PassParams& p, float2 (&v)[EX::E], float2* smem, int grp, int t) {
  using SH = RowShape<EX>;
  constexpr int E = EX::E, M = EX::M, ROWS = SH::ROWS;
  const int row = grp >> 1, r = grp & 1;
  EX::inv(v, smem + grp * EX::BUF, t, p.twx);
  __syncthreads();  // the exchange buffers alias the half-row buffers
  float2* hrow = smem + (r * ROWS + row) * M;
  if (r) {
    if constexpr (X2) {
      const float2 wt = ldg2(p.wpx + t);
      for_slots(
          [&](auto ec) {
            constexpr int e = decltype(ec)::value;
            hrow[EX::in_pos(t, e)] = c_mulc(v[e], slot_split_twiddle<EX, e>(wt));
          },
          std::make_integer_sequence<int, E>{});
    } else {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int pos = EX::in_pos(t, e);
        hrow[pos] = c_mulc(v[e], ldg2(p.wpx + pos));
      }
    }
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) hrow[EX::in_pos(t, e)] = v[e];
  }
}

// Load the bins of rows y0 .. y0 + nrows - 1 of field f, inverse-transform them and leave both
// halves in natural order in shared memory [r][ROWS][M] at `smem`, the odd one times
// exp(2 pi i pos / P). Ends before the barrier that makes the halves visible.
template <class EX, bool X2>
__device__ __forceinline__ void inverse_rows(const PassParams& p, int f, int y0, int nrows, float2* smem, int grp,
                                             int t) {
  using SH = RowShape<EX>;
  constexpr int E = EX::E, M = EX::M, ROWS = SH::ROWS, LD = SH::LD, NT = SH::THREADS;
  const int row = grp >> 1, r = grp & 1;
  const int ny = p.ny;
  const float2* ws = p.ws + (long long)f * p.ws_stride;
  float2 v[E];
  if constexpr (SH::DIRECT) {
    load_bins<EX>(p, f, y0, nrows, grp, t, v);
  } else {
    // the tile [2M][LD] from the workspace in address order (ROWS rows x 4 lines per block)
    for (int i = threadIdx.x; i < 2 * M * ROWS; i += NT) {
      const int c = i & 3, q = i >> 2;
      const int yo = q % ROWS, blk = q / ROWS;
      smem[SH::tslot(4 * blk + c) * LD + yo] =
          yo < nrows ? ws[((long long)blk * ny + y0 + yo) * 4 + c] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = smem[SH::tslot(r * M + EX::bin(t, e)) * LD + row];
    __syncthreads();  // the tile aliases the exchange buffers
  }
  inverse_halves<EX, X2>(p, v, smem, grp, t);
}

template <class EX, bool X2>
__global__ void __launch_bounds__(RowShape<EX>::THREADS, RowShape<EX>::MINB_INV) k_rows_inv(const __grid_constant__ PassParams p) {
  using SH = RowShape<EX>;
  constexpr int G = EX::G, E = EX::E, M = EX::M, ROWS = SH::ROWS, LD = SH::LD, NT = SH::THREADS;
  TOP_DYN_SMEM(float2, smem);
  int grp, t;
  group_lane<G>(threadIdx.x, grp, t);
  const int row = grp >> 1, r = grp & 1;
  const int y0 = blockIdx.x * ROWS;
  const int nrows = min(ROWS, p.ny - y0);
  const int g = blockIdx.y;
  const int f0 = g * p.group;
  const int f1 = min(f0 + p.group, p.nfields);
  const int ny = p.ny;

  // staged epilogue planes: accumulators and shared mask rows once per block, the saved input
  // and per-field mask rows once per field (copied while the field is transformed)
  const bool staged = epi_staged<EX>(p);
  EpiPlanes ep{};
  const int nx = p.nx;
  const int plane = ROWS * nx;
  const long long row0 = (long long)y0 * nx;
  const ModDev& m = p.mepi;
  const bool grads = p.epi_kind == EPI_MODGRAD && (p.part_phase || p.part_amp || p.part_mask);
  if (staged) {
    float* pl = reinterpret_cast<float*>(smem + SH::SMEM / sizeof(float2));
    auto carve = [&](int floats_per_sample) {
      float* d = pl;
      pl += plane * floats_per_sample;
      return d;
    };
    auto copy_in = [&](float* dst, const float* src, int floats_per_sample) {
      const float4* s4 = reinterpret_cast<const float4*>(src);
      float4* d4 = reinterpret_cast<float4*>(dst);
      const int n4 = nrows * nx * floats_per_sample / 4;
      for (int i = threadIdx.x; i < n4; i += NT) top_cp_async16(d4 + i, s4 + i);
    };
    if (p.epi_kind == EPI_INTENSITY) ep.acc_i = carve(1);
    if (grads) {
      const long long pidx = (long long)g * p.part_stride + row0;
      auto acc = [&](float* dst, const float* src, int fps) {
        if (p.part_accumulate) {
          copy_in(dst, src, fps);
        } else {
          for (int i = threadIdx.x; i < nrows * nx * fps; i += NT) dst[i] = 0.f;
        }
      };
      if (p.part_phase) { ep.acc_ph = carve(1); acc(ep.acc_ph, p.part_phase + pidx, 1); }
      if (p.part_amp) { ep.acc_am = carve(1); acc(ep.acc_am, p.part_amp + pidx, 1); }
      if (p.part_mask) {
        ep.acc_cm = reinterpret_cast<float2*>(carve(2));
        acc(reinterpret_cast<float*>(ep.acc_cm), reinterpret_cast<const float*>(p.part_mask + pidx), 2);
      }
      ep.xs = reinterpret_cast<const float2*>(carve(2));
    }
    if (m.flags & TOP_MOD_PHASE) ep.ph = carve(1);
    if (m.flags & TOP_MOD_AMPLITUDE) ep.am = carve(1);
    if (m.flags & TOP_MOD_COMPLEX) ep.cm = reinterpret_cast<const float2*>(carve(2));
    if (m.stride == 0) {
      if (ep.ph) copy_in(const_cast<float*>(ep.ph), m.phase + row0, 1);
      if (ep.am) copy_in(const_cast<float*>(ep.am), m.amp + row0, 1);
      if (ep.cm) copy_in(reinterpret_cast<float*>(const_cast<float2*>(ep.cm)), reinterpret_cast<const float*>(m.cmask + row0), 2);
    }
  }
  auto stage_field = [&](int f) {
    auto copy_in = [&](float* dst, const float* src, int floats_per_sample) {
      const float4* s4 = reinterpret_cast<const float4*>(src);
      float4* d4 = reinterpret_cast<float4*>(dst);
      const int n4 = nrows * nx * floats_per_sample / 4;
      for (int i = threadIdx.x; i < n4; i += NT) top_cp_async16(d4 + i, s4 + i);
    };
    if (grads)
      copy_in(reinterpret_cast<float*>(const_cast<float2*>(ep.xs)),
              reinterpret_cast<const float*>(p.xs + (long long)f * p.xs_stride + row0), 2);
    if (m.stride != 0) {
      const long long midx = (long long)f * m.stride + row0;
      if (ep.ph) copy_in(const_cast<float*>(ep.ph), m.phase + midx, 1);
      if (ep.am) copy_in(const_cast<float*>(ep.am), m.amp + midx, 1);
      if (ep.cm) copy_in(reinterpret_cast<float*>(const_cast<float2*>(ep.cm)), reinterpret_cast<const float*>(m.cmask + midx), 2);
    }
  };

  // two-stage plans load the next field's bins into the registers the transform has freed while
  // the current field's halves are combined, so the loads overlap the epilogue
  float2 v[E];
  if constexpr (SH::DIRECT) load_bins<EX>(p, f0, y0, nrows, grp, t, v);
#pragma unroll 1
  for (int f = f0; f < f1; ++f) {
    const FieldSet& fs = p.sets[p.set_of[f]];
    if (staged) stage_field(f);
    if constexpr (SH::DIRECT) {
      inverse_halves<EX, X2>(p, v, smem, grp, t);
    } else {
      inverse_rows<EX, X2>(p, f, y0, nrows, smem, grp, t);
    }
    if (staged) top_cp_async_wait_all();
    __syncthreads();
    if constexpr (SH::DIRECT) {
      if (f + 1 < f1) load_bins<EX>(p, f + 1, y0, nrows, grp, t, v);
    }
    // combine the halves over the cropped window, epilogue, coalesced store
    const EpiPlanes* epp = staged ? &ep : nullptr;
    OvAcc acc{0.0, 0.0, 0.0};
    if (p.epi_kind == EPI_FIELD) {
      combine_rows<EX, X2, EPI_FIELD>(p, fs, smem, f, g, f == f0, y0, nrows, epp, acc);
    } else if (p.epi_kind == EPI_INTENSITY) {
      combine_rows<EX, X2, EPI_INTENSITY>(p, fs, smem, f, g, f == f0, y0, nrows, epp, acc);
    } else if (p.epi_kind == EPI_MODGRAD) {
      combine_rows<EX, X2, EPI_MODGRAD>(p, fs, smem, f, g, f == f0, y0, nrows, epp, acc);
    } else {
      combine_rows<EX, X2, EPI_OVERLAP>(p, fs, smem, f, g, f == f0, y0, nrows, epp, acc);
      // the block's sums in a fixed order: every thread's three values, added by thread 0
      __syncthreads();
      double* red = reinterpret_cast<double*>(smem);
      red[3 * threadIdx.x] = acc.re;
      red[3 * threadIdx.x + 1] = acc.im;
      red[3 * threadIdx.x + 2] = acc.pw;
      __syncthreads();
      if (threadIdx.x == 0) {
        double sr = 0.0, si = 0.0, sp = 0.0;
        for (int i = 0; i < NT; ++i) {
          sr += red[3 * i];
          si += red[3 * i + 1];
          sp += red[3 * i + 2];
        }
        double* out = p.ov_part + ((long long)f * gridDim.x + blockIdx.x) * 3;
        out[0] = sr;
        out[1] = si;
        out[2] = sp;
      }
    }
    __syncthreads();
  }
  if (staged) {
    // accumulators of the group back to global memory
    auto copy_out = [&](float* dst, const float* src, int floats_per_sample) {
      float4* d4 = reinterpret_cast<float4*>(dst);
      const float4* s4 = reinterpret_cast<const float4*>(src);
      const int n4 = nrows * nx * floats_per_sample / 4;
      for (int i = threadIdx.x; i < n4; i += NT) d4[i] = s4[i];
    };
    if (ep.acc_i) copy_out(p.outf + (long long)g * p.outf_stride + row0, ep.acc_i, 1);
    const long long pidx = (long long)g * p.part_stride + row0;
    if (ep.acc_ph) copy_out(p.part_phase + pidx, ep.acc_ph, 1);
    if (ep.acc_am) copy_out(p.part_amp + pidx, ep.acc_am, 1);
    if (ep.acc_cm) copy_out(reinterpret_cast<float*>(p.part_mask + pidx), reinterpret_cast<const float*>(ep.acc_cm), 2);
  }
}

// ----------------------------------------------------------------------------- R2 + R1 fused

// Shared memory of a fused chain block, in float2 units: the row-pass region, whose tail past
// the two half rows [2][ROWS][M] also holds the field rows between the two propagations (they
// are written after the exchanges of the inverse transform and read before those of the forward
// one), then the next propagation's source planes, which arrive during the inverse transform.
template <class EN>
__host__ __device__ inline size_t chain_rows_off() {
  return size_t(2) * RowShape<EN>::ROWS * EN::M;
}
template <class EN>
__host__ __device__ inline size_t chain_planes_off(int nx) {
  const size_t end_rows = chain_rows_off<EN>() + size_t(RowShape<EN>::ROWS) * nx;
  const size_t region = RowShape<EN>::SMEM / sizeof(float2);
  return end_rows > region ? end_rows : region;
}
template <class EN>
__host__ __device__ inline size_t chain_smem(const PassParams& next) {
  return sizeof(float2) * chain_planes_off<EN>(next.nx) + sizeof(float) * src_plane_floats(next, RowShape<EN>::ROWS);
}

// The inverse row pass of one propagation (pa) fused with the forward row pass of the next (pb)
// in a system chain (Eq. 1 and Eq. 4 in turn): the field between them stays in shared memory
// and reaches global memory only when it is kept (pa.out). pb's bins replace pa's in the
// workspace, row tile by row tile, each block reading its tile before writing it.
template <class EX, bool X2>
__global__ void __launch_bounds__(RowShape<EX>::THREADS, RowShape<EX>::MINB_INV)
    k_rows_chain(const __grid_constant__ PassParams pa, const __grid_constant__ PassParams pb) {
  using SH = RowShape<EX>;
  constexpr int M = EX::M, ROWS = SH::ROWS, NT = SH::THREADS;
  TOP_DYN_SMEM(float2, smem);
  int grp, t;
  group_lane<EX::G>(threadIdx.x, grp, t);
  const int y0 = blockIdx.x * ROWS;
  const int nrows = min(ROWS, pa.ny - y0);
  const int f = blockIdx.y;
  const int nx = pa.nx;
  float2* rows = smem + chain_rows_off<EX>();  // [ROWS][nx]
  // the next propagation's modulation planes arrive while this one is finished
  const SrcPlanes sp = stage_src_planes<EX>(pb, f, y0, nrows, reinterpret_cast<float*>(smem + chain_planes_off<EX>(nx)));
  inverse_rows<EX, X2>(pa, f, y0, nrows, smem, grp, t);
  __syncthreads();
  if constexpr (X2 && (M / 2) % NT == 0) {
    // nx = M: lower half e + o from slots M/2 on, upper half e - o from slot 0 on
    for (int rr = 0; rr < ROWS; ++rr) {
      const float2* ev = smem + rr * M;
      const float2* od = smem + (ROWS + rr) * M;
      float2* out = pa.out ? pa.out + (long long)f * pa.out_stride + (long long)(y0 + rr) * nx : nullptr;
      const bool live = rr < nrows;
#pragma unroll 4
      for (int i = 0; i < M / NT; ++i) {
        const int x = threadIdx.x + i * NT;
        const bool upper = i >= M / 2 / NT;
        const int pos = upper ? x - M / 2 : x + M / 2;
        float2 val = make_float2(0.f, 0.f);
        if (live) {
          val = upper ? c_sub(ev[pos], od[pos]) : c_add(ev[pos], od[pos]);
          if (out) out[x] = val;
        }
        rows[rr * M + x] = val;
      }
    }
  } else {
  for (int rr = 0; rr < ROWS; ++rr) {
    for (int x = threadIdx.x; x < nx; x += NT) {
      float2 val = make_float2(0.f, 0.f);
      if (rr < nrows) {
        int pos;
        bool upper;
        if constexpr (X2) {
          upper = x >= M / 2;
          pos = upper ? x - M / 2 : x + M / 2;
        } else {
          const int pp = x + pa.ox;
          upper = pp >= M;
          pos = upper ? pp - M : pp;
        }
        const float2 o = smem[(ROWS + rr) * M + pos];
        const float2 ev = smem[rr * M + pos];
        val = upper ? c_sub(ev, o) : c_add(ev, o);
        if (pa.out) pa.out[(long long)f * pa.out_stride + (long long)(y0 + rr) * nx + x] = val;
      }
      rows[rr * nx + x] = val;
    }
  }
  }
  top_cp_async_wait_all();
  __syncthreads();
  if (pb.msrc.flags) {
    modulate_src_rows<EX>(pb, pb.sets[pb.set_of[f]], f, y0, nrows, rows, sp);
    __syncthreads();
  }
  forward_rows<EX, X2>(pb, f, y0, nrows, rows, smem, grp, t);
}

}  // namespace top

#include "top_pair_rows.cuh"

namespace top {

// ----------------------------------------------------------------------------- launchers

template <class K>
inline cudaError_t set_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Blocks of a kernel resident on the whole device at the given block shape (0 if unknown).
template <class K>
inline int resident_blocks(K kernel, int threads, size_t smem) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess)
    return 0;
  return sms * per_sm;
}

#ifndef TOP_L2_AHEAD
#define TOP_L2_AHEAD 1
#endif
// How far ahead the column pass prefetches, in hundredths of a wave of resident blocks.
#ifndef TOP_L2_WAVES
#define TOP_L2_WAVES 100
#endif

// Whether the pair-local row passes take the rows of plan EX at padding exactly 2.
#ifndef TOP_PAIR_ROWS
#define TOP_PAIR_ROWS 1
#endif
template <class EX>
constexpr bool pair_rows() {
  return TOP_PAIR_ROWS && PairRows<EX>::OK;
}
// Epilogues the pair-local inverse pass covers.
inline bool pair_epilogue(const PassParams& p) {
  return p.nx % 4 == 0 && (p.epi_kind == EPI_FIELD || p.epi_kind == EPI_INTENSITY ||
                           (p.epi_kind == EPI_MODGRAD && !p.part_amp && !p.part_mask));
}

// Largest shared memory of a pair-local block: the exchange buffers and, after them, two rows of
// staged operands (at most eight floats a sample).
template <class EX>
constexpr size_t pair_smem_max() {
  return PairRows<EX>::SMEM + sizeof(float) * 2 * 8 * EX::M;
}

// The pair-local forward pass stages its source row in the pair's exchange buffers.
template <class EX>
inline bool pair_fwd_fits(const PassParams& p) {
  return p.nx % 4 == 0 && size_t(pair_src_floats(p)) * sizeof(float) <= 2 * EX::BUF * sizeof(float2);
}

// The pair kernels are compiled for the modulation flag sets of common elements (none, a lens or
// a phase mask behind an aperture) and for flags read at run time.
constexpr uint32_t kLensCirc = TOP_MOD_LENS | TOP_MOD_CIRC;
constexpr uint32_t kPhaseCirc = TOP_MOD_PHASE | TOP_MOD_CIRC;

template <class EX, uint32_t MF>
cudaError_t launch_rows_fwd_pair_k(const PassParams& p, cudaStream_t s) {
  using PR = PairRows<EX>;
  static const cudaError_t attr = set_smem(k_rows_fwd_pair<EX, MF>, PR::SMEM);
  if (attr != cudaSuccess) return attr;
  static const int resident = resident_blocks(k_rows_fwd_pair<EX, MF>, PR::THREADS, PR::SMEM);
  PassParams q = p;
  q.l2_ahead = TOP_L2_AHEAD && !(p.tune_rows & TOP_TUNE_NO_L2_FWD) ? resident : 0;
  dim3 grid((p.ny + PR::ROWS - 1) / PR::ROWS, p.nfields);
  TOP_LAUNCH((k_rows_fwd_pair<EX, MF>), grid, PR::THREADS, PR::SMEM, s, q);
  return cudaGetLastError();
}

template <class EX>
cudaError_t launch_rows_fwd_pair(const PassParams& p, cudaStream_t s) {
  if (p.msrc.flags == 0) return launch_rows_fwd_pair_k<EX, 0>(p, s);
  if (p.msrc.flags == kLensCirc) return launch_rows_fwd_pair_k<EX, kLensCirc>(p, s);
  return launch_rows_fwd_pair_k<EX, TOP_MOD_DYNAMIC>(p, s);
}

template <class EX, int KIND, uint32_t MF>
cudaError_t launch_rows_inv_pair_k(const PassParams& p, cudaStream_t s) {
  using PR = PairRows<EX>;
  static const cudaError_t attr = set_smem(k_rows_inv_pair<EX, KIND, MF>, pair_smem_max<EX>());
  if (attr != cudaSuccess) return attr;
  PassParams q = p;
  // a field epilogue has no group: a block runs its rows of a few consecutive fields
  if (KIND == EPI_FIELD) q.group = p.nfields < tune_span(p.tune_rows) ? p.nfields : tune_span(p.tune_rows);
  const size_t bytes = PR::SMEM + sizeof(float) * 2 * size_t((pair_epi_floats<KIND>(q) + 3) & ~3);
  dim3 grid((q.ny + PR::ROWS - 1) / PR::ROWS, (q.nfields + q.group - 1) / q.group);
  TOP_LAUNCH((k_rows_inv_pair<EX, KIND, MF>), grid, PR::THREADS, bytes, s, q);
  return cudaGetLastError();
}

template <class EX>
cudaError_t launch_rows_inv_pair(const PassParams& p, cudaStream_t s) {
  const uint32_t fl = p.mepi.flags;
  if (p.epi_kind == EPI_FIELD)
    return fl == 0 ? launch_rows_inv_pair_k<EX, EPI_FIELD, 0>(p, s) : launch_rows_inv_pair_k<EX, EPI_FIELD, TOP_MOD_DYNAMIC>(p, s);
  if (p.epi_kind == EPI_INTENSITY)
    return fl == 0 ? launch_rows_inv_pair_k<EX, EPI_INTENSITY, 0>(p, s)
                   : launch_rows_inv_pair_k<EX, EPI_INTENSITY, TOP_MOD_DYNAMIC>(p, s);
  return fl == kPhaseCirc ? launch_rows_inv_pair_k<EX, EPI_MODGRAD, kPhaseCirc>(p, s)
                          : launch_rows_inv_pair_k<EX, EPI_MODGRAD, TOP_MOD_DYNAMIC>(p, s);
}

template <class EX, uint32_t MF>
cudaError_t launch_rows_chain_pair_k(const PassParams& pa, const PassParams& pb, cudaStream_t s) {
  using PR = PairRows<EX>;
  static const cudaError_t attr = set_smem(k_rows_chain_pair<EX, MF>, pair_smem_max<EX>());
  if (attr != cudaSuccess) return attr;
  const size_t bytes = PR::SMEM + sizeof(float) * 2 * size_t((pair_mod_floats(pb.msrc.flags, pb.nx) + 3) & ~3);
  dim3 grid((pa.ny + PR::ROWS - 1) / PR::ROWS, pa.nfields);
  TOP_LAUNCH((k_rows_chain_pair<EX, MF>), grid, PR::THREADS, bytes, s, pa, pb);
  return cudaGetLastError();
}

template <class EX>
cudaError_t launch_rows_chain_pair(const PassParams& pa, const PassParams& pb, cudaStream_t s) {
  const uint32_t fl = pb.msrc.flags;
  if (fl == kLensCirc) return launch_rows_chain_pair_k<EX, kLensCirc>(pa, pb, s);
  if (fl == kPhaseCirc) return launch_rows_chain_pair_k<EX, kPhaseCirc>(pa, pb, s);
  if (fl == 0) return launch_rows_chain_pair_k<EX, 0>(pa, pb, s);
  return launch_rows_chain_pair_k<EX, TOP_MOD_DYNAMIC>(pa, pb, s);
}

template <class EX, bool X2>
cudaError_t launch_rows_fwd_t(const PassParams& p, cudaStream_t s) {
  using SH = RowShape<EX>;
  const auto launch = [&](auto kernel) {
    static const cudaError_t attr = set_smem(kernel, SH::SMEM_SRC_MAX);
    if (attr != cudaSuccess) return attr;
    dim3 grid((p.ny + SH::ROWS - 1) / SH::ROWS, p.nfields);
    const size_t bytes = SH::SMEM + (src_staged<EX>(p) ? sizeof(float) * src_plane_floats(p, SH::ROWS) : 0);
    TOP_LAUNCH(kernel, grid, SH::THREADS, bytes, s, p);
    return cudaGetLastError();
  };
  if constexpr (SH::FWD_B2) {
    return launch(k_rows_fwd_b2<EX, X2>);
  } else {
    return launch(k_rows_fwd<EX, X2>);
  }
}


template <class EY, bool X2>
cudaError_t launch_cols_t(const PassParams& p, cudaStream_t s) {
  using SH = ColShape<EY>;
  static const cudaError_t attr = set_smem(k_cols<EY, X2>, SH::SMEM_MAX);
  if (attr != cudaSuccess) return attr;
  const size_t bytes = SH::template smem<X2>(p.ny);
  static const int resident = resident_blocks(k_cols<EY, X2>, SH::THREADS, bytes);
  PassParams q = p;
  q.l2_ahead = TOP_L2_AHEAD && !(p.tune_cols & TOP_TUNE_NO_L2_COLS) ? resident * TOP_L2_WAVES / 100 : 0;
  dim3 grid((p.Px + SH::COLS - 1) / SH::COLS, p.nfields);
  TOP_LAUNCH((k_cols<EY, X2>), grid, SH::THREADS, bytes, s, q);
  return cudaGetLastError();
}

template <class EX, bool X2>
cudaError_t launch_rows_inv_t(const PassParams& p, cudaStream_t s) {
  using SH = RowShape<EX>;
  static const cudaError_t attr = set_smem(k_rows_inv<EX, X2>, SH::SMEM_EPI_MAX);
  if (attr != cudaSuccess) return attr;
  dim3 grid((p.ny + SH::ROWS - 1) / SH::ROWS, (p.nfields + p.group - 1) / p.group);
  const size_t bytes =
      SH::SMEM + (epi_staged<EX>(p) ? sizeof(float) * size_t(epi_plane_floats(p)) * SH::ROWS * p.nx : 0);
  TOP_LAUNCH((k_rows_inv<EX, X2>), grid, SH::THREADS, bytes, s, p);
  return cudaGetLastError();
}

template <class EX, bool X2>
cudaError_t launch_rows_chain_t(const PassParams& pa, const PassParams& pb, cudaStream_t s) {
  using SH = RowShape<EX>;
  static const cudaError_t attr = set_smem(k_rows_chain<EX, X2>, kChainSmemMax);
  if (attr != cudaSuccess) return attr;
  const size_t bytes = chain_smem<EX>(pb);
  if (bytes > kChainSmemMax) return cudaErrorInvalidValue;
  dim3 grid((pa.ny + SH::ROWS - 1) / SH::ROWS, pa.nfields);
  TOP_LAUNCH((k_rows_chain<EX, X2>), grid, SH::THREADS, bytes, s, pa, pb);
  return cudaGetLastError();
}

// padding exactly 2 along an axis: n = M and the field sits at M/2
inline bool exact2(int n, int M, int o) { return n == M && o == M / 2; }

template <class EX>
cudaError_t launch_rows_fwd(const PassParams& p, cudaStream_t s) {
  if constexpr (pair_rows<EX>()) {
    if (exact2(p.nx, p.Mx, p.ox) && pair_fwd_fits<EX>(p) && !(p.tune_rows & TOP_TUNE_CLASSIC_FWD))
      return launch_rows_fwd_pair<EX>(p, s);
  }
  return exact2(p.nx, p.Mx, p.ox) ? launch_rows_fwd_t<EX, true>(p, s) : launch_rows_fwd_t<EX, false>(p, s);
}

template <class EY>
cudaError_t launch_cols(const PassParams& p, cudaStream_t s) {
  return exact2(p.ny, p.My, p.oy) ? launch_cols_t<EY, true>(p, s) : launch_cols_t<EY, false>(p, s);
}

template <class EX>
cudaError_t launch_rows_chain(const PassParams& pa, const PassParams& pb, cudaStream_t s) {
  if constexpr (pair_rows<EX>()) {
    if (exact2(pa.nx, pa.Mx, pa.ox) && pa.nx % 4 == 0 && !(pa.tune_rows & TOP_TUNE_CLASSIC_CHAIN))
      return launch_rows_chain_pair<EX>(pa, pb, s);
  }
  return exact2(pa.nx, pa.Mx, pa.ox) ? launch_rows_chain_t<EX, true>(pa, pb, s) : launch_rows_chain_t<EX, false>(pa, pb, s);
}

template <class EX>
cudaError_t launch_rows_inv(const PassParams& p, cudaStream_t s) {
  if constexpr (pair_rows<EX>()) {
    if (exact2(p.nx, p.Mx, p.ox) && pair_epilogue(p) && !(p.tune_rows & TOP_TUNE_CLASSIC_INV))
      return launch_rows_inv_pair<EX>(p, s);
  }
  return exact2(p.nx, p.Mx, p.ox) ? launch_rows_inv_t<EX, true>(p, s) : launch_rows_inv_t<EX, false>(p, s);
}

}  // namespace top
