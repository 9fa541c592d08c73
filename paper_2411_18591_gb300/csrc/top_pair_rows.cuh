// Row passes of the two-stage plans that give each half line one warp, at padding exactly 2
// (n = M samples at offset M/2): the two warps of a row trade halves through shared memory once
// per direction, with no block barrier and no row buffer (included by top_passes.cuh).
//
// At padding 2 every stage-0 position pos of a half line stands for one field sample,
// x(pos) = pos + M/2 below M/2 and pos - M/2 above (the fold of Eq. 4's zero-padded row has a
// single term per slot). The even half's input at pos is psi[x(pos)], the odd half's is
// -/+ w^pos psi[x(pos)] with w = exp(-2 pi i / P); after the inverse transforms
// psi[x(pos)] = E[pos] -/+ O'[pos], O' = conj(w^pos) O. Lane t holds the same positions in both
// warps, so the even warp owns the slots with pos < M/2 and the odd warp the others: each warp
// computes the samples of its own slots (combine, modulation of Eq. 1, epilogue) and receives
// the rest from its partner. For these plans pos < M/2 exactly when e mod R0 < R0/2, so the
// split is fixed at compile time per slot.
#pragma once

#include "top_passes.cuh"

namespace top {

// Blocks per SM the pair-local inverse pass is compiled for (its group loop holds the next
// field's bins, this field's samples and the group sums in registers at once).
#ifndef TOP_PAIR_INV_MINB
#define TOP_PAIR_INV_MINB 3
#endif
// Blocks per SM the pair-local fused row pass is compiled for.
#ifndef TOP_PAIR_CHAIN_MINB
#define TOP_PAIR_CHAIN_MINB 4
#endif
// Whether the fused row pass runs its forward transform in the compact (looped) form too.
#ifndef TOP_CHAIN_FWD_COMPACT
#define TOP_CHAIN_FWD_COMPACT 1
#endif
// Whether the inverse pass loads the next field's bins before this field's epilogue.
#ifndef TOP_PAIR_PREFETCH
#define TOP_PAIR_PREFETCH 1
#endif

template <class EX>
struct PairRows {
  // two-stage plans with one butterfly a thread (direct bins) and one warp per half line
  static constexpr bool OK = EX::NS == 2 && EX::E == EX::RL && EX::G == 32 && (EX::M / EX::RL) % 4 == 0 &&
                             EX::radix(0) % 2 == 0;
  static constexpr int ROWS = 2;                     // rows per block (named barrier ids 1 .. ROWS)
  static constexpr int THREADS = 2 * ROWS * EX::G;   // one warp per half line
  static constexpr size_t SMEM = sizeof(float2) * 2 * ROWS * EX::BUF;
  static constexpr int H = EX::E / 2;                // own slots of a warp
  static constexpr int R0 = EX::radix(0);
  // k-th slot below M/2 (its partner above M/2 is lo(k) + R0/2, at position + M/2)
  __host__ __device__ static constexpr int lo(int k) { return (k / (R0 / 2)) * R0 + k % (R0 / 2); }
  __host__ __device__ static constexpr int hi(int k) { return lo(k) + R0 / 2; }
};

// Modulation flags a pair kernel is compiled for; TOP_MOD_DYNAMIC reads them at run time.
constexpr uint32_t TOP_MOD_DYNAMIC = 0xffffffffu;

template <uint32_t MF>
__device__ __forceinline__ uint32_t mod_flags(const ModDev& m) {
  return MF == TOP_MOD_DYNAMIC ? m.flags : MF;
}

// The two warps of row `row` of the block.
__device__ __forceinline__ void pair_sync(int row) { top_named_barrier(1 + row, 64); }

// Bins of half r of row y of field f straight from the workspace (four lanes read one sector).
template <class EX>
__device__ __forceinline__ void pair_load_bins(const PassParams& p, int f, int y, int r, int t, float2 (&v)[EX::E]) {
  const float2* wp = p.ws + (long long)f * p.ws_stride + direct_base<EX>(r, t, y, p.ny);
  const int step = (EX::M / EX::RL) * p.ny;
#pragma unroll
  for (int e = 0; e < EX::E; ++e) v[e] = wp[e * step];
}

template <class EX>
__device__ __forceinline__ void pair_store_bins(const PassParams& p, int f, int y, int r, int t,
                                                const float2 (&v)[EX::E]) {
  float2* wp = p.ws + (long long)f * p.ws_stride + direct_base<EX>(r, t, y, p.ny);
  const int step = (EX::M / EX::RL) * p.ny;
#pragma unroll
  for (int e = 0; e < EX::E; ++e) wp[e * step] = v[e];
}

// The block l2_ahead blocks later in launch order (the next wave of resident blocks), whose source
// rows the forward pass prefetches into L2.
__device__ __forceinline__ bool ahead_block(const PassParams& p, int& f, int& tile) {
  if (p.l2_ahead <= 0) return false;
  const long long lb = (long long)blockIdx.y * gridDim.x + blockIdx.x + p.l2_ahead;
  if (lb >= (long long)gridDim.x * gridDim.y) return false;
  f = int(lb / gridDim.x);
  tile = int(lb % gridDim.x);
  return true;
}

// Positions of lane t: own slot k of warp r sits at lo_pos(k) + (r ? M/2 : 0), its field sample
// (and the partner's slot k) at x(k) = lo_pos(k) + (r ? 0 : M/2).
template <class EX>
__device__ __forceinline__ int lo_pos(int t, int k) {
  return EX::in_pos(t, PairRows<EX>::lo(k));
}

// After the inverse transforms (v = E in the even warp, O' in the odd one): trade the partner's
// slots and return this warp's own samples psi[x(k)] in o.
template <class EX>
__device__ __forceinline__ void pair_combine(const float2 (&v)[EX::E], float2 (&o)[PairRows<EX>::H], float2* mine,
                                             const float2* theirs, int r, int t, int row) {
  using PR = PairRows<EX>;
  constexpr int HM = EX::M / 2;
  const int own_off = r ? HM : 0, x_off = r ? 0 : HM;
  EX::sync_group();  // this warp's last reads of its exchange buffer are done
#pragma unroll
  for (int k = 0; k < PR::H; ++k) mine[lo_pos<EX>(t, k) + x_off] = r ? v[PR::lo(k)] : v[PR::hi(k)];
  pair_sync(row);
#pragma unroll
  for (int k = 0; k < PR::H; ++k) {
    const float2 q = theirs[lo_pos<EX>(t, k) + own_off];
    o[k] = r ? c_add(q, v[PR::hi(k)]) : c_sub(v[PR::lo(k)], q);
  }
}

// This warp's own samples in o: trade them so both warps hold every slot in v, and apply the odd
// half's fold twiddle. Ends with the pair barrier after which the exchange buffers are free. (The
// positions written here are disjoint from those pair_combine wrote, so no barrier is needed
// between the two.)
template <class EX>
__device__ __forceinline__ void pair_spread(float2 (&v)[EX::E], const float2 (&o)[PairRows<EX>::H], float2* mine,
                                            const float2* theirs, int r, int t, int row, const float2* __restrict__ wp) {
  using PR = PairRows<EX>;
  constexpr int HM = EX::M / 2;
  const int own_off = r ? HM : 0, x_off = r ? 0 : HM;
#pragma unroll
  for (int k = 0; k < PR::H; ++k) mine[lo_pos<EX>(t, k) + own_off] = o[k];
  pair_sync(row);
#pragma unroll
  for (int k = 0; k < PR::H; ++k) {
    const float2 q = theirs[lo_pos<EX>(t, k) + x_off];
    v[PR::lo(k)] = r ? q : o[k];
    v[PR::hi(k)] = r ? o[k] : q;
  }
  if (r) {
    const float2 wt = ldg2(wp + t);
    for_slots(
        [&](auto ec) {
          constexpr int e = decltype(ec)::value;
          constexpr bool low = (e % PR::R0) < PR::R0 / 2;
          const float2 w = slot_split_twiddle<EX, e>(wt);
          v[e] = c_mul(v[e], low ? c_neg(w) : w);
        },
        std::make_integer_sequence<int, EX::E>{});
  }
  pair_sync(row);
}

// Inverse transform of the bins in v, then the odd half's unfold twiddle (v = E or O').
template <class EX, bool COMPACT = false>
__device__ __forceinline__ void pair_inverse(const PassParams& p, float2 (&v)[EX::E], float2* mine, int r, int t) {
  if constexpr (COMPACT) {
    EX::inv_compact(v, mine, t, p.twx);
  } else {
    EX::inv(v, mine, t, p.twx);
  }
  if (r) {
    const float2 wt = ldg2(p.wpx + t);
    for_slots(
        [&](auto ec) {
          constexpr int e = decltype(ec)::value;
          v[e] = c_mulc(v[e], slot_split_twiddle<EX, e>(wt));
        },
        std::make_integer_sequence<int, EX::E>{});
  }
}

// ----------------------------------------------------------------------------- staged operands

// The per-sample operands of a modulation (Eq. 1) for one row, staged in shared memory by the
// pair with 16-byte asynchronous copies (complex mask first, then phase and amplitude; every part
// a whole number of 16-byte units when nx is a multiple of 4). Lens factors are read from their
// table in global memory (the same few KB for every row of a field, so they stay in L1).
struct PairPlanes {
  const float2* cm;
  const float* ph;
  const float* am;
};

// Floats per row that the staged operands of modulation flags take.
__host__ __device__ inline int pair_mod_floats(uint32_t flags, int nx) {
  int n = 0;
  if (flags & TOP_MOD_COMPLEX) n += 2 * nx;
  if (flags & TOP_MOD_PHASE) n += nx;
  if (flags & TOP_MOD_AMPLITUDE) n += nx;
  return n;
}

// Copy `floats` floats (a multiple of 4, both ends 16-byte aligned) with the pair's 64 threads.
__device__ __forceinline__ void pair_copy(float* dst, const float* src, int floats, int lane64) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
  float4* d4 = reinterpret_cast<float4*>(dst);
  for (int i = lane64; i < floats / 4; i += 64) top_cp_async16(d4 + i, s4 + i);
}

// Issue the copies of row y's modulation operands (field f) into `dst`; returns the views.
__device__ __forceinline__ PairPlanes pair_stage_mod(const ModDev& m, uint32_t flags, int f, int y, int nx,
                                                     float* dst, int lane64) {
  PairPlanes pp{};
  const long long row0 = (long long)f * m.stride + (long long)y * nx;
  if (flags & TOP_MOD_COMPLEX) {
    pair_copy(dst, reinterpret_cast<const float*>(m.cmask + row0), 2 * nx, lane64);
    pp.cm = reinterpret_cast<const float2*>(dst);
    dst += 2 * nx;
  }
  if (flags & TOP_MOD_PHASE) {
    pair_copy(dst, m.phase + row0, nx, lane64);
    pp.ph = dst;
    dst += nx;
  }
  if (flags & TOP_MOD_AMPLITUDE) {
    pair_copy(dst, m.amp + row0, nx, lane64);
    pp.am = dst;
  }
  return pp;
}

// Per-row constants of a modulation: aperture range and the lens factor of the row.
struct ModRow {
  int2 rg;
  float2 ly;
  const float2* lx;
};
__device__ __forceinline__ ModRow mod_row(const ModDev& m, uint32_t flags, const float2* lx, const float2* ly_tab,
                                          int y, int nx) {
  ModRow mr;
  mr.rg = (flags & TOP_MOD_CIRC) ? __ldg(m.circ + y) : make_int2(0, nx - 1);
  mr.ly = (flags & TOP_MOD_LENS) ? ldg2(ly_tab + y) : make_float2(1.f, 0.f);
  mr.lx = lx;
  return mr;
}

// M(x, y) of Eq. 1 from staged operands, in the order of mod_value.
__device__ __forceinline__ float2 mod_staged(uint32_t flags, int conj, const PairPlanes& pp, const ModRow& mr, int x) {
  float2 r = make_float2(1.f, 0.f);
  if (flags & TOP_MOD_COMPLEX) r = pp.cm[x];
  if (flags & TOP_MOD_AMPLITUDE) r = c_scale(r, pp.am[x]);
  if (flags & TOP_MOD_PHASE) r = c_mul(r, cis(pp.ph[x]));
  if (flags & TOP_MOD_LENS) r = c_mul(r, c_mul(ldg2(mr.lx + x), mr.ly));
  if ((flags & TOP_MOD_CIRC) && (x < mr.rg.x || x > mr.rg.y)) r = make_float2(0.f, 0.f);
  return conj ? c_conj(r) : r;
}

// Floats per row the pair-local forward pass stages: the source row (the field, or the saved field
// and the intensity gradient) and the source modulation's operands.
__host__ __device__ inline int pair_src_floats(const PassParams& p) {
  return (p.src_kind == SRC_INTENSITY ? 3 : 2) * p.nx + pair_mod_floats(p.msrc.flags, p.nx);
}

// ----------------------------------------------------------------------------- R1

// The source row and its operands are staged in the pair's two exchange buffers (they are read
// before the first exchange), so the pass needs no shared memory beyond the transforms'.
template <class EX, uint32_t MF>
__global__ void __launch_bounds__(PairRows<EX>::THREADS, 4) k_rows_fwd_pair(const __grid_constant__ PassParams p) {
  using PR = PairRows<EX>;
  TOP_DYN_SMEM(float2, smem);
  const int grp = threadIdx.x >> 5, t = threadIdx.x & 31;
  const int row = grp >> 1, r = grp & 1;
  const int lane64 = threadIdx.x & 63;
  const int y = blockIdx.x * PR::ROWS + row;
  const int f = blockIdx.y;
  const int nx = p.nx;
  const bool live = y < p.ny;
  const FieldSet& fs = p.sets[p.set_of[f]];
  float2* mine = smem + grp * EX::BUF;
  const float2* theirs = smem + (grp ^ 1) * EX::BUF;
  float* stage = reinterpret_cast<float*>(smem + 2 * row * EX::BUF);
  const bool inten = p.src_kind == SRC_INTENSITY;
  const ModDev& m = p.msrc;
  const uint32_t flags = mod_flags<MF>(m);
  if (threadIdx.x == 0) {
    int fa, tile;
    if (ahead_block(p, fa, tile)) {
      const int ya = tile * PR::ROWS, na = min(PR::ROWS, p.ny - ya);
      const long long rowa = (long long)ya * nx;
      const float2* src = inten ? p.psi + (long long)fa * p.psi_stride + rowa : field_in(p, fa) + rowa;
      top_prefetch_l2(src, unsigned(na) * nx * 8u);
      if (inten) top_prefetch_l2(p.gI + (long long)(fa / p.src_group) * p.gI_stride + rowa, unsigned(na) * nx * 4u);
    }
  }
  PairPlanes pp{};
  if (live) {
    const long long row0 = (long long)y * nx;
    const float2* src = inten ? p.psi + (long long)f * p.psi_stride + row0 : field_in(p, f) + row0;
    pair_copy(stage, reinterpret_cast<const float*>(src), 2 * nx, lane64);
    if (inten) pair_copy(stage + 2 * nx, p.gI + (long long)(f / p.src_group) * p.gI_stride + row0, nx, lane64);
    pp = pair_stage_mod(m, flags, f, y, nx, stage + (inten ? 3 : 2) * nx, lane64);
  }
  top_cp_async_wait_all();
  pair_sync(row);
  const float2* srow = reinterpret_cast<const float2*>(stage);
  const float* gi = stage + 2 * nx;
  const float w2 = inten ? 2.f * (p.weights ? __ldg(p.weights + f) : 1.f) : 1.f;
  const ModRow mr = mod_row(m, flags, fs.src_lx, fs.src_ly, live ? y : 0, nx);
  const int x0 = t + (r ? 0 : EX::M / 2);
  float2 o[PR::H];
#pragma unroll
  for (int k = 0; k < PR::H; ++k) {
    const int x = x0 + (lo_pos<EX>(t, k) - t);
    float2 s = make_float2(0.f, 0.f);
    if (live) {
      s = srow[x];
      if (inten) s = c_scale(s, w2 * gi[x]);
      if (flags) s = c_mul(s, mod_staged(flags, m.conj, pp, mr, x));
    }
    o[k] = s;
  }
  pair_sync(row);  // both warps are done with the staged row before the exchanges overwrite it
  float2 v[EX::E];
  pair_spread<EX>(v, o, mine, theirs, r, t, row, p.wpx);
  EX::fwd(v, mine, t, p.twx);
  if (live) pair_store_bins<EX>(p, f, y, r, t, v);
}

// ----------------------------------------------------------------------------- R2

// Floats per row the pair-local inverse pass stages after the exchange buffers: the epilogue
// modulation's operands and, for the phase gradient, the saved modulation input.
template <int KIND>
__host__ __device__ inline int pair_epi_floats(const PassParams& p) {
  return pair_mod_floats(p.mepi.flags, p.nx) + (KIND == EPI_MODGRAD && p.part_phase ? 2 * p.nx : 0);
}

// Epilogues of the pair-local inverse pass: EPI_FIELD, EPI_INTENSITY (summed over the group in
// registers, field order), EPI_MODGRAD with at most the phase partials (summed the same way).
// A block runs its rows of p.group consecutive fields (with TOP_PAIR_PREFETCH, loading the next
// field's bins while the current one's epilogue runs); the operands of field f are copied while
// its rows are transformed.
template <class EX, int KIND, uint32_t MF>
__global__ void __launch_bounds__(PairRows<EX>::THREADS, TOP_PAIR_INV_MINB) k_rows_inv_pair(const __grid_constant__ PassParams p) {
  using PR = PairRows<EX>;
  constexpr int E = EX::E, H = PR::H;
  TOP_DYN_SMEM(float2, smem);
  const int grp = threadIdx.x >> 5, t = threadIdx.x & 31;
  const int row = grp >> 1, r = grp & 1;
  const int lane64 = threadIdx.x & 63;
  const int y = blockIdx.x * PR::ROWS + row;
  const int g = blockIdx.y;
  const int f0 = g * p.group;
  const int f1 = min(f0 + p.group, p.nfields);
  const bool live = y < p.ny;
  const int nx = p.nx;
  float2* mine = smem + grp * EX::BUF;
  const float2* theirs = smem + (grp ^ 1) * EX::BUF;
  const int sf = (pair_epi_floats<KIND>(p) + 3) & ~3;
  float* stage = reinterpret_cast<float*>(smem + 2 * PR::ROWS * EX::BUF) + row * sf;
  const ModDev& m = p.mepi;
  const uint32_t flags = mod_flags<MF>(m);
  const bool partial = KIND == EPI_MODGRAD && p.part_phase != nullptr;
  constexpr bool ACC = KIND == EPI_INTENSITY || KIND == EPI_MODGRAD;
  const int x0 = t + (r ? 0 : EX::M / 2);
  // sums over the group, one per own slot
  float acc[H];
  if constexpr (ACC) {
#pragma unroll
    for (int k = 0; k < H; ++k) acc[k] = 0.f;
    if (partial && p.part_accumulate && live) {
      const float* src = p.part_phase + (long long)g * p.part_stride + (long long)y * nx;
#pragma unroll
      for (int k = 0; k < H; ++k) acc[k] = src[x0 + (lo_pos<EX>(t, k) - t)];
    }
  }
  float2 v[E];
  if (live) {
    pair_load_bins<EX>(p, f0, y, r, t, v);
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = make_float2(0.f, 0.f);
  }
#pragma unroll 1
  for (int f = f0; f < f1; ++f) {
    const FieldSet& fs = p.sets[p.set_of[f]];
    PairPlanes pp{};
    const float2* xs = nullptr;
    if (live && sf) {
      // this field's operands arrive while its rows are transformed
      pp = pair_stage_mod(m, flags, f, y, nx, stage, lane64);
      if (partial) {
        float* xdst = stage + pair_mod_floats(flags, nx);
        pair_copy(xdst, reinterpret_cast<const float*>(p.xs + (long long)f * p.xs_stride + (long long)y * nx), 2 * nx,
                  lane64);
        xs = reinterpret_cast<const float2*>(xdst);
      }
    }
    pair_inverse<EX, true>(p, v, mine, r, t);
    float2 o[H];
    pair_combine<EX>(v, o, mine, theirs, r, t, row);
#if TOP_PAIR_PREFETCH
    // the next field's bins load while this field's epilogue runs
    if (live && f + 1 < f1) pair_load_bins<EX>(p, f + 1, y, r, t, v);
#endif
    if (sf) {
      top_cp_async_wait_all();
      pair_sync(row);  // the partner's copies of the operands are visible
    }
    if (live) {
      const ModRow mr = mod_row(m, flags, fs.epi_lx, fs.epi_ly, y, nx);
      const float w = KIND == EPI_INTENSITY && p.weights ? __ldg(p.weights + f) : 1.f;
      float2* fout = KIND == EPI_FIELD ? field_out(p, f) + (long long)y * nx
                     : (p.out ? p.out + (long long)f * p.out_stride + (long long)y * nx : nullptr);
#pragma unroll
      for (int k = 0; k < H; ++k) {
        const int x = x0 + (lo_pos<EX>(t, k) - t);
        float2 val = o[k];
        if constexpr (KIND == EPI_FIELD) {
          if (flags) val = c_mul(val, mod_staged(flags, m.conj, pp, mr, x));
          fout[x] = val;
        } else if constexpr (KIND == EPI_INTENSITY) {
          if (flags) val = c_mul(val, mod_staged(flags, m.conj, pp, mr, x));
          if (fout) fout[x] = val;
          acc[k] += w * fmaf(val.x, val.x, val.y * val.y);
        } else {  // EPI_MODGRAD: val = dL/dy with y = M x
          const float2 mv = mod_staged(flags, 0, pp, mr, x);
          if (fout) fout[x] = c_mulc(val, mv);
          if (partial) {
            const float2 ys = c_mul(mv, xs[x]);
            acc[k] += fmaf(val.y, ys.x, -val.x * ys.y);  // Im(val conj(y))
          }
        }
      }
    }
    pair_sync(row);  // the partner is done with this warp's buffers before they are reused
#if !TOP_PAIR_PREFETCH
    if (live && f + 1 < f1) pair_load_bins<EX>(p, f + 1, y, r, t, v);
#endif
  }
  if constexpr (ACC) {
    if (live && (KIND == EPI_INTENSITY || partial)) {
      float* dst = KIND == EPI_INTENSITY ? p.outf + (long long)g * p.outf_stride + (long long)y * nx
                                         : p.part_phase + (long long)g * p.part_stride + (long long)y * nx;
#pragma unroll
      for (int k = 0; k < H; ++k) dst[x0 + (lo_pos<EX>(t, k) - t)] = acc[k];
    }
  }
}

// ----------------------------------------------------------------------------- R2 + R1 fused

// The inverse rows of one propagation (pa), the next propagation's source modulation and its
// forward rows (pb) of a system chain, as k_rows_chain does, pair-local. The next source's
// operands are staged after the exchange buffers while the rows are transformed.
template <class EX, uint32_t MF>
__global__ void __launch_bounds__(PairRows<EX>::THREADS, TOP_PAIR_CHAIN_MINB)
    k_rows_chain_pair(const __grid_constant__ PassParams pa, const __grid_constant__ PassParams pb) {
  using PR = PairRows<EX>;
  TOP_DYN_SMEM(float2, smem);
  const int grp = threadIdx.x >> 5, t = threadIdx.x & 31;
  const int row = grp >> 1, r = grp & 1;
  const int lane64 = threadIdx.x & 63;
  const int y = blockIdx.x * PR::ROWS + row;
  const int f = blockIdx.y;
  const bool live = y < pa.ny;
  const int nx = pa.nx;
  float2* mine = smem + grp * EX::BUF;
  const float2* theirs = smem + (grp ^ 1) * EX::BUF;
  const ModDev& m = pb.msrc;
  const uint32_t flags = mod_flags<MF>(m);
  const FieldSet& fsb = pb.sets[pb.set_of[f]];
  const int sf = (pair_mod_floats(flags, nx) + 3) & ~3;
  float* stage = reinterpret_cast<float*>(smem + 2 * PR::ROWS * EX::BUF) + row * sf;
  PairPlanes pp{};
  if (live && sf) pp = pair_stage_mod(m, flags, f, y, nx, stage, lane64);
  float2 v[EX::E];
  if (live) {
    pair_load_bins<EX>(pa, f, y, r, t, v);
  } else {
#pragma unroll
    for (int e = 0; e < EX::E; ++e) v[e] = make_float2(0.f, 0.f);
  }
  pair_inverse<EX, true>(pa, v, mine, r, t);
  float2 o[PR::H];
  pair_combine<EX>(v, o, mine, theirs, r, t, row);
  if (sf) {
    top_cp_async_wait_all();
    pair_sync(row);  // the partner's copies of the operands are visible
  }
  const ModRow mr = mod_row(m, flags, fsb.src_lx, fsb.src_ly, live ? y : 0, nx);
  float2* kept = pa.out ? pa.out + (long long)f * pa.out_stride + (long long)y * nx : nullptr;
  const int x0 = t + (r ? 0 : EX::M / 2);
#pragma unroll
  for (int k = 0; k < PR::H; ++k) {
    const int x = x0 + (lo_pos<EX>(t, k) - t);
    float2 val = live ? o[k] : make_float2(0.f, 0.f);
    if (live && kept) kept[x] = val;
    if (live && flags) val = c_mul(val, mod_staged(flags, m.conj, pp, mr, x));
    o[k] = val;
  }
  pair_spread<EX>(v, o, mine, theirs, r, t, row, pb.wpx);
#if TOP_CHAIN_FWD_COMPACT
  EX::fwd_compact(v, mine, t, pb.twx);
#else
  EX::fwd(v, mine, t, pb.twx);
#endif
  if (live) pair_store_bins<EX>(pb, f, y, r, t, v);
}

}  // namespace top
