// The three passes of one batched propagation, Eq. 4 with H_z of Eq. 5:
//
//   R1  rows:    modulate (Eq. 1), zero-pad along x, forward DFT along x,
//                store transposed:  ws[field][kx][y]
//   C   columns: zero-pad along y, forward DFT along y, multiply by H(kx, ky),
//                inverse DFT along y, crop:  ws[field][kx][y] in place
//   R2  rows:    inverse DFT along x, crop, epilogue (modulation, |psi|^2,
//                incoherent sums of Eq. 14, or modulation gradients)
//
// Each padded line of even length P = 2M is handled as its two interleaved
// halves (even and odd frequencies). With a field of n <= P samples at offset
// o, the even half is the M-point DFT of the folded sequence
// v[q] = sum_{p = q mod M} x[p - o] and the odd half that of
// sum_{p = q mod M} x[p - o] exp(-2 pi i p / P). Zero samples of the padding are
// never loaded or transformed, and the inverse only produces the cropped
// window: x[p] = E[p mod M] + exp(2 pi i p / P) O[p mod M].
//
// Layout of the workspace between passes: for each field, Px lines of ny
// samples, line kpos = r Mx + k holding frequency kx = 2 k + r. The column pass
// therefore reads and writes contiguous lines; R1 and R2 move ROWS-sample chunks.
#pragma once

#include <climits>

#include "top_engine.cuh"
#include "top_internal.h"
#include "top_launch.h"

namespace top {

template <class EN>
struct RowShape {
  static constexpr int ROWS = (256 / EN::G) >= 2 ? (256 / EN::G) : 2;
  static constexpr int THREADS = ROWS * EN::G;
  static constexpr int LD = ROWS + 1;  // odd tile stride: conflict-free column writes
  static constexpr int TILE = EN::M * LD;
  static constexpr int XCH = ROWS * EN::BUF;
  static constexpr size_t SMEM = sizeof(float2) * (TILE > XCH ? TILE : XCH);
};

template <class EN>
struct ColShape {
  static constexpr int COLS = (128 / EN::G) >= 1 ? (128 / EN::G) : 1;
  static constexpr int THREADS = COLS * EN::G;
  static constexpr size_t SMEM = sizeof(float2) * COLS * EN::BUF;
};

__device__ __forceinline__ float2 ldg2(const float2* p) { return __ldg(p); }

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
  if (flags & TOP_MOD_PHASE) {
    float s, c;
    sincosf(__ldg(m.phase + idx), &s, &c);
    r = c_mul(r, make_float2(c, s));
  }
  if (flags & TOP_MOD_LENS) r = c_mul(r, c_mul(ldg2(lx + x), ldg2(ly + y)));
  return conj ? c_conj(r) : r;
}

__device__ __forceinline__ float2 load_src(const PassParams& p, const FieldSet& fs, int f, int y, int x) {
  const long long idx = (long long)y * p.nx + x;
  float2 s;
  if (p.src_kind == SRC_FIELD) {
    s = ldg2(p.in + (long long)(f / p.in_repeat) * p.in_stride + idx);
  } else {
    const float gi = __ldg(p.gI + (long long)(f / p.src_group) * p.gI_stride + idx);
    const float w = p.weights ? __ldg(p.weights + f) : 1.f;
    s = c_scale(ldg2(p.psi + (long long)f * p.psi_stride + idx), 2.f * w * gi);
  }
  if (p.msrc.flags) s = c_mul(s, mod_value(p.msrc, p.msrc.flags, p.msrc.conj, fs.src_lx, fs.src_ly, f, y, x, p.nx));
  return s;
}

// ----------------------------------------------------------------------------- R1

template <class EX>
__global__ void __launch_bounds__(RowShape<EX>::THREADS) k_rows_fwd(const __grid_constant__ PassParams p) {
  constexpr int G = EX::G, E = EX::E, M = EX::M;
  constexpr int ROWS = RowShape<EX>::ROWS, LD = RowShape<EX>::LD;
  TOP_DYN_SMEM(float2, smem);
  const int grp = threadIdx.x / G, t = threadIdx.x - grp * G;
  const int y0 = blockIdx.x * ROWS, y = y0 + grp;
  const int f = blockIdx.y;
  const bool valid = y < p.ny;
  const FieldSet& fs = p.sets[p.set_of[f]];
  float2* buf = smem + grp * EX::BUF;

#pragma unroll 1
  for (int r = 0; r < 2; ++r) {
    float2 v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int pos = EX::in_pos(t, e);
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int x = pos + c * M - p.ox;
        if (valid && x >= 0 && x < p.nx) {
          float2 s = load_src(p, fs, f, y, x);
          if (r) {
            const float2 w = ldg2(p.wpx + pos);
            s = c_mul(s, c ? c_neg(w) : w);
          }
          acc = c_add(acc, s);
        }
      }
      v[e] = acc;
    }
    EX::fwd(v, buf, t, p.twx);
    __syncthreads();  // line buffers alias the tile
#pragma unroll
    for (int e = 0; e < E; ++e) smem[EX::bin(t, e) * LD + grp] = v[e];
    __syncthreads();
    float2* dst = p.ws + (long long)f * p.ws_stride + (long long)(r * M) * p.ny;
    for (int idx = threadIdx.x; idx < M * ROWS; idx += blockDim.x) {
      const int k = idx / ROWS, row = idx - (idx / ROWS) * ROWS;
      if (y0 + row < p.ny) dst[(long long)k * p.ny + y0 + row] = smem[k * LD + row];
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------- C

__device__ __forceinline__ float2 transfer_value(const PassParams& p, const FieldSet& fs, float2 cxh, float ux,
                                                 int kc, int ky) {
  const float4 hy = __ldg(fs.hy + ky);
  float2 h = c_mul(cxh, make_float2(hy.x, hy.y));
  if (p.method == TOP_AS) {
    if (kc != INT_MAX) {
      const int sy = ky < (p.Py + 1) / 2 ? ky : ky - p.Py;
      if (abs(sy) > kc) return make_float2(0.f, 0.f);
    }
    // AS remainder beyond the separable Fresnel phase: cr * g(u), g(u) = -(u^2/4)/(sqrt(1-u) + 1 - u/2)
    const float u = ux + hy.z;
    const float sq = sqrtf(fmaxf(1.f - u, 0.f));
    const float rr = fs.cr * (-0.25f * u * u) / (sq + 1.f - 0.5f * u);
    float s, c;
    sincosf(rr, &s, &c);
    h = c_mul(h, make_float2(c, s));
  }
  return p.adjoint ? c_conj(h) : h;
}

template <class EY>
__global__ void __launch_bounds__(ColShape<EY>::THREADS) k_cols(const __grid_constant__ PassParams p) {
  constexpr int G = EY::G, E = EY::E, M = EY::M, COLS = ColShape<EY>::COLS;
  TOP_DYN_SMEM(float2, smem);
  const int grp = threadIdx.x / G, t = threadIdx.x - grp * G;
  const int col = blockIdx.x * COLS + grp;
  const int f = blockIdx.y;
  const bool valid = col < p.Px;
  const int cc = valid ? col : 0;
  const FieldSet& fs = p.sets[p.set_of[f]];
  float2* buf = smem + grp * EY::BUF;
  float2* line = p.ws + (long long)f * p.ws_stride + (long long)cc * p.ny;

  const int rx = cc >= p.Mx ? 1 : 0;
  const int kx = 2 * (cc - rx * p.Mx) + rx;
  const float4 hx = __ldg(fs.hx + kx);
  const float2 cxh = c_mul(fs.cg, make_float2(hx.x, hx.y));
  const int kc = fs.kcut ? __ldg(fs.kcut + kx) : INT_MAX;

  float2 acc[E];
  float2 v[E];
#pragma unroll 1
  for (int r = 0; r < 2; ++r) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int pos = EY::in_pos(t, e);
      float2 a = make_float2(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int yy = pos + c * M - p.oy;
        if (valid && yy >= 0 && yy < p.ny) {
          float2 s = line[yy];
          if (r) {
            const float2 w = ldg2(p.wpy + pos);
            s = c_mul(s, c ? c_neg(w) : w);
          }
          a = c_add(a, s);
        }
      }
      v[e] = a;
    }
    EY::fwd(v, buf, t, p.twy);
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = c_mul(v[e], transfer_value(p, fs, cxh, hx.z, kc, 2 * EY::bin(t, e) + r));
    EY::inv(v, buf, t, p.twy);
    if (r == 0) {
#pragma unroll
      for (int e = 0; e < E; ++e) acc[e] = v[e];
    }
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int pos = EY::in_pos(t, e);
    const float2 o = c_mulc(v[e], ldg2(p.wpy + pos));
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int yy = pos + c * M - p.oy;
      if (valid && yy >= 0 && yy < p.ny) line[yy] = c ? c_sub(acc[e], o) : c_add(acc[e], o);
    }
  }
}

// ----------------------------------------------------------------------------- R2

// Epilogue of one output sample val = psi(y, x) of field f in group g.
__device__ __forceinline__ void epilogue(const PassParams& p, const FieldSet& fs, int f, int g, bool first, int y,
                                         int x, float2 val) {
  const long long idx = (long long)y * p.nx + x;
  if (p.epi_kind == EPI_FIELD) {
    if (p.mepi.flags) val = c_mul(val, mod_value(p.mepi, p.mepi.flags, p.mepi.conj, fs.epi_lx, fs.epi_ly, f, y, x, p.nx));
    p.out[(long long)f * p.out_stride + idx] = val;
  } else if (p.epi_kind == EPI_INTENSITY) {
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

template <class EX>
__global__ void __launch_bounds__(RowShape<EX>::THREADS) k_rows_inv(const __grid_constant__ PassParams p) {
  constexpr int G = EX::G, E = EX::E, M = EX::M;
  constexpr int ROWS = RowShape<EX>::ROWS, LD = RowShape<EX>::LD;
  TOP_DYN_SMEM(float2, smem);
  const int grp = threadIdx.x / G, t = threadIdx.x - grp * G;
  const int y0 = blockIdx.x * ROWS, y = y0 + grp;
  const bool valid = y < p.ny;
  const int g = blockIdx.y;
  const int f0 = g * p.group;
  const int f1 = min(f0 + p.group, p.nfields);
  float2* buf = smem + grp * EX::BUF;

#pragma unroll 1
  for (int f = f0; f < f1; ++f) {
    const FieldSet& fs = p.sets[p.set_of[f]];
    float2 acc[E];
    float2 v[E];
#pragma unroll 1
    for (int r = 0; r < 2; ++r) {
      __syncthreads();
      const float2* src = p.ws + (long long)f * p.ws_stride + (long long)(r * M) * p.ny;
      for (int idx = threadIdx.x; idx < M * ROWS; idx += blockDim.x) {
        const int k = idx / ROWS, row = idx - (idx / ROWS) * ROWS;
        smem[k * LD + row] = (y0 + row < p.ny) ? src[(long long)k * p.ny + y0 + row] : make_float2(0.f, 0.f);
      }
      __syncthreads();
#pragma unroll
      for (int e = 0; e < E; ++e) v[e] = smem[EX::bin(t, e) * LD + grp];
      __syncthreads();  // tile reads done before the aliased line buffers are written
      EX::inv(v, buf, t, p.twx);
      if (r == 0) {
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] = v[e];
      }
    }
    if (valid) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int pos = EX::in_pos(t, e);
        const float2 o = c_mulc(v[e], ldg2(p.wpx + pos));
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int x = pos + c * M - p.ox;
          if (x >= 0 && x < p.nx) epilogue(p, fs, f, g, f == f0, y, x, c ? c_sub(acc[e], o) : c_add(acc[e], o));
        }
      }
    }
  }
}

// ----------------------------------------------------------------------------- launchers

template <class K>
inline cudaError_t set_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <class EX>
cudaError_t launch_rows_fwd(const PassParams& p, cudaStream_t s) {
  using SH = RowShape<EX>;
  static const cudaError_t attr = set_smem(k_rows_fwd<EX>, SH::SMEM);
  if (attr != cudaSuccess) return attr;
  dim3 grid((p.ny + SH::ROWS - 1) / SH::ROWS, p.nfields);
  TOP_LAUNCH(k_rows_fwd<EX>, grid, SH::THREADS, SH::SMEM, s, p);
  return cudaGetLastError();
}

template <class EY>
cudaError_t launch_cols(const PassParams& p, cudaStream_t s) {
  using SH = ColShape<EY>;
  static const cudaError_t attr = set_smem(k_cols<EY>, SH::SMEM);
  if (attr != cudaSuccess) return attr;
  dim3 grid((p.Px + SH::COLS - 1) / SH::COLS, p.nfields);
  TOP_LAUNCH(k_cols<EY>, grid, SH::THREADS, SH::SMEM, s, p);
  return cudaGetLastError();
}

template <class EX>
cudaError_t launch_rows_inv(const PassParams& p, cudaStream_t s) {
  using SH = RowShape<EX>;
  static const cudaError_t attr = set_smem(k_rows_inv<EX>, SH::SMEM);
  if (attr != cudaSuccess) return attr;
  dim3 grid((p.ny + SH::ROWS - 1) / SH::ROWS, (p.nfields + p.group - 1) / p.group);
  TOP_LAUNCH(k_rows_inv<EX>, grid, SH::THREADS, SH::SMEM, s, p);
  return cudaGetLastError();
}

}  // namespace top
