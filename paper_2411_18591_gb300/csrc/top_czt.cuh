// Line transforms of arbitrary length by Bluestein's chirp-z method, on the engines of
// top_engine.cuh.
//
// For the forward DFT X[k] = sum_n x[n] exp(-2 pi i n k / P), n k = (n^2 + k^2 - (k - n)^2) / 2 gives
// X[k] = c[k] sum_n (x[n] c[n]) b[k - n] with c[n] = exp(-i pi n^2 / P) and b[m] = conj(c[m]) = b[-m].
// The sum over n < P is a linear convolution, which a circular one of length L >= 2P - 1 holds
// unaliased at k < P: conv = IFFT_L(FFT_L(a) * FFT_L(b_L)) with b_L the m in (-P, P) of b wrapped
// modulo L. The inverse DFT is the same with c and b conjugated. Between a forward and an inverse
// transform (CZT_FILTER) the chirps cancel: the inverse transform's input is conv[k] H[k] / L.
//
// k_czt runs each L-point transform on an L-point engine (L up to 4096). k_czt_split, for L = 8192,
// runs them as two L/2-point halves on an engine of M = L/2, as the propagation passes do: a (at
// most P <= L/2 samples) gives the even bins as FFT_M(a) and the odd ones as FFT_M(a[n] w^n) with
// w = exp(-2 pi i / L); the product with the chirp transform is taken per half (tables split by
// parity, in the engine's slot order), and the convolution's first L/2 samples are
// IFFT_M(even) + w^-n IFFT_M(odd), combined through shared memory. Group r of a line is half r.
#pragma once

#include "top_engine.cuh"
#include "top_internal.h"
#include "top_launch.h"

namespace top {

// Lines per block: 128 threads (at least one line).
template <class EN>
struct CztShape {
  static constexpr int LINES = EN::G >= 128 ? 1 : 128 / EN::G;
  static constexpr int THREADS = LINES * EN::G;
  static constexpr size_t SMEM = sizeof(float2) * size_t(LINES) * EN::BUF;
  // 128 registers a thread (the three-stage plans spill some, and still run faster than with
  // two blocks per SM and no spills)
  static constexpr int MINB = 4;
};

// conv = IFFT_L(FFT_L(v) * bh) (unnormalised), natural order in and out; bh in the engine's slot
// order (entry e G + t: the bin lane t holds in slot e), so a warp's reads are consecutive
template <class EN>
__device__ __forceinline__ void czt_convolve(float2 (&v)[EN::E], float2* buf, int t, const float2* __restrict__ tw,
                                             const float2* __restrict__ bh) {
  EN::fwd(v, buf, t, tw);
#pragma unroll
  for (int e = 0; e < EN::E; ++e) v[e] = c_mul(v[e], __ldg(bh + e * EN::G + t));
  EN::inv(v, buf, t, tw);
}

template <class EN>
__global__ void __launch_bounds__(CztShape<EN>::THREADS, CztShape<EN>::MINB) k_czt(const __grid_constant__ CztParams p) {
  constexpr int G = EN::G, E = EN::E;
  TOP_DYN_SMEM(float2, smem);
  const int grp = threadIdx.x / G, t = threadIdx.x - grp * G;
  const int line = blockIdx.x * CztShape<EN>::LINES + grp;
  const int f = blockIdx.y;
  const bool live = line < p.nlines;  // the group still runs its transforms (barriers)
  const int li = live ? line : 0;
  float2* buf = smem + grp * EN::BUF;
  const float2* in = p.in + (long long)(f / p.in_repeat) * p.in_fstride + li * p.in_lstride;
  const bool inv = p.mode == CZT_INV;

  // a[n] = x[n - off] c[n] (conj(c[n]) for the inverse) on the line's samples, zero elsewhere
  float2 v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int n = EN::in_pos(t, e);
    const int j = n - p.off_in;
    float2 a = make_float2(0.f, 0.f);
    if (live && j >= 0 && j < p.n_in) {
      const float2 x = in[j];
      const float2 c = __ldg(p.chirp + n);
      a = inv ? c_mulc(x, c) : c_mul(x, c);
    }
    v[e] = a;
  }
  czt_convolve<EN>(v, buf, t, p.tw, inv ? p.bh_inv : p.bh_fwd);

  if (p.mode == CZT_FILTER) {
    // X[k] H[k] conj(c[k]) = conv[k] H[k] / L at k < P (the chirps cancel), zero beyond
    const float2* hrow = p.h[f] + (long long)li * p.P;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k = EN::in_pos(t, e);
      float2 hv = make_float2(0.f, 0.f);
      if (k < p.P) {
        hv = __ldg(hrow + k);
        if (p.adjoint) hv.y = -hv.y;
      }
      v[e] = c_scale(c_mul(v[e], hv), p.inv_l);
    }
    czt_convolve<EN>(v, buf, t, p.tw, p.bh_inv);
  }

  // the window of X[k] = c[k] conv[k] / L (conj(c[k]) after an inverse transform)
  const bool post_conj = p.mode != CZT_FWD;
  float2* out = p.out + (long long)f * p.out_fstride + li * p.out_lstride;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = EN::in_pos(t, e);
    const int j = k - p.k0;
    if (live && j >= 0 && j < p.n_out) {
      const float2 c = __ldg(p.chirp + k);
      out[j] = c_scale(post_conj ? c_mulc(v[e], c) : c_mul(v[e], c), p.inv_l);
    }
  }
}

template <class EN>
cudaError_t launch_czt(const CztParams& p, cudaStream_t s) {
  using SH = CztShape<EN>;
  if (SH::SMEM > 48 * 1024) {
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_czt<EN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SH::SMEM);
    if (attr != cudaSuccess) return attr;
  }
  dim3 grid((p.nlines + SH::LINES - 1) / SH::LINES, p.nfields);
  TOP_LAUNCH(k_czt<EN>, grid, SH::THREADS, SH::SMEM, s, p);
  return cudaGetLastError();
}


// Lines per block: 128 threads where the two halves of a line fit (at least one line).
template <class EN>
struct CztSplitShape {
  static constexpr int LINES = 2 * EN::G >= 128 ? 1 : 128 / (2 * EN::G);
  static constexpr int THREADS = LINES * 2 * EN::G;
  // per line: the combined samples [M] and one exchange buffer per half
  static constexpr size_t SMEM = sizeof(float2) * size_t(LINES) * (EN::M + 2 * EN::BUF);
  static constexpr int MINB = THREADS == 128 ? 4 : 2;  // 128 registers a thread
};

// One half of a circular convolution of length 2M: v holds this half's input slots (natural
// positions in_pos(t, e) < M, zero past the sequence), already times w^pos for the odd half;
// leaves IFFT_M(FFT_M(v) * bh_r) (unnormalised) in natural order.
template <class EN>
__device__ __forceinline__ void czt_half(float2 (&v)[EN::E], float2* buf, int t, const float2* __restrict__ tw,
                                         const float2* __restrict__ bh_r) {
  constexpr int E = EN::E, CH = E % 8 == 0 ? 8 : E;
  EN::fwd(v, buf, t, tw);
  // eight slots at a time: the compiler barrier keeps all the table loads from being hoisted at once
#pragma unroll
  for (int e0 = 0; e0 < E; e0 += CH) {
#pragma unroll
    for (int e = e0; e < e0 + CH; ++e) v[e] = c_mul(v[e], __ldg(bh_r + e * EN::G + t));
    asm volatile("" ::: "memory");
  }
  EN::inv(v, buf, t, tw);
}

// The halves of conv = IFFT_L(FFT_L(a) bh) for the slots in v (half r of a line), combined into
// comb[n] = even[n] + w^-n odd[n] through the odd half's exchange buffer obuf. Ends after the
// barrier that makes comb visible.
template <class EN>
__device__ __forceinline__ void czt_split_convolve(float2 (&v)[EN::E], float2* buf, float2* obuf, float2* comb, int r, int t,
                                             const float2* __restrict__ tw, const float2* __restrict__ bh_r,
                                             const float2* __restrict__ wsplit) {
  constexpr int E = EN::E, CH = E % 8 == 0 ? 8 : E;
  czt_half<EN>(v, buf, t, tw, bh_r);
  EN::sync_group();  // the odd half's exchange buffer becomes its output
  if (r) {
#pragma unroll
    for (int e0 = 0; e0 < E; e0 += CH) {
#pragma unroll
      for (int e = e0; e < e0 + CH; ++e) {
        const int n = EN::in_pos(t, e);
        obuf[n] = c_mulc(v[e], __ldg(wsplit + n));
      }
      asm volatile("" ::: "memory");
    }
  }
  __syncthreads();
  if (!r) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int n = EN::in_pos(t, e);
      comb[n] = c_add(v[e], obuf[n]);
    }
  }
  __syncthreads();
}

template <class EN>
__global__ void __launch_bounds__(CztSplitShape<EN>::THREADS, CztSplitShape<EN>::MINB) k_czt_split(const __grid_constant__ CztParams p) {
  constexpr int G = EN::G, E = EN::E, M = EN::M;
  TOP_DYN_SMEM(float2, smem);
  const int grp = threadIdx.x / G, t = threadIdx.x - grp * G;
  const int ln = grp >> 1, r = grp & 1;
  const int line = blockIdx.x * CztSplitShape<EN>::LINES + ln;
  const int f = blockIdx.y;
  const bool live = line < p.nlines;  // the groups still run their transforms (barriers)
  const int li = live ? line : 0;
  float2* comb = smem + ln * (M + 2 * EN::BUF);  // combined samples [M]
  float2* buf = comb + M + r * EN::BUF;           // this half's exchange buffer
  float2* obuf = comb + M + EN::BUF;              // the odd half's buffer, later its output
  const float2* in = p.in + (long long)(f / p.in_repeat) * p.in_fstride + li * p.in_lstride;
  const bool inv = p.mode == CZT_INV;

  // a[n] = x[n - off] c[n] (conj(c[n]) for the inverse), times w^n in the odd half; eight slots at
  // a time (the compiler barrier keeps all the slots' loads from being hoisted at once)
  constexpr int CH = E % 8 == 0 ? 8 : E;
  float2 v[E];
#pragma unroll
  for (int e0 = 0; e0 < E; e0 += CH) {
#pragma unroll
    for (int e = e0; e < e0 + CH; ++e) {
      const int n = EN::in_pos(t, e);
      const int j = n - p.off_in;
      float2 a = make_float2(0.f, 0.f);
      if (live && j >= 0 && j < p.n_in) {
        const float2 x = in[j];
        const float2 c = __ldg(p.chirp + n);
        a = inv ? c_mulc(x, c) : c_mul(x, c);
        if (r) a = c_mul(a, __ldg(p.wsplit + n));
      }
      v[e] = a;
    }
    asm volatile("" ::: "memory");
  }

  czt_split_convolve<EN>(v, buf, obuf, comb, r, t, p.tw, (inv ? p.bh_inv : p.bh_fwd) + r * M, p.wsplit);

  if (p.mode == CZT_FILTER) {
    // X[k] H[k] conj(c[k]) = conv[k] H[k] / L at k < P (the chirps cancel), zero beyond; times
    // w^k in the odd half
    const float2* hrow = p.h[f] + (long long)li * p.P;
#pragma unroll
    for (int e0 = 0; e0 < E; e0 += CH) {
#pragma unroll
      for (int e = e0; e < e0 + CH; ++e) {
        const int k = EN::in_pos(t, e);
        float2 a = make_float2(0.f, 0.f);
        if (k < p.P) {
          float2 hv = __ldg(hrow + k);
          if (p.adjoint) hv.y = -hv.y;
          a = c_scale(c_mul(comb[k], hv), p.inv_l);
          if (r) a = c_mul(a, __ldg(p.wsplit + k));
        }
        v[e] = a;
      }
      asm volatile("" ::: "memory");
    }
    __syncthreads();  // every lane has read comb before the next combine writes it
    czt_split_convolve<EN>(v, buf, obuf, comb, r, t, p.tw, p.bh_inv + r * M, p.wsplit);
  }

  // the window of X[k] = c[k] conv[k] / L (conj(c[k]) after an inverse transform), stored by both
  // halves from the combined samples
  const bool post_conj = p.mode != CZT_FWD;
  float2* out = p.out + (long long)f * p.out_fstride + li * p.out_lstride;
  if (live) {
    for (int j = r * G + t; j < p.n_out; j += 2 * G) {
      const int k = p.k0 + j;
      const float2 c = __ldg(p.chirp + k);
      const float2 x = comb[k];
      out[j] = c_scale(post_conj ? c_mulc(x, c) : c_mul(x, c), p.inv_l);
    }
  }
}

template <class EN>
cudaError_t launch_czt_split(const CztParams& p, cudaStream_t s) {
  using SH = CztSplitShape<EN>;
  if (SH::SMEM > 48 * 1024) {
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_czt_split<EN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SH::SMEM);
    if (attr != cudaSuccess) return attr;
  }
  dim3 grid((p.nlines + SH::LINES - 1) / SH::LINES, p.nfields);
  TOP_LAUNCH(k_czt_split<EN>, grid, SH::THREADS, SH::SMEM, s, p);
  return cudaGetLastError();
}

}  // namespace top
