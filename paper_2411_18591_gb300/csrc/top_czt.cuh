// Line transforms of arbitrary length by Bluestein's chirp-z method, on the engines of
// top_engine.cuh (a power-of-two L-point transform per line, L >= 2P - 1).
//
// For the forward DFT X[k] = sum_n x[n] exp(-2 pi i n k / P), n k = (n^2 + k^2 - (k - n)^2) / 2 gives
// X[k] = c[k] sum_n (x[n] c[n]) b[k - n] with c[n] = exp(-i pi n^2 / P) and b[m] = conj(c[m]) = b[-m].
// The sum over n < P is a linear convolution, which a circular one of length L >= 2P - 1 holds
// unaliased at k < P: conv = IFFT_L(FFT_L(a) * FFT_L(b_L)) with b_L the m in (-P, P) of b wrapped
// modulo L. The inverse DFT is the same with c and b conjugated. Between a forward and an inverse
// transform (CZT_FILTER) the chirps cancel: the inverse transform's input is conv[k] H[k] / L.
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
  static constexpr int MINB = 4;  // 128 registers a thread
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

}  // namespace top
