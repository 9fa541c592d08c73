// Register-resident mixed-radix FFT engine for sm_103a.
//
// One line of length M (a row or a column of the zero-padded field, or one half
// of it, see top_passes.cuh) is owned by G consecutive threads; each thread holds
// E = M / G complex samples in registers. The transform is a sequence of radix-R
// stages (R in {2, 3, 4, 5} and their products, each done in registers with
// compile-time twiddles); between stages the samples are exchanged through a
// padded shared-memory line buffer.
//
// Forward: decimation in frequency, natural-order input, digit-reversed output.
// Inverse: the mirror-image decimation in time, digit-reversed input, natural
// output, unnormalised. A forward transform followed by a point-wise product
// and the inverse therefore needs no reordering pass at all: the frequency-
// domain product (the transfer function H_z of Eq. 5) is applied to the
// samples where the forward transform leaves them.
//
// Stage s has radix R_s and span SP_s = R_{s+1} ... R_{NS-1}. Its butterfly b
// (0 <= b < M / R_s) reads positions blk * R_s * SP_s + i + j * SP_s with
// blk = b / SP_s, i = b % SP_s, j = 0 .. R_s - 1. The forward butterfly is an
// R_s-point DFT followed by the twiddles w_{R_s SP_s}^{i j}; the inverse applies
// the conjugate twiddles first and then the inverse DFT.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "top_launch.h"

#include <utility>

namespace top {

// ----------------------------------------------------------------------------- complex helpers

// Sums and differences of complex samples are single packed-pair instructions (two FP32 lanes
// in one 64-bit register pair, round to nearest like the scalar forms).
__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) {
  float2 r;
  asm("{.reg .b64 pa, pb, pr;\n\t"
      "mov.b64 pa, {%2, %3};\n\t"
      "mov.b64 pb, {%4, %5};\n\t"
      "sub.rn.f32x2 pr, pa, pb;\n\t"
      "mov.b64 {%0, %1}, pr;}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
// Scalar forms, where an operand is a quarter-turn rotation that the scalar instructions absorb
// (a packed pair would need the swapped components moved into a register pair first).
__device__ __forceinline__ float2 s_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 s_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 c_mulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 c_conj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 c_scale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 c_neg(float2 a) { return make_float2(-a.x, -a.y); }
// multiply by +i or -i
__device__ __forceinline__ float2 c_mul_i(float2 a) { return make_float2(-a.y, a.x); }
__device__ __forceinline__ float2 c_mul_mi(float2 a) { return make_float2(a.y, -a.x); }

// ----------------------------------------------------------------------------- compile-time trig

constexpr double kCxPi = 3.14159265358979323846264338327950288;

// Taylor series on [-pi/4, pi/4]; used only to fold constants at compile time.
__host__ __device__ constexpr double cx_sin_poly(double x) {
  double x2 = x * x, term = x, sum = x;
  for (int n = 1; n <= 12; ++n) {
    term = -term * x2 / double((2 * n) * (2 * n + 1));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double cx_cos_poly(double x) {
  double x2 = x * x, term = 1.0, sum = 1.0;
  for (int n = 1; n <= 12; ++n) {
    term = -term * x2 / double((2 * n - 1) * (2 * n));
    sum += term;
  }
  return sum;
}
// cos / sin of 2 pi m / n, reduced to the nearest quarter turn with integer arithmetic.
__host__ __device__ constexpr double cx_cos2pi(long m, long n) {
  m %= n;
  if (m < 0) m += n;
  const long q = (8 * m + n) / (2 * n);  // nearest quarter turn
  const double r = 2.0 * kCxPi * double(4 * m - q * n) / double(4 * n);
  switch (q & 3) {
    case 0: return cx_cos_poly(r);
    case 1: return -cx_sin_poly(r);
    case 2: return -cx_cos_poly(r);
    default: return cx_sin_poly(r);
  }
}
__host__ __device__ constexpr double cx_sin2pi(long m, long n) {
  m %= n;
  if (m < 0) m += n;
  const long q = (8 * m + n) / (2 * n);
  const double r = 2.0 * kCxPi * double(4 * m - q * n) / double(4 * n);
  switch (q & 3) {
    case 0: return cx_sin_poly(r);
    case 1: return cx_cos_poly(r);
    case 2: return -cx_sin_poly(r);
    default: return -cx_cos_poly(r);
  }
}

// a * exp(DIR * 2 pi i MM / NN) with the constant folded; quarter and eighth turns are exact.
template <int DIR, long MM, long NN>
__device__ __forceinline__ float2 tw_const(float2 a) {
  constexpr long m = ((MM % NN) + NN) % NN;
  if constexpr (m == 0) {
    return a;
  } else if constexpr ((4 * m) % NN == 0) {
    constexpr int q = int((4 * m) / NN);
    if constexpr (q == 2) {
      return c_neg(a);
    } else if constexpr ((q == 1) == (DIR > 0)) {
      return c_mul_i(a);
    } else {
      return c_mul_mi(a);
    }
  } else if constexpr ((8 * m) % NN == 0) {
    constexpr float h = 0.70710678118654752440f;
    constexpr float sc = cx_cos2pi(m, NN) > 0 ? 1.f : -1.f;
    constexpr float ss = (DIR * cx_sin2pi(m, NN)) > 0 ? 1.f : -1.f;
    return make_float2(h * (sc * a.x - ss * a.y), h * (ss * a.x + sc * a.y));
  } else {
    constexpr float c = float(cx_cos2pi(m, NN));
    constexpr float s = float(DIR * cx_sin2pi(m, NN));
    return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
  }
}

// ----------------------------------------------------------------------------- in-register DFTs
// dft<N, S, DIR>(v): in-place N-point DFT of v[0], v[S], ..., v[(N-1) S], natural order
// in and out, X[k] = sum_n x[n] exp(DIR 2 pi i n k / N) (DIR = -1 forward, +1 inverse).

template <int N>
struct FirstFactor {
  static constexpr int value = (N % 4 == 0 && N != 4)   ? 4
                               : (N % 2 == 0 && N != 2) ? 2
                               : (N % 3 == 0 && N != 3) ? 3
                               : (N % 5 == 0 && N != 5) ? 5
                                                        : N;
};

template <int N, int S, int DIR>
__device__ __forceinline__ void dft(float2* v);

template <int S, int DIR>
__device__ __forceinline__ void dft2(float2* v) {
  const float2 a = v[0], b = v[S];
  v[0] = c_add(a, b);
  v[S] = c_sub(a, b);
}

template <int S, int DIR>
__device__ __forceinline__ void dft3(float2* v) {
  constexpr float c = -0.5f;
  constexpr float s = DIR * 0.86602540378443864676f;  // DIR sin(2 pi / 3)
  const float2 x0 = v[0], x1 = v[S], x2 = v[2 * S];
  const float2 t = c_add(x1, x2), d = c_sub(x1, x2);
  const float2 m = make_float2(fmaf(c, t.x, x0.x), fmaf(c, t.y, x0.y));
  const float2 id = make_float2(-s * d.y, s * d.x);  // i s d
  v[0] = c_add(x0, t);
  v[S] = s_add(m, id);
  v[2 * S] = s_sub(m, id);
}

template <int S, int DIR>
__device__ __forceinline__ void dft4(float2* v) {
  const float2 x0 = v[0], x1 = v[S], x2 = v[2 * S], x3 = v[3 * S];
  const float2 a = c_add(x0, x2), b = c_sub(x0, x2);
  const float2 c = c_add(x1, x3), d = c_sub(x1, x3);
  const float2 wd = DIR > 0 ? c_mul_i(d) : c_mul_mi(d);  // exp(DIR i pi/2) d
  v[0] = c_add(a, c);
  v[2 * S] = c_sub(a, c);
  v[S] = s_add(b, wd);
  v[3 * S] = s_sub(b, wd);
}

template <int S, int DIR>
__device__ __forceinline__ void dft5(float2* v) {
  constexpr float c1 = 0.30901699437494742410f;   // cos(2 pi / 5)
  constexpr float c2 = -0.80901699437494742410f;  // cos(4 pi / 5)
  constexpr float s1 = DIR * 0.95105651629515357212f;
  constexpr float s2 = DIR * 0.58778525229247312917f;
  const float2 x0 = v[0];
  const float2 a1 = c_add(v[S], v[4 * S]), b1 = c_sub(v[S], v[4 * S]);
  const float2 a2 = c_add(v[2 * S], v[3 * S]), b2 = c_sub(v[2 * S], v[3 * S]);
  const float2 m1 = make_float2(fmaf(c1, a1.x, fmaf(c2, a2.x, x0.x)), fmaf(c1, a1.y, fmaf(c2, a2.y, x0.y)));
  const float2 m2 = make_float2(fmaf(c2, a1.x, fmaf(c1, a2.x, x0.x)), fmaf(c2, a1.y, fmaf(c1, a2.y, x0.y)));
  // n1 = s1 b1 + s2 b2, n2 = s2 b1 - s1 b2; terms are i * n
  const float2 n1 = make_float2(fmaf(s1, b1.x, s2 * b2.x), fmaf(s1, b1.y, s2 * b2.y));
  const float2 n2 = make_float2(fmaf(s2, b1.x, -s1 * b2.x), fmaf(s2, b1.y, -s1 * b2.y));
  v[0] = c_add(x0, c_add(a1, a2));
  v[S] = s_add(m1, c_mul_i(n1));
  v[4 * S] = s_sub(m1, c_mul_i(n1));
  v[2 * S] = s_add(m2, c_mul_i(n2));
  v[3 * S] = s_sub(m2, c_mul_i(n2));
}

// element I of an A x B block (index I = B k1 + n2) gets w_N^{n2 k1}
template <int A, int B, int S, int DIR, int... I>
__device__ __forceinline__ void apply_inner_twiddles(float2* v, std::integer_sequence<int, I...>) {
  ((v[I * S] = tw_const<DIR, long(I % B) * long(I / B), long(A * B)>(v[I * S])), ...);
}

template <int A, int B, int S, int... I>
__device__ __forceinline__ void digit_permute(float2* v, std::integer_sequence<int, I...>) {
  // out[k1 + A k2] = in[B k1 + k2]; I enumerates the output index k = k1 + A k2
  float2 t[A * B] = {v[(B * (I % A) + I / A) * S]...};
  ((v[I * S] = t[I]), ...);
}

template <int N, int S, int DIR>
__device__ __forceinline__ void dft_composite(float2* v) {
  constexpr int A = FirstFactor<N>::value;
  constexpr int B = N / A;
  // A-point DFTs over n1 for each n2 (elements B n1 + n2)
#pragma unroll
  for (int n2 = 0; n2 < B; ++n2) dft<A, B * S, DIR>(v + n2 * S);
  apply_inner_twiddles<A, B, S, DIR>(v, std::make_integer_sequence<int, N>{});
  // B-point DFTs over n2 for each k1 (elements B k1 + n2)
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1) dft<B, S, DIR>(v + B * k1 * S);
  digit_permute<A, B, S>(v, std::make_integer_sequence<int, N>{});
}

template <int N, int S, int DIR>
__device__ __forceinline__ void dft(float2* v) {
  static_assert(N >= 1, "radix");
  if constexpr (N == 1) {
  } else if constexpr (N == 2) {
    dft2<S, DIR>(v);
  } else if constexpr (N == 3) {
    dft3<S, DIR>(v);
  } else if constexpr (N == 4) {
    dft4<S, DIR>(v);
  } else if constexpr (N == 5) {
    dft5<S, DIR>(v);
  } else {
    static_assert(FirstFactor<N>::value != N, "only radices with factors 2, 3, 5 are supported");
    dft_composite<N, S, DIR>(v);
  }
}

// ----------------------------------------------------------------------------- engine

// Stage arithmetic of a radix plan R0 x R1 x R2 x R3 (unused trailing radices are 1).
template <int R0, int R1, int R2, int R3>
struct Radices {
  static constexpr int NS = R3 > 1 ? 4 : R2 > 1 ? 3 : R1 > 1 ? 2 : 1;
  __host__ __device__ static constexpr int radix(int s) {
    return s == 0 ? R0 : s == 1 ? R1 : s == 2 ? R2 : R3;
  }
  __host__ __device__ static constexpr int span(int s) {
    int p = 1;
    for (int i = s + 1; i < NS; ++i) p *= radix(i);
    return p;
  }
  // product R_0 ... R_{s-1}: weight of stage s's digit in the frequency index
  __host__ __device__ static constexpr int weight(int s) {
    int p = 1;
    for (int i = 0; i < s; ++i) p *= radix(i);
    return p;
  }
  __host__ __device__ static constexpr int tw_off(int s) {
    int o = 0;
    for (int i = 0; i < s; ++i)
      if (span(i) > 1) o += (radix(i) - 1) * span(i);
    return o;
  }
  __host__ __device__ static constexpr bool divides(int m, int g) {
    for (int s = 0; s < NS; ++s)
      if ((m / radix(s)) % g != 0) return false;
    return true;
  }
};

template <int M_, int G_, int R0, int R1 = 1, int R2 = 1, int R3 = 1>
struct Engine : Radices<R0, R1, R2, R3> {
  using Rd = Radices<R0, R1, R2, R3>;
  using Rd::NS;
  using Rd::radix;
  using Rd::span;
  using Rd::weight;
  using Rd::tw_off;
  static constexpr int M = M_;
  static constexpr int G = G_;
  static constexpr int E = M / G;
  static_assert(R0 * R1 * R2 * R3 == M, "radices must multiply to M");
  static_assert(M % G == 0, "G must divide M");
  static_assert(Rd::divides(M_, G_), "G must divide M / R_s for every stage");
  static constexpr int TW_SIZE = Rd::tw_off(Rd::NS) > 0 ? Rd::tw_off(Rd::NS) : 1;
  static constexpr int PADW = M / 4 >= 32 ? 32 : (M / 4 >= 1 ? M / 4 : 1);
  // padded line buffer (float2 elements) with one spare slot between lines
  static constexpr int BUF = (M - 1) + (M - 1) / PADW + 2;
  static constexpr int RL = Rd::radix(Rd::NS - 1);

  __device__ __forceinline__ static int padi(int p) { return p + p / PADW; }

  // a group that tiles a warp synchronises with __syncwarp, a group of whole warps with its own
  // named barrier (ids from 15 down, one per group of the block; the pass shapes assert that they
  // stay clear of the column barriers' ids from 1 up), anything else with the whole block
  __device__ __forceinline__ static void sync_group() {
    if constexpr (G <= 32 && 32 % G == 0) {
      __syncwarp();
    } else if constexpr (G % 32 == 0) {
      top_named_barrier(15 - int(threadIdx.x) / G, G);
    } else {
      __syncthreads();
    }
  }

  // position held by slot (q, j) of thread t in the layout of stage S
  template <int S>
  __device__ __forceinline__ static int pos(int t, int q, int j) {
    constexpr int R = radix(S), SP = span(S);
    const int b = t + G * q;
    const int blk = b / SP, i = b - blk * SP;
    return blk * (R * SP) + i + j * SP;
  }

  // Input/output layout (stage 0): slot e = q R0 + j holds position (t + G q) + j SP0.
  __device__ __forceinline__ static int in_pos(int t, int e) {
    const int q = e / R0, j = e - (e / R0) * R0;
    return t + G * q + j * span(0);
  }

  // Frequency layout (last stage): slot e = q RL + j holds the bin kbase(t + G q) + j M / RL.
  __host__ __device__ __forceinline__ static constexpr int kbase(int b) {
    // b = position / RL; digits of stages 0 .. NS-2 of the position b * RL
    int k = 0;
#pragma unroll
    for (int s = 0; s < NS - 1; ++s) {
      const int sp = span(s) / RL;
      k += ((b / sp) % radix(s)) * weight(s);
    }
    return k;
  }
  __device__ __forceinline__ static int bin(int t, int e) {
    const int q = e / RL, j = e - (e / RL) * RL;
    return kbase(t + G * q) + j * (M / RL);
  }
  // Arrays indexed by bin that lanes read or write in the frequency layout: where consecutive
  // lanes hold bins a multiple of 16 apart (sixteen 8-byte entries span the banks once), one
  // spare entry after every 16 spreads a warp's accesses over all banks.
  static constexpr bool BIN_PAD = (kbase(1) - kbase(0)) % 16 == 0;
  __host__ __device__ __forceinline__ static constexpr int bin_slot(int k) { return BIN_PAD ? k + k / 16 : k; }

  template <int S, int DIR>
  __device__ __forceinline__ static void stage(float2 (&v)[E], int t, const float2* __restrict__ tw) {
    constexpr int R = radix(S), SP = span(S), Q = M / (R * G);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      float2* w = v + q * R;
      if constexpr (DIR < 0) {
        dft<R, 1, -1>(w);
        if constexpr (SP > 1) {
          const int i = (t + G * q) % SP;
          const float2* tp = tw + tw_off(S) + i;
#pragma unroll
          for (int j = 1; j < R; ++j) w[j] = c_mul(w[j], __ldg(tp + (j - 1) * SP));
        }
      } else {
        if constexpr (SP > 1) {
          const int i = (t + G * q) % SP;
          const float2* tp = tw + tw_off(S) + i;
#pragma unroll
          for (int j = 1; j < R; ++j) w[j] = c_mulc(w[j], __ldg(tp + (j - 1) * SP));
        }
        dft<R, 1, +1>(w);
      }
    }
  }

  template <int A, int B>
  __device__ __forceinline__ static void exchange(float2 (&v)[E], float2* __restrict__ buf, int t) {
    constexpr int RA = radix(A), QA = M / (RA * G);
    constexpr int RB = radix(B), QB = M / (RB * G);
    sync_group();
#pragma unroll
    for (int q = 0; q < QA; ++q)
#pragma unroll
      for (int j = 0; j < RA; ++j) buf[padi(pos<A>(t, q, j))] = v[q * RA + j];
    sync_group();
#pragma unroll
    for (int q = 0; q < QB; ++q)
#pragma unroll
      for (int j = 0; j < RB; ++j) v[q * RB + j] = buf[padi(pos<B>(t, q, j))];
  }

  // fwd_compact / inv_compact: two-stage plans with equal radices run their two stages as one loop
  // over a single copy of the in-register DFT (half the code of the unrolled form), for kernels
  // whose code otherwise spills out of the instruction cache (the fused row passes hold a forward
  // and an inverse transform); elsewhere the unrolled form measured faster.
  static constexpr bool LOOP2 = NS == 2 && Rd::radix(0) == Rd::radix(1);

  template <int DIR>
  __device__ __forceinline__ static void dfts(float2 (&v)[E]) {
    constexpr int R = radix(0), Q = M / (R * G);
#pragma unroll
    for (int q = 0; q < Q; ++q) dft<R, 1, DIR>(v + q * R);
  }
  // the twiddles of stage 0 (span span(0)), conjugated for the inverse
  template <int DIR>
  __device__ __forceinline__ static void stage0_twiddles(float2 (&v)[E], int t, const float2* __restrict__ tw) {
    constexpr int R = radix(0), SP = span(0), Q = M / (R * G);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      float2* w = v + q * R;
      const int i = (t + G * q) % SP;
      const float2* tp = tw + tw_off(0) + i;
#pragma unroll
      for (int j = 1; j < R; ++j) w[j] = DIR < 0 ? c_mul(w[j], __ldg(tp + (j - 1) * SP)) : c_mulc(w[j], __ldg(tp + (j - 1) * SP));
    }
  }

  __device__ __forceinline__ static void fwd_compact(float2 (&v)[E], float2* buf, int t, const float2* __restrict__ tw) {
    if constexpr (LOOP2) {
#pragma unroll 1
      for (int s = 0; s < 2; ++s) {
        if (s == 1) exchange<0, 1>(v, buf, t);
        dfts<-1>(v);
        if (s == 0) stage0_twiddles<-1>(v, t, tw);
      }
    } else {
      fwd(v, buf, t, tw);
    }
  }
  __device__ __forceinline__ static void inv_compact(float2 (&v)[E], float2* buf, int t, const float2* __restrict__ tw) {
    if constexpr (LOOP2) {
#pragma unroll 1
      for (int s = 0; s < 2; ++s) {
        if (s == 1) {
          exchange<1, 0>(v, buf, t);
          stage0_twiddles<+1>(v, t, tw);
        }
        dfts<+1>(v);
      }
    } else {
      inv(v, buf, t, tw);
    }
  }

  // forward DFT: natural-order input (in_pos layout) -> digit-reversed bins (bin layout)
  __device__ __forceinline__ static void fwd(float2 (&v)[E], float2* buf, int t, const float2* __restrict__ tw) {
    stage<0, -1>(v, t, tw);
    if constexpr (NS > 1) {
      exchange<0, 1>(v, buf, t);
      stage<1, -1>(v, t, tw);
    }
    if constexpr (NS > 2) {
      exchange<1, 2>(v, buf, t);
      stage<2, -1>(v, t, tw);
    }
    if constexpr (NS > 3) {
      exchange<2, 3>(v, buf, t);
      stage<3, -1>(v, t, tw);
    }
  }

  // unnormalised inverse DFT: bin layout -> natural order (in_pos layout)
  __device__ __forceinline__ static void inv(float2 (&v)[E], float2* buf, int t, const float2* __restrict__ tw) {
    if constexpr (NS > 3) {
      stage<3, +1>(v, t, tw);
      exchange<3, 2>(v, buf, t);
    }
    if constexpr (NS > 2) {
      stage<2, +1>(v, t, tw);
      exchange<2, 1>(v, buf, t);
    }
    if constexpr (NS > 1) {
      stage<1, +1>(v, t, tw);
      exchange<1, 0>(v, buf, t);
    }
    stage<0, +1>(v, t, tw);
  }
};

}  // namespace top
