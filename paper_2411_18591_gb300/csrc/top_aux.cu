#include "top_aux.h"

#include <cstring>

#include <algorithm>

#include "top_passes.cuh"

namespace top {

// out[f] = M_f * in[f] (Eq. 1), conj(M_f) where the modulation asks for it; fields of a repeat
// group (in_repeat > 1) read their group's input
__global__ void __launch_bounds__(256) k_modulate(const __grid_constant__ PassParams p) {
  const long long plane = (long long)p.ny * p.nx;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int f = blockIdx.y;
  if (i >= plane) return;
  const int y = int(i / p.nx), x = int(i - (long long)y * p.nx);
  const FieldSet& fs = p.sets[p.set_of[f]];
  const float2 m = mod_value(p.msrc, p.msrc.flags, p.msrc.conj, fs.src_lx, fs.src_ly, f, y, x, p.nx);
  const int fi = p.in_repeat > 1 ? f / p.in_repeat : f;  // fields in repeat groups share an input
  p.out[(long long)f * plane + i] = c_mul(p.in[(long long)fi * plane + i], m);
}

// Backward of y = M x: grad_in = conj(M) g; parameter gradients summed over the fields of a
// group in field order (one thread per pixel, so the sum order is fixed).
__global__ void __launch_bounds__(256) k_modulate_backward(const __grid_constant__ PassParams p) {
  const long long plane = (long long)p.ny * p.nx;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= plane) return;
  const int y = int(i / p.nx), x = int(i - (long long)y * p.nx);
  const int f0 = blockIdx.y * p.group, f1 = min(f0 + p.group, p.nfields);
  float gp = 0.f, ga = 0.f;
  float2 gm = make_float2(0.f, 0.f);
  const ModDev& m = p.msrc;
  for (int f = f0; f < f1; ++f) {
    const FieldSet& fs = p.sets[p.set_of[f]];
    const float2 g = ldg2(p.in + (long long)f * plane + i);
    const float2 mv = mod_value(m, m.flags, 0, fs.src_lx, fs.src_ly, f, y, x, p.nx);
    if (p.out) p.out[(long long)f * plane + i] = c_mulc(g, mv);
    if (p.xs) {
      const float2 xs = ldg2(p.xs + (long long)f * plane + i);
      if (p.part_phase) {
        const float2 ys = c_mul(mv, xs);
        gp += fmaf(g.y, ys.x, -g.x * ys.y);
      }
      if (p.part_amp) {
        const float2 d = c_mul(mod_value(m, m.flags & ~TOP_MOD_AMPLITUDE, 0, fs.src_lx, fs.src_ly, f, y, x, p.nx), xs);
        ga += fmaf(g.x, d.x, g.y * d.y);
      }
      if (p.part_mask) {
        const float2 r = c_mul(mod_value(m, m.flags & ~TOP_MOD_COMPLEX, 0, fs.src_lx, fs.src_ly, f, y, x, p.nx), xs);
        gm = c_add(gm, c_mulc(g, r));
      }
    }
  }
  if (p.xs) {
    const long long o = (long long)blockIdx.y * plane + i;  // group plane (shared mask: one group)
    if (p.part_phase) p.part_phase[o] = p.part_accumulate ? p.part_phase[o] + gp : gp;
    if (p.part_amp) p.part_amp[o] = p.part_accumulate ? p.part_amp[o] + ga : ga;
    if (p.part_mask) p.part_mask[o] = p.part_accumulate ? c_add(p.part_mask[o], gm) : gm;
  }
}

__global__ void __launch_bounds__(256) k_reduce_partials(const float* part_phase, const float* part_amp,
                                                         const float2* part_mask, int ngroups, long long plane,
                                                         float* phase, float* amp, float2* mask) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= plane) return;
  if (phase) {
    float s = 0.f;
    for (int g = 0; g < ngroups; ++g) s += part_phase[(long long)g * plane + i];
    phase[i] = s;
  }
  if (amp) {
    float s = 0.f;
    for (int g = 0; g < ngroups; ++g) s += part_amp[(long long)g * plane + i];
    amp[i] = s;
  }
  if (mask) {
    float2 s = make_float2(0.f, 0.f);
    for (int g = 0; g < ngroups; ++g) s = c_add(s, part_mask[(long long)g * plane + i]);
    mask[i] = s;
  }
}

// MSE: each of kMseBlocks blocks sums a fixed strided subset in float64 (fixed tree order),
// then one block sums the partials in a fixed order.
__global__ void __launch_bounds__(256) k_mse_partial(long long n, const float* I, const float* T, float* grad,
                                                     double* partial) {
  __shared__ double red[256];
  double acc = 0.0;
  const float scale = float(2.0 / double(n));
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float r = I[i] - T[i];
    acc += double(r) * double(r);
    if (grad) grad[i] = scale * r;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(256) k_mse_final(long long n, const double* partial, int np, double* loss) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += partial[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = red[0] / double(n);
}

// A chunk of words carried in the kernel's parameters.
constexpr int kPutWords = 1024;
struct PutChunk {
  unsigned long long w[kPutWords];
};

__global__ void __launch_bounds__(256) k_put(unsigned long long* dst, int n, const __grid_constant__ PutChunk c) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = c.w[i];
}

cudaError_t launch_put(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes % 8 != 0) return cudaErrorInvalidValue;
  const size_t words = bytes / 8;
  auto* d = static_cast<unsigned long long*>(dst);
  const auto* h = static_cast<const unsigned char*>(src);
  PutChunk c;
  for (size_t w0 = 0; w0 < words; w0 += kPutWords) {
    const int n = int(words - w0 < size_t(kPutWords) ? words - w0 : size_t(kPutWords));
    std::memcpy(c.w, h + w0 * 8, size_t(n) * 8);
    TOP_LAUNCH(k_put, 1, 256, 0, s, d + w0, n, c);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_modulate(const PassParams& p, cudaStream_t s) {
  const long long plane = (long long)p.ny * p.nx;
  dim3 grid(unsigned((plane + 255) / 256), p.nfields);
  TOP_LAUNCH(k_modulate, grid, 256, 0, s, p);
  return cudaGetLastError();
}

cudaError_t launch_modulate_backward(const PassParams& p, cudaStream_t s) {
  const long long plane = (long long)p.ny * p.nx;
  dim3 grid(unsigned((plane + 255) / 256), (p.nfields + p.group - 1) / p.group);
  TOP_LAUNCH(k_modulate_backward, grid, 256, 0, s, p);
  return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const float* part_phase, const float* part_amp, const float2* part_mask,
                                   int ngroups, long long plane, float* phase, float* amp, float2* mask,
                                   cudaStream_t s) {
  TOP_LAUNCH(k_reduce_partials, unsigned((plane + 255) / 256), 256, 0, s, part_phase, part_amp, part_mask, ngroups,
             plane, phase, amp, mask);
  return cudaGetLastError();
}

// Transfer function (Eq. 5; the Fresnel form for method TOP_FRESNEL_TF) on one quadrant of
// the padded frequency grid, in float64: f = |k| / (P d), the AS radicand evaluated as
// ((1 / (lambda lambda)) - fx fx) - fy fy with every operation rounded on its own (no fused
// multiply-add, so the evanescent decision is the same as an IEEE evaluation of that
// expression), H = 0 where it is negative, else exp(2 pi i z sqrt(radicand)). Phases are
// reduced in cycles (c - rint(c) is exact) before the sine and cosine.
__device__ __forceinline__ float2 transfer_value(int akx, int aky, int Py, int Px, double dy, double dx, double lam,
                                                 double z, int method) {
  const double fx = double(akx) / (double(Px) * dx);
  const double fy = double(aky) / (double(Py) * dy);
  const double fx2 = __dmul_rn(fx, fx), fy2 = __dmul_rn(fy, fy);
  const double norm = 1.0 / (double(Py) * double(Px));
  double cyc;
  if (method == TOP_AS) {
    const double rad = __dsub_rn(__dsub_rn(1.0 / __dmul_rn(lam, lam), fx2), fy2);
    if (rad < 0.0) return make_float2(0.f, 0.f);
    const double c = __dmul_rn(z, sqrt(rad));
    cyc = c - rint(c);
  } else {
    const double a = z / lam;
    const double b = 0.5 * lam * z * (fx2 + fy2);
    cyc = (a - rint(a)) - (b - rint(b));
  }
  double sn, cs;
  sincospi(2.0 * cyc, &sn, &cs);
  return make_float2(float(cs * norm), float(sn * norm));
}

__global__ void __launch_bounds__(256) k_transfer_table(float2* hq, int Py, int Px, double dy, double dx, double lam,
                                                        double z, int method) {
  const int my = Py / 2, even = my / 2 + 1;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int akx = blockIdx.y;
  if (j > my + 1) return;
  float2* out = hq + (long long)akx * (my + 2) + j;
  if (j == my + 1) {
    *out = make_float2(0.f, 0.f);
    return;
  }
  const int aky = j < even ? 2 * j : 2 * (j - even) + 1;
  *out = transfer_value(akx, aky, Py, Px, dy, dx, lam, z, method);
}

// The same values on the whole padded grid in natural order, one row per kx: h[kx Py + ky], with
// |k| = min(k, P - k) (any Py, Px).
__global__ void __launch_bounds__(256) k_transfer_full(float2* h, int Py, int Px, double dy, double dx, double lam,
                                                       double z, int method) {
  const int ky = blockIdx.x * blockDim.x + threadIdx.x;
  const int kx = blockIdx.y;
  if (ky >= Py) return;
  h[(long long)kx * Py + ky] = transfer_value(min(kx, Px - kx), min(ky, Py - ky), Py, Px, dy, dx, lam, z, method);
}

// out[b][c][r] = in[b][r][c] for [rows][cols] planes, through a 32 x 33 shared tile.
__global__ void __launch_bounds__(256) k_transpose_rect(const float2* in, float2* out, int rows, int cols) {
  __shared__ float2 tile[32][33];
  const long long base = (long long)blockIdx.z * rows * cols;
  const int bc = blockIdx.x * 32, br = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int r = br + j, c = bc + threadIdx.x;
    if (r < rows && c < cols) tile[j][threadIdx.x] = in[base + (long long)r * cols + c];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int c = bc + j, r = br + threadIdx.x;
    if (r < rows && c < cols) out[base + (long long)c * rows + r] = tile[threadIdx.x][j];
  }
}

// h_z(x, y) dx dy of Eq. 3 at x = sx dx, y = sy dy with (sx, sy) the signed lags of the grid:
// h = z / (i lambda d) (1 + i / (k d)) exp(i k d) / d = (z / (lambda d^2)) (1/(k d) - i) exp(i k d),
// the phase k d reduced in cycles (d / lambda - rint) before the sine and cosine.
__global__ void __launch_bounds__(256) k_di_samples(float2* out, int Py, int Px, double dy, double dx, double lam,
                                                    double z) {
  const int ix = blockIdx.x * blockDim.x + threadIdx.x;
  const int iy = blockIdx.y;
  if (ix >= Px) return;
  const int sx = ix < (Px + 1) / 2 ? ix : ix - Px;
  const int sy = iy < (Py + 1) / 2 ? iy : iy - Py;
  const double x = sx * dx, y = sy * dy;
  const double r2 = x * x + y * y + z * z;
  const double d = sqrt(r2);
  const double amp = z / (lam * r2) * (dx * dy);
  const double a = lam / (2.0 * 3.14159265358979323846 * d);  // 1 / (k d)
  const double c = d / lam;
  double sn, cs;
  sincospi(2.0 * (c - rint(c)), &sn, &cs);
  out[(long long)iy * Px + ix] = make_float2(float(amp * (a * cs + sn)), float(amp * (a * sn - cs)));
}

cudaError_t launch_di_samples(float2* out, int Py, int Px, double dy, double dx, double lam, double z, cudaStream_t s) {
  dim3 grid((Px + 255) / 256, Py);
  TOP_LAUNCH(k_di_samples, grid, 256, 0, s, out, Py, Px, dy, dx, lam, z);
  return cudaGetLastError();
}

// One warp per field: lanes take tiles lane, lane + 32, ... in order, then a fixed butterfly.
__global__ void __launch_bounds__(32) k_overlap_finish(const double* part, int ntiles, double area, double* overlap,
                                                       double* power) {
  const int f = blockIdx.x;
  const int lane = threadIdx.x;
  double sr = 0.0, si = 0.0, sp = 0.0;
  const double* pf = part + (long long)f * ntiles * 3;
  for (int i = lane; i < ntiles; i += 32) {
    sr += pf[3 * i];
    si += pf[3 * i + 1];
    sp += pf[3 * i + 2];
  }
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
    sp += __shfl_xor_sync(0xffffffffu, sp, o);
  }
  if (lane == 0) {
    overlap[2 * f] = sr * area;
    overlap[2 * f + 1] = si * area;
    if (power) power[f] = sp * area;
  }
}

cudaError_t launch_overlap_finish(const double* part, int ntiles, int nfields, double area, double* overlap,
                                  double* power, cudaStream_t s) {
  if (nfields < 1) return cudaSuccess;
  TOP_LAUNCH(k_overlap_finish, nfields, 32, 0, s, part, ntiles, area, overlap, power);
  return cudaGetLastError();
}

__global__ void k_overlap_loss_value(const double* overlap, long long batch, double* loss) {
  double l = 0.0;
  for (long long b = 0; b < batch; ++b) {
    const double re = overlap[2 * b], im = overlap[2 * b + 1];
    l += 1.0 - (re * re + im * im);
  }
  loss[0] = l / double(batch);
}

__global__ void __launch_bounds__(256) k_overlap_grad(const double* overlap, long long batch, const float2* target,
                                                      long long target_stride, long long plane, double area,
                                                      float2* grad) {
  const double s = -2.0 * area / double(batch);
  const long long total = batch * plane;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < total; j += (long long)gridDim.x * blockDim.x) {
    const long long b = j / plane, i = j - b * plane;
    const float2 c = make_float2(float(s * overlap[2 * b]), float(s * overlap[2 * b + 1]));
    grad[j] = c_mul(c, ldg2(target + b * target_stride + i));
  }
}

cudaError_t launch_overlap_loss(const double* overlap, long long batch, const float2* target, long long target_stride,
                                long long plane, double area, double* loss, float2* grad, cudaStream_t s) {
  TOP_LAUNCH(k_overlap_loss_value, 1, 1, 0, s, overlap, batch, loss);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !grad) return e;
  const long long blocks = (batch * plane + 255) / 256;
  TOP_LAUNCH(k_overlap_grad, unsigned(blocks < 152 * 64 ? blocks : 152 * 64), 256, 0, s, overlap, batch, target,
             target_stride, plane, area, grad);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------- Jones matrices

__device__ __forceinline__ float2 jones_at(const float2* J, const Jones3& ju, int k, long long px, long long plane) {
  return J ? ldg2(J + k * plane + px) : ju.m[k];
}

__global__ void __launch_bounds__(256) k_jones(const float2* in, float2* out, long long groups, long long inner,
                                               long long plane, const float2* J, const Jones3 ju) {
  const long long total = groups * inner * plane;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < total; j += (long long)gridDim.x * blockDim.x) {
    const long long px = j % plane, q = j / plane;
    const long long o = q / inner, i = q - o * inner;
    const long long base = (o * 3 * inner + i) * plane + px, cs = inner * plane;
    const float2 a0 = ldg2(in + base), a1 = ldg2(in + base + cs), a2 = ldg2(in + base + 2 * cs);
    float2 r[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      r[c] = c_add(c_add(c_mul(jones_at(J, ju, 3 * c, px, plane), a0), c_mul(jones_at(J, ju, 3 * c + 1, px, plane), a1)),
                   c_mul(jones_at(J, ju, 3 * c + 2, px, plane), a2));
    }
    out[base] = r[0];
    out[base + cs] = r[1];
    out[base + 2 * cs] = r[2];
  }
}

cudaError_t launch_jones(const float2* in, float2* out, long long groups, long long inner, long long plane,
                         const float2* J, Jones3 ju, cudaStream_t s) {
  const long long n = groups * inner * plane;
  if (n == 0) return cudaSuccess;
  const long long blocks = (n + 255) / 256;
  TOP_LAUNCH(k_jones, unsigned(blocks < 152 * 32 ? blocks : 152 * 32), 256, 0, s, in, out, groups, inner, plane, J, ju);
  return cudaGetLastError();
}

// one thread per pixel: grad_in for every polarised field, grad_J summed over them in order
__global__ void __launch_bounds__(256) k_jones_backward(const float2* in, const float2* gout, float2* gin, float2* gJ,
                                                        long long groups, long long inner, long long plane,
                                                        const float2* J, const Jones3 ju) {
  const long long px = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (px >= plane) return;
  float2 acc[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k] = make_float2(0.f, 0.f);
  const long long cs = inner * plane;
  for (long long o = 0; o < groups; ++o) {
    for (long long i = 0; i < inner; ++i) {
      const long long base = (o * 3 * inner + i) * plane + px;
      const float2 g0 = ldg2(gout + base), g1 = ldg2(gout + base + cs), g2 = ldg2(gout + base + 2 * cs);
      if (gJ) {
        const float2 x[3] = {ldg2(in + base), ldg2(in + base + cs), ldg2(in + base + 2 * cs)};
        const float2 g[3] = {g0, g1, g2};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) acc[3 * a + b] = c_add(acc[3 * a + b], c_mulc(g[a], x[b]));
      }
      if (gin) {
        float2 r[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          // (J^H g)_b = sum_a conj(J_ab) g_a
          r[b] = c_add(c_add(c_mul(c_conj(jones_at(J, ju, b, px, plane)), g0),
                             c_mul(c_conj(jones_at(J, ju, 3 + b, px, plane)), g1)),
                       c_mul(c_conj(jones_at(J, ju, 6 + b, px, plane)), g2));
        }
        gin[base] = r[0];
        gin[base + cs] = r[1];
        gin[base + 2 * cs] = r[2];
      }
    }
  }
  if (gJ) {
#pragma unroll
    for (int k = 0; k < 9; ++k) gJ[k * plane + px] = acc[k];
  }
}

cudaError_t launch_jones_backward(const float2* in, const float2* gout, float2* gin, float2* gJ, long long groups,
                                  long long inner, long long plane, const float2* J, Jones3 ju, cudaStream_t s) {
  if (plane == 0) return cudaSuccess;
  TOP_LAUNCH(k_jones_backward, unsigned((plane + 255) / 256), 256, 0, s, in, gout, gin, gJ, groups, inner, plane, J, ju);
  return cudaGetLastError();
}

// power: kPowerBlocks blocks per field, each a float64 grid-stride sum and a fixed-order tree
__global__ void __launch_bounds__(256) k_power_partial(const float2* field, long long plane, double* partial) {
  __shared__ double red[256];
  const long long b = blockIdx.y;
  const float2* f = field + b * plane;
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < plane; i += (long long)gridDim.x * blockDim.x) {
    const float2 v = ldg2(f + i);
    acc = fma(double(v.x), double(v.x), fma(double(v.y), double(v.y), acc));
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[b * gridDim.x + blockIdx.x] = red[0];
}

__global__ void k_power_finish(const double* partial, long long batch, int nblk, double area, double* power) {
  const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  double s = 0.0;
  for (int k = 0; k < nblk; ++k) s += partial[b * nblk + k];
  power[b] = s * area;
}

cudaError_t launch_field_power(const float2* field, long long batch, long long plane, double area, double* partial,
                               double* power, cudaStream_t s) {
  if (batch == 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  for (long long b0 = 0; b0 < batch && e == cudaSuccess; b0 += 65535) {
    const long long nb = batch - b0 < 65535 ? batch - b0 : 65535;
    dim3 grid(kPowerBlocks, unsigned(nb));
    TOP_LAUNCH(k_power_partial, grid, 256, 0, s, field + b0 * plane, plane, partial + b0 * kPowerBlocks);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  TOP_LAUNCH(k_power_finish, unsigned((batch + 255) / 256), 256, 0, s, partial, batch, kPowerBlocks, area, power);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------- resampling

// Output sample j of an axis at fractional input index u = (j - (n_out-1)/2) d_out / d_in +
// (n_in-1)/2 (float64, each operation rounded on its own): nearest takes floor(u + 1/2) with weight
// 1, bilinear floor(u) with 1 - t and floor(u) + 1 with t = u - floor(u).
__device__ __forceinline__ void axis_weights(int j, int n_in, double d_in, int n_out, double d_out, int mode, int& i0,
                                             float& w0, float& w1) {
  const double u = __dadd_rn(__ddiv_rn(__dmul_rn(__dsub_rn(double(j), (n_out - 1) / 2.0), d_out), d_in), (n_in - 1) / 2.0);
  if (mode == 0) {
    i0 = int(floor(__dadd_rn(u, 0.5)));
    w0 = 1.f;
    w1 = 0.f;
  } else {
    const double f = floor(u);
    i0 = int(f);
    const double t = __dsub_rn(u, f);
    w0 = float(1.0 - t);
    w1 = float(t);
  }
}

__global__ void __launch_bounds__(256) k_resample(const float2* in, float2* out, ResampleGeom g) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int a = blockIdx.y;
  const long long b = blockIdx.z;
  if (c >= g.nx2) return;
  int iy, ix;
  float wy0, wy1, wx0, wx1;
  axis_weights(a, g.ny, g.dy, g.ny2, g.dy2, g.mode, iy, wy0, wy1);
  axis_weights(c, g.nx, g.dx, g.nx2, g.dx2, g.mode, ix, wx0, wx1);
  const float2* f = in + b * (long long)g.ny * g.nx;
  float2 acc = make_float2(0.f, 0.f);
  const float wy[2] = {wy0, wy1}, wx[2] = {wx0, wx1};
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const int y = iy + p;
    if (wy[p] == 0.f || y < 0 || y >= g.ny) continue;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int x = ix + q;
      if (wx[q] == 0.f || x < 0 || x >= g.nx) continue;
      acc = c_add(acc, c_scale(ldg2(f + (long long)y * g.nx + x), wy[p] * wx[q]));
    }
  }
  out[(b * g.ny2 + a) * (long long)g.nx2 + c] = acc;
}

// first output index j whose sample can reach input index i (a safe lower bound, refined by the
// exact weights in the caller's loop)
__device__ __forceinline__ int first_reach(int i, int n_in, double d_in, int n_out, double d_out) {
  const double j = (double(i) - 1.0 - (n_in - 1) / 2.0) * d_in / d_out + (n_out - 1) / 2.0;
  return max(0, int(floor(j)) - 1);
}

// transpose: every input sample gathers the output samples that weigh it, in a fixed order
__global__ void __launch_bounds__(256) k_resample_t(const float2* gout, float2* gin, ResampleGeom g) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  const long long b = blockIdx.z;
  if (x >= g.nx) return;
  const float2* go = gout + b * (long long)g.ny2 * g.nx2;
  float2 acc = make_float2(0.f, 0.f);
  for (int a = first_reach(y, g.ny, g.dy, g.ny2, g.dy2); a < g.ny2; ++a) {
    int iy;
    float wy0, wy1;
    axis_weights(a, g.ny, g.dy, g.ny2, g.dy2, g.mode, iy, wy0, wy1);
    if (iy > y) break;
    const float wy = iy == y ? wy0 : (iy + 1 == y ? wy1 : 0.f);
    if (wy == 0.f) continue;
    for (int c = first_reach(x, g.nx, g.dx, g.nx2, g.dx2); c < g.nx2; ++c) {
      int ix;
      float wx0, wx1;
      axis_weights(c, g.nx, g.dx, g.nx2, g.dx2, g.mode, ix, wx0, wx1);
      if (ix > x) break;
      const float wx = ix == x ? wx0 : (ix + 1 == x ? wx1 : 0.f);
      if (wx == 0.f) continue;
      acc = c_add(acc, c_scale(ldg2(go + (long long)a * g.nx2 + c), wy * wx));
    }
  }
  gin[(b * g.ny + y) * (long long)g.nx + x] = acc;
}

cudaError_t launch_resample(const float2* in, float2* out, long long batch, ResampleGeom rg, int transpose,
                            cudaStream_t s) {
  for (long long b0 = 0; b0 < batch; b0 += 65535) {
    const unsigned nb = unsigned(batch - b0 < 65535 ? batch - b0 : 65535);
    if (!transpose) {
      dim3 grid(unsigned((rg.nx2 + 255) / 256), unsigned(rg.ny2), nb);
      TOP_LAUNCH(k_resample, grid, 256, 0, s, in + b0 * (long long)rg.ny * rg.nx, out + b0 * (long long)rg.ny2 * rg.nx2, rg);
    } else {
      dim3 grid(unsigned((rg.nx + 255) / 256), unsigned(rg.ny), nb);
      TOP_LAUNCH(k_resample_t, grid, 256, 0, s, in + b0 * (long long)rg.ny2 * rg.nx2, out + b0 * (long long)rg.ny * rg.nx, rg);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_transfer_table(float2* hq, int Py, int Px, double dy, double dx, double lam, double z, int method,
                                  cudaStream_t s) {
  const int my = Py / 2;
  dim3 grid((my + 2 + 255) / 256, Px / 2 + 1);
  TOP_LAUNCH(k_transfer_table, grid, 256, 0, s, hq, Py, Px, dy, dx, lam, z, method);
  return cudaGetLastError();
}

// out_b = 2 w_b gI[b / group] psi_b: the source of the intensity backward (Eq. 14, chain rule).
__global__ void __launch_bounds__(256) k_intensity_source(const float2* psi, const float* gI, const float* weights,
                                                          int group, long long plane, float2* out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long b = blockIdx.y;
  if (i >= plane) return;
  const float w = weights ? weights[b] : 1.f;
  const float g = gI[(b / group) * plane + i];
  out[b * plane + i] = c_scale(psi[b * plane + i], 2.f * w * g);
}

// I[g] = sum over the group's fields, in field order, of w_b |psi_b|^2 (Eq. 14).
__global__ void __launch_bounds__(256) k_intensity_sum(const float2* psi, const float* weights, int group,
                                                       long long plane, float* out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long g = blockIdx.y;
  if (i >= plane) return;
  float acc = 0.f;
  for (long long b = g * group; b < (g + 1) * group; ++b) {
    const float2 v = psi[b * plane + i];
    const float w = weights ? weights[b] : 1.f;
    const float e = w * fmaf(v.x, v.x, v.y * v.y);
    acc = b == g * group ? e : acc + e;
  }
  out[g * plane + i] = acc;
}

// Partial sums of Eq. 7 over the fields of a batch: block (tile, b) adds psi conj(phi) and |psi|^2
// over samples tile * 256 + tid + k * ntiles * 256 in float64, then the block's threads in a fixed
// order, into part[(b ntiles + tile) 3 + {0, 1, 2}] (the layout k_overlap_finish reads).
__global__ void __launch_bounds__(256) k_overlap_partials(const float2* psi, const float2* target,
                                                          long long target_stride, long long plane, double* part) {
  __shared__ double red[3 * 256];
  const int tile = blockIdx.x, ntiles = gridDim.x;
  const long long b = blockIdx.y;
  double re = 0.0, im = 0.0, pw = 0.0;
  for (long long i = (long long)tile * 256 + threadIdx.x; i < plane; i += (long long)ntiles * 256) {
    const float2 v = psi[b * plane + i];
    const float2 t = target[b * target_stride + i];
    const double vx = v.x, vy = v.y, px = t.x, py = t.y;
    re = fma(vx, px, fma(vy, py, re));
    im = fma(vy, px, fma(-vx, py, im));
    pw = fma(vx, vx, fma(vy, vy, pw));
  }
  red[3 * threadIdx.x] = re;
  red[3 * threadIdx.x + 1] = im;
  red[3 * threadIdx.x + 2] = pw;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sr = 0.0, si = 0.0, sp = 0.0;
    for (int k = 0; k < 256; ++k) {
      sr += red[3 * k];
      si += red[3 * k + 1];
      sp += red[3 * k + 2];
    }
    double* out = part + (b * ntiles + tile) * 3;
    out[0] = sr;
    out[1] = si;
    out[2] = sp;
  }
}

cudaError_t launch_overlap_partials(const float2* psi, const float2* target, long long target_stride, long long batch,
                                    long long plane, int ntiles, double* part, cudaStream_t s) {
  for (long long b0 = 0; b0 < batch; b0 += 65535) {
    const unsigned nb = unsigned(std::min<long long>(65535, batch - b0));
    TOP_LAUNCH(k_overlap_partials, dim3(ntiles, nb), 256, 0, s, psi + b0 * plane, target + b0 * target_stride,
               target_stride, plane, part + b0 * ntiles * 3);
  }
  return cudaGetLastError();
}

cudaError_t launch_intensity_source(const float2* psi, const float* gI, const float* weights, int group,
                                    long long batch, long long plane, float2* out, cudaStream_t s) {
  const long long step = 65535 - 65535 % group;  // launches of whole groups
  for (long long b0 = 0; b0 < batch; b0 += step) {
    const unsigned nb = unsigned(std::min<long long>(step, batch - b0));
    dim3 grid(unsigned((plane + 255) / 256), nb);
    TOP_LAUNCH(k_intensity_source, grid, 256, 0, s, psi + b0 * plane, gI + (b0 / group) * plane,
               weights ? weights + b0 : nullptr, group, plane, out + b0 * plane);
  }
  return cudaGetLastError();
}

cudaError_t launch_intensity_sum(const float2* psi, const float* weights, int group, long long ngroups, long long plane,
                                 float* out, cudaStream_t s) {
  for (long long g0 = 0; g0 < ngroups; g0 += 65535) {
    const unsigned ng = unsigned(std::min<long long>(65535, ngroups - g0));
    dim3 grid(unsigned((plane + 255) / 256), ng);
    TOP_LAUNCH(k_intensity_sum, grid, 256, 0, s, psi + g0 * group * plane, weights ? weights + g0 * group : nullptr,
               group, plane, out + g0 * plane);
  }
  return cudaGetLastError();
}

cudaError_t launch_transfer_full(float2* h, int Py, int Px, double dy, double dx, double lam, double z, int method,
                                 cudaStream_t s) {
  dim3 grid((Py + 255) / 256, Px);
  TOP_LAUNCH(k_transfer_full, grid, 256, 0, s, h, Py, Px, dy, dx, lam, z, method);
  return cudaGetLastError();
}

cudaError_t launch_transpose_rect(const float2* in, float2* out, long long batch, int rows, int cols, cudaStream_t s) {
  for (long long b0 = 0; b0 < batch; b0 += 65535) {
    const unsigned nb = unsigned(std::min<long long>(65535, batch - b0));
    dim3 grid((cols + 31) / 32, (rows + 31) / 32, nb);
    const long long off = b0 * rows * cols;
    TOP_LAUNCH(k_transpose_rect, grid, dim3(32, 8), 0, s, in + off, out + off, rows, cols);
  }
  return cudaGetLastError();
}

cudaError_t launch_mse(long long n, const float* I, const float* T, float* grad, double* partial, double* loss,
                       cudaStream_t s) {
  TOP_LAUNCH(k_mse_partial, kMseBlocks, 256, 0, s, n, I, T, grad, partial);
  TOP_LAUNCH(k_mse_final, 1, 256, 0, s, n, partial, kMseBlocks, loss);
  return cudaGetLastError();
}

}  // namespace top

namespace top {

// ----------------------------------------------------------------------------- coherence

__device__ __forceinline__ float2 coh_mask(const PassParams& p, int r) {
  const int y = r / p.nx, x = r - (r / p.nx) * p.nx;
  const FieldSet& fs = p.sets[0];
  return mod_value(p.msrc, p.msrc.flags, 0, fs.src_lx, fs.src_ly, 0, y, x, p.nx);
}

// out(r1, r2) = M(r1) conj(M(r2)) in(r1, r2)  (Eq. 12), or its conjugate factor for the backward
__global__ void __launch_bounds__(256) k_coh_modulate(const float2* in, float2* out, const __grid_constant__ PassParams p,
                                                      int n, int conj_mask) {
  const int r2 = blockIdx.x * blockDim.x + threadIdx.x;
  const int r1 = blockIdx.y;
  const long long b = blockIdx.z;
  if (r2 >= n) return;
  float2 d = c_mulc(coh_mask(p, r1), coh_mask(p, r2));
  if (conj_mask) d = c_conj(d);
  const long long i = (b * n + r1) * n + r2;
  out[i] = c_mul(in[i], d);
}

// batched square transpose through a 32 x 33 shared tile
__global__ void __launch_bounds__(256) k_transpose(const float2* in, float2* out, int n) {
  __shared__ float2 tile[32][33];
  const long long base = (long long)blockIdx.z * n * n;
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int r = by + j, c = bx + threadIdx.x;
    if (r < n && c < n) tile[j][threadIdx.x] = in[base + (long long)r * n + c];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int r = bx + j, c = by + threadIdx.x;
    if (r < n && c < n) out[base + (long long)r * n + c] = tile[threadIdx.x][j];
  }
}

__global__ void __launch_bounds__(256) k_coh_diag(const float2* gamma, float* inten, int n) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const long long b = blockIdx.y;
  if (r < n) inten[b * n + r] = gamma[(b * n + r) * n + r].x;
}

__global__ void __launch_bounds__(256) k_coh_diag_backward(const float* gI, float2* grad, int n) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const long long b = blockIdx.y;
  if (r < n) grad[(b * n + r) * n + r] = make_float2(gI[b * n + r], 0.f);
}

// M(s) for every s of the grid (the mask of Eq. 12, evaluated once for the gradient sums)
__global__ void __launch_bounds__(256) k_coh_mask_values(const __grid_constant__ PassParams p, int n, float2* mv) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) mv[s] = coh_mask(p, s);
}

// row term: one block per r, fixed tree order over s; batch summed in order
__global__ void __launch_bounds__(256) k_coh_grad_rows(const float2* G, const float2* Gm, const float2* mv, int n,
                                                       long long batch, float2* gm) {
  __shared__ float2 red[256];
  const int r = blockIdx.x;
  float2 acc = make_float2(0.f, 0.f);
  for (long long b = 0; b < batch; ++b) {
    const long long row = (b * n + r) * n;
    for (int s = threadIdx.x; s < n; s += blockDim.x) acc = c_add(acc, c_mul(c_mulc(G[row + s], Gm[row + s]), mv[s]));
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] = c_add(red[threadIdx.x], red[threadIdx.x + k]);
    __syncthreads();
  }
  if (threadIdx.x == 0) gm[r] = red[0];
}

// column term, partial sums: block (32 r, kCohWarps warps) of slice `split` of the s range; warp w
// sums its part of the slice in order (over the batch, then s), and the warps' sums are added in
// warp order: part[split][r]
constexpr int kCohSplit = 16;
constexpr int kCohWarps = 8;
__global__ void __launch_bounds__(32 * kCohWarps) k_coh_grad_cols_part(const float2* G, const float2* Gm, const float2* mv,
                                                                       int n, long long batch, float2* part) {
  __shared__ float2 red[kCohWarps][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int r = blockIdx.x * 32 + lane;
  const int per = (n + kCohSplit * kCohWarps - 1) / (kCohSplit * kCohWarps);
  const int s0 = (blockIdx.y * kCohWarps + w) * per, s1 = min(n, s0 + per);
  float2 acc = make_float2(0.f, 0.f);
  if (r < n) {
    for (long long b = 0; b < batch; ++b)
      for (int s = s0; s < s1; ++s) {
        const long long i = (b * n + s) * n + r;
        acc = c_add(acc, c_mul(c_mulc(Gm[i], G[i]), mv[s]));
      }
  }
  red[w][lane] = acc;
  __syncthreads();
  if (w == 0 && r < n) {
    float2 t = red[0][lane];
    for (int k = 1; k < kCohWarps; ++k) t = c_add(t, red[k][lane]);
    part[(long long)blockIdx.y * n + r] = t;
  }
}

// g_M(r) = row term + the column slices in order; then the parameter gradients
__global__ void __launch_bounds__(256) k_coh_grad_finish(const __grid_constant__ PassParams p, int n,
                                                         const float2* gm_rows, const float2* part, float* gphase,
                                                         float* gamp, float2* gmask) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  float2 acc = gm_rows[r];
  for (int k = 0; k < kCohSplit; ++k) acc = c_add(acc, part[(long long)k * n + r]);
  // acc = g_M(r) for the complex mask value M(r)
  const int y = r / p.nx, x = r - (r / p.nx) * p.nx;
  const FieldSet& fs = p.sets[0];
  const ModDev& m = p.msrc;
  const float2 mval = mod_value(m, m.flags, 0, fs.src_lx, fs.src_ly, 0, y, x, p.nx);
  if (gphase) gphase[r] = fmaf(mval.x, acc.y, -mval.y * acc.x);  // Im(conj(M) g_M)
  if (gamp) {
    const float2 ra = mod_value(m, m.flags & ~TOP_MOD_AMPLITUDE, 0, fs.src_lx, fs.src_ly, 0, y, x, p.nx);
    gamp[r] = fmaf(acc.x, ra.x, acc.y * ra.y);  // Re(conj(g_M) R_A)
  }
  if (gmask) {
    const float2 rc = mod_value(m, m.flags & ~TOP_MOD_COMPLEX, 0, fs.src_lx, fs.src_ly, 0, y, x, p.nx);
    gmask[r] = c_mulc(acc, rc);  // g_M conj(R_C)
  }
}

size_t coh_mask_grads_work(int n) { return sizeof(float2) * size_t(n) * (2 + kCohSplit); }

cudaError_t launch_coh_modulate(const float2* in, float2* out, const PassParams& p, long long batch, int conj_mask,
                                cudaStream_t s) {
  const int n = p.ny * p.nx;
  dim3 grid((n + 255) / 256, n, unsigned(batch));
  TOP_LAUNCH(k_coh_modulate, grid, 256, 0, s, in, out, p, n, conj_mask);
  return cudaGetLastError();
}

cudaError_t launch_transpose(const float2* in, float2* out, long long batch, int n, cudaStream_t s) {
  dim3 grid((n + 31) / 32, (n + 31) / 32, unsigned(batch));
  TOP_LAUNCH(k_transpose, grid, dim3(32, 8), 0, s, in, out, n);
  return cudaGetLastError();
}

cudaError_t launch_coh_diag(const float2* gamma, float* inten, long long batch, int n, cudaStream_t s) {
  dim3 grid((n + 255) / 256, unsigned(batch));
  TOP_LAUNCH(k_coh_diag, grid, 256, 0, s, gamma, inten, n);
  return cudaGetLastError();
}

cudaError_t launch_coh_diag_backward(const float* gI, float2* grad, long long batch, int n, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(float2) * size_t(batch) * n * n, s);
  if (e != cudaSuccess) return e;
  dim3 grid((n + 255) / 256, unsigned(batch));
  TOP_LAUNCH(k_coh_diag_backward, grid, 256, 0, s, gI, grad, n);
  return cudaGetLastError();
}

cudaError_t launch_coh_mask_grads(const float2* G, const float2* gamma_in, const PassParams& p, long long batch,
                                  float2* gm_work, float* grad_phase, float* grad_amp, float2* grad_mask,
                                  cudaStream_t s) {
  const int n = p.ny * p.nx;
  float2* rows = gm_work;
  float2* mv = gm_work + n;
  float2* part = gm_work + 2 * size_t(n);
  TOP_LAUNCH(k_coh_mask_values, (n + 255) / 256, 256, 0, s, p, n, mv);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  TOP_LAUNCH(k_coh_grad_rows, n, 256, 0, s, G, gamma_in, mv, n, batch, rows);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  TOP_LAUNCH(k_coh_grad_cols_part, dim3((n + 31) / 32, kCohSplit), 32 * kCohWarps, 0, s, G, gamma_in, mv, n, batch, part);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  TOP_LAUNCH(k_coh_grad_finish, (n + 255) / 256, 256, 0, s, p, n, rows, part, grad_phase, grad_amp, grad_mask);
  return cudaGetLastError();
}

}  // namespace top
