// Auxiliary kernels: standalone modulation (Eq. 1) and its backward, deterministic
// reductions of modulation-gradient partials, the MSE detector loss, the transfer-function
// table (Eq. 5 and the Fresnel form).
#pragma once

#include <cuda_runtime.h>

#include "top_internal.h"

namespace top {

constexpr int kMseBlocks = 1024;

// Write `bytes` (a multiple of 8) from host memory to device memory `dst` in stream order by kernel
// launches whose parameters carry the bytes: no host-to-device copy from pageable memory (which
// waits for the stream and cannot be captured in a CUDA graph), no pinned staging to keep alive.
cudaError_t launch_put(void* dst, const void* src, size_t bytes, cudaStream_t s);

// Device address of the static scratch of top_propagate_noalloc (TOP_NOALLOC_SCRATCH_BYTES) on the
// current device, looked up with cudaGetSymbolAddress on the first call per device.
cudaError_t noalloc_scratch_address(void** out);

cudaError_t launch_modulate(const PassParams& p, cudaStream_t s);
cudaError_t launch_modulate_backward(const PassParams& p, cudaStream_t s);
cudaError_t launch_reduce_partials(const float* part_phase, const float* part_amp, const float2* part_mask,
                                   int ngroups, long long plane, float* phase, float* amp, float2* mask,
                                   cudaStream_t s);
cudaError_t launch_mse(long long n, const float* I, const float* T, float* grad, double* partial, double* loss,
                       cudaStream_t s);
// Samples of h_z (Eq. 3) times dx dy at the signed lags of a Py x Px grid, row-major (float64
// arithmetic, rounded once), the kernel of the Direct Integration method.
cudaError_t launch_di_samples(float2* out, int Py, int Px, double dy, double dx, double lam, double z, cudaStream_t s);
// Overlaps of Eq. 7 and powers per field from the row-tile partial sums of an EPI_OVERLAP pass:
// overlap[2 f] + i overlap[2 f + 1] = area sum_tiles, power[f] = area sum_tiles (fixed order).
cudaError_t launch_overlap_finish(const double* part, int ntiles, int nfields, double area, double* overlap,
                                  double* power, cudaStream_t s);
// L = mean_b (1 - |O_b|^2) into loss[0] and, when grad is non-null, grad_b = -(2/B) O_b phi_b area.
cudaError_t launch_overlap_loss(const double* overlap, long long batch, const float2* target, long long target_stride,
                                long long plane, double area, double* loss, float2* grad, cudaStream_t s);
// Jones matrices (§5.1) on three-component fields: field (o 3 + c) inner + i holds component c of
// polarised field (o, i). J: per-pixel planes [3][3][plane] or, when null, the uniform matrix ju.
struct Jones3 {
  float2 m[9];
};
cudaError_t launch_jones(const float2* in, float2* out, long long groups, long long inner, long long plane,
                         const float2* J, Jones3 ju, cudaStream_t s);
// grad_in = J^H grad_out (optional) and grad_J = sum over the polarised fields of grad_out conj(in)^T
// per pixel (optional, per-pixel J only), the sum in field order.
cudaError_t launch_jones_backward(const float2* in, const float2* gout, float2* gin, float2* gJ, long long groups,
                                  long long inner, long long plane, const float2* J, Jones3 ju, cudaStream_t s);
// power[b] = area sum |field_b|^2 (float64, fixed order); partial: batch * kPowerBlocks doubles.
constexpr int kPowerBlocks = 64;
cudaError_t launch_field_power(const float2* field, long long batch, long long plane, double area, double* partial,
                               double* power, cudaStream_t s);
// Interpolation between centred grids (nearest: mode 0, bilinear: 1) and its transpose.
struct ResampleGeom {
  int ny, nx, ny2, nx2;
  double dy, dx, dy2, dx2;
  int mode;
};
cudaError_t launch_resample(const float2* in, float2* out, long long batch, ResampleGeom rg, int transpose,
                            cudaStream_t s);
// Quadrant table of H / (Py Px) for one (lambda, z) in the FieldSet::hq layout (float64 arithmetic).
cudaError_t launch_transfer_table(float2* hq, int Py, int Px, double dy, double dx, double lam, double z, int method,
                                  cudaStream_t s);
// The same values on the whole grid in natural order, h[kx Py + ky] (the Bluestein column lines).
cudaError_t launch_transfer_full(float2* h, int Py, int Px, double dy, double dx, double lam, double z, int method,
                                 cudaStream_t s);
// Intensity (Eq. 14) as separate passes: out_b = 2 w_b gI[b / group] psi_b (the backward's source),
// and I[g] = sum over group g's fields, in field order, of w_b |psi_b|^2. weights may be null (1).
cudaError_t launch_intensity_source(const float2* psi, const float* gI, const float* weights, int group,
                                    long long batch, long long plane, float2* out, cudaStream_t s);
cudaError_t launch_intensity_sum(const float2* psi, const float* weights, int group, long long ngroups, long long plane,
                                 float* out, cudaStream_t s);
// Per-field partial sums of Eq. 7 (psi conj(phi), |psi|^2; float64, fixed order) in ntiles tiles,
// part[(b ntiles + tile) 3 + c], for launch_overlap_finish; target_stride 0 shares phi.
cudaError_t launch_overlap_partials(const float2* psi, const float2* target, long long target_stride, long long batch,
                                    long long plane, int ntiles, double* part, cudaStream_t s);
// Whole propagations of 64 x 64 fields at padding 2 in one kernel (top_onchip.cu), for plain
// requests: a field source without modulation and a field epilogue without modulation.
bool onchip_supported(const PassParams& p);
cudaError_t launch_onchip(const PassParams& p, cudaStream_t s);
// out[b][c][r] = in[b][r][c] for a batch of [rows][cols] planes.
cudaError_t launch_transpose_rect(const float2* in, float2* out, long long batch, int rows, int cols, cudaStream_t s);

}  // namespace top

namespace top {

// Mutual coherence (Eq. 12-13), tensors [batch][n][n] with n = ny * nx.
cudaError_t launch_coh_modulate(const float2* in, float2* out, const PassParams& p, long long batch, int conj_mask,
                                cudaStream_t s);
cudaError_t launch_transpose(const float2* in, float2* out, long long batch, int n, cudaStream_t s);
cudaError_t launch_coh_diag(const float2* gamma, float* inten, long long batch, int n, cudaStream_t s);
cudaError_t launch_coh_diag_backward(const float* gI, float2* grad, long long batch, int n, cudaStream_t s);
// g_M(r) = sum_s G(r,s) conj(Gm(r,s)) M(s) + sum_s conj(G(s,r)) Gm(s,r) M(s), summed over the batch,
// then turned into phase / amplitude / complex-mask gradients; gm_work holds
// coh_mask_grads_work(ny nx) bytes (the row terms, the mask values and the column slices; the
// column sum runs in slices over the grid, each slice in a fixed order, the slices in order).
size_t coh_mask_grads_work(int n);
cudaError_t launch_coh_mask_grads(const float2* G, const float2* gamma_in, const PassParams& p, long long batch,
                                  float2* gm_work, float* grad_phase, float* grad_amp, float2* grad_mask,
                                  cudaStream_t s);

}  // namespace top
