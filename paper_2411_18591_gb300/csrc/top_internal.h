// Host/device shared structures of the propagation library.
//
// Every launch receives its parameters by value (a PassParams of a few KB in the
// kernel parameter space), so a call needs no host-to-device copies and stays
// capturable in a CUDA graph once its tables exist.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/top.h"

namespace top {

constexpr int kMaxSets = 24;      // distinct (lambda, z) parameter sets per launch
constexpr int kMaxFields = 2048;  // fields per launch (larger batches run in chunks)

// One (lambda, z) parameter set: the transfer function and the lens factors, computed in
// float64 and rounded to float32. H depends on the frequencies only through fx^2 and fy^2, so
// one quadrant is stored: hq[|kx| (My + 2) + j] = H(|kx|, |ky|) / (Py Px) for |kx| <= Px / 2,
// with the even |ky| = 2 j at j < My/2 + 1, the odd |ky| = 2 (j - My/2 - 1) + 1 after them and
// one zero entry that makes rows whole 16-byte units (one row per |kx|; a column half reads the
// even or the odd part of its row).
struct FieldSet {
  const float2* hq;      // [Px/2 + 1][My + 2]
  const float2* src_lx;  // lens factor tables of the source-side modulation: [nx], [ny]
  const float2* src_ly;
  const float2* epi_lx;  // lens factor tables of the epilogue-side modulation
  const float2* epi_ly;
};

// Element modulation (Eq. 1) applied in a prologue or epilogue.
struct ModDev {
  uint32_t flags;          // TOP_MOD_*
  int conj;                // apply conj(M)
  const float2* cmask;     // complex mask
  const float* amp;        // amplitude
  const float* phase;      // phase
  long long stride;        // elements between consecutive fields' masks (0 = shared)
  const int2* circ;        // [ny] inclusive x range inside the aperture per row (x > y: empty)
};

enum SrcKind : int {
  SRC_FIELD = 0,      // v = modsrc * in[f]
  SRC_INTENSITY = 1,  // v = modsrc * 2 w_f gI[f / group] psi[f]
};

enum EpiKind : int {
  EPI_FIELD = 0,      // out[f] = modepi * v
  EPI_INTENSITY = 1,  // I[g] += w_f |modepi * v|^2 over the group; optional out[f] = modepi * v
  EPI_MODGRAD = 2,    // gradient of a modulation y = M x: grad_in = conj(M) v, grads of M (partials)
  EPI_OVERLAP = 3,    // per row tile: sums of psi conj(phi) and |psi|^2, psi = modepi * v (Eq. 7); optional out[f]
};

struct PassParams {
  // geometry of the padded problem
  int ny, nx;      // field samples
  int Py, Px;      // padded sizes (even; each handled as two interleaved halves)
  int My, Mx;      // Py / 2, Px / 2
  int oy, ox;      // offset of the field in the padded grid
  int nfields;     // fields in this launch
  int group;       // fields per epilogue group (R2 grid.y = ceil(nfields / group))
  int src_group;   // fields sharing one intensity-gradient plane (SRC_INTENSITY)
  int in_repeat;   // SRC_FIELD: output field f reads input field f / in_repeat
  int method;      // top_method
  int adjoint;     // use conj(H)
  int src_kind;
  int epi_kind;
  int fp64_r;      // reserved
  int l2_ahead;    // blocks ahead whose input a block prefetches into L2 (0: none)
  uint32_t tune_rows;  // TOP_TUNE_* choices for the row passes (of Mx) and the column pass (of My)
  uint32_t tune_cols;

  // buffers (element strides per field)
  const float2* in;   long long in_stride;
  // ragged batches: per-field device pointers (device arrays of nfields entries) that replace
  // in + f * in_stride and out + f * out_stride when non-null
  const float2* const* in_list;
  float2* const* out_list;
  // per-field transfer-function tables (device array of nfields entries) that replace
  // sets[set_of[f]].hq in the column pass when non-null (ragged batches: no limit on the sets)
  const float2* const* hq_list;
  float2* ws;         long long ws_stride;   // pass workspace [field][Px][ny]
  float2* out;        long long out_stride;
  float* outf;        long long outf_stride; // intensity output per group / partial sums per group
  const float2* psi;  long long psi_stride;  // saved output field (SRC_INTENSITY)
  const float2* xs;   long long xs_stride;   // saved input x of the modulation (EPI_MODGRAD, modulate backward)
  const float* gI;    long long gI_stride;   // intensity gradient per group (SRC_INTENSITY)
  const float* weights;                      // per field or null
  float* part_phase;  float* part_amp;  float2* part_mask;  long long part_stride;  // EPI_MODGRAD partials per group
  int part_accumulate;                       // add to the partials instead of overwriting (later chunks)

  // engine tables
  const float2* twx;  // stage twiddles of the x engine
  const float2* twy;
  const float2* wpx;  // exp(-2 pi i p / Px), p < Mx
  const float2* wpy;

  // EPI_OVERLAP: target phi (+ f * target_stride) and float64 partial sums [field][row tile][3]
  // (re and im of sum psi conj(phi), sum |psi|^2)
  const float2* target; long long target_stride;
  double* ov_part;
  // shared sources (input_repeat): the column pass stores the forward spectrum of every column in
  // its register order (spec_out, one spectrum per launch field), or starts from the spectrum of
  // field f / in_repeat (spec_in) instead of loading, folding and transforming its columns.
  // Spectrum of field s, column kpos, half r, slot e, lane t at ((s Px + kpos) 2 + r) M + e G + t.
  float2* spec_out;
  const float2* spec_in;
  // column pass as the second half of a forward 2-D transform: bins of columns kx <= Px/2 go to
  // this quadrant table (FieldSet::hq layout) times hq_scale, nothing else is written
  float2* hq_out;
  float hq_scale;

  ModDev msrc;  // modulation applied to the R1 source
  ModDev mepi;  // modulation applied in the R2 epilogue

  int nsets;
  FieldSet sets[kMaxSets];
  unsigned char set_of[kMaxFields];
};

// Kernel launch timing kinds (instrumentation)
// Floats per R1 block of the planes staged besides the field rows: the intensity gradient
// (SRC_INTENSITY) and the phase, amplitude and complex mask of the source modulation.
__host__ __device__ inline size_t src_plane_floats(const PassParams& p, int rows) {
  const size_t plane = size_t(rows) * size_t(p.nx);
  size_t n = 0;
  if (p.src_kind == SRC_INTENSITY) n += plane;
  if (p.msrc.flags & TOP_MOD_PHASE) n += plane;
  if (p.msrc.flags & TOP_MOD_AMPLITUDE) n += plane;
  if (p.msrc.flags & TOP_MOD_COMPLEX) n += 2 * plane;
  return n;
}

// Line transforms of any length P by Bluestein's chirp-z method (padded sizes without a plan of
// their own): with c[n] = exp(-i pi n^2 / P), the DFT is X[k] = c[k] sum_n (x[n] c[n]) conj(c[k - n]),
// a convolution done as an L-point FFT (L >= 2P - 1), a product with the transform of the chirp
// (in bins) and an inverse L-point FFT; the inverse DFT uses the conjugate chirps.
enum CztMode : int {
  CZT_FWD = 0,     // forward DFT of the zero-padded line
  CZT_INV = 1,     // inverse DFT (unnormalised), then the output window
  CZT_FILTER = 2,  // forward DFT, times the transfer function (conjugated for the adjoint), inverse DFT, window
};

struct CztParams {
  const float2* in;      // line i of field f at in + (f / in_repeat) in_fstride + i in_lstride
  long long in_fstride;
  long long in_lstride;
  int in_repeat;
  float2* out;           // window sample k - k0 of line i of field f at out + f out_fstride + i out_lstride
  long long out_fstride;
  long long out_lstride;
  int nlines, nfields;
  int P;                 // DFT length
  int n_in, off_in;      // the line's samples sit at [off_in, off_in + n_in) of the zero-padded line
  int k0, n_out;         // output window
  int mode;              // CztMode
  int adjoint;
  float inv_l;           // 1 / L, L the convolution length
  const float2* chirp;   // c[n], n < P
  // L-point transforms of conj(c) (forward) and c (inverse) on the lags (-P, P), entry e G + t = the
  // bin lane t of the transforming engine holds in slot e; for L = 8192 split by parity (half r,
  // bins 2k + r, at r L/2, on the 4096-point engine)
  const float2* bh_fwd;
  const float2* bh_inv;
  const float2* tw;      // stage twiddles of the transforming engine
  const float2* wsplit;  // L = 8192: exp(-2 pi i p / L), p < L/2
  const float2* const* h;  // CZT_FILTER: per field, rows [line][P] of H / (Py Px) in natural order
};

// The autotune table (top_tune.cu): TOP_TUNE_* flags per line length M (0: the defaults).
uint32_t tune_flags(int M);
bool tune_flags_valid(uint32_t flags);
void tune_set(int M, uint32_t flags);
void tune_clear();
bool tune_save(const char* path, std::string* err);
bool tune_load(const char* path, std::string* err);
// Fields per block of the pair-local inverse pass with a field epilogue under tuning flags.
inline int tune_span(uint32_t flags) {
  const uint32_t c = (flags >> 8) & 7u;
  return c == 0 ? 4 : 1 << (c - 1);
}

// Largest dynamic shared memory of a fused chain block (R2 of one propagation + R1 of the next).
constexpr size_t kChainSmemMax = 227 * 1024;

enum KernelKind : int { KK_ROWS_FWD = 0, KK_COLS, KK_ROWS_INV, KK_AUX, KK_ROWS_CHAIN, KK_ONCHIP, KK_COUNT };

}  // namespace top
