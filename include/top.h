/*
 * top.h -- C ABI of a GB300 (sm_103a) library for differentiable free-space
 * propagation of sampled scalar optical fields (TorchOptics, arXiv 2411.18591).
 *
 * The library implements, in its own CUDA kernels (no cuFFT):
 *   - angular-spectrum (AS) propagation, Eq. 4 with the transfer function of
 *     Eq. 5, and the Fresnel transfer-function variant named in §3;
 *   - configurable zero padding and cropping (§3);
 *   - element modulation, Eq. 1 (phase masks, amplitude masks, complex masks,
 *     thin lenses and circular apertures, §2 and §5.4), fused into the
 *     propagation passes;
 *   - detector intensity |psi|^2 and the incoherent sum of Eq. 14, fused;
 *   - the hand-written adjoint (backward) of all of the above (§4);
 *   - mutual-coherence modulation and propagation, Eq. 12-13 (§5.2).
 *
 * Conventions shared by every call
 *   - Fields are complex64 (interleaved float re, im), row-major
 *     [batch][ny][nx], x fastest. Intensities and phases are float32.
 *   - All field, mask and gradient buffers are DEVICE memory owned by the
 *     caller and must be 16-byte aligned; the library never frees them.
 *     Wavelength and distance arrays (lambda, z) are HOST arrays of doubles.
 *   - Padded size per axis P = floor(pad * n + 0.5) (P >= n); the field sits at
 *     offset floor((P - n) / 2) of the padded grid and is cropped from the same
 *     window. Frequencies are f_k = k / (P d) with k in FFT order. The forward
 *     DFT is unnormalised and the inverse carries 1 / (Py Px).
 *   - AS transfer function H = exp(2 pi i z sqrt(1/lambda^2 - fx^2 - fy^2)), set
 *     to 0 where the radicand is negative (evanescent cutoff). Fresnel transfer
 *     function H = exp(2 pi i z / lambda) exp(-i pi lambda z (fx^2 + fy^2)).
 *   - Gradients use the real-loss convention g = dL/dRe + i dL/dIm, so the
 *     backward of a complex-linear map A is its adjoint A^H.
 *   - Calls are asynchronous on the caller's CUDA stream (cudaStream_t passed as
 *     void*, NULL = legacy default stream). Argument errors are detected on the
 *     host before anything is launched. Nothing throws across the ABI; every
 *     call returns a top_status and top_last_error() gives a message for the
 *     calling thread.
 *   - Transfer-function, lens and aperture tables are built on first use of a
 *     parameter set and cached in the handle; the handle's workspace grows on
 *     first use of a grid size. Make one warm-up call with each parameter set
 *     before capturing a stream into a CUDA graph (table building and workspace
 *     growth allocate and copy synchronously).
 *   - Results are deterministic: batch reductions use a fixed order, no atomics.
 *   - One handle must not be used from two host threads at the same time.
 */
#ifndef TOP_H_
#define TOP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TOP_ABI_VERSION 1

typedef enum top_status {
  TOP_OK = 0,
  TOP_ERR_INVALID_ARG = 1, /* bad size, spacing, wavelength, pointer or alignment */
  TOP_ERR_UNSUPPORTED = 2, /* valid request outside what the kernels implement */
  TOP_ERR_OOM = 3,         /* device allocation failed (workspace or tables) */
  TOP_ERR_CUDA = 4,        /* a CUDA runtime call failed */
  TOP_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
  TOP_ERR_INTERNAL = 6
} top_status;

/* Propagation method (§3): angular spectrum (Eq. 4-5) or Fresnel transfer function. */
/* TOP_AS: angular spectrum (Eq. 4-5). TOP_FRESNEL_TF: Fresnel transfer function (§3).
 * TOP_DI: Direct Integration (§3): Eq. 2 as the convolution with h_z (Eq. 3) sampled at the
 * grid's lags, by FFT; needs a padded size of at least 2n - 1 per axis and z > 0.
 * TOP_AUTO: per field, AS when z < z_critical (Eq. 6, the smaller of n dx^2 / lambda and
 * n dy^2 / lambda) and DI otherwise, the paper's default choice. */
typedef enum top_method { TOP_AS = 0, TOP_FRESNEL_TF = 1, TOP_DI = 2, TOP_AUTO = 3 } top_method;

typedef struct top_ctx* top_handle;

/* Planar sampling grid shared by all fields of a call (§3: "a discrete grid that is
 * uniformly sampled over the xy-plane"). */
typedef struct top_grid {
  int64_t batch;  /* number of fields (or coherence tensors), >= 1 */
  int32_t ny, nx; /* samples per field, >= 1 */
  double dy, dx;  /* sample spacing in metres, > 0 */
  double pad;     /* zero-padding factor per axis, P = floor(pad*n + 0.5) >= n */
  int32_t method; /* top_method */
  int32_t input_repeat; /* forward calls only: input field b / input_repeat feeds output field b (0 or 1:
                           one input per output). Broadcasts one object over consecutive wavelengths
                           (Listing 5). Must divide batch; backward calls require 0 or 1. */
} top_grid;

/* Element modulation M(x, y) of Eq. 1, a product of the enabled factors:
 *   TOP_MOD_COMPLEX    complex64 mask [ny][nx]
 *   TOP_MOD_AMPLITUDE  float32 amplitude A [ny][nx]
 *   TOP_MOD_PHASE      float32 phase phi [ny][nx], factor exp(i phi)
 *   TOP_MOD_LENS       thin lens exp(-i pi (x^2 + y^2) / (lambda f)) (§2 Lens, §5.4)
 *   TOP_MOD_CIRC       circular aperture: 1 where x^2 + y^2 <= R^2, else 0 (§5.4)
 * Sample positions are x_i = (i - (nx-1)/2) dx, y_j = (j - (ny-1)/2) dy. */
#define TOP_MOD_COMPLEX 0x1u
#define TOP_MOD_AMPLITUDE 0x2u
#define TOP_MOD_PHASE 0x4u
#define TOP_MOD_LENS 0x8u
#define TOP_MOD_CIRC 0x10u

typedef struct top_mod {
  uint32_t flags;         /* OR of TOP_MOD_* (0 = identity) */
  int32_t reserved;
  const void* mask;       /* TOP_MOD_COMPLEX: complex64, device */
  const float* amplitude; /* TOP_MOD_AMPLITUDE: float32, device */
  const float* phase;     /* TOP_MOD_PHASE: float32, device */
  int64_t batch_stride;   /* elements between the masks of consecutive fields; 0 = one mask for all */
  double focal_length;    /* TOP_MOD_LENS: f in metres (non-zero) */
  double radius;          /* TOP_MOD_CIRC: R in metres (>= 0) */
} top_mod;

/* Gradients of a modulation's parameters (backward of Eq. 1), accumulated over the
 * batch in a fixed order when the mask is shared (batch_stride == 0), per field
 * otherwise. Any output pointer may be NULL. */
typedef struct top_mod_grads {
  const void* saved_in; /* complex64 [batch][ny][nx]: the field x that entered M in the forward pass */
  float* grad_phase;    /* dL/dphi, float32 */
  float* grad_amplitude;/* dL/dA, float32 */
  void* grad_mask;      /* dL/dRe M + i dL/dIm M, complex64 */
} top_mod_grads;

/* ---------------------------------------------------------------- handle and errors */

/* Create a handle bound to CUDA device `device`. Returns TOP_ERR_CUDA without a GPU. */
top_status top_create(top_handle* out, int device);
/* Synchronise the device, free the workspace and cached tables, destroy the handle. */
top_status top_destroy(top_handle h);
/* Message of the last failing call on this host thread ("" if none). Never NULL. */
const char* top_last_error(void);
/* Static name of a status code. */
const char* top_status_string(top_status s);
/* TOP_ABI_VERSION of the loaded library. */
int top_version(void);
/* Cap on the handle's workspace in bytes (default 8 GiB, at least 1 MiB: TOP_ERR_INVALID_ARG
 * below); larger batches run in chunks, and a call whose smallest chunk needs more returns
 * TOP_ERR_OOM before launching anything. */
top_status top_set_workspace_limit(top_handle h, uint64_t bytes);

/* Host-only plan query: padded sizes and per-field workspace bytes of a propagation.
 * Validates `g` exactly like the propagation calls. Padded sizes P = floor(pad n + 0.5) of
 * 2 x {16 .. 4096 powers of two, 250, 500, 768, 1000} have FFT plans of their own (one
 * field-sized workspace buffer); any other size up to 4096 per axis goes through Bluestein
 * transforms (two buffers); larger unplanned sizes return TOP_ERR_UNSUPPORTED. */
top_status top_plan_query(const top_grid* g, int64_t* py, int64_t* px, uint64_t* workspace_per_field);

/* Eq. 6: z_critical = L dx / lambda. AS is the accurate method for z < z_critical. */
double top_zcritical(double L, double dx, double lambda);

/* ---------------------------------------------------------------- propagation (Eq. 4-5) */

/* out = post * P_z(pre * in) for every field (Eq. 1 then Eq. 4, then Eq. 1).
 * in, out: complex64 [batch][ny][nx] device (in == out allowed).
 * lambda, z: host arrays of n_lz values, n_lz == 1 (shared) or == batch (per field).
 * pre, post: modulations or NULL.
 * Padded sizes without an FFT plan of their own (odd, or with prime factors above 5; up to
 * 4096 per axis) use Bluestein line transforms: the same result (a DFT of length P per axis),
 * with modulations, intensities and the intensity backward's source as separate passes, and
 * modulation gradients from the adjoint propagation by the modulation's own backward; this holds
 * for the backward, intensity, overlap, chain and ragged calls and for TOP_DI (its kernel
 * transformed by the same line transforms) too. The no-alloc call needs a planned size
 * (TOP_ERR_UNSUPPORTED). */
top_status top_propagate(top_handle h, const top_grid* g, const void* in, void* out,
                         const double* lambda, const double* z, int64_t n_lz,
                         const top_mod* pre, const top_mod* post, void* stream);

/* A ragged batch (fields of different sizes, spacings, wavelengths and distances, §5.3-style
 * mixed workloads): field i has its own grid grids[i] (batch 1, input_repeat 0 or 1),
 * wavelength lambda[i], distance z[i] and device buffers in[i] -> out[i] (complex64 [ny][nx],
 * 16-byte aligned; in[i] == out[i] allowed). out[i] = P_z(in[i]) (Eq. 4), or the adjoint
 * P_z^H when `backward` is non-zero. Fields with the same size and padded size share one launch
 * of each pass whatever their method, spacing, wavelength and distance (per-field pointers to the
 * fields and to their transfer-function tables replace the batch strides; up to 2048 fields a
 * launch, fewer when the workspace limit asks for it); padded sizes without a plan of their own
 * run field by field through the Bluestein transforms. The per-field lists reach the device
 * through the parameters of small kernels in stream order (no host-to-device copy), so once the
 * handle holds the tables and workspace a call launches kernels only. grids, in, out, lambda, z
 * are host arrays of `count` entries. Results equal top_propagate / top_propagate_backward per
 * field. */
top_status top_propagate_ragged(top_handle h, int count, const top_grid* grids, const void* const* in,
                                void* const* out, const double* lambda, const double* z, int backward, void* stream);

/* One stage of a system chain: the field entering the stage is multiplied by `pre` (Eq. 1;
 * NULL: none) and propagated by `z` (Eq. 4). `keep`, when non-NULL, receives the stage's output
 * field (complex64 [batch][ny][nx] device, caller-owned); the last stage's must be NULL. */
typedef struct top_stage {
  double z;
  const top_mod* pre;
  void* keep;
} top_stage;

/* A system of §2 (elements in sequence, Fig. 1) on every field: x_0 = in and
 * x_k = P_{z_k}(pre_k x_{k-1}) for k = 1 .. nstages, with the inverse row pass of each stage and
 * the forward row pass of the next fused into one kernel, so x_k reaches global memory only
 * through stages[k-1].keep. The last field x_K goes to `out` (may be NULL when `intensity` is
 * given) and, when `intensity` is non-NULL, |x_K|^2 summed over each `group` consecutive fields
 * (Eq. 14) to intensity [batch / group][ny][nx] (float32). g->input_repeat as in top_propagate.
 * lambda: host, n_lz values (1 or batch), shared by every stage. Results equal the same
 * sequence of top_propagate calls; a boundary whose modulation planes would not fit in shared
 * memory runs as two launches (through `keep`, or a field-sized scratch in the workspace). */
top_status top_fused_chain(top_handle h, const top_grid* g, const void* in, void* out, float* intensity,
                           int64_t group, const double* lambda, int64_t n_lz, const top_stage* stages,
                           int nstages, void* stream);

/* Backward of a chain ending at the grouped intensity (§4 through a System of §2): with the
 * forward chain of top_fused_chain (x_k = P_{z_k}(pre_k x_{k-1}), k = 1 .. nstages, the same
 * `stages` in forward order; their keep pointers are not used) and
 * I[b / group] = sum of |x_K|^2 over each group of fields (Eq. 14), given the saved last field
 * `field` = x_K (complex64 [batch][ny][nx]) and grad_intensity = dL/dI ([batch / group][ny][nx]
 * float32): g_K = 2 dL/dI x_K, then for k = K .. 1 h_k = P_{z_k}^H g_k (conj(H)) and
 * g_{k-1} = conj(pre_k) h_k. grad_in (may be NULL when first_grads asks for a gradient) receives
 * g_0; first_grads (may be NULL) the gradients of stages[0].pre's phase / amplitude / mask from
 * h_1 and its saved_in = x_0, as top_propagate_backward gives them. Each stage boundary (inverse
 * rows of one adjoint propagation, conj(pre) of its element, forward rows of the next) is one
 * fused row pass; padded sizes without a plan, or boundaries whose operands do not fit, run as
 * separate propagations through a field-sized scratch with the same results. Results equal the
 * sequence top_propagate_intensity_backward (stage K, post NULL) then top_propagate_backward
 * (stage k with post = pre_{k+1}) down to stage 1. lambda: host, n_lz values (1 or batch);
 * g->input_repeat 0 or 1. */
top_status top_fused_chain_backward(top_handle h, const top_grid* g, const void* field, const float* grad_intensity,
                                    int64_t group, const double* lambda, int64_t n_lz, const top_stage* stages,
                                    int nstages, const top_mod_grads* first_grads, void* grad_in, void* stream);

/* Bytes of the library's static device scratch used by top_propagate_noalloc. */
#define TOP_NOALLOC_SCRATCH_BYTES (64u << 20)

/* out = P_z(in) for every field (Eq. 4 with H of Eq. 5, or the Fresnel form) without a
 * handle and without allocating device memory. The paper has no counterpart: this is an
 * engineering variant of top_propagate (pre = post = NULL, input_repeat 0 or 1) for callers
 * that cannot allocate -- a process whose device memory is held by another allocator (a
 * cudaMalloc here would fail or force that allocator to release its cache), or a caller that
 * must not stall other streams (a handle grows its workspace with a device-wide synchronise,
 * cudaFree and cudaMalloc) -- and for callers that hold no handle.
 *
 * Scratch: the twiddle and transfer-function tables and the frequency-domain workspace of
 * each chunk of fields live in one static device array of TOP_NOALLOC_SCRATCH_BYTES per
 * device (the current device of the calling thread). The array sits in a device-code module of
 * its own: a device holds it from the first no-alloc call there until the process exits (or from
 * context creation when CUDA loads modules eagerly, CUDA_MODULE_LOADING=EAGER); processes that
 * never make the call do not pay for it under CUDA's default lazy loading. Every call rewrites
 * the tables on `stream` (twiddles written by kernels that carry them in their parameters,
 * transfer functions built by a kernel), so nothing in the scratch needs to start at zero.
 * Fields are processed in chunks that fit: a chunk of n fields needs n * Px * ny * 8 bytes of
 * workspace and one table of (Px/2 + 1)(Py/2 + 2) * 8 bytes per distinct (lambda, z) among them
 * (at most 24), and the chunk is the largest n that fits (1024^2 fields at 2x padding: 16 MiB of
 * workspace and 8.4 MiB of table each, so three fields of one (lambda, z), or two of two). A grid
 * whose single field and table do not fit is rejected with TOP_ERR_UNSUPPORTED before
 * anything is launched.
 * The first call on a device looks up the scratch address (cudaGetSymbolAddress, which loads
 * that module): make it before any stream capture. Calls share the scratch, so two calls in
 * flight at once on one device (other streams, other threads) race; order them on one stream or
 * synchronise between them.
 * in, out: complex64 [batch][ny][nx] device, 16-byte aligned (in == out allowed); lambda, z:
 * host arrays of n_lz values (1 or batch). Results equal top_propagate's bit for bit. */
top_status top_propagate_noalloc(const top_grid* g, const void* in, void* out, const double* lambda,
                                 const double* z, int64_t n_lz, void* stream);

/* Backward of top_propagate (§4): grad_in = conj(pre) * P_z^H(conj(post) * grad_out),
 * P_z^H using conj(H). grad_in may be NULL when only `pre_grads` is wanted.
 * pre_grads (may be NULL): gradients of pre's phase / amplitude / mask; needs
 * pre_grads->saved_in = the `in` of the forward call. */
top_status top_propagate_backward(top_handle h, const top_grid* g, const void* grad_out, void* grad_in,
                                  const double* lambda, const double* z, int64_t n_lz,
                                  const top_mod* pre, const top_mod* post,
                                  const top_mod_grads* pre_grads, void* stream);

/* Detector intensity fused into the propagation (Eq. 14):
 * I[b / group] = sum over each consecutive group of `group` fields of w_b |post * P_z(pre * in_b)|^2.
 * intensity: float32 [batch/group][ny][nx]; weights: device float32 [batch] or NULL (all 1);
 * field_out: complex64 [batch][ny][nx] or NULL, receives post * P_z(pre * in) (needed by the backward). */
top_status top_propagate_intensity(top_handle h, const top_grid* g, const void* in, void* field_out,
                                   float* intensity, int64_t group, const float* weights,
                                   const double* lambda, const double* z, int64_t n_lz,
                                   const top_mod* pre, const top_mod* post, void* stream);

/* Backward of top_propagate_intensity: with psi = the saved field_out,
 * grad_in = conj(pre) * P_z^H(conj(post) * 2 w_b grad_I[b/group] psi_b); pre_grads as in
 * top_propagate_backward. grad_intensity: float32 [batch/group][ny][nx]. */
top_status top_propagate_intensity_backward(top_handle h, const top_grid* g, const void* field,
                                            const float* grad_intensity, void* grad_in, int64_t group,
                                            const float* weights, const double* lambda, const double* z,
                                            int64_t n_lz, const top_mod* pre, const top_mod* post,
                                            const top_mod_grads* pre_grads, void* stream);

/* Detector intensity of fields already at the detector (Eq. 14, without a propagation):
 * I[b / group] = sum over each consecutive group of `group` fields of w_b |field_b|^2, summed in
 * field order. field: complex64 [batch][ny][nx] device; intensity: float32 [batch/group][ny][nx]
 * device; weights: device float32 [batch] or NULL (all 1); group >= 1 divides batch. The grid's
 * spacing, padding and method are not used. Errors: TOP_ERR_INVALID_ARG before any launch. */
top_status top_intensity(top_handle h, const top_grid* g, const void* field, float* intensity, int64_t group,
                         const float* weights, void* stream);

/* Backward of top_intensity: grad_field_b = 2 w_b grad_I[b / group] field_b (the gradient of a
 * real loss in the g = dL/dRe + i dL/dIm convention). grad_intensity: float32 [batch/group][ny][nx];
 * grad_field: complex64 [batch][ny][nx] (grad_field == field allowed). */
top_status top_intensity_backward(top_handle h, const top_grid* g, const void* field, const float* grad_intensity,
                                  void* grad_field, int64_t group, const float* weights, void* stream);

/* ---------------------------------------------------------------- modulation (Eq. 1) */

/* out = M * in, point-wise (in == out allowed). lambda (host, n_lz values) is used by lenses only. */
top_status top_modulate(top_handle h, const top_grid* g, const top_mod* mod, const void* in, void* out,
                        const double* lambda, int64_t n_lz, void* stream);

/* Backward of top_modulate: grad_in = conj(M) * grad_out (grad_in may be NULL) and the
 * parameter gradients of `grads` (grads->saved_in = the forward `in`). */
top_status top_modulate_backward(top_handle h, const top_grid* g, const top_mod* mod, const void* grad_out,
                                 void* grad_in, const top_mod_grads* grads, const double* lambda,
                                 int64_t n_lz, void* stream);

/* ---------------------------------------------------------------- losses */

/* The overlap integral of Eq. 7 at the output of a propagation, fused into its last pass: for
 * every field O_b = sum_{x,y} psi_b conj(phi_b) dx dy and its power sum |psi_b|^2 dx dy, with
 * psi_b = post * P_z(pre * in_b) (Eq. 1, Eq. 4). target phi: complex64 device, [ny][nx]
 * (target_stride 0, shared) or [batch][ny][nx] (target_stride ny nx). overlap: device
 * double[2 batch] (re, im per field); power: device double[batch] or NULL; field_out: psi
 * (complex64 [batch][ny][nx]) or NULL, in which case psi is never written. The sums are
 * float64 in a fixed order (deterministic). */
top_status top_propagate_overlap(top_handle h, const top_grid* g, const void* in, void* field_out,
                                 const void* target, int64_t target_stride, double* overlap, double* power,
                                 const double* lambda, const double* z, int64_t n_lz, const top_mod* pre,
                                 const top_mod* post, void* stream);

/* Loss of Eq. 7 averaged over the batch, L = mean_b (1 - |O_b|^2), from the overlaps of
 * top_propagate_overlap (device double[2 batch]) into loss (device double[1]); when grad is
 * non-NULL also dL/dpsi_b = -(2 / batch) O_b phi_b dx dy (complex64 [batch][ny][nx], the
 * real-loss convention), ready for top_propagate_backward. g gives batch, ny, nx, dy, dx. */
top_status top_overlap_loss(top_handle h, const top_grid* g, const double* overlap, const void* target,
                            int64_t target_stride, double* loss, void* grad, void* stream);

/* L = mean((I - T)^2) over n elements and grad = 2 (I - T) / n (float32, device; grad may be
 * NULL). loss: device double[1]. Deterministic two-stage reduction. */
top_status top_mse_loss(top_handle h, int64_t n, const float* intensity, const float* target, double* loss,
                        float* grad, void* stream);

/* ---------------------------------------------------------------- unequal spacings (§3) */

typedef enum top_interp { TOP_NEAREST = 0, TOP_BILINEAR = 1 } top_interp;

/* A field on g's centred grid (sample i at (i - (n-1)/2) d) interpolated onto the centred grid
 * (ny_out, nx_out, dy_out, dx_out), as the paper does after propagating on the input spacing:
 * output sample j sits at fractional input index u = (j - (n_out-1)/2) d_out / d + (n-1)/2
 * (float64), TOP_NEAREST takes sample floor(u + 1/2), TOP_BILINEAR weighs floor(u) and
 * floor(u) + 1 by 1 - t and t (t = u - floor(u)); samples outside the input grid count as zero.
 * in: complex64 [batch][g->ny][g->nx], out: [batch][ny_out][nx_out] (distinct buffers).
 * backward != 0 applies the transpose (the gradient): in is then [batch][ny_out][nx_out] and
 * out [batch][g->ny][g->nx], each input sample gathering its terms in a fixed order. */
top_status top_resample(top_handle h, const top_grid* g, int ny_out, int nx_out, double dy_out, double dx_out,
                        int mode, int backward, const void* in, void* out, void* stream);

/* ---------------------------------------------------------------- polarisation (§5.1) */

/* Jones-matrix modulation |psi_out(r)> = J(r) |psi_in(r)> of polarised fields with three
 * components (x, y, z). Field index b = (o * 3 + c) * inner + i holds component c of polarised
 * field (o, i): g->batch = 3 * inner * (number of polarised fields); inner = 1 is the
 * [fields][3][ny][nx] layout, inner = W the (object, component, wavelength) order of a
 * polychromatic batch. J: device complex64 [3][3][ny][nx] (spatially varying, row-major
 * matrix index) or NULL, then j_uniform: host double[18], one 3x3 matrix row-major as
 * (re, im) pairs. A 2x2 Jones matrix acts on (x, y) with J_zz = 1 and zero z couplings.
 * in == out allowed. */
top_status top_jones(top_handle h, const top_grid* g, int64_t inner, const void* J, const double* j_uniform,
                     const void* in, void* out, void* stream);

/* Backward of top_jones: grad_in = J^H grad_out per pixel (grad_in may be NULL, must not
 * alias grad_out) and, for spatially varying J only, grad_J = sum over the polarised fields of
 * grad_out conj(saved_in)^T per pixel (device complex64 [3][3][ny][nx], or NULL), summed in
 * field order. */
top_status top_jones_backward(top_handle h, const top_grid* g, int64_t inner, const void* J, const double* j_uniform,
                              const void* saved_in, const void* grad_out, void* grad_in, void* grad_J, void* stream);

/* Jones matrices of the polarisation elements of §5.1 (the polariser, circular polariser and
 * waveplate calls of the paper's polarisation listings), written as the j_uniform argument of
 * top_jones: out is host double[18], one 3x3 matrix row-major as (re, im) pairs, with the 2x2
 * block on (x, y) and J_zz = 1, zero z couplings. Host-only, no device work; out is caller-owned.
 * TOP_ERR_INVALID_ARG for a NULL out or a non-finite angle, out untouched then.
 *   linear polariser, transmission axis at theta to x: J = u u^T, u = (cos theta, sin theta);
 *   circular polariser passing (1, i h)/sqrt 2 (h = +1 or -1): J = v v^H;
 *   waveplate with its fast axis at theta and the given retardance (pi/2 quarter-wave, pi
 *   half-wave): J = u u^T + exp(i retardance) w w^T, w = (-sin theta, cos theta). */
top_status top_jones_linear_polarizer(double theta, double* out);
top_status top_jones_circular_polarizer(int handedness, double* out);
top_status top_jones_waveplate(double retardance, double theta, double* out);

/* Power of every field, sum |psi_b|^2 dx dy (device double[batch]; float64, fixed order). */
top_status top_field_power(top_handle h, const top_grid* g, const void* field, double* power, void* stream);

/* ---------------------------------------------------------------- mutual coherence (§5.2) */

/* Gamma_out = P_z (M(r1) M*(r2) Gamma_in) P_z^H  (Eq. 12 then Eq. 13): h_z acts on
 * (y1, x1) and h_z* on (y2, x2). gamma_in, gamma_out: complex64
 * [batch][ny][nx][ny][nx] device (distinct buffers). mask: M or NULL. lambda, z: host,
 * one value each (shared by the batch). Uses workspace of one Gamma tensor. */
top_status top_propagate_coherence(top_handle h, const top_grid* g, const void* gamma_in, void* gamma_out,
                                   const double* lambda, const double* z, const top_mod* mask, void* stream);

/* Backward of top_propagate_coherence: grad_in = M*(r1) M(r2) (P_z^H G P_z) (grad_in may be
 * NULL) and the gradients of the mask parameters (grads->saved_in = the forward gamma_in). */
top_status top_propagate_coherence_backward(top_handle h, const top_grid* g, const void* grad_out,
                                            void* grad_in, const double* lambda, const double* z,
                                            const top_mod* mask, const top_mod_grads* grads, void* stream);

/* Intensity Gamma(r, r) of each coherence tensor: float32 [batch][ny][nx]. */
top_status top_coherence_intensity(top_handle h, const top_grid* g, const void* gamma, float* intensity,
                                   void* stream);

/* Backward of top_coherence_intensity: grad_gamma = diag(grad_I) (all other elements 0). */
top_status top_coherence_intensity_backward(top_handle h, const top_grid* g, const float* grad_intensity,
                                            void* grad_gamma, void* stream);

/* ---------------------------------------------------------------- autotuning */

/* Pass variants the autotuner chooses between, per line length M = P/2 (flags 0: the defaults).
 * Row passes of M (the x axis) read the row bits, the column pass of M (the y axis) the column
 * bit. TOP_TUNE_CLASSIC_*: the block-cooperative row kernels instead of the pair-local ones (plans
 * of one warp a half line at padding 2); TOP_TUNE_NO_L2_*: no L2 prefetch of the next wave's
 * inputs; bits 8-10 (TOP_TUNE_SPAN): fields per block of the inverse row pass with a field
 * epilogue, c -> 2^(c - 1) (0: 4); TOP_TUNE_THREE_PASS (read for M = 64): fields of 64 x 64 at
 * padding 2 go through the three passes and the workspace instead of the one-kernel on-chip
 * propagation (plain propagations: no modulation, a field epilogue). */
#define TOP_TUNE_CLASSIC_FWD 0x1u
#define TOP_TUNE_CLASSIC_INV 0x2u
#define TOP_TUNE_CLASSIC_CHAIN 0x4u
#define TOP_TUNE_NO_L2_COLS 0x8u
#define TOP_TUNE_NO_L2_FWD 0x10u
#define TOP_TUNE_SPAN(c) ((uint32_t)(c) << 8)
#define TOP_TUNE_THREE_PASS 0x800u

/* Measure the pass variants on g's geometry (padded sizes with a plan of their own; g->batch
 * fields of scratch, allocated and freed by the call -- 16 or more fields at 1024^2 give passes
 * long enough to time) with CUDA events, keep for every pass kind the fastest, and record the
 * choices in the process-wide table for Px/2 (row bits) and Py/2 (column bit). Synchronises the
 * device. rows_flags / cols_flags (may be NULL) receive the entries written. */
top_status top_autotune(top_handle h, const top_grid* g, uint32_t* rows_flags, uint32_t* cols_flags);
/* The process-wide table, host-only: set, get (0 when absent), clear. Invalid flags:
 * TOP_ERR_INVALID_ARG. */
top_status top_autotune_set(int line_length, uint32_t flags);
top_status top_autotune_get(int line_length, uint32_t* flags);
top_status top_autotune_clear(void);
/* Write the table to a text file (a header line, one "M flags" line per entry, and a line with
 * the FNV-1a checksum of everything before it), or replace the table by a file's contents. A
 * missing, truncated, altered or malformed file is refused with TOP_ERR_INVALID_ARG and leaves
 * the table unchanged. The first top_create of a process loads the file named by the environment
 * variable TOP_AUTOTUNE_CACHE, if set (a refused file leaves the defaults, and the handle is
 * created all the same). */
top_status top_autotune_save(const char* path);
top_status top_autotune_load(const char* path);

/* ---------------------------------------------------------------- instrumentation */

/* Enable (1) or disable (0) CUDA-event timing of every kernel launched by the handle. */
top_status top_profile_enable(top_handle h, int enable);
/* Drain the recorded events (synchronising on them) and return per-kind totals.
 * kinds (up to `cap` entries) get static names, ms the summed milliseconds and count the
 * launches since the last call; *n receives the number of kinds written. The kinds are
 * "rows_fwd" (forward row passes), "cols" (column passes), "rows_inv" (inverse row passes),
 * "aux" (losses, reductions, modulations and the other auxiliary kernels) and "rows_chain"
 * (the fused inverse-and-forward row passes between the stages of a system chain). */
top_status top_profile_read(top_handle h, int cap, const char** kinds, double* ms, int64_t* count, int* n);

#ifdef __cplusplus
}
#endif

#endif /* TOP_H_ */
