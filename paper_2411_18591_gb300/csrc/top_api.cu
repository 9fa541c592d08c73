// C ABI of the propagation library: handle, argument validation, float64 table
// caches, workspace management and the launch sequence of each call.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <complex>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <utility>
#include <vector>

#include "top_aux.h"
#include "top_dispatch.h"
#include "top_internal.h"

using namespace top;

// ============================================================================= errors

namespace {

thread_local std::string t_last_error;

top_status fail(top_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_last_error = buf;
  return s;
}

top_status cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? TOP_ERR_OOM : TOP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define TOP_CUDA(call, what)                         \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

#define TOP_TRY(call)                    \
  do {                                   \
    top_status s_ = (call);              \
    if (s_ != TOP_OK) return s_;         \
  } while (0)

uint64_t bits(double d) {
  uint64_t u;
  std::memcpy(&u, &d, sizeof u);
  return u;
}

}  // namespace

// ============================================================================= handle

struct TransferEntry {
  float2* hq = nullptr;
};

// Bluestein tables of one line length P (CztParams): convolution length L = 2M, chirp, chirp
// transforms split by parity, M-point engine twiddles, split twiddles of L.
struct CztPlan {
  int L = 0;
  const float2* chirp = nullptr;
  const float2* bh_fwd = nullptr;  // halves in the M-point engine's slot order
  const float2* bh_inv = nullptr;
  const float2* tw = nullptr;
  const float2* wsplit = nullptr;
};

struct top_ctx {
  int device = 0;
  uint64_t ws_limit = 8ull << 30;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  void* coh = nullptr;  // one coherence tensor of scratch for the transposes
  size_t coh_bytes = 0;
  void* chain = nullptr;  // the intermediate fields of a chain at a padded size without a plan
  size_t chain_bytes = 0;
  void* cohg = nullptr;  // the coherence backward's G' when the caller wants no grad_in
  size_t cohg_bytes = 0;
  std::vector<void*> allocs;  // cached tables, freed with the handle
  std::map<int, float2*> eng_tw;
  std::map<int, float2*> split_tw;
  std::map<std::array<uint64_t, 7>, TransferEntry> transfer;
  std::map<std::array<uint64_t, 4>, float2*> lens;
  std::map<std::array<uint64_t, 5>, int2*> circ;
  std::map<int, CztPlan> czt;                               // Bluestein tables per line length
  std::map<std::array<uint64_t, 7>, float2*> transfer_full;  // natural-order H for Bluestein columns
  // instrumentation
  bool prof = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  std::vector<cudaEvent_t> pool;
  double prof_ms[KK_COUNT] = {};
  long long prof_cnt[KK_COUNT] = {};
};

namespace {

top_status bind(top_handle h) {
  TOP_CUDA(cudaSetDevice(h->device), "cudaSetDevice");
  return TOP_OK;
}

template <class T>
top_status upload(top_handle h, const std::vector<T>& host, T** out) {
  void* p = nullptr;
  TOP_CUDA(cudaMalloc(&p, std::max<size_t>(sizeof(T), host.size() * sizeof(T))), "cudaMalloc(table)");
  h->allocs.push_back(p);
  if (!host.empty()) TOP_CUDA(cudaMemcpy(p, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice), "cudaMemcpy(table)");
  *out = static_cast<T*>(p);
  return TOP_OK;
}

top_status ensure_workspace(top_handle h, size_t bytes) {
  if (bytes <= h->ws_bytes) return TOP_OK;
  if (h->ws) {
    TOP_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize(workspace growth)");
    cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_bytes = 0;
  }
  const size_t rounded = (bytes + (1u << 20) - 1) & ~size_t((1u << 20) - 1);
  cudaError_t e = cudaMalloc(&h->ws, rounded);
  if (e != cudaSuccess) {
    h->ws = nullptr;
    return cuda_fail(e, "cudaMalloc(workspace)");
  }
  h->ws_bytes = rounded;
  return TOP_OK;
}

cudaEvent_t take_event(top_handle h) {
  if (!h->pool.empty()) {
    cudaEvent_t e = h->pool.back();
    h->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Launch with optional CUDA-event timing on the launching stream.
template <class F>
top_status timed(top_handle h, int kind, cudaStream_t st, const char* what, F&& launch) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (h->prof) {
    a = take_event(h);
    b = take_event(h);
    cudaEventRecord(a, st);
  }
  cudaError_t e = launch();
  if (h->prof) {
    cudaEventRecord(b, st);
    h->pending.push_back({kind, {a, b}});
  }
  if (e != cudaSuccess) return cuda_fail(e, what);
  return TOP_OK;
}

// ============================================================================= engines and tables

bool find_engine(int M, EngineInfo* info) {
  return engine_info_small(M, info) || engine_info_mid(M, info) || engine_info_m1024(M, info) ||
         engine_info_large(M, info) || engine_info_mixed(M, info);
}

cudaError_t launch_pass(int kind, int M, const PassParams& p, cudaStream_t s, const PassParams* next = nullptr) {
  bool found = false;
  cudaError_t e = launch_pass_small(kind, M, p, next, s, &found);
  if (found) return e;
  e = launch_pass_mid(kind, M, p, next, s, &found);
  if (found) return e;
  e = launch_pass_m1024(kind, M, p, next, s, &found);
  if (found) return e;
  e = launch_pass_large(kind, M, p, next, s, &found);
  if (found) return e;
  e = launch_pass_mixed(kind, M, p, next, s, &found);
  if (found) return e;
  return cudaErrorInvalidValue;
}

// Bluestein line pass with convolution length L: one L-point engine up to 4096, two halves on the
// 4096-point engine for 8192.
cudaError_t launch_czt_pass(int L, const CztParams& p, cudaStream_t s) {
  bool found = false;
  cudaError_t e;
  if (L > 4096) {
    e = launch_czt_split_large(L / 2, p, s, &found);
    return found ? e : cudaErrorInvalidValue;
  }
  e = launch_czt_small(L, p, s, &found);
  if (found) return e;
  e = launch_czt_mid(L, p, s, &found);
  if (found) return e;
  e = launch_czt_m1024(L, p, s, &found);
  if (found) return e;
  e = launch_czt_large(L, p, s, &found);
  if (found) return e;
  return cudaErrorInvalidValue;
}

// Fields of a repeat group (input_repeat) share one source when the source modulation does not
// depend on the wavelength: no lens, and masks shared by the batch.
bool shared_source(const top_mod* m) {
  return !m || m->flags == 0 || (!(m->flags & TOP_MOD_LENS) && m->batch_stride == 0);
}

// The forward half of a propagation whose fields come in repeat groups with one source each: R1
// and the forward column transforms run once per source (these parameters) into `spec`, then every
// field's column pass starts from its source's spectrum (H of its own wavelength, inverse, crop),
// with the same results as R1 and the column pass per field.
PassParams source_params(const PassParams& p, int repeat, float2* spec) {
  PassParams ps = p;
  ps.nfields = p.nfields / repeat;
  ps.in_repeat = 1;
  for (int s = 0; s < ps.nfields; ++s) ps.set_of[s] = p.set_of[s * repeat];
  ps.spec_out = spec;
  return ps;
}

// (cos, sin) of pi * x for a float64 x, with x reduced modulo 2 exactly (fmod is exact).
void cis_pi(double x, double* c, double* s) {
  double r = std::fmod(x, 2.0);
  if (r > 1.0) r -= 2.0;
  if (r < -1.0) r += 2.0;
  *c = std::cos(M_PI * r);
  *s = std::sin(M_PI * r);
}

// exp(-2 pi i m / n) for integers, m reduced modulo n first
float2 unit_root(long long m, long long n) {
  m %= n;
  if (m < 0) m += n;
  double c, s;
  cis_pi(-2.0 * double(m) / double(n), &c, &s);
  return make_float2(float(c), float(s));
}

// Stage twiddles w_{R SP}^{i j} of an engine plan, in the layout the device reads.
top_status engine_twiddles(top_handle h, int M, const float2** out) {
  auto it = h->eng_tw.find(M);
  if (it != h->eng_tw.end()) {
    *out = it->second;
    return TOP_OK;
  }
  EngineInfo info;
  if (!find_engine(M, &info)) return fail(TOP_ERR_UNSUPPORTED, "no FFT engine for line length %d", M);
  std::vector<float2> tw(std::max(1, info.tw_size));
  size_t off = 0;
  for (int s = 0; s < info.NS; ++s) {
    int sp = 1;
    for (int i = s + 1; i < info.NS; ++i) sp *= info.R[i];
    if (sp <= 1) continue;
    const int r = info.R[s], L = r * sp;
    for (int j = 1; j < r; ++j)
      for (int i = 0; i < sp; ++i) tw[off + size_t(j - 1) * sp + i] = unit_root((long long)i * j, L);
    off += size_t(r - 1) * sp;
  }
  if ((int)off > std::max(1, info.tw_size)) return fail(TOP_ERR_INTERNAL, "twiddle table size mismatch");
  float2* d = nullptr;
  TOP_TRY(upload(h, tw, &d));
  h->eng_tw[M] = d;
  *out = d;
  return TOP_OK;
}

// exp(-2 pi i p / P) for p < P / 2: the twiddles that fold and unfold the two halves.
top_status split_twiddles(top_handle h, int P, const float2** out) {
  auto it = h->split_tw.find(P);
  if (it != h->split_tw.end()) {
    *out = it->second;
    return TOP_OK;
  }
  std::vector<float2> w(P / 2);
  for (int p = 0; p < P / 2; ++p) w[p] = unit_root(p, P);
  float2* d = nullptr;
  TOP_TRY(upload(h, w, &d));
  h->split_tw[P] = d;
  *out = d;
  return TOP_OK;
}

long long signed_index(long long k, long long P) { return k < (P + 1) / 2 ? k : k - P; }
double freq(long long k, long long P, double d) { return double(signed_index(k, P)) / (double(P) * d); }

// Direct Integration table: the forward 2-D DFT of h_z (Eq. 3) sampled at the padded grid's signed
// lags (times dx dy), divided by Py Px, into the quadrant layout (h_z is even in x and y, so its
// transform is too). The samples are taken in float64 and transformed by the library's own row
// pass and a forward-only column pass, through temporary buffers freed before returning.
top_status di_table(top_handle h, int Py, int Px, double dy, double dx, double lam, double z, cudaStream_t st,
                    float2* hq) {
  const float2 *twx, *twy, *wpx, *wpy;
  TOP_TRY(engine_twiddles(h, Px / 2, &twx));
  TOP_TRY(engine_twiddles(h, Py / 2, &twy));
  TOP_TRY(split_twiddles(h, Px, &wpx));
  TOP_TRY(split_twiddles(h, Py, &wpy));
  const size_t plane = size_t(Py) * size_t(Px);
  void* buf = nullptr;
  TOP_CUDA(cudaMalloc(&buf, 2 * plane * sizeof(float2)), "cudaMalloc(DI kernel samples)");
  float2* samples = static_cast<float2*>(buf);
  float2* ws = samples + plane;
  PassParams p{};
  p.ny = Py;
  p.nx = Px;
  p.Py = Py;
  p.Px = Px;
  p.My = Py / 2;
  p.Mx = Px / 2;
  p.method = TOP_DI;
  p.src_kind = SRC_FIELD;
  p.epi_kind = EPI_FIELD;
  p.in = samples;
  p.in_stride = (long long)plane;
  p.in_repeat = 1;
  p.ws = ws;
  p.ws_stride = (long long)plane;
  p.twx = twx;
  p.twy = twy;
  p.wpx = wpx;
  p.wpy = wpy;
  p.nfields = 1;
  p.nsets = 1;
  p.group = 1;
  p.src_group = 1;
  p.hq_out = hq;
  p.hq_scale = float(1.0 / (double(Py) * double(Px)));
  cudaError_t e = launch_di_samples(samples, Py, Px, dy, dx, lam, z, st);
  if (e == cudaSuccess) e = launch_pass(PASS_ROWS_FWD, Px / 2, p, st);
  if (e == cudaSuccess) e = launch_pass(PASS_COLS, Py / 2, p, st);
  const cudaError_t es = cudaStreamSynchronize(st);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_fail(e, "DI table");
  if (es != cudaSuccess) return cuda_fail(es, "cudaStreamSynchronize(DI table)");
  return TOP_OK;
}

// Quadrant table of the transfer function for one (lambda, z) (Eq. 5 and the Fresnel form),
// built in float64 on the device on first use and cached; the build is waited for, so later
// calls on any stream may read it.
top_status transfer_tables(top_handle h, int Py, int Px, double dy, double dx, double lam, double z, int method,
                           cudaStream_t st, TransferEntry* out) {
  const std::array<uint64_t, 7> key = {uint64_t(Py), uint64_t(Px), bits(dy), bits(dx), bits(lam), bits(z),
                                       uint64_t(method)};
  auto it = h->transfer.find(key);
  if (it != h->transfer.end()) {
    *out = it->second;
    return TOP_OK;
  }
  TransferEntry te;
  void* p = nullptr;
  TOP_CUDA(cudaMalloc(&p, size_t(Px / 2 + 1) * size_t(Py / 2 + 2) * sizeof(float2)), "cudaMalloc(transfer table)");
  h->allocs.push_back(p);
  te.hq = static_cast<float2*>(p);
  if (method == TOP_DI) {
    TOP_TRY(di_table(h, Py, Px, dy, dx, lam, z, st, te.hq));
  } else {
    TOP_CUDA(launch_transfer_table(te.hq, Py, Px, dy, dx, lam, z, method, st), "transfer table");
  }
  TOP_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize(transfer table)");
  h->transfer[key] = te;
  *out = te;
  return TOP_OK;
}

// The method of one field: TOP_AUTO picks AS below z_critical (Eq. 6, the smaller of the two
// axes' n d^2 / lambda) and DI above it.
int resolve_method(const top_grid* g, int ny, int nx, double lam, double z) {
  if (g->method != TOP_AUTO) return g->method;
  const double zc = std::min(double(nx) * g->dx * g->dx / lam, double(ny) * g->dy * g->dy / lam);
  return z < zc ? TOP_AS : TOP_DI;
}

// Transfer table of one field with its method resolved and the DI conditions checked.
top_status field_transfer(top_handle h, const top_grid* g, int ny, int nx, int Py, int Px, double lam, double z,
                          cudaStream_t st, TransferEntry* te) {
  const int m = resolve_method(g, ny, nx, lam, z);
  if (m == TOP_DI) {
    if (Py < 2 * ny - 1 || Px < 2 * nx - 1)
      return fail(TOP_ERR_INVALID_ARG, "DI needs padded sizes >= 2 n - 1 (got %dx%d for %dx%d; pad >= 2)", Py, Px, ny, nx);
    if (!(z > 0)) return fail(TOP_ERR_INVALID_ARG, "DI needs z > 0 (got %g)", z);
  }
  return transfer_tables(h, Py, Px, g->dy, g->dx, lam, z, m, st, te);
}

// Thin-lens factor table exp(-i pi s^2 / (lambda f)) along one axis (s = (i - (n-1)/2) d).
top_status lens_table(top_handle h, int n, double d, double lam, double f, const float2** out) {
  const std::array<uint64_t, 4> key = {uint64_t(n), bits(d), bits(lam), bits(f)};
  auto it = h->lens.find(key);
  if (it != h->lens.end()) {
    *out = it->second;
    return TOP_OK;
  }
  std::vector<float2> t(n);
  for (int i = 0; i < n; ++i) {
    const double s = (double(i) - double(n - 1) / 2.0) * d;
    double c, sn;
    cis_pi(-(s * s) / (lam * f), &c, &sn);
    t[i] = make_float2(float(c), float(sn));
  }
  float2* dp = nullptr;
  TOP_TRY(upload(h, t, &dp));
  h->lens[key] = dp;
  *out = dp;
  return TOP_OK;
}

// Circular aperture: per row the inclusive x range with x^2 + y^2 <= R^2 (float64, pixel centres).
top_status circ_table(top_handle h, int ny, int nx, double dy, double dx, double R, const int2** out) {
  const std::array<uint64_t, 5> key = {uint64_t(ny), uint64_t(nx), bits(dy), bits(dx), bits(R)};
  auto it = h->circ.find(key);
  if (it != h->circ.end()) {
    *out = it->second;
    return TOP_OK;
  }
  std::vector<int2> t(ny);
  const double r2 = R * R;
  for (int j = 0; j < ny; ++j) {
    const double yv = (double(j) - double(ny - 1) / 2.0) * dy;
    const double y2 = yv * yv;
    int lo = nx, hi = -1;
    for (int i = 0; i < nx; ++i) {
      const double xv = (double(i) - double(nx - 1) / 2.0) * dx;
      if (xv * xv + y2 <= r2) {
        lo = std::min(lo, i);
        hi = std::max(hi, i);
      }
    }
    t[j] = make_int2(lo, hi);
  }
  int2* dp = nullptr;
  TOP_TRY(upload(h, t, &dp));
  h->circ[key] = dp;
  *out = dp;
  return TOP_OK;
}

// ============================================================================= validation

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

struct Geometry {
  int ny, nx, Py, Px, oy, ox;
};

top_status padded(int n, double pad, int* P) {
  const double v = std::floor(pad * double(n) + 0.5);
  if (!(v >= double(n)) || v > 1048576.0) return fail(TOP_ERR_INVALID_ARG, "padded size %.0f invalid for n = %d", v, n);
  *P = int(v);
  return TOP_OK;
}

top_status check_grid(const top_grid* g, Geometry* geo) {
  if (!g) return fail(TOP_ERR_INVALID_ARG, "grid is NULL");
  if (g->batch < 1) return fail(TOP_ERR_INVALID_ARG, "batch must be >= 1 (got %lld)", (long long)g->batch);
  if (g->ny < 1 || g->nx < 1) return fail(TOP_ERR_INVALID_ARG, "ny, nx must be >= 1 (got %d, %d)", g->ny, g->nx);
  if (!(std::isfinite(g->dy) && g->dy > 0) || !(std::isfinite(g->dx) && g->dx > 0))
    return fail(TOP_ERR_INVALID_ARG, "spacing must be finite and > 0");
  if (!(std::isfinite(g->pad) && g->pad >= 1.0)) return fail(TOP_ERR_INVALID_ARG, "pad must be finite and >= 1");
  if (g->method != TOP_AS && g->method != TOP_FRESNEL_TF && g->method != TOP_DI && g->method != TOP_AUTO)
    return fail(TOP_ERR_INVALID_ARG, "unknown method %d", g->method);
  if (g->input_repeat < 0 || (g->input_repeat > 1 && g->batch % g->input_repeat != 0))
    return fail(TOP_ERR_INVALID_ARG, "input_repeat (%d) must be 0, 1 or a divisor of batch", g->input_repeat);
  geo->ny = g->ny;
  geo->nx = g->nx;
  TOP_TRY(padded(g->ny, g->pad, &geo->Py));
  TOP_TRY(padded(g->nx, g->pad, &geo->Px));
  geo->oy = (geo->Py - g->ny) / 2;
  geo->ox = (geo->Px - g->nx) / 2;
  return TOP_OK;
}

bool has_engines(const Geometry& geo) {
  EngineInfo info;
  for (int P : {geo.Py, geo.Px})
    if (P % 2 != 0 || !find_engine(P / 2, &info)) return false;
  return true;
}

top_status check_engines(const Geometry& geo) {
  if (!has_engines(geo))
    return fail(TOP_ERR_UNSUPPORTED,
                "padded size %d x %d has no FFT plan of its own (planned: 2 x {16 .. 4096 powers of two, 250, 500, 768, "
                "1000}); other sizes up to 4096 go through Bluestein transforms, which do not take this call",
                geo.Py, geo.Px);
  return TOP_OK;
}

top_status check_lz(const top_grid* g, const double* lam, const double* z, int64_t n_lz, bool need_z) {
  if (!lam || (need_z && !z)) return fail(TOP_ERR_INVALID_ARG, "lambda / z arrays are NULL");
  if (n_lz != 1 && n_lz != g->batch)
    return fail(TOP_ERR_INVALID_ARG, "n_lz must be 1 or batch (%lld), got %lld", (long long)g->batch, (long long)n_lz);
  for (int64_t i = 0; i < n_lz; ++i) {
    if (!(std::isfinite(lam[i]) && lam[i] > 0)) return fail(TOP_ERR_INVALID_ARG, "lambda[%lld] must be finite and > 0", (long long)i);
    if (need_z && !std::isfinite(z[i])) return fail(TOP_ERR_INVALID_ARG, "z[%lld] must be finite", (long long)i);
  }
  return TOP_OK;
}

top_status check_ptr(const void* p, const char* name) {
  if (!p) return fail(TOP_ERR_INVALID_ARG, "%s is NULL", name);
  if (!aligned16(p)) return fail(TOP_ERR_INVALID_ARG, "%s is not 16-byte aligned", name);
  return TOP_OK;
}

top_status check_mod(const top_mod* m, const char* name) {
  if (!m || m->flags == 0) return TOP_OK;
  const uint32_t all = TOP_MOD_COMPLEX | TOP_MOD_AMPLITUDE | TOP_MOD_PHASE | TOP_MOD_LENS | TOP_MOD_CIRC;
  if (m->flags & ~all) return fail(TOP_ERR_INVALID_ARG, "%s: unknown modulation flags 0x%x", name, m->flags);
  if ((m->flags & TOP_MOD_COMPLEX)) TOP_TRY(check_ptr(m->mask, "modulation mask"));
  if ((m->flags & TOP_MOD_AMPLITUDE)) TOP_TRY(check_ptr(m->amplitude, "modulation amplitude"));
  if ((m->flags & TOP_MOD_PHASE)) TOP_TRY(check_ptr(m->phase, "modulation phase"));
  if ((m->flags & TOP_MOD_LENS) && !(std::isfinite(m->focal_length) && m->focal_length != 0.0))
    return fail(TOP_ERR_INVALID_ARG, "%s: focal length must be finite and non-zero", name);
  if ((m->flags & TOP_MOD_CIRC) && !(std::isfinite(m->radius) && m->radius >= 0.0))
    return fail(TOP_ERR_INVALID_ARG, "%s: aperture radius must be finite and >= 0", name);
  if (m->batch_stride < 0) return fail(TOP_ERR_INVALID_ARG, "%s: batch_stride must be >= 0", name);
  return TOP_OK;
}

ModDev mod_dev(const top_mod* m, int conj, const int2* circ) {
  ModDev d{};
  if (!m) return d;
  d.flags = m->flags;
  d.conj = conj;
  d.cmask = static_cast<const float2*>(m->mask);
  d.amp = m->amplitude;
  d.phase = m->phase;
  d.stride = m->batch_stride;
  d.circ = circ;
  return d;
}

// Per-field masks (batch_stride != 0) are addressed relative to the first field of a launch.
ModDev offset_mod(ModDev d, long long pos) {
  if (d.stride) {
    if (d.cmask) d.cmask += pos * d.stride;
    if (d.amp) d.amp += pos * d.stride;
    if (d.phase) d.phase += pos * d.stride;
  }
  return d;
}

// ============================================================================= propagation driver

struct Request {
  const top_grid* g;
  const double* lam;
  const double* z;
  int64_t n_lz;
  int adjoint;
  int src_kind;
  const void* in;
  const void* psi_src;  // SRC_INTENSITY saved field
  const float* gI;
  const float* weights;
  int64_t group;  // intensity group (SRC_INTENSITY / EPI_INTENSITY)
  const top_mod* msrc;
  int msrc_conj;
  int epi_kind;
  void* out;
  float* outf;
  const top_mod* mepi;
  int mepi_conj;
  const top_mod_grads* grads;  // EPI_MODGRAD
  const void* target;          // EPI_OVERLAP: phi, shared (target_stride 0) or per field
  int64_t target_stride;
  double* ov_out;              // EPI_OVERLAP: [2 batch] overlaps, [batch] powers (may be null)
  double* pw_out;
  // upstream adjoint stages of a fused backward chain, run before this propagation: stage j
  // propagates by up[j].z with conj(H) (up[0] starts from this request's source), then its field
  // is multiplied by conj(up[j].pre) and enters stage j + 1, the last one this propagation (whose
  // own source modulation is then null); each boundary is one fused row pass
  const top_stage* up;
  int n_up;
};

// A scratch buffer owned by the handle, grown on demand (the previous contents are not kept).
top_status grow_scratch(void** buf, size_t* have, size_t bytes, const char* what) {
  if (*have < bytes) {
    if (*buf) {
      TOP_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize(scratch growth)");
      cudaFree(*buf);
      *buf = nullptr;
      *have = 0;
    }
    cudaError_t e = cudaMalloc(buf, bytes);
    if (e != cudaSuccess) {
      *buf = nullptr;
      return cuda_fail(e, what);
    }
    *have = bytes;
  }
  return TOP_OK;
}

// One field-sized (or coherence-tensor-sized) scratch buffer per handle.
top_status coh_scratch(top_handle h, size_t bytes, void** out) {
  TOP_TRY(grow_scratch(&h->coh, &h->coh_bytes, bytes, "cudaMalloc(coherence scratch)"));
  *out = h->coh;
  return TOP_OK;
}

// ============================================================================= Bluestein path

// In-place radix-2 FFT in float64, X[k] = sum_n x[n] exp(-2 pi i n k / L), L a power of two.
void host_fft(std::vector<std::complex<double>>& a) {
  const size_t L = a.size();
  for (size_t i = 1, j = 0; i < L; ++i) {
    size_t bit = L >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  for (size_t len = 2; len <= L; len <<= 1) {
    for (size_t k = 0; k < len / 2; ++k) {
      double c, sn;
      cis_pi(-2.0 * double(k) / double(len), &c, &sn);
      const std::complex<double> w(c, sn);
      for (size_t i = 0; i < L; i += len) {
        const std::complex<double> u = a[i + k], v = a[i + k + len / 2] * w;
        a[i + k] = u + v;
        a[i + k + len / 2] = u - v;
      }
    }
  }
}

// The frequency bin that lane t of an engine holds in slot e after its forward transform (the
// engine's digit-reversed output order): slot e = q RL + j holds bin kbase(t + G q) + j M / RL, where
// kbase gathers the digits of stages 0 .. NS-2 of the position (t + G q) RL.
int engine_bin(const EngineInfo& info, int t, int e) {
  const int NS = info.NS, RL = info.R[NS - 1];
  auto span = [&](int s) {
    int p = 1;
    for (int i = s + 1; i < NS; ++i) p *= info.R[i];
    return p;
  };
  auto weight = [&](int s) {
    int p = 1;
    for (int i = 0; i < s; ++i) p *= info.R[i];
    return p;
  };
  const int q = e / RL, j = e % RL, b = t + info.G * q;
  int k = 0;
  for (int s = 0; s < NS - 1; ++s) k += ((b / (span(s) / RL)) % info.R[s]) * weight(s);
  return k + j * (info.M / RL);
}

// Tables of the Bluestein transforms of length P: c[n] = exp(-i pi n^2 / P) with n^2 reduced
// modulo 2 P in integers (exact), and the L-point transforms of conj(c) and c on the lags
// (-P, P) wrapped modulo L, in float64, rounded once.
top_status czt_plan(top_handle h, int P, CztPlan* out) {
  auto it = h->czt.find(P);
  if (it != h->czt.end()) {
    *out = it->second;
    return TOP_OK;
  }
  int L = 16;
  while (L < 2 * P - 1) L *= 2;
  if (L > 8192)
    return fail(TOP_ERR_UNSUPPORTED, "padded size %d has no FFT plan and is above the 4096 points of the Bluestein "
                "transforms", P);
  std::vector<float2> chirp(P);
  std::vector<std::complex<double>> bf(L), bi(L);
  for (int n = 0; n < P; ++n) {
    const unsigned long long r = ((unsigned long long)n * (unsigned long long)n) % (2ull * (unsigned long long)P);
    double c, sn;
    cis_pi(-double(r) / double(P), &c, &sn);
    chirp[n] = make_float2(float(c), float(sn));
    bf[n] = std::complex<double>(c, -sn);
    bi[n] = std::complex<double>(c, sn);
    if (n > 0) {
      bf[L - n] = bf[n];
      bi[L - n] = bi[n];
    }
  }
  host_fft(bf);
  host_fft(bi);
  // in the slot order of the engine that runs the transforms, so a warp reads consecutive entries
  // (entry e G + t holds the bin lane t keeps in slot e after the forward transform): the L-point
  // engine, or for L = 8192 the 4096-point one with the table split by parity (half r holds the
  // bins 2k + r, at r M)
  const bool split = L > 4096;
  const int M = split ? L / 2 : L;
  EngineInfo info;
  if (!find_engine(M, &info)) return fail(TOP_ERR_INTERNAL, "no %d-point engine for the Bluestein transforms", M);
  std::vector<float2> hf(L), hi(L);
  const int E = M / info.G;
  for (int r = 0; r < (split ? 2 : 1); ++r)
    for (int t = 0; t < info.G; ++t)
      for (int e = 0; e < E; ++e) {
        const int k = split ? 2 * engine_bin(info, t, e) + r : engine_bin(info, t, e);
        hf[size_t(r) * M + size_t(e) * info.G + t] = make_float2(float(bf[k].real()), float(bf[k].imag()));
        hi[size_t(r) * M + size_t(e) * info.G + t] = make_float2(float(bi[k].real()), float(bi[k].imag()));
      }
  CztPlan plan;
  plan.L = L;
  float2 *dc = nullptr, *df = nullptr, *di = nullptr;
  TOP_TRY(upload(h, chirp, &dc));
  TOP_TRY(upload(h, hf, &df));
  TOP_TRY(upload(h, hi, &di));
  plan.chirp = dc;
  plan.bh_fwd = df;
  plan.bh_inv = di;
  TOP_TRY(engine_twiddles(h, M, &plan.tw));
  if (split) TOP_TRY(split_twiddles(h, L, &plan.wsplit));
  h->czt[P] = plan;
  *out = plan;
  return TOP_OK;
}

// H / (Py Px) on the whole grid in natural order, one row per kx (cached per parameter set).
top_status transfer_full_table(top_handle h, int Py, int Px, double dy, double dx, double lam, double z, int method,
                               cudaStream_t st, const float2** out) {
  const std::array<uint64_t, 7> key = {uint64_t(Py), uint64_t(Px), bits(dy), bits(dx), bits(lam), bits(z),
                                       uint64_t(method)};
  auto it = h->transfer_full.find(key);
  if (it != h->transfer_full.end()) {
    *out = it->second;
    return TOP_OK;
  }
  void* p = nullptr;
  TOP_CUDA(cudaMalloc(&p, size_t(Px) * size_t(Py) * sizeof(float2)), "cudaMalloc(transfer table)");
  h->allocs.push_back(p);
  float2* tab = static_cast<float2*>(p);
  if (method == TOP_DI) {
    // DI: the sampled kernel h_z dx dy at the grid's signed lags, forward-transformed by Bluestein
    // rows, a transpose and Bluestein columns into [kx][ky], divided by Py Px
    CztPlan cx, cy;
    TOP_TRY(czt_plan(h, Px, &cx));
    TOP_TRY(czt_plan(h, Py, &cy));
    const size_t plane = size_t(Py) * size_t(Px);
    void* buf = nullptr;
    TOP_CUDA(cudaMalloc(&buf, 2 * plane * sizeof(float2)), "cudaMalloc(DI kernel samples)");
    float2* a = static_cast<float2*>(buf);
    float2* b = a + plane;
    CztParams r{};
    r.mode = CZT_FWD;
    r.in = a;
    r.in_fstride = (long long)plane;
    r.in_lstride = Px;
    r.in_repeat = 1;
    r.out = b;
    r.out_fstride = (long long)plane;
    r.out_lstride = Px;
    r.nlines = Py;
    r.nfields = 1;
    r.P = Px;
    r.n_in = Px;
    r.off_in = 0;
    r.k0 = 0;
    r.n_out = Px;
    r.inv_l = float(1.0 / double(cx.L));
    r.chirp = cx.chirp;
    r.bh_fwd = cx.bh_fwd;
    r.bh_inv = cx.bh_inv;
    r.tw = cx.tw;
    r.wsplit = cx.wsplit;
    CztParams c = r;
    c.in = a;
    c.in_lstride = Py;
    c.out = tab;
    c.out_lstride = Py;
    c.nlines = Px;
    c.P = Py;
    c.n_in = Py;
    c.n_out = Py;
    c.inv_l = float(1.0 / (double(cy.L) * double(Py) * double(Px)));
    c.chirp = cy.chirp;
    c.bh_fwd = cy.bh_fwd;
    c.bh_inv = cy.bh_inv;
    c.tw = cy.tw;
    c.wsplit = cy.wsplit;
    cudaError_t e = launch_di_samples(a, Py, Px, dy, dx, lam, z, st);
    if (e == cudaSuccess) e = launch_czt_pass(cx.L, r, st);
    if (e == cudaSuccess) e = launch_transpose_rect(b, a, 1, Py, Px, st);
    if (e == cudaSuccess) e = launch_czt_pass(cy.L, c, st);
    const cudaError_t es = cudaStreamSynchronize(st);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(e, "DI table");
    if (es != cudaSuccess) return cuda_fail(es, "cudaStreamSynchronize(DI table)");
  } else {
    TOP_CUDA(launch_transfer_full(tab, Py, Px, dy, dx, lam, z, method, st), "transfer table");
    TOP_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize(transfer table)");
  }
  h->transfer_full[key] = tab;
  *out = tab;
  return TOP_OK;
}

// Lens tables of fields [pos, pos + n) as the parameter sets of one modulation launch.
top_status fill_lens_sets(top_handle h, const top_grid* g, const top_mod* mod, const double* lambda,
                                 int64_t n_lz, int64_t pos, int64_t n, PassParams* p) {
  p->nsets = 0;
  for (int64_t b = pos; b < pos + n; ++b) {
    FieldSet fs{};
    if (mod->flags & TOP_MOD_LENS) {
      const double lam = lambda[n_lz == 1 ? 0 : b];
      TOP_TRY(lens_table(h, g->nx, g->dx, lam, mod->focal_length, &fs.src_lx));
      TOP_TRY(lens_table(h, g->ny, g->dy, lam, mod->focal_length, &fs.src_ly));
    }
    fs.epi_lx = fs.src_lx;
    fs.epi_ly = fs.src_ly;
    int k = 0;
    while (k < p->nsets && std::memcmp(&p->sets[k], &fs, sizeof fs) != 0) ++k;
    if (k == p->nsets) {
      if (p->nsets == kMaxSets) return fail(TOP_ERR_INTERNAL, "lens set overflow");
      p->sets[p->nsets++] = fs;
    }
    p->set_of[b - pos] = (unsigned char)k;
  }
  return TOP_OK;
}

// out[f] = M_f in[f / repeat] (conj(M_f) with conj) for fields [pos, pos + n) of a call.
top_status modulate_fields(top_handle h, const top_grid* g, const Geometry& geo, const top_mod* mod, int conj,
                           const double* lam, int64_t n_lz, int64_t pos, int64_t n, const float2* in, int repeat,
                           float2* out, cudaStream_t st) {
  const int2* circ = nullptr;
  if (mod->flags & TOP_MOD_CIRC) TOP_TRY(circ_table(h, geo.ny, geo.nx, g->dy, g->dx, mod->radius, &circ));
  const ModDev base = mod_dev(mod, conj, circ);
  const long long plane = (long long)geo.ny * geo.nx;
  for (int64_t c = 0; c < n; c += kMaxSets) {
    const int64_t m = std::min<int64_t>(kMaxSets, n - c);
    PassParams p{};
    p.ny = geo.ny;
    p.nx = geo.nx;
    TOP_TRY(fill_lens_sets(h, g, mod, lam, n_lz, pos + c, m, &p));
    p.nfields = int(m);
    p.msrc = offset_mod(base, pos + c);
    // a repeat group never straddles the chunks of kMaxSets fields when repeat divides them
    p.in_repeat = repeat;
    p.in = in + (repeat > 1 ? c / repeat : c) * plane;
    p.out = out + c * plane;
    TOP_TRY(timed(h, KK_AUX, st, "modulate", [&] { return launch_modulate(p, st); }));
  }
  return TOP_OK;
}

// A field-to-field propagation (modulations before and after as separate passes) whose padded
// size has no plan of its own (odd, or with prime factors above 5), up to 4096 points per axis:
// rows by Bluestein forward transforms, a transpose, each column's forward transform, H and
// inverse transform in one Bluestein line pass, a transpose back and the rows' inverse
// transforms with the crop.
top_status bluestein_fields(top_handle h, const Request& q, const Geometry& geo, cudaStream_t st) {
  const top_grid* g = q.g;
  const int64_t B = g->batch;
  const long long plane = (long long)geo.ny * geo.nx;
  const int repeat = g->input_repeat > 1 ? g->input_repeat : 1;
  CztPlan cx, cy;
  TOP_TRY(czt_plan(h, geo.Px, &cx));
  TOP_TRY(czt_plan(h, geo.Py, &cy));
  std::vector<const float2*> tables(B);
  for (int64_t b = 0; b < B; ++b) {
    const double lam = q.lam[q.n_lz == 1 ? 0 : b], z = q.z[q.n_lz == 1 ? 0 : b];
    const int method = resolve_method(g, geo.ny, geo.nx, lam, z);
    if (method == TOP_DI) {
      if (geo.Py < 2 * geo.ny - 1 || geo.Px < 2 * geo.nx - 1)
        return fail(TOP_ERR_INVALID_ARG, "DI needs padded sizes >= 2 n - 1 (got %dx%d for %dx%d; pad >= 2)", geo.Py,
                    geo.Px, geo.ny, geo.nx);
      if (!(z > 0)) return fail(TOP_ERR_INVALID_ARG, "DI needs z > 0 (got %g)", z);
    }
    TOP_TRY(transfer_full_table(h, geo.Py, geo.Px, g->dy, g->dx, lam, z, method, st, &tables[b]));
  }
  const long long wplane = (long long)geo.ny * geo.Px;
  const bool pre = q.msrc && q.msrc->flags;
  const bool post = q.mepi && q.mepi->flags;
  const size_t per_field = sizeof(float2) * size_t(2 * wplane + (pre ? plane : 0)) + sizeof(void*);
  int64_t chunk = std::max<int64_t>(1, int64_t((h->ws_limit > 4096 ? h->ws_limit - 4096 : 0) / per_field));
  chunk = std::min<int64_t>({chunk, B, 65535});
  if (repeat > 1) {
    // whole repeat groups per chunk, and per modulation launch (kMaxSets fields)
    if (pre && kMaxSets % repeat != 0)
      return fail(TOP_ERR_UNSUPPORTED, "input_repeat %d with a source modulation on a Bluestein size needs a divisor "
                  "of %d", repeat, kMaxSets);
    chunk = std::max<int64_t>(repeat, chunk - chunk % repeat);
  }
  TOP_TRY(ensure_workspace(h, size_t(chunk) * (per_field - sizeof(void*)) + 256 + size_t(chunk) * sizeof(void*)));
  float2* w1 = static_cast<float2*>(h->ws);
  float2* w2 = w1 + chunk * wplane;
  float2* src = w2 + chunk * wplane;
  char* tail = reinterpret_cast<char*>(w1) + size_t(chunk) * (per_field - sizeof(void*));
  tail = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(tail) + 255) & ~uintptr_t(255));
  const float2** d_h = reinterpret_cast<const float2**>(tail);
  const float2* in = static_cast<const float2*>(q.in);
  float2* out = static_cast<float2*>(q.out);
  for (int64_t pos = 0; pos < B; pos += chunk) {
    const int64_t n = std::min<int64_t>(chunk, B - pos);
    const float2* fin = in + (pos / repeat) * plane;
    int in_rep = repeat;
    if (pre) {
      TOP_TRY(modulate_fields(h, g, geo, q.msrc, q.msrc_conj, q.lam, q.n_lz, pos, n, fin, repeat, src, st));
      fin = src;
      in_rep = 1;
    }
    TOP_CUDA(cudaMemcpyAsync(d_h, tables.data() + pos, size_t(n) * sizeof(void*), cudaMemcpyHostToDevice, st),
             "cudaMemcpyAsync(transfer table pointers)");
    CztParams r{};
    r.mode = CZT_FWD;
    r.in = fin;
    r.in_fstride = plane;
    r.in_lstride = geo.nx;
    r.in_repeat = in_rep;
    r.out = w1;
    r.out_fstride = wplane;
    r.out_lstride = geo.Px;
    r.nlines = geo.ny;
    r.nfields = int(n);
    r.P = geo.Px;
    r.n_in = geo.nx;
    r.off_in = geo.ox;
    r.k0 = 0;
    r.n_out = geo.Px;
    r.inv_l = 1.f / float(cx.L);
    r.chirp = cx.chirp;
    r.bh_fwd = cx.bh_fwd;
    r.bh_inv = cx.bh_inv;
    r.tw = cx.tw;
    r.wsplit = cx.wsplit;
    TOP_TRY(timed(h, KK_ROWS_FWD, st, "Bluestein rows", [&] { return launch_czt_pass(cx.L, r, st); }));
    TOP_TRY(timed(h, KK_AUX, st, "transpose", [&] { return launch_transpose_rect(w1, w2, n, geo.ny, geo.Px, st); }));
    CztParams c{};
    c.mode = CZT_FILTER;
    c.adjoint = q.adjoint;
    c.in = w2;
    c.in_fstride = wplane;
    c.in_lstride = geo.ny;
    c.in_repeat = 1;
    c.out = w2;
    c.out_fstride = wplane;
    c.out_lstride = geo.ny;
    c.nlines = geo.Px;
    c.nfields = int(n);
    c.P = geo.Py;
    c.n_in = geo.ny;
    c.off_in = geo.oy;
    c.k0 = geo.oy;
    c.n_out = geo.ny;
    c.inv_l = 1.f / float(cy.L);
    c.chirp = cy.chirp;
    c.bh_fwd = cy.bh_fwd;
    c.bh_inv = cy.bh_inv;
    c.tw = cy.tw;
    c.wsplit = cy.wsplit;
    c.h = d_h;
    TOP_TRY(timed(h, KK_COLS, st, "Bluestein columns", [&] { return launch_czt_pass(cy.L, c, st); }));
    TOP_TRY(timed(h, KK_AUX, st, "transpose", [&] { return launch_transpose_rect(w2, w1, n, geo.Px, geo.ny, st); }));
    CztParams v = r;
    v.mode = CZT_INV;
    v.in = w1;
    v.in_fstride = wplane;
    v.in_lstride = geo.Px;
    v.in_repeat = 1;
    v.out = out + pos * plane;
    v.out_fstride = plane;
    v.out_lstride = geo.nx;
    v.n_in = geo.Px;
    v.off_in = 0;
    v.k0 = geo.ox;
    v.n_out = geo.nx;
    TOP_TRY(timed(h, KK_ROWS_INV, st, "Bluestein inverse rows", [&] { return launch_czt_pass(cx.L, v, st); }));
    if (post)
      TOP_TRY(modulate_fields(h, g, geo, q.mepi, q.mepi_conj, q.lam, q.n_lz, pos, n, out + pos * plane, 1,
                              out + pos * plane, st));
  }
  return TOP_OK;
}

// The propagation calls at padded sizes without a plan of their own: the intensity backward's
// source (2 w gI psi), the detector intensity (Eq. 14) and the overlap sums (Eq. 7) run as
// separate passes around bluestein_fields, and modulation gradients follow the adjoint
// propagation through the modulation's own backward.
top_status run_bluestein(top_handle h, const Request& q, const Geometry& geo, cudaStream_t st) {
  const top_grid* g = q.g;
  TOP_TRY(bind(h));
  const int64_t B = g->batch;
  const long long plane = (long long)geo.ny * geo.nx;
  const bool need_src = q.src_kind == SRC_INTENSITY;
  const bool need_field = q.epi_kind == EPI_MODGRAD || ((q.epi_kind == EPI_INTENSITY || q.epi_kind == EPI_OVERLAP) && !q.out);
  constexpr int kOvTiles = 64;  // partial sums per field of the overlap (fixed order)
  const size_t ov_bytes = q.epi_kind == EPI_OVERLAP ? sizeof(double) * 3 * kOvTiles * size_t(B) : 0;
  float2* scratch = nullptr;
  if (need_src || need_field || ov_bytes) {
    void* p = nullptr;
    TOP_TRY(coh_scratch(h, sizeof(float2) * size_t(B) * size_t(plane) * size_t(int(need_src) + int(need_field)) + ov_bytes,
                        &p));
    scratch = static_cast<float2*>(p);
  }
  float2* src_buf = scratch;
  float2* field_buf = need_src ? scratch + B * plane : scratch;
  Request r = q;
  if (need_src) {
    TOP_TRY(timed(h, KK_AUX, st, "intensity source", [&] {
      return launch_intensity_source(static_cast<const float2*>(q.psi_src), q.gI, q.weights, int(q.group), B, plane,
                                     src_buf, st);
    }));
    r.src_kind = SRC_FIELD;
    r.in = src_buf;
  }
  if (q.epi_kind == EPI_FIELD) return bluestein_fields(h, r, geo, st);
  if (q.epi_kind == EPI_MODGRAD) {
    // the adjoint propagation into a scratch field, then the modulation's own backward (input
    // gradient conj(M) g and the parameter gradients from the saved input)
    r.epi_kind = EPI_FIELD;
    r.out = field_buf;
    r.mepi = nullptr;
    r.grads = nullptr;
    TOP_TRY(bluestein_fields(h, r, geo, st));
    return top_modulate_backward(h, g, q.mepi, field_buf, q.out, q.grads, q.lam, q.n_lz, st);
  }
  // EPI_INTENSITY / EPI_OVERLAP: the (modulated) field, kept in field_out when given, then the
  // group sums of Eq. 14 or the overlaps and powers of Eq. 7
  float2* field = q.out ? static_cast<float2*>(q.out) : field_buf;
  r.epi_kind = EPI_FIELD;
  r.out = field;
  TOP_TRY(bluestein_fields(h, r, geo, st));
  if (q.epi_kind == EPI_INTENSITY)
    return timed(h, KK_AUX, st, "intensity", [&] {
      return launch_intensity_sum(field, q.weights, int(q.group), B / q.group, plane, q.outf, st);
    });
  double* part = reinterpret_cast<double*>(scratch + B * plane * (int(need_src) + int(need_field)));
  TOP_TRY(timed(h, KK_AUX, st, "overlap partial sums", [&] {
    return launch_overlap_partials(field, static_cast<const float2*>(q.target), q.target_stride, B, plane, kOvTiles,
                                   part, st);
  }));
  return timed(h, KK_AUX, st, "overlap sums", [&] {
    return launch_overlap_finish(part, kOvTiles, int(B), g->dy * g->dx, q.ov_out, q.pw_out, st);
  });
}

top_status run_propagation(top_handle h, const Request& q, cudaStream_t st);

// Whether every boundary of a request's upstream stages runs as one fused row pass: the next
// stage's source operands fit the fused kernel's shared memory (as in run_chain).
bool upstream_fuses(const Geometry& geo, const Request& q) {
  EngineInfo ex;
  if (!find_engine(geo.Px / 2, &ex)) return false;
  for (int j = 0; j < q.n_up; ++j) {
    PassParams probe{};
    probe.nx = geo.nx;
    probe.src_kind = SRC_FIELD;
    probe.msrc = mod_dev(q.up[j].pre, 1, nullptr);
    const size_t planes = src_plane_floats(probe, ex.rows);
    const size_t rows_end = sizeof(float2) * (size_t(2) * ex.rows * ex.M + size_t(ex.rows) * geo.nx);
    const size_t bytes = std::max(rows_end, ex.row_smem) + sizeof(float) * planes;
    if (!((planes == 0 || geo.nx % 4 == 0) && bytes <= kChainSmemMax)) return false;
  }
  return true;
}

// The upstream stages of a request one propagation at a time through a field-sized scratch (sizes
// without a plan of their own, or boundaries that do not fuse), then the request itself; the same
// results as the fused passes.
top_status run_upstream_unfused(top_handle h, const Request& q, cudaStream_t st) {
  const int64_t B = q.g->batch;
  const size_t plane = size_t(q.g->ny) * size_t(q.g->nx);
  TOP_TRY(grow_scratch(&h->chain, &h->chain_bytes, sizeof(float2) * size_t(B) * plane, "cudaMalloc(chain scratch)"));
  void* tmp = h->chain;
  for (int j = 0; j < q.n_up; ++j) {
    const std::vector<double> zj(size_t(q.n_lz), q.up[j].z);
    Request r{};
    r.g = q.g; r.lam = q.lam; r.z = zj.data(); r.n_lz = q.n_lz; r.adjoint = 1;
    if (j == 0) {
      r.src_kind = q.src_kind; r.in = q.in; r.psi_src = q.psi_src; r.gI = q.gI; r.group = q.group;
      r.weights = q.weights;
    } else {
      r.src_kind = SRC_FIELD; r.in = tmp; r.group = 1;
      r.msrc = q.up[j - 1].pre; r.msrc_conj = 1;
    }
    r.epi_kind = EPI_FIELD; r.out = tmp;
    TOP_TRY(run_propagation(h, r, st));
  }
  Request m = q;
  m.up = nullptr; m.n_up = 0;
  m.src_kind = SRC_FIELD; m.in = tmp; m.psi_src = nullptr; m.gI = nullptr; m.weights = nullptr; m.group = 1;
  m.msrc = q.up[q.n_up - 1].pre; m.msrc_conj = 1;
  return run_propagation(h, m, st);
}

top_status run_propagation(top_handle h, const Request& q, cudaStream_t st) {
  const top_grid* g = q.g;
  Geometry geo;
  TOP_TRY(check_grid(g, &geo));
  const bool planned = has_engines(geo);
  TOP_TRY(check_lz(g, q.lam, q.z, q.n_lz, true));
  TOP_TRY(check_mod(q.msrc, "source modulation"));
  TOP_TRY(check_mod(q.mepi, "epilogue modulation"));
  const int64_t B = g->batch;
  if (q.adjoint && g->input_repeat > 1) return fail(TOP_ERR_INVALID_ARG, "input_repeat applies to forward calls only");
  if (g->input_repeat > 1 && q.in && q.in == q.out)
    return fail(TOP_ERR_INVALID_ARG, "input_repeat > 1 needs distinct input and output buffers");
  if (q.src_kind == SRC_FIELD) TOP_TRY(check_ptr(q.in, "input field"));
  if (q.src_kind == SRC_INTENSITY) {
    TOP_TRY(check_ptr(q.psi_src, "saved field"));
    TOP_TRY(check_ptr(q.gI, "intensity gradient"));
  }
  if (q.group < 1 || B % q.group != 0)
    return fail(TOP_ERR_INVALID_ARG, "group (%lld) must be >= 1 and divide batch (%lld)", (long long)q.group, (long long)B);
  if (q.group > kMaxFields) return fail(TOP_ERR_UNSUPPORTED, "group larger than %d fields", kMaxFields);
  if (q.weights && !aligned16(q.weights)) return fail(TOP_ERR_INVALID_ARG, "weights not 16-byte aligned");
  if (q.epi_kind == EPI_FIELD) TOP_TRY(check_ptr(q.out, "output field"));
  if (q.epi_kind == EPI_INTENSITY) {
    TOP_TRY(check_ptr(q.outf, "intensity"));
    if (q.out) TOP_TRY(check_ptr(q.out, "field output"));
  }
  if (q.epi_kind == EPI_OVERLAP) {
    TOP_TRY(check_ptr(q.target, "target"));
    if (q.target_stride != 0 && q.target_stride != (int64_t)geo.ny * geo.nx)
      return fail(TOP_ERR_INVALID_ARG, "target_stride must be 0 (shared) or ny * nx (per field)");
    if (!q.ov_out || (reinterpret_cast<uintptr_t>(q.ov_out) & 7u) || (reinterpret_cast<uintptr_t>(q.pw_out) & 7u))
      return fail(TOP_ERR_INVALID_ARG, "overlap must be a non-NULL, 8-byte aligned device array (power too when given)");
    if (q.out) TOP_TRY(check_ptr(q.out, "field output"));
  }
  const top_mod_grads* gr = q.grads;
  const bool want_pgrads = q.epi_kind == EPI_MODGRAD && gr && (gr->grad_phase || gr->grad_amplitude || gr->grad_mask);
  if (q.epi_kind == EPI_MODGRAD) {
    if (q.out) TOP_TRY(check_ptr(q.out, "grad_in"));
    if (want_pgrads) {
      TOP_TRY(check_ptr(gr->saved_in, "pre_grads->saved_in"));
      if (!q.mepi || q.mepi->flags == 0) return fail(TOP_ERR_INVALID_ARG, "modulation gradients need a modulation");
      if (gr->grad_phase && !(q.mepi->flags & TOP_MOD_PHASE)) return fail(TOP_ERR_INVALID_ARG, "grad_phase needs TOP_MOD_PHASE");
      if (gr->grad_amplitude && !(q.mepi->flags & TOP_MOD_AMPLITUDE)) return fail(TOP_ERR_INVALID_ARG, "grad_amplitude needs TOP_MOD_AMPLITUDE");
      if (gr->grad_mask && !(q.mepi->flags & TOP_MOD_COMPLEX)) return fail(TOP_ERR_INVALID_ARG, "grad_mask needs TOP_MOD_COMPLEX");
      for (const void* p : {(const void*)gr->grad_phase, (const void*)gr->grad_amplitude, (const void*)gr->grad_mask})
        if (p && !aligned16(p)) return fail(TOP_ERR_INVALID_ARG, "gradient output not 16-byte aligned");
    }
  }
  if (q.n_up > 0) {
    if (!q.adjoint || q.msrc) return fail(TOP_ERR_INTERNAL, "upstream stages need an adjoint request without a source modulation");
    for (int j = 0; j < q.n_up; ++j) {
      if (!std::isfinite(q.up[j].z)) return fail(TOP_ERR_INVALID_ARG, "stage %d: z must be finite", j);
      TOP_TRY(check_mod(q.up[j].pre, "stage modulation"));
    }
    if (!planned || !upstream_fuses(geo, q)) return run_upstream_unfused(h, q, st);
  }
  if (!planned) return run_bluestein(h, q, geo, st);
  TOP_TRY(bind(h));

  // engine and split twiddles
  const float2 *twx, *twy, *wpx, *wpy;
  TOP_TRY(engine_twiddles(h, geo.Px / 2, &twx));
  TOP_TRY(engine_twiddles(h, geo.Py / 2, &twy));
  TOP_TRY(split_twiddles(h, geo.Px, &wpx));
  TOP_TRY(split_twiddles(h, geo.Py, &wpy));
  const int2* circ_src = nullptr;
  const int2* circ_epi = nullptr;
  if (q.msrc && (q.msrc->flags & TOP_MOD_CIRC)) TOP_TRY(circ_table(h, geo.ny, geo.nx, g->dy, g->dx, q.msrc->radius, &circ_src));
  if (q.mepi && (q.mepi->flags & TOP_MOD_CIRC)) TOP_TRY(circ_table(h, geo.ny, geo.nx, g->dy, g->dx, q.mepi->radius, &circ_epi));

  // per-field parameter sets (the source-side lens tables of this propagation belong to its
  // source modulation, or with upstream stages to the last boundary's)
  const top_mod* src_mod = q.n_up > 0 ? q.up[q.n_up - 1].pre : q.msrc;
  std::vector<FieldSet> field_sets(B);
  for (int64_t b = 0; b < B; ++b) {
    const int64_t i = q.n_lz == 1 ? 0 : b;
    TransferEntry te;
    TOP_TRY(field_transfer(h, g, geo.ny, geo.nx, geo.Py, geo.Px, q.lam[i], q.z[i], st, &te));
    FieldSet fs{};
    fs.hq = te.hq;
    if (src_mod && (src_mod->flags & TOP_MOD_LENS)) {
      TOP_TRY(lens_table(h, geo.nx, g->dx, q.lam[i], src_mod->focal_length, &fs.src_lx));
      TOP_TRY(lens_table(h, geo.ny, g->dy, q.lam[i], src_mod->focal_length, &fs.src_ly));
    }
    if (q.mepi && (q.mepi->flags & TOP_MOD_LENS)) {
      TOP_TRY(lens_table(h, geo.nx, g->dx, q.lam[i], q.mepi->focal_length, &fs.epi_lx));
      TOP_TRY(lens_table(h, geo.ny, g->dy, q.lam[i], q.mepi->focal_length, &fs.epi_ly));
    }
    field_sets[b] = fs;
  }
  // upstream stages: stage j's transfer table and the lens tables of the boundary modulation its
  // forward row pass applies (none for the first, which starts from the request's source)
  std::vector<std::vector<FieldSet>> up_sets(size_t(q.n_up), std::vector<FieldSet>(B));
  std::vector<const int2*> up_circ(size_t(q.n_up), nullptr);
  for (int j = 0; j < q.n_up; ++j) {
    const top_mod* bm = j > 0 ? q.up[j - 1].pre : nullptr;
    if (q.up[j].pre && (q.up[j].pre->flags & TOP_MOD_CIRC))
      TOP_TRY(circ_table(h, geo.ny, geo.nx, g->dy, g->dx, q.up[j].pre->radius, &up_circ[j]));
    for (int64_t b = 0; b < B; ++b) {
      const int64_t i = q.n_lz == 1 ? 0 : b;
      TransferEntry te;
      TOP_TRY(field_transfer(h, g, geo.ny, geo.nx, geo.Py, geo.Px, q.lam[i], q.up[j].z, st, &te));
      FieldSet fs{};
      fs.hq = te.hq;
      if (bm && (bm->flags & TOP_MOD_LENS)) {
        TOP_TRY(lens_table(h, geo.nx, g->dx, q.lam[i], bm->focal_length, &fs.src_lx));
        TOP_TRY(lens_table(h, geo.ny, g->dy, q.lam[i], bm->focal_length, &fs.src_ly));
      }
      up_sets[j][b] = fs;
    }
  }
  if (q.n_up > 0 && q.msrc == nullptr && src_mod && (src_mod->flags & TOP_MOD_CIRC))
    TOP_TRY(circ_table(h, geo.ny, geo.nx, g->dy, g->dx, src_mod->radius, &circ_src));
  auto same_one = [](const FieldSet& a, const FieldSet& b) { return std::memcmp(&a, &b, sizeof(FieldSet)) == 0; };
  // fields share a parameter-set slot when every stage's set agrees
  auto same_field = [&](int64_t a, int64_t b) {
    if (!same_one(field_sets[a], field_sets[b])) return false;
    for (int j = 0; j < q.n_up; ++j)
      if (!same_one(up_sets[j][a], up_sets[j][b])) return false;
    return true;
  };

  // epilogue grouping and workspace
  const long long plane = (long long)geo.ny * geo.nx;
  const bool shared_mask = q.mepi && q.mepi->batch_stride == 0;
  int64_t group = 1;
  if (q.epi_kind == EPI_INTENSITY) group = q.group;
  const bool partials = want_pgrads && shared_mask;
  const int rows_per_cta_guess = 8;
  if (partials) {
    const int64_t tiles = (geo.ny + rows_per_cta_guess - 1) / rows_per_cta_guess;
    const int64_t want_groups = std::max<int64_t>(1, (4 * 152 + tiles - 1) / tiles);
    group = std::max<int64_t>(1, (B + want_groups - 1) / want_groups);
  }
  // plain propagations of 64 x 64 fields at padding 2 run as one on-chip kernel (no workspace)
  const bool onchip = geo.Py == 128 && geo.Px == 128 && geo.ny == 64 && geo.nx == 64 && q.n_up == 0 &&
                      q.src_kind == SRC_FIELD && !(q.msrc && q.msrc->flags) && q.epi_kind == EPI_FIELD &&
                      !(q.mepi && q.mepi->flags) && !(tune_flags(geo.Px / 2) & TOP_TUNE_THREE_PASS);
  const size_t ws_field = onchip ? 0 : size_t(geo.Px) * size_t(geo.ny) * sizeof(float2);
  EngineInfo ex_info;
  find_engine(geo.Px / 2, &ex_info);
  const int ntiles = (geo.ny + ex_info.rows - 1) / ex_info.rows;  // R2 row tiles (overlap partial sums)
  size_t part_bytes_per_group = 0;
  if (q.epi_kind == EPI_OVERLAP) part_bytes_per_group = size_t(ntiles) * 3 * sizeof(double);
  if (partials) {
    if (gr->grad_phase) part_bytes_per_group += plane * sizeof(float);
    if (gr->grad_amplitude) part_bytes_per_group += plane * sizeof(float);
    if (gr->grad_mask) part_bytes_per_group += plane * sizeof(float2);
  }
  // chunk: a multiple of every grouping (intensity planes never straddle chunks), <= kMaxFields,
  // workspace within the limit
  const int64_t src_group = q.src_kind == SRC_INTENSITY ? q.group : 1;
  const int64_t epi_align = q.epi_kind == EPI_INTENSITY ? group : 1;
  const int64_t in_repeat = (q.src_kind == SRC_FIELD && g->input_repeat > 1) ? g->input_repeat : 1;
  const int64_t align = std::lcm(std::lcm(src_group, epi_align), in_repeat);
  if (align > kMaxFields) return fail(TOP_ERR_UNSUPPORTED, "intensity group larger than %d fields", kMaxFields);
  int64_t chunk = std::min<int64_t>(B, kMaxFields);
  chunk = std::max<int64_t>(align, chunk - chunk % align);
  // broadcast sources: one forward spectrum per source (Px x Py samples) after the partials
  const bool share = q.src_kind == SRC_FIELD && in_repeat > 1 && shared_source(q.msrc) && !onchip;
  const size_t spec_src = share ? size_t(geo.Px) * size_t(geo.Py) * sizeof(float2) : 0;
  auto need = [&](int64_t c) {
    const int64_t ng = (c + group - 1) / group;
    return size_t(c) * ws_field + size_t(ng) * part_bytes_per_group + 256 + size_t(c / in_repeat) * spec_src + 256;
  };
  while (chunk > align && need(chunk) > h->ws_limit) chunk = std::max<int64_t>(align, (chunk / 2) - (chunk / 2) % align);
  if (need(chunk) > h->ws_limit)
    return fail(TOP_ERR_OOM, "one group of fields needs %zu bytes of workspace, above the limit %llu", need(chunk),
                (unsigned long long)h->ws_limit);
  TOP_TRY(ensure_workspace(h, need(chunk)));
  float2* ws = static_cast<float2*>(h->ws);
  char* part_base = reinterpret_cast<char*>(h->ws) + size_t(chunk) * ws_field;
  part_base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(part_base) + 255) & ~uintptr_t(255));
  const int64_t ngroups_chunk = (chunk + group - 1) / group;
  float2* spec = nullptr;
  if (share) {
    char* sb = part_base + size_t(ngroups_chunk) * part_bytes_per_group;
    spec = reinterpret_cast<float2*>((reinterpret_cast<uintptr_t>(sb) + 255) & ~uintptr_t(255));
  }
  float* part_phase = nullptr;
  float* part_amp = nullptr;
  float2* part_mask = nullptr;
  if (partials) {
    // chunks may hold different numbers of groups (the parameter-set limit can end a chunk early),
    // so the partial planes start at zero and every chunk adds to them
    char* pb = part_base;
    if (gr->grad_phase) { part_phase = reinterpret_cast<float*>(pb); pb += ngroups_chunk * plane * sizeof(float); }
    if (gr->grad_amplitude) { part_amp = reinterpret_cast<float*>(pb); pb += ngroups_chunk * plane * sizeof(float); }
    if (gr->grad_mask) { part_mask = reinterpret_cast<float2*>(pb); pb += ngroups_chunk * plane * sizeof(float2); }
    TOP_CUDA(cudaMemsetAsync(part_base, 0, size_t(pb - part_base), st), "cudaMemsetAsync(gradient partials)");
  }

  PassParams p{};
  p.ny = geo.ny;
  p.nx = geo.nx;
  p.Py = geo.Py;
  p.Px = geo.Px;
  p.My = geo.Py / 2;
  p.Mx = geo.Px / 2;
  p.oy = geo.oy;
  p.ox = geo.ox;
  p.tune_rows = tune_flags(geo.Px / 2);
  p.tune_cols = tune_flags(geo.Py / 2);
  p.method = g->method;
  p.adjoint = q.adjoint;
  p.src_kind = q.src_kind;
  p.epi_kind = q.epi_kind;
  p.twx = twx;
  p.twy = twy;
  p.wpx = wpx;
  p.wpy = wpy;
  const ModDev msrc_base = q.n_up > 0 ? mod_dev(src_mod, 1, circ_src) : mod_dev(q.msrc, q.msrc_conj, circ_src);
  const ModDev mepi_base = mod_dev(q.mepi, q.mepi_conj, circ_epi);
  p.ws = ws;
  p.ws_stride = (long long)geo.Px * geo.ny;
  p.in_stride = plane;
  p.out_stride = plane;
  p.psi_stride = plane;
  p.xs_stride = plane;
  p.gI_stride = plane;
  p.outf_stride = plane;
  p.part_stride = plane;

  std::vector<PassParams> pu(size_t(q.n_up));
  int64_t pos = 0;
  while (pos < B) {
    // grow the chunk field by field while the distinct parameter sets fit (one representative
    // field per set)
    int64_t n = 0;
    p.nsets = 0;
    std::vector<int64_t> rep;
    while (pos + n < B && n < chunk) {
      // a whole aligned group of fields at a time
      int64_t gend = std::min<int64_t>(B, pos + n + align);
      std::vector<int64_t> rep2 = rep;
      unsigned char idx_tmp[kMaxFields];
      bool ok = true;
      for (int64_t b = pos + n; b < gend; ++b) {
        size_t k = 0;
        while (k < rep2.size() && !same_field(rep2[k], b)) ++k;
        if (k == rep2.size()) {
          if ((int)rep2.size() == kMaxSets) { ok = false; break; }
          rep2.push_back(b);
        }
        idx_tmp[b - pos - n] = (unsigned char)k;
      }
      if (!ok) break;
      rep = rep2;
      std::memcpy(p.set_of + n, idx_tmp, size_t(gend - pos - n));
      n = gend - pos;
    }
    p.nsets = int(rep.size());
    for (size_t k = 0; k < rep.size(); ++k) p.sets[k] = field_sets[rep[k]];
    if (n == 0) return fail(TOP_ERR_UNSUPPORTED, "a group of fields uses more than %d (lambda, z) sets", kMaxSets);
    p.nfields = int(n);
    p.group = int(group);
    p.src_group = int(src_group);
    p.in_repeat = int(in_repeat);
    p.msrc = offset_mod(msrc_base, pos);
    p.mepi = offset_mod(mepi_base, pos);
    p.in = q.src_kind == SRC_FIELD ? static_cast<const float2*>(q.in) + (pos / in_repeat) * plane : nullptr;
    p.psi = nullptr;
    if (q.src_kind == SRC_INTENSITY) {
      p.psi = static_cast<const float2*>(q.psi_src) + pos * plane;
      p.gI = q.gI + (pos / q.group) * plane;
    }
    p.weights = q.weights ? q.weights + pos : nullptr;
    p.out = q.out ? static_cast<float2*>(q.out) + pos * plane : nullptr;
    p.outf = q.outf ? q.outf + (pos / group) * plane : nullptr;
    if (q.epi_kind == EPI_MODGRAD) {
      p.xs = want_pgrads ? static_cast<const float2*>(gr->saved_in) + pos * plane : nullptr;
      if (partials) {
        p.part_phase = part_phase;
        p.part_amp = part_amp;
        p.part_mask = part_mask;
        p.part_stride = plane;
        p.part_accumulate = 1;
      } else if (want_pgrads) {  // per-field masks: write straight into the outputs
        p.part_phase = gr->grad_phase ? gr->grad_phase + pos * plane : nullptr;
        p.part_amp = gr->grad_amplitude ? gr->grad_amplitude + pos * plane : nullptr;
        p.part_mask = gr->grad_mask ? static_cast<float2*>(gr->grad_mask) + pos * plane : nullptr;
        p.part_stride = plane;
        p.part_accumulate = 0;
      }
      // partial planes are reused by every chunk (group g of each chunk adds to plane g);
      // per-field gradients use groups of one field
      p.group = partials ? int(group) : 1;
    }
    if (q.n_up > 0) {
      // upstream adjoint stages: the first from this request's source, each boundary (inverse rows
      // of one stage, conj(pre) of its element, forward rows of the next) one fused pass
      for (int j = 0; j < q.n_up; ++j) {
        PassParams& u = pu[j];
        u = p;
        for (size_t k = 0; k < rep.size(); ++k) u.sets[k] = up_sets[j][rep[k]];
        u.epi_kind = EPI_FIELD;
        u.out = nullptr;
        u.outf = nullptr;
        u.mepi = ModDev{};
        u.group = 1;
        u.part_phase = nullptr;
        u.part_amp = nullptr;
        u.part_mask = nullptr;
        u.xs = nullptr;
        if (j > 0) {
          u.src_kind = SRC_FIELD;
          u.msrc = offset_mod(mod_dev(q.up[j - 1].pre, 1, up_circ[j - 1]), pos);
        } else {
          u.msrc = ModDev{};
        }
      }
      TOP_TRY(timed(h, KK_ROWS_FWD, st, "rows forward pass", [&] { return launch_pass(PASS_ROWS_FWD, p.Mx, pu[0], st); }));
      TOP_TRY(timed(h, KK_COLS, st, "column pass", [&] { return launch_pass(PASS_COLS, p.My, pu[0], st); }));
      for (int j = 0; j < q.n_up; ++j) {
        PassParams nxt = j + 1 < q.n_up ? pu[j + 1] : p;
        nxt.src_kind = SRC_FIELD;
        TOP_TRY(timed(h, KK_ROWS_CHAIN, st, "fused row pass",
                      [&] { return launch_pass(PASS_ROWS_CHAIN, p.Mx, pu[j], st, &nxt); }));
        TOP_TRY(timed(h, KK_COLS, st, "column pass", [&] { return launch_pass(PASS_COLS, p.My, nxt, st); }));
      }
    } else if (onchip) {
      if (!onchip_supported(p)) return fail(TOP_ERR_INTERNAL, "on-chip propagation chosen for a request it does not take");
      TOP_TRY(timed(h, KK_ONCHIP, st, "on-chip propagation", [&] { return launch_onchip(p, st); }));
      pos += n;
      continue;
    } else if (share) {
      const PassParams ps = source_params(p, int(in_repeat), spec);
      PassParams pc = p;
      pc.spec_in = spec;
      TOP_TRY(timed(h, KK_ROWS_FWD, st, "rows forward pass (sources)", [&] { return launch_pass(PASS_ROWS_FWD, p.Mx, ps, st); }));
      TOP_TRY(timed(h, KK_COLS, st, "column spectra (sources)", [&] { return launch_pass(PASS_COLS, p.My, ps, st); }));
      TOP_TRY(timed(h, KK_COLS, st, "column pass from spectra", [&] { return launch_pass(PASS_COLS, p.My, pc, st); }));
    } else {
      TOP_TRY(timed(h, KK_ROWS_FWD, st, "rows forward pass", [&] { return launch_pass(PASS_ROWS_FWD, p.Mx, p, st); }));
      TOP_TRY(timed(h, KK_COLS, st, "column pass", [&] { return launch_pass(PASS_COLS, p.My, p, st); }));
    }
    if (q.epi_kind == EPI_OVERLAP) {
      p.target = static_cast<const float2*>(q.target) + pos * q.target_stride;
      p.target_stride = q.target_stride;
      p.ov_part = reinterpret_cast<double*>(part_base);
    }
    TOP_TRY(timed(h, KK_ROWS_INV, st, "rows inverse pass", [&] { return launch_pass(PASS_ROWS_INV, p.Mx, p, st); }));
    if (q.epi_kind == EPI_OVERLAP) {
      TOP_TRY(timed(h, KK_AUX, st, "overlap sums", [&] {
        return launch_overlap_finish(p.ov_part, ntiles, int(n), g->dy * g->dx, q.ov_out + 2 * pos,
                                     q.pw_out ? q.pw_out + pos : nullptr, st);
      }));
    }
    pos += n;
  }
  if (partials) {
    TOP_TRY(timed(h, KK_AUX, st, "gradient reduction", [&] {
      return launch_reduce_partials(part_phase, part_amp, part_mask, int(ngroups_chunk), plane, gr->grad_phase,
                                    gr->grad_amplitude, static_cast<float2*>(gr->grad_mask), st);
    }));
  }
  return TOP_OK;
}

// ============================================================================= fused system chain

// x_0 = in, x_k = P_{z_k}(pre_k x_{k-1}); the inverse row pass of stage k and the forward row
// pass of stage k+1 run as one kernel where the next source's staged planes fit (else the pair
// runs as two launches through `keep` or a field scratch in the workspace, with the same results).
top_status run_chain(top_handle h, const top_grid* g, const void* in, void* out, float* inten, int64_t group,
                     const double* lam, int64_t n_lz, const top_stage* stages, int K, cudaStream_t st) {
  Geometry geo;
  TOP_TRY(check_grid(g, &geo));
  TOP_TRY(check_lz(g, lam, nullptr, n_lz, false));
  if (!stages || K < 1) return fail(TOP_ERR_INVALID_ARG, "a chain needs at least one stage");
  for (int k = 0; k < K; ++k) {
    if (!std::isfinite(stages[k].z)) return fail(TOP_ERR_INVALID_ARG, "stage %d: z must be finite", k);
    TOP_TRY(check_mod(stages[k].pre, "stage modulation"));
    if (stages[k].keep) TOP_TRY(check_ptr(stages[k].keep, "stage keep buffer"));
  }
  if (stages[K - 1].keep) return fail(TOP_ERR_INVALID_ARG, "the last stage's field goes to out; its keep must be NULL");
  const int64_t B = g->batch;
  TOP_TRY(check_ptr(in, "input field"));
  if (!out && !inten) return fail(TOP_ERR_INVALID_ARG, "a chain needs out, intensity or both");
  if (out) TOP_TRY(check_ptr(out, "output field"));
  if (inten) {
    TOP_TRY(check_ptr(inten, "intensity"));
    if (group < 1 || B % group != 0)
      return fail(TOP_ERR_INVALID_ARG, "group (%lld) must be >= 1 and divide batch (%lld)", (long long)group, (long long)B);
    if (group > kMaxFields) return fail(TOP_ERR_UNSUPPORTED, "group larger than %d fields", kMaxFields);
  }
  const int64_t in_repeat = g->input_repeat > 1 ? g->input_repeat : 1;
  if (in_repeat > 1) {
    if (in == out) return fail(TOP_ERR_INVALID_ARG, "input_repeat > 1 needs distinct input and output buffers");
    for (int k = 0; k < K; ++k)
      if (stages[k].keep == in) return fail(TOP_ERR_INVALID_ARG, "input_repeat > 1 needs keep buffers apart from the input");
  }
  TOP_TRY(bind(h));
  if (!has_engines(geo)) {
    // a padded size without a plan of its own: the stages one by one through the Bluestein path,
    // each stage's field to its keep buffer or to one scratch field set (in place from the second
    // stage on), the last stage's to out and the intensity
    for (int P : {geo.Py, geo.Px})
      if (2 * P - 1 > 8192) TOP_TRY(check_engines(geo));
    const long long plane = (long long)geo.ny * geo.nx;
    TOP_TRY(grow_scratch(&h->chain, &h->chain_bytes, sizeof(float2) * size_t(B) * size_t(plane),
                         "cudaMalloc(chain scratch)"));
    float2* tmp = static_cast<float2*>(h->chain);
    const void* cur = in;
    for (int k = 0; k < K; ++k) {
      top_grid gk = *g;
      if (k > 0) gk.input_repeat = 0;
      const std::vector<double> zk(size_t(n_lz), stages[k].z);
      Request q{};
      q.g = &gk; q.lam = lam; q.z = zk.data(); q.n_lz = n_lz; q.adjoint = 0;
      q.src_kind = SRC_FIELD; q.in = cur; q.group = 1;
      q.msrc = stages[k].pre; q.msrc_conj = 0;
      q.epi_kind = EPI_FIELD;
      void* dst = nullptr;
      if (k + 1 < K) {
        dst = stages[k].keep ? stages[k].keep : static_cast<void*>(tmp);
        q.out = dst;
      } else if (inten) {
        q.epi_kind = EPI_INTENSITY; q.out = out; q.outf = inten; q.group = group;
      } else {
        q.out = out;
      }
      TOP_TRY(run_bluestein(h, q, geo, st));
      cur = dst;
    }
    return TOP_OK;
  }

  const float2 *twx, *twy, *wpx, *wpy;
  TOP_TRY(engine_twiddles(h, geo.Px / 2, &twx));
  TOP_TRY(engine_twiddles(h, geo.Py / 2, &twy));
  TOP_TRY(split_twiddles(h, geo.Px, &wpx));
  TOP_TRY(split_twiddles(h, geo.Py, &wpy));
  std::vector<const int2*> circ(K, nullptr);
  for (int k = 0; k < K; ++k)
    if (stages[k].pre && (stages[k].pre->flags & TOP_MOD_CIRC))
      TOP_TRY(circ_table(h, geo.ny, geo.nx, g->dy, g->dx, stages[k].pre->radius, &circ[k]));
  // per stage and field: the transfer table of (lambda, z_k) and the lens tables of pre_k
  std::vector<std::vector<FieldSet>> fsets(K, std::vector<FieldSet>(B));
  for (int k = 0; k < K; ++k) {
    const top_mod* m = stages[k].pre;
    for (int64_t b = 0; b < B; ++b) {
      const int64_t i = n_lz == 1 ? 0 : b;
      TransferEntry te;
      TOP_TRY(field_transfer(h, g, geo.ny, geo.nx, geo.Py, geo.Px, lam[i], stages[k].z, st, &te));
      FieldSet fs{};
      fs.hq = te.hq;
      if (m && (m->flags & TOP_MOD_LENS)) {
        TOP_TRY(lens_table(h, geo.nx, g->dx, lam[i], m->focal_length, &fs.src_lx));
        TOP_TRY(lens_table(h, geo.ny, g->dy, lam[i], m->focal_length, &fs.src_ly));
      }
      fsets[k][b] = fs;
    }
  }
  auto same = [](const FieldSet& a, const FieldSet& b) { return std::memcmp(&a, &b, sizeof(FieldSet)) == 0; };

  // stage boundaries that fuse: the next source's planes fit and are 16-byte rows
  EngineInfo ex;
  find_engine(geo.Px / 2, &ex);
  std::vector<char> fused(K, 0);  // fused[k]: stage k-1 -> k in one kernel
  bool scratch = false;
  for (int k = 1; k < K; ++k) {
    PassParams probe{};
    probe.nx = geo.nx;
    probe.src_kind = SRC_FIELD;
    probe.msrc = mod_dev(stages[k].pre, 0, nullptr);
    const size_t planes = src_plane_floats(probe, ex.rows);
    // the field rows sit past the two half rows, the planes past the rows and the row-pass region
    const size_t rows_end = sizeof(float2) * (size_t(2) * ex.rows * ex.M + size_t(ex.rows) * geo.nx);
    const size_t bytes = std::max(rows_end, ex.row_smem) + sizeof(float) * planes;
    fused[k] = (planes == 0 || geo.nx % 4 == 0) && bytes <= kChainSmemMax;
    if (!fused[k] && !stages[k - 1].keep) scratch = true;
  }

  const long long plane = (long long)geo.ny * geo.nx;
  const int64_t align = std::lcm(inten ? group : int64_t(1), in_repeat);
  if (align > kMaxFields) return fail(TOP_ERR_UNSUPPORTED, "intensity group larger than %d fields", kMaxFields);
  const size_t ws_field = size_t(geo.Px) * size_t(geo.ny) * sizeof(float2);
  const size_t scr_field = scratch ? size_t(plane) * sizeof(float2) : 0;
  const bool share = in_repeat > 1 && shared_source(stages[0].pre);
  const size_t spec_src = share ? size_t(geo.Px) * size_t(geo.Py) * sizeof(float2) : 0;
  int64_t chunk = std::min<int64_t>(B, kMaxFields);
  chunk = std::max<int64_t>(align, chunk - chunk % align);
  auto need = [&](int64_t c) { return size_t(c) * (ws_field + scr_field) + 256 + size_t(c / in_repeat) * spec_src + 256; };
  while (chunk > align && need(chunk) > h->ws_limit) chunk = std::max<int64_t>(align, (chunk / 2) - (chunk / 2) % align);
  if (need(chunk) > h->ws_limit)
    return fail(TOP_ERR_OOM, "one group of fields needs %zu bytes of workspace, above the limit %llu", need(chunk),
                (unsigned long long)h->ws_limit);
  TOP_TRY(ensure_workspace(h, need(chunk)));
  float2* ws = static_cast<float2*>(h->ws);
  float2* scr = scratch ? ws + size_t(chunk) * size_t(geo.Px) * size_t(geo.ny) : nullptr;
  float2* spec = nullptr;
  if (share) {
    char* sb = reinterpret_cast<char*>(h->ws) + size_t(chunk) * (ws_field + scr_field);
    spec = reinterpret_cast<float2*>((reinterpret_cast<uintptr_t>(sb) + 255) & ~uintptr_t(255));
  }

  PassParams base{};
  base.ny = geo.ny;
  base.nx = geo.nx;
  base.Py = geo.Py;
  base.Px = geo.Px;
  base.My = geo.Py / 2;
  base.Mx = geo.Px / 2;
  base.oy = geo.oy;
  base.ox = geo.ox;
  base.tune_rows = tune_flags(geo.Px / 2);
  base.tune_cols = tune_flags(geo.Py / 2);
  base.method = g->method;
  base.src_kind = SRC_FIELD;
  base.epi_kind = EPI_FIELD;
  base.twx = twx;
  base.twy = twy;
  base.wpx = wpx;
  base.wpy = wpy;
  base.ws = ws;
  base.ws_stride = (long long)geo.Px * geo.ny;
  base.in_stride = plane;
  base.out_stride = plane;
  base.psi_stride = plane;
  base.xs_stride = plane;
  base.gI_stride = plane;
  base.outf_stride = plane;
  base.part_stride = plane;
  base.group = 1;
  base.src_group = 1;
  base.in_repeat = 1;

  std::vector<PassParams> ps(K, base);
  int64_t pos = 0;
  while (pos < B) {
    // grow the chunk by aligned groups while the distinct parameter sets fit
    int64_t n = 0;
    std::vector<int64_t> rep;  // a field of each chunk-local set
    unsigned char set_of[kMaxFields];
    while (pos + n < B && n < chunk) {
      const int64_t gend = std::min<int64_t>(B, pos + n + align);
      std::vector<int64_t> rep2 = rep;
      unsigned char idx[kMaxFields];
      bool ok = true;
      for (int64_t b = pos + n; b < gend; ++b) {
        size_t k = 0;
        while (k < rep2.size() && !same(fsets[0][rep2[k]], fsets[0][b])) ++k;
        if (k == rep2.size()) {
          if ((int)rep2.size() == kMaxSets) { ok = false; break; }
          rep2.push_back(b);
        }
        idx[b - pos - n] = (unsigned char)k;
      }
      if (!ok) break;
      rep = rep2;
      std::memcpy(set_of + n, idx, size_t(gend - pos - n));
      n = gend - pos;
    }
    if (n == 0) return fail(TOP_ERR_UNSUPPORTED, "a group of fields uses more than %d (lambda, z) sets", kMaxSets);
    for (int k = 0; k < K; ++k) {
      PassParams& p = ps[k];
      p.nfields = int(n);
      p.nsets = int(rep.size());
      for (size_t q = 0; q < rep.size(); ++q) p.sets[q] = fsets[k][rep[q]];
      std::memcpy(p.set_of, set_of, size_t(n));
      p.msrc = offset_mod(mod_dev(stages[k].pre, 0, circ[k]), pos);
      p.in = nullptr;
      p.in_repeat = 1;
      p.out = stages[k].keep ? static_cast<float2*>(stages[k].keep) + pos * plane : nullptr;
      p.epi_kind = EPI_FIELD;
      p.group = 1;
      p.outf = nullptr;
    }
    ps[0].in = static_cast<const float2*>(in) + (pos / in_repeat) * plane;
    ps[0].in_repeat = int(in_repeat);
    PassParams& last = ps[K - 1];
    last.out = out ? static_cast<float2*>(out) + pos * plane : nullptr;
    if (inten) {
      last.epi_kind = EPI_INTENSITY;
      last.group = int(group);
      last.outf = inten + (pos / group) * plane;
    }
    if (share) {
      const PassParams psrc = source_params(ps[0], int(in_repeat), spec);
      PassParams pc = ps[0];
      pc.spec_in = spec;
      TOP_TRY(timed(h, KK_ROWS_FWD, st, "rows forward pass (sources)", [&] { return launch_pass(PASS_ROWS_FWD, geo.Px / 2, psrc, st); }));
      TOP_TRY(timed(h, KK_COLS, st, "column spectra (sources)", [&] { return launch_pass(PASS_COLS, geo.Py / 2, psrc, st); }));
      TOP_TRY(timed(h, KK_COLS, st, "column pass from spectra", [&] { return launch_pass(PASS_COLS, geo.Py / 2, pc, st); }));
    } else {
      TOP_TRY(timed(h, KK_ROWS_FWD, st, "rows forward pass", [&] { return launch_pass(PASS_ROWS_FWD, geo.Px / 2, ps[0], st); }));
      TOP_TRY(timed(h, KK_COLS, st, "column pass", [&] { return launch_pass(PASS_COLS, geo.Py / 2, ps[0], st); }));
    }
    for (int k = 1; k < K; ++k) {
      if (fused[k]) {
        TOP_TRY(timed(h, KK_ROWS_CHAIN, st, "fused row pass",
                      [&] { return launch_pass(PASS_ROWS_CHAIN, geo.Px / 2, ps[k - 1], st, &ps[k]); }));
      } else {
        // two launches through the kept field or the scratch
        PassParams pa = ps[k - 1], pb = ps[k];
        if (!pa.out) pa.out = scr;
        pb.in = pa.out;
        TOP_TRY(timed(h, KK_ROWS_INV, st, "rows inverse pass", [&] { return launch_pass(PASS_ROWS_INV, geo.Px / 2, pa, st); }));
        TOP_TRY(timed(h, KK_ROWS_FWD, st, "rows forward pass", [&] { return launch_pass(PASS_ROWS_FWD, geo.Px / 2, pb, st); }));
      }
      TOP_TRY(timed(h, KK_COLS, st, "column pass", [&] { return launch_pass(PASS_COLS, geo.Py / 2, ps[k], st); }));
    }
    TOP_TRY(timed(h, KK_ROWS_INV, st, "rows inverse pass", [&] { return launch_pass(PASS_ROWS_INV, geo.Px / 2, last, st); }));
    pos += n;
  }
  return TOP_OK;
}

// ============================================================================= ragged batches

// Fields of different sizes, spacings, wavelengths and distances, each with its own buffers.
// Fields with the same padded geometry and method run together, per-field pointers replacing
// the batch strides (device arrays in the workspace tail).
top_status run_ragged(top_handle h, int count, const top_grid* grids, const void* const* in, void* const* out,
                      const double* lam, const double* z, int backward, cudaStream_t st) {
  if (count < 0) return fail(TOP_ERR_INVALID_ARG, "count must be >= 0");
  if (count == 0) return TOP_OK;
  if (!grids || !in || !out || !lam || !z) return fail(TOP_ERR_INVALID_ARG, "grids, in, out, lambda and z must not be NULL");
  std::vector<Geometry> geos(count);
  for (int i = 0; i < count; ++i) {
    const top_grid* g = &grids[i];
    TOP_TRY(check_grid(g, &geos[i]));
    if (g->batch != 1) return fail(TOP_ERR_INVALID_ARG, "ragged field %d: batch must be 1 (got %lld)", i, (long long)g->batch);
    if (g->input_repeat > 1) return fail(TOP_ERR_INVALID_ARG, "ragged field %d: input_repeat must be 0 or 1", i);
    if (!(std::isfinite(lam[i]) && lam[i] > 0)) return fail(TOP_ERR_INVALID_ARG, "lambda[%d] must be finite and > 0", i);
    if (!std::isfinite(z[i])) return fail(TOP_ERR_INVALID_ARG, "z[%d] must be finite", i);
    TOP_TRY(check_ptr(in[i], "ragged input field"));
    TOP_TRY(check_ptr(out[i], "ragged output field"));
  }
  TOP_TRY(bind(h));
  // fields at padded sizes without a plan of their own go one by one through the Bluestein path
  for (int i = 0; i < count; ++i) {
    if (has_engines(geos[i])) continue;
    Request q{};
    q.g = &grids[i]; q.lam = &lam[i]; q.z = &z[i]; q.n_lz = 1; q.adjoint = backward ? 1 : 0;
    q.src_kind = SRC_FIELD; q.in = in[i]; q.group = 1;
    q.epi_kind = EPI_FIELD; q.out = out[i];
    TOP_TRY(run_bluestein(h, q, geos[i], st));
  }
  // groups of one geometry (padded sizes and the field's size), in first-appearance order: fields of
  // any method, wavelength, distance and spacing share a launch (each column reads its own table)
  std::vector<std::vector<int>> groups;
  std::vector<std::array<int, 4>> keys;
  for (int i = 0; i < count; ++i) {
    const Geometry& q = geos[i];
    if (!has_engines(q)) continue;
    const std::array<int, 4> key = {q.ny, q.nx, q.Py, q.Px};
    size_t k = 0;
    while (k < keys.size() && keys[k] != key) ++k;
    if (k == keys.size()) {
      keys.push_back(key);
      groups.emplace_back();
    }
    groups[k].push_back(i);
  }
  for (const auto& grp : groups) {
    const Geometry geo = geos[grp[0]];
    const long long plane = (long long)geo.ny * geo.nx;
    const float2 *twx, *twy, *wpx, *wpy;
    TOP_TRY(engine_twiddles(h, geo.Px / 2, &twx));
    TOP_TRY(engine_twiddles(h, geo.Py / 2, &twy));
    TOP_TRY(split_twiddles(h, geo.Px, &wpx));
    TOP_TRY(split_twiddles(h, geo.Py, &wpy));
    const int64_t nf = int64_t(grp.size());
    std::vector<const float2*> tables(nf);
    for (int64_t j = 0; j < nf; ++j) {
      const int i = grp[j];
      TransferEntry te;
      TOP_TRY(field_transfer(h, &grids[i], geo.ny, geo.nx, geo.Py, geo.Px, lam[i], z[i], st, &te));
      tables[j] = te.hq;
    }
    const size_t ws_field = size_t(geo.Px) * size_t(geo.ny) * sizeof(float2);
    const size_t ptr_field = 3 * sizeof(void*);
    int64_t chunk = std::min<int64_t>(nf, kMaxFields);
    auto need = [&](int64_t c) { return size_t(c) * ws_field + 256 + size_t(c) * ptr_field; };
    while (chunk > 1 && need(chunk) > h->ws_limit) chunk /= 2;
    if (need(chunk) > h->ws_limit)
      return fail(TOP_ERR_OOM, "one field needs %zu bytes of workspace, above the limit %llu", need(chunk),
                  (unsigned long long)h->ws_limit);
    TOP_TRY(ensure_workspace(h, need(chunk)));
    float2* ws = static_cast<float2*>(h->ws);
    char* tail = reinterpret_cast<char*>(h->ws) + size_t(chunk) * ws_field;
    tail = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(tail) + 255) & ~uintptr_t(255));
    void** d_lists = reinterpret_cast<void**>(tail);  // [in][out][table], chunk entries each

    PassParams p{};
    p.ny = geo.ny;
    p.nx = geo.nx;
    p.Py = geo.Py;
    p.Px = geo.Px;
    p.My = geo.Py / 2;
    p.Mx = geo.Px / 2;
    p.oy = geo.oy;
    p.ox = geo.ox;
    p.tune_rows = tune_flags(geo.Px / 2);
    p.tune_cols = tune_flags(geo.Py / 2);
    p.method = grids[grp[0]].method;
    p.adjoint = backward ? 1 : 0;
    p.src_kind = SRC_FIELD;
    p.epi_kind = EPI_FIELD;
    p.twx = twx;
    p.twy = twy;
    p.wpx = wpx;
    p.wpy = wpy;
    p.ws = ws;
    p.ws_stride = (long long)geo.Px * geo.ny;
    p.in_stride = plane;
    p.out_stride = plane;
    p.group = 1;
    p.src_group = 1;
    p.in_repeat = 1;
    p.in_list = reinterpret_cast<const float2* const*>(d_lists);
    p.out_list = reinterpret_cast<float2* const*>(d_lists + chunk);
    p.hq_list = reinterpret_cast<const float2* const*>(d_lists + 2 * chunk);
    p.nsets = 1;  // no lens tables; every column pass reads its field's table from hq_list
    std::vector<const void*> lists(3 * size_t(chunk));
    int64_t pos = 0;
    while (pos < nf) {
      const int64_t n = std::min<int64_t>(chunk, nf - pos);
      for (int64_t j = 0; j < n; ++j) {
        lists[j] = in[grp[pos + j]];
        lists[size_t(chunk) + j] = out[grp[pos + j]];
        lists[2 * size_t(chunk) + j] = tables[pos + j];
      }
      // the lists are rewritten in stream order after the previous chunk's kernels, by kernels
      // that carry them in their parameters
      TOP_CUDA(launch_put(d_lists, lists.data(), lists.size() * sizeof(void*), st), "ragged field lists");
      p.nfields = int(n);
      if (onchip_supported(p) && !(tune_flags(geo.Px / 2) & TOP_TUNE_THREE_PASS)) {
        // 64 x 64 fields at padding 2: the same on-chip kernel as a single call's
        TOP_TRY(timed(h, KK_ONCHIP, st, "on-chip propagation", [&] { return launch_onchip(p, st); }));
        pos += n;
        continue;
      }
      TOP_TRY(timed(h, KK_ROWS_FWD, st, "rows forward pass", [&] { return launch_pass(PASS_ROWS_FWD, p.Mx, p, st); }));
      TOP_TRY(timed(h, KK_COLS, st, "column pass", [&] { return launch_pass(PASS_COLS, p.My, p, st); }));
      TOP_TRY(timed(h, KK_ROWS_INV, st, "rows inverse pass", [&] { return launch_pass(PASS_ROWS_INV, p.Mx, p, st); }));
      pos += n;
    }
  }
  return TOP_OK;
}

}  // namespace

// ============================================================================= C ABI

extern "C" {

const char* top_last_error(void) { return t_last_error.c_str(); }

const char* top_status_string(top_status s) {
  switch (s) {
    case TOP_OK: return "TOP_OK";
    case TOP_ERR_INVALID_ARG: return "TOP_ERR_INVALID_ARG";
    case TOP_ERR_UNSUPPORTED: return "TOP_ERR_UNSUPPORTED";
    case TOP_ERR_OOM: return "TOP_ERR_OOM";
    case TOP_ERR_CUDA: return "TOP_ERR_CUDA";
    case TOP_ERR_TIMEOUT: return "TOP_ERR_TIMEOUT";
    case TOP_ERR_INTERNAL: return "TOP_ERR_INTERNAL";
  }
  return "TOP_ERR_UNKNOWN";
}

int top_version(void) { return TOP_ABI_VERSION; }

double top_zcritical(double L, double dx, double lambda) { return L * dx / lambda; }

top_status top_create(top_handle* out, int device) {
  if (!out) return fail(TOP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= count) return fail(TOP_ERR_INVALID_ARG, "device %d out of range (%d devices)", device, count);
  TOP_CUDA(cudaSetDevice(device), "cudaSetDevice");
  static std::once_flag tune_once;
  std::call_once(tune_once, [] {
    const char* path = std::getenv("TOP_AUTOTUNE_CACHE");
    std::string err;
    if (path && *path) tune_load(path, &err);  // a refused file leaves the defaults
  });
  top_ctx* h = new top_ctx();
  h->device = device;
  *out = h;
  return TOP_OK;
}

top_status top_autotune(top_handle h, const top_grid* g, uint32_t* rows_flags, uint32_t* cols_flags) {
  if (!h) return fail(TOP_ERR_INVALID_ARG, "handle is NULL");
  Geometry geo;
  TOP_TRY(check_grid(g, &geo));
  TOP_TRY(check_engines(geo));
  if (!has_engines(geo)) return fail(TOP_ERR_UNSUPPORTED, "autotune needs padded sizes with a plan of their own");
  TOP_TRY(bind(h));
  const int64_t B = g->batch;
  const size_t bytes = sizeof(float2) * size_t(B) * size_t(geo.ny) * size_t(geo.nx);
  void *x = nullptr, *y = nullptr, *gi = nullptr;
  TOP_CUDA(cudaMalloc(&x, bytes), "cudaMalloc(autotune fields)");
  if (cudaMalloc(&y, bytes) != cudaSuccess || cudaMalloc(&gi, bytes / 2) != cudaSuccess) {
    cudaFree(x);
    cudaFree(y);
    return fail(TOP_ERR_OOM, "cudaMalloc(autotune fields) failed");
  }
  cudaMemset(x, 0x3c, bytes);  // every float 0.0115
  cudaMemset(gi, 0x3c, bytes / 2);
  const int Mx = geo.Px / 2, My = geo.Py / 2;
  const uint32_t row_bits = TOP_TUNE_CLASSIC_FWD | TOP_TUNE_CLASSIC_INV | TOP_TUNE_CLASSIC_CHAIN | TOP_TUNE_NO_L2_FWD |
                            TOP_TUNE_SPAN(7);
  const uint32_t col_bits = TOP_TUNE_NO_L2_COLS;
  const uint32_t keep_x = tune_flags(Mx), keep_y = tune_flags(My);
  const bool keep_prof = h->prof;
  // launches the caller profiled before this call keep their totals
  for (auto& pe : h->pending) {
    float ms = 0.f;
    cudaEventSynchronize(pe.second.second);
    if (cudaEventElapsedTime(&ms, pe.second.first, pe.second.second) == cudaSuccess) {
      h->prof_ms[pe.first] += ms;
      h->prof_cnt[pe.first] += 1;
    }
    h->pool.push_back(pe.second.first);
    h->pool.push_back(pe.second.second);
  }
  h->pending.clear();
  auto apply = [&](uint32_t rows, uint32_t cols) {
    tune_set(Mx, (tune_flags(Mx) & ~row_bits) | rows);
    tune_set(My, (tune_flags(My) & ~col_bits) | cols);
  };
  top_mod lens{};
  lens.flags = TOP_MOD_LENS;
  lens.focal_length = 0.1;
  const double lam = 532e-9, z = 0.01;
  const top_stage stages[2] = {{z, nullptr, nullptr}, {z, &lens, nullptr}};
  top_grid gg = *g;
  gg.input_repeat = 0;
  // one candidate: a propagation and a two-stage chain, the mean milliseconds per kind over 3 runs
  auto measure = [&](uint32_t rows, uint32_t cols, double (&t)[KK_COUNT]) -> top_status {
    apply(rows, cols);
    for (int rep = 0; rep < 4; ++rep) {
      h->prof = rep > 0;
      Request q{};
      q.g = &gg; q.lam = &lam; q.z = &z; q.n_lz = 1; q.src_kind = SRC_FIELD; q.in = x; q.group = 1;
      q.epi_kind = EPI_FIELD; q.out = y;
      TOP_TRY(run_propagation(h, q, nullptr));
      // the backward from an intensity (the other source the forward rows see)
      Request b{};
      b.g = &gg; b.lam = &lam; b.z = &z; b.n_lz = 1; b.adjoint = 1; b.src_kind = SRC_INTENSITY; b.psi_src = x;
      b.gI = static_cast<const float*>(gi); b.group = 1; b.epi_kind = EPI_FIELD; b.out = y;
      TOP_TRY(run_propagation(h, b, nullptr));
      TOP_TRY(run_chain(h, &gg, x, y, nullptr, 1, &lam, 1, stages, 2, nullptr));
    }
    h->prof = false;
    TOP_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize(autotune)");
    for (int k = 0; k < KK_COUNT; ++k) t[k] = 0.0;
    for (auto& pe : h->pending) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, pe.second.first, pe.second.second) == cudaSuccess) t[pe.first] += ms / 3.0;
      h->pool.push_back(pe.second.first);
      h->pool.push_back(pe.second.second);
    }
    h->pending.clear();
    return TOP_OK;
  };
  double A[KK_COUNT], Bc[KK_COUNT], C[KK_COUNT], D[KK_COUNT], E[KK_COUNT];
  top_status st = measure(0, 0, A);
  if (st == TOP_OK) st = measure(TOP_TUNE_CLASSIC_FWD | TOP_TUNE_CLASSIC_INV | TOP_TUNE_CLASSIC_CHAIN, 0, Bc);
  if (st == TOP_OK) st = measure(TOP_TUNE_NO_L2_FWD | TOP_TUNE_SPAN(1), TOP_TUNE_NO_L2_COLS, C);
  if (st == TOP_OK) st = measure(TOP_TUNE_SPAN(2), 0, D);
  if (st == TOP_OK) st = measure(TOP_TUNE_SPAN(4), 0, E);
  h->prof = keep_prof;
  cudaFree(x);
  cudaFree(y);
  cudaFree(gi);
  if (st != TOP_OK) {
    tune_set(Mx, keep_x);
    tune_set(My, keep_y);
    return st;
  }
  // a variant replaces the default only when it is more than 2 % faster
  auto better = [](double cand, double base) { return cand < 0.98 * base; };
  uint32_t rows = 0, cols = 0;
  double fwd = A[KK_ROWS_FWD];
  if (better(Bc[KK_ROWS_FWD], fwd)) { rows |= TOP_TUNE_CLASSIC_FWD; fwd = Bc[KK_ROWS_FWD]; }
  if (better(C[KK_ROWS_FWD], fwd)) { rows = (rows & ~TOP_TUNE_CLASSIC_FWD) | TOP_TUNE_NO_L2_FWD; }
  double inv = A[KK_ROWS_INV];
  uint32_t inv_bits = 0;
  const std::pair<double, uint32_t> inv_cands[] = {{Bc[KK_ROWS_INV], TOP_TUNE_CLASSIC_INV}, {C[KK_ROWS_INV], TOP_TUNE_SPAN(1)},
                                                   {D[KK_ROWS_INV], TOP_TUNE_SPAN(2)}, {E[KK_ROWS_INV], TOP_TUNE_SPAN(4)}};
  for (const auto& c : inv_cands)
    if (better(c.first, inv)) { inv = c.first; inv_bits = c.second; }
  rows |= inv_bits;
  if (better(Bc[KK_ROWS_CHAIN], A[KK_ROWS_CHAIN])) rows |= TOP_TUNE_CLASSIC_CHAIN;
  if (better(C[KK_COLS], A[KK_COLS])) cols |= TOP_TUNE_NO_L2_COLS;
  apply(rows, cols);
  if (rows_flags) *rows_flags = tune_flags(Mx);
  if (cols_flags) *cols_flags = tune_flags(My);
  return TOP_OK;
}

top_status top_autotune_set(int line_length, uint32_t flags) {
  if (line_length < 1 || line_length > (1 << 20)) return fail(TOP_ERR_INVALID_ARG, "line length %d out of range", line_length);
  if (!tune_flags_valid(flags)) return fail(TOP_ERR_INVALID_ARG, "unknown autotune flags 0x%x", flags);
  tune_set(line_length, flags);
  return TOP_OK;
}

top_status top_autotune_get(int line_length, uint32_t* flags) {
  if (!flags) return fail(TOP_ERR_INVALID_ARG, "flags is NULL");
  *flags = tune_flags(line_length);
  return TOP_OK;
}

top_status top_autotune_clear(void) {
  tune_clear();
  return TOP_OK;
}

top_status top_autotune_save(const char* path) {
  if (!path) return fail(TOP_ERR_INVALID_ARG, "path is NULL");
  std::string err;
  if (!tune_save(path, &err)) return fail(TOP_ERR_INVALID_ARG, "autotune cache %s: %s", path, err.c_str());
  return TOP_OK;
}

top_status top_autotune_load(const char* path) {
  if (!path) return fail(TOP_ERR_INVALID_ARG, "path is NULL");
  std::string err;
  if (!tune_load(path, &err)) return fail(TOP_ERR_INVALID_ARG, "autotune cache %s: %s", path, err.c_str());
  return TOP_OK;
}

top_status top_destroy(top_handle h) {
  if (!h) return fail(TOP_ERR_INVALID_ARG, "handle is NULL");
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  for (void* p : h->allocs) cudaFree(p);
  if (h->ws) cudaFree(h->ws);
  if (h->coh) cudaFree(h->coh);
  if (h->cohg) cudaFree(h->cohg);
  if (h->chain) cudaFree(h->chain);
  for (auto& pe : h->pending) {
    cudaEventDestroy(pe.second.first);
    cudaEventDestroy(pe.second.second);
  }
  for (cudaEvent_t e : h->pool) cudaEventDestroy(e);
  delete h;
  return TOP_OK;
}

top_status top_set_workspace_limit(top_handle h, uint64_t bytes) {
  if (!h) return fail(TOP_ERR_INVALID_ARG, "handle is NULL");
  if (bytes < (1u << 20)) return fail(TOP_ERR_INVALID_ARG, "workspace limit below 1 MiB");
  h->ws_limit = bytes;
  return TOP_OK;
}

top_status top_plan_query(const top_grid* g, int64_t* py, int64_t* px, uint64_t* workspace_per_field) {
  Geometry geo;
  TOP_TRY(check_grid(g, &geo));
  // sizes without a plan of their own take Bluestein transforms (up to 4096 points per axis,
  // two field-sized buffers)
  const bool planned = has_engines(geo);
  if (!planned) {
    for (int P : {geo.Py, geo.Px})
      if (2 * P - 1 > 8192) TOP_TRY(check_engines(geo));
  }
  if (py) *py = geo.Py;
  if (px) *px = geo.Px;
  if (workspace_per_field)
    *workspace_per_field = uint64_t(planned ? 1 : 2) * uint64_t(geo.Px) * uint64_t(geo.ny) * sizeof(float2);
  return TOP_OK;
}

top_status top_propagate(top_handle h, const top_grid* g, const void* in, void* out, const double* lambda,
                         const double* z, int64_t n_lz, const top_mod* pre, const top_mod* post, void* stream) {
  if (!h) return fail(TOP_ERR_INVALID_ARG, "handle is NULL");
  Request q{};
  q.g = g; q.lam = lambda; q.z = z; q.n_lz = n_lz; q.adjoint = 0;
  q.src_kind = SRC_FIELD; q.in = in; q.group = 1;
  q.msrc = pre; q.msrc_conj = 0;
  q.epi_kind = EPI_FIELD; q.out = out; q.mepi = post; q.mepi_conj = 0;
  return run_propagation(h, q, static_cast<cudaStream_t>(stream));
}

top_status top_propagate_overlap(top_handle h, const top_grid* g, const void* in, void* field_out,
                                 const void* target, int64_t target_stride, double* overlap, double* power,
                                 const double* lambda, const double* z, int64_t n_lz, const top_mod* pre,
                                 const top_mod* post, void* stream) {
  if (!h) return fail(TOP_ERR_INVALID_ARG, "handle is NULL");
  Request q{};
  q.g = g; q.lam = lambda; q.z = z; q.n_lz = n_lz; q.adjoint = 0;
  q.src_kind = SRC_FIELD; q.in = in; q.group = 1;
  q.msrc = pre; q.msrc_conj = 0;
  q.epi_kind = EPI_OVERLAP; q.out = field_out; q.mepi = post; q.mepi_conj = 0;
  q.target = target; q.target_stride = target_stride; q.ov_out = overlap; q.pw_out = power;
  return run_propagation(h, q, static_cast<cudaStream_t>(stream));
}

top_status top_overlap_loss(top_handle h, const top_grid* g, const double* overlap, const void* target,
                            int64_t target_stride, double* loss, void* grad, void* stream) {
  if (!h) return fail(TOP_ERR_INVALID_ARG, "handle is NULL");
  if (!g) return fail(TOP_ERR_INVALID_ARG, "grid is NULL");
  if (g->batch < 1 || g->ny < 1 || g->nx < 1) return fail(TOP_ERR_INVALID_ARG, "batch, ny and nx must be >= 1");
  if (!(std::isfinite(g->dy) && g->dy > 0) || !(std::isfinite(g->dx) && g->dx > 0))
    return fail(TOP_ERR_INVALID_ARG, "spacing must be finite and > 0");
  const long long plane = (long long)g->ny * g->nx;
  if (!overlap || (reinterpret_cast<uintptr_t>(overlap) & 7u) || !loss || (reinterpret_cast<uintptr_t>(loss) & 7u))
    return fail(TOP_ERR_INVALID_ARG, "overlap and loss must be non-NULL, 8-byte aligned device arrays");
  if (grad) {
    TOP_TRY(check_ptr(grad, "grad"));
    TOP_TRY(check_ptr(target, "target"));
    if (target_stride != 0 && target_stride != plane)
      return fail(TOP_ERR_INVALID_ARG, "target_stride must be 0 (shared) or ny * nx (per field)");
  }
  TOP_TRY(bind(h));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return timed(h, KK_AUX, st, "overlap loss", [&] {
    return launch_overlap_loss(overlap, g->batch, static_cast<const float2*>(target), target_stride, plane,
                               g->dy * g->dx, loss, static_cast<float2*>(grad), st);
  });
}

// The Jones matrices of the elements of §5.1 as 3 x 3 matrices on (x, y, z), row-major (re, im)
// pairs: the 2 x 2 block acts on (x, y), the z component passes unchanged (J_zz = 1).
static void jones_put(double* out, const double (&re)[4], const double (&im)[4]) {
  for (int k = 0; k < 18; ++k) out[k] = 0.0;
  const int at[4] = {0, 1, 3, 4};  // (x, x), (x, y), (y, x), (y, y) in the 3 x 3 order
  for (int k = 0; k < 4; ++k) {
    out[2 * at[k]] = re[k];
    out[2 * at[k] + 1] = im[k];
  }
  out[2 * 8] = 1.0;
}

top_status top_jones_linear_polarizer(double theta, double* out) {
  if (!out) return fail(TOP_ERR_INVALID_ARG, "output matrix is NULL");
  if (!std::isfinite(theta)) return fail(TOP_ERR_INVALID_ARG, "theta must be finite");
  // projector on the transmission axis (cos theta, sin theta)
  const double c = std::cos(theta), s = std::sin(theta);
  jones_put(out, {c * c, c * s, s * c, s * s}, {0.0, 0.0, 0.0, 0.0});
  return TOP_OK;
}

top_status top_jones_circular_polarizer(int handedness, double* out) {
  if (!out) return fail(TOP_ERR_INVALID_ARG, "output matrix is NULL");
  if (handedness != 1 && handedness != -1) return fail(TOP_ERR_INVALID_ARG, "handedness must be +1 or -1");
  // projector on (1, i h) / sqrt 2: entries 1/2, -i h/2, i h/2, 1/2
  const double h = 0.5 * handedness;
  jones_put(out, {0.5, 0.0, 0.0, 0.5}, {0.0, -h, h, 0.0});
  return TOP_OK;
}

top_status top_jones_waveplate(double retardance, double theta, double* out) {
  if (!out) return fail(TOP_ERR_INVALID_ARG, "output matrix is NULL");
  if (!std::isfinite(retardance) || !std::isfinite(theta))
    return fail(TOP_ERR_INVALID_ARG, "retardance and theta must be finite");
  // fast axis u = (cos theta, sin theta) passes unchanged, the slow axis v = (-sin theta, cos theta)
  // is delayed by exp(i retardance): J = u u^T + exp(i retardance) v v^T
  const double c = std::cos(theta), s = std::sin(theta);
  const double er = std::cos(retardance), ei = std::sin(retardance);
  const double uu[4] = {c * c, c * s, s * c, s * s};
  const double vv[4] = {s * s, -s * c, -c * s, c * c};
  double re[4], im[4];
  for (int k = 0; k < 4; ++k) {
    re[k] = uu[k] + er * vv[k];
    im[k] = ei * vv[k];
  }
  jones_put(out, re, im);
  return TOP_OK;
}

static top_status jones_common(const top_grid* g, int64_t inner, const void* J, const double* ju, Jones3* m,
                               int64_t* groups) {
  if (!g) return fail(TOP_ERR_INVALID_ARG, "grid is NULL");
  if (g->batch < 1 || g->ny < 1 || g->nx < 1) return fail(TOP_ERR_INVALID_ARG, "batch, ny and nx must be >= 1");
  if (inner < 1 || g->batch % (3 * inner) != 0)
    return fail(TOP_ERR_INVALID_ARG, "batch (%lld) must be 3 * inner (%lld) * the number of polarised fields",
                (long long)g->batch, (long long)inner);
  *groups = g->batch / (3 * inner);
  if (J) {
    TOP_TRY(check_ptr(J, "Jones planes"));
  } else {
    if (!ju) return fail(TOP_ERR_INVALID_ARG, "give either Jones planes or a uniform Jones matrix");
    for (int k = 0; k < 9; ++k) {
      if (!std::isfinite(ju[2 * k]) || !std::isfinite(ju[2 * k + 1])) return fail(TOP_ERR_INVALID_ARG, "Jones matrix entries must be finite");
      m->m[k] = make_float2(float(ju[2 * k]), float(ju[2 * k + 1]));
    }
  }
  return TOP_OK;
}

top_status top_jones(top_handle h, const top_grid* g, int64_t inner, const void* J, const double* j_uniform,
                     const void* in, void* out, void* stream) {
  if (!h) return fail(TOP_ERR_INVALID_ARG, "handle is NULL");
  Jones3 m{};
  int64_t groups = 0;
  TOP_TRY(jones_common(g, inner, J, j_uniform, &m, &groups));
  TOP_TRY(check_ptr(in, "input field"));
  TOP_TRY(check_ptr(out, "output field"));
  TOP_TRY(bind(h));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return timed(h, KK_AUX, st, "Jones modulation", [&] {
    return launch_jones(static_cast<const float2*>(in), static_cast<float2*>(out), groups, inner,
                        (long long)g->ny * g->nx, static_cast<const float2*>(J), m, st);
  });
}

top_status top_jones_backward(top_handle h, const top_grid* g, int64_t inner, const void* J, const double* j_uniform,
                              const void* saved_in, const void* grad_out, void* grad_in, void* grad_J, void* stream) {
  if (!h) return fail(TOP_ERR_INVALID_ARG, "handle is NULL");
  Jones3 m{};
  int64_t groups = 0;
  TOP_TRY(jones_common(g, inner, J, j_uniform, &m, &groups));
  TOP_TRY(check_ptr(grad_out, "grad_out"));
  if (grad_in) TOP_TRY(check_ptr(grad_in, "grad_in"));
  if (grad_J) {
    if (!J) return fail(TOP_ERR_INVALID_ARG, "grad_J needs spatially varying Jones planes");
    TOP_TRY(check_ptr(grad_J, "grad_J"));
    TOP_TRY(check_ptr(saved_in, "saved_in"));
  }
  if (grad_in && grad_in == grad_out) return fail(TOP_ERR_INVALID_ARG, "grad_in must not alias grad_out");
  TOP_TRY(bind(h));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return timed(h, KK_AUX, st, "Jones backward", [&] {
    return launch_jones_backward(static_cast<const float2*>(saved_in), static_cast<const float2*>(grad_out),
                                 static_cast<float2*>(grad_in), static_cast<float2*>(grad_J), groups, inner,
                                 (long long)g->ny * g->nx, static_cast<const float2*>(J), m, st);
  });
}

top_status top_field_power(top_handle h, const top_grid* g, const void* field, double* power, void* stream) {
  if (!h) return fail(TOP_ERR_INVALID_ARG, "handle is NULL");
  if (!g) return fail(TOP_ERR_INVALID_ARG, "grid is NULL");
  if (g->batch < 1 || g->ny < 1 || g->nx < 1) return fail(TOP_ERR_INVALID_ARG, "batch, ny and nx must be >= 1");
  if (!(std::isfinite(g->dy) && g->dy > 0) || !(std::isfinite(g->dx) && g->dx > 0))
    return fail(TOP_ERR_INVALID_ARG, "spacing must be finite and > 0");
  TOP_TRY(check_ptr(field, "field"));
  if (!power || (reinterpret_cast<uintptr_t>(power) & 7u)) return fail(TOP_ERR_INVALID_ARG, "power must be a non-NULL, 8-byte aligned device array");
  TOP_TRY(bind(h));
  // partial sums in a small region at the end of the workspace
  const size_t bytes = size_t(g->batch) * kPowerBlocks * sizeof(double) + 256;
  if (h->ws_bytes < bytes) TOP_TRY(ensure_workspace(h, bytes));
  double* partial = reinterpret_cast<double*>(static_cast<char*>(h->ws) + h->ws_bytes - size_t(g->batch) * kPowerBlocks * sizeof(double));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return timed(h, KK_AUX, st, "field power", [&] {
    return launch_field_power(static_cast<const float2*>(field), g->batch, (long long)g->ny * g->nx, g->dy * g->dx,
                              partial, power, st);
  });
}

top_status top_resample(top_handle h, const top_grid* g, int ny_out, int nx_out, double dy_out, double dx_out, int mode,
                        int backward, const void* in, void* out, void* stream) {
  if (!h) return fail(TOP_ERR_INVALID_ARG, "handle is NULL");
  if (!g) return fail(TOP_ERR_INVALID_ARG, "grid is NULL");
  if (g->batch < 1 || g->ny < 1 || g->nx < 1 || ny_out < 1 || nx_out < 1)
    return fail(TOP_ERR_INVALID_ARG, "batch and all grid sizes must be >= 1");
  for (double d : {g->dy, g->dx, dy_out, dx_out})
    if (!(std::isfinite(d) && d > 0)) return fail(TOP_ERR_INVALID_ARG, "spacings must be finite and > 0");
  if (mode != TOP_NEAREST && mode != TOP_BILINEAR) return fail(TOP_ERR_INVALID_ARG, "unknown interpolation mode %d", mode);
  TOP_TRY(check_ptr(in, "input"));
  TOP_TRY(check_ptr(out, "output"));
  if (in == out) return fail(TOP_ERR_INVALID_ARG, "input and output must be distinct");
  TOP_TRY(bind(h));
  ResampleGeom rg{g->ny, g->nx, ny_out, nx_out, g->dy, g->dx, dy_out, dx_out, mode};
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return timed(h, KK_AUX, st, "resample", [&] {
    return launch_resample(static_cast<const float2*>(in), static_cast<float2*>(out), g->batch, rg, backward ? 1 : 0, st);
  });
}

top_status top_propagate_ragged(top_handle h, int count, const top_grid* grids, const void* const* in,
                                void* const* out, const double* lambda, const double* z, int backward, void* stream) {
  if (!h) return fail(TOP_ERR_INVALID_ARG, "handle is NULL");
  return run_ragged(h, count, grids, in, out, lambda, z, backward, static_cast<cudaStream_t>(stream));
}

top_status top_fused_chain(top_handle h, const top_grid* g, const void* in, void* out, float* intensity,
                           int64_t group, const double* lambda, int64_t n_lz, const top_stage* stages, int nstages,
                           void* stream) {
  if (!h) return fail(TOP_ERR_INVALID_ARG, "handle is NULL");
  return run_chain(h, g, in, out, intensity, group, lambda, n_lz, stages, nstages, static_cast<cudaStream_t>(stream));
}

top_status top_propagate_backward(top_handle h, const top_grid* g, const void* grad_out, void* grad_in,
                                  const double* lambda, const double* z, int64_t n_lz, const top_mod* pre,
                                  const top_mod* post, const top_mod_grads* pre_grads, void* stream) {
  if (!h) return fail(TOP_ERR_INVALID_ARG, "handle is NULL");
  Request q{};
  q.g = g; q.lam = lambda; q.z = z; q.n_lz = n_lz; q.adjoint = 1;
  q.src_kind = SRC_FIELD; q.in = grad_out; q.group = 1;
  q.msrc = post; q.msrc_conj = 1;
  const bool pg = pre_grads && (pre_grads->grad_phase || pre_grads->grad_amplitude || pre_grads->grad_mask);
  if (pg) {
    q.epi_kind = EPI_MODGRAD; q.out = grad_in; q.mepi = pre; q.mepi_conj = 0; q.grads = pre_grads;
  } else {
    if (!grad_in) return fail(TOP_ERR_INVALID_ARG, "grad_in is NULL and no modulation gradient requested");
    q.epi_kind = EPI_FIELD; q.out = grad_in; q.mepi = pre; q.mepi_conj = 1;
  }
  return run_propagation(h, q, static_cast<cudaStream_t>(stream));
}

top_status top_propagate_intensity(top_handle h, const top_grid* g, const void* in, void* field_out,
                                   float* intensity, int64_t group, const float* weights, const double* lambda,
                                   const double* z, int64_t n_lz, const top_mod* pre, const top_mod* post,
                                   void* stream) {
  if (!h) return fail(TOP_ERR_INVALID_ARG, "handle is NULL");
  Request q{};
  q.g = g; q.lam = lambda; q.z = z; q.n_lz = n_lz; q.adjoint = 0;
  q.src_kind = SRC_FIELD; q.in = in; q.group = group; q.weights = weights;
  q.msrc = pre; q.msrc_conj = 0;
  q.epi_kind = EPI_INTENSITY; q.out = field_out; q.outf = intensity; q.mepi = post; q.mepi_conj = 0;
  return run_propagation(h, q, static_cast<cudaStream_t>(stream));
}

top_status top_fused_chain_backward(top_handle h, const top_grid* g, const void* field, const float* grad_intensity,
                                    int64_t group, const double* lambda, int64_t n_lz, const top_stage* stages,
                                    int nstages, const top_mod_grads* first_grads, void* grad_in, void* stream) {
  if (!h) return fail(TOP_ERR_INVALID_ARG, "handle is NULL");
  if (!g) return fail(TOP_ERR_INVALID_ARG, "grid is NULL");
  if (!stages || nstages < 1) return fail(TOP_ERR_INVALID_ARG, "a chain needs at least one stage");
  if (g->input_repeat > 1) return fail(TOP_ERR_INVALID_ARG, "the backward of a chain takes input_repeat 0 or 1");
  for (int k = 0; k < nstages; ++k) {
    if (!std::isfinite(stages[k].z)) return fail(TOP_ERR_INVALID_ARG, "stage %d: z must be finite", k);
    TOP_TRY(check_mod(stages[k].pre, "stage modulation"));
  }
  // stage 0's adjoint is the request; stages K-1 .. 1 run upstream of it, in that order
  std::vector<top_stage> up;
  for (int k = nstages - 1; k >= 1; --k) up.push_back(stages[k]);
  std::vector<double> z0(size_t(std::max<int64_t>(1, n_lz)), stages[0].z);
  Request q{};
  q.g = g; q.lam = lambda; q.z = z0.data(); q.n_lz = n_lz; q.adjoint = 1;
  q.src_kind = SRC_INTENSITY; q.psi_src = field; q.gI = grad_intensity; q.group = group;
  q.up = up.empty() ? nullptr : up.data();
  q.n_up = int(up.size());
  const top_mod* pre0 = stages[0].pre;
  const bool pg = first_grads && (first_grads->grad_phase || first_grads->grad_amplitude || first_grads->grad_mask);
  if (pg) {
    q.epi_kind = EPI_MODGRAD; q.out = grad_in; q.mepi = pre0; q.mepi_conj = 0; q.grads = first_grads;
  } else {
    if (!grad_in) return fail(TOP_ERR_INVALID_ARG, "grad_in is NULL and no modulation gradient requested");
    q.epi_kind = EPI_FIELD; q.out = grad_in; q.mepi = pre0; q.mepi_conj = 1;
  }
  return run_propagation(h, q, static_cast<cudaStream_t>(stream));
}

top_status top_propagate_intensity_backward(top_handle h, const top_grid* g, const void* field,
                                            const float* grad_intensity, void* grad_in, int64_t group,
                                            const float* weights, const double* lambda, const double* z,
                                            int64_t n_lz, const top_mod* pre, const top_mod* post,
                                            const top_mod_grads* pre_grads, void* stream) {
  if (!h) return fail(TOP_ERR_INVALID_ARG, "handle is NULL");
  Request q{};
  q.g = g; q.lam = lambda; q.z = z; q.n_lz = n_lz; q.adjoint = 1;
  q.src_kind = SRC_INTENSITY; q.psi_src = field; q.gI = grad_intensity; q.group = group; q.weights = weights;
  q.msrc = post; q.msrc_conj = 1;
  const bool pg = pre_grads && (pre_grads->grad_phase || pre_grads->grad_amplitude || pre_grads->grad_mask);
  if (pg) {
    q.epi_kind = EPI_MODGRAD; q.out = grad_in; q.mepi = pre; q.mepi_conj = 0; q.grads = pre_grads;
  } else {
    if (!grad_in) return fail(TOP_ERR_INVALID_ARG, "grad_in is NULL and no modulation gradient requested");
    q.epi_kind = EPI_FIELD; q.out = grad_in; q.mepi = pre; q.mepi_conj = 1;
  }
  return run_propagation(h, q, static_cast<cudaStream_t>(stream));
}

// ----------------------------------------------------------------------------- modulation

static top_status modulation_common(top_handle h, const top_grid* g, const top_mod* mod, const double* lambda,
                                    int64_t n_lz, Geometry* geo, PassParams* p) {
  TOP_TRY(check_grid(g, geo));
  if (!mod) return fail(TOP_ERR_INVALID_ARG, "modulation is NULL");
  TOP_TRY(check_mod(mod, "modulation"));
  if (mod->flags & TOP_MOD_LENS) TOP_TRY(check_lz(g, lambda, nullptr, n_lz, false));
  TOP_TRY(bind(h));
  const int2* circ = nullptr;
  if (mod->flags & TOP_MOD_CIRC) TOP_TRY(circ_table(h, geo->ny, geo->nx, g->dy, g->dx, mod->radius, &circ));
  *p = PassParams{};
  p->ny = geo->ny;
  p->nx = geo->nx;
  p->msrc = mod_dev(mod, 0, circ);
  p->mepi = p->msrc;
  return TOP_OK;
}

top_status top_modulate(top_handle h, const top_grid* g, const top_mod* mod, const void* in, void* out,
                        const double* lambda, int64_t n_lz, void* stream) {
  if (!h) return fail(TOP_ERR_INVALID_ARG, "handle is NULL");
  Geometry geo;
  PassParams p;
  TOP_TRY(modulation_common(h, g, mod, lambda, n_lz, &geo, &p));
  TOP_TRY(check_ptr(in, "input field"));
  TOP_TRY(check_ptr(out, "output field"));
  const ModDev base = p.msrc;
  const long long plane = (long long)geo.ny * geo.nx;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int64_t pos = 0; pos < g->batch; pos += kMaxSets) {
    const int64_t n = std::min<int64_t>(kMaxSets, g->batch - pos);
    TOP_TRY(fill_lens_sets(h, g, mod, lambda, n_lz, pos, n, &p));
    p.nfields = int(n);
    p.msrc = offset_mod(base, pos);
    p.in = static_cast<const float2*>(in) + pos * plane;
    p.out = static_cast<float2*>(out) + pos * plane;
    TOP_TRY(timed(h, KK_AUX, st, "modulate", [&] { return launch_modulate(p, st); }));
  }
  return TOP_OK;
}

top_status top_modulate_backward(top_handle h, const top_grid* g, const top_mod* mod, const void* grad_out,
                                 void* grad_in, const top_mod_grads* grads, const double* lambda, int64_t n_lz,
                                 void* stream) {
  if (!h) return fail(TOP_ERR_INVALID_ARG, "handle is NULL");
  Geometry geo;
  PassParams p;
  TOP_TRY(modulation_common(h, g, mod, lambda, n_lz, &geo, &p));
  TOP_TRY(check_ptr(grad_out, "grad_out"));
  if (grad_in) TOP_TRY(check_ptr(grad_in, "grad_in"));
  const bool pg = grads && (grads->grad_phase || grads->grad_amplitude || grads->grad_mask);
  if (pg) {
    TOP_TRY(check_ptr(grads->saved_in, "grads->saved_in"));
    if (grads->grad_phase && !(mod->flags & TOP_MOD_PHASE)) return fail(TOP_ERR_INVALID_ARG, "grad_phase needs TOP_MOD_PHASE");
    if (grads->grad_amplitude && !(mod->flags & TOP_MOD_AMPLITUDE)) return fail(TOP_ERR_INVALID_ARG, "grad_amplitude needs TOP_MOD_AMPLITUDE");
    if (grads->grad_mask && !(mod->flags & TOP_MOD_COMPLEX)) return fail(TOP_ERR_INVALID_ARG, "grad_mask needs TOP_MOD_COMPLEX");
  }
  if (!grad_in && !pg) return fail(TOP_ERR_INVALID_ARG, "nothing to compute");
  // the lens factor varies with the field's wavelength; all other factors are per pixel
  const long long plane = (long long)geo.ny * geo.nx;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool shared = mod->batch_stride == 0;
  const ModDev base = p.msrc;
  // with a shared mask the first chunk writes the gradients and later chunks add to them
  for (int64_t pos = 0; pos < g->batch; pos += kMaxSets) {
    const int64_t n = std::min<int64_t>(kMaxSets, g->batch - pos);
    TOP_TRY(fill_lens_sets(h, g, mod, lambda, n_lz, pos, n, &p));
    p.nfields = int(n);
    p.in = static_cast<const float2*>(grad_out) + pos * plane;
    p.out = grad_in ? static_cast<float2*>(grad_in) + pos * plane : nullptr;
    p.xs = pg ? static_cast<const float2*>(grads->saved_in) + pos * plane : nullptr;
    p.msrc = offset_mod(base, pos);
    const long long goff = shared ? 0 : pos * plane;
    p.part_phase = pg && grads->grad_phase ? grads->grad_phase + goff : nullptr;
    p.part_amp = pg && grads->grad_amplitude ? grads->grad_amplitude + goff : nullptr;
    p.part_mask = pg && grads->grad_mask ? static_cast<float2*>(grads->grad_mask) + goff : nullptr;
    p.part_accumulate = (shared && pos > 0) ? 1 : 0;
    p.group = shared ? int(n) : 1;
    TOP_TRY(timed(h, KK_AUX, st, "modulate backward", [&] { return launch_modulate_backward(p, st); }));
  }
  return TOP_OK;
}

// ----------------------------------------------------------------------------- loss

top_status top_mse_loss(top_handle h, int64_t n, const float* intensity, const float* target, double* loss,
                        float* grad, void* stream) {
  if (!h) return fail(TOP_ERR_INVALID_ARG, "handle is NULL");
  if (n < 1) return fail(TOP_ERR_INVALID_ARG, "n must be >= 1");
  TOP_TRY(check_ptr(intensity, "intensity"));
  TOP_TRY(check_ptr(target, "target"));
  TOP_TRY(check_ptr(loss, "loss"));
  if (grad) TOP_TRY(check_ptr(grad, "grad"));
  TOP_TRY(bind(h));
  // partial sums live in a small region at the end of the workspace
  const size_t bytes = kMseBlocks * sizeof(double) + 256;
  if (h->ws_bytes < bytes) TOP_TRY(ensure_workspace(h, bytes));
  double* partial = reinterpret_cast<double*>(static_cast<char*>(h->ws) + h->ws_bytes - kMseBlocks * sizeof(double));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return timed(h, KK_AUX, st, "mse loss", [&] { return launch_mse(n, intensity, target, grad, partial, loss, st); });
}

// ----------------------------------------------------------------------------- mutual coherence


// Mask parameters of a coherence modulation M(r) (single wavelength).
static top_status coh_mask_params(top_handle h, const top_grid* g, const top_mod* mask, double lam, PassParams* p) {
  *p = PassParams{};
  p->ny = g->ny;
  p->nx = g->nx;
  const int2* circ = nullptr;
  if (mask->flags & TOP_MOD_CIRC) TOP_TRY(circ_table(h, g->ny, g->nx, g->dy, g->dx, mask->radius, &circ));
  p->msrc = mod_dev(mask, 0, circ);
  FieldSet fs{};
  if (mask->flags & TOP_MOD_LENS) {
    TOP_TRY(lens_table(h, g->nx, g->dx, lam, mask->focal_length, &fs.src_lx));
    TOP_TRY(lens_table(h, g->ny, g->dy, lam, mask->focal_length, &fs.src_ly));
  }
  p->nsets = 1;
  p->sets[0] = fs;
  return TOP_OK;
}

static top_status coh_check(const top_grid* g, const double* lambda, const double* z, const top_mod* mask) {
  Geometry geo;
  TOP_TRY(check_grid(g, &geo));
  TOP_TRY(check_engines(geo));
  TOP_TRY(check_lz(g, lambda, z, 1, true));
  TOP_TRY(check_mod(mask, "coherence mask"));
  if (mask && mask->flags && mask->batch_stride != 0) return fail(TOP_ERR_INVALID_ARG, "coherence mask must be shared (batch_stride 0)");
  const long long n = (long long)g->ny * g->nx;
  if (n * n * g->batch > (1ll << 40)) return fail(TOP_ERR_INVALID_ARG, "coherence tensor too large");
  return TOP_OK;
}

// P or P^H applied over r2 (each r1 slice), then over r1 via two batched transposes (Eq. 13).
static top_status coh_two_sided(top_handle h, const top_grid* g, const void* src, void* dst, const double* lambda,
                                const double* z, int adjoint_r2, cudaStream_t st) {
  const int n = g->ny * g->nx;
  top_grid fg = *g;
  fg.batch = g->batch * n;
  Request q{};
  q.g = &fg; q.lam = lambda; q.z = z; q.n_lz = 1; q.adjoint = adjoint_r2;
  q.src_kind = SRC_FIELD; q.in = src; q.group = 1;
  q.epi_kind = EPI_FIELD; q.out = dst;
  TOP_TRY(run_propagation(h, q, st));
  void* tmp = nullptr;
  TOP_TRY(coh_scratch(h, sizeof(float2) * size_t(g->batch) * n * n, &tmp));
  TOP_TRY(timed(h, KK_AUX, st, "transpose", [&] {
    return launch_transpose(static_cast<const float2*>(dst), static_cast<float2*>(tmp), g->batch, n, st);
  }));
  q.in = tmp; q.out = tmp; q.adjoint = 1 - adjoint_r2;
  TOP_TRY(run_propagation(h, q, st));
  return timed(h, KK_AUX, st, "transpose", [&] {
    return launch_transpose(static_cast<const float2*>(tmp), static_cast<float2*>(dst), g->batch, n, st);
  });
}

top_status top_propagate_coherence(top_handle h, const top_grid* g, const void* gamma_in, void* gamma_out,
                                   const double* lambda, const double* z, const top_mod* mask, void* stream) {
  if (!h) return fail(TOP_ERR_INVALID_ARG, "handle is NULL");
  TOP_TRY(coh_check(g, lambda, z, mask));
  TOP_TRY(check_ptr(gamma_in, "gamma_in"));
  TOP_TRY(check_ptr(gamma_out, "gamma_out"));
  if (gamma_in == gamma_out) return fail(TOP_ERR_INVALID_ARG, "gamma_in and gamma_out must be distinct");
  TOP_TRY(bind(h));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const void* src = gamma_in;
  if (mask && mask->flags) {
    PassParams mp;
    TOP_TRY(coh_mask_params(h, g, mask, lambda[0], &mp));
    TOP_TRY(timed(h, KK_AUX, st, "coherence modulation", [&] {
      return launch_coh_modulate(static_cast<const float2*>(gamma_in), static_cast<float2*>(gamma_out), mp, g->batch, 0, st);
    }));
    src = gamma_out;
  }
  // Gamma_z = P Gamma P^H: conj(H) over (y2, x2), H over (y1, x1)
  return coh_two_sided(h, g, src, gamma_out, lambda, z, 1, st);
}

top_status top_propagate_coherence_backward(top_handle h, const top_grid* g, const void* grad_out, void* grad_in,
                                            const double* lambda, const double* z, const top_mod* mask,
                                            const top_mod_grads* grads, void* stream) {
  if (!h) return fail(TOP_ERR_INVALID_ARG, "handle is NULL");
  TOP_TRY(coh_check(g, lambda, z, mask));
  TOP_TRY(check_ptr(grad_out, "grad_out"));
  const bool pg = grads && (grads->grad_phase || grads->grad_amplitude || grads->grad_mask);
  if (grad_in) TOP_TRY(check_ptr(grad_in, "grad_in"));
  if (!grad_in && !pg) return fail(TOP_ERR_INVALID_ARG, "nothing to compute");
  if (pg) {
    if (!mask || !mask->flags) return fail(TOP_ERR_INVALID_ARG, "mask gradients need a mask");
    TOP_TRY(check_ptr(grads->saved_in, "grads->saved_in"));
    if (grads->grad_phase && !(mask->flags & TOP_MOD_PHASE)) return fail(TOP_ERR_INVALID_ARG, "grad_phase needs TOP_MOD_PHASE");
    if (grads->grad_amplitude && !(mask->flags & TOP_MOD_AMPLITUDE)) return fail(TOP_ERR_INVALID_ARG, "grad_amplitude needs TOP_MOD_AMPLITUDE");
    if (grads->grad_mask && !(mask->flags & TOP_MOD_COMPLEX)) return fail(TOP_ERR_INVALID_ARG, "grad_mask needs TOP_MOD_COMPLEX");
  }
  if (grad_in == grad_out) return fail(TOP_ERR_INVALID_ARG, "grad_in and grad_out must be distinct");
  TOP_TRY(bind(h));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int n = g->ny * g->nx;
  const size_t tensor = sizeof(float2) * size_t(g->batch) * n * n;
  // G' = P^H G P lands in grad_in, or (when the caller wants no grad_in) in a scratch tensor the
  // handle keeps: the two-sided propagation uses the workspace and the transpose scratch already
  void* dst = grad_in;
  if (!dst) {
    TOP_TRY(grow_scratch(&h->cohg, &h->cohg_bytes, tensor, "cudaMalloc(coherence gradient)"));
    dst = h->cohg;
  }
  top_status s = coh_two_sided(h, g, grad_out, dst, lambda, z, 0, st);
  if (s == TOP_OK && pg) {
    PassParams mp;
    s = coh_mask_params(h, g, mask, lambda[0], &mp);
    const size_t work = coh_mask_grads_work(int(n)) + 256;
    if (s == TOP_OK && h->ws_bytes < work) s = ensure_workspace(h, work);
    if (s == TOP_OK)
      s = timed(h, KK_AUX, st, "coherence mask gradients", [&] {
        return launch_coh_mask_grads(static_cast<const float2*>(dst), static_cast<const float2*>(grads->saved_in), mp,
                                     g->batch, static_cast<float2*>(h->ws), grads->grad_phase, grads->grad_amplitude,
                                     static_cast<float2*>(grads->grad_mask), st);
      });
  }
  if (s == TOP_OK && grad_in && mask && mask->flags) {
    PassParams mp;
    s = coh_mask_params(h, g, mask, lambda[0], &mp);
    if (s == TOP_OK)
      s = timed(h, KK_AUX, st, "coherence modulation backward", [&] {
        return launch_coh_modulate(static_cast<const float2*>(dst), static_cast<float2*>(dst), mp, g->batch, 1, st);
      });
  }
  return s;
}

static top_status intensity_check(top_handle h, const top_grid* g, const void* field, const void* other, int64_t group,
                                  const float* weights, long long* plane) {
  if (!h) return fail(TOP_ERR_INVALID_ARG, "handle is NULL");
  Geometry geo;
  TOP_TRY(check_grid(g, &geo));
  TOP_TRY(check_ptr(field, "field"));
  TOP_TRY(check_ptr(other, "intensity or gradient"));
  if (group < 1 || g->batch % group != 0)
    return fail(TOP_ERR_INVALID_ARG, "group (%lld) must be >= 1 and divide batch (%lld)", (long long)group,
                (long long)g->batch);
  if (group > 65535) return fail(TOP_ERR_UNSUPPORTED, "group larger than 65535 fields");
  if (weights && !aligned16(weights)) return fail(TOP_ERR_INVALID_ARG, "weights not 16-byte aligned");
  *plane = (long long)g->ny * g->nx;
  return TOP_OK;
}

top_status top_intensity(top_handle h, const top_grid* g, const void* field, float* intensity, int64_t group,
                         const float* weights, void* stream) {
  long long plane = 0;
  TOP_TRY(intensity_check(h, g, field, intensity, group, weights, &plane));
  TOP_TRY(bind(h));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return timed(h, KK_AUX, st, "intensity", [&] {
    return launch_intensity_sum(static_cast<const float2*>(field), weights, int(group), g->batch / group, plane,
                                intensity, st);
  });
}

top_status top_intensity_backward(top_handle h, const top_grid* g, const void* field, const float* grad_intensity,
                                  void* grad_field, int64_t group, const float* weights, void* stream) {
  long long plane = 0;
  TOP_TRY(intensity_check(h, g, field, grad_field, group, weights, &plane));
  TOP_TRY(check_ptr(grad_intensity, "grad_intensity"));
  TOP_TRY(bind(h));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return timed(h, KK_AUX, st, "intensity backward", [&] {
    return launch_intensity_source(static_cast<const float2*>(field), grad_intensity, weights, int(group), g->batch,
                                   plane, static_cast<float2*>(grad_field), st);
  });
}

top_status top_coherence_intensity(top_handle h, const top_grid* g, const void* gamma, float* intensity, void* stream) {
  if (!h) return fail(TOP_ERR_INVALID_ARG, "handle is NULL");
  Geometry geo;
  TOP_TRY(check_grid(g, &geo));
  TOP_TRY(check_ptr(gamma, "gamma"));
  TOP_TRY(check_ptr(intensity, "intensity"));
  TOP_TRY(bind(h));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return timed(h, KK_AUX, st, "coherence intensity", [&] {
    return launch_coh_diag(static_cast<const float2*>(gamma), intensity, g->batch, g->ny * g->nx, st);
  });
}

top_status top_coherence_intensity_backward(top_handle h, const top_grid* g, const float* grad_intensity,
                                            void* grad_gamma, void* stream) {
  if (!h) return fail(TOP_ERR_INVALID_ARG, "handle is NULL");
  Geometry geo;
  TOP_TRY(check_grid(g, &geo));
  TOP_TRY(check_ptr(grad_intensity, "grad_intensity"));
  TOP_TRY(check_ptr(grad_gamma, "grad_gamma"));
  TOP_TRY(bind(h));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return timed(h, KK_AUX, st, "coherence intensity backward", [&] {
    return launch_coh_diag_backward(grad_intensity, static_cast<float2*>(grad_gamma), g->batch, g->ny * g->nx, st);
  });
}

// ----------------------------------------------------------------------------- instrumentation

top_status top_profile_enable(top_handle h, int enable) {
  if (!h) return fail(TOP_ERR_INVALID_ARG, "handle is NULL");
  h->prof = enable != 0;
  return TOP_OK;
}

top_status top_profile_read(top_handle h, int cap, const char** kinds, double* ms, int64_t* count, int* n) {
  if (!h) return fail(TOP_ERR_INVALID_ARG, "handle is NULL");
  for (auto& pe : h->pending) {
    float t = 0.f;
    cudaEventSynchronize(pe.second.second);
    if (cudaEventElapsedTime(&t, pe.second.first, pe.second.second) == cudaSuccess) {
      h->prof_ms[pe.first] += t;
      h->prof_cnt[pe.first] += 1;
    }
    h->pool.push_back(pe.second.first);
    h->pool.push_back(pe.second.second);
  }
  h->pending.clear();
  static const char* names[KK_COUNT] = {"rows_fwd", "cols", "rows_inv", "aux", "rows_chain", "onchip"};
  int w = 0;
  for (int k = 0; k < KK_COUNT && w < cap; ++k, ++w) {
    if (kinds) kinds[w] = names[k];
    if (ms) ms[w] = h->prof_ms[k];
    if (count) count[w] = h->prof_cnt[k];
    h->prof_ms[k] = 0;
    h->prof_cnt[k] = 0;
  }
  if (n) *n = w;
  return TOP_OK;
}

}  // extern "C"

// ============================================================================= static-scratch propagation

namespace {

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Address of the static scratch on the current device (looked up once per device).
top_status noalloc_scratch(void** out) {
  const cudaError_t e = noalloc_scratch_address(out);
  if (e == cudaErrorInvalidDevice) return fail(TOP_ERR_UNSUPPORTED, "device beyond the ones the static scratch supports");
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
  return TOP_OK;
}

// Host image of an engine's stage twiddles (the same float64 arithmetic as the handle's cached ones).
void noalloc_engine_twiddles(int M, std::vector<float2>& tw) {
  EngineInfo info;
  find_engine(M, &info);
  tw.assign(std::max(1, info.tw_size), make_float2(0.f, 0.f));
  size_t off = 0;
  for (int s = 0; s < info.NS; ++s) {
    int sp = 1;
    for (int i = s + 1; i < info.NS; ++i) sp *= info.R[i];
    if (sp <= 1) continue;
    const int r = info.R[s], L = r * sp;
    for (int j = 1; j < r; ++j)
      for (int i = 0; i < sp; ++i) tw[off + size_t(j - 1) * sp + i] = unit_root((long long)i * j, L);
    off += size_t(r - 1) * sp;
  }
}

// Append a table to the host image at a 256-byte boundary; returns its byte offset.
template <class T>
size_t put(std::vector<unsigned char>& img, const std::vector<T>& v) {
  const size_t off = align256(img.size());
  img.resize(off + v.size() * sizeof(T));
  if (!v.empty()) std::memcpy(img.data() + off, v.data(), v.size() * sizeof(T));
  return off;
}

top_status propagate_noalloc(const top_grid* g, const void* in, void* out, const double* lam, const double* z,
                             int64_t n_lz, cudaStream_t st) {
  Geometry geo;
  TOP_TRY(check_grid(g, &geo));
  TOP_TRY(check_engines(geo));
  TOP_TRY(check_lz(g, lam, z, n_lz, true));
  if (g->input_repeat > 1) return fail(TOP_ERR_UNSUPPORTED, "top_propagate_noalloc takes input_repeat 0 or 1");
  if (g->method != TOP_AS && g->method != TOP_FRESNEL_TF)
    return fail(TOP_ERR_UNSUPPORTED, "top_propagate_noalloc takes the AS and Fresnel methods");
  TOP_TRY(check_ptr(in, "input field"));
  TOP_TRY(check_ptr(out, "output field"));
  const int64_t B = g->batch;
  const long long plane = (long long)geo.ny * geo.nx;

  // scratch budget: the twiddles, table slots for the distinct (lambda, z) sets, then the workspace
  EngineInfo ix, iy;
  find_engine(geo.Px / 2, &ix);
  find_engine(geo.Py / 2, &iy);
  const size_t tw_bytes = align256(std::max(1, ix.tw_size) * sizeof(float2)) +
                          align256(std::max(1, iy.tw_size) * sizeof(float2)) +
                          align256(size_t(geo.Px / 2) * sizeof(float2)) + align256(size_t(geo.Py / 2) * sizeof(float2));
  const size_t set_bytes = align256(size_t(geo.Px / 2 + 1) * size_t(geo.Py / 2 + 2) * sizeof(float2));
  const size_t ws_field = size_t(geo.Px) * size_t(geo.ny) * sizeof(float2);
  const size_t cap = TOP_NOALLOC_SCRATCH_BYTES;
  if (tw_bytes + set_bytes + ws_field > cap)
    return fail(TOP_ERR_UNSUPPORTED,
                "one %dx%d field (padded %dx%d) needs %zu bytes of static scratch (workspace %zu + tables %zu), "
                "above the %zu bytes of top_propagate_noalloc",
                geo.ny, geo.nx, geo.Py, geo.Px, tw_bytes + set_bytes + ws_field, ws_field, tw_bytes + set_bytes, cap);
  int64_t distinct = 0;
  {
    std::vector<std::pair<uint64_t, uint64_t>> all;
    for (int64_t i = 0; i < n_lz; ++i) all.emplace_back(bits(lam[i]), bits(z[i]));
    std::sort(all.begin(), all.end());
    distinct = std::unique(all.begin(), all.end()) - all.begin();
  }
  // the chunk first: the most fields n whose workspace and min(n, distinct, kMaxSets) tables fit
  auto fits = [&](int64_t n) {
    const int64_t sets = std::min<int64_t>({n, distinct, int64_t(kMaxSets)});
    return tw_bytes + size_t(sets) * set_bytes + size_t(n) * ws_field <= cap;
  };
  int64_t chunk = std::min<int64_t>(B, kMaxFields);
  while (chunk > 1 && !fits(chunk)) --chunk;
  const int slots = int(std::min<int64_t>({chunk, distinct, int64_t(kMaxSets)}));
  const size_t table_bytes = tw_bytes + size_t(slots) * set_bytes;

  void* scratch = nullptr;
  TOP_TRY(noalloc_scratch(&scratch));
  unsigned char* base = static_cast<unsigned char*>(scratch);
  float2* ws = reinterpret_cast<float2*>(base + table_bytes);

  // twiddles: written in stream order by kernels that carry them in their parameters (no copy from
  // pageable host memory)
  std::vector<float2> twx, twy, wpx(geo.Px / 2), wpy(geo.Py / 2);
  noalloc_engine_twiddles(geo.Px / 2, twx);
  noalloc_engine_twiddles(geo.Py / 2, twy);
  for (int q = 0; q < geo.Px / 2; ++q) wpx[q] = unit_root(q, geo.Px);
  for (int q = 0; q < geo.Py / 2; ++q) wpy[q] = unit_root(q, geo.Py);
  std::vector<unsigned char> img;
  const size_t o_twx = put(img, twx), o_twy = put(img, twy), o_wpx = put(img, wpx), o_wpy = put(img, wpy);
  if (img.size() > tw_bytes) return fail(TOP_ERR_INTERNAL, "static twiddle image above its reserved size");
  img.resize((img.size() + 7) & ~size_t(7));
  TOP_CUDA(launch_put(base, img.data(), img.size(), st), "static twiddles");

  PassParams p{};
  p.ny = geo.ny;
  p.nx = geo.nx;
  p.Py = geo.Py;
  p.Px = geo.Px;
  p.My = geo.Py / 2;
  p.Mx = geo.Px / 2;
  p.oy = geo.oy;
  p.ox = geo.ox;
  p.tune_rows = tune_flags(geo.Px / 2);
  p.tune_cols = tune_flags(geo.Py / 2);
  p.method = g->method;
  p.adjoint = 0;
  p.src_kind = SRC_FIELD;
  p.epi_kind = EPI_FIELD;
  p.twx = reinterpret_cast<const float2*>(base + o_twx);
  p.twy = reinterpret_cast<const float2*>(base + o_twy);
  p.wpx = reinterpret_cast<const float2*>(base + o_wpx);
  p.wpy = reinterpret_cast<const float2*>(base + o_wpy);
  p.ws = ws;
  p.ws_stride = (long long)geo.Px * geo.ny;
  p.in_stride = plane;
  p.out_stride = plane;
  p.psi_stride = plane;
  p.xs_stride = plane;
  p.gI_stride = plane;
  p.outf_stride = plane;
  p.part_stride = plane;
  p.group = 1;
  p.src_group = 1;
  p.in_repeat = 1;

  std::vector<std::pair<uint64_t, uint64_t>> keys;
  int64_t pos = 0;
  while (pos < B) {
    // fields of this chunk and their distinct (lambda, z) sets, one table slot each
    keys.clear();
    int64_t n = 0;
    while (pos + n < B && n < chunk) {
      const int64_t i = n_lz == 1 ? 0 : pos + n;
      const std::pair<uint64_t, uint64_t> key{bits(lam[i]), bits(z[i])};
      size_t k = 0;
      while (k < keys.size() && keys[k] != key) ++k;
      if (k == keys.size()) {
        if ((int)keys.size() == slots) break;
        keys.push_back(key);
        float2* hq = reinterpret_cast<float2*>(base + tw_bytes + k * set_bytes);
        TOP_CUDA(launch_transfer_table(hq, geo.Py, geo.Px, g->dy, g->dx, lam[i], z[i], g->method, st), "transfer table");
        FieldSet fs{};
        fs.hq = hq;
        p.sets[k] = fs;
      }
      p.set_of[n] = (unsigned char)k;
      ++n;
    }
    p.nsets = int(keys.size());
    p.nfields = int(n);
    p.in = static_cast<const float2*>(in) + pos * plane;
    p.out = static_cast<float2*>(out) + pos * plane;
    if (onchip_supported(p) && !(tune_flags(p.Mx) & TOP_TUNE_THREE_PASS)) {
      // 64 x 64 fields at padding 2: the on-chip kernel, as top_propagate runs them
      TOP_CUDA(launch_onchip(p, st), "on-chip propagation");
      pos += n;
      continue;
    }
    TOP_CUDA(launch_pass(PASS_ROWS_FWD, p.Mx, p, st), "rows forward pass");
    TOP_CUDA(launch_pass(PASS_COLS, p.My, p, st), "column pass");
    TOP_CUDA(launch_pass(PASS_ROWS_INV, p.Mx, p, st), "rows inverse pass");
    pos += n;
  }
  return TOP_OK;
}

}  // namespace

extern "C" top_status top_propagate_noalloc(const top_grid* g, const void* in, void* out, const double* lambda,
                                            const double* z, int64_t n_lz, void* stream) {
  return propagate_noalloc(g, in, out, lambda, z, n_lz, static_cast<cudaStream_t>(stream));
}
