// Internal types and device helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/fstat.h"

namespace fstat {

// ---------------------------------------------------------------- constants
constexpr int kMaxDet = FSTAT_MAX_DET;
constexpr int kSkyBlock = 256;      // threads per block of the per-SSB-sample kernel
constexpr int kMinLog2 = 5;         // FFT pass lengths 32 .. 4096 (pass B rows)
constexpr int kMaxLog2 = 12;
constexpr int kMaxLog2A = 13;       // pass A columns up to 8192 (FP32 plans)

// Per-sky constants, written by k_sky_setup / k_sky_finalize (device memory).
struct SkyConst {
  double alpha, delta;
  double cos_alpha, sin_alpha;
  double nx, ny, nz;          // unit vector to the source
  double t_b0;                // start of the SSB grid
  double j_ref;               // (t_ref - t_b0) / dt
  // antenna patterns a = sum_i ca[X][i] h_i, b = sum_i cb[X][i] h_i with
  // h = (1, cos 2H, sin 2H, cos H, sin H), H = alpha - (lon + ph0 + W_rot t)
  double ca[kMaxDet][5];
  double cb[kMaxDet][5];
  double A, B, C, D;
  double kA, kB, kC;          // 2A/D, 2B/D, 4C/D  (2F = kB|Fa|^2 + kA|Fb|^2 - kC Re FaFb*)
  float kAf, kBf, kCf;
};

// Per-template spindown phase polynomial in s = j - J (J = rint(j_ref)):
// phi(s) = p0 + p1 s + p2 s^2 + p3 s^3 cycles.  Double-float split for the
// FP32 path (hi + lo carries ~48 bits), FP64 for the FP64 path.
struct TmplCoef {
  float hi[4], lo[4];
  double p[4];
  int J;
  int pad_;
};

// Spindown phase polynomial of one template (eqs. Fa, Fb: Phi_s =
// 2 pi (f1dot tau^2/2 + f2dot tau^3/6)) for samples j with tau_j = (j - jr) dt,
// expanded in s = j - J.  J is the integer nearest jr clamped into the data
// [0, n - 1], so |s| < n < 2^24 stays exact in FP32 wherever the reference
// time lies; p0, a phase common to every sample that cancels in 2F, is
// reduced mod 1.
__host__ __device__ inline TmplCoef spin_coef(double jr, int64_t n, double dt, double f1dot, double f2dot) {
  double J = rint(jr);
  if (!(J >= 0.0)) J = 0.0;
  if (J > (double)(n - 1)) J = (double)(n - 1);
  const double e = jr - J;  // tau_j = (s - e) dt
  const double c2 = f1dot * dt * dt / 2.0;
  const double c3 = f2dot * dt * dt * dt / 6.0;
  TmplCoef c;
  c.p[3] = c3;
  c.p[2] = c2 - 3.0 * c3 * e;
  c.p[1] = -2.0 * c2 * e + 3.0 * c3 * e * e;
  const double p0 = c2 * e * e - c3 * e * e * e;
  c.p[0] = p0 - rint(p0);
  for (int q = 0; q < 4; ++q) {
    const float h = (float)c.p[q];
    c.hi[q] = h;
    c.lo[q] = (float)(c.p[q] - (double)h);
  }
  c.J = (int)J;
  c.pad_ = 0;
  return c;
}

// Largest spindown phase excursion over the data (cycles) that the FP32
// path's double-float evaluation reduces mod 1 exactly (its reduced phase
// then stays within [-0.57, 0.57] cycles).  tmax bounds |tau| over the data
// samples; twice max |Phi_s| / 2 pi bounds the excursion.
constexpr double kMaxSpinCycles = 1048576.0;  // 2^20
inline bool spin_in_range(double tmax, double f1dot, double f2dot) {
  const double b = fabs(f1dot) * tmax * tmax + fabs(f2dot) * tmax * tmax * tmax / 3.0;
  return b < kMaxSpinCycles;
}

// Streaming multiprocessors of the current device (host; cached per device).
int device_sm_count();

// One entry of the sky-independent timing table (sky.cu): cos, sin of the
// orbital phase and of the sidereal rotation angle.
struct alignas(32) TimeTab {
  double co, so, cq, sq;
};

// Per-sky timing at one node (see Geo::nodes).
struct alignas(32) SkyNode {
  double tm_det;  // t_m,X(t0 + j dt)
  double v;       // (T - t0) / dt - j, T + t_m,X(T) = t_b^j
  double a, b;    // antenna patterns at T
};
// The same nodes for the FP32 (mixed-precision) path: v = vi + vf with
// vi = rint(v) exact and |vf| <= 1/2 in FP32, dv = v(next node) - v (small:
// the delay's change over kNodeStep samples), a, b in FP32; and the step-iii
// phase f_h t_m at the detector-time node as its fraction phf (|phf| <= 1/2)
// and its change to the next node dph (below a cycle), both formed in FP64.
struct alignas(32) NodeF32 {
  float a, b, vf, dv;
  int vi;
  float phf, dph;
  int pad_;
};
constexpr int kNodeStep = 16;  // samples between timing nodes
inline int sky_nodes(int64_t n) { return (int)((n + kNodeStep - 1) / kNodeStep) + 3; }

// Geometry constants for one plan (kernel argument, by value).
struct Geo {
  double c, au, r_earth, w_rot, w_orb, cos_obl, sin_obl, orb_ph0, sid_ph0;
  double lat[kMaxDet], lon[kMaxDet], gam[kMaxDet];
  double rcl[kMaxDet], rsl[kMaxDet];   // r_earth cos(lat), r_earth sin(lat)
  double w[kMaxDet];                   // noise weights of the rescaled series, sigma_ref^2 / (2 sigma_X^2)
  double inv_sigma_ref;                // z is stored divided by sigma_ref (smallest sigma_X)
  double t0, dt, f_het, t_ref;
  int64_t n;                           // samples per detector
  int n_det, dterms;
  int interp;                          // FSTAT_INTERP_*
  double clon[kMaxDet], slon[kMaxDet]; // cos, sin of the longitudes
  // Sky-independent timing table (sky.cu): cos, sin of the orbital phase and
  // of the sidereal rotation angle at t = tab_t0 + i / tab_inv_h.
  const TimeTab* tab;
  double tab_t0, tab_inv_h;
  int tab_n;
  // Roemer delay t_m of the current sky position for each detector on the
  // same grid, [X * tab_n + i] (rewritten by every per-sky run)
  double* tm_tab;
  // Per-sky timing nodes every kNodeStep samples (sky.cu), [X * n_nodes + m]
  // for sample j = (m - 1) kNodeStep: t_m at the detector time, and at the
  // SSB epoch the delay correction v = u - j and the antenna patterns a, b
  SkyNode* nodes;
  NodeF32* nodes32;                    // the same nodes in FP32 (mixed path)
  int n_nodes;
};

// ---------------------------------------------------- pair of complex values
// The two transforms Fa and Fb of one template share every index and
// twiddle, so kernels carry them together: (a.re, a.im, b.re, b.im).
template <typename T> struct Pair { T ar, ai, br, bi; };

template <typename T> __device__ __forceinline__ Pair<T> padd(const Pair<T>& x, const Pair<T>& y) {
  return {x.ar + y.ar, x.ai + y.ai, x.br + y.br, x.bi + y.bi};
}
template <typename T> __device__ __forceinline__ Pair<T> psub(const Pair<T>& x, const Pair<T>& y) {
  return {x.ar - y.ar, x.ai - y.ai, x.br - y.br, x.bi - y.bi};
}
// multiply both members by the complex number (c, s)
template <typename T> __device__ __forceinline__ Pair<T> pmul(const Pair<T>& x, T c, T s) {
  return {x.ar * c - x.ai * s, x.ar * s + x.ai * c, x.br * c - x.bi * s, x.br * s + x.bi * c};
}
// multiply by -i
template <typename T> __device__ __forceinline__ Pair<T> pmul_mi(const Pair<T>& x) {
  return {x.ai, -x.ar, x.bi, -x.br};
}
template <typename T> __device__ __forceinline__ Pair<T> pzero() { return {T(0), T(0), T(0), T(0)}; }

// memory images: float pair = float4 (16 B); double pair = 2 x double2 (32 B)
template <typename T> struct PairMem;
template <> struct PairMem<float> { using type = float4; };
template <> struct PairMem<double> { struct alignas(16) type { double2 a, b; }; };

__device__ __forceinline__ Pair<float> pload(const float4* p) {
  float4 v = *p; return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ void pstore(float4* p, const Pair<float>& x) {
  *p = make_float4(x.ar, x.ai, x.br, x.bi);
}
__device__ __forceinline__ Pair<double> pload(const PairMem<double>::type* p) {
  double2 a = p->a, b = p->b; return {a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ void pstore(PairMem<double>::type* p, const Pair<double>& x) {
  p->a = make_double2(x.ar, x.ai); p->b = make_double2(x.br, x.bi);
}
__device__ __forceinline__ Pair<float> pload_g(const float4* __restrict__ p) {
  float4 v = __ldg(p); return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Pair<double> pload_g(const PairMem<double>::type* __restrict__ p) {
  double2 a = __ldg(&p->a), b = __ldg(&p->b); return {a.x, a.y, b.x, b.y};
}

__device__ __forceinline__ void sincospi_t(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void sincospi_t(double x, double* s, double* c) { sincospi(x, s, c); }

// ------------------------------------------------------------ host helpers
void launch_sky(const Geo& g, int precision, double alpha, double delta, const void* const* xh,
                const int* xh_dtype, void* z, void* G, int n1, int64_t lc, double* partials,
                int n_blocks, SkyConst* sky, int* err, cudaStream_t st);
// Timing table: entries needed to cover [t_lo, t_hi] at spacing h, and the
// kernel that fills them (FP64 sincos, once per plan).
int time_table_entries(double t_lo, double t_hi, double h);
cudaError_t launch_time_table(const Geo& g, TimeTab* tab, cudaStream_t st);
void launch_tmpl_coef(const SkyConst* sky, double dt, int64_t n, const fstat_template* tmpl,
                      const int* order, int first, int count, TmplCoef* out, cudaStream_t st);
void launch_check_finite(const void* x, int dtype, int64_t n, int* err, cudaStream_t st);
// Gradient (adjoint.cu): per-plan sample tables and per-call scratch.
size_t grad_table_bytes(int n_det, int64_t n);
cudaError_t launch_grad_tables(const Geo& g, const void* const* xh, const int* dtype, void* base,
                               cudaStream_t st);
size_t grad_scratch_bytes(int n_cand, const Geo& g);
cudaError_t launch_grad(const Geo& g, const void* tables, const fstat_candidate* cand_dev, int n_cand,
                        void* scratch, float* twoF, float* grad, cudaStream_t st);

// Twiddle tables (tables.cu): pointers into one device block.
struct TwiddleTables {
  const void* a;   // pass A Stockham roots, N2 entries
  const void* b;   // pass B Stockham roots, N1 entries
  size_t bytes;
};
TwiddleTables twiddle_layout(int precision, int log2n1, int log2n2, void* base);
cudaError_t build_twiddles(int precision, int log2n1, int log2n2, void* base, cudaStream_t st);

// Arguments of pass B's other epilogues: peaks mode reduces one template's
// 2F in the kernel instead of writing it bin by bin (fstat_compute_peaks);
// accumulate mode adds it to a row at a bin offset (fstat_semicoherent).
struct PeakArgs {
  unsigned long long* band_key;  // this template's row of band keys, or nullptr
  fstat_peak* peaks;             // crossing list [cap]
  unsigned long long* count;     // list counter, or nullptr (no list)
  long long cap;
  long long tmpl;                // template index stored with each crossing
  float thr;
  int log2_band;                 // log2(bins per band)
  int shift;                     // accumulate: bin m adds to bin m - shift
  int* err;                      // where a pass records FSTAT_ERR_TIMEOUT, or nullptr
  int wait_limit;                // polls of a tile's first bulk-copy wait (<= 0 with
                                 // wait_set: give up at once; unset: the default)
  int wait_set;
};

// Band key: order-preserving image of the float 2F in the high word, the
// complement of the bin in the low word, so an unsigned maximum picks the
// largest 2F and, among equal values, the smallest bin.  0 = no value.
__device__ __forceinline__ unsigned long long band_key(float v, unsigned bin) {
  unsigned u = __float_as_uint(v);
  u ^= (u & 0x80000000u) ? 0xffffffffu : 0x80000000u;
  return ((unsigned long long)u << 32) | (unsigned long long)(0xffffffffu - bin);
}

// FFT passes; ca / cb = columns / rows per CTA (0 = default for the length),
// va / vb = radix schedule: bit 0 radix-8 first, bit 1 single shared
// buffer, bit 2 (pass B) tiles by bulk tensor copies, bit 3 (pass A) three
// CTAs per SM, va 16 (8192-point columns) the next column's samples staged
// by a bulk copy under the transform.  res > 0: persistent grid of at most
// res CTAs per SM (0 = every resident CTA).  err: where a pass records a
// timed-out wait (FSTAT_ERR_TIMEOUT), or nullptr; wait_limit >= 0: polls of
// pass A's staged-column waits (timeout tests).
cudaError_t launch_pass_a_f32(int log2_n2, int ca, int va, const void* G, int64_t lc, int64_t n, int n1,
                              const void* twA, const TmplCoef* coef, void* Z, cudaStream_t st, int res = 0,
                              int* err = nullptr, int wait_limit = -1);
// pk == nullptr: write 2F to out[n_fft]; otherwise reduce it as pk says.
// err: where a pass records a timed-out wait (FSTAT_ERR_TIMEOUT), or nullptr
// wait_limit >= 0: polls of each tile's first bulk-copy wait (timeout tests)
cudaError_t launch_pass_b_f32(int log2_n1, int cb, int vb, const void* Z, int n2, const void* twB,
                              const SkyConst* sky, float* out, cudaStream_t st,
                              const PeakArgs* pk = nullptr, int res = 0, int* err = nullptr,
                              int wait_limit = -1);
cudaError_t launch_pass_a_f64(int log2_n2, int ca, int va, const void* G, int64_t lc, int64_t n, int n1,
                              const void* twA, const TmplCoef* coef, void* Z, cudaStream_t st, int res = 0,
                              int* err = nullptr, int wait_limit = -1);
cudaError_t launch_pass_b_f64(int log2_n1, int cb, int vb, const void* Z, int n2, const void* twB,
                              const SkyConst* sky, float* out, cudaStream_t st,
                              const PeakArgs* pk = nullptr, int res = 0, int* err = nullptr,
                              int wait_limit = -1);
cudaError_t launch_pass_b_peak_f32(int log2_n1, int cb, int vb, const void* Z, int n2, const void* twB,
                                   const SkyConst* sky, const PeakArgs& pk, cudaStream_t st, int res = 0);
cudaError_t launch_pass_b_peak_f64(int log2_n1, int cb, int vb, const void* Z, int n2, const void* twB,
                                   const SkyConst* sky, const PeakArgs& pk, cudaStream_t st, int res = 0);
// Accumulate mode: out[m - shift] += 2F[m] for 0 <= m - shift < n_fft.
cudaError_t launch_pass_b_acc_f32(int log2_n1, int cb, int vb, const void* Z, int n2, const void* twB,
                                  const SkyConst* sky, float* out, int shift, cudaStream_t st, int res = 0,
                                  int* err = nullptr, int wait_limit = -1);
cudaError_t launch_pass_b_acc_f64(int log2_n1, int cb, int vb, const void* Z, int n2, const void* twB,
                                  const SkyConst* sky, float* out, int shift, cudaStream_t st, int res = 0,
                                  int* err = nullptr, int wait_limit = -1);
// PeakArgs' wait fields from a plan's setting (< 0: the default limit)
inline void set_wait(PeakArgs& a, int wait_limit) {
  a.wait_set = wait_limit >= 0;
  a.wait_limit = wait_limit >= 0 ? wait_limit : 0;
}
// One persistent launch of both FFT passes over T templates of one sky
// group (fft_fused.cuh).  kRing intermediates in flight; launch state of
// queue_ints(T) ints, zeroed before every launch.
constexpr int kRing = 3;
constexpr int kQueueHead = 4;
inline size_t queue_ints(int T) { return (size_t)kQueueHead + 2 * (size_t)T; }

struct FusedArgs {
  const float4* G;        // column-major resampled pairs (per-sky work)
  int64_t lc;             // column length of G
  int n;                  // samples
  int n1, n2;             // split: n1 columns of n2 points (pass A), n2 rows of n1 points (pass B)
  const TmplCoef* coef;   // [T] spindown coefficients of the launch's templates
  const int* ord;         // [T] caller's template index of each (row = ord mod out_rows)
  int64_t out_rows;
  float* out;             // 2F rows of n1 * n2 floats
  const SkyConst* sky;
  float4* Z[kRing];       // intermediates
  int* q;                 // launch state (queue_ints(T) ints)
  int T;
  int na, nb, total;      // tiles per template of pass A, of pass B; items in the launch
  int* err;               // sticky error of the plan
  int wait_limit;         // polls of the first waits (when wait_set), else the defaults
  int wait_set;
};

// The fused launch for FP32 plans, compiled for the splits fused_supported
// names (cudaErrorInvalidConfiguration otherwise).
bool fused_supported(int log2n1, int log2n2);
cudaError_t launch_fused_f32(int log2n1, int log2n2, const FusedArgs& a, cudaStream_t st);

// Band keys of n rows x n_bands -> maximum 2F and its bin (band_bin may be null).
cudaError_t launch_band_decode(const unsigned long long* keys, int64_t count, float* band_max,
                               int32_t* band_bin, cudaStream_t st);

}  // namespace fstat
