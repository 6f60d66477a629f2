// Per-sky kernels: Sec. 3 steps (iii), (iv), (v) of the resampling method,
// antenna weighting, the noise-weighted detector sum, and the antenna-pattern
// integrals A, B, C, D of eq. (Fstat).  The result G = (G_a, G_b) is stored
// in the column-major layout the FFT pass A reads: element j goes to
// G[(j mod n1) * lc + j / n1].
//
// Timing (t_m, the inversion T + t_m(T) = t_b, u = (T - t0)/dt) is FP64 in
// both precisions; f_h t_m is reduced mod 1 in FP64 before the sincos.

#include <math.h>

#include <algorithm>
#include <cmath>

#include "fstat_internal.cuh"

// Negative control for the parity tests (never in the regular build): with
// FSTAT_NEGCTRL_FP32_TIMING defined, f_h t_m and the sample position
// u = (T - t0) / dt are formed in FP32 instead of FP64, the precision loss
// the FP64 timing exists to prevent.  A test builds this variant separately
// and checks that its 2F fails the tolerance the regular build meets.
#ifdef FSTAT_NEGCTRL_FP32_TIMING
constexpr bool kNegCtrlFp32 = true;
#else
constexpr bool kNegCtrlFp32 = false;
#endif

namespace fstat {

namespace {

struct Rot { double c, s; };  // cos, sin of the detector's sidereal angle

// The orbital phase and the sidereal rotation angle enter the timing only
// through their cosines and sines, which the plan tabulates every 30 s
// (k_time_table, FP64 sincos once per entry) over the span the timing can
// reach.  Per sky position the Roemer delay of each detector is then
// tabulated at the same nodes (k_sky_table), and every timing evaluation
// is the cubic Lagrange interpolation through the four nearest nodes.  The
// interpolation error in t_m is ~1e-14 s (rotation term:
// (w_rot h)^4 * 9/16/24 * R_E/c at h = 30 s), below the FP64 rounding of
// t_m itself.
struct TabPos {
  int i;                      // first of the four nodes
  double w0, w1, w2, w3;      // Lagrange weights
};

__device__ __forceinline__ TabPos tab_pos(const Geo& g, double t) {
  const double x = (t - g.tab_t0) * g.tab_inv_h;
  int i = (int)floor(x) - 1;                       // nodes i .. i + 3
  i = i < 0 ? 0 : (i > g.tab_n - 4 ? g.tab_n - 4 : i);
  const double f = x - (double)(i + 1);            // position from node i + 1
  const double fm = f - 1.0, fp = f + 1.0, f2 = f - 2.0;
  TabPos p;
  p.i = i;
  p.w0 = -f * fm * f2 * (1.0 / 6.0);
  p.w1 = fp * fm * f2 * 0.5;
  p.w2 = -fp * f * f2 * 0.5;
  p.w3 = fp * f * fm * (1.0 / 6.0);
  return p;
}

// Roemer delay t_m,X(t) of the current sky position (Sec. 2 phase model).
__device__ __forceinline__ double tm_eval(const Geo& g, int X, double t) {
  const TabPos p = tab_pos(g, t);
  const double* v = g.tm_tab + (int64_t)X * g.tab_n + p.i;
  return p.w0 * v[0] + p.w1 * v[1] + p.w2 * v[2] + p.w3 * v[3];
}

// t_m,X(t) and its derivative dt_m/dt (derivative of the same cubic)
__device__ __forceinline__ double tm_eval_d(const Geo& g, int X, double t, double* dtm) {
  const TabPos p = tab_pos(g, t);
  const double f = (t - g.tab_t0) * g.tab_inv_h - (double)(p.i + 1);
  const double f2 = f * f;
  const double d0 = -(3.0 * f2 - 6.0 * f + 2.0) * (1.0 / 6.0);
  const double d1 = (3.0 * f2 - 4.0 * f - 1.0) * 0.5;
  const double d2 = -(3.0 * f2 - 2.0 * f - 2.0) * 0.5;
  const double d3 = (3.0 * f2 - 1.0) * (1.0 / 6.0);
  const double* v = g.tm_tab + (int64_t)X * g.tab_n + p.i;
  *dtm = (d0 * v[0] + d1 * v[1] + d2 * v[2] + d3 * v[3]) * g.tab_inv_h;
  return p.w0 * v[0] + p.w1 * v[1] + p.w2 * v[2] + p.w3 * v[3];
}

// cos, sin of detector X's sidereal angle lon + rotation angle at t
__device__ __forceinline__ Rot rot_eval(const Geo& g, int X, double t) {
  const TabPos p = tab_pos(g, t);
  const TimeTab a = g.tab[p.i], b = g.tab[p.i + 1], c = g.tab[p.i + 2], d = g.tab[p.i + 3];
  const double cq = p.w0 * a.cq + p.w1 * b.cq + p.w2 * c.cq + p.w3 * d.cq;
  const double sq = p.w0 * a.sq + p.w1 * b.sq + p.w2 * c.sq + p.w3 * d.sq;
  return Rot{g.clon[X] * cq - g.slon[X] * sq, g.slon[X] * cq + g.clon[X] * sq};
}

__global__ void k_time_table(Geo g, TimeTab* __restrict__ tab) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.tab_n; i += gridDim.x * blockDim.x) {
    const double t = g.tab_t0 + (double)i / g.tab_inv_h;
    double so, co, sq, cq;
    sincos(g.orb_ph0 + g.w_orb * t, &so, &co);
    sincos(g.sid_ph0 + g.w_rot * t, &sq, &cq);
    tab[i] = TimeTab{co, so, cq, sq};
  }
}

// t_m = (r_orb + r_rot) . n / c at every node, for every detector
__global__ void k_sky_table(Geo g, const SkyConst* __restrict__ skyp) {
  const SkyConst& s = *skyp;
  const double py = g.cos_obl * s.ny + g.sin_obl * s.nz;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.tab_n; i += gridDim.x * blockDim.x) {
    const TimeTab e = g.tab[i];
    const double orb = g.au * (e.co * s.nx + e.so * py);
    for (int X = 0; X < g.n_det; ++X) {
      const double cp = g.clon[X] * e.cq - g.slon[X] * e.sq;
      const double sp = g.slon[X] * e.cq + g.clon[X] * e.sq;
      const double rot = g.rcl[X] * (cp * s.nx + sp * s.ny) + g.rsl[X] * s.nz;
      g.tm_tab[(int64_t)X * g.tab_n + i] = (orb + rot) / g.c;
    }
  }
}

// a(t), b(t) from the harmonic coefficients and the sidereal angle (JKS 1998
// eqs. 12-13): H = alpha - phi, h = (1, cos 2H, sin 2H, cos H, sin H).
__device__ __forceinline__ void antenna(const SkyConst& s, int X, const Rot& r, double* a, double* b) {
  const double ca = s.cos_alpha, sa = s.sin_alpha;
  double cH = ca * r.c + sa * r.s;
  double sH = sa * r.c - ca * r.s;
  double c2H = cH * cH - sH * sH;
  double s2H = 2.0 * sH * cH;
  *a = s.ca[X][0] + s.ca[X][1] * c2H + s.ca[X][2] * s2H + s.ca[X][3] * cH + s.ca[X][4] * sH;
  *b = s.cb[X][0] + s.cb[X][1] * c2H + s.cb[X][2] * s2H + s.cb[X][3] * cH + s.cb[X][4] * sH;
}

__global__ void k_sky_setup(Geo g, double alpha, double delta, SkyConst* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  SkyConst s;
  s.alpha = alpha;
  s.delta = delta;
  s.cos_alpha = cos(alpha);
  s.sin_alpha = sin(alpha);
  s.nx = cos(delta) * s.cos_alpha;
  s.ny = cos(delta) * s.sin_alpha;
  s.nz = sin(delta);
  // SSB grid start: t0 + orbital Roemer delay at the data midpoint
  double t_mid = g.t0 + 0.5 * (double)g.n * g.dt;
  double so, co;
  sincos(g.orb_ph0 + g.w_orb * t_mid, &so, &co);
  double orb = g.au * (co * s.nx + so * (g.cos_obl * s.ny + g.sin_obl * s.nz));
  s.t_b0 = g.t0 + orb / g.c;
  s.j_ref = (g.t_ref - s.t_b0) / g.dt;
  double sd = sin(delta), cd = cos(delta), s2d = sin(2.0 * delta), c2d = cos(2.0 * delta);
  for (int X = 0; X < kMaxDet; ++X) {
    for (int i = 0; i < 5; ++i) { s.ca[X][i] = 0.0; s.cb[X][i] = 0.0; }
    if (X >= g.n_det) continue;
    double lam = g.lat[X], gam = g.gam[X];
    double s2g = sin(2.0 * gam), c2g = cos(2.0 * gam);
    double sl = sin(lam), cl = cos(lam), s2l = sin(2.0 * lam), c2l = cos(2.0 * lam);
    s.ca[X][0] = 0.75 * s2g * cl * cl * cd * cd;
    s.ca[X][1] = s2g * (3.0 - c2l) * (3.0 - c2d) / 16.0;
    s.ca[X][2] = -0.25 * c2g * sl * (3.0 - c2d);
    s.ca[X][3] = 0.25 * s2g * s2l * s2d;
    s.ca[X][4] = -0.5 * c2g * cl * s2d;
    s.cb[X][0] = 0.0;
    s.cb[X][1] = c2g * sl * sd;
    s.cb[X][2] = 0.25 * s2g * (3.0 - c2l) * sd;
    s.cb[X][3] = c2g * cl * cd;
    s.cb[X][4] = 0.5 * s2g * s2l * cd;
  }
  s.A = s.B = s.C = s.D = 0.0;
  s.kA = s.kB = s.kC = 0.0;
  s.kAf = s.kBf = s.kCf = 0.0f;
  *out = s;
}

// Cubic Lagrange weights at f = r / kNodeStep between nodes 0 and 1 of
// nodes at -1, 0, 1, 2 (dyadic f: every weight is exact in FP64).
// FP32 tap weights: the quotient by the hardware reciprocal (2 ulp; its
// denominator len sin(pi (d - m)/len) lies between ~pi |d - m| and D + 1),
// and the Hamming taper's sine and cosine of an angle within +-pi/2 by the
// hardware unit (~4e-7 absolute on a factor near 1).  The Dirichlet sines
// themselves keep the accurate sincospi (their arguments can be tiny).  FP64
// keeps exact division and sincospi throughout.
__device__ __forceinline__ float tap_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double tap_div(double a, double b) { return a / b; }
__device__ __forceinline__ void taper_sincospi(float x, float* s, float* c) {
  __sincosf(3.14159265358979323846f * x, s, c);
}
__device__ __forceinline__ void taper_sincospi(double x, double* s, double* c) { sincospi(x, s, c); }

// Per-tap constants of the interpolation kernel, one aligned entry per tap
// m = -D..D: cos, sin(pi m / len) (the Dirichlet denominator by angle
// addition) and cos, sin(pi m / (D + 1)) (the taper).
template <typename T> struct alignas(4 * sizeof(T)) TapK {
  T c, s, tc, ts;
};

__device__ __forceinline__ void node_weights(int r, double* w) {
  const double f = (double)r * (1.0 / kNodeStep);
  const double fm = f - 1.0, fp = f + 1.0, f2 = f - 2.0;
  w[0] = -f * fm * f2 * (1.0 / 6.0);
  w[1] = fp * fm * f2 * 0.5;
  w[2] = -fp * f * f2 * 0.5;
  w[3] = fp * f * fm * (1.0 / 6.0);
}

// Timing nodes of the current sky position (FP64, every kNodeStep samples,
// from sample -kNodeStep on): the Roemer delay at the detector time, and at
// the SSB epoch t_b^j the detector epoch T (T + t_m(T) = t_b^j: the
// fixed-point start T0 = t_b - t_m(t_b), then one Newton step; |dt_m/dT|
// ~ 1e-4 puts T0 within ~0.05 s of the root and |d2t_m/dT2| ~ 1e-10 /s the
// Newton step within ~1e-13 s of it, the root three fixed-point iterations
// reach), stored as v = (T - t0)/dt - j, and the antenna patterns at T.
// Between nodes every per-sample quantity is the cubic interpolant through
// the four nearest nodes: t_m, T and a, b are smooth on the scale of the
// node spacing (rotation: (w_rot h)^4 R_E/c ~ 1e-14 s at h = 32 s), so the
// interpolation error is below the FP64 rounding of the quantities.
__global__ void k_sky_nodes(Geo g, const SkyConst* __restrict__ skyp) {
  const SkyConst& s = *skyp;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < g.n_nodes; m += gridDim.x * blockDim.x) {
    const double j = (double)(m - 1) * kNodeStep;
    const double td = g.t0 + j * g.dt;
    const double tb = s.t_b0 + j * g.dt;
    for (int X = 0; X < g.n_det; ++X) {
      double T_ = tb - tm_eval(g, X, tb);
      {
        double dtm;
        const double tm = tm_eval_d(g, X, T_, &dtm);
        T_ -= (T_ + tm - tb) / (1.0 + dtm);
      }
      SkyNode nd;
      nd.tm_det = tm_eval(g, X, td);
      nd.v = (T_ - g.t0) / g.dt - j;
      antenna(s, X, rot_eval(g, X, T_), &nd.a, &nd.b);
      g.nodes[(int64_t)X * g.n_nodes + m] = nd;
    }
  }
}

// FP32 image of the nodes for the mixed path (NodeF32): the delay split
// into its exact integer part and an FP32 fraction, and its FP32 change to
// the next node, formed in FP64 from the FP64 nodes.
__global__ void k_sky_nodes32(Geo g) {
  const int64_t total = (int64_t)g.n_det * g.n_nodes;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int m = (int)(i % g.n_nodes);
    const SkyNode nd = g.nodes[i];
    const bool next = m + 1 < g.n_nodes;
    NodeF32 f;
    const double vi = rint(nd.v);
    f.a = (float)nd.a;
    f.b = (float)nd.b;
    f.vi = (int)vi;
    f.vf = (float)(nd.v - vi);
    f.dv = next ? (float)(g.nodes[i + 1].v - nd.v) : 0.f;
    const double ph = g.f_het * nd.tm_det;
    f.phf = (float)(ph - rint(ph));
    f.dph = next ? (float)(g.f_het * (g.nodes[i + 1].tm_det - nd.tm_det)) : 0.f;
    f.pad_ = 0;
    g.nodes32[i] = f;
  }
}

// Step (iii): z = x_h exp(-i 2 pi frac(f_h t_m(t_k))), stored divided by a
// common sigma_ref.  Rescaling every detector's series by the same factor,
// with weights w_X = sigma_ref^2 / (2 sigma_X^2), scales G by sigma_ref and
// A, B, C by sigma_ref^2, which leaves eq. (Fstat) unchanged while every FP32
// value stays O(1) whatever the units of x_h (strain-scaled data would
// overflow 1/(2 sigma^2) and |Fa|^2 in FP32).  t_m from the timing nodes.
template <typename TIn, typename TZ>
__global__ void k_detector_phase(Geo g, int X, const TIn* __restrict__ xh, TZ* __restrict__ z) {
  __shared__ double s_w[kNodeStep][4];  // the node weights, by sample mod kNodeStep
  __shared__ float s_wf[kNodeStep][4];
  if (threadIdx.x < kNodeStep) {
    node_weights(threadIdx.x, s_w[threadIdx.x]);
#pragma unroll
    for (int q = 0; q < 4; ++q) s_wf[threadIdx.x][q] = (float)s_w[threadIdx.x][q];
  }
  __syncthreads();
  // FP32 path: the phase's fraction from the FP32 node image (the cubic
  // written about the segment's node, |result| <~ 1/2 before the final
  // reduction); FP64 plans and the negative control form f_h t_m in FP64
  constexpr bool kSplit = sizeof(TZ) == sizeof(float2) && !kNegCtrlFp32;
  const SkyNode* nd = g.nodes + (int64_t)X * g.n_nodes;
  const NodeF32* nf32 = g.nodes32 + (int64_t)X * g.n_nodes;
  const float isf = (float)g.inv_sigma_ref;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < g.n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = k / kNodeStep + 1;
    double ph = 0.0;  // FP64 path: the phase in cycles, in [0, 1)
    float phs = 0.f;  // FP32 path: the same, in [-1/2, 1/2]
    if constexpr (kSplit) {
      const float* wf = s_wf[k % kNodeStep];
      const NodeF32* nf = nf32 + m;
      const float d0 = nf[0].dph;
      const float p = nf[0].phf + ((wf[2] * d0 + wf[3] * (d0 + nf[1].dph)) - wf[0] * nf[-1].dph);
      phs = p - rintf(p);
    } else {
      const double* w = s_w[k % kNodeStep];
      const double tm = w[0] * nd[m - 1].tm_det + w[1] * nd[m].tm_det + w[2] * nd[m + 1].tm_det + w[3] * nd[m + 2].tm_det;
      ph = g.f_het * tm;
      if constexpr (kNegCtrlFp32) ph = (double)((float)g.f_het * (float)tm);
      ph -= floor(ph);
    }
    TIn x = xh[k];
    const double is = g.inv_sigma_ref;
    if constexpr (kSplit) {
      float sn, cs;
      sincospif(2.0f * phs, &sn, &cs);
      float xr, xi;
      if constexpr (sizeof(TIn) == sizeof(float2)) {
        xr = x.x * isf;
        xi = x.y * isf;
      } else {
        xr = (float)((double)x.x * is);
        xi = (float)((double)x.y * is);
      }
      z[k] = make_float2(xr * cs + xi * sn, xi * cs - xr * sn);
    } else if constexpr (sizeof(TZ) == sizeof(float2)) {
      float sn, cs;
      sincospif(2.0f * (float)ph, &sn, &cs);
      float xr = (float)((double)x.x * is), xi = (float)((double)x.y * is);
      z[k] = make_float2(xr * cs + xi * sn, xi * cs - xr * sn);
    } else {
      double sn, cs;
      sincospi(2.0 * ph, &sn, &cs);
      double xr = (double)x.x * is, xi = (double)x.y * is;
      z[k] = make_double2(xr * cs + xi * sn, xi * cs - xr * sn);
    }
  }
}

// Steps (iv) + (v) + antenna weighting + detector sum, one SSB sample per
// thread.  The sample positions u(j) of a block's kSkyBlock consecutive SSB
// samples increase with j and span kSkyBlock samples give or take the
// delay's drift, so the block stages the detector samples its taps can
// touch, [rint(u_first) - D, rint(u_last) + D] (rounded out to float4
// boundaries), in shared memory with coalesced 16-byte loads, and the taps
// read them from there.  The tap weights W(d - m) use angle addition from
// per-block tables of cos, sin(pi m / len) and of the taper's
// cos, sin(pi m / (D + 1)), m = -D..D: two sine/cosine evaluations per
// sample instead of two per tap.
//
// FP64 work per sample is kept to what needs it: the sample position u and
// a, b for the weighted sum G come from the FP32 image of the nodes in the
// mixed path (u's integer part exact, its fraction to ~6e-8 samples; G
// itself is FP32; the FP64 path keeps FP64 throughout);
// and A, B, C per 16-sample segment: with a(r) = sum_q W_rq a_q the cubic
// interpolant of the segment's four node values a_q, the segment's
// sum_r a(r)^2 is the quadratic form a^T M a with M = sum_r W_r W_r^T
// (and likewise b^T M b, a^T M b), exact algebra in FP64, one thread per
// detector and segment after the sample loop; segments with invalid
// samples (the data's edges) sum per sample.
constexpr int kMaxD = 32;
constexpr int kWin = kSkyBlock + 2 * kMaxD + 8;  // staged window, samples (covers the drift); even
static_assert(kWin % 2 == 0, "whole 16-byte loads of complex64 samples");

template <typename T, typename TZ>
__global__ void __launch_bounds__(kSkyBlock)
k_resample(Geo g, const SkyConst* __restrict__ skyp, const TZ* __restrict__ z,
           typename PairMem<T>::type* __restrict__ G, int n1, int64_t lc, double* __restrict__ partials) {
  (void)skyp;  // the sky position enters through the timing nodes
  __shared__ __align__(16) TZ win[kWin];
  __shared__ TapK<T> tk[2 * kMaxD + 1];
  __shared__ long long s_span[2];
  __shared__ double s_w[kNodeStep][4], s_m[4][4];  // node weights by j mod kNodeStep; segment matrix M
  __shared__ float s_wf[kNodeStep][4];
  __shared__ bool s_full[kMaxDet][kSkyBlock / kNodeStep];  // segment fully valid, per detector
  static_assert(kSkyBlock % 32 == 0 && kNodeStep == 16, "two whole segments per warp");
  static_assert(kMaxDet * (kSkyBlock / kNodeStep) <= kSkyBlock, "one thread per detector and segment");
  const int D = g.dterms;
  const T nT = (T)g.n;
  // Dirichlet kernel of the full series (length N) or of the 2D + 1 taps
  // themselves; the Hamming taper only for the default kernel
  const T len = g.interp == FSTAT_INTERP_PERIODIC ? (T)(2 * D + 1) : nT;
  const bool taper = g.interp == FSTAT_INTERP_TAPERED;
  const T inv_taper = (T)1 / (T)(D + 1);
  for (int m = threadIdx.x; m <= 2 * D; m += blockDim.x) {
    T sn, cs;
    TapK<T> q;
    sincospi_t((T)(m - D) / len, &sn, &cs);
    q.c = cs;
    q.s = sn;
    sincospi_t((T)(m - D) * inv_taper, &sn, &cs);
    q.tc = cs;
    q.ts = sn;
    tk[m] = q;
  }
  if (threadIdx.x < kNodeStep) {
    node_weights(threadIdx.x, s_w[threadIdx.x]);
#pragma unroll
    for (int q = 0; q < 4; ++q) s_wf[threadIdx.x][q] = (float)s_w[threadIdx.x][q];
  }
  __shared__ float s_wx[kMaxDet];  // noise weights in FP32 (the mixed path's G)
  if (threadIdx.x < g.n_det) s_wx[threadIdx.x] = (float)g.w[threadIdx.x];
  __syncthreads();
  if (threadIdx.x < 16) {
    const int q = threadIdx.x >> 2, r2 = threadIdx.x & 3;
    double m = 0.0;
    for (int r = 0; r < kNodeStep; ++r) m += s_w[r][q] * s_w[r][r2];
    s_m[q][r2] = m;  // visible after the barriers in the detector loop
  }
  const int64_t j0 = (int64_t)blockIdx.x * blockDim.x;
  int64_t j = j0 + threadIdx.x;
  const int64_t j_last = min(j0 + (int64_t)blockDim.x, g.n) - 1;
  const double* wn = s_w[j % kNodeStep];
  const float* wf = s_wf[j % kNodeStep];
  const unsigned lane = threadIdx.x & 31;
  double sa = 0.0, sb = 0.0, sab = 0.0;
  bool summed = false;  // this thread added to sa, sb, sab
  Pair<T> acc = pzero<T>();
  for (int X = 0; X < g.n_det; ++X) {
    // steps (iv)-(v): the sample position u of T (T + t_m(T) = t_b^j) and
    // the antenna patterns at T, interpolated between the timing nodes
    const int64_t node0 = (int64_t)X * g.n_nodes + (min(j, j_last) / kNodeStep + 1);
    const SkyNode* nd = g.nodes + node0;
    // k0 = rint(u) and dlt = u - k0 for u = j + v.  FP32 path: v = vi + vf
    // at this segment's node, plus the weighted node-to-node changes (the
    // interpolating cubic written about that node), so the integer part is
    // exact and only the fraction, |f| <~ 1/2, is rounded to FP32.  FP64
    // plans (and the FP32-timing negative control) form u in FP64.
    long long k0;
    T dlt;
    if constexpr (sizeof(T) == sizeof(float) && !kNegCtrlFp32) {
      const NodeF32* nf = g.nodes32 + node0;
      const float dv0 = nf[0].dv;
      const float f = nf[0].vf + ((wf[2] * dv0 + wf[3] * (dv0 + nf[1].dv)) - wf[0] * nf[-1].dv);
      const float rf = rintf(f);
      k0 = j + nf[0].vi + (long long)rf;
      dlt = f - rf;
    } else {
      double u = (double)j + (wn[0] * nd[-1].v + wn[1] * nd[0].v + wn[2] * nd[1].v + wn[3] * nd[2].v);
      if constexpr (kNegCtrlFp32) u = (double)((float)j + (float)(u - (double)j));
      k0 = __double2ll_rn(u);
      dlt = (T)(u - (double)k0);
    }
    // the block's window of detector samples (u is monotonic in j)
    __syncthreads();  // the previous detector's window has been read
    if (j == j0) s_span[0] = k0;
    if (j == j_last) s_span[1] = k0;
    __syncthreads();
    constexpr int PER = 16 / (int)sizeof(TZ);          // samples per 16-byte load
    // window start rounded down so that the element index X n + lo in the
    // series buffer (16-byte aligned base) is a multiple of PER
    long long lo = s_span[0] - D;
    lo -= (((int64_t)X * g.n + lo) % PER + PER) % PER;
    long long hi = s_span[1] + D;
    if (hi - lo + 1 > kWin) hi = lo + kWin - 1;       // drift beyond the window: taps past it read global
    const TZ* zx = z + (int64_t)X * g.n;
    {
      const long long n_vec = (hi - lo + PER) / PER;
      for (long long q = threadIdx.x; q < n_vec; q += blockDim.x) {
        const long long k = lo + q * PER;
        if (k >= 0 && k + PER <= g.n) {
          *reinterpret_cast<float4*>(win + q * PER) = *reinterpret_cast<const float4*>(zx + k);
        } else {
#pragma unroll
          for (int e = 0; e < PER; ++e) {
            const long long kk = k + e;
            TZ v{};
            if (kk >= 0 && kk < g.n) v = zx[kk];
            win[q * PER + e] = v;
          }
        }
      }
    }
    __syncthreads();
    // A, B, C: fully valid 16-sample segments are summed after this loop
    // (one thread per detector and segment); the others per sample here
    const bool valid = j < g.n && k0 >= 0 && k0 <= g.n - 1;
    const unsigned vmask = __ballot_sync(0xffffffffu, valid);
    const bool seg_full = ((vmask >> (lane & 16u)) & 0xffffu) == 0xffffu;
    if ((lane & 15u) == 0) s_full[X][threadIdx.x / kNodeStep] = seg_full;
    const double w = g.w[X];
    if (!seg_full && valid) {
      const double a = wn[0] * nd[-1].a + wn[1] * nd[0].a + wn[2] * nd[1].a + wn[3] * nd[2].a;
      const double b = wn[0] * nd[-1].b + wn[1] * nd[0].b + wn[2] * nd[1].b + wn[3] * nd[2].b;
      summed = true;
      sa += w * a * a;
      sb += w * b * b;
      sab += w * a * b;
    }
    if (!valid) continue;

    auto tap = [&](long long k) -> TZ {
      const long long i = k - lo;
      return (i >= 0 && i < kWin) ? win[i] : zx[k];
    };
    T zr = 0, zi = 0;
    if (dlt == (T)0) {
      TZ v = tap(k0);
      zr = (T)v.x;
      zi = (T)v.y;
    } else {
      T d = dlt, sd, cd_, sdl, cdl, sdt = 0, cdt = 0;
      sincospi_t(d, &sd, &cd_);
      sincospi_t(d / len, &sdl, &cdl);
      if (taper) taper_sincospi(d * inv_taper, &sdt, &cdt);
      auto weight = [&](int m) -> T {
        // sin(pi (d - m)) = (-1)^m sin(pi d); sin(pi (d - m)/len) by angle addition
        const TapK<T> q = tk[m + D];
        const T num = (m & 1) ? -sd : sd;
        const T sx = sdl * q.c - cdl * q.s;
        T wgt = tap_div(num, len * sx);
        if (taper) wgt *= (T)0.54 + (T)0.46 * (cdt * q.tc + sdt * q.ts);
        return wgt;
      };
      const long long i0 = k0 - D - lo;  // window index of tap -D
      if (k0 - D >= 0 && k0 + D < g.n && i0 >= 0 && i0 + 2 * D < kWin) {
        // every tap inside the data and the staged window (the usual case):
        // the same sum without per-tap checks
        const TZ* wp = win + i0;
        for (int m = -D; m <= D; ++m) {
          const T wgt = weight(m);
          const TZ v = wp[m + D];
          zr += (T)v.x * wgt;
          zi += (T)v.y * wgt;
        }
      } else {
        for (int m = -D; m <= D; ++m) {
          const long long k = k0 + m;
          if (k < 0 || k >= g.n) continue;
          const T wgt = weight(m);
          const TZ v = tap(k);
          zr += (T)v.x * wgt;
          zi += (T)v.y * wgt;
        }
      }
    }
    // the antenna-weighted detector sum G (FP32 a, b in the mixed path)
    T wa, wb;
    if constexpr (sizeof(T) == sizeof(float)) {
      const NodeF32* ab = g.nodes32 + node0;
      const float a = wf[0] * ab[-1].a + wf[1] * ab[0].a + wf[2] * ab[1].a + wf[3] * ab[2].a;
      const float b = wf[0] * ab[-1].b + wf[1] * ab[0].b + wf[2] * ab[1].b + wf[3] * ab[2].b;
      const float wx = s_wx[X];
      wa = wx * a;
      wb = wx * b;
    } else {
      const double a = wn[0] * nd[-1].a + wn[1] * nd[0].a + wn[2] * nd[1].a + wn[3] * nd[2].a;
      const double b = wn[0] * nd[-1].b + wn[1] * nd[0].b + wn[2] * nd[1].b + wn[3] * nd[2].b;
      wa = (T)(w * a);
      wb = (T)(w * b);
    }
    acc.ar += wa * zr;
    acc.ai += wa * zi;
    acc.br += wb * zr;
    acc.bi += wb * zi;
  }
  if (j < g.n) {
    int64_t n1i = j % n1, n2i = j / n1;
    pstore(G + n1i * lc + n2i, acc);
  }
  // the fully valid segments' A, B, C: sum_r a(r)^2 over a segment = a^T M a
  // in the four node values (likewise b^T M b, a^T M b), one thread per
  // detector and segment, all lanes of a warp busy
  __syncthreads();
  constexpr int kSeg = kSkyBlock / kNodeStep;
  if (threadIdx.x < g.n_det * kSeg) {
    const int X = threadIdx.x / kSeg, sg = threadIdx.x % kSeg;
    if (s_full[X][sg]) {
      const SkyNode* nd = g.nodes + (int64_t)X * g.n_nodes + (j0 / kNodeStep + sg + 1);
      const double av[4] = {nd[-1].a, nd[0].a, nd[1].a, nd[2].a};
      const double bv[4] = {nd[-1].b, nd[0].b, nd[1].b, nd[2].b};
      double aMa = 0.0, bMb = 0.0, aMb = 0.0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        double ma = 0.0, mb = 0.0;
#pragma unroll
        for (int r2 = 0; r2 < 4; ++r2) {
          ma += s_m[q][r2] * av[r2];
          mb += s_m[q][r2] * bv[r2];
        }
        aMa += av[q] * ma;
        bMb += bv[q] * mb;
        aMb += av[q] * mb;
      }
      const double w = g.w[X];
      summed = true;
      sa += w * aMa;
      sb += w * bMb;
      sab += w * aMb;
    }
  }
  // block reduction of the A, B, C partial sums (fixed order).  Only the
  // warps that summed anything reduce (the segment sums sit in the first
  // n_det kSeg threads, per-sample sums arise only at the data's edges):
  // the others' zeros would not change a bit of the result.
  __shared__ double red[3][kSkyBlock / 32];
  if (__any_sync(0xffffffffu, summed)) {
    for (int o = 16; o > 0; o >>= 1) {
      sa += __shfl_down_sync(0xffffffffu, sa, o);
      sb += __shfl_down_sync(0xffffffffu, sb, o);
      sab += __shfl_down_sync(0xffffffffu, sab, o);
    }
  }
  const int wid = threadIdx.x >> 5;
  if (lane == 0) { red[0][wid] = sa; red[1][wid] = sb; red[2][wid] = sab; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double A = 0, B = 0, C = 0;
    for (int i = 0; i < kSkyBlock / 32; ++i) { A += red[0][i]; B += red[1][i]; C += red[2][i]; }
    partials[3 * blockIdx.x + 0] = A;
    partials[3 * blockIdx.x + 1] = B;
    partials[3 * blockIdx.x + 2] = C;
  }
}

__global__ void __launch_bounds__(1024)
k_sky_finalize(const double* __restrict__ partials, int nblocks, SkyConst* sky, int* err) {
  __shared__ double red[3][1024];
  double A = 0, B = 0, C = 0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
    A += partials[3 * i + 0];
    B += partials[3 * i + 1];
    C += partials[3 * i + 2];
  }
  red[0][threadIdx.x] = A;
  red[1][threadIdx.x] = B;
  red[2][threadIdx.x] = C;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[0][threadIdx.x] += red[0][threadIdx.x + o];
      red[1][threadIdx.x] += red[1][threadIdx.x + o];
      red[2][threadIdx.x] += red[2][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    A = red[0][0];
    B = red[1][0];
    C = red[2][0];
    double D = A * B - C * C;
    sky->A = A;
    sky->B = B;
    sky->C = C;
    sky->D = D;
    bool ok = isfinite(D) && D > 1e-12 * A * B && A > 0.0 && B > 0.0;
    if (!ok) {
      atomicCAS(err, 0, FSTAT_ERR_DEGENERATE);
      D = 1.0;
      A = B = C = 0.0;
    }
    sky->kA = 2.0 * A / D;
    sky->kB = 2.0 * B / D;
    sky->kC = 4.0 * C / D;
    sky->kAf = (float)sky->kA;
    sky->kBf = (float)sky->kB;
    sky->kCf = (float)sky->kC;
  }
}

// Per-template spindown polynomial in s = j - J (see TmplCoef).
__global__ void k_tmpl_coef(const SkyConst* __restrict__ sky, double dt, int64_t n,
                            const fstat_template* __restrict__ tmpl, const int* __restrict__ order,
                            int first, int count, TmplCoef* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const fstat_template tp = tmpl[order[first + i]];
  out[first + i] = spin_coef(sky->j_ref, n, dt, tp.f1dot, tp.f2dot);
}

// (after k_sky_table on the same stream: the phase uses this sky's t_m)
template <typename TIn, typename TZ>
void launch_phase(const Geo& g, int X, const void* xh, void* z, cudaStream_t st) {
  int blocks = (int)((g.n + 255) / 256);
  if (blocks > device_sm_count() * 64) blocks = device_sm_count() * 64;
  k_detector_phase<TIn, TZ><<<blocks, 256, 0, st>>>(g, X, (const TIn*)xh, (TZ*)z + (int64_t)X * g.n);
}

}  // namespace

int time_table_entries(double t_lo, double t_hi, double h) {
  return (int)std::ceil((t_hi - t_lo) / h) + 1;
}

cudaError_t launch_time_table(const Geo& g, TimeTab* tab, cudaStream_t st) {
  const int blocks = (g.tab_n + 255) / 256;
  k_time_table<<<blocks, 256, 0, st>>>(g, tab);
  return cudaGetLastError();
}

void launch_sky(const Geo& g, int precision, double alpha, double delta, const void* const* xh,
                const int* xh_dtype, void* z, void* G, int n1, int64_t lc, double* partials,
                int n_blocks, SkyConst* sky, int* err, cudaStream_t st) {
  k_sky_setup<<<1, 32, 0, st>>>(g, alpha, delta, sky);
  k_sky_table<<<(g.tab_n + 255) / 256, 256, 0, st>>>(g, sky);
  k_sky_nodes<<<(g.n_nodes + 127) / 128, 128, 0, st>>>(g, sky);
  if (precision != FSTAT_FP64) {
    const int64_t total = (int64_t)g.n_det * g.n_nodes;
    k_sky_nodes32<<<(int)std::min<int64_t>((total + 255) / 256, 8 * device_sm_count()), 256, 0, st>>>(g);
  }
  for (int X = 0; X < g.n_det; ++X) {
    bool in64 = xh_dtype[X] == FSTAT_C128;
    if (precision == FSTAT_FP64) {
      if (in64) launch_phase<double2, double2>(g, X, xh[X], z, st);
      else launch_phase<float2, double2>(g, X, xh[X], z, st);
    } else {
      if (in64) launch_phase<double2, float2>(g, X, xh[X], z, st);
      else launch_phase<float2, float2>(g, X, xh[X], z, st);
    }
  }
  if (precision == FSTAT_FP64) {
    k_resample<double, double2><<<n_blocks, kSkyBlock, 0, st>>>(
        g, sky, (const double2*)z, (PairMem<double>::type*)G, n1, lc, partials);
  } else {
    k_resample<float, float2><<<n_blocks, kSkyBlock, 0, st>>>(
        g, sky, (const float2*)z, (float4*)G, n1, lc, partials);
  }
  k_sky_finalize<<<1, 1024, 0, st>>>(partials, n_blocks, sky, err);
}

void launch_tmpl_coef(const SkyConst* sky, double dt, int64_t n, const fstat_template* tmpl,
                      const int* order, int first, int count, TmplCoef* out, cudaStream_t st) {
  if (count <= 0) return;
  k_tmpl_coef<<<(count + 127) / 128, 128, 0, st>>>(sky, dt, n, tmpl, order, first, count, out);
}

// Scan an input series for NaN/Inf.
template <typename TIn>
__global__ void k_check_finite(const TIn* __restrict__ x, int64_t n, int* err) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    TIn v = x[k];
    if (!isfinite((double)v.x) || !isfinite((double)v.y)) atomicCAS(err, 0, FSTAT_ERR_NONFINITE);
  }
}

void launch_check_finite(const void* x, int dtype, int64_t n, int* err, cudaStream_t st) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > device_sm_count() * 32) blocks = device_sm_count() * 32;
  if (dtype == FSTAT_C128) k_check_finite<double2><<<blocks, 256, 0, st>>>((const double2*)x, n, err);
  else k_check_finite<float2><<<blocks, 256, 0, st>>>((const float2*)x, n, err);
}

}  // namespace fstat
