// 2F and its gradient in (f, f1dot, alpha, delta) at arbitrary parameters.
//
// The refined statistic is eq. (Fstat) with the demodulation integrals of
// eqs. (Fa_DET)/(Fb_DET) (Sec. 2) summed directly over detector samples at
// a single frequency:
//
//   Phi_k = (f - f_h) tau_k + f_h t_m(t_k) + f1dot tau_k^2/2 + f2dot tau_k^3/6   [cycles]
//   tau_k = t_k - t_ref + t_m(t_k),   t_m = (r(t_k) / c) . n(alpha, delta)
//   Fa = sum_X w_X sum_k x_X[k] a_X(t_k) e^{-i 2 pi Phi_k},  Fb with b,
//   a = d(t_k) : e+(alpha, delta),  b = d(t_k) : ex(alpha, delta)
//
// t_m is linear in the sky vector n and a, b are linear in the detector
// tensor d(t_k), so r(t_k)/c and d(t_k) are sky-independent per-sample
// tables built once per plan.  Per candidate and sample the phase is
// evaluated in double-float (FP32 pairs, ~48-bit) arithmetic; the sums of
// Fa, Fb, their derivatives, and A, B, C (with their sky derivatives) are
// FP32 two-level sums reduced in FP64.  d(2F) follows by the chain rule.

#include <math.h>

#include "fstat_internal.cuh"

namespace fstat {
namespace adj {

constexpr int kWarps = 8;          // candidates per CTA (one warp each)
constexpr int kChunk = 1 << 17;    // samples per CTA (over all detectors)
constexpr int kInner = 64;         // first-level summation length per lane
constexpr int kAcc = 29;           // accumulated quantities per candidate

// ------------------------------------------------------------ double-float
struct df {
  float h, l;
};
__device__ __forceinline__ df df_from(double x) {
  float h = (float)x;
  return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.h, b.h);
  float e = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
  float h = __fadd_rn(s.h, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s.h))};
}
__device__ __forceinline__ df df_mul(df a, df b) {
  float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  float h = __fadd_rn(p, e);
  return {h, __fsub_rn(e, __fsub_rn(h, p))};
}
__device__ __forceinline__ df df_mulf(df a, float b) {
  float p = __fmul_rn(a.h, b);
  float e = fmaf(a.h, b, -p);
  e = fmaf(a.l, b, e);
  float h = __fadd_rn(p, e);
  return {h, __fsub_rn(e, __fsub_rn(h, p))};
}
// fractional part of a double-float in [-1/2, 1/2]
__device__ __forceinline__ float df_frac(df a) {
  float k = rintf(a.h);
  return __fadd_rn(__fsub_rn(a.h, k), a.l);
}

// ------------------------------------------------------------ tables, consts
// Per sample (detector-major, k fastest): r/c as double-float, detector
// tensor components (xx, yy, zz, xy, xz, yz), normalised data.
struct SampleTabs {
  float4* rc;   // (x.h, x.l, y.h, y.l) per sample
  float2* rcz;  // (z.h, z.l)
  float4* d0;   // (xx, yy, zz, xy)
  float2* d1;   // (xz, yz)
  float2* x;    // x_h / sigma_ref
};

struct CandConst {
  df nx, ny, nz;                 // sky vector
  float dna[3], dnd[3];          // d n / d alpha, d n / d delta
  float ep[6], ex[6];            // e+ and ex weights for (xx, yy, zz, xy, xz, yz), off-diagonals doubled
  float epa[6], epd[6], exa[6], exd[6];
  df fmh;                        // f - f_h
  df fh;                         // f_h
  df f1h;                        // f1dot / 2
  df f2s;                        // f2dot / 6
  float f, f1, f2;               // for dPhi/dt_m = f + f1dot tau + f2dot tau^2 / 2
  float pad_;
};

__global__ void k_tables(Geo g, int X, const void* __restrict__ xh, int dtype, SampleTabs tab) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < g.n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double t = g.t0 + (double)k * g.dt;
    double so, co, sp, cp;
    sincos(g.orb_ph0 + g.w_orb * t, &so, &co);
    const double ph = g.lon[X] + g.sid_ph0 + g.w_rot * t;
    sincos(ph, &sp, &cp);
    const double rx = (g.au * co + g.rcl[X] * cp) / g.c;
    const double ry = (g.au * g.cos_obl * so + g.rcl[X] * sp) / g.c;
    const double rz = (g.au * g.sin_obl * so + g.rsl[X]) / g.c;
    const int64_t i = (int64_t)X * g.n + k;
    float hx = (float)rx, hy = (float)ry, hz = (float)rz;
    tab.rc[i] = make_float4(hx, (float)(rx - hx), hy, (float)(ry - hy));
    tab.rcz[i] = make_float2(hz, (float)(rz - hz));
    // detector tensor d = (u u^T - v v^T)/2, arms at gamma -/+ 45 deg from East towards North
    const double sl = sin(g.lat[X]), cl = cos(g.lat[X]);
    const double e[3] = {-sp, cp, 0.0};
    const double nn[3] = {-sl * cp, -sl * sp, cl};
    const double g1 = g.gam[X] - 0.78539816339744830962, g2 = g.gam[X] + 0.78539816339744830962;
    double u[3], v[3];
    for (int q = 0; q < 3; ++q) {
      u[q] = cos(g1) * e[q] + sin(g1) * nn[q];
      v[q] = cos(g2) * e[q] + sin(g2) * nn[q];
    }
    auto dd = [&](int p, int q) { return 0.5 * (u[p] * u[q] - v[p] * v[q]); };
    tab.d0[i] = make_float4((float)dd(0, 0), (float)dd(1, 1), (float)dd(2, 2), (float)dd(0, 1));
    tab.d1[i] = make_float2((float)dd(0, 2), (float)dd(1, 2));
    double xr, xi;
    if (dtype == FSTAT_C128) {
      double2 v2 = ((const double2*)xh)[k];
      xr = v2.x; xi = v2.y;
    } else {
      float2 v2 = ((const float2*)xh)[k];
      xr = v2.x; xi = v2.y;
    }
    tab.x[i] = make_float2((float)(xr * g.inv_sigma_ref), (float)(xi * g.inv_sigma_ref));
  }
}

// polarisation tensors and their sky derivatives for one candidate
__global__ void k_cand_consts(const fstat_candidate* __restrict__ cand, int n, double f_het,
                              CandConst* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const fstat_candidate c = cand[i];
  const double sa = sin(c.alpha), ca = cos(c.alpha), sd = sin(c.delta), cd = cos(c.delta);
  CandConst k;
  k.nx = df_from(cd * ca);
  k.ny = df_from(cd * sa);
  k.nz = df_from(sd);
  const double dna[3] = {-cd * sa, cd * ca, 0.0};
  const double dnd[3] = {-sd * ca, -sd * sa, cd};
  const double x[3] = {sa, -ca, 0.0};
  const double y[3] = {-sd * ca, -sd * sa, cd};
  const double xa[3] = {ca, sa, 0.0};
  const double ya[3] = {sd * sa, -sd * ca, 0.0};
  const double xd[3] = {0.0, 0.0, 0.0};
  const double yd[3] = {-cd * ca, -cd * sa, -sd};
  const int P[6] = {0, 1, 2, 0, 0, 1}, Q[6] = {0, 1, 2, 1, 2, 2};
  for (int m = 0; m < 6; ++m) {
    const int p = P[m], q = Q[m];
    const double w = m < 3 ? 1.0 : 2.0;  // off-diagonal terms appear twice in d : e
    k.ep[m] = (float)(w * (x[p] * x[q] - y[p] * y[q]));
    k.ex[m] = (float)(w * (x[p] * y[q] + y[p] * x[q]));
    k.epa[m] = (float)(w * (xa[p] * x[q] + x[p] * xa[q] - ya[p] * y[q] - y[p] * ya[q]));
    k.epd[m] = (float)(w * (xd[p] * x[q] + x[p] * xd[q] - yd[p] * y[q] - y[p] * yd[q]));
    k.exa[m] = (float)(w * (xa[p] * y[q] + x[p] * ya[q] + ya[p] * x[q] + y[p] * xa[q]));
    k.exd[m] = (float)(w * (xd[p] * y[q] + x[p] * yd[q] + yd[p] * x[q] + y[p] * xd[q]));
  }
  for (int q = 0; q < 3; ++q) {
    k.dna[q] = (float)dna[q];
    k.dnd[q] = (float)dnd[q];
  }
  k.fmh = df_from(c.f - f_het);
  k.fh = df_from(f_het);
  k.f1h = df_from(c.f1dot / 2.0);
  k.f2s = df_from(c.f2dot / 6.0);
  k.f = (float)c.f;
  k.f1 = (float)c.f1dot;
  k.f2 = (float)c.f2dot;
  k.pad_ = 0.f;
  out[i] = k;
}

// accumulated quantities (kAcc): 0-1 Fa, 2-3 Fb, 4-7 dFa,dFb/df, 8-11 d/df1dot,
// 12-15 d/dalpha, 16-19 d/ddelta, 20-22 A,B,C, 23-25 dA,dB,dC/dalpha, 26-28 d/ddelta
__global__ void __launch_bounds__(kWarps * 32, 3)
k_partial(Geo g, SampleTabs tab, const CandConst* __restrict__ cc, int n_cand, int n_chunks,
          double* __restrict__ partial) {
  __shared__ CandConst sc[kWarps];
  // second-level sums of every lane, in shared memory so that the registers
  // hold the candidate's constants instead (same FP32 arithmetic)
  __shared__ float s_outer[kWarps][kAcc][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cand = blockIdx.x * kWarps + warp;
  const int chunk = blockIdx.y;
  if (threadIdx.x < kWarps && blockIdx.x * kWarps + threadIdx.x < n_cand)
    sc[threadIdx.x] = cc[blockIdx.x * kWarps + threadIdx.x];
  __syncthreads();
  if (cand >= n_cand) return;
  const CandConst& K = sc[warp];
  const int64_t total = (int64_t)g.n_det * g.n;
  const int64_t beg = (int64_t)chunk * kChunk;
  const int64_t end = beg + kChunk < total ? beg + kChunk : total;
  const df dt = df_from(g.dt);
  const df c0 = df_from(g.t0 - g.t_ref);
  const float two_pi = 6.28318530717958647692f;

  float inner[kAcc];
  float* outer = &s_outer[warp][0][lane];  // element q at outer[32 q]
#pragma unroll
  for (int q = 0; q < kAcc; ++q) outer[32 * q] = 0.f;
  int cnt = 0;
#pragma unroll
  for (int q = 0; q < kAcc; ++q) inner[q] = 0.f;
  // detector X and sample k of index i, advanced incrementally (no 64-bit
  // division, no double->float conversion per sample)
  int X = (int)((beg + lane) / g.n);
  int k = (int)(beg + lane - (int64_t)X * g.n);
  float w = X < g.n_det ? (float)g.w[X] : 0.f;
  for (int64_t i = beg + lane; i < end; i += 32, k += 32) {
    while (k >= g.n) {
      k -= (int)g.n;
      ++X;
      w = (float)g.w[X];
    }
    const float4 r4 = __ldg(&tab.rc[i]);
    const float2 rz = __ldg(&tab.rcz[i]);
    const float4 d0 = __ldg(&tab.d0[i]);
    const float2 d1 = __ldg(&tab.d1[i]);
    const float2 xv = __ldg(&tab.x[i]);
    // t_m = (r/c) . n in double-float
    df tm = df_add(df_add(df_mul({r4.x, r4.y}, K.nx), df_mul({r4.z, r4.w}, K.ny)), df_mul({rz.x, rz.y}, K.nz));
    // tau = k dt + (t0 - t_ref) + t_m
    df tk = df_add(df_mulf(dt, (float)k), c0);
    df tau = df_add(tk, tm);
    // Phi = (f - f_h) tau + f_h t_m + f1dot tau^2/2 + f2dot tau^3/6
    df tau2 = df_mul(tau, tau);
    df ph = df_add(df_add(df_mul(K.fmh, tau), df_mul(K.fh, tm)),
                   df_add(df_mul(K.f1h, tau2), df_mul(K.f2s, df_mul(tau2, tau))));
    const float fr = df_frac(ph);
    float sn, cs;
    __sincosf(two_pi * fr, &sn, &cs);
    // e = w x exp(-i 2 pi Phi)
    const float er = w * (xv.x * cs + xv.y * sn);
    const float ei = w * (xv.y * cs - xv.x * sn);
    const float D[6] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y};
    float a = 0.f, b = 0.f, aa = 0.f, ad = 0.f, ba = 0.f, bd = 0.f;
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      a = fmaf(D[m], K.ep[m], a);
      b = fmaf(D[m], K.ex[m], b);
      aa = fmaf(D[m], K.epa[m], aa);
      ad = fmaf(D[m], K.epd[m], ad);
      ba = fmaf(D[m], K.exa[m], ba);
      bd = fmaf(D[m], K.exd[m], bd);
    }
    const float tauf = tau.h;
    const float dpdt = K.f + K.f1 * tauf + 0.5f * K.f2 * tauf * tauf;  // dPhi/dt_m
    const float tma = r4.x * K.dna[0] + r4.z * K.dna[1] + rz.x * K.dna[2];
    const float tmd = r4.x * K.dnd[0] + r4.z * K.dnd[1] + rz.x * K.dnd[2];
    // d/dtheta of e * pat = e * (pat_theta - i 2 pi Phi_theta pat)
    const float pf = two_pi * tauf, p1 = two_pi * 0.5f * tauf * tauf;
    const float pa = two_pi * dpdt * tma, pd = two_pi * dpdt * tmd;
    inner[0] += er * a;  inner[1] += ei * a;
    inner[2] += er * b;  inner[3] += ei * b;
    // (-i p) e pat = p pat (ei, -er)
    inner[4] += pf * a * ei;  inner[5] -= pf * a * er;
    inner[6] += pf * b * ei;  inner[7] -= pf * b * er;
    inner[8] += p1 * a * ei;  inner[9] -= p1 * a * er;
    inner[10] += p1 * b * ei; inner[11] -= p1 * b * er;
    inner[12] += er * aa + pa * a * ei;  inner[13] += ei * aa - pa * a * er;
    inner[14] += er * ba + pa * b * ei;  inner[15] += ei * ba - pa * b * er;
    inner[16] += er * ad + pd * a * ei;  inner[17] += ei * ad - pd * a * er;
    inner[18] += er * bd + pd * b * ei;  inner[19] += ei * bd - pd * b * er;
    inner[20] += w * a * a;
    inner[21] += w * b * b;
    inner[22] += w * a * b;
    inner[23] += 2.f * w * a * aa;
    inner[24] += 2.f * w * b * ba;
    inner[25] += w * (aa * b + a * ba);
    inner[26] += 2.f * w * a * ad;
    inner[27] += 2.f * w * b * bd;
    inner[28] += w * (ad * b + a * bd);
    if (++cnt == kInner) {
#pragma unroll
      for (int q = 0; q < kAcc; ++q) { outer[32 * q] += inner[q]; inner[q] = 0.f; }
      cnt = 0;
    }
  }
  double* dst = partial + ((int64_t)cand * n_chunks + chunk) * kAcc;
#pragma unroll
  for (int q = 0; q < kAcc; ++q) {
    double v = (double)outer[32 * q] + (double)inner[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) dst[q] = v;
  }
}

// sum the chunk partials (fixed order) and apply the chain rule in FP64
__global__ void k_finalize(const double* __restrict__ partial, int n_cand, int n_chunks,
                           float* __restrict__ twoF, float* __restrict__ grad) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_cand) return;
  double s[kAcc];
  for (int q = 0; q < kAcc; ++q) s[q] = 0.0;
  for (int c = 0; c < n_chunks; ++c)
    for (int q = 0; q < kAcc; ++q) s[q] += partial[((int64_t)i * n_chunks + c) * kAcc + q];
  const double A = s[20], B = s[21], C = s[22];
  const double D = A * B - C * C;
  const double far = s[0], fai = s[1], fbr = s[2], fbi = s[3];
  const double fa2 = far * far + fai * fai, fb2 = fbr * fbr + fbi * fbi, re = far * fbr + fai * fbi;
  const double N = B * fa2 + A * fb2 - 2.0 * C * re;
  twoF[i] = (float)(2.0 * N / D);
  for (int j = 0; j < 4; ++j) {
    const double dar = s[4 + 4 * j], dai = s[5 + 4 * j], dbr = s[6 + 4 * j], dbi = s[7 + 4 * j];
    const double dfa2 = 2.0 * (far * dar + fai * dai);
    const double dfb2 = 2.0 * (fbr * dbr + fbi * dbi);
    const double dre = dar * fbr + dai * fbi + far * dbr + fai * dbi;
    double dA = 0.0, dB = 0.0, dC = 0.0;
    if (j == 2) { dA = s[23]; dB = s[24]; dC = s[25]; }
    if (j == 3) { dA = s[26]; dB = s[27]; dC = s[28]; }
    const double dN = dB * fa2 + B * dfa2 + dA * fb2 + A * dfb2 - 2.0 * (dC * re + C * dre);
    const double dD = dA * B + A * dB - 2.0 * C * dC;
    grad[4 * i + j] = (float)(2.0 * (dN * D - N * dD) / (D * D));
  }
}

}  // namespace adj

size_t grad_table_bytes(int n_det, int64_t n) {
  return (size_t)n_det * n * (16 + 8 + 16 + 8 + 8) + 256;
}

cudaError_t launch_grad_tables(const Geo& g, const void* const* xh, const int* dtype, void* base,
                               cudaStream_t st) {
  const int64_t tot = (int64_t)g.n_det * g.n;
  adj::SampleTabs tab;
  char* p = (char*)base;
  tab.rc = (float4*)p; p += 16 * tot;
  tab.d0 = (float4*)p; p += 16 * tot;
  tab.rcz = (float2*)p; p += 8 * tot;
  tab.d1 = (float2*)p; p += 8 * tot;
  tab.x = (float2*)p;
  int blocks = (int)((g.n + 255) / 256);
  if (blocks > device_sm_count() * 32) blocks = device_sm_count() * 32;
  for (int X = 0; X < g.n_det; ++X)
    adj::k_tables<<<blocks, 256, 0, st>>>(g, X, xh[X], dtype[X], tab);
  return cudaGetLastError();
}

size_t grad_scratch_bytes(int n_cand, const Geo& g) {
  const int64_t tot = (int64_t)g.n_det * g.n;
  const int chunks = (int)((tot + adj::kChunk - 1) / adj::kChunk);
  return (size_t)n_cand * sizeof(adj::CandConst) + (size_t)n_cand * chunks * adj::kAcc * sizeof(double) + 512;
}

cudaError_t launch_grad(const Geo& g, const void* tables, const fstat_candidate* cand_dev, int n_cand,
                        void* scratch, float* twoF, float* grad, cudaStream_t st) {
  const int64_t tot = (int64_t)g.n_det * g.n;
  const int chunks = (int)((tot + adj::kChunk - 1) / adj::kChunk);
  adj::SampleTabs tab;
  char* p = (char*)tables;
  tab.rc = (float4*)p; p += 16 * tot;
  tab.d0 = (float4*)p; p += 16 * tot;
  tab.rcz = (float2*)p; p += 8 * tot;
  tab.d1 = (float2*)p; p += 8 * tot;
  tab.x = (float2*)p;
  adj::CandConst* cc = (adj::CandConst*)scratch;
  double* partial = (double*)((char*)scratch + (((size_t)n_cand * sizeof(adj::CandConst) + 255) & ~(size_t)255));
  adj::k_cand_consts<<<(n_cand + 127) / 128, 128, 0, st>>>(cand_dev, n_cand, g.f_het, cc);
  dim3 grid((n_cand + adj::kWarps - 1) / adj::kWarps, chunks);
  adj::k_partial<<<grid, adj::kWarps * 32, 0, st>>>(g, tab, cc, n_cand, chunks, partial);
  adj::k_finalize<<<(n_cand + 127) / 128, 128, 0, st>>>(partial, n_cand, chunks, twoF, grad);
  return cudaGetLastError();
}

}  // namespace fstat
