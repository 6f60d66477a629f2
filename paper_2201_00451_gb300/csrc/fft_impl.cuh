// Batched Stockham FFT for the template loop: Sec. 3 steps (vi) and (vii).
//
// For one template, Fa and Fb are forward DFTs of length N = n_fft of the
// zero-padded, spindown-corrected series y[j] = G[j] exp(-i 2 pi phi(j)),
// j < n (eqs. Fa, Fb).  N = N1 * N2 is split four-step style:
//
//   pass A (column n1 < N1):  Y[n1][k2] = W_N^{n1 k2} sum_{n2} y[n1 + N1 n2] W_N2^{n2 k2}
//   pass B (row k2 < N2):     X[k2 + N2 k1] = sum_{n1} Y[n1][k2] W_N1^{n1 k1}
//
// Each column / row FFT runs in shared memory as Stockham radix-16/8/4
// passes (out-of-place index map, in-place buffer, butterflies in
// registers).  Pass A computes the spindown phase on the fly, pass B
// evaluates eq. (Fstat) on the final butterfly outputs and stores 2F in
// ascending frequency (fftshift folded into the index).  Fa and Fb travel
// together as one 16-byte (FP32) / 32-byte (FP64) element, so every index,
// twiddle and phase is computed once for both.
//
// Twiddles are computed per butterfly: one sine/cosine of the reduced angle
// (hardware sine/cosine in FP32, sincospi in FP64) and powers by binary
// splitting.  CA / CB, the columns / rows per CTA, are template parameters
// chosen per FFT length by the autotuner.
#pragma once

#include <cuda.h>  // CUtensorMap (encoded through the runtime's driver entry point)
#include <stdint.h>
#include <string.h>

#include "fstat_internal.cuh"

namespace fstat {
namespace fft {

#ifndef FSTAT_PASSB_TABLE
#define FSTAT_PASSB_TABLE 0
#endif
// Stockham twiddles are computed (hardware sine/cosine of the reduced angle
// and powers) in both passes; the table variant of pass B (build with
// -DFSTAT_PASSB_TABLE=1) measured 11% slower on GB300 at n_fft = 2^22.
constexpr bool kPassBTable = FSTAT_PASSB_TABLE != 0;

#ifndef FSTAT_PIPELINE
#define FSTAT_PIPELINE 1
#endif
#ifndef FSTAT_R8_MINB
#define FSTAT_R8_MINB 1
#endif
// FSTAT_PIPELINE = 1: persistent CTAs prefetch the next tile with cp.async;
// 0: one tile per CTA, loaded straight into registers.
constexpr bool kPipeline = FSTAT_PIPELINE != 0;
// minimum resident CTAs requested for radix-8 variants (0 = no register cap)
constexpr int kR8MinBlocks = FSTAT_R8_MINB;

template <typename T> struct TwT;
template <> struct TwT<float> { using type = float2; };
template <> struct TwT<double> { using type = double2; };

// ------------------------------------------------------------ radix schedule
// V = 0: radix-16 first (fewest shared-memory passes, 16 points per thread);
// Schedule code V: bit 0 (lengths >= 1024) = radix-8 first (8 points per
// thread, half the registers, one more pass); bit 1 = one shared buffer
// (no prefetch), half the shared memory, and for radix-16 CTAs of up to
// 256 threads a register cap (128) that lets two CTAs share an SM; bit 3
// (pass A, with bit 1, radix-16) = a tighter cap (80) for three CTAs per
// SM; bit 2 (pass B) = tiles loaded by bulk tensor copies (TMA) instead of
// per-thread 16-byte copies; bit 3 (pass B, per-thread copies, one
// buffer) = the first half of the next tile's rows copied into a staging
// area of their own as soon as the first pass has read this tile's (the
// second half as before, once the last pass has read the buffer); bit 2
// (pass A, fused kernel only) = the
// column staged densely by one bulk copy; bit 4 (pass A, one column per
// CTA: 16 at 8192 points, 18 at 4096 points with the two-per-SM register
// cap of bit 1) = the next column's samples copied densely by one bulk copy
// into a staging area of their own while this column is transformed.  The first
// radix is the largest.
__host__ __device__ constexpr bool r8(int L, int V) { return (V & 1) && L >= 1024; }
__host__ __device__ constexpr int np_of(int L, int V) {
  return r8(L, V) ? (L == 8192 ? 5 : 4) : (L <= 256 ? 2 : (L <= 4096 ? 3 : 4));
}
__host__ __device__ constexpr int r_of(int L, int p, int V) {
  return r8(L, V)   ? (L == 8192 ? (p < 4 ? 8 : 2) : (p < 3 ? 8 : L / 512))
       : L == 32    ? (p == 0 ? 8 : 4)
       : L == 64    ? 8
       : L == 128   ? (p == 0 ? 16 : 8)
       : L == 256   ? 16
       : L == 512   ? 8
       : L == 1024  ? (p == 0 ? 16 : 8)
       : L == 2048  ? (p == 2 ? 8 : 16)
       : L == 8192  ? (p == 3 ? 2 : 16)  // pass A only: 16 x 16 x 16 x 2
       : 16;  // 4096
}
__host__ __device__ constexpr int ns_of(int L, int p, int V) {
  return p == 0 ? 1 : ns_of(L, p - 1, V) * r_of(L, p - 1, V);
}
__host__ __device__ constexpr int log2c(int x) { return x <= 1 ? 0 : 1 + log2c(x / 2); }

// product of the schedule's radices (must be L)
__host__ __device__ constexpr int radix_product(int L, int V, int p = 0) {
  return p == np_of(L, V) ? 1 : r_of(L, p, V) * radix_product(L, V, p + 1);
}

template <typename T, int L, int V = 0> struct Shape {
  static constexpr int NP = np_of(L, V);
  static constexpr int R0 = r_of(L, 0, V);        // largest radix, points per thread
  static constexpr int TPC = L / R0;              // threads per column
  static constexpr int PS = log2c(R0);            // shared-memory padding shift
  static constexpr int LP = L + (L >> PS);        // padded column length
  static constexpr int RL = r_of(L, NP - 1, V);   // last radix
  static constexpr int NSL = L / RL;              // span of the last pass
  static constexpr int CA_DEF = TPC >= 128 ? 1 : 128 / TPC;
  static constexpr int CB_MIN = sizeof(T) == 4 ? 2 : 1;
  static constexpr int CB_DEF = TPC >= 128 ? CB_MIN : (128 / TPC > CB_MIN ? 128 / TPC : CB_MIN);
  using PM = typename PairMem<T>::type;
  using TW = typename TwT<T>::type;
  // every pass's radix divides the points per thread (each thread owns whole
  // butterflies of every pass, the last one included) and the radices
  // multiply to L
  static_assert(radix_product(L, V) == L, "radix schedule does not multiply to the length");
  static_assert(R0 % RL == 0 && R0 >= RL, "the last pass's butterflies do not cover the points of a thread");
};

// Shared memory of a persistent pass kernel: NBUF padded buffers of C
// columns; two (prefetch the next tile while transforming this one) when
// they fit, else one.
constexpr size_t kSmemCap = (size_t)220 * 1024;
template <typename T, int L, int C, int V = 0> struct Buf {
  static constexpr size_t ONE = (size_t)C * Shape<T, L, V>::LP * sizeof(typename Shape<T, L, V>::PM);
  static constexpr int NBUF = (kPipeline && !(V & 2) && !(V & 8) && !(V & 16) && 2 * ONE <= kSmemCap) ? 2 : 1;
  static constexpr size_t BYTES = NBUF * ONE;
};

// Peaks mode: a persistent pass-B CTA keeps the band keys of up to
// kPeakBands bands in shared memory across its tiles and flushes them to
// global memory once, when every band spans whole output rows (then each
// band's bins in a tile sit in the same threads in every tile).
constexpr int kPeakBands = 1024;
// pass-B epilogues: store 2F, reduce it (peaks), add it to a shifted row
constexpr int kStore = 0, kPeaks = 1, kAccumulate = 2;
// With one buffer the tile's 2F goes to a region of its own (SEP, when it
// fits) instead of the buffer, so that the next tile's copies can start
// early as in the other epilogues.  Layout: buffers, band keys, 2F tile.
template <typename T, int L, int C, int V> struct PeakSmem {
  static constexpr size_t EXTRA = (size_t)kPeakBands * sizeof(unsigned long long);
  static constexpr bool ACC = kPipeline && Buf<T, L, C, V>::BYTES + EXTRA <= 227 * 1024;
  static constexpr size_t KEYS_END = Buf<T, L, C, V>::BYTES + (ACC ? EXTRA : 0);
  static constexpr size_t SF = (size_t)L * C * sizeof(float);
  static constexpr bool SEP = kPipeline && Buf<T, L, C, V>::NBUF == 1 && KEYS_END + SF <= 227 * 1024;
  static constexpr size_t BYTES = KEYS_END + (SEP ? SF : 0);
};

template <typename T, int L, int C, int V = 0> constexpr bool cfg_ok() {
  using S = Shape<T, L, V>;
  return C * S::TPC >= 32 && C * S::TPC <= 1024 && Buf<T, L, C, V>::ONE <= kSmemCap;
}

// 16-byte asynchronous global -> shared copies (completion tracked by
// commit groups; cp.async.wait_group is a hardware wait, not a spin loop).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
template <typename PM> __device__ __forceinline__ void cp_pair(PM* dst, const PM* src) {
  cp_async16(dst, src);
  if constexpr (sizeof(PM) == 32) cp_async16((char*)dst + 16, (const char*)src + 16);
}

// Bulk tensor copies (TMA) for pass B's tiles: one thread issues a few 2D
// box copies of the intermediate into shared memory, completion is counted
// in bytes on an mbarrier, and every thread waits on the barrier's phase.
// Each wait gives up after kWaitLimit polls (a GPU that stopped delivering
// copies must not hang the kernel): it then records FSTAT_ERR_TIMEOUT and
// the kernel returns.
constexpr int kWaitLimit = 1 << 22;
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int limit = kWaitLimit) {
  for (int i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// order this thread's earlier shared-memory accesses before async-proxy writes
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::
          "r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// rows per box of a pass-B tile load (the box height limit is 256)
constexpr int kTmaRows = 256;
// contiguous bulk copy global -> shared (16-byte aligned addresses, size a
// multiple of 16), completion counted in bytes on the mbarrier
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// load with acquire semantics at GPU scope (a counter another CTA releases)
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// order this thread's earlier generic-proxy accesses to global memory (and
// what it acquired) before its later async-proxy (bulk copy) accesses
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;\n" ::: "memory");
}

__device__ __forceinline__ int pad_idx(int pos, int ps) { return pos + (pos >> ps); }

template <typename TW> __device__ __forceinline__ TW tw_ld(const TW* p) { return __ldg(p); }

// (cos, sin) of 2 pi x for x in turns.  FP32: reduce x to [-1/2, 1/2] (exact)
// and use the hardware sine/cosine, accurate to ~4e-7 absolute on [-pi, pi];
// FP64: sincospi.
__device__ __forceinline__ void turn_sincos(float x, float* s, float* c) {
  const float r = x - rintf(x);
  __sincosf(6.28318530717958647692f * r, s, c);
}
__device__ __forceinline__ void turn_sincos(double x, double* s, double* c) {
  sincospi(2.0 * x, s, c);
}

// wc[q] + i ws[q] = (c + i s)^q for q = 0..R-1 by binary splitting (the
// error grows with log2 q, not q).
template <typename T, int R>
__device__ __forceinline__ void powers(T c, T s, T* wc, T* ws) {
  wc[0] = (T)1; ws[0] = (T)0;
  wc[1] = c; ws[1] = s;
#pragma unroll
  for (int q = 2; q < R; ++q) {
    const int h = q / 2, l = q - h;
    wc[q] = wc[h] * wc[l] - ws[h] * ws[l];
    ws[q] = wc[h] * ws[l] + ws[h] * wc[l];
  }
}

// ------------------------------------------------------------- small DFTs
template <typename T> __device__ __forceinline__ Pair<T> w8_1(const Pair<T>& x) {  // * (1 - i)/sqrt2
  const T r = (T)0.70710678118654752440;
  return {(x.ar + x.ai) * r, (x.ai - x.ar) * r, (x.br + x.bi) * r, (x.bi - x.br) * r};
}
template <typename T> __device__ __forceinline__ Pair<T> w8_3(const Pair<T>& x) {  // * (-1 - i)/sqrt2
  const T r = (T)0.70710678118654752440;
  return {(x.ai - x.ar) * r, -(x.ar + x.ai) * r, (x.bi - x.br) * r, -(x.br + x.bi) * r};
}

template <typename T> __device__ __forceinline__ void dft4(Pair<T>& x0, Pair<T>& x1, Pair<T>& x2, Pair<T>& x3) {
  Pair<T> t0 = padd(x0, x2), t1 = psub(x0, x2), t2 = padd(x1, x3), t3 = pmul_mi(psub(x1, x3));
  x0 = padd(t0, t2);
  x2 = psub(t0, t2);
  x1 = padd(t1, t3);
  x3 = psub(t1, t3);
}

template <typename T> __device__ __forceinline__ void dft8(Pair<T>* x) {
  Pair<T> e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
  Pair<T> o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
  dft4(e0, e1, e2, e3);
  dft4(o0, o1, o2, o3);
  o1 = w8_1(o1);
  o2 = pmul_mi(o2);
  o3 = w8_3(o3);
  x[0] = padd(e0, o0); x[4] = psub(e0, o0);
  x[1] = padd(e1, o1); x[5] = psub(e1, o1);
  x[2] = padd(e2, o2); x[6] = psub(e2, o2);
  x[3] = padd(e3, o3); x[7] = psub(e3, o3);
}

template <typename T> __device__ __forceinline__ void dft16(Pair<T>* x) {
  Pair<T> e[8], o[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) { e[k] = x[2 * k]; o[k] = x[2 * k + 1]; }
  dft8(e);
  dft8(o);
  const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173;  // cos, sin of pi/8
  o[1] = pmul(o[1], c1, -s1);
  o[2] = w8_1(o[2]);
  o[3] = pmul(o[3], s1, -c1);
  o[4] = pmul_mi(o[4]);
  o[5] = pmul(o[5], -s1, -c1);
  o[6] = w8_3(o[6]);
  o[7] = pmul(o[7], -c1, -s1);
#pragma unroll
  for (int k = 0; k < 8; ++k) { x[k] = padd(e[k], o[k]); x[k + 8] = psub(e[k], o[k]); }
}

// The same transforms when the upper half of the inputs is zero (x[R/2..R)
// unread): the zero-padded first pass of pass A when every column holds at
// most L/2 samples.  Same output order as dft4/dft8/dft16; the first
// add/subtract level of the even/odd split drops out.
template <typename T> __device__ __forceinline__ void dft4_half(Pair<T>& x0, Pair<T>& x1, Pair<T>& x2,
                                                               Pair<T>& x3) {
  const Pair<T> a = x0, t3 = pmul_mi(x1);
  x2 = psub(a, x1);
  x0 = padd(a, x1);
  x1 = padd(a, t3);
  x3 = psub(a, t3);
}
template <typename T> __device__ __forceinline__ void dft8_half(Pair<T>* x) {
  Pair<T> e0 = x[0], e1 = x[2], e2, e3;
  Pair<T> o0 = x[1], o1 = x[3], o2, o3;
  dft4_half(e0, e1, e2, e3);
  dft4_half(o0, o1, o2, o3);
  o1 = w8_1(o1);
  o2 = pmul_mi(o2);
  o3 = w8_3(o3);
  x[0] = padd(e0, o0); x[4] = psub(e0, o0);
  x[1] = padd(e1, o1); x[5] = psub(e1, o1);
  x[2] = padd(e2, o2); x[6] = psub(e2, o2);
  x[3] = padd(e3, o3); x[7] = psub(e3, o3);
}
template <typename T> __device__ __forceinline__ void dft16_half(Pair<T>* x) {
  Pair<T> e[8], o[8];
#pragma unroll
  for (int k = 0; k < 4; ++k) { e[k] = x[2 * k]; o[k] = x[2 * k + 1]; }
  dft8_half(e);
  dft8_half(o);
  const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173;  // cos, sin of pi/8
  o[1] = pmul(o[1], c1, -s1);
  o[2] = w8_1(o[2]);
  o[3] = pmul(o[3], s1, -c1);
  o[4] = pmul_mi(o[4]);
  o[5] = pmul(o[5], -s1, -c1);
  o[6] = w8_3(o[6]);
  o[7] = pmul(o[7], -c1, -s1);
#pragma unroll
  for (int k = 0; k < 8; ++k) { x[k] = padd(e[k], o[k]); x[k + 8] = psub(e[k], o[k]); }
}
template <typename T, int R> __device__ __forceinline__ void dft(Pair<T>* x) {
  if constexpr (R == 2) { Pair<T> a = x[0], b = x[1]; x[0] = padd(a, b); x[1] = psub(a, b); }
  else if constexpr (R == 4) dft4(x[0], x[1], x[2], x[3]);
  else if constexpr (R == 8) dft8(x);
  else dft16(x);
}

template <typename T, int R> __device__ __forceinline__ void dft_half(Pair<T>* x) {
  if constexpr (R == 8) dft8_half(x);
  else if constexpr (R == 16) dft16_half(x);
  else {
#pragma unroll
    for (int s = R / 2; s < R; ++s) x[s] = pzero<T>();
    dft<T, R>(x);
  }
}

// --------------------------------------------------------- Stockham passes
// After pass 0 (done by the caller, in registers), store it and run passes
// 1..NP-1.  On return v holds the last pass's outputs: butterfly
// b = t + q * TPC, output index b + s * NSL in v[q * RL + s].
// Shared-memory address of logical position pos is pad(pos) * STRIDE.
// at_free() runs once the last pass has read the buffer into registers (all
// threads past the barrier that follows): the buffer is free from there on.
struct NoOp {
  __device__ __forceinline__ void operator()() const {}
};
template <typename T, int L, int V, int STRIDE, int P, bool TABLE, typename F = NoOp>
__device__ __forceinline__ void passes(Pair<T>* v, typename PairMem<T>::type* buf, int t,
                                       const typename TwT<T>::type* __restrict__ twL, const F& at_free = F()) {
  using S = Shape<T, L, V>;
  constexpr int R = r_of(L, P, V);
  constexpr int NS = ns_of(L, P, V);
  constexpr int NB = S::R0 / R;  // butterflies per thread
  constexpr int STEP = L / (NS * R);
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int b = t + q * S::TPC;
#pragma unroll
    for (int s = 0; s < R; ++s) v[q * R + s] = pload(buf + pad_idx(b + s * (L / R), S::PS) * STRIDE);
  }
  __syncthreads();
  if constexpr (P + 1 == S::NP) at_free();
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int b = t + q * S::TPC;
    if constexpr (TABLE) {
      const int k = (b & (NS - 1)) * STEP;
#pragma unroll
      for (int s = 1; s < R; ++s) {
        const auto w = tw_ld(twL + k * s);
        v[q * R + s] = pmul(v[q * R + s], (T)w.x, (T)w.y);
      }
    } else if (NS > 1) {
      T sn, cs, wc[R], ws[R];
      turn_sincos(-(T)(b & (NS - 1)) / (T)(NS * R), &sn, &cs);
      powers<T, R>(cs, sn, wc, ws);
#pragma unroll
      for (int s = 1; s < R; ++s) v[q * R + s] = pmul(v[q * R + s], wc[s], ws[s]);
    }
    dft<T, R>(v + q * R);
  }
  if constexpr (P + 1 < S::NP) {
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int b = t + q * S::TPC;
      const int base = (b / NS) * NS * R + (b & (NS - 1));
#pragma unroll
      for (int s = 0; s < R; ++s) pstore(buf + pad_idx(base + s * NS, S::PS) * STRIDE, v[q * R + s]);
    }
    __syncthreads();
    passes<T, L, V, STRIDE, P + 1, TABLE, F>(v, buf, t, twL, at_free);
  }
}

// store pass-0 outputs (one radix-R0 butterfly per thread, Ns = 1)
template <typename T, int L, int V, int STRIDE>
__device__ __forceinline__ void store_pass0(const Pair<T>* v, typename PairMem<T>::type* buf, int t) {
  using S = Shape<T, L, V>;
#pragma unroll
  for (int s = 0; s < S::R0; ++s) pstore(buf + pad_idx(t * S::R0 + s, S::PS) * STRIDE, v[s]);
  __syncthreads();
}

// ----------------------------------------------------- spindown phase
// e^{-i 2 pi phi(s)}, phi = ((p3 s + p2) s + p1) s + p0 cycles, s exact in FP32.
// FP32 path: Horner in double-float (error-free products and sums with
// explicitly rounded operations so the compiler cannot contract them), mod
// 1 in double-float, then the rotation of the reduced phase f in [-1/2, 1/2]
// (|2 pi f| <= pi, where the hardware sine/cosine is accurate to ~4e-7).
__device__ __forceinline__ void spin_rot(const TmplCoef& c, int si, float* cs, float* sn) {
  const float s = (float)si;
  float h = c.hi[3], l = c.lo[3];
#pragma unroll
  for (int q = 2; q >= 0; --q) {
    float p = __fmul_rn(h, s);
    float e = fmaf(h, s, -p);
    e = fmaf(l, s, e);
    float S = __fadd_rn(p, c.hi[q]);
    float bb = __fsub_rn(S, p);
    float err = __fadd_rn(__fsub_rn(p, __fsub_rn(S, bb)), __fsub_rn(c.hi[q], bb));
    err = __fadd_rn(err, __fadd_rn(e, c.lo[q]));
    h = __fadd_rn(S, err);
    l = __fsub_rn(err, __fsub_rn(h, S));
  }
  const float k = rintf(h);
  const float f = __fadd_rn(__fsub_rn(h, k), l);
  float sv, cv;
  __sincosf(6.28318530717958647692f * f, &sv, &cv);
  *cs = cv;
  *sn = -sv;
}
__device__ __forceinline__ void spin_rot(const TmplCoef& c, int si, double* cs, double* sn) {
  const double s = (double)si;
  double ph = ((c.p[3] * s + c.p[2]) * s + c.p[1]) * s + c.p[0];
  double f = ph - rint(ph);
  double sv, cv;
  sincospi(2.0 * f, &sv, &cv);
  *cs = cv;
  *sn = -sv;
}

// ------------------------------------------------------------- pass A
// One tile = CA columns.  `staged`: the column samples were copied to `buf`
// (at padded natural positions) by cp.async, or densely (one bulk copy) to
// `buf` or, with schedule bit 4, to the separate area `stg`; otherwise they
// are loaded from global memory straight into registers.  at_staged() runs
// once every thread has read `stg` (after the barrier that ends the first
// pass's stores).
template <typename T, int L, int CA, int V, bool STAGED, typename F = NoOp, typename H = NoOp>
__device__ __forceinline__ void pass_a_tile(int tile, typename PairMem<T>::type* buf, int c, int t,
                                            const typename PairMem<T>::type* __restrict__ G, int64_t lc,
                                            int n, int n1, const typename TwT<T>::type* __restrict__ twL,
                                            const TmplCoef& tc, T inv_n,
                                            typename PairMem<T>::type* __restrict__ Z, const F& at_free = F(),
                                            const typename PairMem<T>::type* stg = nullptr,
                                            const H& at_staged = H()) {
  using S = Shape<T, L, V>;
  using PM = typename PairMem<T>::type;
  // staged column: padded positions (per-thread copies) or dense (one bulk copy)
  constexpr bool kSep = (V & 16) != 0;
  constexpr bool kDense = (V & 4) != 0 || kSep;
  const int col = tile * CA + c;
  const PM* gcol = G + (int64_t)col * lc;
  Pair<T> v[S::R0];
  auto load = [&](int s) {
    const int n2 = t + s * S::TPC;
    const int j = col + n1 * n2;
    if (j < n) {
      Pair<T> g = STAGED ? pload(kSep ? stg + n2 : buf + (kDense ? n2 : pad_idx(n2, S::PS))) : pload_g(gcol + n2);
      T cs, sn;
      spin_rot(tc, j - tc.J, &cs, &sn);
      v[s] = pmul(g, cs, sn);
    } else {
      v[s] = pzero<T>();
    }
  };
  // zero padding to at least twice the data (n <= n1 L / 2): no column has
  // a sample at n2 >= L/2, the upper half of every first butterfly is zero
  const bool half = (int64_t)n1 * (L / 2) >= (int64_t)n;
  if (half) {
#pragma unroll
    for (int s = 0; s < S::R0 / 2; ++s) load(s);
  } else {
#pragma unroll
    for (int s = 0; s < S::R0; ++s) load(s);
  }
  if constexpr (STAGED && !kSep) __syncthreads();  // the staged column is overwritten below
  if (half) dft_half<T, S::R0>(v);
  else dft<T, S::R0>(v);
  store_pass0<T, L, V, 1>(v, buf, t);
  at_staged();
  passes<T, L, V, 1, 1, false, F>(v, buf, t, twL, at_free);

  // four-step twiddle W_N^{col k2} = W_N^{col b} (W_N^{col NSL})^s for
  // k2 = b + s * NSL, and store Z[col][k2]
  T sc, ss, stc[S::RL], sts[S::RL];
  turn_sincos(-(T)(col * S::NSL) * inv_n, &ss, &sc);
  powers<T, S::RL>(sc, ss, stc, sts);
  PM* zrow = Z + (int64_t)col * L;
  constexpr int NB = S::R0 / S::RL;
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int b = t + q * S::TPC;
    T bc, bs;
    turn_sincos(-(T)(col * b) * inv_n, &bs, &bc);
    Pair<T>* x = v + q * S::RL;
#pragma unroll
    for (int s = 0; s < S::RL; ++s) {
      const T wc = bc * stc[s] - bs * sts[s];
      const T ws = bc * sts[s] + bs * stc[s];
      pstore(zrow + b + s * S::NSL, pmul(x[s], wc, ws));
    }
  }
}

template <typename T, int L, int C, int V> constexpr int min_blocks() {
  // radix-8 variants: ask for enough resident CTAs to cap registers at 64;
  // one-buffer radix-16 variants of up to 256 threads: two CTAs per SM
  // (three with bit 3), which their shared memory allows
  constexpr int threads = C * Shape<T, L, V>::TPC;
  constexpr int want = 65536 / (threads * 64);
  if constexpr ((V & 1) == 0 && (V & 2) != 0) return threads <= 256 ? ((V & 8) ? 3 : 2) : 1;
  return ((V & 1) && kR8MinBlocks > 0 && want > 1) ? want : 1;
}

// Direct mode (kPipeline = false): one tile per CTA.  Pipelined mode: the
// CTA transforms tiles b, b + grid, ...; the next tile's samples are copied
// asynchronously into the other buffer while the current one is
// transformed in place, or, with one buffer, into that buffer as soon as
// the last Stockham pass has read it (under that pass and the epilogue).
template <typename T, int L, int CA, int V>
__global__ void __launch_bounds__(CA * Shape<T, L, V>::TPC, (min_blocks<T, L, CA, V>()))
k_pass_a(const typename PairMem<T>::type* __restrict__ G, int64_t lc, int n, int n1,
         const typename TwT<T>::type* __restrict__ twL, const TmplCoef* __restrict__ coefp,
         typename PairMem<T>::type* __restrict__ Z, int* __restrict__ err, int wait_limit) {
  using S = Shape<T, L, V>;
  using B = Buf<T, L, CA, V>;
  using PM = typename PairMem<T>::type;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  PM* smem = reinterpret_cast<PM*>(smem_raw);
  const int c = threadIdx.x / S::TPC;
  const int t = threadIdx.x % S::TPC;
  const TmplCoef tc = *coefp;
  const int log2N = log2c(L) + 31 - __clz(n1);
  const T inv_n = (T)1 / (T)(1 << log2N);
  if constexpr (!kPipeline) {
    pass_a_tile<T, L, CA, V, false>(blockIdx.x, smem + c * S::LP, c, t, G, lc, n, n1, twL, tc, inv_n, Z);
  } else if constexpr ((V & 16) != 0) {
    // Input double-buffered: thread 0 copies the next column's samples
    // (those with j = col + n1 n2 < n, contiguous in G) densely into the
    // staging area behind the column buffer with one bulk copy, counted in
    // bytes on an mbarrier, as soon as every thread has read the current
    // column's; the copy runs under the whole transform.  Copy u completes
    // phase u.
    static_assert(CA == 1 && B::NBUF == 1 && sizeof(T) == 4, "separate staging: one FP32 column per CTA");
    static_assert(L * sizeof(PM) < (1u << 20), "mbarrier transaction count");
    const int n_tiles = n1;
    const int m_max = (n + n1 - 1) / n1;  // samples in column 0, the most of any column
    PM* stg = smem + S::LP;
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(stg + m_max);
    if (threadIdx.x == 0) {
      mbar_init(bar, 1);
      mbar_fence_init();
    }
    __syncthreads();
    unsigned issued = 0, waited = 0;
    auto issue = [&](int col) {
      const int m = col < n ? (n - col + n1 - 1) / n1 : 0;
      fence_proxy_async();  // the staging area's earlier reads precede the copy
      mbar_expect_tx(bar, (unsigned)(m * sizeof(PM)));
      if (m > 0) bulk_load(stg, G + (int64_t)col * lc, (unsigned)(m * sizeof(PM)), bar);
      ++issued;
    };
    int tile = blockIdx.x;
    if (threadIdx.x == 0 && tile < n_tiles) issue(tile);
    bool all_ok = true;
    for (; tile < n_tiles; tile += gridDim.x) {
      // the plan may shorten this wait (tests of the timeout path); the
      // drain below always keeps the full limit
      const bool ok = mbar_wait(bar, waited & 1u, wait_limit >= 0 ? wait_limit : kWaitLimit);
      if (ok) ++waited;
      all_ok = __syncthreads_and(ok) != 0;
      if (!all_ok) break;
      const int next = tile + gridDim.x;
      pass_a_tile<T, L, CA, V, true>(tile, smem, c, t, G, lc, n, n1, twL, tc, inv_n, Z, NoOp(), stg, [&] {
        if (threadIdx.x == 0 && next < n_tiles) issue(next);
      });
    }
    if (!all_ok) {
      // a wait ran out: record it, then give the copy still in flight a
      // bounded chance to land before the CTA's shared memory goes away
      if (threadIdx.x == 0) {
        if (err) atomicCAS(err, 0, FSTAT_ERR_TIMEOUT);
        for (unsigned u = waited; u < issued; ++u) mbar_wait(bar, u & 1u);
      }
      return;
    }
  } else {
    const int n_tiles = n1 / CA;
    auto stage = [&](int it) { return smem + (B::NBUF == 2 ? (it & 1) : 0) * (CA * S::LP) + c * S::LP; };
    auto prefetch = [&](int tile, PM* dst) {
      const int col = tile * CA + c;
      const PM* gcol = G + (int64_t)col * lc;
#pragma unroll
      for (int s = 0; s < S::R0; ++s) {
        const int n2 = t + s * S::TPC;
        if (col + n1 * n2 < n) cp_pair(dst + pad_idx(n2, S::PS), gcol + n2);
      }
    };
    int tile = blockIdx.x;
    if (tile < n_tiles) prefetch(tile, stage(0));
    cp_async_commit();
    for (int it = 0; tile < n_tiles; ++it, tile += gridDim.x) {
      PM* buf = stage(it);
      const int next = tile + gridDim.x;
      if constexpr (B::NBUF == 2) {
        if (next < n_tiles) prefetch(next, stage(it + 1));
        cp_async_commit();
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();
      if constexpr (B::NBUF == 2) {
        pass_a_tile<T, L, CA, V, true>(tile, buf, c, t, G, lc, n, n1, twL, tc, inv_n, Z);
        __syncthreads();  // this buffer is the prefetch target two tiles on
      } else {
        // no barrier after the tile: it stopped reading the buffer before
        // the barrier at which the next tile's copies were issued
        pass_a_tile<T, L, CA, V, true>(tile, buf, c, t, G, lc, n, n1, twL, tc, inv_n, Z, [&] {
          if (next < n_tiles) prefetch(next, buf);
          cp_async_commit();
        });
      }
    }
  }
}

// ------------------------------------------------------------- pass B
// Peaks epilogue.  sf holds the tile's 2F as [r][c] (r = ascending row of
// the output, c = column of the CTA), so bin m = k2_0 + c + n2 r increases
// with the flat index f = r CB + c.  Each thread takes E consecutive
// values.  Band boundaries fall on multiples of a power of two in f (every
// band is 2^log2_band consecutive bins and k2_0 is a multiple of CB), so
// when no thread's run straddles one, the lanes of one band form an
// aligned power-of-two group: a masked butterfly gives the group maximum
// and the group's first lane alone updates the band key.
template <int CB, int E>
__device__ __forceinline__ void peak_epilogue(const float* sf, int k2_0, int n2, const PeakArgs& pk,
                                              unsigned long long* ks) {
  constexpr unsigned FULL = 0xffffffffu;
  const int f0 = threadIdx.x * E;
  float v[E];
  if constexpr (E % 4 == 0) {
#pragma unroll
    for (int j = 0; j < E; j += 4) {
      const float4 q = *reinterpret_cast<const float4*>(sf + f0 + j);
      v[j] = q.x; v[j + 1] = q.y; v[j + 2] = q.z; v[j + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < E; ++j) v[j] = sf[f0 + j];
  }
  auto bin = [&](int f) { return (unsigned)(k2_0 + (f & (CB - 1)) + n2 * (f / CB)); };
  float best = v[0];
  int jb = 0;
#pragma unroll
  for (int j = 1; j < E; ++j)
    if (v[j] > best) { best = v[j]; jb = j; }
  const int lane = threadIdx.x & 31;
  if (pk.count && __any_sync(FULL, best > pk.thr)) {
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const bool hit = v[j] > pk.thr;
      const unsigned bal = __ballot_sync(FULL, hit);
      if (!bal) continue;
      const int leader = __ffs(bal) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(pk.count, (unsigned long long)__popc(bal));
      base = __shfl_sync(FULL, base, leader);
      if (hit) {
        const unsigned long long idx = base + __popc(bal & ((1u << lane) - 1u));
        if (idx < (unsigned long long)pk.cap) {
          fstat_peak e;
          e.tmpl = pk.tmpl;
          e.bin = (int32_t)bin(f0 + j);
          e.twoF = v[j];
          pk.peaks[idx] = e;
        }
      }
    }
  }
  if (pk.band_key) {
    // shared keys of this CTA when it accumulates, else the global row
    unsigned long long* keys = ks ? ks : pk.band_key;
    const int lb = pk.log2_band;
    // a band is a run of 2^lp consecutive f: CB W / n2 when it spans whole
    // rows, else the CTA's part of one row (at most CB values)
    constexpr int LCB = log2c(CB), LE = log2c(E);
    const int ln2 = 31 - __clz(n2);
    const int lp = lb >= ln2 ? LCB + lb - ln2 : (lb < LCB ? lb : LCB);
    // In shared keys, a band within one warp's values has a single writer
    // (the same lane in every tile), so a plain update suffices.
    const bool excl = ks != nullptr && lp <= LE + 5;
    auto update = [&](unsigned b, unsigned long long key) {
      if (excl) {
        if (key > keys[b]) keys[b] = key;
      } else {
        atomicMax(keys + b, key);
      }
    };
    if (lp >= LE) {
      // the run lies in one band; lanes of a band form an aligned group
      const unsigned band = bin(f0) >> lb;
      unsigned long long key = band_key(best, bin(f0 + jb));
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long ok = __shfl_xor_sync(FULL, key, o);
        if (o < (1 << (lp - LE)) && ok > key) key = ok;
      }
      if ((lane & ((1 << (lp - LE < 5 ? lp - LE : 5)) - 1)) == 0) update(band, key);
    } else {
      // runs of P values, each one band, inside this thread's values
      const int pm = (1 << lp) - 1;
      float bv = v[0];
      int bj = 0;
#pragma unroll
      for (int j = 1; j < E; ++j) {
        if ((j & pm) == 0) {
          update(bin(f0 + bj) >> lb, band_key(bv, bin(f0 + bj)));
          bv = v[j]; bj = j;
        } else if (v[j] > bv) {
          bv = v[j]; bj = j;
        }
      }
      update(bin(f0 + bj) >> lb, band_key(bv, bin(f0 + bj)));
    }
  }
}

// Schedule bit 3: rows [0, L/2) of the tile come from `stg` (same layout
// as the buffer), and at_staged() runs once every thread has read them.
template <typename T, int L, int CB, int V, bool STAGED, int MODE, typename F = NoOp, typename H = NoOp>
__device__ __forceinline__ void pass_b_tile(int tile, typename PairMem<T>::type* buf, int c, int t,
                                            const typename PairMem<T>::type* __restrict__ Z, int n2,
                                            const typename TwT<T>::type* __restrict__ twL, T kA, T kB, T kC,
                                            float* __restrict__ out, const PeakArgs& pk,
                                            unsigned long long* ks, float* sf_sep, const F& at_free = F(),
                                            const typename PairMem<T>::type* stg = nullptr,
                                            const H& at_staged = H()) {
  using S = Shape<T, L, V>;
  const int k2 = tile * CB + c;
  constexpr int NB = S::R0 / S::RL;
  // accumulate mode: the running sums this thread adds to, loaded before
  // the transform so their latency hides under it
  float acc[MODE == kAccumulate ? S::R0 : 1];
  if constexpr (MODE == kAccumulate) {
#pragma unroll
    for (int q = 0; q < NB; ++q)
#pragma unroll
      for (int s = 0; s < S::RL; ++s) {
        const int r = (t + q * S::TPC + s * S::NSL + L / 2) & (L - 1);
        const int mg = k2 + n2 * r - pk.shift;
        acc[q * S::RL + s] = (unsigned)mg < (unsigned)(n2 * L) ? out[mg] : 0.f;
      }
  }
  Pair<T> v[S::R0];
  // staged rows: padded positions (per-thread copies) or dense rows (TMA boxes)
  constexpr bool kDense = (V & 4) != 0;
#pragma unroll
  for (int s = 0; s < S::R0; ++s)
    v[s] = STAGED ? pload(((V & 8) && s < S::R0 / 2 ? stg : buf) +
                          (kDense ? t + s * S::TPC : pad_idx(t + s * S::TPC, S::PS)) * CB)
                  : pload_g(Z + (int64_t)(t + s * S::TPC) * n2 + k2);
  if constexpr (STAGED) {
    __syncthreads();  // the staged rows are overwritten below
    at_staged();
  }
  dft<T, S::R0>(v);
  store_pass0<T, L, V, CB>(v, buf, t);
  passes<T, L, V, CB, 1, kPassBTable && sizeof(T) == 4, F>(v, buf, t, twL, at_free);

  // peaks epilogue: the tile's 2F in its own region, or in the CTA's stage
  // once every thread is done with it as the exchange buffer
  float* sf = sf_sep ? sf_sep : reinterpret_cast<float*>(buf - c);
  if constexpr (MODE == kPeaks) {
    if (!sf_sep) __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int b = t + q * S::TPC;
#pragma unroll
    for (int s = 0; s < S::RL; ++s) {
      const Pair<T>& x = v[q * S::RL + s];
      const int k1 = b + s * S::NSL;
      T fa2 = x.ar * x.ar + x.ai * x.ai;
      T fb2 = x.br * x.br + x.bi * x.bi;
      T re = x.ar * x.br + x.ai * x.bi;
      T tf = kB * fa2 + kA * fb2 - kC * re;
      const int r = (k1 + L / 2) & (L - 1);
      if constexpr (MODE == kPeaks) {
        sf[r * CB + c] = (float)tf;
      } else if constexpr (MODE == kAccumulate) {
        // semi-coherent sum: this segment's bin m adds to global bin m - shift
        const int mg = k2 + n2 * r - pk.shift;
        if ((unsigned)mg < (unsigned)(n2 * L)) out[mg] = acc[q * S::RL + s] + (float)tf;
      } else {
        __stcs(out + k2 + n2 * r, (float)tf);  // streaming store: keep G and Z in L2
      }
    }
  }
  if constexpr (MODE == kPeaks) {
    __syncthreads();
    peak_epilogue<CB, L * CB / (CB * S::TPC)>(sf, tile * CB, n2, pk, ks);
  }
}

template <typename T, int L, int CB, int V, int MODE>
__global__ void __launch_bounds__(CB * Shape<T, L, V>::TPC, (min_blocks<T, L, CB, V>()))
k_pass_b(const typename PairMem<T>::type* __restrict__ Z, int n2,
         const typename TwT<T>::type* __restrict__ twL, const SkyConst* __restrict__ sky,
         float* __restrict__ out, const PeakArgs pk, const __grid_constant__ CUtensorMap zmap) {
  using S = Shape<T, L, V>;
  using B = Buf<T, L, CB, V>;
  using PM = typename PairMem<T>::type;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  PM* smem = reinterpret_cast<PM*>(smem_raw);
  const int c = threadIdx.x % CB;
  const int t = threadIdx.x / CB;
  T kA, kB, kC;
  if constexpr (sizeof(T) == 4) { kA = sky->kAf; kB = sky->kBf; kC = sky->kCf; }
  else { kA = sky->kA; kB = sky->kB; kC = sky->kC; }
  // peaks mode with whole-row bands: this CTA's band keys in shared memory
  unsigned long long* ks = nullptr;
  float* sf_sep = nullptr;
  if constexpr (MODE == kPeaks && PeakSmem<T, L, CB, V>::SEP)
    sf_sep = reinterpret_cast<float*>(smem_raw + PeakSmem<T, L, CB, V>::KEYS_END);
  int n_bands = 0;
  if constexpr (MODE == kPeaks && PeakSmem<T, L, CB, V>::ACC) {
    if (pk.band_key && pk.log2_band >= 31 - __clz(n2)) {
      n_bands = (L * n2) >> pk.log2_band;
      if (n_bands <= kPeakBands) {
        ks = reinterpret_cast<unsigned long long*>(smem_raw + Buf<T, L, CB, V>::BYTES);
        for (int b = threadIdx.x; b < n_bands; b += blockDim.x) ks[b] = 0ull;
        // visible to the epilogue after the tile loop's first barrier
      }
    }
  }
  if constexpr (!kPipeline) {
    pass_b_tile<T, L, CB, V, false, MODE>(blockIdx.x, smem + c, c, t, Z, n2, twL, kA, kB, kC, out, pk, ks,
                                          nullptr);
  } else if constexpr ((V & 4) != 0) {
    // Tiles by bulk tensor copies: thread 0 loads tile k's CB columns of
    // all L rows as boxes of kTmaRows rows into stage k mod NBUF, counted
    // on that stage's mbarrier; use u of a stage completes phase u.  With
    // one stage (and no peaks epilogue that reuses it) the next tile's
    // copies start as soon as the last Stockham pass has read the stage.
    constexpr bool kEarly = B::NBUF == 1 && (MODE != kPeaks || PeakSmem<T, L, CB, V>::SEP);
    __shared__ unsigned long long s_bar[2];
    const int n_tiles = n2 / CB;
    if (threadIdx.x == 0) {
      mbar_init(&s_bar[0], 1);
      mbar_init(&s_bar[1], 1);
      mbar_fence_init();
    }
    __syncthreads();
    unsigned issued[2] = {0u, 0u};  // loads issued per stage (thread 0)
    unsigned waited[2] = {0u, 0u};  // loads waited for per stage (every thread)
    auto issue = [&](int tl, int b) {
      PM* dst = smem + b * (CB * S::LP);
      fence_proxy_async();  // the stage's earlier reads and writes precede the copy
      mbar_expect_tx(&s_bar[b], (unsigned)(L * CB * sizeof(PM)));
#pragma unroll 1
      for (int r = 0; r < L; r += kTmaRows)
        tma_load_2d(dst + r * CB, &zmap, tl * CB * (int)(sizeof(PM) / sizeof(float)), r, &s_bar[b]);
      ++issued[b];
    };
    int tile = blockIdx.x;
    if (threadIdx.x == 0 && tile < n_tiles) issue(tile, 0);
    bool all_ok = true;  // CTA-wide: every thread's wait succeeded
    int it = 0;
    for (; tile < n_tiles; ++it, tile += gridDim.x) {
      const int b = B::NBUF == 2 ? (it & 1) : 0;
      if (threadIdx.x == 0) {
        if constexpr (B::NBUF == 2) {
          if (tile + (int)gridDim.x < n_tiles) issue(tile + gridDim.x, b ^ 1);
        } else if constexpr (!kEarly) {
          if (it > 0) issue(tile, 0);  // the previous tile released the only stage
        }
      }
      // the plan may shorten this first wait (tests of the timeout path); the
      // drain below always keeps the full limit
      const bool ok = mbar_wait(&s_bar[b], waited[b] & 1u, pk.wait_set ? pk.wait_limit : kWaitLimit);
      if (ok) ++waited[b];
      all_ok = __syncthreads_and(ok) != 0;
      if (!all_ok) break;
      if constexpr (kEarly) {
        // no barrier after the tile: it stopped reading the stage before the
        // barrier at which thread 0 issued the next tile's copies
        const int next = tile + gridDim.x;
        pass_b_tile<T, L, CB, V, true, MODE>(tile, smem + c, c, t, Z, n2, twL, kA, kB, kC, out, pk, ks, sf_sep,
                                             [&] {
                                               if (threadIdx.x == 0 && next < n_tiles) issue(next, 0);
                                             });
      } else {
        pass_b_tile<T, L, CB, V, true, MODE>(tile, smem + b * (CB * S::LP) + c, c, t, Z, n2, twL, kA, kB, kC,
                                             out, pk, ks, sf_sep);
        fence_proxy_async();  // this thread's accesses to the stage precede the next bulk copy into it
        __syncthreads();      // this stage is the load target NBUF tiles on
      }
    }
    if (!all_ok) {
      // a wait ran out: record it, then give the loads still in flight a
      // bounded chance to land before the CTA's shared memory goes away
      if (threadIdx.x == 0) {
        if (pk.err) atomicCAS(pk.err, 0, FSTAT_ERR_TIMEOUT);
        for (int b = 0; b < 2; ++b)
          for (unsigned u = waited[b]; u < issued[b]; ++u) mbar_wait(&s_bar[b], u & 1u);
      }
      return;
    }
    if constexpr (MODE == kPeaks) {
      if (ks) {
        if constexpr (kEarly) __syncthreads();  // else the loop ended on one
        // every tile's keys are in
        for (int b = threadIdx.x; b < n_bands; b += blockDim.x)
          if (ks[b]) atomicMax(pk.band_key + b, ks[b]);
      }
    }
  } else {
    const int n_tiles = n2 / CB;
    auto stage = [&](int it) { return smem + (B::NBUF == 2 ? (it & 1) : 0) * (CB * S::LP) + c; };
    // rows [s0 R0/16 .. ) of the tile: s in [s0, s1) of each thread's rows t + s TPC
    auto prefetch_rows = [&](int tile, PM* dst, int s0, int s1) {
      const int k2 = tile * CB + c;
#pragma unroll
      for (int s = 0; s < S::R0; ++s) {
        if (s < s0 || s >= s1) continue;
        const int n1 = t + s * S::TPC;
        cp_pair(dst + pad_idx(n1, S::PS) * CB, Z + (int64_t)n1 * n2 + k2);
      }
    };
    // bit 3: the first half of the rows in their own staging area
    constexpr bool kSplit = (V & 8) != 0;
    static_assert(!kSplit || (B::NBUF == 1 && MODE != kPeaks && sizeof(T) == 4), "split staging: one buffer");
    PM* stg = kSplit ? smem + CB * S::LP + c : nullptr;
    constexpr int kLo = kSplit ? S::R0 / 2 : 0;
    auto prefetch = [&](int tile, PM* dst) { prefetch_rows(tile, dst, kLo, S::R0); };
    // with one buffer (and no peaks epilogue that reuses it) the next
    // tile's copies start as soon as the last Stockham pass has read it
    constexpr bool kEarly = B::NBUF == 1 && (MODE != kPeaks || PeakSmem<T, L, CB, V>::SEP);
    int tile = blockIdx.x;
    if constexpr (B::NBUF == 2 || kEarly) {
      if (tile < n_tiles) {
        if constexpr (kSplit) prefetch_rows(tile, stg, 0, kLo);
        prefetch(tile, stage(0));
      }
      cp_async_commit();
    }
    for (int it = 0; tile < n_tiles; ++it, tile += gridDim.x) {
      PM* buf = stage(it);
      const int next = tile + gridDim.x;
      if constexpr (B::NBUF == 2) {
        if (next < n_tiles) prefetch(next, stage(it + 1));
        cp_async_commit();
        cp_async_wait<1>();
      } else if constexpr (kEarly) {
        cp_async_wait<0>();
      } else {
        prefetch(tile, buf);
        cp_async_commit();
        cp_async_wait<0>();
      }
      __syncthreads();
      if constexpr (kEarly) {
        // no barrier after the tile: it stopped reading the buffer before
        // the barrier at which the next tile's copies were issued
        pass_b_tile<T, L, CB, V, true, MODE>(
            tile, buf, c, t, Z, n2, twL, kA, kB, kC, out, pk, ks, sf_sep,
            [&] {
              if (next < n_tiles) prefetch(next, buf);
              cp_async_commit();
            },
            stg, [&] {
              if constexpr (kSplit) {
                if (next < n_tiles) prefetch_rows(next, stg, 0, kLo);
                cp_async_commit();
              }
            });
      } else {
        pass_b_tile<T, L, CB, V, true, MODE>(tile, buf, c, t, Z, n2, twL, kA, kB, kC, out, pk, ks, sf_sep);
        __syncthreads();  // this buffer is the prefetch target two tiles on
      }
    }
    if constexpr (MODE == kPeaks) {
      if (ks) {
        if constexpr (kEarly) __syncthreads();  // else the loop ended on one
        // every tile's keys are in
        for (int b = threadIdx.x; b < n_bands; b += blockDim.x)
          if (ks[b]) atomicMax(pk.band_key + b, ks[b]);
      }
    }
  }
}

// ------------------------------------------------------------- launchers
// Resident CTAs of a persistent kernel: SM count x CTAs per SM (queried
// once per kernel instantiation).
template <typename K>
cudaError_t resident_ctas(K kernel, int threads, size_t smem, int* out, int* out_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  *out = sms * per_sm;
  *out_per_sm = per_sm;
  return cudaSuccess;
}

// Persistent grid: every resident CTA, or at most `res` per SM (res > 0),
// which leaves room on each SM for a CTA of the other pass of a
// neighbouring template running on another stream.
inline int persistent_grid(int tiles, int ctas, int per_sm, int res) {
  int g = ctas;
  if (res > 0 && res < per_sm) g = ctas / per_sm * res;
  return (!kPipeline || tiles < g) ? tiles : g;
}

// Dynamic shared memory a CTA may opt into (227 KB on sm_100 / sm_103).
constexpr size_t kSmemOptIn = (size_t)227 * 1024;

template <typename T, int L, int CA, int V>
cudaError_t run_a(const void* G, int64_t lc, int64_t n, int n1, const void* twA, const TmplCoef* coef, void* Z,
                  int* err, int wait_limit, cudaStream_t st, int res) {
  using S = Shape<T, L, V>;
  using PM = typename S::PM;
  // separate staging (bit 4): the column buffer, the most samples of any
  // column (dense) and the mbarrier, sized per launch
  size_t smem = Buf<T, L, CA, V>::BYTES;
  if constexpr ((V & 16) != 0) {
    smem += (size_t)((n + n1 - 1) / n1) * sizeof(PM) + 16;
    if (smem > kSmemOptIn) return cudaErrorInvalidConfiguration;
  }
  constexpr int threads = CA * S::TPC;
  // resident CTAs for this launch's shared memory (separate staging: it
  // depends on the plan, so the query is redone when it changes)
  static int ctas = 0, per_sm = 0;
  static size_t ctas_smem = 0;
  if (!ctas || ctas_smem != smem) {
    cudaError_t e = resident_ctas(k_pass_a<T, L, CA, V>, threads, smem, &ctas, &per_sm);
    if (e != cudaSuccess) return e;
    ctas_smem = smem;
  }
  if (n1 % CA) return cudaErrorInvalidConfiguration;
  const int tiles = n1 / CA;
  using TW = typename S::TW;
  const int grid = persistent_grid(tiles, ctas, per_sm, res);
  k_pass_a<T, L, CA, V><<<grid, threads, smem, st>>>((const PM*)G, lc, (int)n, n1, (const TW*)twA, coef, (PM*)Z, err,
                                                     wait_limit);
  return cudaGetLastError();
}

// cuTensorMapEncodeTiled, through the runtime's driver entry point (the
// library does not link the driver API).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
inline EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
  }
  return fn;
}

// Tensor map of pass B's input (FP32 pairs): L rows of n2 pairs, i.e. rows
// of 4 n2 floats at a pitch of 16 n2 bytes; a box is CB pairs (16 CB bytes,
// a multiple of 16) by min(L, kTmaRows) rows.  Box x coordinates are
// multiples of 4 CB floats, so every copy starts on a 16-byte boundary.
inline cudaError_t z_tensor_map(CUtensorMap* map, const void* Z, int L, int n2, int CB) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  if (((uintptr_t)Z & 15) || CB * 4 > 256) return cudaErrorInvalidValue;
  const cuuint64_t dims[2] = {(cuuint64_t)n2 * 4, (cuuint64_t)L};
  const cuuint64_t strides[1] = {(cuuint64_t)n2 * 16};
  const cuuint32_t box[2] = {(cuuint32_t)(CB * 4), (cuuint32_t)(L < kTmaRows ? L : kTmaRows)};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(Z), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <typename T, int L, int CB, int V, int MODE>
cudaError_t run_b(const void* Z, int n2, const void* twB, const SkyConst* sky, float* out, const PeakArgs& pk,
                  cudaStream_t st, int res) {
  using S = Shape<T, L, V>;
  // split staging (bit 3): half a tile more
  constexpr size_t smem = MODE == kPeaks ? PeakSmem<T, L, CB, V>::BYTES
                          : (V & 8)      ? Buf<T, L, CB, V>::BYTES + Buf<T, L, CB, V>::ONE / 2
                                         : Buf<T, L, CB, V>::BYTES;
  if constexpr (smem > kSmemOptIn) return cudaErrorInvalidConfiguration;
  constexpr int threads = CB * S::TPC;
  static_assert(MODE != kPeaks || (L * CB * sizeof(float) <= Buf<T, L, CB, V>::ONE), "peaks epilogue reuses the stage");
  static_assert(MODE != kPeaks || threads % 32 == 0, "peaks epilogue works on whole warps");
  static int ctas = 0, per_sm = 0;
  if (!ctas) {
    cudaError_t e = resident_ctas(k_pass_b<T, L, CB, V, MODE>, threads, smem, &ctas, &per_sm);
    if (e != cudaSuccess) return e;
  }
  if (n2 % CB) return cudaErrorInvalidConfiguration;
  const int tiles = n2 / CB;
  const int grid = persistent_grid(tiles, ctas, per_sm, res);
  CUtensorMap zmap;
  memset(&zmap, 0, sizeof(zmap));
  if constexpr ((V & 4) != 0) {
    static_assert(sizeof(T) == 4 && kPipeline, "TMA tiles: FP32, persistent pass");
    static_assert(L * CB * sizeof(typename S::PM) < (1u << 20), "mbarrier transaction count");
    const cudaError_t e = z_tensor_map(&zmap, Z, L, n2, CB);
    if (e != cudaSuccess) return e;
  }
  k_pass_b<T, L, CB, V, MODE><<<grid, threads, smem, st>>>(
      (const typename S::PM*)Z, n2, (const typename S::TW*)twB, sky, out, pk, zmap);
  return cudaGetLastError();
}

// CTA shapes compiled per length: the default plus wider ones and the
// radix-8 schedule, only for the lengths the configured workloads use
// (512..4096) and only in FP32.
template <int L> constexpr bool wide_variants() { return L >= 512; }

// shape code: c = columns (A) / rows (B) per CTA, 0 = default; v = schedule
template <typename T, int L, int V>
cudaError_t pick_a_v(int ca, const void* G, int64_t lc, int64_t n, int n1, const void* twA, const TmplCoef* coef,
                     void* Z, int* err, int wait_limit, cudaStream_t st, int res) {
  switch (ca) {
    case 1: if constexpr (cfg_ok<T, L, 1, V>()) return run_a<T, L, 1, V>(G, lc, n, n1, twA, coef, Z, err, wait_limit, st, res); break;
    case 2: if constexpr (cfg_ok<T, L, 2, V>()) return run_a<T, L, 2, V>(G, lc, n, n1, twA, coef, Z, err, wait_limit, st, res); break;
    case 4: if constexpr (cfg_ok<T, L, 4, V>()) return run_a<T, L, 4, V>(G, lc, n, n1, twA, coef, Z, err, wait_limit, st, res); break;
    default: break;
  }
  return cudaErrorInvalidConfiguration;
}

template <typename T, int L>
cudaError_t pick_a(int ca, int v, const void* G, int64_t lc, int64_t n, int n1, const void* twA, const TmplCoef* coef,
                   void* Z, int* err, int wait_limit, cudaStream_t st, int res) {
  using S = Shape<T, L, 0>;
  if (ca <= 0) ca = S::CA_DEF;
  if (v == 0 && ca == S::CA_DEF) return run_a<T, L, S::CA_DEF, 0>(G, lc, n, n1, twA, coef, Z, err, wait_limit, st, res);
  if constexpr (sizeof(T) == 4 && wide_variants<L>()) {
    if (v == 0) return pick_a_v<T, L, 0>(ca, G, lc, n, n1, twA, coef, Z, err, wait_limit, st, res);
    if (v == 2) return pick_a_v<T, L, 2>(ca, G, lc, n, n1, twA, coef, Z, err, wait_limit, st, res);
    if constexpr (L >= 1024) {
      if (v == 1) return pick_a_v<T, L, 1>(ca, G, lc, n, n1, twA, coef, Z, err, wait_limit, st, res);
      if (v == 3) return pick_a_v<T, L, 3>(ca, G, lc, n, n1, twA, coef, Z, err, wait_limit, st, res);
      if (v == 10) return pick_a_v<T, L, 10>(ca, G, lc, n, n1, twA, coef, Z, err, wait_limit, st, res);
    }
    if constexpr (L == 8192 && kPipeline) {
      if (v == 16 && ca == 1) return run_a<T, L, 1, 16>(G, lc, n, n1, twA, coef, Z, err, wait_limit, st, res);
    }
    if constexpr (L == 4096 && kPipeline) {  // 256 threads: two CTAs per SM
      if (v == 18 && ca == 1) return run_a<T, L, 1, 18>(G, lc, n, n1, twA, coef, Z, err, wait_limit, st, res);
    }
  }
  return cudaErrorInvalidConfiguration;
}

template <typename T, int L, int V, int MODE>
cudaError_t pick_b_v(int cb, const void* Z, int n2, const void* twB, const SkyConst* sky, float* out,
                     const PeakArgs& pk, cudaStream_t st, int res) {
  switch (cb) {
    case 1: if constexpr (cfg_ok<T, L, 1, V>()) return run_b<T, L, 1, V, MODE>(Z, n2, twB, sky, out, pk, st, res); break;
    case 2: if constexpr (cfg_ok<T, L, 2, V>()) return run_b<T, L, 2, V, MODE>(Z, n2, twB, sky, out, pk, st, res); break;
    case 4: if constexpr (cfg_ok<T, L, 4, V>()) return run_b<T, L, 4, V, MODE>(Z, n2, twB, sky, out, pk, st, res); break;
    case 8: if constexpr (cfg_ok<T, L, 8, V>()) return run_b<T, L, 8, V, MODE>(Z, n2, twB, sky, out, pk, st, res); break;
    default: break;
  }
  return cudaErrorInvalidConfiguration;
}

template <typename T, int L, int MODE>
cudaError_t pick_b(int cb, int v, const void* Z, int n2, const void* twB, const SkyConst* sky, float* out,
                   const PeakArgs& pk, cudaStream_t st, int res) {
  using S = Shape<T, L, 0>;
  if (cb <= 0) cb = S::CB_DEF;
  // the peaks epilogue's band keys and 2F tile leave no room for the split
  // staging of schedule 8: the same transform with schedule 0 instead
  if (MODE == kPeaks && v == 8) v = 0;
  if (v == 0 && cb == S::CB_DEF) return run_b<T, L, S::CB_DEF, 0, MODE>(Z, n2, twB, sky, out, pk, st, res);
  if constexpr (sizeof(T) == 4 && wide_variants<L>()) {
    if (v == 0) return pick_b_v<T, L, 0, MODE>(cb, Z, n2, twB, sky, out, pk, st, res);
    if (v == 2) return pick_b_v<T, L, 2, MODE>(cb, Z, n2, twB, sky, out, pk, st, res);
    if constexpr (L >= 1024) {
      if (v == 1) return pick_b_v<T, L, 1, MODE>(cb, Z, n2, twB, sky, out, pk, st, res);
      if (v == 3) return pick_b_v<T, L, 3, MODE>(cb, Z, n2, twB, sky, out, pk, st, res);
      if constexpr (kPipeline) {  // tiles by bulk tensor copies
        if (v == 4) return pick_b_v<T, L, 4, MODE>(cb, Z, n2, twB, sky, out, pk, st, res);
        if (v == 5) return pick_b_v<T, L, 5, MODE>(cb, Z, n2, twB, sky, out, pk, st, res);
        if (v == 6) return pick_b_v<T, L, 6, MODE>(cb, Z, n2, twB, sky, out, pk, st, res);
        if (v == 7) return pick_b_v<T, L, 7, MODE>(cb, Z, n2, twB, sky, out, pk, st, res);
        if constexpr (MODE != kPeaks) {  // half the next tile staged apart
          if (v == 8) return pick_b_v<T, L, 8, MODE>(cb, Z, n2, twB, sky, out, pk, st, res);
        }
      }
    }
  }
  return cudaErrorInvalidConfiguration;
}

#define FSTAT_LEN_CASES(F, ...)            \
  case 5: return F<T, 32 __VA_ARGS__;    \
  case 6: return F<T, 64 __VA_ARGS__;    \
  case 7: return F<T, 128 __VA_ARGS__;   \
  case 8: return F<T, 256 __VA_ARGS__;   \
  case 9: return F<T, 512 __VA_ARGS__;   \
  case 10: return F<T, 1024 __VA_ARGS__; \
  case 11: return F<T, 2048 __VA_ARGS__; \
  case 12: return F<T, 4096 __VA_ARGS__;

// 8192-point columns (FP32 only: one padded column of FP64 pairs would not
// fit shared memory), compiled in a translation unit of their own
cudaError_t pick_a_8192(int ca, int v, const void* G, int64_t lc, int64_t n, int n1, const void* twA,
                        const TmplCoef* coef, void* Z, int* err, int wait_limit, cudaStream_t st, int res);

template <typename T>
cudaError_t dispatch_a(int log2_n2, int ca, int v, const void* G, int64_t lc, int64_t n, int n1, const void* twA,
                       const TmplCoef* coef, void* Z, int* err, int wait_limit, cudaStream_t st, int res = 0) {
  switch (log2_n2) {
    FSTAT_LEN_CASES(pick_a, >(ca, v, G, lc, n, n1, twA, coef, Z, err, wait_limit, st, res))
    case 13:
      if constexpr (sizeof(T) == 4) return pick_a_8192(ca, v, G, lc, n, n1, twA, coef, Z, err, wait_limit, st, res);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int MODE>
cudaError_t dispatch_b(int log2_n1, int cb, int v, const void* Z, int n2, const void* twB, const SkyConst* sky,
                       float* out, const PeakArgs& pk, cudaStream_t st, int res = 0) {
  switch (log2_n1) {
    FSTAT_LEN_CASES(pick_b, , MODE>(cb, v, Z, n2, twB, sky, out, pk, st, res))
    default: return cudaErrorInvalidValue;
  }
}

#undef FSTAT_LEN_CASES

}  // namespace fft
}  // namespace fstat
