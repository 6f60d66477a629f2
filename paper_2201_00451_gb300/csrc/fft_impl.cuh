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
// together as one 16-byte (FP32) / 32-byte (FP64) element.
#pragma once

#include "fstat_internal.cuh"

namespace fstat {
namespace fft {

// ------------------------------------------------------------ radix schedule
__host__ __device__ constexpr int np_of(int L) { return L <= 256 ? 2 : 3; }
__host__ __device__ constexpr int r_of(int L, int p) {
  return L == 32    ? (p == 0 ? 8 : 4)
       : L == 64    ? 8
       : L == 128   ? (p == 0 ? 16 : 8)
       : L == 256   ? 16
       : L == 512   ? 8
       : L == 1024  ? (p == 0 ? 16 : 8)
       : L == 2048  ? (p == 2 ? 8 : 16)
       : 16;  // 4096
}
__host__ __device__ constexpr int ns_of(int L, int p) { return p == 0 ? 1 : ns_of(L, p - 1) * r_of(L, p - 1); }
__host__ __device__ constexpr int log2c(int x) { return x <= 1 ? 0 : 1 + log2c(x / 2); }

template <typename T, int L> struct Shape {
  static constexpr int NP = np_of(L);
  static constexpr int R0 = r_of(L, 0);           // largest radix, points per thread
  static constexpr int TPC = L / R0;              // threads per column
  static constexpr int PS = log2c(R0);            // shared-memory padding shift
  static constexpr int LP = L + (L >> PS);        // padded column length
  static constexpr int RL = r_of(L, NP - 1);      // last radix
  static constexpr int NSL = L / RL;              // span of the last pass
  static constexpr int CA = TPC >= 128 ? 1 : 128 / TPC;                       // columns / CTA (A)
  static constexpr int CB0 = sizeof(T) == 4 ? 2 : 1;
  static constexpr int CB = TPC >= 128 ? CB0 : (128 / TPC > CB0 ? 128 / TPC : CB0);  // rows / CTA (B)
  using PM = typename PairMem<T>::type;
  static constexpr size_t SMEM_A = (size_t)CA * LP * sizeof(PM);
  static constexpr size_t SMEM_B = (size_t)CB * LP * sizeof(PM);
};

__device__ __forceinline__ int pad_idx(int pos, int ps) { return pos + (pos >> ps); }

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

template <typename T, int R> __device__ __forceinline__ void dft(Pair<T>* x) {
  if constexpr (R == 2) { Pair<T> a = x[0], b = x[1]; x[0] = padd(a, b); x[1] = psub(a, b); }
  else if constexpr (R == 4) dft4(x[0], x[1], x[2], x[3]);
  else if constexpr (R == 8) dft8(x);
  else dft16(x);
}

// x[q] *= w^q for q = 1..R-1, w = (c + i s); powers by binary splitting
// (error grows with log2 q, not q).
template <typename T, int R> __device__ __forceinline__ void twiddle(Pair<T>* x, T c, T s) {
  T wc[R], ws[R];
  wc[0] = (T)1; ws[0] = (T)0;
  wc[1] = c; ws[1] = s;
#pragma unroll
  for (int q = 2; q < R; ++q) {
    const int h = q / 2, l = q - h;
    wc[q] = wc[h] * wc[l] - ws[h] * ws[l];
    ws[q] = wc[h] * ws[l] + ws[h] * wc[l];
  }
#pragma unroll
  for (int q = 1; q < R; ++q) x[q] = pmul(x[q], wc[q], ws[q]);
}

// --------------------------------------------------------- Stockham passes
// After pass 0 (done by the caller, in registers), store it and run passes
// 1..NP-1.  On return v holds the last pass's outputs: butterfly
// b = t + q * TPC, output index b + s * NSL in v[q * RL + s].
// Shared-memory address of logical position pos is pad(pos) * STRIDE.
template <typename T, int L, int STRIDE, int P>
__device__ __forceinline__ void passes(Pair<T>* v, typename PairMem<T>::type* buf, int t) {
  using S = Shape<T, L>;
  constexpr int R = r_of(L, P);
  constexpr int NS = ns_of(L, P);
  constexpr int NB = S::R0 / R;  // butterflies per thread
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int b = t + q * S::TPC;
#pragma unroll
    for (int s = 0; s < R; ++s) v[q * R + s] = pload(buf + pad_idx(b + s * (L / R), S::PS) * STRIDE);
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int b = t + q * S::TPC;
    const int k = b & (NS - 1);
    if (NS > 1) {
      T sn, cs;
      sincospi_t((T)(-2 * k) / (T)(NS * R), &sn, &cs);
      twiddle<T, R>(v + q * R, cs, sn);
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
    passes<T, L, STRIDE, P + 1>(v, buf, t);
  }
}

// store pass-0 outputs (one radix-R0 butterfly per thread, Ns = 1)
template <typename T, int L, int STRIDE>
__device__ __forceinline__ void store_pass0(const Pair<T>* v, typename PairMem<T>::type* buf, int t) {
  using S = Shape<T, L>;
#pragma unroll
  for (int s = 0; s < S::R0; ++s) pstore(buf + pad_idx(t * S::R0 + s, S::PS) * STRIDE, v[s]);
  __syncthreads();
}

// ----------------------------------------------------- spindown phase
// e^{-i 2 pi phi(s)}, phi = ((p3 s + p2) s + p1) s + p0 cycles, s exact in FP32.
// FP32 path: Horner in double-float (error-free products and sums with
// explicitly rounded operations so the compiler cannot contract them).
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
  sincospif(2.0f * f, &sv, &cv);
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
template <typename T, int L>
__global__ void __launch_bounds__(Shape<T, L>::CA * Shape<T, L>::TPC)
k_pass_a(const typename PairMem<T>::type* __restrict__ G, int64_t lc, int n, int n1, int log2N,
         const TmplCoef* __restrict__ coefp, typename PairMem<T>::type* __restrict__ Z) {
  using S = Shape<T, L>;
  using PM = typename PairMem<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PM* smem = reinterpret_cast<PM*>(smem_raw);
  const int c = threadIdx.x / S::TPC;
  const int t = threadIdx.x % S::TPC;
  const int col = blockIdx.x * S::CA + c;
  PM* buf = smem + c * S::LP;
  const TmplCoef tc = *coefp;
  const PM* gcol = G + (int64_t)col * lc;

  Pair<T> v[S::R0];
#pragma unroll
  for (int s = 0; s < S::R0; ++s) {
    const int n2 = t + s * S::TPC;
    const int j = col + n1 * n2;
    if (j < n) {
      Pair<T> g = pload_g(gcol + n2);
      T cs, sn;
      spin_rot(tc, j - tc.J, &cs, &sn);
      v[s] = pmul(g, cs, sn);
    } else {
      v[s] = pzero<T>();
    }
  }
  dft<T, S::R0>(v);
  store_pass0<T, L, 1>(v, buf, t);
  passes<T, L, 1, 1>(v, buf, t);

  // four-step twiddle W_N^{col k2}, k2 = b + s * NSL, and store Z[col][k2]
  const T scale = (T)2 / (T)(1 << log2N);
  PM* zrow = Z + (int64_t)col * L;
  constexpr int NB = S::R0 / S::RL;
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int b = t + q * S::TPC;
    T s0, c0, s1, c1;
    sincospi_t(-(T)(col * b) * scale, &s0, &c0);
    sincospi_t(-(T)(col * S::NSL) * scale, &s1, &c1);
    Pair<T>* x = v + q * S::RL;
#pragma unroll
    for (int s = 0; s < S::RL; ++s) x[s] = pmul(x[s], c0, s0);
    twiddle<T, S::RL>(x, c1, s1);
#pragma unroll
    for (int s = 0; s < S::RL; ++s) pstore(zrow + b + s * S::NSL, x[s]);
  }
}

// ------------------------------------------------------------- pass B
template <typename T, int L>
__global__ void __launch_bounds__(Shape<T, L>::CB * Shape<T, L>::TPC)
k_pass_b(const typename PairMem<T>::type* __restrict__ Z, int n2, const SkyConst* __restrict__ sky,
         float* __restrict__ out) {
  using S = Shape<T, L>;
  using PM = typename PairMem<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PM* smem = reinterpret_cast<PM*>(smem_raw);
  const int c = threadIdx.x % S::CB;
  const int t = threadIdx.x / S::CB;
  const int k2 = blockIdx.x * S::CB + c;
  PM* buf = smem + c;

  Pair<T> v[S::R0];
#pragma unroll
  for (int s = 0; s < S::R0; ++s) v[s] = pload_g(Z + (int64_t)(t + s * S::TPC) * n2 + k2);
  dft<T, S::R0>(v);
  store_pass0<T, L, S::CB>(v, buf, t);
  passes<T, L, S::CB, 1>(v, buf, t);

  T kA, kB, kC;
  if constexpr (sizeof(T) == 4) { kA = sky->kAf; kB = sky->kBf; kC = sky->kCf; }
  else { kA = sky->kA; kB = sky->kB; kC = sky->kC; }
  constexpr int NB = S::R0 / S::RL;
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
      const int m = k2 + n2 * ((k1 + L / 2) & (L - 1));
      out[m] = (float)tf;
    }
  }
}

template <typename T, int L>
cudaError_t run_a(const void* G, int64_t lc, int64_t n, int n1, int log2N, const TmplCoef* coef,
                  void* Z, cudaStream_t st) {
  using S = Shape<T, L>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_pass_a<T, L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)S::SMEM_A);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_pass_a<T, L><<<n1 / S::CA, S::CA * S::TPC, S::SMEM_A, st>>>(
      (const typename S::PM*)G, lc, (int)n, n1, log2N, coef, (typename S::PM*)Z);
  return cudaGetLastError();
}

template <typename T, int L>
cudaError_t run_b(const void* Z, int n2, const SkyConst* sky, float* out, cudaStream_t st) {
  using S = Shape<T, L>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_pass_b<T, L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)S::SMEM_B);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_pass_b<T, L><<<n2 / S::CB, S::CB * S::TPC, S::SMEM_B, st>>>((const typename S::PM*)Z, n2, sky, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch_a(int log2_n2, const void* G, int64_t lc, int64_t n, int n1, int log2N,
                       const TmplCoef* coef, void* Z, cudaStream_t st) {
  switch (log2_n2) {
    case 5: return run_a<T, 32>(G, lc, n, n1, log2N, coef, Z, st);
    case 6: return run_a<T, 64>(G, lc, n, n1, log2N, coef, Z, st);
    case 7: return run_a<T, 128>(G, lc, n, n1, log2N, coef, Z, st);
    case 8: return run_a<T, 256>(G, lc, n, n1, log2N, coef, Z, st);
    case 9: return run_a<T, 512>(G, lc, n, n1, log2N, coef, Z, st);
    case 10: return run_a<T, 1024>(G, lc, n, n1, log2N, coef, Z, st);
    case 11: return run_a<T, 2048>(G, lc, n, n1, log2N, coef, Z, st);
    case 12: return run_a<T, 4096>(G, lc, n, n1, log2N, coef, Z, st);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t dispatch_b(int log2_n1, const void* Z, int n2, const SkyConst* sky, float* out, cudaStream_t st) {
  switch (log2_n1) {
    case 5: return run_b<T, 32>(Z, n2, sky, out, st);
    case 6: return run_b<T, 64>(Z, n2, sky, out, st);
    case 7: return run_b<T, 128>(Z, n2, sky, out, st);
    case 8: return run_b<T, 256>(Z, n2, sky, out, st);
    case 9: return run_b<T, 512>(Z, n2, sky, out, st);
    case 10: return run_b<T, 1024>(Z, n2, sky, out, st);
    case 11: return run_b<T, 2048>(Z, n2, sky, out, st);
    case 12: return run_b<T, 4096>(Z, n2, sky, out, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fft
}  // namespace fstat
