// One persistent launch over many templates: both FFT passes of Sec. 3
// steps (vi)-(vii) for every template of a sky group, pulled as work items
// from a queue by CTAs that stay resident for the whole launch.
//
// Items.  Template k has NA = n1 / CA pass-A tiles (CA columns each) and
// NB = n2 / CB pass-B tiles (CB rows each).  The queue order is
//   A(0) | A(1) + B(0) | A(2) + B(1) | ... | A(T-1) + B(T-2) | B(T-1)
// where each middle group interleaves the tiles of A(g) and B(g - 1), with
// every A(g) tile within the first NA + NB/2 positions, so that A(g) is
// complete before the B(g) tiles of the next group are taken.  The
// intermediate of template k lives in ring slot k mod kRing.
//
// Dependencies.  A B(k) tile reads every column of template k's
// intermediate: it waits until all NA tiles of A(k) are done.  An A(k) tile
// overwrites ring slot k mod kRing: it waits until all NB tiles of
// B(k - kRing) are done.  Items are taken in queue order (one atomic
// counter) and every item depends only on items earlier in that order, so
// the earliest unfinished item can always run: the launch cannot deadlock,
// whether or not all of its CTAs are resident at once.  Every wait is
// bounded: a wait that runs out records FSTAT_ERR_TIMEOUT, raises the
// launch's abort flag (which the other CTAs' waits watch), lets this CTA's
// bulk copies in flight land, and returns.
//
// Loads.  Both kinds of tile are loaded into the CTA's one shared buffer by
// bulk copies that thread 0 issues, counted in bytes on one mbarrier: a
// pass-A tile as CA contiguous column copies of G (dense staging), a pass-B
// tile as 2D tensor boxes of the ring slot's intermediate.  The next item's
// copies are issued as soon as the current item's last Stockham pass has
// read the buffer, when its dependency is already met (else at its start).
// Completion: every thread's stores, a CTA barrier, then thread 0 releases
// the item (fence + atomic add on the template's counter); a consumer's
// thread 0 acquires the counter and fences the async proxy before its
// bulk copies read the data.
#pragma once

#include "fft_impl.cuh"

namespace fstat {
namespace fft {

using fstat::FusedArgs;
using fstat::kRing;
using fstat::kQueueHead;

struct ZMaps {
  CUtensorMap m[kRing];
};

struct Item {
  int kind;  // 0 = pass-A tile, 1 = pass-B tile
  int k;     // template (within the launch)
  int tile;
};

__device__ __forceinline__ Item decode_item(int i, int NA, int NB, int T) {
  if (i < NA) return Item{0, 0, i};
  const int j = i - NA;
  const int GRP = NA + NB;
  const int g = 1 + j / GRP;
  const int p = j - (g - 1) * GRP;
  if (g >= T) return Item{1, T - 1, p};  // last group: B(T - 1) only
  const int W = NA + NB / 2;             // A(g) tiles lie within [0, W)
  if (p < W) {
    const int cnt = (int)((int64_t)(p + 1) * NA / W);  // A tiles among positions 0..p
    const int cntp = (int)((int64_t)p * NA / W);
    if (cnt > cntp) return Item{0, g, cnt - 1};
    return Item{1, g - 1, p - cnt};
  }
  return Item{1, g - 1, p - NA};
}

constexpr int kDepPolls = 1 << 22;  // dependency polls (each after a ~0.1-0.3 us sleep)

// 2F rows are written with streaming stores as in the two-launch path

template <int LA, int CA, int VA, int LB, int CB, int VB>
struct FusedShape {
  using SA = Shape<float, LA, VA>;
  using SB = Shape<float, LB, VB>;
  static constexpr int NT = CA * SA::TPC;
  static_assert(NT == CB * SB::TPC, "both passes run with the CTA's thread count");
  static_assert((VA & 6) == 6 && (VB & 6) == 6, "one buffer, dense staging by bulk copies");
  static constexpr size_t ONE_A = (size_t)CA * SA::LP * sizeof(float4);
  static constexpr size_t ONE_B = (size_t)CB * SB::LP * sizeof(float4);
  static constexpr size_t SMEM = ONE_A > ONE_B ? ONE_A : ONE_B;
  static constexpr int MINB = NT <= 256 ? 2 : 1;
  static_assert(LB * CB * sizeof(float4) < (1u << 20), "mbarrier transaction count");
};

// Thread 0's side of the queue: is the item's dependency met (acquire)?
__device__ __forceinline__ bool item_ready(const FusedArgs& a, const Item& it) {
  const int* done = a.q + kQueueHead;
  if (it.kind == 0) return it.k < kRing || ld_acquire(done + a.T + it.k - kRing) >= a.nb;
  return ld_acquire(done + it.k) >= a.na;
}

// Bounded wait for the item's dependency; false (abort flag raised, a
// timeout recorded if this wait ran out) when the launch gives up.
__device__ __noinline__ bool item_wait(const FusedArgs& a, const Item& it, int limit) {
  volatile int* abort_flag = a.q + 1;
  for (int i = 0; i < limit; ++i) {
    if (item_ready(a, it)) return true;
    if (*abort_flag) return false;
    __nanosleep(128);
  }
  if (a.err) atomicCAS(a.err, 0, FSTAT_ERR_TIMEOUT);
  atomicExch(a.q + 1, 1);
  return false;
}

// Thread 0: the item's bulk copies into the CTA's buffer, counted on bar.
template <int LA, int CA, int LB, int CB>
__device__ __noinline__ void item_issue(const FusedArgs& a, const ZMaps& zm, const Item& it, float4* smem,
                                        unsigned long long* bar) {
  constexpr int LPA = LA + (LA >> log2c(r_of(LA, 0, 6)));
  fence_proxy_async_global();  // what item_ready acquired precedes the copies
  fence_proxy_async();         // this CTA's earlier use of the buffer precedes them
  if (it.kind == 0) {
    const unsigned bytes = (unsigned)(a.lc * sizeof(float4));
    mbar_expect_tx(bar, bytes * CA);
#pragma unroll 1
    for (int c = 0; c < CA; ++c) bulk_load(smem + c * LPA, a.G + (int64_t)(it.tile * CA + c) * a.lc, bytes, bar);
  } else {
    mbar_expect_tx(bar, (unsigned)(LB * CB * sizeof(float4)));
    const CUtensorMap* map = &zm.m[it.k % kRing];
#pragma unroll 1
    for (int r = 0; r < LB; r += kTmaRows) tma_load_2d(smem + r * CB, map, it.tile * CB * 4, r, bar);
  }
}

template <int LA, int CA, int VA, int LB, int CB, int VB>
__global__ void __launch_bounds__(FusedShape<LA, CA, VA, LB, CB, VB>::NT, FusedShape<LA, CA, VA, LB, CB, VB>::MINB)
k_fused(const __grid_constant__ FusedArgs a, const __grid_constant__ ZMaps zm) {
  using FS = FusedShape<LA, CA, VA, LB, CB, VB>;
  using SA = typename FS::SA;
  static_assert(SA::LP == LA + (LA >> log2c(r_of(LA, 0, 6))), "staging layout of item_issue");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float4* smem = reinterpret_cast<float4*>(smem_raw);
  // queue state shared by the CTA (kept out of registers, which the FFT
  // passes need): current and next item, stop flag, whether the next
  // item's copies are in flight, and the mbarrier uses issued / waited
  __shared__ unsigned long long bar;
  __shared__ int s_cur, s_next, s_stop, s_loaded;
  __shared__ unsigned s_issued, s_waited;

  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
    s_cur = atomicAdd(a.q, 1);
    s_loaded = 0;
    s_issued = 0;
    s_waited = 0;
  }
  __syncthreads();
  bool failed = false;
  for (;;) {
    if (s_cur >= a.total) break;
    if (threadIdx.x == 0) {
      // the current item's copies (unless issued early), then the next item
      const Item it = decode_item(s_cur, a.na, a.nb, a.T);
      bool ok = true;
      if (!s_loaded) {
        ok = item_wait(a, it, a.wait_set ? a.wait_limit : kDepPolls);
        if (ok) {
          item_issue<LA, CA, LB, CB>(a, zm, it, smem, &bar);
          ++s_issued;
        }
      }
      const bool stop = !ok || *((volatile int*)(a.q + 1));
      s_next = stop ? a.total : atomicAdd(a.q, 1);
      s_stop = stop;
      s_loaded = 0;
    }
    __syncthreads();
    if (s_stop) { failed = true; break; }
    const bool got = mbar_wait(&bar, s_waited & 1u, a.wait_set ? a.wait_limit : kWaitLimit);
    if (__syncthreads_and(got) == 0) {
      if (threadIdx.x == 0) {
        if (a.err) atomicCAS(a.err, 0, FSTAT_ERR_TIMEOUT);
        atomicExch(a.q + 1, 1);
      }
      failed = true;
      break;
    }
    // the next item's copies, as soon as this item has read the buffer
    auto at_free = [&] {
      if (threadIdx.x == 0 && s_next < a.total) {
        const Item ni = decode_item(s_next, a.na, a.nb, a.T);
        if (item_ready(a, ni)) {
          item_issue<LA, CA, LB, CB>(a, zm, ni, smem, &bar);
          ++s_issued;
          s_loaded = 1;
        }
      }
    };
    {
      const Item it = decode_item(s_cur, a.na, a.nb, a.T);
      if (it.kind == 0) {
        const int cA = threadIdx.x / SA::TPC, tA = threadIdx.x % SA::TPC;
        const float inv_n = 1.f / (float)((int64_t)a.n1 * a.n2);
        pass_a_tile<float, LA, CA, VA, true>(it.tile, smem + cA * SA::LP, cA, tA, a.G, a.lc, a.n, a.n1,
                                             (const float2*)nullptr, a.coef[it.k], inv_n, a.Z[it.k % kRing],
                                             at_free);
      } else {
        const int cB = threadIdx.x % CB, tB = threadIdx.x / CB;
        const SkyConst& sk = *a.sky;
        float* row = a.out + (int64_t)(a.ord[it.k] % a.out_rows) * ((int64_t)a.n1 * a.n2);
        const PeakArgs pk{};
        pass_b_tile<float, LB, CB, VB, true, kStore>(it.tile, smem + cB, cB, tB, a.Z[it.k % kRing], a.n2,
                                                     (const float2*)nullptr, sk.kAf, sk.kBf, sk.kCf, row, pk,
                                                     nullptr, nullptr, at_free);
      }
    }
    __syncthreads();  // every thread's stores of this item are issued
    if (threadIdx.x == 0) {
      const Item it = decode_item(s_cur, a.na, a.nb, a.T);
      __threadfence();
      atomicAdd(a.q + kQueueHead + (it.kind == 0 ? 0 : a.T) + it.k, 1);
      s_cur = s_next;
      ++s_waited;
    }
    __syncthreads();
  }
  if (failed && threadIdx.x == 0) {
    // let the copies this CTA issued land before its shared memory goes away
    for (unsigned u = s_waited; u < s_issued; ++u) mbar_wait(&bar, u & 1u);
  }
}

template <int LA, int CA, int VA, int LB, int CB, int VB>
cudaError_t run_fused(const FusedArgs& in, cudaStream_t st) {
  using FS = FusedShape<LA, CA, VA, LB, CB, VB>;
  static int ctas = 0, per_sm = 0;
  if (!ctas) {
    cudaError_t e = resident_ctas(k_fused<LA, CA, VA, LB, CB, VB>, FS::NT, FS::SMEM, &ctas, &per_sm);
    if (e != cudaSuccess) return e;
  }
  if (in.n1 != LB || in.n2 != LA || in.n1 % CA || in.n2 % CB || in.T < 1 || in.lc < 1 || in.lc > LA)
    return cudaErrorInvalidConfiguration;
  if ((uintptr_t)in.G & 15) return cudaErrorInvalidValue;
  FusedArgs a = in;
  a.na = in.n1 / CA;
  a.nb = in.n2 / CB;
  const int64_t total = (int64_t)a.T * (a.na + a.nb);
  if (total >= INT32_MAX) return cudaErrorInvalidValue;
  a.total = (int)total;
  ZMaps zm;
  memset(&zm, 0, sizeof(zm));
  for (int r = 0; r < kRing; ++r) {
    const cudaError_t e = z_tensor_map(&zm.m[r], a.Z[r], LB, a.n2, CB);
    if (e != cudaSuccess) return e;
  }
  const int grid = a.total < ctas ? a.total : ctas;
  k_fused<LA, CA, VA, LB, CB, VB><<<grid, FS::NT, FS::SMEM, st>>>(a, zm);
  return cudaGetLastError();
}

}  // namespace fft
}  // namespace fstat
