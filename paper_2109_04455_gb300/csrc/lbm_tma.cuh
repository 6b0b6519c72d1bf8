// TMA-staged bulk step of the ADR lattices.
//
// A persistent grid walks the row tiles (kBlockX nodes of one lattice row).
// For each tile one thread issues 1D bulk copies (cp.async.bulk, the TMA
// engine's linear mode) of every population plane's source row segment --
// row y - c_iy, columns [x0 - M, x0 + kBlockX + M) with a 16-byte margin M --
// plus the tile's velocity and link words into shared memory, completing on
// an mbarrier.  Two stages: while the block computes tile k from shared
// memory, the copies of tile k+1 are in flight.  The bytes in flight no
// longer depend on registers, which is what limits the 2-byte loads of the
// half-precision path in the register-staged kernel.
//
// Every copy starts on a 16-byte boundary (x0 is a multiple of kBlockX,
// nx_pad of 32 elements, M * sizeof(S) = 16) and has a length that is a
// multiple of 16 bytes; a copy that would leave the population buffer is
// not issued -- only boundary nodes (rows 0 and ny-1, columns 0 and nx-1)
// would read it, and those are updated by the boundary kernel instead.
// Waits are bounded: after kTmaWaitLimit polls a block records the failure
// in *status, waits (bounded) for its own copies still in flight, and
// returns.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

constexpr long long kTmaWaitLimit = 1ll << 24;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar,
                                                      uint32_t bytes) {
  asm volatile(
      "mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
          smem_u32(bar)),
      "r"(bytes)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src,
                                         uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// bounded wait on one phase of an mbarrier; false if the limit was reached
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar,
                                                  uint32_t parity) {
  for (long long it = 0; it < kTmaWaitLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

template <class P, int NS>
struct TmaLayout {
  using S = typename P::S;
  using T = typename P::T;
  static constexpr int kM = 16 / static_cast<int>(sizeof(S));  // margin
  static constexpr int kRow = kBlockX + 2 * kM;                 // elements
  static constexpr int kPlanes = NS * 9;
  static constexpr size_t kPop = sizeof(S) * kRow * kPlanes;     // bytes
  static constexpr size_t kU = sizeof(T) * kBlockX;              // one u row
  static constexpr size_t kLinks = sizeof(uint32_t) * kBlockX;
  // half storage: reference rows y-1, y, y+1 of every species (16-byte
  // margins)
  static constexpr int kMR = 16 / static_cast<int>(sizeof(RefT));
  static constexpr int kRefRow = kBlockX + 2 * kMR;
  static constexpr size_t kRef = P::kDev ? sizeof(RefT) * kRefRow * 3 * NS : 0;
  static constexpr size_t kStage = kPop + 2 * kU + kLinks + kRef;
  static constexpr size_t kBytes = 2 * kStage + 16;               // + 2 barriers
  static_assert(kPop % 16 == 0 && kU % 16 == 0, "16-byte aligned regions");
};

template <class P, int NS, int MODE>
__global__ void __launch_bounds__(kBlockX, 1)
    adr_tma_kernel(const AdrArgs a, int *status) {
  using S = typename P::S;
  using T = typename P::T;
  using L = TmaLayout<P, NS>;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + 2 * L::kStage);
  __shared__ int s_abort;

  const long long np = a.nx_pad, plane = a.plane;
  const int nxb = (a.nx_pad + kBlockX - 1) / kBlockX;
  const long long ntiles = static_cast<long long>(nxb) * a.ny;
  const S *src = static_cast<const S *>(a.src);
  const long long total = static_cast<long long>(L::kPlanes) * plane;
  const T *U = static_cast<const T *>(a.u);

  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_fence_init();
    s_abort = 0;
  }
  __syncthreads();

  // warp 0: copies of tile t into stage st, one copy per lane.  Copy q:
  // q < planes: population plane q; then u_x, u_y, the link words; then
  // (half storage) the 3 reference rows of every species.
  constexpr int kCopies = L::kPlanes + 3 + (P::kDev ? 3 * NS : 0);
  auto issue = [&](long long t, int st) {
    const int lane = threadIdx.x & 31;
    unsigned char *base = smem + st * L::kStage;
    const long long y = t / nxb;
    const long long x0 = (t % nxb) * kBlockX;
    const long long left = a.nx_pad - x0;              // multiple of 32
    const long long width = left < kBlockX ? left : kBlockX;
    const long long n0 = y * np + x0;
    // this lane's copies: destination, source, bytes (0 = not issued)
    unsigned char *dq[2] = {nullptr, nullptr};
    const void *sq[2] = {nullptr, nullptr};
    uint32_t bq[2] = {0u, 0u};
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int q = lane + 32 * r;
      if (q >= kCopies) continue;
      if (q < L::kPlanes) {
        const int i = q % 9;
        const long long plen = width + L::kM + (left > kBlockX ? L::kM : 0);
        const long long start = q * plane + (y - cy(i)) * np + x0 - L::kM;
        if (start >= 0 && start + plen <= total) {
          dq[r] = base + static_cast<size_t>(q) * L::kRow * sizeof(S);
          sq[r] = src + start;
          bq[r] = static_cast<uint32_t>(plen * sizeof(S));
        }
      } else if (q < L::kPlanes + 3) {
        const int j = q - L::kPlanes;   // 0: u_x, 1: u_y, 2: links
        dq[r] = base + L::kPop + j * L::kU;
        sq[r] = j < 2 ? static_cast<const void *>(U + j * plane + n0)
                      : static_cast<const void *>(a.links + n0);
        bq[r] = static_cast<uint32_t>(width * (j < 2 ? sizeof(T) : sizeof(uint32_t)));
      } else {
        const int qq = q - L::kPlanes - 3;   // species qq / 3, row y - 1 + qq % 3
        long long rlen = width + L::kMR + (left > kBlockX ? L::kMR : 0);
        long long start = (qq / 3) * plane + (y - 1 + qq % 3) * np + x0 - L::kMR;
        long long skip = 0;
        if (start < 0 && start + L::kMR >= 0) {
          // first row of species 0: drop the left margin (only column 0, a
          // boundary node, would read it)
          skip = L::kMR;
          start += skip;
          rlen -= skip;
        }
        if (start >= 0 && start + rlen <= static_cast<long long>(NS) * plane) {
          dq[r] = base + L::kPop + 2 * L::kU + L::kLinks +
                  (static_cast<size_t>(qq) * L::kRefRow + skip) * sizeof(RefT);
          sq[r] = a.rsrc + start;
          bq[r] = static_cast<uint32_t>(rlen * sizeof(RefT));
        }
      }
    }
    const uint32_t bytes = __reduce_add_sync(0xffffffffu, bq[0] + bq[1]);
    if (lane == 0) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&bars[st], bytes);
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 2; ++r)
      if (bq[r]) bulk_g2s(dq[r], sq[r], bq[r], &bars[st]);
  };

  uint32_t phase[2] = {0u, 0u};
  long long t = blockIdx.x;
  if (t < ntiles && threadIdx.x < 32) issue(t, 0);
  int k = 0;
  for (; t < ntiles; t += gridDim.x, ++k) {
    const int st = k & 1;
    const long long tn = t + gridDim.x;
    if (tn < ntiles && threadIdx.x < 32) issue(tn, st ^ 1);
    if (!mbar_wait_bounded(&bars[st], phase[st])) s_abort = 1;
    __syncthreads();
    if (s_abort) {
      if (threadIdx.x == 0) {
        atomicExch(status, 1);
        // the other stage may still be filling: let it land before exit
        if (tn < ntiles) mbar_wait_bounded(&bars[st ^ 1], phase[st ^ 1]);
      }
      return;
    }
    phase[st] ^= 1u;

    const unsigned char *base = smem + st * L::kStage;
    const S *rows = reinterpret_cast<const S *>(base);
    const T *su = reinterpret_cast<const T *>(base + L::kPop);
    const uint32_t *sl = reinterpret_cast<const uint32_t *>(base + L::kPop + 2 * L::kU);
    const RefT *sr = reinterpret_cast<const RefT *>(base + L::kPop + 2 * L::kU + L::kLinks);
    const long long y = t / nxb;
    const int x = static_cast<int>((t % nxb) * kBlockX) + threadIdx.x;
    const long long n = y * np + x;
    T acc[2 * NS];
#pragma unroll
    for (int q = 0; q < 2 * NS; ++q) acc[q] = T(0);
    if (x < a.nx_pad && sl[threadIdx.x] == 0u) {
      S *__restrict__ dst = static_cast<S *>(a.dst);
      T *__restrict__ cp = static_cast<T *>(a.cprev);
      T prev[NS];
      if (MODE == kAdrCheck) {
#pragma unroll
        for (int s = 0; s < NS; ++s) prev[s] = cp[s * plane + n];
      }
      T E[9];
      eq_factors<T>(su[threadIdx.x], su[kBlockX + threadIdx.x], E);
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        T g[9];
        T c = T(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          g[i] = P::load(rows[(s * 9 + i) * L::kRow + L::kM + threadIdx.x - cx(i)]);
          if constexpr (P::kDev)   // reference of the source node x - c_i
            g[i] += Lattice<T>::w(i) *
                    __half2float(sr[(s * 3 + 1 - cy(i)) * L::kRefRow + L::kMR + threadIdx.x - cx(i)]);
          c += g[i];
        }
        const T om = pick<T>(a.omega[s], a.fomega[s]);
        T cq = c;
        if constexpr (P::kDev) {
          cq = ref_round(c);
          a.rdst[s * plane + n] = __float2half_rn(c);
        }
#pragma unroll
        for (int i = 0; i < 9; ++i)
          dst[(long long)(s * 9 + i) * plane + n] =
              P::store(g[i] + om * (c * E[i] - g[i]) - adr_unref<P>(i, cq));
        if (MODE == kAdrCheck) {
          acc[2 * s] += absT(c - prev[s]);
          acc[2 * s + 1] += absT(c);
          cp[s * plane + n] = c;
        }
      }
    }
    if (MODE == kAdrCheck) block_sum_store<2 * NS, T>(acc, a.partials + t * (2 * NS));
    __syncthreads();  // stage st is free for the copies of tile k + 2
  }
}

// Whether a precision's bulk step uses the TMA-staged kernel (see the
// measurements in the design notes; the register-staged kernel is the
// default).
#ifndef LBM_ADR_TMA_F32
#define LBM_ADR_TMA_F32 0
#endif
#ifndef LBM_ADR_TMA_F16
#define LBM_ADR_TMA_F16 0
#endif
template <class P>
constexpr bool adr_uses_tma() {
  return sizeof(typename P::S) == 2 ? LBM_ADR_TMA_F16 != 0
                                    : (sizeof(typename P::S) == 4 ? LBM_ADR_TMA_F32 != 0
                                                                  : false);
}

}  // namespace lbm
