// Pass A with its input tiles staged by the Tensor Memory Accelerator.
//
// The direct pass A (update_x_body) runs one CTA per tile: each thread loads
// its column of W, psi and the update input, transforms, updates and stores.
// At 512^3 complex64 one 512-thread CTA fills an SM, so the loads, the two
// transforms and the stores of a tile do not overlap.  Here a persistent CTA
// per SM walks the tiles k = blockIdx.x, blockIdx.x + gridDim.x, ... with a
// two-stage pipeline: while it transforms tile k, the TMA unit copies the
// W, psi and update-input tiles of the next tile into the other stage of
// shared memory (cp.async.bulk.tensor.2d, completion counted in bytes on an
// mbarrier).  Threads read their column from the staged tile, and the
// arithmetic is the same core as the direct kernel's (update_x_core).
//
// Tensor maps (built on the host per plan, kept in device memory): every
// lattice viewed as a 2D tensor of N rows (x, stride N^2 sites) by N^2 sites
// (y, z), in elements of one site (8 bytes for complex64, 4 for FP32 V); a
// box is XT sites by min(N, 256) rows, so a tile takes
// N / 256 boxes per array.  Every box starts at a column k * XT, a multiple
// of 16 bytes, as the copies require.
//
// Waits are bounded: a thread that finds its stage's barrier incomplete after
// TMA_WAIT_LIMIT tries (each try suspends the thread for at most about
// TMA_TRY_NS nanoseconds, so about a second in all) gives up; the CTA then sets the plan's error flag,
// waits (bounded again) for the copies it has issued, and returns.  The host
// reports the flag as QFD_ERR_TIMEOUT.  test_skip = 1 arms the barriers
// without issuing any copy, so that every wait runs out: the test of that
// path (no copy is in flight when the CTA returns).
#pragma once

#include <cuda.h>  // CUtensorMap

#include "qfd_kernels.cuh"

namespace qfd {

constexpr uint32_t TMA_WAIT_LIMIT = 1u << 19;
constexpr uint32_t TMA_TRY_NS = 2000;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make the initialised barriers visible to the asynchronous (TMA) proxy
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// the tensor maps were written by a host copy before the launch
__device__ __forceinline__ void fence_tensormap(const void* map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}
// arrive on the barrier and add `bytes` to the transaction count of its phase
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(TMA_TRY_NS)
      : "memory");
  return ok != 0;
}
// bounded wait for the phase of parity `parity` of the barrier
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// 2D tiled copy of the box at element coordinates (x0, x1) into shared memory
__device__ __forceinline__ void tma_load_2d(void* dst, const void* map, int x0, int x1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x0), "r"(x1), "r"(smem_u32(bar))
      : "memory");
}

// Launch shape of the TMA-staged pass A: XT sites a tile (so that two stages
// of W, psi and the update input and the exchange tile fit in shared memory),
// T = N / 8 threads a column, one CTA per SM.  Complex64 at N = 256, 512, 1024.
template <class A, int N> struct TmaShape {
  static constexpr bool OK = A::id == 1 && (N == 256 || N == 512 || N == 1024);
  static constexpr int XT = N == 256 ? 16 : N == 512 ? 8 : 4;
  static constexpr int T = N / FftPlan<N>::E;
  static constexpr int THREADS = T * XT;
  static constexpr int BOXR = N < 256 ? N : 256;  // rows of a box
  static constexpr int NBOX = N / BOXR;
  static constexpr size_t WB = (size_t)N * XT * sizeof(typename A::C);  // one W or psi tile
  static constexpr size_t UB = (size_t)N * XT * sizeof(typename A::U);  // one update-input tile
  static constexpr size_t STAGE = 2 * WB + UB;
  // two stages, the exchange tile, the barriers, and room to align the base
  // to 128 bytes (the dynamic region follows the kernel's static buffers)
  static constexpr size_t SMEM = 2 * STAGE + WB + 2 * sizeof(uint64_t) + 128;
  static_assert(!OK || SMEM <= 227 * 1024, "shared memory of one CTA");
};

template <class A, int N, int STATS>
__global__ void __launch_bounds__(TmaShape<A, N>::THREADS, 1)
k_update_x_tma(const __grid_constant__ BatchU b, uint32_t scaled, int test_skip) {
  using C = typename A::C;
  using U = typename A::U;
  using TS = TmaShape<A, N>;
  constexpr int XT = TS::XT, T = TS::T, E = FftPlan<N>::E;
  constexpr int NT = N * N / XT;  // tiles of a lattice
  extern __shared__ __align__(128) unsigned char smraw[];
  unsigned char* sbase = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 127) & ~(uintptr_t)127);
  unsigned char* stage[2] = {sbase, sbase + TS::STAGE};
  C* exch = reinterpret_cast<C*>(sbase + 2 * TS::STAGE);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sbase + 2 * TS::STAGE + TS::WB);
  const int lat = blockIdx.y;
  const void* mapW = b.tmap[lat][0];
  const void* mapP = b.tmap[lat][1];
  const void* mapU = b.tmap[lat][2];
  C* W = static_cast<C*>(b.W[lat]);
  C* psi = static_cast<C*>(b.psi[lat]);
  const double* scale = (scaled >> lat) & 1u ? b.scale[lat] : nullptr;
  const int tid = threadIdx.x;
  const int col = tid % XT, t = tid / XT;
  const int k0 = blockIdx.x, g = gridDim.x;

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_tensormap(mapW);
    fence_tensormap(mapP);
    fence_tensormap(mapU);
    fence_async_shared();
  }
  __syncthreads();
  // thread 0: copy the W, psi and update-input tiles of tile k into stage s
  auto issue = [&](int k, int s) {
    mbar_arrive_expect_tx(&bars[s], (uint32_t)TS::STAGE);
    if (test_skip) return;
    unsigned char* d = stage[s];
    for (int r = 0; r < TS::NBOX; ++r) {
      const int x1 = r * TS::BOXR;
      tma_load_2d(d + (size_t)x1 * XT * sizeof(C), mapW, k * XT, x1, &bars[s]);
      tma_load_2d(d + TS::WB + (size_t)x1 * XT * sizeof(C), mapP, k * XT, x1, &bars[s]);
      tma_load_2d(d + 2 * TS::WB + (size_t)x1 * XT * sizeof(U), mapU, k * XT, x1, &bars[s]);
    }
  };
  if (tid == 0) {
    if (k0 < NT) issue(k0, 0);
    if (k0 + g < NT) issue(k0 + g, 1);
  }
  typename A::Acc nacc;
  typename A::Full facc;
  bool failed = false;
  int it = 0;
  for (int k = k0; k < NT; k += g, ++it) {
    const int s = it & 1;
    const bool ok = mbar_wait_bounded(&bars[s], (uint32_t)(it >> 1) & 1u, TMA_WAIT_LIMIT);
    if (!__syncthreads_and(ok)) {
      failed = true;
      break;
    }
    const C* Ws = reinterpret_cast<const C*>(stage[s]);
    const C* Ps = reinterpret_cast<const C*>(stage[s] + TS::WB);
    const U* Us = reinterpret_cast<const U*>(stage[s] + 2 * TS::WB);
    C v[E], ps[E];
    U cf[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int j = (t + m * T) * XT + col;
      v[m] = Ws[j];
      ps[m] = Ps[j];
      cf[m] = Us[j];
    }
    __syncthreads();  // stage s is read: refill it with the tile after next
    if (tid == 0 && k + 2 * g < NT) issue(k + 2 * g, s);
    update_x_core<A, N, STATS, XT>(v, ps, cf, t, col, (int64_t)k * XT + col, W, psi, b.up[lat],
                                   static_cast<const typename A::VT*>(b.V[lat]), scale, b.scale_f[lat],
                                   static_cast<const C*>(b.tw[lat]), exch, nacc, facc);
  }
  if (failed) {
    // the copies issued for iterations it and it + 1 may still be in flight:
    // wait for them (bounded) before the CTA's shared memory is released
    if (tid == 0) {
      atomicExch(b.err[lat], 1);
      if (!test_skip) {
        for (int j = it; j < it + 2; ++j)
          if (k0 + j * g < NT) mbar_wait_bounded(&bars[j & 1], (uint32_t)(j >> 1) & 1u, 4u * TMA_WAIT_LIMIT);
      }
    }
    __syncthreads();
    return;
  }
  if constexpr (STATS == STATS_NORM) norm_reduce_store<A>(nacc, b.part[lat]);
  if constexpr (STATS == STATS_FULL) full_store<A>(facc, b.part[lat]);
}

}  // namespace qfd
