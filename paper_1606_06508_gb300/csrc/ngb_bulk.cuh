// ngb_bulk.cuh -- binary32 quaternions (Algorithm 7) staged through shared
// memory by bulk copies of the tensor-memory-accelerator engine
// (cp.async.bulk, completion counted on an mbarrier), an alternative to the
// register-staged k_small_vec16, taken only on request (NGB_QUAT_BULK=1).
//
// Measured on 2^26 quaternions (fraction of the measured HBM copy
// bandwidth; k_small_vec16 0.98 on the same boxes): tiles of 256 x U
// quaternions with S stages, (U, S) = (4, 4) 0.87, (1, 8) 0.85, (2, 6) 0.83,
// (4, 2) 0.82, (2, 4) 0.81, (2, 10) 0.70.  The kernel's work per byte (the
// branch order of Algorithm 7, the IEEE square root and reciprocal) keeps
// the ALU busy; a block that waits for its tile, computes, meets at a
// barrier and refills leaves more idle time than k_small_vec16's 32 warps
// per SM with six 16-byte loads in flight per lane, which already keep about
// 100 KB per SM on the way from HBM.
//
// Each block of BULK_THREADS threads keeps BULK_STAGES tiles of BULK_TILE
// quaternions (16 KiB) in flight: thread 0 arms the stage's mbarrier with
// the tile's byte count and issues one bulk copy global -> shared; every
// thread waits for the stage's phase, normalizes its BULK_U quaternions
// (thread t takes tile positions t, t + 256, ...: consecutive 16-byte shared
// reads and coalesced 16-byte evict-first global stores), and after a block
// barrier thread 0 refills the stage with the block's tile BULK_STAGES
// ahead.  Blocks stride over the tiles (grid: one wave).
//
// Waits are bounded: a wait that has not seen its phase after about 2^31
// clock cycles sets bit 1 of g_bulk_state, the block waits (bounded again) for the
// copies it issued and leaves.  Only device memory is read this way (the
// launcher checks the pointer); bulk copies need 16-byte aligned addresses
// and sizes, which 16-byte quaternions starting at a 16-byte aligned array
// give for every tile, the last one included.
#pragma once
#include <stdint.h>

#include "ngb_arith.cuh"

namespace ngb {

constexpr int BULK_THREADS = 256;
constexpr int BULK_U = 4;                          // quaternions per thread and tile
constexpr int BULK_STAGES = 4;                     // tiles in flight per block
constexpr int BULK_TILE = BULK_THREADS * BULK_U;   // quaternions per tile
constexpr size_t BULK_SMEM = (size_t)BULK_STAGES * BULK_TILE * 16 + BULK_STAGES * sizeof(uint64_t);
constexpr long long BULK_WAIT_CYCLES = 1ll << 31;

// State of this path in the process, read by ngb_quat_bulk_state(): bit 0
// once the kernel has run, bit 1 when a block's wait gave up (never
// expected; the tiles it did not reach keep whatever their outputs held).
__device__ unsigned g_bulk_state;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, unsigned parity) {
  uint32_t done;
  asm volatile(
      "{\n"
      "  .reg .pred p;\n"
      "  mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "  selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(done)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return done != 0;
}
// Wait for the phase of parity `parity` to complete, at most BULK_WAIT_CYCLES.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* b, unsigned parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(b, parity))
    if (clock64() - t0 > BULK_WAIT_CYCLES) return false;
  return true;
}
// One bulk copy of `bytes` (a multiple of 16, 16-byte aligned ends) from
// global to shared memory, completing on mbarrier b.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(b))
               : "memory");
}

__global__ void __launch_bounds__(BULK_THREADS) k_quat_bulk(const float* __restrict__ x, float* y, VecOut<float> out,
                                                            int64_t count, int quat_zero) {
  extern __shared__ __align__(128) unsigned char bulk_smem[];
  float4* buf = reinterpret_cast<float4*>(bulk_smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(bulk_smem + (size_t)BULK_STAGES * BULK_TILE * 16);
  const int t = threadIdx.x;
  const int64_t ntiles = (count + BULK_TILE - 1) / BULK_TILE;
  const float4* x4 = reinterpret_cast<const float4*>(x);
  auto issue = [&](int s, int64_t tile) {  // thread 0
    const int64_t q0 = tile * BULK_TILE;
    const int64_t nq = count - q0 < BULK_TILE ? count - q0 : BULK_TILE;
    const unsigned bytes = (unsigned)(nq * 16);
    mbar_arrive_expect_tx(&full[s], bytes);
    bulk_copy_g2s(buf + (size_t)s * BULK_TILE, x4 + q0, bytes, &full[s]);
  };
  if (t == 0) {
    for (int s = 0; s < BULK_STAGES; ++s) mbar_init(&full[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int s = 0; s < BULK_STAGES; ++s) {
      const int64_t tile = blockIdx.x + (int64_t)s * gridDim.x;
      if (tile < ntiles) issue(s, tile);
    }
  }
  if (blockIdx.x == 0 && t == 0) atomicOr(&g_bulk_state, 1u);
  __syncthreads();
  int64_t it = 0;
  bool alive = true;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int s = (int)(it % BULK_STAGES);
    const unsigned parity = (unsigned)((it / BULK_STAGES) & 1);
    const bool ok = mbar_wait_bounded(&full[s], parity);
    alive = __syncthreads_and(ok) != 0;
    if (!alive) break;
    const int64_t q0 = tile * BULK_TILE;
    const float4* b = buf + (size_t)s * BULK_TILE;
#pragma unroll
    for (int u = 0; u < BULK_U; ++u) {
      const int k = u * BULK_THREADS + t;
      const int64_t i = q0 + k;
      if (i < count) {
        const float4 v = b[k];
        float xv[4] = {v.x, v.y, v.z, v.w}, yv[4], r, h;
        const int code = normalize_small<float, 4>(xv, yv, r, h, quat_zero != 0);
        if (y) __stcs(reinterpret_cast<float4*>(y) + i, make_float4(yv[0], yv[1], yv[2], yv[3]));
        out.put(i, r, h, code);
      }
    }
    __syncthreads();  // every thread has read stage s
    if (t == 0) {
      const int64_t next = tile + (int64_t)BULK_STAGES * gridDim.x;
      if (next < ntiles) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(s, next);
      }
    }
  }
  if (!alive) {
    if (t == 0) {
      atomicOr(&g_bulk_state, 2u);
      // the copies this block issued and did not consume: tiles it .. it + STAGES - 1
      for (int64_t j = it; j < it + BULK_STAGES; ++j) {
        const int64_t tile = blockIdx.x + j * gridDim.x;
        if (tile < ntiles) mbar_wait_bounded(&full[j % BULK_STAGES], (unsigned)((j / BULK_STAGES) & 1));
      }
    }
    __syncthreads();
  }
}

}  // namespace ngb
