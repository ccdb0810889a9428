// kernels_ragged.cuh -- ragged batches (vector i = x[offsets[i] .. offsets[i+1]))
// forward and backward; instantiated per precision by ragged_f32.cu and
// ragged_f64.cu.
//
// 1. k_classify reads the int64 offsets once, skips (and flags) vectors with
//    bad offsets, finishes zero-length vectors (norm +0), and appends every
//    other vector index to one of the lists by length: the block list
//    (n > warp_max), the warp list (thread_max < n <= warp_max), in binary64
//    two group lists for the shorter warp-sized vectors (n <= 64: groups of
//    8 lanes; n <= 128: groups of 16 lanes; csrc/ngb_grouppath.cuh), and the
//    thread list (n <= thread_max; n <= 4 always).  Appends are aggregated
//    per block: one atomic per block and list.
// 2. Forward: k_ragged runs one wave of persistent blocks that take work from
//    the lists, longest vectors first, through atomic tickets: whole blocks
//    on block items, warps on batches of warp items, groups of lanes on group
//    items, lanes on thread items.  Warps and blocks stream their vector
//    (three passes, a few partial sums per lane) instead of holding it, so
//    the kernel keeps few registers and many loads in flight; in binary32 a
//    warp prefetches its next item into L2 once pass 1 has read the current
//    one.
//    Groups hold their (short) vector in registers.  No block ever waits for
//    another.
// 3. Backward: one plain grid-stride kernel per list (k_ragged_bwd_blocks,
//    k_ragged_bwd_warps, k_ragged_bwd_groups, k_ragged_bwd_threads).
// Every mapping evaluates the same operations in the same order (the paper's
// Algorithms 3-7 for n <= 4, the order CR(n) for n >= 5), so the results do
// not depend on the mapping, the grid or the order in which items are taken.
#pragma once
#include "ngb_internal.h"
#include "ngb_grouppath.cuh"
#include "ngb_threadpath.cuh"

namespace ngb {

constexpr int CLASSIFY_THREADS = 1024;
constexpr int WARP_BATCH = 8;     // warp items per ticket (binary32 ragged, prefetch after pass 1: 4 1.941 ms, 8 1.933 ms;
                                  // binary64 ragged: 4 7.293 ms, 8 7.288 ms)
constexpr int THREAD_BATCH = 4;   // 32-item groups per ticket
constexpr int GROUP_BATCH = 4;    // rounds of 32 / W group items per ticket

// The longest vectors of the group lists (0: no group list).  binary64
// only: there the per-vector steps run on the scarce FP64 pipe, and a group
// of W lanes shares each of their instructions among 32 / W vectors.
template <typename T> __host__ __device__ constexpr int group8_max() { return sizeof(T) == 8 ? 64 : 0; }
template <typename T> __host__ __device__ constexpr int group16_max() { return sizeof(T) == 8 ? 128 : 0; }
static_assert(ragged_lists(4) == 3 && group8_max<float>() == 0 && group16_max<float>() == 0,
              "binary32 scratch holds three lists");
static_assert(ragged_lists(8) == NLISTS, "binary64 scratch holds every list");

template <typename T>
__global__ void __launch_bounds__(CLASSIFY_THREADS)
    k_classify(const int64_t* __restrict__ off, int64_t count, int64_t capacity, int thread_max, int warp_max,
               int validate, RaggedScratch sc, VecOut<T> zero_out) {
  __shared__ int wcount[CLASSIFY_THREADS / 32][NLISTS];
  __shared__ int wbase[CLASSIFY_THREADS / 32][NLISTS];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  for (int64_t base = (int64_t)blockIdx.x * CLASSIFY_THREADS; base < count;
       base += (int64_t)gridDim.x * CLASSIFY_THREADS) {
    const int64_t i = base + t;
    int b = -1;
    if (i < count) {
      const int64_t s = off[i], e = off[i + 1];
      const int64_t n = e - s;
      // capacity > 0: ends past the caller's buffer are bad; capacity < 0: the
      // batch has no element array, so every vector of positive length is bad
      const bool bad = n < 0 || n > MAX_LEN || s < 0 || (capacity > 0 && e > capacity) ||
                       (capacity < 0 && n > 0) || (validate && i == 0 && s != 0);
      if (bad) {
        atomicOr(sc.status, 1);
      } else if (n == 0) {
        zero_out.put(i, T(0), T(0), CODE_ZERO);
      } else {
        // n <= 4 always runs Algorithms 5-7 in one thread
        if (n <= thread_max || n <= 4) b = LIST_THREAD;
        else if (n > warp_max) b = LIST_BLOCK;
        else if (n <= group8_max<T>()) b = LIST_GROUP8;
        else if (n <= group16_max<T>()) b = LIST_GROUP16;
        else b = LIST_WARP;
      }
    }
    unsigned ball[NLISTS];
#pragma unroll
    for (int k = 0; k < NLISTS; ++k) {
      ball[k] = __ballot_sync(FULL, b == k);
      if (lane == 0) wcount[w][k] = __popc(ball[k]);
    }
    __syncthreads();
    if (w == 0) {  // per bucket: exclusive scan of the 32 warp counts by shuffles, one atomic per block
      static_assert(CLASSIFY_THREADS == 1024, "one warp count per lane");
#pragma unroll
      for (int k = 0; k < NLISTS; ++k) {
        const int c = wcount[lane][k];
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(FULL, incl, o);
          if (lane >= o) incl += v;
        }
        int g = 0;
        if (lane == 31 && incl) g = atomicAdd(&sc.counts[k], incl);
        g = __shfl_sync(FULL, g, 31);
        wbase[lane][k] = g + incl - c;
      }
    }
    __syncthreads();
    if (b >= 0) {
      unsigned mine = 0;
#pragma unroll
      for (int k = 0; k < NLISTS; ++k)
        if (b == k) mine = ball[k];
      sc.items[(int64_t)b * count + wbase[w][b] + __popc(mine & lt_mask)] = (int32_t)i;
    }
    __syncthreads();
  }
}

template <typename T>
struct RaggedArgs {
  const T* x;          // forward input, or y for the backward pass
  T* y;                // forward output (nullable: norm only), or grad
  const T* g;          // backward: upstream gradient
  const T* h_in;       // backward: saved h
  const int8_t* c_in;  // backward: saved code
  VecOut<T> out;       // forward per-vector outputs
  const int64_t* off;
  RaggedScratch sc;
  int64_t count;
};

// Forward persistent kernel, B threads per block (128 or 256), resident
// threads per SM as ragged_min_blocks asks.
// L2 prefetch of the next warp item's vector (within the ticket), issued
// once pass 1 has read the current item, so that the prefetched lines wait in
// L2 for passes 2 and 3 of the current item only.  Measured on the ragged
// binary32 workload (time per step; DRAM reads of the 10^6-vector case):
// no prefetch 2.125 ms (1575 MB); the whole next item before the current
// item 1.99 ms (1719 MB: prefetched lines evicted before use), its first
// 2, 4 or 8 KiB 2.08, 2.05, 2.02 ms; the whole next item after pass 1
// 1.93 ms (1592 MB).  Earlier tests with the prefetch before the item: a
// whole ticket at once or the next ticket taken one ahead were slower.
// binary64, bound by the FP64 pipe: 0.401 -> 0.388 of the copy bandwidth
// with the prefetch before the item: off.
constexpr bool WARP_PREFETCH_F32 = true, WARP_PREFETCH_F64 = false;
template <typename T>
__host__ __device__ constexpr bool warp_prefetch() { return sizeof(T) == 4 ? WARP_PREFETCH_F32 : WARP_PREFETCH_F64; }

// Prefetch n values from p into L2, one 128-byte line per lane and step
// (every address lies inside the range).
template <typename T>
__device__ __forceinline__ void prefetch_range_l2(const T* p, int64_t n, int lane) {
  const char* c = reinterpret_cast<const char*>(p);
  const int64_t bytes = n * (int64_t)sizeof(T);
  for (int64_t b = (int64_t)lane * 128; b < bytes; b += 32 * 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(c + b));
}


// Group items of list `list`: each warp takes GROUP_BATCH rounds of 32 / W
// items per ticket, one item per group of W lanes.
template <typename T, int W>
__device__ __forceinline__ void ragged_group_items(const RaggedArgs<T>& a, int list, int lane) {
  constexpr int PER = 32 / W;
  const int cnt = a.sc.counts[list];
  const int32_t* L = a.sc.items + (int64_t)list * a.count;
  for (;;) {
    int base = 0;
    if (lane == 0) base = atomicAdd(&a.sc.tickets[list], PER * GROUP_BATCH);
    base = __shfl_sync(FULL, base, 0);
    if (base >= cnt) break;
#pragma unroll 1
    for (int j = 0; j < GROUP_BATCH; ++j) {
      const int it = base + PER * j + lane / W;
      if (it < cnt) {  // the same in every lane of a group
        const int64_t vec = L[it];
        const int64_t s = a.off[vec];
        const int n = (int)(a.off[vec + 1] - s);
        group_forward<T, W>(a.x + s, a.y ? a.y + s : nullptr, n, lane, a.out, vec);
      }
    }
  }
}

// Resident threads per SM asked of the persistent forward: 5 x 256 for
// binary32 (at most 48 registers), 4 x 256 for binary64 (at most 64; 48
// bytes of spill; against 3 x 256 at 80 registers: ragged binary64 forward
// 7.29 -> 7.02 ms, forward + backward 1.652 -> 1.630 ms).
template <typename T>
constexpr int ragged_min_blocks(int B) { return sizeof(T) == 4 ? 5 * 256 / B : 4 * 256 / B; }

// The descriptors of the items of one warp ticket (in shared memory: the
// kernel's registers are at their cap).
struct TicketItems {
  int64_t s[WARP_BATCH];
  int32_t n[WARP_BATCH];
  int32_t vec[WARP_BATCH];
};

template <typename T, int B>
__global__ void __launch_bounds__(B, ragged_min_blocks<T>(B)) k_ragged(RaggedArgs<T> a) {
  __shared__ BlockShared<T, B> sh;
  __shared__ TicketItems tk[B / 32];
  const int t = threadIdx.x, lane = t & 31;
  const int nblk = a.sc.counts[LIST_BLOCK], nwarp = a.sc.counts[LIST_WARP], nthr = a.sc.counts[LIST_THREAD];
  const int32_t* Lb = a.sc.items + LIST_BLOCK * a.count;
  const int32_t* Lw = a.sc.items + LIST_WARP * a.count;
  const int32_t* Lt = a.sc.items + LIST_THREAD * a.count;

  // block items, one ticket per item
  for (;;) {
    if (t == 0) sh.item = atomicAdd(&a.sc.tickets[LIST_BLOCK], 1);
    __syncthreads();
    const int it = sh.item;
    __syncthreads();
    if (it >= nblk) break;
    const int64_t vec = Lb[it];
    const int64_t s = a.off[vec];
    const int n = (int)(a.off[vec + 1] - s);
    block_forward_stream<T, B>(a.x + s, a.y ? a.y + s : nullptr, n, a.out, vec, sh);
  }

  // warp items, WARP_BATCH per ticket.  binary32 (warp_prefetch) prefetches
  // the next item of the ticket into L2 during the current item.
  for (;;) {
    int base = 0;
    if (lane == 0) base = atomicAdd(&a.sc.tickets[LIST_WARP], WARP_BATCH);
    base = __shfl_sync(FULL, base, 0);
    if (base >= nwarp) break;
    if constexpr (sizeof(T) == 8) {
      // binary64: two items at a time share one square root and reciprocal
      // (warp_forward_stream_batch; the pair's vectors stay in L1 between
      // passes 2 and 3).  Measured: forward 7.34 -> 7.29 ms, forward +
      // backward 1.67 -> 1.645 ms; four at a time 7.34 and 1.63 ms.
      for (int j = 0; j < WARP_BATCH && base + j < nwarp; j += 2) {
        const int nb = (nwarp - (base + j)) < 2 ? (nwarp - (base + j)) : 2;
        auto item = [&](int jj, const T*& xr, T*& yr, int& nn, int64_t& vec) {
          vec = Lw[base + j + jj];
          const int64_t s = a.off[vec];
          nn = (int)(a.off[vec + 1] - s);
          xr = a.x + s;
          yr = a.y ? a.y + s : nullptr;
        };
        warp_forward_stream_batch<T, 2, MAX_LEN, true>(item, nb, lane, a.out);
      }
    } else {
      // the ticket's item descriptors, read by lanes 0 .. WARP_BATCH-1 together
      TicketItems& d = tk[t >> 5];
      if (lane < WARP_BATCH && base + lane < nwarp) {
        const int32_t v = Lw[base + lane];
        const int64_t s0 = a.off[v];
        d.vec[lane] = v;
        d.s[lane] = s0;
        d.n[lane] = (int)(a.off[v + 1] - s0);
      }
      __syncwarp();
      const int nb = nwarp - base < WARP_BATCH ? nwarp - base : WARP_BATCH;
      for (int j = 0; j < nb; ++j) {
        const int64_t s = d.s[j];
        // the next item of the ticket is prefetched into L2 once pass 1 has
        // read this one (see WARP_PREFETCH_F32)
        auto prefetch_next = [&]() {
          if (warp_prefetch<T>() && j + 1 < nb) prefetch_range_l2(a.x + d.s[j + 1], d.n[j + 1], lane);
        };
        warp_forward_stream<T>(a.x + s, a.y ? a.y + s : nullptr, d.n[j], lane, a.out, d.vec[j], prefetch_next);
      }
      __syncwarp();  // the next ticket rewrites the descriptors
    }
  }

  // group items (binary64): groups of 16, then of 8 lanes
  if constexpr (group16_max<T>() > 0) ragged_group_items<T, 16>(a, LIST_GROUP16, lane);
  if constexpr (group8_max<T>() > 0) ragged_group_items<T, 8>(a, LIST_GROUP8, lane);

  // thread items, THREAD_BATCH groups of 32 per ticket
  for (;;) {
    int base = 0;
    if (lane == 0) base = atomicAdd(&a.sc.tickets[LIST_THREAD], 32 * THREAD_BATCH);
    base = __shfl_sync(FULL, base, 0);
    if (base >= nthr) break;
#pragma unroll 1
    for (int j = 0; j < THREAD_BATCH; ++j) {
      const int it = base + 32 * j + lane;
      if (it < nthr) {
        const int64_t vec = Lt[it];
        const int64_t s = a.off[vec];
        const int n = (int)(a.off[vec + 1] - s);
        thread_item_fwd<T>(a.x + s, a.y ? a.y + s : nullptr, n, a.out, vec);
      }
    }
  }
}

// Backward, block list: one block per vector, grid-stride over the list.
template <typename T, int B>
__global__ void __launch_bounds__(B) k_ragged_bwd_blocks(RaggedArgs<T> a) {
  __shared__ BlockShared<T, B> sh;
  const int nblk = a.sc.counts[LIST_BLOCK];
  const int32_t* Lb = a.sc.items + LIST_BLOCK * a.count;
  for (int it = blockIdx.x; it < nblk; it += gridDim.x) {
    const int64_t vec = Lb[it];
    const int64_t s = a.off[vec];
    const int n = (int)(a.off[vec + 1] - s);
    block_backward_stream<T, B>(a.x + s, a.g + s, a.y + s, n, a.h_in[vec], a.c_in[vec], sh);
  }
}

// Backward, warp list: one warp per vector, warp-stride over the list.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 3 : 1) k_ragged_bwd_warps(RaggedArgs<T> a) {
  const int lane = threadIdx.x & 31;
  const int nwarp = a.sc.counts[LIST_WARP];
  const int32_t* Lw = a.sc.items + LIST_WARP * a.count;
  const int w0 = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
  for (int it = w0; it < nwarp; it += nw) {
    const int64_t vec = Lw[it];
    const int64_t s = a.off[vec];
    const int n = (int)(a.off[vec + 1] - s);
    warp_backward_stream<T>(a.x + s, a.g + s, a.y + s, n, lane, a.h_in[vec], a.c_in[vec]);
  }
}

// Backward, a group list: one group of W lanes per vector, 32 / W vectors per
// warp, warp-stride over the list.  Three blocks of 256 per SM (binary64:
// 80 registers and 16 bytes of spill, against 2 blocks at 104 registers;
// with the thread kernel below, forward + backward 1.652 -> 1.635 ms).
template <typename T, int W>
__global__ void __launch_bounds__(256, 3) k_ragged_bwd_groups(RaggedArgs<T> a, int list) {
  constexpr int PER = 32 / W;
  const int lane = threadIdx.x & 31;
  const int cnt = a.sc.counts[list];
  const int32_t* L = a.sc.items + (int64_t)list * a.count;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t it0 = w0 * PER; it0 < cnt; it0 += nw * PER) {
    const int64_t it = it0 + lane / W;
    if (it < cnt) {  // the same in every lane of a group
      const int64_t vec = L[it];
      const int64_t s = a.off[vec];
      const int n = (int)(a.off[vec + 1] - s);
      group_backward<T, W>(a.x + s, a.g + s, a.y + s, n, lane, a.h_in[vec], a.c_in[vec]);
    }
  }
}

// Backward, thread list: one thread per vector, grid-stride over the list
// (three blocks of 256 per SM, as the group kernel).
template <typename T>
__global__ void __launch_bounds__(256, 3) k_ragged_bwd_threads(RaggedArgs<T> a) {
  const int nthr = a.sc.counts[LIST_THREAD];
  const int32_t* Lt = a.sc.items + LIST_THREAD * a.count;
  const int stride = (int)((int64_t)gridDim.x * blockDim.x);
  for (int it = (int)((int64_t)blockIdx.x * blockDim.x + threadIdx.x); it < nthr; it += stride) {
    const int64_t vec = Lt[it];
    const int64_t s = a.off[vec];
    const int n = (int)(a.off[vec + 1] - s);
    thread_item_bwd<T>(a.x + s, a.g + s, a.y + s, n, a.h_in[vec], a.c_in[vec]);
  }
}

// ---------------------------------------------------------------------------
template <typename K>
inline int wave_of(K kernel, int threads) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
  if (per_sm < 1) per_sm = 1;
  return per_sm * device_sm_count();
}

template <typename T>
inline int full_wave_dispatch(const RaggedMapping& m) {
  return m.block_threads == 128 ? wave_of(k_ragged<T, 128>, 128) : wave_of(k_ragged<T, 256>, 256);
}

template <typename T>
inline void launch_backward_lists(const RaggedArgs<T>& a, const RaggedMapping& m, cudaStream_t s) {
  const int cap = m.grid_blocks > 0 ? m.grid_blocks : 1 << 30;
  auto clamp = [cap](int g) { return g < cap ? g : cap; };
  if (m.block_threads == 128) {
    k_ragged_bwd_blocks<T, 128><<<clamp(wave_of(k_ragged_bwd_blocks<T, 128>, 128)), 128, 0, s>>>(a);
  } else {
    k_ragged_bwd_blocks<T, 256><<<clamp(wave_of(k_ragged_bwd_blocks<T, 256>, 256)), 256, 0, s>>>(a);
  }
  k_ragged_bwd_warps<T><<<clamp(wave_of(k_ragged_bwd_warps<T>, 256)), 256, 0, s>>>(a);
  if constexpr (group16_max<T>() > 0)
    k_ragged_bwd_groups<T, 16><<<clamp(wave_of(k_ragged_bwd_groups<T, 16>, 256)), 256, 0, s>>>(a, LIST_GROUP16);
  if constexpr (group8_max<T>() > 0)
    k_ragged_bwd_groups<T, 8><<<clamp(wave_of(k_ragged_bwd_groups<T, 8>, 256)), 256, 0, s>>>(a, LIST_GROUP8);
  k_ragged_bwd_threads<T><<<clamp(wave_of(k_ragged_bwd_threads<T>, 256)), 256, 0, s>>>(a);
}

template <typename T>
inline void launch_persistent(const RaggedArgs<T>& a, const RaggedMapping& m, cudaStream_t s) {
  const int grid = m.grid_blocks > 0 ? m.grid_blocks : full_wave_dispatch<T>(m);
  if (m.block_threads == 128) k_ragged<T, 128><<<grid, 128, 0, s>>>(a);
  else k_ragged<T, 256><<<grid, 256, 0, s>>>(a);
}

template <typename T>
cudaError_t launch_ragged_impl(const T* x, T* y, T* norm, T* saved_h, int8_t* saved_code, const T* g, const T* h_in,
                               const int8_t* code_in, T* grad, const int64_t* offsets, int64_t count,
                               int64_t capacity, bool validate, const RaggedMapping& map, const RaggedScratch& sc,
                               bool backward, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(sc.counts, 0, 2 * NLISTS * sizeof(int32_t), s);  // counts, tickets: adjacent
  if (e != cudaSuccess) return e;
  {
    const int64_t blocks_needed = (count + CLASSIFY_THREADS - 1) / CLASSIFY_THREADS;
    const int64_t cap = (int64_t)device_sm_count() * 2;
    const int grid = (int)(blocks_needed < cap ? (blocks_needed > 0 ? blocks_needed : 1) : cap);
    VecOut<T> zo = backward ? VecOut<T>{nullptr, nullptr, nullptr} : VecOut<T>{norm, saved_h, saved_code};
    k_classify<T><<<grid, CLASSIFY_THREADS, 0, s>>>(offsets, count, capacity, map.thread_max, map.warp_max,
                                                     validate ? 1 : 0, sc, zo);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  RaggedArgs<T> a;
  a.off = offsets;
  a.sc = sc;
  a.count = count;
  if (!backward) {
    a.x = x; a.y = y; a.g = nullptr; a.h_in = nullptr; a.c_in = nullptr;
    a.out = VecOut<T>{norm, saved_h, saved_code};
    launch_persistent<T>(a, map, s);
  } else {
    a.x = x; a.y = grad; a.g = g; a.h_in = h_in; a.c_in = code_in;
    a.out = VecOut<T>{nullptr, nullptr, nullptr};
    launch_backward_lists<T>(a, map, s);
  }
  return cudaGetLastError();
}

}  // namespace ngb
