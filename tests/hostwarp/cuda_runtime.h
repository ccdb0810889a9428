// Host emulation of the CUDA thread model that the warp and block forms of
// the kernels' arithmetic (csrc/ngb_rowpath.cuh) use, so that they compile
// with a host C++ compiler and run on CPU for tests
// (tests/rowpath_host_check.cpp).
//
// One block of `n` threads runs as n std::threads.  A warp collective with
// mask m exchanges values through per-thread slots and meets the other lanes
// of m (in the same warp) at a barrier of popcount(m) participants, twice:
// after every lane has written, and after every lane has read.  Half-warp
// groups (masks 0x0000FFFF and 0xFFFF0000) therefore proceed independently,
// as they do on the GPU.  __syncthreads is a barrier of the whole block.
// The arithmetic intrinsics come from ngb_host_intrinsics.h.
#pragma once
#include <barrier>
#include <cstdint>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <utility>
#include <vector>

#include "../hostcuda/ngb_host_intrinsics.h"

struct float4 { float x, y, z, w; };
struct double2 { double x, y; };
inline float4 make_float4(float a, float b, float c, float d) { return {a, b, c, d}; }
inline double2 make_double2(double a, double b) { return {a, b}; }
inline int __ffs(int v) { return __builtin_ffs(v); }
inline int __popc(unsigned v) { return __builtin_popcount(v); }
template <typename T> inline T __ldcs(const T* p) { return *p; }
template <typename T> inline void __stcs(T* p, T v) { *p = v; }

namespace hemu {

struct Team {
  unsigned n;
  std::barrier<> block_bar;
  std::vector<uint64_t> slot;
  std::mutex mu;
  std::map<std::pair<unsigned, unsigned>, std::unique_ptr<std::barrier<>>> groups;
  explicit Team(unsigned n_) : n(n_), block_bar(n_), slot(n_) {}
  std::barrier<>& group(unsigned warp, unsigned mask) {
    std::lock_guard<std::mutex> g(mu);
    auto& p = groups[{warp, mask}];
    if (!p) p.reset(new std::barrier<>(__builtin_popcount(mask)));
    return *p;
  }
};

inline thread_local Team* team = nullptr;
inline thread_local unsigned tid = 0;

template <typename T> inline uint64_t to_bits(T v) {
  uint64_t u = 0;
  std::memcpy(&u, &v, sizeof(T));
  return u;
}
template <typename T> inline T from_bits(uint64_t u) {
  T v;
  std::memcpy(&v, &u, sizeof(T));
  return v;
}

// Every lane of `mask` publishes v; f(values of the group's lanes) runs after
// all have published; the slots are reused only after all have read.
template <typename T, typename F>
inline auto exchange(unsigned mask, T v, F f) {
  const unsigned w = tid / 32;
  team->slot[tid] = to_bits(v);
  auto& b = team->group(w, mask);
  b.arrive_and_wait();
  auto r = f(w * 32);
  b.arrive_and_wait();
  return r;
}

// Runs fn() on a block of n threads and waits for them.
template <typename F>
inline void run_block(unsigned n, F fn) {
  Team t(n);
  std::vector<std::thread> ts;
  ts.reserve(n);
  for (unsigned i = 0; i < n; ++i)
    ts.emplace_back([&t, i, &fn] {
      team = &t;
      tid = i;
      fn();
    });
  for (auto& th : ts) th.join();
}

struct V3 { unsigned x, y, z; };

}  // namespace hemu

#define threadIdx (hemu::V3{hemu::tid, 0, 0})
#define blockIdx (hemu::V3{0, 0, 0})
#define blockDim (hemu::V3{hemu::team->n, 1, 1})
#define gridDim (hemu::V3{1, 1, 1})

template <typename T>
inline T __shfl_sync(unsigned mask, T v, int src) {
  return hemu::exchange(mask, v, [src](unsigned base) { return hemu::from_bits<T>(hemu::team->slot[base + (src & 31)]); });
}
template <typename T>
inline T __shfl_xor_sync(unsigned mask, T v, int o) {
  const unsigned lane = hemu::tid & 31;
  return __shfl_sync(mask, v, (int)(lane ^ (unsigned)o));
}
inline unsigned __ballot_sync(unsigned mask, int p) {
  return hemu::exchange(mask, (uint64_t)(p != 0), [mask](unsigned base) {
    unsigned r = 0;
    for (unsigned l = 0; l < 32; ++l)
      if ((mask >> l) & 1u) r |= (hemu::team->slot[base + l] ? 1u : 0u) << l;
    return r;
  });
}
inline bool __any_sync(unsigned mask, int p) { return __ballot_sync(mask, p) != 0u; }
inline bool __all_sync(unsigned mask, int p) { return __ballot_sync(mask, p) == mask; }
inline unsigned __reduce_max_sync(unsigned mask, unsigned v) {
  return hemu::exchange(mask, v, [mask](unsigned base) {
    unsigned r = 0;
    for (unsigned l = 0; l < 32; ++l)
      if ((mask >> l) & 1u) r = std::max(r, (unsigned)hemu::team->slot[base + l]);
    return r;
  });
}
inline unsigned __reduce_min_sync(unsigned mask, unsigned v) {
  return hemu::exchange(mask, v, [mask](unsigned base) {
    unsigned r = 0xFFFFFFFFu;
    for (unsigned l = 0; l < 32; ++l)
      if ((mask >> l) & 1u) r = std::min(r, (unsigned)hemu::team->slot[base + l]);
    return r;
  });
}
inline void __syncthreads() { hemu::team->block_bar.arrive_and_wait(); }
inline int __syncthreads_or(int p) {
  hemu::team->slot[hemu::tid] = p ? 1u : 0u;
  hemu::team->block_bar.arrive_and_wait();
  int r = 0;
  for (unsigned i = 0; i < hemu::team->n; ++i) r |= hemu::team->slot[i] ? 1 : 0;
  hemu::team->block_bar.arrive_and_wait();
  return r;
}
