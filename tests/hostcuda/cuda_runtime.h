// Host stand-ins for the CUDA declarations that the per-thread arithmetic of
// csrc/ngb_arith.cuh uses, so that it compiles with a host C++ compiler for
// CPU tests (tests/kernel_host_check.cpp).  The arithmetic intrinsics come
// from ngb_host_intrinsics.h; the warp collectives are declared for the
// members of MagTrack that the per-thread paths never call, and act on a
// single lane.
#pragma once
#include "ngb_host_intrinsics.h"

template <typename T>
inline T __shfl_xor_sync(unsigned, T v, int) { return v; }
inline bool __any_sync(unsigned, bool p) { return p; }
inline unsigned __reduce_max_sync(unsigned, unsigned v) { return v; }
inline unsigned __reduce_min_sync(unsigned, unsigned v) { return v; }
