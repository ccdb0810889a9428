// Host build of the warp and block forms of the kernels' arithmetic
// (csrc/ngb_rowpath.cuh), run on an emulated block of threads
// (tests/hostwarp/cuda_runtime.h), for CPU tests against the oracle.  The
// loops over rows follow the row kernels with a grid of one block.
//
//   rowpath_host_check <f32|f64> <n> <path> <in> <out>
//
// Forward paths read count x n values and write y (count x n), r, h (count
// each) and code (count bytes):
//   warp    rows in registers, one warp per row (warp_load + warp_forward_loaded;
//           16-byte chunks for binary32 when n % 4 == 0), n <= 1024
//   half    binary32, one row per half-warp (half_forward_f32<4>), 128 < n <= 256, n % 4 == 0
//   stream  one warp streaming the row (warp_forward_stream)
//   batch   one warp streaming 4 rows with one square root and reciprocal
//           (warp_forward_stream_batch)
//   block   one block of 256 threads streaming the row (block_forward_stream)
//   pairs   one warp streaming 2 rows of different lengths with one square
//           root and reciprocal and the partial-round skip (the ragged
//           binary64 warp items: warp_forward_stream_batch<T, 2, MAX_LEN, true>);
//           row i holds a vector of length n - (i mod 5) (at least 5)
//   thread  one thread per row (the ragged thread items, thread_item_fwd),
//           n <= 16; row i holds a vector of length 1 + i mod n
//   group8, group16  groups of W = 8 or 16 lanes, 32 / W rows per warp
//           (csrc/ngb_grouppath.cuh), n <= 8 W; row i holds a vector of
//           length n - (i mod 5) (at least 5) in its first components, so
//           that the groups of a warp differ in length
// Backward paths read y, g (count x n each), h (count) and code (count bytes)
// and write grad (count x n): warp_bwd (n <= 1024), stream_bwd, block_bwd,
// group8_bwd, group16_bwd (lengths as the group forward paths), thread_bwd
// (n <= 16, one thread per row, the ragged thread items; row i holds a
// vector of length 1 + i mod n).
// Path ghr: see run_ghr.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "ngb_grouppath.cuh"
#include "ngb_threadpath.cuh"

using namespace ngb;

static int chunks(int n, int per) {
  int c = 1;
  while (c * per < n) c *= 2;
  return c;
}

template <typename T>
struct Rows {
  int64_t count = 0;
  int n = 0;
  std::vector<T> x, y, g, r, h, grad;
  std::vector<int8_t> code;
};

template <typename T, int V, int CH>
static void warp_rows(Rows<T>& d) {
  hemu::run_block(64, [&] {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = threadIdx.x >> 5, nw = 2;
    VecOut<T> out{d.r.data(), d.h.data(), d.code.data()};
    for (int64_t row = w0; row < d.count; row += nw) {
      T v[CH][V];
      warp_load<T, V, CH>(d.x.data() + row * d.n, d.n, lane, v);
      warp_forward_loaded<T, V, CH>(v, d.x.data() + row * d.n, d.y.data() + row * d.n, d.n, lane, out, row);
    }
  });
}

template <typename T, int V, int CH>
static void warp_rows_bwd(Rows<T>& d) {
  hemu::run_block(64, [&] {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = threadIdx.x >> 5, nw = 2;
    for (int64_t row = w0; row < d.count; row += nw)
      warp_backward<T, V, CH>(d.y.data() + row * d.n, d.g.data() + row * d.n, d.grad.data() + row * d.n, d.n, lane,
                              d.h[row], d.code[row]);
  });
}

template <typename T, bool BWD>
static void warp_dispatch(Rows<T>& d) {
  const int n = d.n;
  if (sizeof(T) == 4 && n % 4 == 0) {
    constexpr int W = sizeof(T) == 4 ? 4 : 1;
    switch (chunks(n, 32 * W)) {
      case 1: return BWD ? warp_rows_bwd<T, W, 1>(d) : warp_rows<T, W, 1>(d);
      case 2: return BWD ? warp_rows_bwd<T, W, 2>(d) : warp_rows<T, W, 2>(d);
      case 4: return BWD ? warp_rows_bwd<T, W, 4>(d) : warp_rows<T, W, 4>(d);
      default: return BWD ? warp_rows_bwd<T, W, 8>(d) : warp_rows<T, W, 8>(d);
    }
  }
  switch (chunks(n, 32)) {
    case 1: return BWD ? warp_rows_bwd<T, 1, 1>(d) : warp_rows<T, 1, 1>(d);
    case 2: return BWD ? warp_rows_bwd<T, 1, 2>(d) : warp_rows<T, 1, 2>(d);
    case 4: return BWD ? warp_rows_bwd<T, 1, 4>(d) : warp_rows<T, 1, 4>(d);
    case 8: return BWD ? warp_rows_bwd<T, 1, 8>(d) : warp_rows<T, 1, 8>(d);
    case 16: return BWD ? warp_rows_bwd<T, 1, 16>(d) : warp_rows<T, 1, 16>(d);
    default: return BWD ? warp_rows_bwd<T, 1, 32>(d) : warp_rows<T, 1, 32>(d);
  }
}

// Row lengths of the group paths.
static int group_len(int n, int64_t row) {
  const int m = n - (int)(row % 5);
  return m < 5 ? 5 : m;
}

template <typename T, int W, bool BWD>
static void group_rows(Rows<T>& d) {
  constexpr int PER = 32 / W;
  hemu::run_block(64, [&] {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = threadIdx.x >> 5, nw = 2;
    VecOut<T> out{d.r.data(), d.h.data(), d.code.data()};
    for (int64_t r0 = w0 * PER; r0 < d.count; r0 += nw * PER) {
      const int64_t row = r0 + lane / W;
      if (row >= d.count) continue;
      const int len = group_len(d.n, row);
      if (BWD)
        group_backward<T, W>(d.y.data() + row * d.n, d.g.data() + row * d.n, d.grad.data() + row * d.n, len, lane,
                             d.h[row], d.code[row]);
      else
        group_forward<T, W>(d.x.data() + row * d.n, d.y.data() + row * d.n, len, lane, out, row);
    }
  });
}

template <typename T>
static void run_path(Rows<T>& d, const std::string& path) {
  VecOut<T> out{d.r.data(), d.h.data(), d.code.data()};
  const int n = d.n;
  if (path == "warp") {
    warp_dispatch<T, false>(d);
  } else if (path == "warp_bwd") {
    warp_dispatch<T, true>(d);
  } else if (path == "half") {
    if constexpr (sizeof(T) == 4) {
      hemu::run_block(64, [&] {
        const int lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
        const unsigned gmask = half ? 0xFFFF0000u : 0x0000FFFFu;
        const int64_t w0 = threadIdx.x >> 5, nw = 2;
        for (int64_t r0 = 2 * w0; r0 < d.count; r0 += 2 * nw) {
          const int64_t row = r0 + half;
          const bool valid = row < d.count;
          const int64_t rr = valid ? row : r0;
          half_forward_f32<4>(d.x.data() + rr * n, valid ? d.y.data() + rr * n : nullptr, n, hl, gmask, out, rr,
                              valid);
        }
      });
    }
  } else if (path == "pairs") {
    hemu::run_block(64, [&] {
      const int lane = threadIdx.x & 31;
      const int64_t w0 = threadIdx.x >> 5, nw = 2;
      for (int64_t g = w0 * 2; g < d.count; g += nw * 2) {
        const int nb = (int)((d.count - g) < 2 ? (d.count - g) : 2);
        auto item = [&](int j, const T*& xr, T*& yr, int& nn, int64_t& vec) {
          vec = g + j;
          xr = d.x.data() + vec * n;
          yr = d.y.data() + vec * n;
          nn = group_len(n, vec);
        };
        warp_forward_stream_batch<T, 2, MAX_LEN, true>(item, nb, lane, out);
      }
    });
  } else if (path == "group8" || path == "group16" || path == "group8_bwd" || path == "group16_bwd") {
    const bool bwd = path.size() > 4 && path.compare(path.size() - 4, 4, "_bwd") == 0;
    const int W = path.compare(0, 7, "group16") == 0 ? 16 : 8;
    if (n > 8 * W) {
      fprintf(stderr, "group paths take n <= 8 W\n");
      exit(2);
    }
    if (W == 8) bwd ? group_rows<T, 8, true>(d) : group_rows<T, 8, false>(d);
    else bwd ? group_rows<T, 16, true>(d) : group_rows<T, 16, false>(d);
  } else if (path == "stream") {
    hemu::run_block(64, [&] {
      const int lane = threadIdx.x & 31;
      for (int64_t row = threadIdx.x >> 5; row < d.count; row += 2)
        warp_forward_stream<T>(d.x.data() + row * n, d.y.data() + row * n, n, lane, out, row);
    });
  } else if (path == "thread") {  // one thread per row, row i of length 1 + i mod n (n <= 16)
    hemu::run_block(32, [&] {
      for (int64_t row = threadIdx.x; row < d.count; row += 32)
        thread_item_fwd<T>(d.x.data() + row * n, d.y.data() + row * n, 1 + (int)(row % n), out, row);
    });
  } else if (path == "thread_bwd") {  // one thread per row, row i of length 1 + i mod n (n <= 16)
    hemu::run_block(32, [&] {
      for (int64_t row = threadIdx.x; row < d.count; row += 32)
        thread_item_bwd<T>(d.y.data() + row * n, d.g.data() + row * n, d.grad.data() + row * n,
                           1 + (int)(row % n), d.h[row], d.code[row]);
    });
  } else if (path == "stream_bwd") {
    hemu::run_block(64, [&] {
      const int lane = threadIdx.x & 31;
      for (int64_t row = threadIdx.x >> 5; row < d.count; row += 2)
        warp_backward_stream<T>(d.y.data() + row * n, d.g.data() + row * n, d.grad.data() + row * n, n, lane,
                                d.h[row], d.code[row]);
    });
  } else if (path == "batch") {
    constexpr int NB = 4;
    hemu::run_block(64, [&] {
      const int lane = threadIdx.x & 31;
      const int64_t w0 = threadIdx.x >> 5, nw = 2;
      for (int64_t g = w0 * NB; g < d.count; g += nw * NB) {
        const int nb = (int)((d.count - g) < NB ? (d.count - g) : NB);
        auto item = [&](int j, const T*& xr, T*& yr, int& nn, int64_t& vec) {
          vec = g + j;
          xr = d.x.data() + vec * n;
          yr = d.y.data() + vec * n;
          nn = n;
        };
        warp_forward_stream_batch<T, NB, MAX_LEN>(item, nb, lane, out);
      }
    });
  } else if (path == "block") {
    BlockShared<T, 256> sh;
    hemu::run_block(256, [&] {
      for (int64_t row = 0; row < d.count; ++row)
        block_forward_stream<T, 256>(d.x.data() + row * n, d.y.data() + row * n, n, out, row, sh);
    });
  } else if (path == "block_bwd") {
    BlockShared<T, 256> sh;
    hemu::run_block(256, [&] {
      for (int64_t row = 0; row < d.count; ++row)
        block_backward_stream<T, 256>(d.y.data() + row * n, d.g.data() + row * n, d.grad.data() + row * n, n,
                                      d.h[row], d.code[row], sh);
    });
  } else {
    fprintf(stderr, "unknown path %s\n", path.c_str());
    exit(2);
  }
}

template <typename T>
static int run(int n, const std::string& path, const char* in, const char* outp) {
  FILE* f = fopen(in, "rb");
  if (!f) { perror(in); return 2; }
  fseek(f, 0, SEEK_END);
  const long bytes = ftell(f);
  fseek(f, 0, SEEK_SET);
  const bool bwd = path.size() > 4 && path.compare(path.size() - 4, 4, "_bwd") == 0;
  Rows<T> d;
  d.n = n;
  d.count = bwd ? bytes / (long)(2 * n * sizeof(T) + sizeof(T) + 1) : bytes / (long)(n * sizeof(T));
  const size_t m = (size_t)d.count * n;
  auto rd = [&](void* p, size_t b) {
    if (b && fread(p, 1, b, f) != b) { fprintf(stderr, "short read\n"); exit(2); }
  };
  d.code.assign(d.count, 0);
  d.r.assign(d.count, T(0));
  d.h.assign(d.count, T(0));
  if (bwd) {
    d.y.resize(m);
    d.g.resize(m);
    d.grad.assign(m, T(0));
    rd(d.y.data(), m * sizeof(T));
    rd(d.g.data(), m * sizeof(T));
    rd(d.h.data(), d.count * sizeof(T));
    rd(d.code.data(), d.count);
  } else {
    d.x.resize(m);
    d.y.assign(m, T(0));
    rd(d.x.data(), m * sizeof(T));
  }
  fclose(f);
  run_path<T>(d, path);
  FILE* o = fopen(outp, "wb");
  if (!o) { perror(outp); return 2; }
  if (bwd) {
    fwrite(d.grad.data(), sizeof(T), m, o);
  } else {
    fwrite(d.y.data(), sizeof(T), m, o);
    fwrite(d.r.data(), sizeof(T), d.count, o);
    fwrite(d.h.data(), sizeof(T), d.count, o);
    fwrite(d.code.data(), 1, d.count, o);
  }
  fclose(o);
  return 0;
}

// Path "ghr" (f64): the decision of grad_h_in_range against brute force.
// Reads count rows of y (n values), g (n values), dot (1) and h (1), all
// binary64 in that order per array (y of every row, then g, dot, h), and
// writes count bytes: 0 when products_in_range(keys of y, key of dot) fails
// (the decision is not taken), else 1 + the decision; then count bytes: 1
// when every d_k = RN(g_k - RN(y_k dot)) satisfies f64emu::mul_in_range(d_k, h)
// and no g_k or p_k exceeds biased exponent 2045 (f64emu::add_signed's range).
static int run_ghr(int n, const char* inp, const char* outp) {
  FILE* f = fopen(inp, "rb");
  if (!f) { perror(inp); return 2; }
  fseek(f, 0, SEEK_END);
  const long bytes = ftell(f);
  fseek(f, 0, SEEK_SET);
  const long count = bytes / (long)((2 * n + 2) * sizeof(double));
  std::vector<double> y((size_t)count * n), g((size_t)count * n), dot(count), h(count);
  auto rd = [&](void* p, size_t b) {
    if (b && fread(p, 1, b, f) != b) { fprintf(stderr, "short read\n"); exit(2); }
  };
  rd(y.data(), y.size() * sizeof(double));
  rd(g.data(), g.size() * sizeof(double));
  rd(dot.data(), dot.size() * sizeof(double));
  rd(h.data(), h.size() * sizeof(double));
  fclose(f);
  std::vector<unsigned char> decision(count), brute(count);
  for (long i = 0; i < count; ++i) {
    MagTrack<double> ry, rg, rdot;
    for (int k = 0; k < n; ++k) {
      ry.take(y[(size_t)i * n + k]);
      rg.take(g[(size_t)i * n + k]);
    }
    rdot.take(dot[i]);
    decision[i] = products_in_range(ry, rdot) ? (unsigned char)(1 + (grad_h_in_range(ry, rg, rdot, h[i]) ? 1 : 0)) : 0;
    bool all = true;
    for (int k = 0; k < n; ++k) {
      volatile double p = y[(size_t)i * n + k] * dot[i];
      volatile double d = g[(size_t)i * n + k] - p;
      uint64_t db, hb;
      const double dv = d, hv = h[i];
      memcpy(&db, &dv, 8);
      memcpy(&hb, &hv, 8);
      uint64_t gb, pb;
      const double gv = g[(size_t)i * n + k], pv = p;
      memcpy(&gb, &gv, 8);
      memcpy(&pb, &pv, 8);
      // f64emu::add_signed forms d_k when neither operand exceeds exponent 2045
      all = all && f64emu::mul_in_range(db, hb) && ((gb >> 52) & 0x7FF) <= 2045 && ((pb >> 52) & 0x7FF) <= 2045;
    }
    brute[i] = all ? 1 : 0;
  }
  FILE* o = fopen(outp, "wb");
  if (!o) { perror(outp); return 2; }
  fwrite(decision.data(), 1, count, o);
  fwrite(brute.data(), 1, count, o);
  fclose(o);
  return 0;
}

int main(int argc, char** argv) {
  if (argc != 6) {
    fprintf(stderr, "usage: %s f32|f64 n path in out\n", argv[0]);
    return 2;
  }
  if (!strcmp(argv[3], "ghr")) return run_ghr(atoi(argv[2]), argv[4], argv[5]);
  const int n = atoi(argv[2]);
  const bool short_ok = !strcmp(argv[3], "thread_bwd") || !strcmp(argv[3], "thread");
  if (n < (short_ok ? 1 : 5) || n > (short_ok ? 16 : MAX_LEN)) { fprintf(stderr, "n out of range for the path\n"); return 2; }
  return !strcmp(argv[1], "f32") ? run<float>(n, argv[3], argv[4], argv[5]) : run<double>(n, argv[3], argv[4], argv[5]);
}
