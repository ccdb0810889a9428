// Host build of the kernels' per-thread arithmetic (csrc/ngb_arith.cuh, with
// tests/hostcuda/cuda_runtime.h for the CUDA intrinsics), for CPU tests
// against the oracle.
//
//   kernel_host_check <f32|f64> <dim> <mode> <quat_zero> <in> <out>
//
// Forward modes read count x dim values from <in> and write y (count x dim),
// r (count), h (count) and code (count bytes) to <out>:
//   fwd     the library's per-vector forward: normalize_small (dim <= 4) or
//           normalize_thread_generic (5 <= dim <= 16)
//   hw      normalize_small_hw, the hardware-operation form alone (dim <= 4)
//   padded  binary64: the components zero-padded to 4 and the integer-pipe
//           form for n <= 4 when in range, else normalize_small_hw (the
//           ragged kernel's thread items)
//   sq64    binary64: the integer-pipe form with the squares on the FP64
//           pipe (the dense kernels' choice for warps that are all in range)
//           when in range, else normalize_small_hw
//   quot1, quot2  dim 3: the quotient Algorithms 1 and 2 (ngb_quotient.cuh);
//           h and code are written as zero
// Mode bwd reads y, g (count x dim each), h (count) and code (count bytes)
// and writes grad (count x dim): backward_small or backward_thread_generic.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "ngb_arith.cuh"
#include "ngb_quotient.cuh"

using namespace ngb;

template <typename T>
static std::vector<T> read_vals(FILE* f, size_t n) {
  std::vector<T> v(n);
  if (n && fread(v.data(), sizeof(T), n, f) != n) { fprintf(stderr, "short read\n"); exit(2); }
  return v;
}

template <typename T, int D>
static int fwd_small(const T* x, T* y, T& r, T& h, bool qz, const char* mode) {
  if (!strcmp(mode, "quot1") || !strcmp(mode, "quot2")) {
    if constexpr (D == 3) {
      const T xv[3] = {x[0], x[1], x[2]};
      T yv[3];
      if (mode[4] == '1') quotient1_3<T>(xv, yv, r);
      else quotient2_3<T>(xv, yv, r);
      for (int k = 0; k < 3; ++k) y[k] = yv[k];
      h = T(0);
      return 0;
    }
    fprintf(stderr, "the quotient modes take dim 3\n");
    exit(2);
  }
  if (!strcmp(mode, "hw")) return normalize_small_hw<T, D>(x, y, r, h, qz);
  if (!strcmp(mode, "sq64")) {
    if constexpr (sizeof(T) == 8) {
      const SmallKeysF64<D> kk(x);
      if (kk.ok) return normalize_small_f64_int<D, true>(x, y, r, h, qz, kk);
      return normalize_small_hw<T, D>(x, y, r, h, qz);
    }
    fprintf(stderr, "sq64 is a binary64 mode\n");
    exit(2);
  }
  if (!strcmp(mode, "padded")) {
    if constexpr (sizeof(T) == 8) {
      double xv[4] = {0, 0, 0, 0}, yv[4];
      for (int k = 0; k < D; ++k) xv[k] = x[k];
      const SmallKeysF64<4> kk(xv);
      if (kk.ok) {
        const int code = normalize_small_f64_int<4>(xv, yv, r, h, false, kk);
        for (int k = 0; k < D; ++k) y[k] = yv[k];
        return code;
      }
      return normalize_small_hw<T, D>(x, y, r, h, false);
    }
    fprintf(stderr, "padded is a binary64 mode\n");
    exit(2);
  }
  return normalize_small<T, D>(x, y, r, h, qz);
}

template <typename T>
static int run(int dim, const char* mode, bool qz, FILE* in, FILE* out) {
  fseek(in, 0, SEEK_END);
  const long bytes = ftell(in);
  fseek(in, 0, SEEK_SET);
  const bool bwd = !strcmp(mode, "bwd");
  const size_t per = bwd ? (2 * dim * sizeof(T) + sizeof(T) + 1) : dim * sizeof(T);
  const size_t count = (size_t)bytes / per;
  if (bwd) {
    std::vector<T> y = read_vals<T>(in, count * dim), g = read_vals<T>(in, count * dim), h = read_vals<T>(in, count);
    std::vector<int8_t> c = read_vals<int8_t>(in, count);
    std::vector<T> grad(count * dim);
    for (size_t i = 0; i < count; ++i) {
      const T* yi = &y[i * dim];
      const T* gi = &g[i * dim];
      T* o = &grad[i * dim];
      switch (dim) {
        case 1: backward_small<T, 1>(yi, gi, h[i], c[i], o); break;
        case 2: backward_small<T, 2>(yi, gi, h[i], c[i], o); break;
        case 3: backward_small<T, 3>(yi, gi, h[i], c[i], o); break;
        case 4: backward_small<T, 4>(yi, gi, h[i], c[i], o); break;
        default: backward_thread_generic<T, 16>(yi, gi, dim, h[i], c[i], o); break;
      }
    }
    fwrite(grad.data(), sizeof(T), grad.size(), out);
    return 0;
  }
  std::vector<T> x = read_vals<T>(in, count * dim), y(count * dim), r(count), h(count);
  std::vector<int8_t> c(count);
  for (size_t i = 0; i < count; ++i) {
    const T* xi = &x[i * dim];
    T* yi = &y[i * dim];
    int code;
    switch (dim) {
      case 1: code = fwd_small<T, 1>(xi, yi, r[i], h[i], qz, mode); break;
      case 2: code = fwd_small<T, 2>(xi, yi, r[i], h[i], qz, mode); break;
      case 3: code = fwd_small<T, 3>(xi, yi, r[i], h[i], qz, mode); break;
      case 4: code = fwd_small<T, 4>(xi, yi, r[i], h[i], qz, mode); break;
      default: code = normalize_thread_generic<T, 16>(xi, yi, dim, r[i], h[i]); break;
    }
    c[i] = (int8_t)code;
  }
  fwrite(y.data(), sizeof(T), y.size(), out);
  fwrite(r.data(), sizeof(T), r.size(), out);
  fwrite(h.data(), sizeof(T), h.size(), out);
  fwrite(c.data(), 1, c.size(), out);
  return 0;
}

int main(int argc, char** argv) {
  if (argc != 7) {
    fprintf(stderr, "usage: %s f32|f64 dim fwd|hw|padded|bwd quat_zero in out\n", argv[0]);
    return 2;
  }
  const int dim = atoi(argv[2]);
  if (dim < 1 || dim > 16) { fprintf(stderr, "dim must be 1..16\n"); return 2; }
  FILE* in = fopen(argv[5], "rb");
  FILE* out = fopen(argv[6], "wb");
  if (!in || !out) { fprintf(stderr, "cannot open files\n"); return 2; }
  const bool qz = atoi(argv[4]) != 0;
  const int rc = !strcmp(argv[1], "f32") ? run<float>(dim, argv[3], qz, in, out) : run<double>(dim, argv[3], qz, in, out);
  fclose(in);
  fclose(out);
  return rc;
}
