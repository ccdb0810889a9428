// api.cu -- the C ABI of libnormgb (declared in include/normgb.h): argument
// checks, dispatch to the kernels, ragged plans (work lists, mapping, CUDA
// graph replay, autotuner) and error reporting.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "normgb.h"
#include "ngb_args.h"
#include "ngb_internal.h"

namespace {

thread_local std::string g_last_error;

ngb_status fail(ngb_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

ngb_status cuda_fail(cudaError_t e, const char* where) {
  return fail(NGB_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

cudaStream_t cs(ngb_stream_t s) { return reinterpret_cast<cudaStream_t>(s); }

bool stream_capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return st != cudaStreamCaptureStatusNone;
}

}  // namespace

namespace ngb {
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace ngb

struct GraphKey {
  const void* p[10];
  int64_t count;
  int validate;
  ngb::RaggedMapping map;
  bool operator==(const GraphKey& o) const {
    return std::memcmp(p, o.p, sizeof(p)) == 0 && count == o.count && validate == o.validate &&
           map.thread_max == o.map.thread_max && map.warp_max == o.map.warp_max &&
           map.block_threads == o.map.block_threads && map.grid_blocks == o.map.grid_blocks;
  }
};

struct ngb_plan {
  int64_t count = 0;
  int32_t dtype_bytes = 0;
  int64_t capacity = 0;
  int device = 0;
  int32_t* buf = nullptr;  // scratch header, then the work lists (ngb::ragged_scratch)
  ngb::RaggedScratch sc{};
  ngb::RaggedMapping map{8, 8192, 256, 0};
  bool graphs = true;
  cudaStream_t cap_stream = nullptr;
  struct Slot {
    cudaGraphExec_t exec = nullptr;
    GraphKey key{};
  } slot[2];
};

namespace {

ngb_status check_plan(ngb_plan* plan, int64_t count, int dtype_bytes) {
  if (!plan) return fail(NGB_ERR_NO_PLAN, "ragged batch (dim == 0) needs a plan from ngb_plan_create");
  if (plan->count != count || plan->dtype_bytes != dtype_bytes)
    return fail(NGB_ERR_NO_PLAN, "plan was created for another count or dtype");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->device)
    return fail(NGB_ERR_INVALID_ARG, "plan belongs to another device than the current one");
  return NGB_OK;
}

template <typename T>
ngb_status run_ragged(ngb_plan* p, const T* x, T* y, T* norm, T* h, int8_t* code, const T* g, const T* h_in,
                      const int8_t* c_in, T* grad, const int64_t* off, bool validate, bool bwd, bool no_elements,
                      cudaStream_t s) {
  ngb::RaggedMapping m = p->map;
  const int64_t capacity = ngb::classifier_capacity(p->capacity, no_elements);
  if (m.grid_blocks <= 0) m.grid_blocks = ngb::ragged_full_wave<T>(m, bwd);
  if (!p->graphs || stream_capturing(s)) {
    cudaError_t e = ngb::launch_ragged<T>(x, y, norm, h, code, g, h_in, c_in, grad, off, p->count, capacity,
                                          validate, m, p->sc, bwd, s);
    return e == cudaSuccess ? NGB_OK : cuda_fail(e, "ragged launch");
  }
  GraphKey k{};
  const void* ptrs[10] = {x, y, norm, h, code, g, h_in, c_in, grad, off};
  std::memcpy(k.p, ptrs, sizeof(ptrs));
  k.count = p->count;
  k.validate = validate ? 1 : 0;
  k.map = m;
  ngb_plan::Slot& sl = p->slot[bwd ? 1 : 0];
  if (!sl.exec || !(sl.key == k)) {
    if (sl.exec) {
      cudaGraphExecDestroy(sl.exec);
      sl.exec = nullptr;
    }
    if (!p->cap_stream) {
      cudaError_t e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(e, "capture stream");
    }
    cudaError_t e = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    cudaError_t le = ngb::launch_ragged<T>(x, y, norm, h, code, g, h_in, c_in, grad, off, p->count, capacity,
                                           validate, m, p->sc, bwd, p->cap_stream);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(p->cap_stream, &graph);
    if (le != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_fail(le, "ragged launch (capture)");
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&sl.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      sl.exec = nullptr;
      return cuda_fail(e, "cudaGraphInstantiate");
    }
    sl.key = k;
  }
  cudaError_t e = cudaGraphLaunch(sl.exec, s);
  return e == cudaSuccess ? NGB_OK : cuda_fail(e, "cudaGraphLaunch");
}

template <typename T>
ngb_status forward(const T* x, T* y, T* norm, T* h, int8_t* code, int64_t count, int32_t dim, const int64_t* off,
                   ngb_plan* plan, uint32_t flags, ngb_stream_t stream) {
  g_last_error.clear();
  const ngb::ArgCheck a = ngb::check_forward(x, count, dim, off, flags);
  if (a.status != NGB_OK) return fail(a.status, a.message);
  if (dim == 0) {
    ngb_status st = check_plan(plan, count, (int)sizeof(T));
    if (st != NGB_OK) return st;
  }
  if (count == 0) return NGB_OK;
  if (dim > 0) {
    cudaError_t e = ngb::launch_fixed_forward<T>(x, y, norm, h, code, count, dim,
                                                 !(flags & NGB_VECTOR_SEMANTICS), cs(stream));
    return e == cudaSuccess ? NGB_OK : cuda_fail(e, "forward launch");
  }
  return run_ragged<T>(plan, x, y, norm, h, code, nullptr, nullptr, nullptr, nullptr, off,
                       (flags & NGB_VALIDATE_OFFSETS) != 0, false, a.no_elements, cs(stream));
}

template <typename T>
ngb_status backward(const T* y, const T* g, const T* h, const int8_t* code, T* grad, int64_t count, int32_t dim,
                    const int64_t* off, ngb_plan* plan, uint32_t flags, ngb_stream_t stream) {
  g_last_error.clear();
  const ngb::ArgCheck a = ngb::check_backward(y, g, h, code, grad, count, dim, off, flags);
  if (a.status != NGB_OK) return fail(a.status, a.message);
  if (dim == 0) {
    ngb_status st = check_plan(plan, count, (int)sizeof(T));
    if (st != NGB_OK) return st;
  }
  if (count == 0) return NGB_OK;
  if (dim > 0) {
    cudaError_t e = ngb::launch_fixed_backward<T>(y, g, h, code, grad, count, dim, cs(stream));
    return e == cudaSuccess ? NGB_OK : cuda_fail(e, "backward launch");
  }
  return run_ragged<T>(plan, y, nullptr, nullptr, nullptr, nullptr, g, h, code, grad, off,
                       (flags & NGB_VALIDATE_OFFSETS) != 0, true, a.no_elements, cs(stream));
}

}  // namespace

// ---------------------------------------------------------------------------
template <typename T>
static ngb_status quotient3_impl(const T* x, T* y, T* norm, int64_t count, int32_t alg, ngb_stream_t stream,
                                 const char* name) {
  g_last_error.clear();
  if (count < 0 || (alg != 1 && alg != 2)) return fail(NGB_ERR_INVALID_ARG, "count < 0 or alg not 1 or 2");
  if (count == 0) return NGB_OK;
  if (!x || !y) return fail(NGB_ERR_INVALID_ARG, "x and y are required");
  cudaError_t e = ngb::launch_quotient3<T>(x, y, norm, count, alg, cs(stream));
  return e == cudaSuccess ? NGB_OK : cuda_fail(e, name);
}

extern "C" {

ngb_status normalize_f32(const float* x, float* y, float* norm, float* saved_h, int8_t* saved_code, int64_t count,
                         int32_t dim, const int64_t* offsets, ngb_plan* plan, uint32_t flags, ngb_stream_t stream) {
  return forward<float>(x, y, norm, saved_h, saved_code, count, dim, offsets, plan, flags, stream);
}

ngb_status normalize_f64(const double* x, double* y, double* norm, double* saved_h, int8_t* saved_code,
                         int64_t count, int32_t dim, const int64_t* offsets, ngb_plan* plan, uint32_t flags,
                         ngb_stream_t stream) {
  return forward<double>(x, y, norm, saved_h, saved_code, count, dim, offsets, plan, flags, stream);
}

ngb_status normalize_backward_f32(const float* y, const float* g, const float* saved_h, const int8_t* saved_code,
                                  float* grad, int64_t count, int32_t dim, const int64_t* offsets, ngb_plan* plan,
                                  uint32_t flags, ngb_stream_t stream) {
  return backward<float>(y, g, saved_h, saved_code, grad, count, dim, offsets, plan, flags, stream);
}

ngb_status normalize_backward_f64(const double* y, const double* g, const double* saved_h,
                                  const int8_t* saved_code, double* grad, int64_t count, int32_t dim,
                                  const int64_t* offsets, ngb_plan* plan, uint32_t flags, ngb_stream_t stream) {
  return backward<double>(y, g, saved_h, saved_code, grad, count, dim, offsets, plan, flags, stream);
}

ngb_status ngb_plan_create(ngb_plan** out, int64_t count, int32_t dtype_bytes, int64_t capacity) {
  g_last_error.clear();
  if (!out) return fail(NGB_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (count < 0 || capacity < 0) return fail(NGB_ERR_INVALID_ARG, "count or capacity < 0");
  if (count > INT32_MAX) return fail(NGB_ERR_UNSUPPORTED, "ragged count >= 2^31");
  if (dtype_bytes != 4 && dtype_bytes != 8) return fail(NGB_ERR_UNSUPPORTED, "dtype_bytes must be 4 or 8");
  ngb_plan* p = new ngb_plan();
  p->count = count;
  p->dtype_bytes = dtype_bytes;
  p->capacity = capacity;
  cudaError_t e = cudaGetDevice(&p->device);
  const size_t words = ngb::SCRATCH_HEADER_WORDS + (size_t)ngb::ragged_lists(dtype_bytes) * (size_t)count;
  if (e == cudaSuccess) e = cudaMalloc(&p->buf, sizeof(int32_t) * words);
  if (e == cudaSuccess) e = cudaMemset(p->buf, 0, sizeof(int32_t) * ngb::SCRATCH_HEADER_WORDS);
  if (e != cudaSuccess) {
    if (p->buf) cudaFree(p->buf);
    delete p;
    return cuda_fail(e, "ngb_plan_create");
  }
  p->sc = ngb::ragged_scratch(p->buf);
  *out = p;
  return NGB_OK;
}

ngb_status ngb_plan_destroy(ngb_plan* p) {
  g_last_error.clear();
  if (!p) return NGB_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != p->device) cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  for (auto& sl : p->slot)
    if (sl.exec) cudaGraphExecDestroy(sl.exec);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  if (p->buf) cudaFree(p->buf);
  if (prev >= 0 && prev != p->device) cudaSetDevice(prev);
  delete p;
  return NGB_OK;
}

ngb_status ngb_plan_set_mapping(ngb_plan* p, int32_t thread_max, int32_t warp_max, int32_t block_threads,
                                int32_t grid_blocks) {
  g_last_error.clear();
  if (!p) return fail(NGB_ERR_INVALID_ARG, "plan is NULL");
  if (thread_max < 4 || thread_max > 16) return fail(NGB_ERR_INVALID_ARG, "thread_max must be in 4..16");
  if (warp_max < thread_max || warp_max > NGB_MAX_LEN)
    return fail(NGB_ERR_INVALID_ARG, "warp_max must be in thread_max..NGB_MAX_LEN");
  if (block_threads != 128 && block_threads != 256) return fail(NGB_ERR_INVALID_ARG, "block_threads must be 128 or 256");
  if (grid_blocks < 0) return fail(NGB_ERR_INVALID_ARG, "grid_blocks < 0");
  p->map = ngb::RaggedMapping{thread_max, warp_max, block_threads, grid_blocks};
  return NGB_OK;
}

ngb_status ngb_plan_get_mapping(const ngb_plan* p, int32_t* thread_max, int32_t* warp_max, int32_t* block_threads,
                                int32_t* grid_blocks) {
  if (!p) return fail(NGB_ERR_INVALID_ARG, "plan is NULL");
  if (thread_max) *thread_max = p->map.thread_max;
  if (warp_max) *warp_max = p->map.warp_max;
  if (block_threads) *block_threads = p->map.block_threads;
  if (grid_blocks) *grid_blocks = p->map.grid_blocks;
  return NGB_OK;
}

ngb_status ngb_plan_set_graphs(ngb_plan* p, int32_t enable) {
  if (!p) return fail(NGB_ERR_INVALID_ARG, "plan is NULL");
  p->graphs = enable != 0;
  return NGB_OK;
}

ngb_status ngb_query_status(ngb_plan* p, ngb_stream_t stream) {
  g_last_error.clear();
  if (!p) return fail(NGB_ERR_INVALID_ARG, "plan is NULL");
  cudaError_t e = cudaStreamSynchronize(cs(stream));
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  int32_t st = 0;
  e = cudaMemcpy(&st, p->sc.status, sizeof(st), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(p->sc.status, 0, sizeof(int32_t));
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  if (st & 1) return fail(NGB_ERR_BAD_OFFSETS, "a ragged vector with bad offsets was skipped");
  return NGB_OK;
}

// ---------------------------------------------------------------------------
// Autotuner
static std::string tune_key(const std::vector<int64_t>& off, int dtype_bytes) {
  cudaDeviceProp prop{};
  int dev = 0;
  cudaGetDevice(&dev);
  cudaGetDeviceProperties(&prop, dev);
  const int64_t count = (int64_t)off.size() - 1;
  const int edges[] = {4, 8, 16, 64, 256, 512, 1024, 4096};
  int64_t hist[9] = {0};
  for (int64_t i = 0; i < count; ++i) {
    const int64_t n = off[i + 1] - off[i];
    int b = 0;
    while (b < 8 && n > edges[b]) ++b;
    hist[b]++;
  }
  std::string k = std::string(prop.name) + "|f" + std::to_string(dtype_bytes * 8) + "|n" + std::to_string(count) +
                  "|e" + std::to_string(off.back());
  for (int b = 0; b < 9; ++b) k += "|" + std::to_string(count ? (hist[b] * 100 + count / 2) / count : 0);
  for (auto& c : k)
    if (c == ' ') c = '_';
  return k;
}

ngb_status ngb_plan_autotune(ngb_plan* p, const int64_t* offsets, const char* cache_path, ngb_stream_t stream) {
  g_last_error.clear();
  if (!p || !offsets) return fail(NGB_ERR_INVALID_ARG, "plan or offsets is NULL");
  if (p->count == 0) return NGB_OK;
  cudaStream_t s = cs(stream);
  std::vector<int64_t> off((size_t)p->count + 1);
  cudaError_t e = cudaMemcpyAsync(off.data(), offsets, sizeof(int64_t) * off.size(), cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "autotune offsets read");
  for (int64_t i = 0; i < p->count; ++i)
    if (off[i + 1] < off[i] || off[i + 1] - off[i] > NGB_MAX_LEN || off[i] < 0)
      return fail(NGB_ERR_BAD_OFFSETS, "autotune: bad offsets");
  const std::string key = tune_key(off, p->dtype_bytes);
  if (cache_path) {
    if (FILE* f = std::fopen(cache_path, "r")) {
      char line[1024];
      while (std::fgets(line, sizeof(line), f)) {
        char k[900];
        int a, b, c, d;
        if (std::sscanf(line, "%899s %d %d %d %d", k, &a, &b, &c, &d) == 5 && key == k) {
          std::fclose(f);
          return ngb_plan_set_mapping(p, a, b, c, d);
        }
      }
      std::fclose(f);
    }
  }
  const int64_t total = off.back();
  void* buf = nullptr;
  e = cudaMalloc(&buf, (size_t)std::max<int64_t>(total, 1) * p->dtype_bytes);
  if (e != cudaSuccess) return cuda_fail(e, "autotune scratch");
  e = cudaMemsetAsync(buf, 0x3c, (size_t)std::max<int64_t>(total, 1) * p->dtype_bytes, s);
  const ngb::RaggedMapping saved = p->map;
  const bool graphs = p->graphs;
  p->graphs = false;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  ngb::RaggedMapping best_map = saved;
  const int tms[] = {4, 8, 16};
  const int wms[] = {2048, 8192, 65536};
  const int bts[] = {128, 256};
  ngb_status st = NGB_OK;
  for (int tm : tms)
    for (int wm : wms)
      for (int bt : bts) {
        p->map = ngb::RaggedMapping{tm, wm, bt, 0};
        float times[3];
        for (int rep = -1; rep < 3 && st == NGB_OK; ++rep) {
          cudaEventRecord(e0, s);
          if (p->dtype_bytes == 4)
            st = normalize_f32((const float*)buf, (float*)buf, nullptr, nullptr, nullptr, p->count, 0, offsets, p, 0,
                               stream);
          else
            st = normalize_f64((const double*)buf, (double*)buf, nullptr, nullptr, nullptr, p->count, 0, offsets, p,
                               0, stream);
          cudaEventRecord(e1, s);
          cudaEventSynchronize(e1);
          float ms = 0;
          cudaEventElapsedTime(&ms, e0, e1);
          if (rep >= 0) times[rep] = ms;
        }
        if (st != NGB_OK) break;
        std::sort(times, times + 3);
        if (times[1] < best) {
          best = times[1];
          best_map = p->map;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  p->graphs = graphs;
  if (st != NGB_OK) {
    p->map = saved;
    return st;
  }
  p->map = best_map;
  if (cache_path) {
    if (FILE* f = std::fopen(cache_path, "a")) {
      std::fprintf(f, "%s %d %d %d %d\n", key.c_str(), best_map.thread_max, best_map.warp_max,
                   best_map.block_threads, best_map.grid_blocks);
      std::fclose(f);
    }
  }
  return NGB_OK;
}

// ---------------------------------------------------------------------------
ngb_status normalize_to_rotation_f32(const float* q, float* R, float* norm, int64_t count, ngb_stream_t stream) {
  g_last_error.clear();
  if (count < 0) return fail(NGB_ERR_INVALID_ARG, "count < 0");
  if (count == 0) return NGB_OK;
  if (!q || !R) return fail(NGB_ERR_INVALID_ARG, "q and R are required");
  cudaError_t e = ngb::launch_rotation<float>(q, R, norm, count, cs(stream));
  return e == cudaSuccess ? NGB_OK : cuda_fail(e, "rotation launch");
}

ngb_status normalize_to_rotation_f64(const double* q, double* R, double* norm, int64_t count, ngb_stream_t stream) {
  g_last_error.clear();
  if (count < 0) return fail(NGB_ERR_INVALID_ARG, "count < 0");
  if (count == 0) return NGB_OK;
  if (!q || !R) return fail(NGB_ERR_INVALID_ARG, "q and R are required");
  cudaError_t e = ngb::launch_rotation<double>(q, R, norm, count, cs(stream));
  return e == cudaSuccess ? NGB_OK : cuda_fail(e, "rotation launch");
}

ngb_status ngb_copy(void* dst, const void* src, int64_t bytes, ngb_stream_t stream) {
  g_last_error.clear();
  if (bytes < 0) return fail(NGB_ERR_INVALID_ARG, "bytes < 0");
  if (bytes == 0) return NGB_OK;
  if (!dst || !src) return fail(NGB_ERR_INVALID_ARG, "dst and src are required");
  cudaError_t e = ngb::launch_copy(dst, src, bytes, cs(stream));
  return e == cudaSuccess ? NGB_OK : cuda_fail(e, "copy launch");
}

ngb_status ngb_fp64_probe(double* out, int32_t blocks, int32_t iters, int64_t* fp64_ops, ngb_stream_t stream) {
  g_last_error.clear();
  if (!out || blocks <= 0 || iters <= 0) return fail(NGB_ERR_INVALID_ARG, "out is required; blocks and iters > 0");
  if (fp64_ops) *fp64_ops = (int64_t)blocks * 256 * 4 * 2 * (int64_t)iters;
  cudaError_t e = ngb::launch_fp64_probe(out, blocks, iters, cs(stream));
  return e == cudaSuccess ? NGB_OK : cuda_fail(e, "fp64 probe launch");
}

ngb_status quotient_normalize3_f32(const float* x, float* y, float* norm, int64_t count, int32_t alg,
                                   ngb_stream_t stream) {
  return quotient3_impl<float>(x, y, norm, count, alg, stream, "quotient_normalize3_f32 launch");
}

ngb_status quotient_normalize3_f64(const double* x, double* y, double* norm, int64_t count, int32_t alg,
                                   ngb_stream_t stream) {
  return quotient3_impl<double>(x, y, norm, count, alg, stream, "quotient_normalize3_f64 launch");
}

ngb_status naive_normalize_f32(const float* x, float* y, int64_t count, int32_t dim, ngb_stream_t stream) {
  g_last_error.clear();
  if (count < 0 || dim < 2 || dim > 4) return fail(NGB_ERR_INVALID_ARG, "count < 0 or dim not in 2..4");
  if (count == 0) return NGB_OK;
  if (!x || !y) return fail(NGB_ERR_INVALID_ARG, "x and y are required");
  cudaError_t e = ngb::launch_naive<float>(x, y, count, dim, cs(stream));
  return e == cudaSuccess ? NGB_OK : cuda_fail(e, "naive launch");
}

ngb_status naive_normalize_f64(const double* x, double* y, int64_t count, int32_t dim, ngb_stream_t stream) {
  g_last_error.clear();
  if (count < 0 || dim < 2 || dim > 4) return fail(NGB_ERR_INVALID_ARG, "count < 0 or dim not in 2..4");
  if (count == 0) return NGB_OK;
  if (!x || !y) return fail(NGB_ERR_INVALID_ARG, "x and y are required");
  cudaError_t e = ngb::launch_naive<double>(x, y, count, dim, cs(stream));
  return e == cudaSuccess ? NGB_OK : cuda_fail(e, "naive launch");
}

ngb_status ngb_shard_range(const int64_t* offsets, int64_t count, int32_t world, int32_t rank, int64_t* begin,
                           int64_t* end) {
  g_last_error.clear();
  if (!begin || !end) return fail(NGB_ERR_INVALID_ARG, "begin and end are required");
  if (count < 0 || world < 1 || rank < 0 || rank >= world)
    return fail(NGB_ERR_INVALID_ARG, "need count >= 0, world >= 1 and 0 <= rank < world");
  // floor(a r / world) without overflow for any int64 a >= 0 and r <= world
  auto part = [world](int64_t a, int64_t r) { return (int64_t)(((__int128)a * r) / world); };
  if (!offsets) {
    *begin = part(count, rank);
    *end = part(count, (int64_t)rank + 1);
    return NGB_OK;
  }
  const int64_t total = offsets[count] - offsets[0];
  auto cut = [&](int64_t r) -> int64_t {
    if (r <= 0) return 0;
    if (r >= world) return count;
    const int64_t target = offsets[0] + part(total, r);
    return (int64_t)(std::lower_bound(offsets, offsets + count, target) - offsets);  // first start >= target
  };
  *begin = cut(rank);
  *end = cut((int64_t)rank + 1);
  return NGB_OK;
}

ngb_status ngb_quat_bulk_state(uint32_t* state) {
  g_last_error.clear();
  if (!state) return fail(NGB_ERR_INVALID_ARG, "state is NULL");
  const cudaError_t e = ngb::quat_bulk_state(state);
  return e == cudaSuccess ? NGB_OK : cuda_fail(e, "ngb_quat_bulk_state");
}

const char* ngb_last_error(void) { return g_last_error.c_str(); }

const char* ngb_version(void) { return "normgb 0.1.0 (sm_103a)"; }

}  // extern "C"
