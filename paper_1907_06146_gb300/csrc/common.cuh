// Shared device/host helpers of the NSSG CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>

#include <nvtx3/nvToolsExt.h>

#include "../../include/ssg.h"

namespace ssg {

// ---------------------------------------------------------------------------------------
// Errors and launches
// ---------------------------------------------------------------------------------------
void set_error(const char* fmt, ...);
extern std::atomic<int64_t> g_launches;   // all threads
// Host-side fault injection (ssg_debug_fail_alloc): while positive, counts scratch
// allocations down; the one that brings it to zero fails as an out-of-memory would.
extern std::atomic<int64_t> g_fail_alloc;
inline bool alloc_fault_injected() {
  if (g_fail_alloc.load(std::memory_order_relaxed) <= 0) return false;
  return g_fail_alloc.fetch_sub(1) == 1;
}
extern thread_local int64_t t_launches;    // this host thread
// Records a failure that a kernel reported through its device status word (read back by
// ssg_last_device_status).
void note_device_status(ssg_status s);

struct Fail {
  ssg_status st;
};

#define SSG_CUDA(call)                                                                 \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      ::ssg::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
      throw ::ssg::Fail{e_ == cudaErrorMemoryAllocation ? SSG_ENOMEM : SSG_ECUDA};     \
    }                                                                                  \
  } while (0)

#define SSG_REQUIRE(cond, st, ...)         \
  do {                                     \
    if (!(cond)) {                         \
      ::ssg::set_error(__VA_ARGS__);       \
      throw ::ssg::Fail{st};               \
    }                                      \
  } while (0)

// Launch a kernel, count it, and turn a launch error into an exception.
#define SSG_LAUNCH(kernel, grid, block, smem, stream, ...)                     \
  do {                                                                         \
    kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);                \
    ::ssg::g_launches.fetch_add(1, std::memory_order_relaxed);                 \
    ++::ssg::t_launches;                                                       \
    cudaError_t e_ = cudaGetLastError();                                       \
    if (e_ != cudaSuccess) {                                                   \
      ::ssg::set_error("%s:%d launch of %s: %s", __FILE__, __LINE__, #kernel,  \
                       cudaGetErrorString(e_));                                \
      throw ::ssg::Fail{SSG_ECUDA};                                            \
    }                                                                          \
  } while (0)

// Stream-ordered scratch buffer, released in stream order when it leaves scope.
// Scratch comes from the current device's default stream-ordered pool.  With the pool's
// default release threshold (0) every stream synchronisation hands its free memory back
// to the driver, and the next allocation maps it again; a build synchronises at its stage
// boundaries, so the pool keeps up to an eighth of the device memory between them
// (once per device, at its first scratch allocation).
inline void keep_pool_memory() {
  static std::mutex mu;
  static std::unordered_map<int, bool> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return;
  done[dev] = true;
  cudaMemPool_t pool;
  size_t free_b = 0, total_b = 0;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess ||
      cudaMemGetInfo(&free_b, &total_b) != cudaSuccess)
    return;
  uint64_t keep = (uint64_t)total_b / 8;
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
}

template <typename T>
struct Scratch {
  T* p = nullptr;
  size_t count = 0;
  cudaStream_t s = nullptr;
  Scratch() = default;
  Scratch(size_t n, cudaStream_t st) { alloc(n, st); }
  void alloc(size_t n, cudaStream_t st) {
    release();
    s = st;
    count = n;
    if (n == 0) return;
    if (alloc_fault_injected()) {
      set_error("scratch allocation of %zu bytes failed: injected", n * sizeof(T));
      throw Fail{SSG_ENOMEM};
    }
    keep_pool_memory();
    cudaError_t e = cudaMallocAsync((void**)&p, n * sizeof(T), st);
    if (e != cudaSuccess) {
      p = nullptr;
      set_error("scratch allocation of %zu bytes failed: %s", n * sizeof(T), cudaGetErrorString(e));
      throw Fail{SSG_ENOMEM};
    }
  }
  void release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
  }
  ~Scratch() { release(); }
  Scratch(const Scratch&) = delete;
  Scratch& operator=(const Scratch&) = delete;
  operator T*() const { return p; }
};

// Event pair for stage timing on a stream.
// A named timer also marks its stage as an NVTX range on the calling thread, so that a
// timeline tool shows the build's stages (the events time the device work).
struct StageTimer {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t s;
  const char* name;
  bool open = false;
  explicit StageTimer(cudaStream_t st, const char* nm = nullptr) : s(st), name(nm) {
    SSG_CUDA(cudaEventCreate(&a));
    SSG_CUDA(cudaEventCreate(&b));
  }
  void start() {
    if (name && !open) {
      nvtxRangePushA(name);
      open = true;
    }
    SSG_CUDA(cudaEventRecord(a, s));
  }
  void stop() {
    SSG_CUDA(cudaEventRecord(b, s));
    if (open) {
      nvtxRangePop();
      open = false;
    }
  }
  double ms() {
    float t = 0.f;
    SSG_CUDA(cudaEventSynchronize(b));
    SSG_CUDA(cudaEventElapsedTime(&t, a, b));
    return (double)t;
  }
  ~StageTimer() {
    if (open) nvtxRangePop();  // a stage left by an error
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

inline int num_sms() {
  static const int sms = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }();
  return sms;
}

// Raises a kernel's dynamic shared-memory limit to at least smem (once per kernel and
// size; the kernel's static shared memory counts on top of it, so even 48 KiB needs the
// raise).  Thread-safe: concurrent builds on several host threads share it.
inline void ensure_smem(const void* kernel, size_t smem) {
  static std::mutex mu;
  static std::unordered_map<const void*, size_t> done;
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = done[kernel];
  if (smem <= cur) return;
  SSG_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  cur = smem;
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// cos(alpha) for alpha in degrees.  Angles whose cosine is rational use the exact value
// (so the 60-degree test is exactly cos > 1/2); others use the C library cosine.
double cos_alpha_of(double alpha_deg);

// ---------------------------------------------------------------------------------------
// Keys: (float distance, int32 id) packed into a uint64 that sorts like the pair.
// ---------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint32_t float_order_bits(float f) {
#ifdef __CUDA_ARCH__
  uint32_t b = __float_as_uint(f);
#else
  uint32_t b;
  memcpy(&b, &f, 4);
#endif
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__host__ __device__ __forceinline__ float order_bits_float(uint32_t u) {
  uint32_t b = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float f;
  memcpy(&f, &b, 4);
  return f;
#endif
}
__host__ __device__ __forceinline__ uint64_t make_key(float d, int32_t id) {
  return ((uint64_t)float_order_bits(d) << 32) | (uint32_t)id;
}
__host__ __device__ __forceinline__ float key_dist(uint64_t k) {
  return order_bits_float((uint32_t)(k >> 32));
}
__host__ __device__ __forceinline__ int32_t key_id(uint64_t k) { return (int32_t)(uint32_t)k; }
constexpr uint64_t KEY_NONE = ~0ull;

// ---------------------------------------------------------------------------------------
// Warp helpers
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Bitonic sort (ascending) of m = power-of-two keys in shared memory by one warp.
__device__ __forceinline__ void warp_sort_keys(uint64_t* a, int m) {
  const int lane = lane_id();
  for (int k = 2; k <= m; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < m; i += 32) {
        int p = i ^ j;
        if (p > i) {
          uint64_t x = a[i], y = a[p];
          bool up = (i & k) == 0;
          if ((x > y) == up) {
            a[i] = y;
            a[p] = x;
          }
        }
      }
      __syncwarp();
    }
  }
}

// The same network for larger m (the pools' 256 keys): each compare-exchange step takes
// the m / 2 pairs (i, i + j), i with bit j clear, four per lane at a time -- all loads,
// then the exchanges (the pairs are disjoint) -- at the cost of more registers.
__device__ __forceinline__ void warp_sort_keys_wide(uint64_t* a, int m) {
  const int lane = lane_id(), half = m >> 1;
  for (int k = 2; k <= m; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      const int lj = 31 - __clz(j);
      for (int q0 = 0; q0 < half; q0 += 128) {
        int ii[4];
        bool act[4];
        uint64_t x[4], y[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int q = q0 + u * 32 + lane;
          act[u] = q < half;
          ii[u] = ((q >> lj) << (lj + 1)) | (q & (j - 1));
          if (act[u]) {
            x[u] = a[ii[u]];
            y[u] = a[ii[u] + j];
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (act[u] && (x[u] > y[u]) == ((ii[u] & k) == 0)) {
            a[ii[u]] = y[u];
            a[ii[u] + j] = x[u];
          }
        }
      }
      __syncwarp();
    }
  }
}

// Same for a whole thread block (blockDim.x threads).
__device__ __forceinline__ void block_sort_keys(uint64_t* a, int m) {
  for (int k = 2; k <= m; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        int p = i ^ j;
        if (p > i) {
          uint64_t x = a[i], y = a[p];
          bool up = (i & k) == 0;
          if ((x > y) == up) {
            a[i] = y;
            a[p] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------------------
// Double-precision reference arithmetic on the float32 inputs.  Differences of two
// floats are exact in double; the sums run in coordinate order with separate multiply
// and add (no fused multiply-add), so the value is the one a plain sequential double
// loop gives.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double dist2_f64(const float* __restrict__ a,
                                            const float* __restrict__ b, int d) {
  double s = 0.0;
  for (int t = 0; t < d; ++t) {
    double u = __dsub_rn((double)a[t], (double)b[t]);
    s = __dadd_rn(s, __dmul_rn(u, u));
  }
  return s;
}

__device__ __forceinline__ double centred_dot_f64(const float* __restrict__ a,
                                                  const float* __restrict__ b,
                                                  const float* __restrict__ o, int d) {
  double s = 0.0;
  for (int t = 0; t < d; ++t) {
    double u = __dsub_rn((double)a[t], (double)o[t]);
    double v = __dsub_rn((double)b[t], (double)o[t]);
    s = __dadd_rn(s, __dmul_rn(u, v));
  }
  return s;
}

// cos of the angle j-i-k from the three centred dot products, 0 for a zero-length edge.
__device__ __forceinline__ double cos_from_gram_f64(double gjk, double gjj, double gkk) {
  if (gjj == 0.0 || gkk == 0.0) return 0.0;
  return __ddiv_rn(gjk, __dsqrt_rn(__dmul_rn(gjj, gkk)));
}

// Unit roundoff of float32.
constexpr double U32 = 5.9604644775390625e-08;  // 2^-24

// Dataset facts gathered at ingest.
struct DataInfo {
  int exact;        // all values integers and every squared distance, norm and partial sum
                    // an integer below 2^24 (2 d max|x|^2 <= 2^24 for non-negative data,
                    // 4 d max|x|^2 <= 2^24 otherwise): fp32 sums are exact
  int bf16_exact;   // exact and max|x| <= 256: bf16 holds every value
  int nonneg;       // no negative value
  float max_norm;   // max over rows of the Euclidean norm (fp32)
  float max_abs;
};

// Exactness of fp32 distance arithmetic on integer data (see DataInfo::exact).
inline bool exact_bound(int d, double max_abs, bool nonneg) {
  return (nonneg ? 2.0 : 4.0) * d * max_abs * max_abs <= 16777216.0;
}

}  // namespace ssg
