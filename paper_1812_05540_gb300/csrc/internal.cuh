// Internal declarations shared by the CUDA translation units of libps.
// Nothing here is part of the public ABI (include/ps.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/ps.h"

#define PS_CUDA(call)                                  \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) {                           \
      ps_internal::set_last_error(e_, #call, __FILE__, __LINE__); \
      return PS_ERR_CUDA;                              \
    }                                                  \
  } while (0)

#define PS_TRY(expr)                 \
  do {                               \
    ps_status s_ = (expr);           \
    if (s_ != PS_OK) return s_;      \
  } while (0)

namespace ps_internal {

// number of kernels launched by this library (for launch accounting)
extern std::atomic<int64_t> g_launches;
// number of device allocations made through Arena::alloc (the library's only device allocation path)
extern std::atomic<int64_t> g_allocs;
#define PS_TICK() ps_internal::g_launches.fetch_add(1, std::memory_order_relaxed)

void set_last_error(cudaError_t e, const char* what, const char* file, int line);
// reason attached to the next PS_ERR_INVALID / PS_ERR_TIMEOUT returned
void set_reason(const char* fmt, ...);
const std::string& last_reason();
const std::string& last_error();

// Device memory owned by one object; every allocation is stream-ordered from a
// library memory pool that keeps freed blocks cached.
struct Arena {
  cudaStream_t stream = 0;
  std::vector<void*> ptrs;
  int64_t bytes = 0;
  int64_t budget = 0;  // 0 = unlimited
  ps_status alloc(void** p, size_t nbytes);
  template <class T>
  ps_status alloc(T** p, size_t count) {
    return alloc(reinterpret_cast<void**>(p), count * sizeof(T));
  }
  void release(void* p);
  void free_all();
};

// the library's stream-ordered memory pool on the current device (null if it could not be created)
cudaMemPool_t pool_for_current_device();

// ---- device utilities (util.cu) ----
// exclusive scan of n int32 counts; out has n+1 entries, out[n] = total (also
// returned in *total when non-null, which synchronises the stream)
ps_status scan_i32(Arena& ar, const int32_t* in, int32_t* out, int64_t n, int32_t* total, cudaStream_t st);
ps_status scan_i64(Arena& ar, const int32_t* in, int64_t* out, int64_t n, int64_t* total, cudaStream_t st);
// deterministic sum (fixed block/tree order) of x[i] over i < n; result on device
ps_status sum_f64(Arena& ar, const double* x, int64_t n, double* d_out, cudaStream_t st);
ps_status max_f64(Arena& ar, const double* x, int64_t n, double* d_out, cudaStream_t st);
// copy int64 row pointers to int32
void rowptr_to_i32(const int64_t* in, int32_t* out, int64_t n, cudaStream_t st);

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline unsigned grid_for(int64_t n, int block) {
  int64_t g = ceil_div(n, block);
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace ps_internal
