// Allocation, error bookkeeping and deterministic scan / reduction kernels.
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "internal.cuh"

namespace ps_internal {

std::atomic<int64_t> g_launches{0};
std::atomic<int64_t> g_allocs{0};
// per host thread, so that concurrent requests of the server keep their own messages
static thread_local std::string g_last_error;

void set_last_error(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s (%s) at %s:%d: %s", cudaGetErrorName(e), what, file, line, cudaGetErrorString(e));
  g_last_error = buf;
}
const std::string& last_error() { return g_last_error; }

static thread_local std::string g_reason;
void set_reason(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_reason = buf;
}
const std::string& last_reason() { return g_reason; }

// One stream-ordered pool per device; freed blocks stay cached in the pool so
// that repeated setups do not pay for cudaMalloc.
cudaMemPool_t pool_for_current_device() {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    if (cudaMemPoolCreate(&pools[dev], &props) != cudaSuccess) {
      pools[dev] = nullptr;
      return nullptr;
    }
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &thr);
  }
  return pools[dev];
}

ps_status Arena::alloc(void** p, size_t nbytes) {
  *p = nullptr;
  if (nbytes == 0) nbytes = 16;
  nbytes = (nbytes + 255) & ~size_t(255);
  if (budget > 0 && bytes + int64_t(nbytes) > budget) return PS_ERR_BUDGET;
  cudaMemPool_t pool = pool_for_current_device();
  cudaError_t e = pool ? cudaMallocFromPoolAsync(p, nbytes, pool, stream) : cudaMallocAsync(p, nbytes, stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_last_error(e, "cudaMallocAsync", __FILE__, __LINE__);
    return e == cudaErrorMemoryAllocation ? PS_ERR_OOM : PS_ERR_CUDA;
  }
  ptrs.push_back(*p);
  bytes += int64_t(nbytes);
  g_allocs.fetch_add(1, std::memory_order_relaxed);
  return PS_OK;
}

void Arena::release(void* p) {
  for (size_t i = 0; i < ptrs.size(); ++i)
    if (ptrs[i] == p) {
      cudaFreeAsync(p, stream);
      ptrs[i] = ptrs.back();
      ptrs.pop_back();
      return;
    }
}

void Arena::free_all() {
  for (void* p : ptrs) cudaFreeAsync(p, stream);
  ptrs.clear();
  bytes = 0;
}

// ---------------------------------------------------------------------------
// exclusive scan: per-block inclusive scans (1024 elements per block), scan of
// block totals (recursive), add-back.
// ---------------------------------------------------------------------------
template <class O>
__global__ void k_block_scan(const int32_t* __restrict__ in, O* __restrict__ out, O* __restrict__ bsum, int64_t n) {
  __shared__ O s[1024];
  int64_t i = int64_t(blockIdx.x) * 1024 + threadIdx.x;
  O v = i < n ? O(in[i]) : O(0);
  s[threadIdx.x] = v;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    O t = threadIdx.x >= off ? s[threadIdx.x - off] : O(0);
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) out[i] = s[threadIdx.x] - v;  // exclusive
  if (threadIdx.x == 1023) bsum[blockIdx.x] = s[1023];
}

template <class O>
__global__ void k_block_scan_o(const O* __restrict__ in, O* __restrict__ out, O* __restrict__ bsum, int64_t n) {
  __shared__ O s[1024];
  int64_t i = int64_t(blockIdx.x) * 1024 + threadIdx.x;
  O v = i < n ? in[i] : O(0);
  s[threadIdx.x] = v;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    O t = threadIdx.x >= off ? s[threadIdx.x - off] : O(0);
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) out[i] = s[threadIdx.x] - v;
  if (threadIdx.x == 1023) bsum[blockIdx.x] = s[1023];
}

template <class O>
__global__ void k_add_offsets(O* __restrict__ out, const O* __restrict__ boff, int64_t n, O* __restrict__ last,
                              const int32_t* __restrict__ in) {
  int64_t i = int64_t(blockIdx.x) * 1024 + threadIdx.x;
  if (i < n) {
    O v = out[i] + boff[blockIdx.x];
    out[i] = v;
    if (i == n - 1) *last = v + O(in[i]);
  }
}

template <class O>
__global__ void k_add_offsets_o(O* __restrict__ out, const O* __restrict__ boff, int64_t n) {
  int64_t i = int64_t(blockIdx.x) * 1024 + threadIdx.x;
  if (i < n) out[i] += boff[blockIdx.x];
}

// exclusive scan of O-typed values in place into out (n entries), no total
template <class O>
static ps_status scan_o(Arena& ar, const O* in, O* out, int64_t n, cudaStream_t st) {
  int64_t nb = ceil_div(n, 1024);
  O* bs = nullptr;
  PS_TRY(ar.alloc(&bs, nb + 1));
  PS_TICK(); k_block_scan_o<O><<<unsigned(nb), 1024, 0, st>>>(in, out, bs, n);
  if (nb > 1) {
    O* bo = nullptr;
    PS_TRY(ar.alloc(&bo, nb + 1));
    PS_TRY(scan_o<O>(ar, bs, bo, nb, st));
    PS_TICK(); k_add_offsets_o<O><<<unsigned(nb), 1024, 0, st>>>(out, bo, n);
    ar.release(bo);
  }
  ar.release(bs);
  return PS_OK;
}

template <class O>
static ps_status scan_impl(Arena& ar, const int32_t* in, O* out, int64_t n, O* total, cudaStream_t st) {
  if (n == 0) {
    PS_CUDA(cudaMemsetAsync(out, 0, sizeof(O), st));
    if (total) *total = 0;
    return PS_OK;
  }
  int64_t nb = ceil_div(n, 1024);
  O* bs = nullptr;
  O* bo = nullptr;
  PS_TRY(ar.alloc(&bs, nb + 1));
  PS_TRY(ar.alloc(&bo, nb + 1));
  PS_TICK(); k_block_scan<O><<<unsigned(nb), 1024, 0, st>>>(in, out, bs, n);
  PS_TRY(scan_o<O>(ar, bs, bo, nb, st));
  PS_TICK(); k_add_offsets<O><<<unsigned(nb), 1024, 0, st>>>(out, bo, n, out + n, in);
  PS_CUDA(cudaGetLastError());
  ar.release(bs);
  ar.release(bo);
  if (total) {
    PS_CUDA(cudaMemcpyAsync(total, out + n, sizeof(O), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
  }
  return PS_OK;
}

ps_status scan_i32(Arena& ar, const int32_t* in, int32_t* out, int64_t n, int32_t* total, cudaStream_t st) {
  return scan_impl<int32_t>(ar, in, out, n, total, st);
}
ps_status scan_i64(Arena& ar, const int32_t* in, int64_t* out, int64_t n, int64_t* total, cudaStream_t st) {
  return scan_impl<int64_t>(ar, in, out, n, total, st);
}

// ---------------------------------------------------------------------------
// deterministic reductions: 256 threads per block, grid-stride in a fixed
// pattern, fixed tree; then one block over the partials.
// ---------------------------------------------------------------------------
template <int OP>
__device__ __forceinline__ double red_op(double a, double b) {
  return OP == 0 ? a + b : fmax(a, b);
}

template <int OP>
__global__ void k_reduce_partial(const double* __restrict__ x, int64_t n, double* __restrict__ part) {
  __shared__ double s[256];
  double acc = OP == 0 ? 0.0 : -INFINITY;
  for (int64_t i = int64_t(blockIdx.x) * 256 + threadIdx.x; i < n; i += int64_t(gridDim.x) * 256)
    acc = red_op<OP>(acc, x[i]);
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if (threadIdx.x < off) s[threadIdx.x] = red_op<OP>(s[threadIdx.x], s[threadIdx.x + off]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

template <int OP>
static ps_status reduce(Arena& ar, const double* x, int64_t n, double* d_out, cudaStream_t st) {
  const int G = 512;
  double* part = nullptr;
  PS_TRY(ar.alloc(&part, G));
  PS_TICK(); k_reduce_partial<OP><<<G, 256, 0, st>>>(x, n, part);
  PS_TICK(); k_reduce_partial<OP><<<1, 256, 0, st>>>(part, G, d_out);
  PS_CUDA(cudaGetLastError());
  ar.release(part);
  return PS_OK;
}

ps_status sum_f64(Arena& ar, const double* x, int64_t n, double* d_out, cudaStream_t st) {
  return reduce<0>(ar, x, n, d_out, st);
}
ps_status max_f64(Arena& ar, const double* x, int64_t n, double* d_out, cudaStream_t st) {
  return reduce<1>(ar, x, n, d_out, st);
}

__global__ void k_rowptr_i32(const int64_t* __restrict__ in, int32_t* __restrict__ out, int64_t n) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) out[i] = int32_t(in[i]);
}
void rowptr_to_i32(const int64_t* in, int32_t* out, int64_t n, cudaStream_t st) {
  PS_TICK(); k_rowptr_i32<<<grid_for(n, 256), 256, 0, st>>>(in, out, n);
}

}  // namespace ps_internal

extern "C" int64_t ps_launch_count(void) { return ps_internal::g_launches.load(); }
extern "C" int64_t ps_alloc_count(void) { return ps_internal::g_allocs.load(); }

extern "C" ps_status ps_pool_bytes(int64_t* reserved, int64_t* used) {
  if (!reserved || !used) return PS_ERR_INVALID;
  *reserved = 0;
  *used = 0;
  cudaMemPool_t pool = ps_internal::pool_for_current_device();
  if (!pool) return PS_OK;
  uint64_t r = 0, u = 0;
  PS_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &r));
  PS_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &u));
  *reserved = int64_t(r);
  *used = int64_t(u);
  return PS_OK;
}
