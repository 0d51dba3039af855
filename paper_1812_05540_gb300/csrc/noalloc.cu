// Residual of the FP64 Jacobian without any device allocation.
//
// Some callers manage every byte of device memory themselves: a simulator that
// reserves its HBM once at start-up so a long run can never fail on an
// allocation midway, or a process whose memory pool is capped by its host
// framework.  Such callers cannot let a library call cudaMalloc (or any routine
// that allocates) inside their Newton loop.  This file gives them
// r = b - A x and ||r||^2 with the only scratch -- the per-block partial sums of
// ||r||^2 -- held in a fixed, file-scope device array.
//
// The scratch array is shared by every call in the process: calls that overlap
// on the GPU (for example on two streams at once) race on it and must be
// serialised by the caller.  Every slot a call reads is written earlier in the
// same call, so nothing has to be cleared between calls.
#include <mutex>

#include "internal.cuh"

namespace {

constexpr int kThreads = 256;                // one warp per block row, 8 rows per block
constexpr int64_t kMaxPartials = 1 << 19;    // blocks of the row kernels (4 MiB of doubles)
constexpr int kFold = 1024;                  // second-stage partials

// per-block partials of the row kernels, then kFold folded partials
static __device__ __align__(256) double g_resid_scratch[kMaxPartials + kFold];

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct Jac64 {
  int64_t nn, nc;
  const int64_t *uu_rp, *uf_rp, *fu_rp, *ff_rp;
  const int32_t *uu_ci, *uf_ci, *fu_ci, *ff_ci;
  const double *uu_v, *uf_v, *fu_v, *ff_v;
};

// displacement rows: r_u = b_u - (A_uu x_u + A_uf x_f), one warp per node
__global__ void __launch_bounds__(kThreads) k_res_u(Jac64 J, const double* __restrict__ x,
                                                    const double* __restrict__ b, double* __restrict__ r,
                                                    double* __restrict__ part) {
  __shared__ double red[kThreads / 32];
  int64_t I = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  double r2 = 0.0;
  if (I < J.nn) {
    const double* xf = x + 3 * J.nn;
    double a[3] = {0.0, 0.0, 0.0};
    int64_t q0 = J.uu_rp[I], nseg = (J.uu_rp[I + 1] - q0) * 3;
    for (int64_t s = lane; s < nseg; s += 32) {
      int64_t q = q0 + s / 3;
      int row = int(s % 3);
      int64_t c = J.uu_ci[q];
      const double* v = J.uu_v + q * 9 + row * 3;
      a[row] += v[0] * x[3 * c] + v[1] * x[3 * c + 1] + v[2] * x[3 * c + 2];
    }
    int64_t p0 = J.uf_rp[I], mseg = (J.uf_rp[I + 1] - p0) * 3;
    for (int64_t s = lane; s < mseg; s += 32) {
      int64_t q = p0 + s / 3;
      int row = int(s % 3);
      int64_t c = J.uf_ci[q];
      const double* v = J.uf_v + q * 6 + row * 2;
      a[row] += v[0] * xf[2 * c] + v[1] * xf[2 * c + 1];
    }
    a[0] = wsum(a[0]);
    a[1] = wsum(a[1]);
    a[2] = wsum(a[2]);
    if (lane < 3) {
      double v = b[3 * I + lane] - a[lane];
      r[3 * I + lane] = v;
      r2 = v * v;
    }
  }
  r2 = wsum(r2);
  if (lane == 0) red[threadIdx.x >> 5] = r2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += red[w];
    part[blockIdx.x] = s;
  }
}

// flow rows: r_f = b_f - (A_fu x_u + A_ff x_f), one warp per cell
__global__ void __launch_bounds__(kThreads) k_res_f(Jac64 J, const double* __restrict__ x,
                                                    const double* __restrict__ b, double* __restrict__ r,
                                                    double* __restrict__ part) {
  __shared__ double red[kThreads / 32];
  int64_t c = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  double r2 = 0.0;
  if (c < J.nc) {
    const double* xf = x + 3 * J.nn;
    double a[2] = {0.0, 0.0};
    int64_t fq0 = J.fu_rp[c], fseg = (J.fu_rp[c + 1] - fq0) * 2;
    for (int64_t s = lane; s < fseg; s += 32) {
      int64_t q = fq0 + s / 2;
      int row = int(s % 2);
      int64_t j3 = int64_t(J.fu_ci[q]) * 3;
      const double* v = J.fu_v + q * 6 + row * 3;
      a[row] += v[0] * x[j3] + v[1] * x[j3 + 1] + v[2] * x[j3 + 2];
    }
    int64_t gq0 = J.ff_rp[c], gseg = (J.ff_rp[c + 1] - gq0) * 2;
    for (int64_t s = lane; s < gseg; s += 32) {
      int64_t q = gq0 + s / 2;
      int row = int(s % 2);
      int64_t j2 = int64_t(J.ff_ci[q]) * 2;
      const double* v = J.ff_v + q * 4 + row * 2;
      a[row] += v[0] * xf[j2] + v[1] * xf[j2 + 1];
    }
    a[0] = wsum(a[0]);
    a[1] = wsum(a[1]);
    if (lane < 2) {
      int64_t o = 3 * J.nn + 2 * c + lane;
      double v = b[o] - a[lane];
      r[o] = v;
      r2 = v * v;
    }
  }
  r2 = wsum(r2);
  if (lane == 0) red[threadIdx.x >> 5] = r2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += red[w];
    part[blockIdx.x] = s;
  }
}

// fixed-order two-stage sum of the block partials
__global__ void k_res_fold(const double* __restrict__ part, int64_t nparts, double* __restrict__ fold) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= kFold) return;
  double s = 0.0;
  for (int64_t i = t; i < nparts; i += kFold) s += part[i];
  fold[t] = s;
}
__global__ void k_res_total(const double* __restrict__ fold, double* __restrict__ out) {
  __shared__ double s[kThreads];
  double a = 0.0;
  for (int i = threadIdx.x; i < kFold; i += kThreads) a += fold[i];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

// device address of the scratch array, looked up once per device
std::mutex g_mu;
double* g_scratch_ptr[64] = {};

ps_status scratch_for_current_device(double** out) {
  int dev = 0;
  PS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    ps_internal::set_reason("device ordinal %d out of range", dev);
    return PS_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    PS_CUDA(cudaGetSymbolAddress(&p, g_resid_scratch));
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return PS_OK;
}

bool shape_ok(const ps_bsr& B, int64_t rows, int64_t cols, int br, int bc) {
  return B.n_brow == rows && B.n_bcol == cols && B.br == br && B.bc == bc && B.rowptr && B.colind && B.val;
}

}  // namespace

extern "C" ps_status ps_residual_noalloc(const ps_jacobian* jac, const ps_grid* grid, const double* x,
                                         const double* b, double* r, double* rnorm2, void* stream) {
  if (!jac || !grid || !x || !b || !r || !rnorm2) {
    ps_internal::set_reason("ps_residual_noalloc: a null pointer argument");
    return PS_ERR_INVALID;
  }
  if (r == x || r == b) {
    ps_internal::set_reason("ps_residual_noalloc: r must not be the same array as x or b");
    return PS_ERR_INVALID;
  }
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) {
    ps_internal::set_reason("ps_residual_noalloc: grid %dx%dx%d has an empty dimension", grid->nx, grid->ny,
                            grid->nz);
    return PS_ERR_INVALID;
  }
  int64_t nn = int64_t(grid->nx + 1) * (grid->ny + 1) * (grid->nz + 1);
  int64_t nc = int64_t(grid->nx) * grid->ny * grid->nz;
  const struct {
    const ps_bsr* B;
    const char* name;
    int64_t rows, cols;
    int br, bc;
  } blocks[4] = {{&jac->A_uu, "A_uu", nn, nn, 3, 3}, {&jac->A_uf, "A_uf", nn, nc, 3, 2},
                 {&jac->A_fu, "A_fu", nc, nn, 2, 3}, {&jac->A_ff, "A_ff", nc, nc, 2, 2}};
  for (const auto& k : blocks)
    if (!shape_ok(*k.B, k.rows, k.cols, k.br, k.bc)) {
      ps_internal::set_reason("ps_residual_noalloc: %s must be %lld x %lld blocks of %dx%d with non-null arrays",
                              k.name, (long long)k.rows, (long long)k.cols, k.br, k.bc);
      return PS_ERR_INVALID;
    }
  const int64_t rows_per_block = kThreads / 32;
  int64_t gu = (nn + rows_per_block - 1) / rows_per_block;
  int64_t gf = (nc + rows_per_block - 1) / rows_per_block;
  if (gu + gf > kMaxPartials) {
    ps_internal::set_reason("ps_residual_noalloc: %lld node + %lld cell rows need %lld blocks of %lld rows, "
                            "more than the fixed scratch of %lld (ceil(nodes/%lld) + ceil(cells/%lld) must be "
                            "at most %lld)",
                            (long long)nn, (long long)nc, (long long)(gu + gf), (long long)rows_per_block,
                            (long long)kMaxPartials, (long long)rows_per_block, (long long)rows_per_block,
                            (long long)kMaxPartials);
    return PS_ERR_INVALID;
  }
  double* scratch = nullptr;
  PS_TRY(scratch_for_current_device(&scratch));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Jac64 J;
  J.nn = nn; J.nc = nc;
  J.uu_rp = jac->A_uu.rowptr; J.uf_rp = jac->A_uf.rowptr; J.fu_rp = jac->A_fu.rowptr; J.ff_rp = jac->A_ff.rowptr;
  J.uu_ci = jac->A_uu.colind; J.uf_ci = jac->A_uf.colind; J.fu_ci = jac->A_fu.colind; J.ff_ci = jac->A_ff.colind;
  J.uu_v = jac->A_uu.val; J.uf_v = jac->A_uf.val; J.fu_v = jac->A_fu.val; J.ff_v = jac->A_ff.val;
  double* part = scratch;
  double* fold = scratch + kMaxPartials;
  PS_TICK(); k_res_u<<<unsigned(gu), kThreads, 0, st>>>(J, x, b, r, part);
  PS_TICK(); k_res_f<<<unsigned(gf), kThreads, 0, st>>>(J, x, b, r, part + gu);
  PS_TICK(); k_res_fold<<<kFold / kThreads, kThreads, 0, st>>>(part, gu + gf, fold);
  PS_TICK(); k_res_total<<<1, kThreads, 0, st>>>(fold, rnorm2);
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}
