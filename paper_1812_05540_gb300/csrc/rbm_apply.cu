// V-cycle of the rigid-body-mode smoothed-aggregation hierarchy (see rbm.cuh): Chebyshev smoothing on
// D^{-1} A with the point diagonal, residual, restriction by R = P^T, coarse correction by P, dense FP64
// solve on the coarsest level.  Block rows are taken by LANES threads that stride over the row's blocks and
// combine their partial sums by shuffles.
#include <type_traits>
#include <utility>

#include "rbm.cuh"

namespace ps_internal {
namespace {

// s[a] = sum over the blocks of row i of M_ij x_j (block BR x BC), all lanes of the row group get the sums
template <class T, int BR, int BC, int LANES>
__device__ __forceinline__ void brow(int64_t i, int sub, bool active, const int32_t* __restrict__ rp,
                                     const int32_t* __restrict__ ci, const T* __restrict__ v, const T* __restrict__ x,
                                     T (&s)[BR]) {
#pragma unroll
  for (int a = 0; a < BR; ++a) s[a] = T(0);
  if (active) {
    const int32_t q1 = rp[i + 1];
    for (int32_t q = rp[i] + sub; q < q1; q += LANES) {
      const int64_t j = ci[q];
      T xj[BC];
#pragma unroll
      for (int e = 0; e < BC; ++e) xj[e] = x[j * BC + e];
      const T* blk = v + int64_t(q) * BR * BC;
#pragma unroll
      for (int a = 0; a < BR; ++a)
#pragma unroll
        for (int e = 0; e < BC; ++e) s[a] += __ldg(blk + a * BC + e) * xj[e];
    }
  }
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1)
#pragma unroll
    for (int a = 0; a < BR; ++a) s[a] += __shfl_xor_sync(0xffffffffu, s[a], o);
}

#define BROW_SETUP                                              \
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; \
  const int64_t i = tid / LANES;                                \
  const int sub = int(tid % LANES);                             \
  const bool active = i < n;

// one Chebyshev step: r = D^{-1} (b - A x); d = c1 d + c2 r (first: d = c2 r); xo = x + d
template <class T, int B, int LANES>
__global__ void k_rb_cheb(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const T* __restrict__ v, const T* __restrict__ dg, const T* __restrict__ b,
                          const T* __restrict__ x, T* __restrict__ xo, T* __restrict__ d, double c1, double c2,
                          int first, int store_d) {
  BROW_SETUP
  T s[B];
  brow<T, B, B, LANES>(i, sub, active, rp, ci, v, x, s);
  if (active && sub == 0)
#pragma unroll
    for (int a = 0; a < B; ++a) {
      const int64_t p = i * B + a;
      const T r = (b[p] - s[a]) / dg[p];
      const T dn = first ? T(c2) * r : T(c1) * d[p] + T(c2) * r;
      xo[p] = x[p] + dn;
      if (store_d) d[p] = dn;
    }
}

// first Chebyshev step from x = 0: x = D^{-1} b / theta (d = x when later steps follow)
template <class T>
__global__ void k_rb_first(int64_t N, const T* __restrict__ dg, const T* __restrict__ b, T* __restrict__ x,
                           T* __restrict__ d, double inv_theta) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= N) return;
  const T xv = (b[t] / dg[t]) * T(inv_theta);
  x[t] = xv;
  if (d) d[t] = xv;
}

// r = b - A x
template <class T, int B, int LANES>
__global__ void k_rb_resid(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const T* __restrict__ v, const T* __restrict__ b, const T* __restrict__ x,
                           T* __restrict__ r) {
  BROW_SETUP
  T s[B];
  brow<T, B, B, LANES>(i, sub, active, rp, ci, v, x, s);
  if (active && sub == 0)
#pragma unroll
    for (int a = 0; a < B; ++a) r[i * B + a] = b[i * B + a] - s[a];
}

// y = M x (or y += M x) with BR x BC blocks
template <class T, int BR, int BC, int LANES>
__global__ void k_rb_spmv(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const T* __restrict__ v, const T* __restrict__ x, T* __restrict__ y, int add) {
  BROW_SETUP
  T s[BR];
  brow<T, BR, BC, LANES>(i, sub, active, rp, ci, v, x, s);
  if (active && sub == 0)
#pragma unroll
    for (int a = 0; a < BR; ++a) y[i * BR + a] = add ? y[i * BR + a] + s[a] : s[a];
}

// coarsest: x = inv b, one warp per row, FP64 sums in both precisions
template <class T>
__global__ void k_rb_dense(int64_t N, const double* __restrict__ inv, const T* __restrict__ b, T* __restrict__ x) {
  const int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= N) return;
  const double* row = inv + w * N;
  double s = 0.0;
  for (int64_t j = lane; j < N; j += 32) s += row[j] * double(b[j]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) x[w] = T(s);
}

template <class F>
void with_lanes(int lanes, F&& f) {
  switch (lanes) {
    case 1: f(std::integral_constant<int, 1>()); break;
    case 2: f(std::integral_constant<int, 2>()); break;
    case 4: f(std::integral_constant<int, 4>()); break;
    case 8: f(std::integral_constant<int, 8>()); break;
    case 16: f(std::integral_constant<int, 16>()); break;
    default: f(std::integral_constant<int, 32>()); break;
  }
}

template <class T>
struct LevelV {
  const T *v, *dg, *pv, *rv;
};
template <class T>
LevelV<T> lview(const RbmLevel& L) {
  if constexpr (sizeof(T) == 4) return {L.vf, L.dgf, L.pvf, L.rvf};
  else return {L.v, L.dg, L.pv, L.rv};
}

// Chebyshev coefficients on [lam / ratio, lam]: step k >= 1 uses c1[k], c2[k]; 1/theta starts a sweep
struct Cheb {
  double inv_theta, c1[8], c2[8];
};
Cheb cheb(double lam, const SmoothParams& sp) {
  Cheb c;
  const double lmax = lam, lmin = lam / sp.ratio;
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  c.inv_theta = 1.0 / theta;
  for (int k = 0; k < 8; ++k) c.c1[k] = c.c2[k] = 0.0;
  for (int k = 1; k < 8 && k < sp.degree; ++k) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    c.c1[k] = rn * rho;
    c.c2[k] = 2.0 * rn / delta;
    rho = rn;
  }
  return c;
}

template <class T, int B>
void cheb_step(const RbmLevel& L, const LevelV<T>& V, const T* b, const T* x, T* xo, T* d, double c1, double c2,
               int first, int store_d, cudaStream_t st) {
  with_lanes(L.lanes, [&](auto LN) {
    constexpr int LA = decltype(LN)::value;
    PS_TICK(); k_rb_cheb<T, B, LA><<<grid_for(L.n * LA, 256), 256, 0, st>>>(L.n, L.rp, L.ci, V.v, V.dg, b, x, xo, d, c1,
                                                                            c2, first, store_d);
  });
}

template <class T, int B>
void level(Rbm& H, int l, const SmoothParams& sp, const T* b, T* out, cudaStream_t st) {
  RbmLevel& L = H.L[l];
  const LevelV<T> V = lview<T>(L);
  const int64_t N = L.n * B;
  if (L.coarsest) {
    PS_TICK(); k_rb_dense<T><<<grid_for(N * 32, 256), 256, 0, st>>>(N, L.inv, b, out);
    return;
  }
  T* x = static_cast<T*>(L.x);
  T* t = static_cast<T*>(L.t);
  T* d = static_cast<T*>(L.d);
  T* r = static_cast<T*>(L.r);
  const Cheb c = cheb(L.lam, sp);
  const int deg = sp.degree < 1 ? 1 : (sp.degree > 8 ? 8 : sp.degree);
  // pre-smoothing from zero
  PS_TICK(); k_rb_first<T><<<grid_for(N, 256), 256, 0, st>>>(N, V.dg, b, x, deg > 1 ? d : nullptr, c.inv_theta);
  T* cur = x;
  T* oth = t;
  for (int k = 1; k < deg; ++k) {
    cheb_step<T, B>(L, V, b, cur, oth, d, c.c1[k], c.c2[k], 0, k < deg - 1, st);
    std::swap(cur, oth);
  }
  // residual, restriction, coarse correction
  with_lanes(L.lanes, [&](auto LN) {
    constexpr int LA = decltype(LN)::value;
    PS_TICK(); k_rb_resid<T, B, LA><<<grid_for(L.n * LA, 256), 256, 0, st>>>(L.n, L.rp, L.ci, V.v, b, cur, r);
  });
  RbmLevel& C = H.L[l + 1];
  T* bc = static_cast<T*>(C.bv);
  T* ec = static_cast<T*>(C.e);
  with_lanes(L.rlane, [&](auto LN) {
    constexpr int LA = decltype(LN)::value;
    PS_TICK(); k_rb_spmv<T, kRbmModes, B, LA><<<grid_for(L.nagg * LA, 256), 256, 0, st>>>(L.nagg, L.rrp, L.rci, V.rv, r,
                                                                                         bc, 0);
  });
  level<T, kRbmModes>(H, l + 1, sp, bc, ec, st);
  with_lanes(L.plane, [&](auto LN) {
    constexpr int LA = decltype(LN)::value;
    PS_TICK(); k_rb_spmv<T, B, kRbmModes, LA><<<grid_for(L.n * LA, 256), 256, 0, st>>>(L.n, L.prp, L.pci, V.pv, ec, cur,
                                                                                      1);
  });
  // post-smoothing from the corrected iterate
  for (int k = 0; k < deg; ++k) {
    T* dst = k == deg - 1 ? out : oth;
    if (k == 0) cheb_step<T, B>(L, V, b, cur, dst, d, 0.0, c.inv_theta, 1, deg > 1, st);
    else cheb_step<T, B>(L, V, b, cur, dst, d, c.c1[k], c.c2[k], 0, k < deg - 1, st);
    oth = cur;
    cur = dst;
  }
}

template <class T>
void launch(Rbm& H, const SmoothParams& sp, const T* b, T* x, cudaStream_t st) {
  if (H.L[0].coarsest) {
    const int64_t N = H.L[0].n * 3;
    PS_TICK(); k_rb_dense<T><<<grid_for(N * 32, 256), 256, 0, st>>>(N, H.L[0].inv, b, x);
    return;
  }
  level<T, 3>(H, 0, sp, b, x, st);
}

}  // namespace

template <class T>
ps_status rbm_alloc_work(Arena& ar, Rbm& H, cudaStream_t st) {
  (void)st;
  for (auto& L : H.L) {
    const size_t m = size_t(L.n) * L.b + 1;
    T *x, *t, *r, *d, *b, *e;
    PS_TRY(ar.alloc(&x, m)); PS_TRY(ar.alloc(&t, m)); PS_TRY(ar.alloc(&r, m)); PS_TRY(ar.alloc(&d, m));
    PS_TRY(ar.alloc(&b, m)); PS_TRY(ar.alloc(&e, m));
    L.x = x; L.t = t; L.r = r; L.d = d; L.bv = b; L.e = e;
  }
  return PS_OK;
}

template <class T>
ps_status rbm_vcycle_direct(Rbm& H, const SmoothParams& sp, const T* b, T* x, cudaStream_t st) {
  launch<T>(H, sp, b, x, st);
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

// about thirty short kernels whose arguments depend only on the hierarchy, b and x: captured once into a
// CUDA graph and replayed; streams that cannot be captured run the kernels directly
template <class T>
ps_status rbm_vcycle(Rbm& H, const SmoothParams& sp, const T* b, T* x, cudaStream_t st) {
  if (H.gexec && H.gb == b && H.gx == x && H.gst == st) {
    PS_CUDA(cudaGraphLaunch(H.gexec, st));
    g_launches.fetch_add(H.gnodes, std::memory_order_relaxed);
    return PS_OK;
  }
  if (st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread) {
    rbm_release_graph(H);
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      launch<T>(H, sp, b, x, st);
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(st, &g);
      if (e == cudaSuccess && g) {
        size_t nodes = 0;
        cudaGraphGetNodes(g, nullptr, &nodes);
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e == cudaSuccess) {
          H.gexec = ex;
          H.gb = b;
          H.gx = x;
          H.gst = st;
          H.gnodes = int64_t(nodes);
          PS_CUDA(cudaGraphLaunch(ex, st));
          return PS_OK;
        }
      }
      cudaGetLastError();
    } else {
      cudaGetLastError();
    }
  }
  return rbm_vcycle_direct<T>(H, sp, b, x, st);
}

template ps_status rbm_alloc_work<float>(Arena&, Rbm&, cudaStream_t);
template ps_status rbm_alloc_work<double>(Arena&, Rbm&, cudaStream_t);
template ps_status rbm_vcycle<float>(Rbm&, const SmoothParams&, const float*, float*, cudaStream_t);
template ps_status rbm_vcycle<double>(Rbm&, const SmoothParams&, const double*, double*, cudaStream_t);
template ps_status rbm_vcycle_direct<float>(Rbm&, const SmoothParams&, const float*, float*, cudaStream_t);
template ps_status rbm_vcycle_direct<double>(Rbm&, const SmoothParams&, const double*, double*, cudaStream_t);

}  // namespace ps_internal
