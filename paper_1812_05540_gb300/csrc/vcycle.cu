// V-cycle apply of the smoothed-aggregation hierarchy (M_uu^{-1} of §5.2 and
// M_pp^{-1} of §5.3): Chebyshev or l1-Jacobi smoothing, residual, restriction
// by R = P^T, coarse correction by P, dense coarsest solve.  Vectors hold nc
// interleaved components (node-major x,y,z for the SDC mechanics operator).
#include <cuda_bf16.h>

#include <cstring>
#include <type_traits>
#include <vector>
#include <utility>

#include "amg.cuh"
#include "gridsync.cuh"

#include <cooperative_groups.h>
#include <map>
#include <mutex>
#include <tuple>

namespace ps_internal {
namespace {

// matrix values as stored (FP64, FP32, or BF16 for the prolongator variant) to the apply precision
template <class T>
__device__ __forceinline__ T val(const T* p) { return __ldg(p); }
template <class T>
__device__ __forceinline__ T val_as(const __nv_bfloat16* p) { return T(__bfloat162float(*p)); }

// a * b + c with one rounding, written out so that every kernel forms the Chebyshev update the same way
// (an implicit contraction of a sum of two products may fuse either product)
__device__ __forceinline__ float mad(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double mad(double a, double b, double c) { return __fma_rn(a, b, c); }

// Programmatic dependent launch.  The V-cycle's kernels after its first are launched with programmatic
// stream serialisation (vl below), so a kernel's CTAs may be scheduled while its predecessor drains.  Every
// such kernel first waits at griddepcontrol.wait, which returns once the predecessor grid has completed and
// its memory operations are visible, and only then reads or writes anything; it then lets its own successor
// launch.  A kernel launched without the attribute passes both instructions at once.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <class T, int NC, int LANES>
struct Row {
  // s[c] = sum_q v[q*NC+c] * x[j*NC+c] over one CSR row with LANES lanes; all lanes get the sum
  template <class XF, class TV>
  __device__ __forceinline__ static void dot(bool active, int32_t q0, int32_t q1, const int32_t* __restrict__ ci,
                                             const TV* __restrict__ v, XF xf, int sub, T (&s)[NC]) {
#pragma unroll
    for (int c = 0; c < NC; ++c) s[c] = T(0);
    if (active)
      for (int32_t q = q0 + sub; q < q1; q += LANES) {
        int32_t j = __ldg(ci + q);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          T a;
          if constexpr (sizeof(TV) == 2) a = val_as<T>(v + int64_t(q) * NC + c);
          else a = T(__ldg(v + int64_t(q) * NC + c));
          s[c] += a * xf(j, c);
        }
      }
#pragma unroll
    for (int off = LANES / 2; off > 0; off >>= 1)
#pragma unroll
      for (int c = 0; c < NC; ++c) s[c] += __shfl_xor_sync(0xffffffffu, s[c], off);
  }
};

// Rows of a level operator in CSR form, LANES threads per row.
template <class T, int NC, int LANES>
struct CsrRows {
  static constexpr int kLanes = LANES;
  const int32_t *rp, *ci;
  const T* v;
  template <class XF>
  __device__ __forceinline__ void dot(int64_t i, int sub, bool active, XF xf, T (&s)[NC]) const {
    int32_t q0 = active ? rp[i] : 0, q1 = active ? rp[i + 1] : 0;
    Row<T, NC, LANES>::dot(active, q0, q1, ci, v, xf, sub, s);
  }
};

// Stencil slot q -> (dx, dy, dz): the full 27-point box (x fastest) or the 7-point star
// (z-1, y-1, x-1, self, x+1, y+1, z+1).
template <int NS>
__device__ __forceinline__ void slot_offset(int q, int& dx, int& dy, int& dz) {
  if constexpr (NS == 27) {
    dx = q % 3 - 1; dy = (q / 3) % 3 - 1; dz = q / 9 - 1;
  } else {
    dx = q == 2 ? -1 : (q == 4 ? 1 : 0);
    dy = q == 1 ? -1 : (q == 5 ? 1 : 0);
    dz = q == 0 ? -1 : (q == 6 ? 1 : 0);
  }
}

// Rows of a level operator on the structured grid (gx x gy x gz rows, x fastest): values by
// stencil slot, [slot][component][row], one thread per row, no column indices.
template <class T, int NC, int NS>
struct StencilRows {
  static constexpr int kLanes = 1;
  int gx, gy, gz;
  int64_t n;
  const T* v;
  template <class XF>
  __device__ __forceinline__ void dot(int64_t i, int, bool active, XF xf, T (&s)[NC]) const {
#pragma unroll
    for (int c = 0; c < NC; ++c) s[c] = T(0);
    if (!active) return;
    // the grid has fewer than 2^31 rows (amg_stencil checks it), so coordinates fit in int
    const int gxy = gx * gy, ii = int(i);
    const int iz = ii / gxy, rem = ii - iz * gxy;
    const int iy = rem / gx, ix = rem - iy * gx;
    const bool inx[3] = {ix > 0, true, ix < gx - 1}, iny[3] = {iy > 0, true, iy < gy - 1},
               inz[3] = {iz > 0, true, iz < gz - 1};
    // values of slots that leave the grid are stored as zero: such a slot reads x at the row
    // itself, so every slot is loaded without a branch and adds exactly zero
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      int dx, dy, dz;
      slot_offset<NS>(q, dx, dy, dz);
      const bool in = inx[dx + 1] && iny[dy + 1] && inz[dz + 1];
      const int64_t j = i + (in ? dx + gx * dy + gxy * dz : 0);
#pragma unroll
      for (int c = 0; c < NC; ++c) s[c] += __ldg(v + (int64_t(q) * NC + c) * n + i) * xf(j, c);
    }
  }
};

#define ROWS_SETUP                                                \
  pdl_enter();                                                    \
  int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;  \
  int64_t i = tid / A::kLanes;                                    \
  int sub = int(tid % A::kLanes);                                 \
  bool active = i < n;

// one Chebyshev step from a nonzero x: r = D^{-1}(b - A x); d = c1 d + c2 r; xo = x + d
// (first == true: d = r / theta, i.e. c1 = 0, c2 = 1/theta); d is stored when store_d (a later step reads it)
template <class T, int NC, class A>
__global__ void k_cheb_step(A a, int64_t n, const T* __restrict__ dg, const T* __restrict__ b,
                            const T* __restrict__ x, T* __restrict__ xo, T* __restrict__ d, double3 c1, double3 c2,
                            int first, int store_d) {
  ROWS_SETUP
  auto xf = [&](int64_t j, int c) { return x[j * NC + c]; };
  T s[NC];
  a.dot(i, sub, active, xf, s);
  if (active && sub == 0) {
    const double a1[3] = {c1.x, c1.y, c1.z}, a2[3] = {c2.x, c2.y, c2.z};
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      T r = (b[i * NC + c] - s[c]) / dg[i * NC + c];
      T dn = first ? T(a2[c]) * r : mad(T(a1[c]), d[i * NC + c], T(a2[c]) * r);
      xo[i * NC + c] = x[i * NC + c] + dn;
      if (store_d) d[i * NC + c] = dn;
    }
  }
}

// The first two Chebyshev steps from x = 0 in one pass.  The first step's iterate x1 = D^{-1} b / theta is
// formed wherever the row touches it (dsi = D^{-1} / theta), so it is neither stored nor read back; then
// r = D^{-1}(b - A x1), d = c1 x1 + c2 r (the first direction is x1 itself), xo = x1 + d, and d is stored
// when later steps need it.
template <class T, int NC, class A>
__global__ void k_cheb_zero2(A a, int64_t n, const T* __restrict__ dg, const T* __restrict__ dsi,
                             const T* __restrict__ b, T* __restrict__ xo, T* __restrict__ d, double3 c1, double3 c2) {
  ROWS_SETUP
  auto xf = [&](int64_t j, int c) { return b[j * NC + c] * dsi[j * NC + c]; };
  T s[NC];
  a.dot(i, sub, active, xf, s);
  if (active && sub == 0) {
    const double a1[3] = {c1.x, c1.y, c1.z}, a2[3] = {c2.x, c2.y, c2.z};
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const T x1 = b[i * NC + c] * dsi[i * NC + c];
      const T r = (b[i * NC + c] - s[c]) / dg[i * NC + c];
      const T dn = mad(T(a1[c]), x1, T(a2[c]) * r);
      xo[i * NC + c] = x1 + dn;
      if (d) d[i * NC + c] = dn;
    }
  }
}

// dsi = D^{-1} / theta per row and component
template <class T, int NC>
__global__ void k_dsi(int64_t n, const T* __restrict__ dg, T* __restrict__ dsi, double3 inv_theta) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const double it[3] = {inv_theta.x, inv_theta.y, inv_theta.z};
  if (t < n * NC) dsi[t] = T(it[t % NC]) / dg[t];
}

// l1-Jacobi: xo = x + (b - A x) / dl1
template <class T, int NC, class A>
__global__ void k_l1_step(A a, int64_t n, const T* __restrict__ dl1, const T* __restrict__ b,
                          const T* __restrict__ x, T* __restrict__ xo) {
  ROWS_SETUP
  auto xf = [&](int64_t j, int c) { return x[j * NC + c]; };
  T s[NC];
  a.dot(i, sub, active, xf, s);
  if (active && sub == 0)
#pragma unroll
    for (int c = 0; c < NC; ++c) xo[i * NC + c] = x[i * NC + c] + (b[i * NC + c] - s[c]) / dl1[i * NC + c];
}

template <class T, int NC>
__global__ void k_l1_first(int64_t n, const T* __restrict__ dl1, const T* __restrict__ b, T* __restrict__ x) {
  pdl_enter();
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < n * NC) x[t] = b[t] / dl1[t];
}

// first Chebyshev step from x = 0: x = D^{-1} b / theta (and d = x when d != nullptr)
template <class T, int NC>
__global__ void k_cheb_first1(int64_t n, const T* __restrict__ dg, const T* __restrict__ b, T* __restrict__ x,
                              T* __restrict__ d, double3 inv_theta) {
  pdl_enter();
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const double it[3] = {inv_theta.x, inv_theta.y, inv_theta.z};
  if (t < n * NC) {
    T v = (b[t] / dg[t]) * T(it[t % NC]);
    x[t] = v;
    if (d) d[t] = v;
  }
}

// r = b - A x
template <class T, int NC, class A>
__global__ void k_resid(A a, int64_t n, const T* __restrict__ b, const T* __restrict__ x, T* __restrict__ r) {
  ROWS_SETUP
  auto xf = [&](int64_t j, int c) { return x[j * NC + c]; };
  T s[NC];
  a.dot(i, sub, active, xf, s);
  if (active && sub == 0)
#pragma unroll
    for (int c = 0; c < NC; ++c) r[i * NC + c] = b[i * NC + c] - s[c];
}

#define ROW_SETUP                                                        \
  pdl_enter();                                                           \
  int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;         \
  int64_t i = tid / LANES;                                               \
  int sub = int(tid % LANES);                                            \
  bool active = i < n;                                                   \
  int32_t q0 = active ? rp[i] : 0, q1 = active ? rp[i + 1] : 0;

// y = M x (restriction with R, or y += P x when add); M's values stored as TV
template <class T, int NC, int LANES, class TV>
__global__ void k_spmv(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                       const TV* __restrict__ v, const T* __restrict__ x, T* __restrict__ y, int add) {
  ROW_SETUP
  auto xf = [&](int32_t j, int c) { return x[int64_t(j) * NC + c]; };
  T s[NC];
  Row<T, NC, LANES>::dot(active, q0, q1, ci, v, xf, sub, s);
  if (active && sub == 0)
#pragma unroll
    for (int c = 0; c < NC; ++c) y[i * NC + c] = add ? y[i * NC + c] + s[c] : s[c];
}

// coarsest: x = inv_c b_c per component, one warp per row; the inverse and the sums stay FP64
// in both precisions (the coarsest solve is one of the FP64 parts of the mixed mode)
template <class T, int NC>
__global__ void k_dense_solve(int64_t n, const double* __restrict__ inv, const T* __restrict__ b, T* __restrict__ x) {
  pdl_enter();
  int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= n * NC) return;
  int c = int(w / n);
  int64_t i = w % n;
  const double* row = inv + (int64_t(c) * n + i) * n;
  double s = 0.0;
  for (int64_t j = lane; j < n; j += 32) s += row[j] * double(b[j * NC + c]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) x[i * NC + c] = T(s);
}

// ---------------------------------------------------------------------------
// The coarse end of the V-cycle in one launch.  Below the finest level every level is small and its kernels
// are bound by launch and drain latency, not bandwidth: about five microseconds per kernel on levels whose
// data moves in one.  k_vcycle_tail runs the steps of levels tail_l0 .. coarsest in order (down: smoothing
// pair, residual, restriction; the dense coarsest solve; up: prolongation, two post steps), each as a
// grid-stride loop over the level's rows, with a barrier between steps: a bounded grid barrier in a
// cooperative launch over the whole GPU (CL = false, from level 1), or the hardware barrier of one
// thread-block cluster (CL = true, from the first level of at most kClusterTailRows rows, where 16 SMs
// stream a level's operator from L2 as fast as the whole GPU and a barrier costs a fraction of a launch).
// Vectors written inside the launch are read through L2 (ld.global.cg).  Each step is the same arithmetic as
// its own kernel (same row split into lanes, same order of sums), so the result is bit-identical to the
// kernel-per-step path.  Used for Chebyshev of degree 2 with FP32 or FP64 transfer operators; other schedules
// keep the kernel-per-step path.
// ---------------------------------------------------------------------------
constexpr int64_t kClusterTailRows = 1024;
constexpr int kTailCluster = 16;
template <class T>
struct TailLevel {
  int64_t n, nnext;
  int lanes, plane, rlane, coarsest;
  const int32_t *rp, *ci, *prp, *pci, *rrp, *rci;
  const T *v, *dg, *dsi, *pv, *rv;
  const double* inv;
  T *x, *t, *r, *d, *b, *e;
  double3 c1, c2, pc2;  // Chebyshev step 1 coefficients, and 1/theta for the first post step
};

// rows [0, n) in groups of LANES lanes; a warp's groups advance together, since the row sums shuffle
// across the whole warp
template <int LANES, class F>
__device__ __forceinline__ void tail_rows(int64_t n, F&& f) {
  constexpr int G = 32 / LANES;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t w = warp; w * G < n; w += nwarps) {
    const int64_t i = w * G + lane / LANES;
    f(i, lane % LANES, i < n);
  }
}

template <class F>
__device__ __forceinline__ void by_lanes(int lanes, F&& f) {
  switch (lanes) {
    case 1: f(std::integral_constant<int, 1>()); break;
    case 2: f(std::integral_constant<int, 2>()); break;
    case 4: f(std::integral_constant<int, 4>()); break;
    case 8: f(std::integral_constant<int, 8>()); break;
    case 16: f(std::integral_constant<int, 16>()); break;
    default: f(std::integral_constant<int, 32>()); break;
  }
}

template <class T, int NC, bool CL>
__global__ void __launch_bounds__(256) k_vcycle_tail(const TailLevel<T>* __restrict__ lv, int nl,
                                                     unsigned long long* bar, int64_t limit, int* err) {
  const unsigned long long G = gridDim.x;
  unsigned long long phase = 0;
  auto sync = [&]() -> bool {
    if constexpr (CL) {
      cooperative_groups::this_cluster().sync();
      return true;
    } else {
      ++phase;
      return grid_barrier(bar, phase * G, limit, err);
    }
  };
  // down the levels
  for (int k = 0; k + 1 < nl; ++k) {
    const TailLevel<T> L = lv[k];
    const double a1[3] = {L.c1.x, L.c1.y, L.c1.z}, a2[3] = {L.c2.x, L.c2.y, L.c2.z};
    // Chebyshev steps 0 and 1 from x = 0 in one pass (as k_cheb_zero2, degree 2: d is not kept)
    by_lanes(L.lanes, [&](auto LN) {
      constexpr int LANES = decltype(LN)::value;
      tail_rows<LANES>(L.n, [&](int64_t i, int sub, bool active) {
        auto xf = [&](int64_t j, int c) { return __ldcg(L.b + j * NC + c) * L.dsi[j * NC + c]; };
        T s[NC];
        CsrRows<T, NC, LANES>{L.rp, L.ci, L.v}.dot(i, sub, active, xf, s);
        if (active && sub == 0)
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            const T x1 = __ldcg(L.b + i * NC + c) * L.dsi[i * NC + c];
            const T r = (__ldcg(L.b + i * NC + c) - s[c]) / L.dg[i * NC + c];
            const T dn = mad(T(a1[c]), x1, T(a2[c]) * r);
            L.x[i * NC + c] = x1 + dn;
          }
      });
    });
    if (!sync()) return;
    // r = b - A x (as k_resid)
    by_lanes(L.lanes, [&](auto LN) {
      constexpr int LANES = decltype(LN)::value;
      tail_rows<LANES>(L.n, [&](int64_t i, int sub, bool active) {
        auto xf = [&](int64_t j, int c) { return __ldcg(L.x + j * NC + c); };
        T s[NC];
        CsrRows<T, NC, LANES>{L.rp, L.ci, L.v}.dot(i, sub, active, xf, s);
        if (active && sub == 0)
#pragma unroll
          for (int c = 0; c < NC; ++c) L.r[i * NC + c] = __ldcg(L.b + i * NC + c) - s[c];
      });
    });
    if (!sync()) return;
    // b_coarse = R r (as k_spmv)
    const TailLevel<T>& C = lv[k + 1];
    T* bc = C.b;
    by_lanes(L.rlane, [&](auto LN) {
      constexpr int LANES = decltype(LN)::value;
      tail_rows<LANES>(L.nnext, [&](int64_t i, int sub, bool active) {
        auto xf = [&](int32_t j, int c) { return __ldcg(L.r + int64_t(j) * NC + c); };
        T s[NC];
        const int32_t q0 = active ? L.rrp[i] : 0, q1 = active ? L.rrp[i + 1] : 0;
        Row<T, NC, LANES>::dot(active, q0, q1, L.rci, L.rv, xf, sub, s);
        if (active && sub == 0)
#pragma unroll
          for (int c = 0; c < NC; ++c) bc[i * NC + c] = s[c];
      });
    });
    if (!sync()) return;
  }
  // coarsest: e = inv b per component, one warp per row (as k_dense_solve)
  {
    const TailLevel<T> L = lv[nl - 1];
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t w = warp; w < L.n * NC; w += nwarps) {
      const int c = int(w / L.n);
      const int64_t i = w % L.n;
      const double* row = L.inv + (int64_t(c) * L.n + i) * L.n;
      double s = 0.0;
      for (int64_t j = lane; j < L.n; j += 32) s += row[j] * double(__ldcg(L.b + j * NC + c));
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) L.e[i * NC + c] = T(s);
    }
    if (!sync()) return;
  }
  // up the levels
  for (int k = nl - 2; k >= 0; --k) {
    const TailLevel<T> L = lv[k];
    const T* ec = lv[k + 1].e;
    const double a1[3] = {L.c1.x, L.c1.y, L.c1.z}, a2[3] = {L.c2.x, L.c2.y, L.c2.z},
                 p2[3] = {L.pc2.x, L.pc2.y, L.pc2.z};
    // x += P e_coarse (as k_spmv with add)
    by_lanes(L.plane, [&](auto LN) {
      constexpr int LANES = decltype(LN)::value;
      tail_rows<LANES>(L.n, [&](int64_t i, int sub, bool active) {
        auto xf = [&](int32_t j, int c) { return __ldcg(ec + int64_t(j) * NC + c); };
        T s[NC];
        const int32_t q0 = active ? L.prp[i] : 0, q1 = active ? L.prp[i + 1] : 0;
        Row<T, NC, LANES>::dot(active, q0, q1, L.pci, L.pv, xf, sub, s);
        if (active && sub == 0)
#pragma unroll
          for (int c = 0; c < NC; ++c) L.x[i * NC + c] = __ldcg(L.x + i * NC + c) + s[c];
      });
    });
    if (!sync()) return;
    // first post step: t = x + d, d = D^{-1}(b - A x) / theta (as k_cheb_step, first)
    by_lanes(L.lanes, [&](auto LN) {
      constexpr int LANES = decltype(LN)::value;
      tail_rows<LANES>(L.n, [&](int64_t i, int sub, bool active) {
        auto xf = [&](int64_t j, int c) { return __ldcg(L.x + j * NC + c); };
        T s[NC];
        CsrRows<T, NC, LANES>{L.rp, L.ci, L.v}.dot(i, sub, active, xf, s);
        if (active && sub == 0)
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            const T r = (__ldcg(L.b + i * NC + c) - s[c]) / L.dg[i * NC + c];
            const T dn = T(p2[c]) * r;
            L.t[i * NC + c] = __ldcg(L.x + i * NC + c) + dn;
            L.d[i * NC + c] = dn;
          }
      });
    });
    if (!sync()) return;
    // second post step: e = t + c1 d + c2 D^{-1}(b - A t) (as k_cheb_step)
    by_lanes(L.lanes, [&](auto LN) {
      constexpr int LANES = decltype(LN)::value;
      tail_rows<LANES>(L.n, [&](int64_t i, int sub, bool active) {
        auto xf = [&](int64_t j, int c) { return __ldcg(L.t + j * NC + c); };
        T s[NC];
        CsrRows<T, NC, LANES>{L.rp, L.ci, L.v}.dot(i, sub, active, xf, s);
        if (active && sub == 0)
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            const T r = (__ldcg(L.b + i * NC + c) - s[c]) / L.dg[i * NC + c];
            const T dn = mad(T(a1[c]), __ldcg(L.d + i * NC + c), T(a2[c]) * r);
            L.e[i * NC + c] = __ldcg(L.t + i * NC + c) + dn;
          }
      });
    });
    if (k > 0 && !sync()) return;
  }
  if constexpr (CL) cooperative_groups::this_cluster().sync();  // no CTA leaves while another may still run
}

template <class T>
struct LevelT {
  const T *v, *dg, *dl1, *pv, *rv;
  const double* inv;
  const T* sv;  // stencil-slot values (level 0 on the structured grid) or null
};
template <class T>
LevelT<T> view(const AmgLevel& L) {
  LevelT<T> o;
  if constexpr (sizeof(T) == 4) {
    o.v = L.vf; o.dg = L.dgf; o.dl1 = L.dl1f; o.pv = L.pvf; o.rv = L.rvf; o.inv = L.inv; o.sv = L.sv_f;
  } else {
    o.v = L.v; o.dg = L.dg; o.dl1 = L.dl1; o.pv = L.pv; o.rv = L.rv; o.inv = L.inv; o.sv = L.sv_d;
  }
  return o;
}

// calls f(rows) with the level's row accessor: stencil slots when the level has them, else CSR
// with the level's lane count
template <class T, int NC, class F>
void with_rows(const AmgLevel& L, const LevelT<T>& V, F&& f) {
  if (V.sv) {
    if constexpr (NC == 3) {
      if (L.sns == 27) { f(StencilRows<T, 3, 27>{L.sgx, L.sgy, L.sgz, L.n, V.sv}); return; }
    } else {
      if (L.sns == 7) { f(StencilRows<T, 1, 7>{L.sgx, L.sgy, L.sgz, L.n, V.sv}); return; }
    }
  }
  switch (L.lanes) {
    case 1: f(CsrRows<T, NC, 1>{L.rp, L.ci, V.v}); break;
    case 2: f(CsrRows<T, NC, 2>{L.rp, L.ci, V.v}); break;
    case 4: f(CsrRows<T, NC, 4>{L.rp, L.ci, V.v}); break;
    case 8: f(CsrRows<T, NC, 8>{L.rp, L.ci, V.v}); break;
    case 16: f(CsrRows<T, NC, 16>{L.rp, L.ci, V.v}); break;
    default: f(CsrRows<T, NC, 32>{L.rp, L.ci, V.v}); break;
  }
}

// Launch state of the V-cycle being enqueued by this host thread: 0 plain launches; 1 the next launch is the
// V-cycle's first (plain), later ones programmatic; 2 programmatic launches.
thread_local int t_pdl = 0;

// launch of a V-cycle kernel with 256 threads per CTA, programmatic when t_pdl says so
template <class... KA, class... Args>
void vl(void (*k)(KA...), unsigned grid, cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = t_pdl == 2 ? 1 : 0;
  if (t_pdl == 1) t_pdl = 2;
  cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

template <class A>
inline unsigned rows_grid(int64_t n) {
  return grid_for(n * A::kLanes, 256);
}

struct ChebCoef {
  double3 inv_theta;
  double3 c1[8], c2[8];  // step k (k = 1..degree-1)
  double3 post_c2;       // 1/theta for the first post step
};

inline ChebCoef cheb_coef(const AmgLevel& L, int nc, const SmoothParams& sp) {
  ChebCoef cc;
  double it[3] = {0, 0, 0}, a1[8][3] = {{0}}, a2[8][3] = {{0}};
  for (int c = 0; c < nc; ++c) {
    double lmax = L.lam[c], lmin = lmax / sp.ratio;
    double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
    double sigma = theta / delta, rho = 1.0 / sigma;
    it[c] = 1.0 / theta;
    for (int k = 1; k < sp.degree && k < 8; ++k) {
      double rn = 1.0 / (2.0 * sigma - rho);
      a1[k][c] = rn * rho;
      a2[k][c] = 2.0 * rn / delta;
      rho = rn;
    }
  }
  cc.inv_theta = make_double3(it[0], it[1], it[2]);
  cc.post_c2 = cc.inv_theta;
  for (int k = 0; k < 8; ++k) {
    cc.c1[k] = make_double3(a1[k][0], a1[k][1], a1[k][2]);
    cc.c2[k] = make_double3(a2[k][0], a2[k][1], a2[k][2]);
  }
  return cc;
}

// Smoothing from x = 0; returns the buffer (x or t) that holds the result.
template <class T, int NC>
T* smooth_zero(const AmgLevel& L, const LevelT<T>& V, const SmoothParams& sp, const T* b, T* x, T* t, T* d,
               cudaStream_t st) {
  int64_t n = L.n;
  T* cur = x;
  T* other = t;
  if (sp.kind == PS_SMOOTH_CHEBYSHEV) {
    ChebCoef cc = cheb_coef(L, NC, sp);
    int deg = sp.degree < 1 ? 1 : (sp.degree > 8 ? 8 : sp.degree);
    int k0 = 1;
    // the fused pair reads b and D^{-1}/theta at every stencil neighbour instead of one iterate; on the
    // 27-point three-component level that doubles the gathered bytes, so there the first step stays apart
    if (deg > 1 && L.dsi && !(NC == 3 && V.sv)) {
      // steps 0 and 1 in one pass
      with_rows<T, NC>(L, V, [&](auto a) {
        using A = decltype(a);
        PS_TICK(); vl(k_cheb_zero2<T, NC, A>, rows_grid<A>(n), st, a, n, V.dg, static_cast<const T*>(L.dsi),
                                                                            b, x, deg > 2 ? d : nullptr, cc.c1[1],
                                                                            cc.c2[1]);
      });
      k0 = 2;
    } else {
      PS_TICK(); vl(k_cheb_first1<T, NC>, grid_for(n * NC, 256), st, n, V.dg, b, x, deg > 1 ? d : nullptr,
                                                                          cc.inv_theta);
    }
    for (int k = k0; k < deg; ++k) {
      with_rows<T, NC>(L, V, [&](auto a) {
        using A = decltype(a);
        PS_TICK(); vl(k_cheb_step<T, NC, A>, rows_grid<A>(n), st, a, n, V.dg, b, cur, other,
                                                                           d, cc.c1[k], cc.c2[k], 0,
                                                                           k < deg - 1);
      });
      std::swap(cur, other);
    }
  } else {
    PS_TICK(); vl(k_l1_first<T, NC>, grid_for(n * NC, 256), st, n, V.dl1, b, x);
    for (int k = 1; k < sp.pre; ++k) {
      with_rows<T, NC>(L, V, [&](auto a) {
        using A = decltype(a);
        PS_TICK(); vl(k_l1_step<T, NC, A>, rows_grid<A>(n), st, a, n, V.dl1, b, cur, other);
      });
      std::swap(cur, other);
    }
  }
  return cur;
}

// Smoothing from the iterate in cur (other is free scratch); result written to out.
template <class T, int NC>
void smooth_post(const AmgLevel& L, const LevelT<T>& V, const SmoothParams& sp, const T* b, T* cur, T* other,
                 T* d, T* out, cudaStream_t st) {
  int64_t n = L.n;
  if (sp.kind == PS_SMOOTH_CHEBYSHEV) {
    ChebCoef cc = cheb_coef(L, NC, sp);
    int deg = sp.degree < 1 ? 1 : (sp.degree > 8 ? 8 : sp.degree);
    for (int k = 0; k < deg; ++k) {
      T* dst = k == deg - 1 ? out : other;
      with_rows<T, NC>(L, V, [&](auto a) {
        using A = decltype(a);
        if (k == 0) {
          PS_TICK(); vl(k_cheb_step<T, NC, A>, rows_grid<A>(n), st, a, n, V.dg, b, cur, dst, d, cc.c1[0],
                                                                             cc.post_c2, 1, deg > 1);
        } else {
          PS_TICK(); vl(k_cheb_step<T, NC, A>, rows_grid<A>(n), st, a, n, V.dg, b, cur, dst, d, cc.c1[k],
                                                                             cc.c2[k], 0, k < deg - 1);
        }
      });
      other = cur;
      cur = dst;
    }
  } else {
    int sweeps = sp.post < 1 ? 1 : sp.post;
    for (int k = 0; k < sweeps; ++k) {
      T* dst = k == sweeps - 1 ? out : other;
      with_rows<T, NC>(L, V, [&](auto a) {
        using A = decltype(a);
        PS_TICK(); vl(k_l1_step<T, NC, A>, rows_grid<A>(n), st, a, n, V.dl1, b, cur, dst);
      });
      other = cur;
      cur = dst;
    }
  }
}

template <class T, int NC, class TV>
void spmv_lanes(int lanes, int64_t n, const int32_t* rp, const int32_t* ci, const TV* v, const T* x, T* y, int add,
                cudaStream_t st) {
  switch (lanes) {
    case 1: PS_TICK(); vl(k_spmv<T, NC, 1, TV>, grid_for(n, 256), st, n, rp, ci, v, x, y, add); break;
    case 2: PS_TICK(); vl(k_spmv<T, NC, 2, TV>, grid_for(n * 2, 256), st, n, rp, ci, v, x, y, add); break;
    case 4: PS_TICK(); vl(k_spmv<T, NC, 4, TV>, grid_for(n * 4, 256), st, n, rp, ci, v, x, y, add); break;
    case 8: PS_TICK(); vl(k_spmv<T, NC, 8, TV>, grid_for(n * 8, 256), st, n, rp, ci, v, x, y, add); break;
    case 16: PS_TICK(); vl(k_spmv<T, NC, 16, TV>, grid_for(n * 16, 256), st, n, rp, ci, v, x, y, add); break;
    default: PS_TICK(); vl(k_spmv<T, NC, 32, TV>, grid_for(n * 32, 256), st, n, rp, ci, v, x, y, add); break;
  }
}

// the tail levels in one launch (one thread-block cluster, or a cooperative launch over the GPU); false when
// the launch was not possible (the caller then runs the kernel-per-step path)
template <class T, int NC>
bool launch_tail(Amg& H, cudaStream_t st) {
  const TailLevel<T>* lv = static_cast<const TailLevel<T>*>(H.tail);
  int nl = H.tail_levels;
  unsigned long long* bar = H.tail_bar;
  int64_t limit = H.spin_limit;
  int* err = H.err;
  if (H.tail_mode == 2) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(H.tail_grid));
    cfg.blockDim = dim3(256);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = unsigned(H.tail_grid);
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, k_vcycle_tail<T, NC, true>, lv, nl, bar, limit, err) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    PS_TICK();
    return true;
  }
  if (cudaMemsetAsync(bar, 0, sizeof(unsigned long long), st) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  void* args[] = {&lv, &nl, &bar, &limit, &err};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_vcycle_tail<T, NC, false>, H.tail_grid, 256, args, 0, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  PS_TICK();
  return true;
}

template <class T, int NC>
void vcycle_level(Amg& H, int l, const SmoothParams& sp, const T* b, T* out, cudaStream_t st) {
  AmgLevel& L = H.L[l];
  LevelT<T> V = view<T>(L);
  int64_t n = L.n;
  if (l >= 1 && l == H.tail_l0 && H.tail && (H.tail_mode == 2 || (H.tail_mode == 1 && H.err)) &&
      b == static_cast<const T*>(L.b) && out == static_cast<T*>(L.e) && launch_tail<T, NC>(H, st))
    return;
  if (L.coarsest) {
    PS_TICK(); vl(k_dense_solve<T, NC>, grid_for(n * NC * 32, 256), st, n, V.inv, b, out);
    return;
  }
  T* x = static_cast<T*>(L.x);
  T* t = static_cast<T*>(L.t);
  T* d = static_cast<T*>(L.d);
  T* r = static_cast<T*>(L.r);
  AmgLevel& C = H.L[l + 1];
  T* bc = static_cast<T*>(C.b);
  T* ec = static_cast<T*>(C.e);
  T* xs = smooth_zero<T, NC>(L, V, sp, b, x, t, d, st);
  with_rows<T, NC>(L, V, [&](auto a) {
    using A = decltype(a);
    PS_TICK(); vl(k_resid<T, NC, A>, rows_grid<A>(n), st, a, n, b, xs, r);
  });
  if (L.rvb && sizeof(T) == 4) spmv_lanes<T, NC>(L.rlane, C.n, L.rrp, L.rci, L.rvb, r, bc, 0, st);
  else spmv_lanes<T, NC>(L.rlane, C.n, L.rrp, L.rci, V.rv, r, bc, 0, st);
  vcycle_level<T, NC>(H, l + 1, sp, bc, ec, st);
  if (L.pvb && sizeof(T) == 4) spmv_lanes<T, NC>(L.plane, n, L.prp, L.pci, L.pvb, ec, xs, 1, st);
  else spmv_lanes<T, NC>(L.plane, n, L.prp, L.pci, V.pv, ec, xs, 1, st);
  smooth_post<T, NC>(L, V, sp, b, xs, xs == x ? t : x, d, out, st);
}

template <class T>
void vcycle_launch(Amg& H, const SmoothParams& sp, const T* b, T* x, cudaStream_t st) {
  t_pdl = H.pdl ? 1 : 0;
  if (H.nc == 3) vcycle_level<T, 3>(H, 0, sp, b, x, st);
  else vcycle_level<T, 1>(H, 0, sp, b, x, st);
  t_pdl = 0;
}

}  // namespace

// descriptors of the tail levels for k_vcycle_tail (Chebyshev degree 2, FP32 or FP64 transfer operators):
// tail_mode 1, the levels below the finest in a cooperative launch; tail_mode 2, the levels from the first
// one of at most kClusterTailRows rows in one thread-block cluster.  Leaves H.tail null when the mode is 0
// or the launch is not possible.
template <class T>
ps_status tail_setup(Arena& ar, Amg& H, const SmoothParams& sp, cudaStream_t st) {
  H.tail = nullptr;
  const int nlev = int(H.L.size());
  if (H.tail_mode == 0 || sp.kind != PS_SMOOTH_CHEBYSHEV || sp.degree != 2 || nlev < 3) return PS_OK;
  int l0 = 1;
  if (H.tail_mode == 2) {
    while (l0 < nlev - 1 && H.L[l0].n > kClusterTailRows) ++l0;
    if (l0 >= nlev - 1) return PS_OK;  // only the coarsest is small: nothing to merge
  }
  for (int l = l0; l < nlev; ++l) {
    const AmgLevel& L = H.L[l];
    if (l < nlev - 1 && (!L.dsi || L.coarsest || L.pvb || L.rvb || L.sv_f || L.sv_d)) return PS_OK;
  }
  if (!H.L[nlev - 1].coarsest) return PS_OK;
  int dev = 0, coop = 0, sms = 0, occ = 0, grid = 0;
  PS_CUDA(cudaGetDevice(&dev));
  if (H.tail_mode == 2) {
    const void* fn = H.nc == 3 ? (const void*)k_vcycle_tail<T, 3, true> : (const void*)k_vcycle_tail<T, 1, true>;
    for (int cs : {kTailCluster, 8}) {
      if (cs > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(unsigned(cs));
      cfg.blockDim = dim3(256);
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = unsigned(cs);
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int ncl = 0;
      if (cudaOccupancyMaxActiveClusters(&ncl, fn, &cfg) == cudaSuccess && ncl >= 1) {
        grid = cs;
        break;
      }
      cudaGetLastError();
    }
    if (grid == 0) return PS_OK;
  } else {
    PS_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    PS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const void* fn = H.nc == 3 ? (const void*)k_vcycle_tail<T, 3, false> : (const void*)k_vcycle_tail<T, 1, false>;
    PS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 256, 0));
    if (!coop || occ < 1) return PS_OK;
    grid = sms * (occ < 2 ? occ : 2);
  }
  std::vector<TailLevel<T>> tl;
  for (int l = l0; l < nlev; ++l) {
    const AmgLevel& L = H.L[l];
    const LevelT<T> V = view<T>(L);
    TailLevel<T> t;
    std::memset(&t, 0, sizeof(t));
    t.n = L.n;
    t.coarsest = L.coarsest ? 1 : 0;
    t.lanes = L.lanes; t.plane = L.plane; t.rlane = L.rlane;
    t.rp = L.rp; t.ci = L.ci; t.v = V.v; t.dg = V.dg; t.dsi = static_cast<const T*>(L.dsi);
    t.inv = L.inv;
    t.x = static_cast<T*>(L.x); t.t = static_cast<T*>(L.t); t.r = static_cast<T*>(L.r);
    t.d = static_cast<T*>(L.d); t.b = static_cast<T*>(L.b); t.e = static_cast<T*>(L.e);
    if (!L.coarsest) {
      t.nnext = H.L[l + 1].n;
      t.prp = L.prp; t.pci = L.pci; t.pv = V.pv;
      t.rrp = L.rrp; t.rci = L.rci; t.rv = V.rv;
      ChebCoef cc = cheb_coef(L, H.nc, sp);
      t.c1 = cc.c1[1]; t.c2 = cc.c2[1]; t.pc2 = cc.post_c2;
    }
    tl.push_back(t);
  }
  TailLevel<T>* d;
  PS_TRY(ar.alloc(&d, tl.size()));
  PS_CUDA(cudaMemcpyAsync(d, tl.data(), sizeof(TailLevel<T>) * tl.size(), cudaMemcpyHostToDevice, st));
  PS_TRY(ar.alloc(&H.tail_bar, 1));
  PS_CUDA(cudaStreamSynchronize(st));
  H.tail = d;
  H.tail_l0 = l0;
  H.tail_levels = int(tl.size());
  H.tail_grid = grid;
  return PS_OK;
}

// ---------------------------------------------------------------------------
// Lanes-per-row autotuner for the CSR kernels of the coarse levels.  For each level below the finest (the
// finest is stencil-indexed on the structured grid, or tuned too when it is not) it times the residual kernel
// of the level operator, and for every level the prolongation and restriction products, with half, the same
// and twice the lanes that the mean row length gives (3 launches each after one warm-up, CUDA events on the
// setup stream), and keeps the fastest; a candidate must beat the default by 3 % to replace it.  The choice
// is cached per process by (value type, components, kind, rows, entries), so equal hierarchies get equal
// schedules.  The lanes change only the order in which a row's products are summed.
// ---------------------------------------------------------------------------
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int64_t, int64_t>, int> g_tune;

template <class F>
int tune_lanes(int kind, int tsize, int nc, int64_t n, int64_t nnz, int def, cudaStream_t st, F&& run) {
  const auto key = std::make_tuple(tsize, nc, kind, n, nnz);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second;
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return def;
  }
  const int cand[3] = {def > 1 ? def / 2 : def, def, def < 32 ? def * 2 : def};
  float best_ms = 0.0f, def_ms = 0.0f;
  int best = def;
  for (int t = 0; t < 3; ++t) {
    const int L = cand[t];
    if (t != 1 && L == def) continue;
    run(L);  // warm-up
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3; ++r) run(L);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (L == def) def_ms = ms;
    if (t == 0 || ms < best_ms) { best_ms = ms; best = L; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  if (best != def && best_ms > 0.97f * def_ms) best = def;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto ins = g_tune.emplace(key, best);
  return ins.first->second;
}

template <class T, int NC>
void autotune_levels(Amg& H, cudaStream_t st) {
  const int nlev = int(H.L.size());
  for (int l = 0; l + 1 < nlev; ++l) {
    AmgLevel& L = H.L[l];
    AmgLevel& C = H.L[l + 1];
    LevelT<T> V = view<T>(L);
    const T* b = static_cast<const T*>(L.b);
    T* x = static_cast<T*>(L.x);
    T* r = static_cast<T*>(L.r);
    const int64_t n = L.n;
    if (!V.sv) {
      L.lanes = tune_lanes(0, int(sizeof(T)), NC, n, L.nnz, L.lanes, st, [&](int lanes) {
        AmgLevel Lt = L;
        Lt.lanes = lanes;
        with_rows<T, NC>(Lt, V, [&](auto a) {
          using A = decltype(a);
          PS_TICK(); k_resid<T, NC, A><<<rows_grid<A>(n), 256, 0, st>>>(a, n, b, x, r);
        });
      });
    }
    if (!L.pvb) {
      L.plane = tune_lanes(1, int(sizeof(T)), NC, n, L.pnnz, L.plane, st, [&](int lanes) {
        spmv_lanes<T, NC>(lanes, n, L.prp, L.pci, V.pv, static_cast<const T*>(C.e), x, 0, st);
      });
      L.rlane = tune_lanes(2, int(sizeof(T)), NC, C.n, L.pnnz, L.rlane, st, [&](int lanes) {
        spmv_lanes<T, NC>(lanes, C.n, L.rrp, L.rci, V.rv, r, static_cast<T*>(C.b), 0, st);
      });
    }
  }
}

template <class T>
ps_status amg_alloc_work(Arena& ar, Amg& H, const SmoothParams& sp, cudaStream_t st) {
  for (auto& L : H.L) {
    size_t m = size_t(L.n) * H.nc + 1;
    T *x, *t, *r, *d, *b, *e;
    PS_TRY(ar.alloc(&x, m)); PS_TRY(ar.alloc(&t, m)); PS_TRY(ar.alloc(&r, m)); PS_TRY(ar.alloc(&d, m));
    PS_TRY(ar.alloc(&b, m)); PS_TRY(ar.alloc(&e, m));
    L.x = x; L.t = t; L.r = r; L.d = d; L.b = b; L.e = e;
    if (sp.kind == PS_SMOOTH_CHEBYSHEV && sp.degree > 1 && !L.coarsest) {
      T* dsi;
      PS_TRY(ar.alloc(&dsi, m));
      ChebCoef cc = cheb_coef(L, H.nc, sp);
      const T* dg = view<T>(L).dg;
      if (H.nc == 3) { PS_TICK(); k_dsi<T, 3><<<grid_for(L.n * 3, 256), 256, 0, st>>>(L.n, dg, dsi, cc.inv_theta); }
      else { PS_TICK(); k_dsi<T, 1><<<grid_for(L.n, 256), 256, 0, st>>>(L.n, dg, dsi, cc.inv_theta); }
      L.dsi = dsi;
    }
  }
  PS_CUDA(cudaGetLastError());
  if (H.autotune) {
    if (H.nc == 3) autotune_levels<T, 3>(H, st);
    else autotune_levels<T, 1>(H, st);
    PS_CUDA(cudaGetLastError());
  }
  return tail_setup<T>(ar, H, sp, st);
}

void amg_release_graph(Amg& H) {
  if (H.gexec) cudaGraphExecDestroy(H.gexec);
  H.gexec = nullptr;
  H.gb = nullptr;
  H.gx = nullptr;
  H.gst = nullptr;
  H.gnodes = 0;
}

// The V-cycle is about thirty short kernels whose arguments depend only on the hierarchy, b and x:
// captured once into a CUDA graph and replayed, so that the coarse levels do not wait on kernel
// launches.  Streams that cannot be captured (the legacy default stream) run the kernels directly.
template <class T>
ps_status amg_vcycle(Amg& H, const SmoothParams& sp, const T* b, T* x, cudaStream_t st) {
  if (H.gexec && H.gb == b && H.gx == x && H.gst == st) {
    PS_CUDA(cudaGraphLaunch(H.gexec, st));
    g_launches.fetch_add(H.gnodes, std::memory_order_relaxed);
    return PS_OK;
  }
  if (st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread) {
    amg_release_graph(H);
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      vcycle_launch<T>(H, sp, b, x, st);
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
          H.gnodes = int64_t(nodes);  // the kernels ticked while capturing run in this first launch
          PS_CUDA(cudaGraphLaunch(ex, st));
          return PS_OK;
        }
      }
      cudaGetLastError();
    } else {
      cudaGetLastError();
    }
  }
  vcycle_launch<T>(H, sp, b, x, st);
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

template <class T>
ps_status amg_vcycle_direct(Amg& H, const SmoothParams& sp, const T* b, T* x, cudaStream_t st) {
  vcycle_launch<T>(H, sp, b, x, st);
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

template ps_status amg_vcycle_direct<double>(Amg&, const SmoothParams&, const double*, double*, cudaStream_t);
template ps_status amg_alloc_work<float>(Arena&, Amg&, const SmoothParams&, cudaStream_t);
template ps_status amg_alloc_work<double>(Arena&, Amg&, const SmoothParams&, cudaStream_t);
template ps_status amg_vcycle<float>(Amg&, const SmoothParams&, const float*, float*, cudaStream_t);
template ps_status amg_vcycle<double>(Amg&, const SmoothParams&, const double*, double*, cudaStream_t);

}  // namespace ps_internal
