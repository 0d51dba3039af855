// FP64 Jacobian SpMV and flexible-GMRES kernels.  Every reduction is taken in
// a fixed order (per-block partial sums, then one block over the partials), so
// repeated solves give identical iterates.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>

#include "gridsync.cuh"
#include "krylov.cuh"

namespace ps_internal {
namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Displacement rows: one warp per node.  A_uu row: 27 blocks x 3 rows = up to
// 81 row segments of 3 doubles; A_uf row: up to 8 blocks x 3 rows of 2 doubles.
__global__ void __launch_bounds__(256) k_spmv_u(JacDev J, const double* __restrict__ x, double* __restrict__ y,
                                                const double* __restrict__ b, double* __restrict__ part) {
  __shared__ double red[8];
  int64_t I = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  double r2 = 0.0;
  if (I < J.nn) {
    const double* xu = x;
    const double* xf = x + 3 * J.nn;
    double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
    int32_t q0 = J.uu_rp[I], q1 = J.uu_rp[I + 1];
    int nseg = (q1 - q0) * 3;
    for (int s = lane; s < nseg; s += 32) {
      int32_t q = q0 + s / 3;
      int r = s % 3;
      int64_t c = J.uu_ci[q];
      const double* v = J.uu_v + int64_t(q) * 9 + r * 3;
      double t = v[0] * xu[3 * c] + v[1] * xu[3 * c + 1] + v[2] * xu[3 * c + 2];
      acc0 += r == 0 ? t : 0.0;
      acc1 += r == 1 ? t : 0.0;
      acc2 += r == 2 ? t : 0.0;
    }
    int32_t p0 = J.uf_rp[I], p1 = J.uf_rp[I + 1];
    int mseg = (p1 - p0) * 3;
    for (int s = lane; s < mseg; s += 32) {
      int32_t q = p0 + s / 3;
      int r = s % 3;
      int64_t c = J.uf_ci[q];
      const double* v = J.uf_v + int64_t(q) * 6 + r * 2;
      double t = v[0] * xf[2 * c] + v[1] * xf[2 * c + 1];
      acc0 += r == 0 ? t : 0.0;
      acc1 += r == 1 ? t : 0.0;
      acc2 += r == 2 ? t : 0.0;
    }
    acc0 = warp_sum(acc0);
    acc1 = warp_sum(acc1);
    acc2 = warp_sum(acc2);
    if (lane < 3) {
      double a = lane == 0 ? acc0 : lane == 1 ? acc1 : acc2;
      if (b) {
        a = b[3 * I + lane] - a;
        r2 = a * a;
      }
      y[3 * I + lane] = a;
    }
  }
  if (part) {
    r2 = warp_sum(r2);
    if (lane == 0) red[threadIdx.x >> 5] = r2;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < 8; ++w) s += red[w];
      part[blockIdx.x] = s;
    }
  }
}

// Flow rows: one warp per cell; lanes 0..15 take the 8 A_fu blocks x 2 rows,
// lanes 16..29 the 7 A_ff blocks x 2 rows.
__global__ void __launch_bounds__(256) k_spmv_f(JacDev J, const double* __restrict__ x, double* __restrict__ y,
                                                const double* __restrict__ b, double* __restrict__ part) {
  __shared__ double red[8];
  int64_t c = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  double r2 = 0.0;
  if (c < J.nc) {
    const double* xu = x;
    const double* xf = x + 3 * J.nn;
    double a0 = 0.0, a1 = 0.0;
    if (lane < 16) {
      int32_t q = J.fu_rp[c] + (lane >> 1);
      int r = lane & 1;
      if (q < J.fu_rp[c + 1]) {
        int64_t J3 = int64_t(J.fu_ci[q]) * 3;
        const double* v = J.fu_v + int64_t(q) * 6 + r * 3;
        double t = v[0] * xu[J3] + v[1] * xu[J3 + 1] + v[2] * xu[J3 + 2];
        if (r == 0) a0 = t; else a1 = t;
      }
    } else {
      int s = lane - 16;
      int32_t q = J.ff_rp[c] + (s >> 1);
      int r = s & 1;
      if (s < 14 && q < J.ff_rp[c + 1]) {
        int64_t j2 = int64_t(J.ff_ci[q]) * 2;
        const double* v = J.ff_v + int64_t(q) * 4 + r * 2;
        double t = v[0] * xf[j2] + v[1] * xf[j2 + 1];
        if (r == 0) a0 = t; else a1 = t;
      }
    }
    a0 = warp_sum(a0);
    a1 = warp_sum(a1);
    if (lane < 2) {
      double a = lane == 0 ? a0 : a1;
      int64_t o = 3 * J.nn + 2 * c + lane;
      if (b) {
        a = b[o] - a;
        r2 = a * a;
      }
      y[o] = a;
    }
  }
  if (part) {
    r2 = warp_sum(r2);
    if (lane == 0) red[threadIdx.x >> 5] = r2;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < 8; ++w) s += red[w];
      part[blockIdx.x] = s;
    }
  }
}

// ---------------------------------------------------------------------------
// Stencil-indexed Jacobian.  Slots: A_uu 27 node neighbours (dk, dj, di) in
// {-1,0,1}^3 ascending, A_uf 8 cells (dk, dj, di) in {-1,0}^3, A_fu 8 nodes in
// {0,1}^3, A_ff 7 cells (z-1, y-1, x-1, self, x+1, y+1, z+1).  Missing
// neighbours are zero blocks, so the sweep needs neither row pointers nor
// column indices and every coefficient load is coalesced across rows.
// ---------------------------------------------------------------------------
struct Geo {
  int nx, ny, nz;
  __device__ __forceinline__ int64_t node(int i, int j, int k) const { return i + int64_t(nx + 1) * (j + int64_t(ny + 1) * k); }
  __device__ __forceinline__ int64_t cell(int i, int j, int k) const { return i + int64_t(nx) * (j + int64_t(ny) * k); }
};

// neighbour of slot s in each family, or -1 when outside the grid
__device__ __forceinline__ int64_t uu_nb(const Geo& g, int i, int j, int k, int s) {
  int a = i + s % 3 - 1, b = j + (s / 3) % 3 - 1, c = k + s / 9 - 1;
  if (a < 0 || b < 0 || c < 0 || a > g.nx || b > g.ny || c > g.nz) return -1;
  return g.node(a, b, c);
}
__device__ __forceinline__ int64_t uf_nb(const Geo& g, int i, int j, int k, int s) {
  int a = i + (s & 1) - 1, b = j + ((s >> 1) & 1) - 1, c = k + (s >> 2) - 1;
  if (a < 0 || b < 0 || c < 0 || a >= g.nx || b >= g.ny || c >= g.nz) return -1;
  return g.cell(a, b, c);
}
__device__ __forceinline__ int64_t fu_nb(const Geo& g, int i, int j, int k, int s) {
  return g.node(i + (s & 1), j + ((s >> 1) & 1), k + (s >> 2));
}
__device__ __forceinline__ int64_t ff_nb(const Geo& g, int i, int j, int k, int s) {
  const int di[7] = {0, 0, -1, 0, 1, 0, 0}, dj[7] = {0, -1, 0, 0, 0, 1, 0}, dk[7] = {-1, 0, 0, 0, 0, 0, 1};
  int a = i + di[s], b = j + dj[s], c = k + dk[s];
  if (a < 0 || b < 0 || c < 0 || a >= g.nx || b >= g.ny || c >= g.nz) return -1;
  return g.cell(a, b, c);
}

// scatter one BSR family into its stencil arrays; flags rows whose pattern is not the stencil
template <int FAM, int NS, int BS>
__global__ void k_to_stencil(Geo g, int64_t nrows, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             const double* __restrict__ v, double* __restrict__ out, int* __restrict__ bad) {
  int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  int i, j, k;
  if (FAM <= 1) { i = int(r % (g.nx + 1)); j = int((r / (g.nx + 1)) % (g.ny + 1)); k = int(r / (int64_t(g.nx + 1) * (g.ny + 1))); }
  else { i = int(r % g.nx); j = int((r / g.nx) % g.ny); k = int(r / (int64_t(g.nx) * g.ny)); }
  int32_t q = rp[r], q1 = rp[r + 1];
  for (int s = 0; s < NS; ++s) {
    int64_t nb = FAM == 0 ? uu_nb(g, i, j, k, s) : FAM == 1 ? uf_nb(g, i, j, k, s) : FAM == 2 ? fu_nb(g, i, j, k, s)
                                                                                          : ff_nb(g, i, j, k, s);
    bool have = nb >= 0 && q < q1 && ci[q] == nb;
    if (nb >= 0 && !have) atomicExch(bad, 1);
    // blocked by 32 rows: [row / 32][slot][entry][row % 32]
    for (int e = 0; e < BS; ++e)
      out[((r >> 5) * int64_t(NS * BS) + s * BS + e) * 32 + (r & 31)] = have ? v[int64_t(q) * BS + e] : 0.0;
    if (have) ++q;
  }
  if (q != q1) atomicExch(bad, 1);
}

__device__ __forceinline__ int64_t clampnb(int64_t nb, int64_t self) { return nb >= 0 ? nb : self; }

// displacement rows, one thread per node
__global__ void __launch_bounds__(256) k_spmv_u_st(JacDev J, const double* __restrict__ x, double* __restrict__ y,
                                                   const double* __restrict__ b, double* __restrict__ part) {
  __shared__ double red[8];
  Geo g{J.nx, J.ny, J.nz};
  int64_t I = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  double r2 = 0.0;
  if (I < J.nn) {
    int i = int(I % (g.nx + 1)), j = int((I / (g.nx + 1)) % (g.ny + 1)), k = int(I / (int64_t(g.nx + 1) * (g.ny + 1)));
    const int64_t n = J.nn;
    const double* xf = x + 3 * n;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
#pragma unroll 3
    for (int s = 0; s < 27; ++s) {
      int64_t c = clampnb(uu_nb(g, i, j, k, s), I);
      const double* A = J.uu_s + (I >> 5) * int64_t(27 * 9 * 32) + (I & 31) + s * 9 * 32;
      double x0 = x[3 * c], x1 = x[3 * c + 1], x2 = x[3 * c + 2];
      // one FMA per block entry (the FP64 pipe is the bound: no separate products or sums)
      a0 = fma(__ldg(A), x0, a0); a0 = fma(__ldg(A + 32), x1, a0); a0 = fma(__ldg(A + 2 * 32), x2, a0);
      a1 = fma(__ldg(A + 3 * 32), x0, a1); a1 = fma(__ldg(A + 4 * 32), x1, a1); a1 = fma(__ldg(A + 5 * 32), x2, a1);
      a2 = fma(__ldg(A + 6 * 32), x0, a2); a2 = fma(__ldg(A + 7 * 32), x1, a2); a2 = fma(__ldg(A + 8 * 32), x2, a2);
    }
#pragma unroll 4
    for (int s = 0; s < 8; ++s) {
      int64_t c = uf_nb(g, i, j, k, s);
      c = c >= 0 ? c : 0;
      const double* A = J.uf_s + (I >> 5) * int64_t(8 * 6 * 32) + (I & 31) + s * 6 * 32;
      double f0 = xf[2 * c], f1 = xf[2 * c + 1];
      a0 = fma(__ldg(A), f0, a0); a0 = fma(__ldg(A + 32), f1, a0);
      a1 = fma(__ldg(A + 2 * 32), f0, a1); a1 = fma(__ldg(A + 3 * 32), f1, a1);
      a2 = fma(__ldg(A + 4 * 32), f0, a2); a2 = fma(__ldg(A + 5 * 32), f1, a2);
    }
    if (b) {
      a0 = b[3 * I] - a0; a1 = b[3 * I + 1] - a1; a2 = b[3 * I + 2] - a2;
      r2 = a0 * a0 + a1 * a1 + a2 * a2;
    }
    y[3 * I] = a0; y[3 * I + 1] = a1; y[3 * I + 2] = a2;
  }
  if (part) {
    r2 = warp_sum(r2);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = r2;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s2 = 0.0;
      for (int w = 0; w < 8; ++w) s2 += red[w];
      part[blockIdx.x] = s2;
    }
  }
}

// flow rows, one thread per cell
__global__ void __launch_bounds__(256) k_spmv_f_st(JacDev J, const double* __restrict__ x, double* __restrict__ y,
                                                   const double* __restrict__ b, double* __restrict__ part) {
  __shared__ double red[8];
  Geo g{J.nx, J.ny, J.nz};
  int64_t C = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  double r2 = 0.0;
  if (C < J.nc) {
    int i = int(C % g.nx), j = int((C / g.nx) % g.ny), k = int(C / (int64_t(g.nx) * g.ny));
    const double* xf = x + 3 * J.nn;
    double a0 = 0.0, a1 = 0.0;
#pragma unroll 4
    for (int s = 0; s < 8; ++s) {
      int64_t c = fu_nb(g, i, j, k, s);
      const double* A = J.fu_s + (C >> 5) * int64_t(8 * 6 * 32) + (C & 31) + s * 6 * 32;
      double x0 = x[3 * c], x1 = x[3 * c + 1], x2 = x[3 * c + 2];
      a0 = fma(__ldg(A), x0, a0); a0 = fma(__ldg(A + 32), x1, a0); a0 = fma(__ldg(A + 2 * 32), x2, a0);
      a1 = fma(__ldg(A + 3 * 32), x0, a1); a1 = fma(__ldg(A + 4 * 32), x1, a1); a1 = fma(__ldg(A + 5 * 32), x2, a1);
    }
#pragma unroll
    for (int s = 0; s < 7; ++s) {
      int64_t c = clampnb(ff_nb(g, i, j, k, s), C);
      const double* A = J.ff_s + (C >> 5) * int64_t(7 * 4 * 32) + (C & 31) + s * 4 * 32;
      double f0 = xf[2 * c], f1 = xf[2 * c + 1];
      a0 = fma(__ldg(A), f0, a0); a0 = fma(__ldg(A + 32), f1, a0);
      a1 = fma(__ldg(A + 2 * 32), f0, a1); a1 = fma(__ldg(A + 3 * 32), f1, a1);
    }
    int64_t o = 3 * J.nn + 2 * C;
    if (b) {
      a0 = b[o] - a0; a1 = b[o + 1] - a1;
      r2 = a0 * a0 + a1 * a1;
    }
    y[o] = a0; y[o + 1] = a1;
  }
  if (part) {
    r2 = warp_sum(r2);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = r2;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s2 = 0.0;
      for (int w = 0; w < 8; ++w) s2 += red[w];
      part[blockIdx.x] = s2;
    }
  }
}

// fold per-block partials into kRedBlocks slots (fixed mapping)
__global__ void k_fold(const double* __restrict__ in, int64_t nin, double* __restrict__ out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= kRedBlocks) return;
  double s = 0.0;
  for (int64_t i = t; i < nin; i += kRedBlocks) s += in[i];
  out[t] = s;
}

__global__ void k_finish_sum(const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double s[256];
  double a = 0.0;
  for (int i = threadIdx.x; i < kRedBlocks; i += 256) a += part[i];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

// ---- multi-dot h = V^T w (columns in chunks of 8) ----
constexpr int kChunk = 8;
__global__ void __launch_bounds__(256) k_multidot(const double* __restrict__ V, int64_t ldv, int m,
                                                  const double* __restrict__ w, int64_t n, int with_norm,
                                                  double* __restrict__ part, const int* __restrict__ gate) {
  if (gate && *gate == 0) return;
  __shared__ double red[kChunk][8];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int mm = m + (with_norm ? 1 : 0);
  for (int c0 = 0; c0 < mm; c0 += kChunk) {
    double acc[kChunk];
#pragma unroll
    for (int k = 0; k < kChunk; ++k) acc[k] = 0.0;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
      double we = w[e];
#pragma unroll
      for (int k = 0; k < kChunk; ++k) {
        int c = c0 + k;
        if (c < m) acc[k] += V[int64_t(c) * ldv + e] * we;
        else if (c == m && with_norm) acc[k] += we * we;
      }
    }
#pragma unroll
    for (int k = 0; k < kChunk; ++k) {
      double v = warp_sum(acc[k]);
      if (lane == 0) red[k][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < kChunk && c0 + threadIdx.x < mm) {
      double s = 0.0;
      for (int q = 0; q < 8; ++q) s += red[threadIdx.x][q];
      part[int64_t(c0 + threadIdx.x) * kRedBlocks + blockIdx.x] = s;
    }
    __syncthreads();
  }
}

// one warp per column: h[c] = sum of the kRedBlocks partials (fixed order)
__global__ void k_multidot_final(const double* __restrict__ part, int mm, double* __restrict__ h,
                                 const int* __restrict__ gate) {
  if (gate && *gate == 0) return;
  int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (c >= mm) return;
  double s = 0.0;
  for (int i = lane; i < kRedBlocks; i += 32) s += part[int64_t(c) * kRedBlocks + i];
  s = warp_sum(s);
  if (lane == 0) h[c] = s;
}

__global__ void __launch_bounds__(256) k_mupdate(const double* __restrict__ V, int64_t ldv, int m,
                                                 const double* __restrict__ h, double* __restrict__ w, int64_t n,
                                                 double* __restrict__ part, const int* __restrict__ gate) {
  if (gate && *gate == 0) return;
  __shared__ double hs[128];
  __shared__ double red[8];
  for (int c = threadIdx.x; c < m; c += blockDim.x) hs[c] = h[c];
  __syncthreads();
  double r2 = 0.0;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
    double s = w[e];
#pragma unroll 8
    for (int c = 0; c < m; ++c) s -= __ldg(V + int64_t(c) * ldv + e) * hs[c];
    w[e] = s;
    r2 += s * s;
  }
  r2 = warp_sum(r2);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = r2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < 8; ++q) s += red[q];
    part[blockIdx.x] = s;
  }
}

__global__ void k_maxpy(const double* __restrict__ Z, int64_t ldz, int m, const double* __restrict__ y,
                        double* __restrict__ x, int64_t n) {
  __shared__ double ys[128];
  for (int c = threadIdx.x; c < m; c += blockDim.x) ys[c] = y[c];
  __syncthreads();
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
    double s = x[e];
    for (int c = 0; c < m; ++c) s += Z[int64_t(c) * ldz + e] * ys[c];
    x[e] = s;
  }
}

__global__ void k_scale(const double* __restrict__ x, double* __restrict__ y, int64_t n,
                        const double* __restrict__ sc) {
  double a = *sc;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x)
    y[e] = x[e] * a;
}
__global__ void k_zero(double* __restrict__ x, int64_t n) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x)
    x[e] = 0.0;
}

// Daniel-Gragg-Kaufman-Stewart test: reorthogonalise when ||w'|| < ||w|| / sqrt(2)
__global__ void k_arnoldi_check(double* sc, int* flag) {
  flag[0] = (sc[1] < 0.5 * sc[0]) ? 1 : 0;
}

// column j of the Hessenberg matrix, Givens rotations, residual estimate
__global__ void k_arnoldi_finish(double* H, double* cs, double* sn, double* g, const double* h1, const double* h2,
                                 double* sc, int* flag, int m, int j) {
  int re = flag[0];
  double hn2 = re ? sc[2] : sc[1];
  double hn = sqrt(hn2);
  double* col = H + int64_t(j) * (m + 1);
  for (int i = 0; i <= j; ++i) col[i] = h1[i] + (re ? h2[i] : 0.0);
  col[j + 1] = hn;
  for (int i = 0; i < j; ++i) {
    double a = col[i], c = col[i + 1];
    col[i] = cs[i] * a + sn[i] * c;
    col[i + 1] = -sn[i] * a + cs[i] * c;
  }
  double a = col[j], c = col[j + 1];
  double rr = hypot(a, c);
  cs[j] = a / rr;
  sn[j] = c / rr;
  col[j] = rr;
  col[j + 1] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  sc[5] = fabs(g[j + 1]) / sc[7];
  sc[6] = hn;
  sc[4] = hn > 0.0 ? 1.0 / hn : 0.0;
  flag[1] = (isnan(sc[5]) || isnan(hn) || isinf(hn)) ? 1 : 0;
}

__global__ void k_cycle_start(double* g, double* sc, int m) {
  double beta = sqrt(sc[3]);
  for (int i = 0; i <= m; ++i) g[i] = 0.0;
  g[0] = beta;
  sc[4] = beta > 0.0 ? 1.0 / beta : 0.0;
}

__global__ void k_hsolve(const double* H, const double* g, double* y, int m, int k) {
  for (int i = k; i >= 0; --i) {
    double s = g[i];
    for (int c = i + 1; c <= k; ++c) s -= H[int64_t(c) * (m + 1) + i] * y[c];
    y[i] = s / H[int64_t(i) * (m + 1) + i];
  }
}

// ---------------------------------------------------------------------------
// Arnoldi step by modified Gram-Schmidt in one cooperative launch, kS basis
// vectors per sweep.  Modified Gram-Schmidt takes, for k = 0..j in turn,
// h_k = v_k . w_k and w_{k+1} = w_k - h_k v_k.  Expanding w_k over one block B
// of consecutive k gives h_k = v_k . w_B - sum_{l in B, l < k} h_l (v_k . v_l):
// the same coefficients follow from the dots of the block's vectors with the w
// at the block start and the in-block Gram entries v_k . v_l, by a forward
// substitution.  So sweep p forms the block's dots (and, in the last block, the
// Gram entries of the newest vector v_j with its block-mates; older entries are
// kept from the launches that created them), and also applies the update of the
// previous block, whose coefficients the grid barrier between sweeps made known.
// Each sweep costs two FP64 FMAs per row and basis vector, as plain modified
// Gram-Schmidt does, with one grid barrier per kS vectors instead of one per
// vector.  After the last sweep, h_{j+1} = ||w|| and v_{j+1} = w / h_{j+1}.
// Every thread keeps the same rows in every sweep, so w needs no
// synchronisation; after each barrier every CTA sums the CTA partials in one
// fixed order, so all CTAs hold bit-identical coefficients.
// ---------------------------------------------------------------------------
constexpr int kMgsThreads = 256;
constexpr int kS = 8;            // most basis vectors per sweep (row stride of the Gram store)

// Warp sums of R values per lane (R a power of two, at most 32) by a transposing butterfly: at each of
// the first log2(R) levels a lane keeps one half of its values, sends the other half to its partner and
// adds what it receives, so the adds per lane are R/2 + R/4 + ... instead of 5 R.  Afterwards the lanes
// of each group of 32 / R hold the full sum of value *which, the same in every lane of the group.
template <int R>
__device__ __forceinline__ double warp_sum_many(double (&a)[R], int lane, int& which) {
  int idx = 0;
  int mask = 16;
#pragma unroll
  for (int half = R / 2; half >= 1; half /= 2, mask >>= 1) {
    const bool up = (lane & mask) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const double keep = up ? a[half + i] : a[i];
      const double send = up ? a[i] : a[half + i];
      a[i] = keep + __shfl_xor_sync(0xffffffffu, send, mask);
    }
    idx = (idx << 1) | (up ? 1 : 0);
  }
  double v = a[0];
#pragma unroll
  for (; mask > 0; mask >>= 1) v += __shfl_xor_sync(0xffffffffu, v, mask);
  which = idx;
  return v;
}

// Gm[k * kS + (l - S * (k / S))] = v_k . v_l for the block-mates l < k of v_k (S vectors per sweep).
// Rows are taken in pairs (one 16-byte load per vector and pair): the basis columns are ldv apart with
// ldv even, and when n is odd the row n of every column is kept zero, so the last pair adds nothing.
template <int S>
__global__ void __launch_bounds__(kMgsThreads, S <= 4 ? 4 : 2) k_mgs(const double* __restrict__ V, int64_t ldv, int j,
                                                     double* __restrict__ w, int n2, double* __restrict__ h,
                                                     double* __restrict__ Gm, double* __restrict__ sc,
                                                     int* __restrict__ flag, double* __restrict__ part,
                                                     unsigned long long* bar, unsigned long long base, int64_t limit,
                                                     int stall) {
  // test hook: CTA stall - 1 never arrives, so the others' bounded barrier waits run out
  if (stall > 0 && int(blockIdx.x) == stall - 1) return;
  constexpr int R = 2 * S;  // partial sums per sweep: S dots, S - 1 Gram entries, ||w||^2 (last slot)
  __shared__ double red[kMgsThreads / 32][R];
  __shared__ double sums[R];
  __shared__ double scratch[kMgsThreads / 16];
  __shared__ double hs[S];  // the sweep's coefficients
  const int G = gridDim.x, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int stride = G * kMgsThreads, t0 = int(blockIdx.x) * kMgsThreads + int(threadIdx.x);
  const double2* __restrict__ V2 = reinterpret_cast<const double2*>(V);
  double2* __restrict__ w2 = reinterpret_cast<double2*>(w);
  const int64_t ld2 = ldv / 2;
  int* err = flag + 2;
  const int nb = j / S + 1;  // blocks of basis vectors 0..j
  double hp[S];              // coefficients of the previous block
  int pc0 = 0, pcn = 0;      // previous block: first column and size
#pragma unroll
  for (int c = 0; c < S; ++c) hp[c] = 0.0;
  double wn2 = 0.0;
  for (int p = 0; p <= nb; ++p) {
    const int c0 = p * S;
    const int cn = p < nb ? min(S, j + 1 - c0) : 0;  // vectors dotted in this sweep
    const bool last = p == nb - 1;
    const int ng = last ? cn - 1 : 0;                // Gram entries of v_j with its block-mates
    const double2* vprev[S];
    const double2* vcur[S];
#pragma unroll
    for (int c = 0; c < S; ++c) {
      vprev[c] = V2 + int64_t(pc0 + (c < pcn ? c : 0)) * ld2;
      vcur[c] = V2 + int64_t(c0 + (c < cn ? c : 0)) * ld2;
    }
    const double2* vjp = V2 + int64_t(j) * ld2;
    double acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0.0;
    if (p < nb && pcn == S && cn == S && ng == 0) {
      // full blocks: update by the previous block, dots with this one
#pragma unroll(S <= 2 ? 2 : 1)
      for (int e = t0; e < n2; e += stride) {
        double2 we = w2[e];
#pragma unroll
        for (int c = 0; c < S; ++c) {
          const double2 v = __ldcs(vprev[c] + e);
          we.x = fma(-hp[c], v.x, we.x);
          we.y = fma(-hp[c], v.y, we.y);
        }
        w2[e] = we;
#pragma unroll
        for (int c = 0; c < S; ++c) {
          const double2 v = vcur[c][e];
          acc[c] = fma(v.x, we.x, acc[c]);
          acc[c] = fma(v.y, we.y, acc[c]);
        }
      }
    } else if (p < nb && pcn == 0 && cn == S && ng == 0) {
      // first sweep: dots only
#pragma unroll(S <= 2 ? 2 : 1)
      for (int e = t0; e < n2; e += stride) {
        const double2 we = w2[e];
#pragma unroll
        for (int c = 0; c < S; ++c) {
          const double2 v = vcur[c][e];
          acc[c] = fma(v.x, we.x, acc[c]);
          acc[c] = fma(v.y, we.y, acc[c]);
        }
      }
    } else if (p == nb && pcn == S) {
      // last sweep after a full block: update and ||w||^2
#pragma unroll(S <= 2 ? 2 : 1)
      for (int e = t0; e < n2; e += stride) {
        double2 we = w2[e];
#pragma unroll
        for (int c = 0; c < S; ++c) {
          const double2 v = __ldcs(vprev[c] + e);
          we.x = fma(-hp[c], v.x, we.x);
          we.y = fma(-hp[c], v.y, we.y);
        }
        w2[e] = we;
        acc[R - 1] = fma(we.x, we.x, acc[R - 1]);
        acc[R - 1] = fma(we.y, we.y, acc[R - 1]);
      }
    } else {
      // partial blocks (the block holding v_j, and the update by it)
      for (int e = t0; e < n2; e += stride) {
        double2 we = w2[e];
#pragma unroll
        for (int c = 0; c < S; ++c)
          if (c < pcn) {
            const double2 v = __ldcs(vprev[c] + e);
            we.x = fma(-hp[c], v.x, we.x);
            we.y = fma(-hp[c], v.y, we.y);
          }
        if (pcn > 0) w2[e] = we;
        if (p < nb) {
          const double2 vj = ng > 0 ? vjp[e] : make_double2(0.0, 0.0);
#pragma unroll
          for (int c = 0; c < S; ++c)
            if (c < cn) {
              const double2 v = vcur[c][e];
              acc[c] = fma(v.x, we.x, acc[c]);
              acc[c] = fma(v.y, we.y, acc[c]);
              if (c < ng) {
                acc[S + c] = fma(v.x, vj.x, acc[S + c]);
                acc[S + c] = fma(v.y, vj.y, acc[S + c]);
              }
            }
        } else {
          acc[R - 1] = fma(we.x, we.x, acc[R - 1]);
          acc[R - 1] = fma(we.y, we.y, acc[R - 1]);
        }
      }
    }
    // CTA partials of the sweep's sums
    {
      int which = 0;
      const double v = warp_sum_many<R>(acc, lane, which);
      if ((lane & ((32 / R) - 1)) == 0) red[wid][which] = v;
    }
    __syncthreads();
    if (threadIdx.x < R) {
      double t = 0.0;
      for (int q = 0; q < kMgsThreads / 32; ++q) t += red[q][threadIdx.x];
      part[(int64_t(p & 1) * R + threadIdx.x) * G + blockIdx.x] = t;
    }
    if (!grid_barrier(bar, base + (unsigned long long)(p + 1) * G, limit, err)) return;
    // every CTA sums the G partials of each quantity in the same order: kMgsThreads / R threads per
    // quantity, each a strided share, then a fixed shuffle tree and a fixed sum over the warps
    {
      constexpr int TPQ = kMgsThreads / R;
      const int r = threadIdx.x / TPQ, sub = threadIdx.x % TPQ;
      const double* pp = part + (int64_t(p & 1) * R + r) * G;
      double t = 0.0;
      for (int i = sub; i < G; i += TPQ) t += __ldcg(pp + i);
      constexpr int W = TPQ < 32 ? TPQ : 32;
#pragma unroll
      for (int o = W / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o, W);
      if (sub % W == 0) scratch[threadIdx.x / W] = t;
      __syncthreads();
      if (threadIdx.x < R) {
        constexpr int PW = TPQ / W;  // groups of W threads per quantity
        double u = 0.0;
        for (int q = 0; q < PW; ++q) u += scratch[threadIdx.x * PW + q];
        sums[threadIdx.x] = u;
      }
    }
    __syncthreads();
    if (p < nb) {
      // forward substitution with the in-block Gram entries, by one thread; the others read the
      // coefficients from shared memory
      if (threadIdx.x == 0) {
        double hq[S];
#pragma unroll
        for (int c = 0; c < S; ++c) {
          if (c >= cn) { hq[c] = 0.0; continue; }
          double hk = sums[c];
          const int k = c0 + c;
#pragma unroll
          for (int l = 0; l < S; ++l) {
            if (l >= c) break;
            double g = (k == j) ? sums[S + l] : __ldcg(Gm + int64_t(k) * kS + l);
            hk -= hq[l] * g;
          }
          hq[c] = hk;
          hs[c] = hk;
        }
        if (blockIdx.x == 0) {
#pragma unroll
          for (int c = 0; c < S; ++c)
            if (c < cn) h[c0 + c] = hq[c];
          for (int l = 0; l < ng; ++l) Gm[int64_t(j) * kS + l] = sums[S + l];
        }
      }
      __syncthreads();
#pragma unroll
      for (int c = 0; c < S; ++c) hp[c] = hs[c];
      pc0 = c0;
      pcn = cn;
    } else {
      wn2 = sums[R - 1];
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc[1] = wn2;
        flag[0] = 0;
      }
    }
    __syncthreads();  // sums[] and red[] are rewritten in the next sweep
  }
  // the same reciprocal as the Arnoldi finish step computes
  double hn = sqrt(wn2);
  double inv = hn > 0.0 ? 1.0 / hn : 0.0;
  for (int e = t0; e < n2; e += stride) {
    double2 we = w2[e];
    we.x *= inv;
    we.y *= inv;
    w2[e] = we;
  }
}

constexpr int kVecBlocks = 1216;  // 8 x 152 SMs

}  // namespace

ps_status jac_build_stencil(Arena& ar, JacDev& J, bool* ok, cudaStream_t st) {
  Geo g{J.nx, J.ny, J.nz};
  int* bad;
  PS_TRY(ar.alloc(&bad, 1));
  PS_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
  const size_t bn = size_t((J.nn + 31) / 32) * 32, bc = size_t((J.nc + 31) / 32) * 32;  // whole 32-row blocks
  PS_TRY(ar.alloc(&J.uu_s, size_t(27) * 9 * bn));
  PS_TRY(ar.alloc(&J.uf_s, size_t(8) * 6 * bn));
  PS_TRY(ar.alloc(&J.fu_s, size_t(8) * 6 * bc));
  PS_TRY(ar.alloc(&J.ff_s, size_t(7) * 4 * bc));
  PS_TICK(); k_to_stencil<0, 27, 9><<<grid_for(J.nn, 256), 256, 0, st>>>(g, J.nn, J.uu_rp, J.uu_ci, J.uu_v, J.uu_s, bad);
  PS_TICK(); k_to_stencil<1, 8, 6><<<grid_for(J.nn, 256), 256, 0, st>>>(g, J.nn, J.uf_rp, J.uf_ci, J.uf_v, J.uf_s, bad);
  PS_TICK(); k_to_stencil<2, 8, 6><<<grid_for(J.nc, 256), 256, 0, st>>>(g, J.nc, J.fu_rp, J.fu_ci, J.fu_v, J.fu_s, bad);
  PS_TICK(); k_to_stencil<3, 7, 4><<<grid_for(J.nc, 256), 256, 0, st>>>(g, J.nc, J.ff_rp, J.ff_ci, J.ff_v, J.ff_s, bad);
  PS_CUDA(cudaGetLastError());
  int h = 0;
  PS_CUDA(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  PS_CUDA(cudaStreamSynchronize(st));
  ar.release(bad);
  *ok = h == 0;
  if (!*ok) {
    ar.release(J.uu_s); ar.release(J.uf_s); ar.release(J.fu_s); ar.release(J.ff_s);
    J.uu_s = J.uf_s = J.fu_s = J.ff_s = nullptr;
  }
  return PS_OK;
}

ps_status jac_refresh_stencil(Arena& ar, JacDev& J, int mask, cudaStream_t st) {
  if (!J.uu_s) return PS_OK;
  Geo g{J.nx, J.ny, J.nz};
  int* bad;
  PS_TRY(ar.alloc(&bad, 1));
  PS_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
  if (mask & 1) { PS_TICK(); k_to_stencil<0, 27, 9><<<grid_for(J.nn, 256), 256, 0, st>>>(g, J.nn, J.uu_rp, J.uu_ci, J.uu_v, J.uu_s, bad); }
  if (mask & 2) { PS_TICK(); k_to_stencil<1, 8, 6><<<grid_for(J.nn, 256), 256, 0, st>>>(g, J.nn, J.uf_rp, J.uf_ci, J.uf_v, J.uf_s, bad); }
  if (mask & 4) { PS_TICK(); k_to_stencil<2, 8, 6><<<grid_for(J.nc, 256), 256, 0, st>>>(g, J.nc, J.fu_rp, J.fu_ci, J.fu_v, J.fu_s, bad); }
  if (mask & 8) { PS_TICK(); k_to_stencil<3, 7, 4><<<grid_for(J.nc, 256), 256, 0, st>>>(g, J.nc, J.ff_rp, J.ff_ci, J.ff_v, J.ff_s, bad); }
  PS_CUDA(cudaGetLastError());
  PS_CUDA(cudaStreamSynchronize(st));
  ar.release(bad);
  return PS_OK;
}

void jac_spmv(const JacDev& J, const double* x, double* y, const double* b, double* part, cudaStream_t st) {
  if (J.uu_s) {
    int64_t gu = ceil_div(J.nn, 256), gf = ceil_div(J.nc, 256);
    double* pu = part ? part + kRedBlocks : nullptr;
    double* pf = part ? part + kRedBlocks + gu : nullptr;
    PS_TICK(); k_spmv_u_st<<<unsigned(gu), 256, 0, st>>>(J, x, y, b, pu);
    PS_TICK(); k_spmv_f_st<<<unsigned(gf), 256, 0, st>>>(J, x, y, b, pf);
    if (part) { PS_TICK(); k_fold<<<grid_for(kRedBlocks, 256), 256, 0, st>>>(part + kRedBlocks, gu + gf, part); }
    return;
  }
  int64_t gu = ceil_div(J.nn * 32, 256), gf = ceil_div(J.nc * 32, 256);
  // partial sums: u blocks first, then f blocks, folded into kRedBlocks slots
  double* pu = part ? part + kRedBlocks : nullptr;
  double* pf = part ? part + kRedBlocks + gu : nullptr;
  PS_TICK(); k_spmv_u<<<unsigned(gu), 256, 0, st>>>(J, x, y, b, pu);
  PS_TICK(); k_spmv_f<<<unsigned(gf), 256, 0, st>>>(J, x, y, b, pf);
  if (part) { PS_TICK(); k_fold<<<grid_for(kRedBlocks, 256), 256, 0, st>>>(part + kRedBlocks, gu + gf, part); }
}

void multidot(const double* V, int64_t ldv, int m, const double* w, int64_t n, double* part, double* h,
              int with_norm, const int* gate, cudaStream_t st) {
  PS_TICK(); k_multidot<<<kRedBlocks, 256, 0, st>>>(V, ldv, m, w, n, with_norm, part, gate);
  int mm = m + (with_norm ? 1 : 0);
  PS_TICK(); k_multidot_final<<<grid_for(int64_t(mm) * 32, 256), 256, 0, st>>>(part, mm, h, gate);
}

void mupdate(const double* V, int64_t ldv, int m, const double* h, double* w, int64_t n, double* part,
             double* norm2, const int* gate, cudaStream_t st) {
  PS_TICK(); k_mupdate<<<kRedBlocks, 256, 0, st>>>(V, ldv, m, h, w, n, part, gate);
  PS_TICK(); k_finish_sum<<<1, 256, 0, st>>>(part, norm2);
}

void maxpy(const double* Z, int64_t ldz, int m, const double* y, double* x, int64_t n, cudaStream_t st) {
  PS_TICK(); k_maxpy<<<kVecBlocks, 256, 0, st>>>(Z, ldz, m, y, x, n);
}
void finish_sum(const double* part, double* out, cudaStream_t st) { PS_TICK(); k_finish_sum<<<1, 256, 0, st>>>(part, out); }
void scale_vec(const double* x, double* y, int64_t n, const double* scale, cudaStream_t st) {
  PS_TICK(); k_scale<<<kVecBlocks, 256, 0, st>>>(x, y, n, scale);
}
void fill_zero(double* x, int64_t n, cudaStream_t st) { PS_TICK(); k_zero<<<kVecBlocks, 256, 0, st>>>(x, n); }

ps_status mgs_grid(int* blocks) {
  // blocks[i]: co-resident CTAs of the sweep width 1 << i (1, 2, 4, 8), 0 without cooperative launch
  int dev = 0, sms = 0, coop = 0;
  PS_CUDA(cudaGetDevice(&dev));
  PS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  PS_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  const void* fns[4] = {(const void*)k_mgs<1>, (const void*)k_mgs<2>, (const void*)k_mgs<4>, (const void*)k_mgs<8>};
  for (int i = 0; i < 4; ++i) {
    int occ = 0;
    PS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fns[i], kMgsThreads, 0));
    blocks[i] = coop ? sms * std::min(occ, 4) : 0;
  }
  return PS_OK;
}

int mgs_gram_stride() { return kS; }
int mgs_partials() { return 4 * kS; }

bool mgs_step(const double* V, int64_t ldv, int j, double* w, int64_t n, KrylovState& K, double* part,
              const int* blocks_by_sweep,
              unsigned long long* bar, unsigned long long* base, int64_t limit, int stall, int sweep,
              cudaStream_t st) {
  const int S = sweep >= 8 ? 8 : sweep >= 4 ? 4 : sweep >= 2 ? 2 : 1;
  int blocks = blocks_by_sweep[S == 8 ? 3 : S == 4 ? 2 : S == 2 ? 1 : 0];
  if (blocks <= 0) return false;
  // small systems use fewer CTAs (at least 16 rows per thread) so that concurrent requests overlap
  int64_t want = (n + int64_t(kMgsThreads) * 16 - 1) / (int64_t(kMgsThreads) * 16);
  if (want < blocks) blocks = int(want < 1 ? 1 : want);
  // rows in pairs: 16-byte aligned columns an even ldv apart, and pair indices that stay in int range
  const int64_t n2l = (n + 1) / 2;
  if ((ldv & 1) || ldv < 2 * n2l || (reinterpret_cast<uintptr_t>(V) & 15) || (reinterpret_cast<uintptr_t>(w) & 15) ||
      n2l + int64_t(blocks) * kMgsThreads > int64_t(INT32_MAX))
    return false;
  int n2 = int(n2l);
  unsigned long long b0 = *base;
  double* h = K.h1;
  double* Gm = K.gram;
  double* sc = K.sc;
  int* flag = K.flag;
  void* args[] = {&V, &ldv, &j, &w, &n2, &h, &Gm, &sc, &flag, &part, &bar, &b0, &limit, &stall};
  const void* fn = S == 8 ? (const void*)k_mgs<8> : S == 4 ? (const void*)k_mgs<4> : S == 2 ? (const void*)k_mgs<2>
                                                                                     : (const void*)k_mgs<1>;
  if (cudaLaunchCooperativeKernel(fn, blocks, kMgsThreads, args, 0, st) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  PS_TICK();
  *base = b0 + (unsigned long long)(j / S + 2) * blocks;
  return true;
}

void arnoldi_check(KrylovState& K, cudaStream_t st) { PS_TICK(); k_arnoldi_check<<<1, 1, 0, st>>>(K.sc, K.flag); }
void arnoldi_finish(KrylovState& K, int m, int j, cudaStream_t st) {
  PS_TICK(); k_arnoldi_finish<<<1, 1, 0, st>>>(K.H, K.cs, K.sn, K.g, K.h1, K.h2, K.sc, K.flag, m, j);
}
void cycle_start(KrylovState& K, int m, cudaStream_t st) { PS_TICK(); k_cycle_start<<<1, 1, 0, st>>>(K.g, K.sc, m); }
void hessenberg_solve(KrylovState& K, int m, int k, cudaStream_t st) { PS_TICK(); k_hsolve<<<1, 1, 0, st>>>(K.H, K.g, K.y, m, k); }

}  // namespace ps_internal
