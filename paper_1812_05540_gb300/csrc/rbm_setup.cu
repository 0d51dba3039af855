// Setup of the rigid-body-mode smoothed-aggregation hierarchy (see rbm.cuh).  Compiled without
// floating-point contraction; every sum runs in a fixed order (ascending block column, then ascending entry
// index), so the aggregates and operators reproduce the plain sequential definition bit for bit.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "rbm.cuh"

namespace ps_internal {
namespace {

constexpr int kMaxRowAgg = 512;    // distinct aggregates among the block columns of one row of A

// the six rigid-body modes at node I: translations along x, y, z and rotations about the axes through the
// grid's centre, (0, -z, y), (z, 0, -x), (-y, x, 0), coordinates in cell widths; rows (x, y, z) of 6
__global__ void k_rbm_modes(int nx, int ny, int nz, int64_t nn, double* __restrict__ B) {
  const int64_t I = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (I >= nn) return;
  const int64_t i = I % (nx + 1), j = (I / (nx + 1)) % (ny + 1), k = I / (int64_t(nx + 1) * (ny + 1));
  const double x = double(i) - 0.5 * nx, y = double(j) - 0.5 * ny, z = double(k) - 0.5 * nz;
  double* r = B + I * 3 * kRbmModes;
  for (int e = 0; e < 3 * kRbmModes; ++e) r[e] = 0.0;
  r[0 * 6 + 0] = 1.0; r[1 * 6 + 1] = 1.0; r[2 * 6 + 2] = 1.0;
  r[1 * 6 + 3] = -z; r[2 * 6 + 3] = y;
  r[0 * 6 + 4] = z;  r[2 * 6 + 4] = -x;
  r[0 * 6 + 5] = -y; r[1 * 6 + 5] = x;
}

// strength value of each block: its Frobenius norm (entries in row-major order)
__global__ void k_block_norm(int64_t nnzb, int bs, const double* __restrict__ v, double* __restrict__ s) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= nnzb) return;
  double a = 0.0;
  for (int e = 0; e < bs; ++e) a = a + v[q * bs + e] * v[q * bs + e];
  s[q] = sqrt(a);
}

// point diagonal, and the Gershgorin ratio sum_j |a_ij| / |a_ii| of each point row
__global__ void k_block_diag_gersh(int64_t n, int b, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                   const double* __restrict__ v, double* __restrict__ dg, double* __restrict__ ratio) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n * b) return;
  const int64_t i = t / b;
  const int a = int(t % b);
  double s = 0.0, d = 0.0;
  for (int32_t q = rp[i]; q < rp[i + 1]; ++q)
    for (int e = 0; e < b; ++e) {
      const double x = v[(int64_t(q) * b + a) * b + e];
      s = s + fabs(x);
      if (ci[q] == i && e == a) d = x;
    }
  dg[t] = d;
  ratio[t] = s / fabs(d);
}

// block rows whose off-diagonal blocks are all zero (Dirichlet nodes): no prolongator row
__global__ void k_block_excl(int64_t n, int b, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             const double* __restrict__ v, uint8_t* __restrict__ excl) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint8_t ex = 1;
  for (int32_t q = rp[i]; q < rp[i + 1]; ++q)
    if (ci[q] != i)
      for (int e = 0; e < b * b; ++e)
        if (v[int64_t(q) * b * b + e] != 0.0) ex = 0;
  excl[i] = ex;
}

__global__ void k_count_by(int64_t n, const int32_t* __restrict__ key, int32_t* __restrict__ cnt) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n && key[i] >= 0) atomicAdd(&cnt[key[i]], 1);
}
__global__ void k_fill_by(int64_t n, const int32_t* __restrict__ key, int32_t* __restrict__ cursor,
                          int32_t* __restrict__ out) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n && key[i] >= 0) out[atomicAdd(&cursor[key[i]], 1)] = int32_t(i);
}
// each group's entries in ascending order (insertion sort; groups are small)
__global__ void k_sort_groups(int64_t ng, const int32_t* __restrict__ off, int32_t* __restrict__ x) {
  const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (g >= ng) return;
  for (int32_t p = off[g] + 1; p < off[g + 1]; ++p) {
    const int32_t v = x[p];
    int32_t q = p - 1;
    while (q >= off[g] && x[q] > v) {
      x[q + 1] = x[q];
      --q;
    }
    x[q + 1] = v;
  }
}

// Tentative prolongator of aggregate a: the modes on its nodes (ascending, b rows each) factored B_a = Q R by
// modified Gram-Schmidt, columns in order; a column whose remainder is at most 1e-10 of its norm gives a zero
// column of Q and a zero row of R.  Q is formed in place in Pt (which holds B's rows on entry), R goes to Bc.
__global__ void k_tentative(int64_t nagg, int b, const int32_t* __restrict__ moff, const int32_t* __restrict__ mem,
                            double* __restrict__ Pt, double* __restrict__ Bc) {
  const int64_t a = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (a >= nagg) return;
  const int32_t m0 = moff[a], m1 = moff[a + 1];
  const int64_t rows = int64_t(m1 - m0) * b;
  auto at = [&](int64_t r, int k) -> double& { return Pt[(int64_t(mem[m0 + r / b]) * b + r % b) * kRbmModes + k]; };
  double R[kRbmModes][kRbmModes];
  for (int r = 0; r < kRbmModes; ++r)
    for (int k = 0; k < kRbmModes; ++k) R[r][k] = 0.0;
  for (int k = 0; k < kRbmModes; ++k) {
    double n0 = 0.0;
    for (int64_t r = 0; r < rows; ++r) n0 = n0 + at(r, k) * at(r, k);
    n0 = sqrt(n0);
    for (int j = 0; j < k; ++j) {
      double c = 0.0;
      for (int64_t r = 0; r < rows; ++r) c = c + at(r, j) * at(r, k);
      R[j][k] = c;
      for (int64_t r = 0; r < rows; ++r) at(r, k) = at(r, k) - c * at(r, j);
    }
    double nk = 0.0;
    for (int64_t r = 0; r < rows; ++r) nk = nk + at(r, k) * at(r, k);
    nk = sqrt(nk);
    if (nk > 1e-10 * n0 && nk > 0.0) {
      R[k][k] = nk;
      for (int64_t r = 0; r < rows; ++r) at(r, k) = at(r, k) / nk;
    } else {
      for (int64_t r = 0; r < rows; ++r) at(r, k) = 0.0;
    }
  }
  for (int r = 0; r < kRbmModes; ++r)
    for (int k = 0; k < kRbmModes; ++k) Bc[(a * kRbmModes + r) * kRbmModes + k] = R[r][k];
}

// copy the modes of aggregated nodes into the Q work space (rows of other nodes stay zero)
__global__ void k_modes_to_pt(int64_t n, int b, const int32_t* __restrict__ agg, const double* __restrict__ B,
                              double* __restrict__ Pt) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n * b * kRbmModes) return;
  const int64_t i = t / (b * kRbmModes);
  Pt[t] = agg[i] >= 0 ? B[t] : 0.0;
}

// distinct aggregates of the block columns of row i, ascending; -1 when there are more than cap
__device__ int row_aggs(int64_t i, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                        const int32_t* __restrict__ agg, int32_t* list, int cap) {
  int c = 0;
  for (int32_t q = rp[i]; q < rp[i + 1]; ++q) {
    const int32_t a = agg[ci[q]];
    if (a < 0) continue;
    int p = c;
    while (p > 0 && list[p - 1] > a) --p;
    if (p > 0 && list[p - 1] == a) continue;
    if (c == cap) return -1;
    for (int s = c; s > p; --s) list[s] = list[s - 1];
    list[p] = a;
    ++c;
  }
  return c;
}

__global__ void k_p_count(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const int32_t* __restrict__ agg, const uint8_t* __restrict__ excl, int32_t* __restrict__ cnt,
                          int* __restrict__ err) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t list[kMaxRowAgg];
  int c = excl[i] ? 0 : row_aggs(i, rp, ci, agg, list, kMaxRowAgg);
  if (c < 0) {
    atomicExch(err, 1);
    c = 0;
  }
  cnt[i] = c;
}

// P = (I - omega D^{-1} A) P_tent with B x 6 blocks, one warp per row: block (i, a) = [a == agg(i)] P_tent(i)
// - (omega / d_i) S, with S the sum over the row's block columns j in aggregate a (ascending) of A_ij P_tent(j).
// Lane 0 lists the row's aggregates into pci (the pattern); then for each aggregate the lanes take the entries
// (r, k) of its block (two per lane where B = 6), each block-product entry summed over its inner index in
// ascending order.
template <int B>
__global__ void __launch_bounds__(256) k_p_fill_w(int64_t n, const int32_t* __restrict__ rp,
                                                  const int32_t* __restrict__ ci, const double* __restrict__ v,
                                                  const int32_t* __restrict__ agg, const uint8_t* __restrict__ excl,
                                                  const double* __restrict__ Pt, const double* __restrict__ dg,
                                                  double omega, const int32_t* __restrict__ prp,
                                                  int32_t* __restrict__ pci, double* __restrict__ pv) {
  constexpr int NE = B * kRbmModes;
  const int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n || excl[i]) return;
  const int32_t o0 = prp[i], c = prp[i + 1] - prp[i];
  if (lane == 0) {
    int32_t list[kMaxRowAgg];
    const int cc = row_aggs(i, rp, ci, agg, list, kMaxRowAgg);
    if (cc == c)
      for (int s = 0; s < c; ++s) pci[o0 + s] = list[s];
    else
      for (int s = 0; s < c; ++s) pci[o0 + s] = -1;  // overflow, reported by k_p_count
  }
  __syncwarp();
  const int32_t q0 = rp[i], q1 = rp[i + 1];
  const int t0 = lane, t1 = lane + 32;
  const int r0 = t0 / kRbmModes, k0 = t0 % kRbmModes, r1 = t1 / kRbmModes, k1 = t1 % kRbmModes;
  const int ai = agg[i];
  for (int s = 0; s < c; ++s) {
    const int32_t a = pci[o0 + s];
    if (a < 0) return;
    double S0 = 0.0, S1 = 0.0;
    for (int32_t q = q0; q < q1; ++q) {
      const int64_t j = ci[q];
      if (agg[j] != a) continue;  // the same for every lane
      const double* vq = v + int64_t(q) * B * B;
      const double* pj = Pt + j * B * kRbmModes;
      if (t0 < NE) {
        double p = 0.0;
#pragma unroll
        for (int e = 0; e < B; ++e) p = p + vq[r0 * B + e] * pj[e * kRbmModes + k0];
        S0 = S0 + p;
      }
      if (t1 < NE) {
        double p = 0.0;
#pragma unroll
        for (int e = 0; e < B; ++e) p = p + vq[r1 * B + e] * pj[e * kRbmModes + k1];
        S1 = S1 + p;
      }
    }
    const int64_t o = o0 + s;
    if (t0 < NE) {
      const double delta = a == ai ? Pt[(i * B + r0) * kRbmModes + k0] : 0.0;
      pv[(o * B + r0) * kRbmModes + k0] = delta - (omega / dg[i * B + r0]) * S0;
    }
    if (t1 < NE) {
      const double delta = a == ai ? Pt[(i * B + r1) * kRbmModes + k1] : 0.0;
      pv[(o * B + r1) * kRbmModes + k1] = delta - (omega / dg[i * B + r1]) * S1;
    }
  }
}

// transpose of a block matrix: entries grouped by column (cursor from the column offsets), then ordered by
// row within each column, then the transposed blocks written out
__global__ void k_t_count(int64_t nnz, const int32_t* __restrict__ ci, int32_t* __restrict__ cnt) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q < nnz) atomicAdd(&cnt[ci[q]], 1);
}
__global__ void k_t_fill(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                         int32_t* __restrict__ cursor, int32_t* __restrict__ src) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int32_t q = rp[i]; q < rp[i + 1]; ++q) src[atomicAdd(&cursor[ci[q]], 1)] = q;
}
// within each output row the source entries ascending (a source entry's position orders it by row)
__global__ void k_t_values(int64_t m, const int32_t* __restrict__ trp, const int32_t* __restrict__ src, int br,
                           int bc, const int32_t* __restrict__ rowof, const double* __restrict__ v,
                           int32_t* __restrict__ tci, double* __restrict__ tv) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= m) return;
  for (int32_t p = trp[j]; p < trp[j + 1]; ++p) {
    const int32_t q = src[p];
    tci[p] = rowof[q];
    for (int a = 0; a < br; ++a)
      for (int e = 0; e < bc; ++e) tv[(int64_t(p) * bc + e) * br + a] = v[(int64_t(q) * br + a) * bc + e];
  }
}
__global__ void k_row_of(int64_t n, const int32_t* __restrict__ rp, int32_t* __restrict__ rowof) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int32_t q = rp[i]; q < rp[i + 1]; ++q) rowof[q] = int32_t(i);
}

// C = X Y with BR x BK blocks of X and BK x BC blocks of Y on C's given sorted pattern, one warp per row of C:
// block (i, j) sums X_ik Y_kj over ascending k (the order of X's row), each entry of a product summing its
// inner index in ascending order by fused multiply-adds.  The warp walks the row's X entries in order; the
// products of one X entry with its Y row go to distinct output blocks, so up to G of them run side by side,
// the lanes taking their entries (G * BR * BC of them) in turn: every output entry is still accumulated by one
// lane at a time, in order, and the lanes stay busy where one 6 x 6 product would leave 28 of 64 slots idle.
template <int BR, int BK, int BC>
__global__ void __launch_bounds__(256) k_bprod(int64_t n, const int32_t* __restrict__ xrp,
                                               const int32_t* __restrict__ xci, const double* __restrict__ xv,
                                               const int32_t* __restrict__ yrp, const int32_t* __restrict__ yci,
                                               const double* __restrict__ yv, const int32_t* __restrict__ crp,
                                               const int32_t* __restrict__ cci, double* __restrict__ cv) {
  constexpr int NE = BR * BC;
  constexpr int G = NE % 32 == 0 ? 1 : (32 % NE == 0 ? 32 / NE : 8);  // products side by side
  const int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  __shared__ int32_t spos_all[8][G];  // output block of each product of a group, per warp (256 threads)
  int32_t* spos = spos_all[(threadIdx.x >> 5) & 7];
  const int32_t c0 = crp[i], c1 = crp[i + 1];
  for (int64_t e = int64_t(c0) * NE + lane; e < int64_t(c1) * NE; e += 32) cv[e] = 0.0;
  __syncwarp();
  for (int32_t q = xrp[i]; q < xrp[i + 1]; ++q) {
    const int32_t k = xci[q];
    const double* X = xv + int64_t(q) * BR * BK;
    const int32_t r1 = yrp[k + 1];
    for (int32_t r0 = yrp[k]; r0 < r1; r0 += G) {
      // lane g < G finds the output block of product r0 + g
      int32_t pos = -1;
      if (lane < G && r0 + lane < r1) {
        const int32_t j = yci[r0 + lane];
        int32_t lo = c0, hi = c1;
        while (lo < hi) {
          const int32_t md = (lo + hi) >> 1;
          if (cci[md] < j) lo = md + 1;
          else hi = md;
        }
        pos = lo < c1 ? lo : -1;  // -1: not in the pattern (cannot happen for a pattern of X Y)
      }
      if (lane < G) spos[lane] = pos;
      __syncwarp();
      for (int t = lane; t < G * NE; t += 32) {
        const int g = t / NE, e = t - g * NE;
        const int32_t pg = spos[g];
        if (r0 + g >= r1 || pg < 0) continue;
        const int a = e / BC, c = e % BC;
        const double* Y = yv + int64_t(r0 + g) * BK * BC;
        double p = 0.0;
#pragma unroll
        for (int f = 0; f < BK; ++f) p = fma(X[a * BK + f], Y[f * BC + c], p);
        double* C = cv + int64_t(pg) * NE;
        C[e] = C[e] + p;
      }
      __syncwarp();
    }
  }
}

// a zero diagonal entry of a coarse operator (a mode its aggregate cannot represent) becomes one
__global__ void k_fix_diag(int64_t n, int b, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           double* __restrict__ v) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int32_t q = rp[i]; q < rp[i + 1]; ++q)
    if (ci[q] == i)
      for (int k = 0; k < b; ++k)
        if (v[(int64_t(q) * b + k) * b + k] == 0.0) v[(int64_t(q) * b + k) * b + k] = 1.0;
}

// dense (n b) x (n b) copy of a block operator, and the identity in inv
__global__ void k_block_dense(int64_t n, int b, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                              const double* __restrict__ v, double* __restrict__ M, double* __restrict__ inv) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t N = n * b;
  if (t >= N) return;
  const int64_t i = t / b;
  const int a = int(t % b);
  inv[t * N + t] = 1.0;
  for (int32_t q = rp[i]; q < rp[i + 1]; ++q)
    for (int e = 0; e < b; ++e) M[t * N + int64_t(ci[q]) * b + e] = v[(int64_t(q) * b + a) * b + e];
}

__global__ void k_to_f32r(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < n) b[t] = float(a[t]);
}

}  // namespace

ps_status rbm_build(Arena& ar, Rbm& H, int nx, int ny, int nz, int64_t nnzb0, const int32_t* rp0, const int32_t* ci0,
                    const double* v0, double theta, int coarse_max, int max_levels, bool mixed, cudaStream_t st) {
  H.L.clear();
  const int64_t nn = int64_t(nx + 1) * (ny + 1) * (nz + 1);
  int* err;
  PS_TRY(ar.alloc(&err, 1));
  PS_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  {
    RbmLevel L0;
    L0.n = nn; L0.b = 3; L0.nnzb = nnzb0;
    L0.rp = const_cast<int32_t*>(rp0); L0.ci = const_cast<int32_t*>(ci0); L0.v = const_cast<double*>(v0);
    PS_TRY(ar.alloc(&L0.B, size_t(nn) * 3 * kRbmModes));
    PS_TICK(); k_rbm_modes<<<grid_for(nn, 256), 256, 0, st>>>(nx, ny, nz, nn, L0.B);
    H.L.push_back(L0);
  }
  for (int l = 0;; ++l) {
    RbmLevel& lev = H.L[l];
    const int64_t n = lev.n, nnzb = lev.nnzb;
    const int b = lev.b;
    lev.lanes = lanes_for(double(nnzb) / double(n > 0 ? n : 1));
    // coarse_max counts nodes: a level is coarsest at 3 coarse_max unknowns, as many as coarse_max nodes carry
    bool coarsest = n * b <= int64_t(3) * coarse_max || l + 1 >= max_levels;
    uint8_t* excl = nullptr;
    if (!coarsest) {
      double* s;
      PS_TRY(ar.alloc(&s, nnzb));
      PS_TICK(); k_block_norm<<<grid_for(nnzb, 256), 256, 0, st>>>(nnzb, b * b, lev.v, s);
      PS_TRY(amg_aggregate_scalar(ar, n, nnzb, lev.rp, lev.ci, s, theta, l, &lev.agg, &lev.nagg, &excl, st));
      ar.release(s);
      if (lev.nagg == 0 || double(n) / double(lev.nagg) < 1.2) coarsest = true;
    }
    double* ratio;
    PS_TRY(ar.alloc(&lev.dg, n * b));
    PS_TRY(ar.alloc(&ratio, n * b));
    PS_TICK(); k_block_diag_gersh<<<grid_for(n * b, 256), 256, 0, st>>>(n, b, lev.rp, lev.ci, lev.v, lev.dg, ratio);
    if (coarsest) {
      ar.release(ratio);
      if (excl) ar.release(excl);
      if (lev.agg) { ar.release(lev.agg); lev.agg = nullptr; }
      lev.nagg = 0;
      lev.coarsest = true;
      const int64_t N = n * b;
      if (N > 12000) {
        set_reason("rigid-body-mode hierarchy: coarsening stalled at level %d with %lld unknowns", l, (long long)N);
        return PS_ERR_INVALID;
      }
      double* M;
      PS_TRY(ar.alloc(&M, size_t(N) * N));
      PS_TRY(ar.alloc(&lev.inv, size_t(N) * N));
      PS_CUDA(cudaMemsetAsync(M, 0, sizeof(double) * N * N, st));
      PS_CUDA(cudaMemsetAsync(lev.inv, 0, sizeof(double) * N * N, st));
      PS_TICK(); k_block_dense<<<grid_for(N, 128), 128, 0, st>>>(n, b, lev.rp, lev.ci, lev.v, M, lev.inv);
      PS_CUDA(cudaGetLastError());
      PS_TRY(amg_dense_inverse(ar, N, M, lev.inv, st));
      ar.release(M);
      if (mixed) {
        PS_TRY(ar.alloc(&lev.dgf, n * b));
        PS_TICK(); k_to_f32r<<<grid_for(n * b, 256), 256, 0, st>>>(lev.dg, lev.dgf, n * b);
      }
      break;
    }
    double* dmax;
    PS_TRY(ar.alloc(&dmax, 1));
    PS_TRY(max_f64(ar, ratio, n * b, dmax, st));
    PS_CUDA(cudaMemcpyAsync(&lev.lam, dmax, sizeof(double), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    ar.release(dmax);
    ar.release(ratio);
    const double omega = (4.0 / 3.0) / lev.lam;
    const int64_t na = lev.nagg;
    // aggregate members, ascending
    int32_t *cnt, *moff, *cursor, *mem;
    PS_TRY(ar.alloc(&cnt, na + 1));
    PS_TRY(ar.alloc(&moff, na + 1));
    PS_TRY(ar.alloc(&cursor, na + 1));
    PS_TRY(ar.alloc(&mem, n + 1));
    PS_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (na + 1), st));
    PS_TICK(); k_count_by<<<grid_for(n, 256), 256, 0, st>>>(n, lev.agg, cnt);
    PS_TRY(scan_i32(ar, cnt, moff, na, nullptr, st));
    PS_CUDA(cudaMemcpyAsync(cursor, moff, sizeof(int32_t) * na, cudaMemcpyDeviceToDevice, st));
    PS_TICK(); k_fill_by<<<grid_for(n, 256), 256, 0, st>>>(n, lev.agg, cursor, mem);
    PS_TICK(); k_sort_groups<<<grid_for(na, 128), 128, 0, st>>>(na, moff, mem);
    // tentative prolongator and coarse modes
    double* Bc;
    PS_TRY(ar.alloc(&lev.Pt, size_t(n) * b * kRbmModes));
    PS_TRY(ar.alloc(&Bc, size_t(na) * kRbmModes * kRbmModes));
    PS_TICK(); k_modes_to_pt<<<grid_for(n * b * kRbmModes, 256), 256, 0, st>>>(n, b, lev.agg, lev.B, lev.Pt);
    PS_TICK(); k_tentative<<<grid_for(na, 64), 64, 0, st>>>(na, b, moff, mem, lev.Pt, Bc);
    PS_CUDA(cudaGetLastError());
    ar.release(cnt); ar.release(cursor); ar.release(mem); ar.release(moff);
    // smoothed prolongator
    uint8_t* bex;
    PS_TRY(ar.alloc(&bex, n));
    PS_TICK(); k_block_excl<<<grid_for(n, 256), 256, 0, st>>>(n, b, lev.rp, lev.ci, lev.v, bex);
    int32_t* pc;
    PS_TRY(ar.alloc(&pc, n + 1));
    PS_TRY(ar.alloc(&lev.prp, n + 1));
    PS_TICK(); k_p_count<<<grid_for(n, 128), 128, 0, st>>>(n, lev.rp, lev.ci, lev.agg, bex, pc, err);
    int32_t pnnz = 0;
    PS_TRY(scan_i32(ar, pc, lev.prp, n, &pnnz, st));
    lev.pnnzb = pnnz;
    PS_TRY(ar.alloc(&lev.pci, size_t(pnnz) + 1));
    PS_TRY(ar.alloc(&lev.pv, (size_t(pnnz) + 1) * b * kRbmModes));
    if (b == 3) {
      PS_TICK(); k_p_fill_w<3><<<grid_for(n * 32, 256), 256, 0, st>>>(n, lev.rp, lev.ci, lev.v, lev.agg, bex, lev.Pt,
                                                                     lev.dg, omega, lev.prp, lev.pci, lev.pv);
    } else if (b == kRbmModes) {
      PS_TICK(); k_p_fill_w<kRbmModes><<<grid_for(n * 32, 256), 256, 0, st>>>(n, lev.rp, lev.ci, lev.v, lev.agg, bex,
                                                                             lev.Pt, lev.dg, omega, lev.prp, lev.pci,
                                                                             lev.pv);
    } else {
      set_reason("rigid-body-mode level with %d x %d blocks", b, b);
      return PS_ERR_INVALID;
    }
    PS_CUDA(cudaGetLastError());
    ar.release(pc); ar.release(bex);
    if (excl) ar.release(excl);
    lev.plane = lanes_for(double(pnnz) / double(n));
    // R = P^T
    int32_t *tc, *tcur, *src, *rowof;
    PS_TRY(ar.alloc(&tc, na + 1));
    PS_TRY(ar.alloc(&lev.rrp, na + 1));
    PS_TRY(ar.alloc(&tcur, na + 1));
    PS_TRY(ar.alloc(&src, size_t(pnnz) + 1));
    PS_TRY(ar.alloc(&rowof, size_t(pnnz) + 1));
    PS_TRY(ar.alloc(&lev.rci, size_t(pnnz) + 1));
    PS_TRY(ar.alloc(&lev.rv, (size_t(pnnz) + 1) * b * kRbmModes));
    PS_CUDA(cudaMemsetAsync(tc, 0, sizeof(int32_t) * (na + 1), st));
    PS_TICK(); k_t_count<<<grid_for(pnnz, 256), 256, 0, st>>>(pnnz, lev.pci, tc);
    PS_TRY(scan_i32(ar, tc, lev.rrp, na, nullptr, st));
    PS_CUDA(cudaMemcpyAsync(tcur, lev.rrp, sizeof(int32_t) * na, cudaMemcpyDeviceToDevice, st));
    PS_TICK(); k_t_fill<<<grid_for(n, 256), 256, 0, st>>>(n, lev.prp, lev.pci, tcur, src);
    PS_TICK(); k_sort_groups<<<grid_for(na, 128), 128, 0, st>>>(na, lev.rrp, src);
    PS_TICK(); k_row_of<<<grid_for(n, 256), 256, 0, st>>>(n, lev.prp, rowof);
    PS_TICK(); k_t_values<<<grid_for(na, 128), 128, 0, st>>>(na, lev.rrp, src, b, kRbmModes, rowof, lev.pv, lev.rci,
                                                               lev.rv);
    PS_CUDA(cudaGetLastError());
    ar.release(tc); ar.release(tcur); ar.release(src); ar.release(rowof);
    lev.rlane = lanes_for(double(pnnz) / double(na));
    // A_c = R (A P): patterns by the SDC hierarchy's SpGEMM, block values by k_bprod
    int32_t *aprp, *apci;
    int64_t apnnz = 0;
    PS_TRY(amg_spgemm_pattern(ar, n, na, lev.rp, lev.ci, nnzb, lev.prp, lev.pci, pnnz, &aprp, &apci, &apnnz, st));
    double* apv;
    PS_TRY(ar.alloc(&apv, (size_t(apnnz) + 1) * b * kRbmModes));
    if (b == 3) {
      PS_TICK(); k_bprod<3, 3, kRbmModes><<<grid_for(n * 32, 256), 256, 0, st>>>(n, lev.rp, lev.ci, lev.v, lev.prp, lev.pci,
                                                                           lev.pv, aprp, apci, apv);
    } else {
      PS_TICK(); k_bprod<6, 6, kRbmModes><<<grid_for(n * 32, 256), 256, 0, st>>>(n, lev.rp, lev.ci, lev.v, lev.prp, lev.pci,
                                                                           lev.pv, aprp, apci, apv);
    }
    RbmLevel C;
    C.n = na; C.b = kRbmModes; C.B = Bc;
    int64_t cnnz = 0;
    PS_TRY(amg_spgemm_pattern(ar, na, na, lev.rrp, lev.rci, pnnz, aprp, apci, apnnz, &C.rp, &C.ci, &cnnz, st));
    C.nnzb = cnnz;
    PS_TRY(ar.alloc(&C.v, (size_t(cnnz) + 1) * kRbmModes * kRbmModes));
    if (b == 3) {
      PS_TICK(); k_bprod<kRbmModes, 3, kRbmModes><<<grid_for(na * 32, 256), 256, 0, st>>>(na, lev.rrp, lev.rci, lev.rv, aprp,
                                                                                   apci, apv, C.rp, C.ci, C.v);
    } else {
      PS_TICK(); k_bprod<kRbmModes, 6, kRbmModes><<<grid_for(na * 32, 256), 256, 0, st>>>(na, lev.rrp, lev.rci, lev.rv, aprp,
                                                                                   apci, apv, C.rp, C.ci, C.v);
    }
    PS_TICK(); k_fix_diag<<<grid_for(na, 256), 256, 0, st>>>(na, kRbmModes, C.rp, C.ci, C.v);
    PS_CUDA(cudaGetLastError());
    ar.release(aprp); ar.release(apci); ar.release(apv);
    int herr = 0;
    PS_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    if (herr) {
      set_reason("rigid-body-mode hierarchy: a row of level %d touches more aggregates than the setup kernels hold", l);
      return PS_ERR_INVALID;
    }
    if (mixed) {
      PS_TRY(ar.alloc(&lev.vf, size_t(nnzb) * b * b));
      PS_TRY(ar.alloc(&lev.dgf, n * b));
      PS_TRY(ar.alloc(&lev.pvf, (size_t(pnnz) + 1) * b * kRbmModes));
      PS_TRY(ar.alloc(&lev.rvf, (size_t(pnnz) + 1) * b * kRbmModes));
      PS_TICK(); k_to_f32r<<<grid_for(nnzb * b * b, 256), 256, 0, st>>>(lev.v, lev.vf, nnzb * b * b);
      PS_TICK(); k_to_f32r<<<grid_for(n * b, 256), 256, 0, st>>>(lev.dg, lev.dgf, n * b);
      PS_TICK(); k_to_f32r<<<grid_for(int64_t(pnnz) * b * kRbmModes, 256), 256, 0, st>>>(lev.pv, lev.pvf,
                                                                                        int64_t(pnnz) * b * kRbmModes);
      PS_TICK(); k_to_f32r<<<grid_for(int64_t(pnnz) * b * kRbmModes, 256), 256, 0, st>>>(lev.rv, lev.rvf,
                                                                                        int64_t(pnnz) * b * kRbmModes);
      PS_CUDA(cudaGetLastError());
    }
    H.L.push_back(C);
    theta *= 0.5;
  }
  ar.release(err);
  return PS_OK;
}

void rbm_release_graph(Rbm& H) {
  if (H.gexec) cudaGraphExecDestroy(H.gexec);
  H.gexec = nullptr;
  H.gb = nullptr;
  H.gx = nullptr;
  H.gst = nullptr;
  H.gnodes = 0;
}

}  // namespace ps_internal
