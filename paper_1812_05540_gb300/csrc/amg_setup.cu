// AMG setup kernels: strength of connection, distance-2 maximal independent
// set, aggregation, smoothed prolongator, transpose, Galerkin product by a
// shared-memory SpGEMM, and the dense inverse of the coarsest operator.
//
// This translation unit is compiled without floating-point contraction and
// every floating-point sum is taken in a fixed order (ascending column / inner
// index), so the aggregates and coarse operators are reproducible bit for bit.
#include <algorithm>
#include <atomic>
#include <climits>
#include <mutex>
#include <cmath>
#include <cstdio>

#include <type_traits>

#include "amg.cuh"
#include "gridsync.cuh"

#include <cooperative_groups.h>

namespace ps_internal {
namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
// MIS priority: (hash(level, i), i), unique per node
__device__ __forceinline__ int64_t mis_key(int64_t i, int level) {
  uint64_t h = mix64((uint64_t(level) << 32) | uint64_t(i));
  return (int64_t(h >> 33) << 32) | i;
}

template <int NC>
__device__ __forceinline__ double abar(const double* v, int64_t q) {
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < NC; ++c) s = s + fabs(v[q * NC + c]);
  return s;
}

template <int NC>
__global__ void k_diag_excl(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            const double* __restrict__ v, double* __restrict__ dgbar, uint8_t* __restrict__ excl,
                            double* __restrict__ dg) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double d = 0.0;
  uint8_t ex = 1;
  for (int32_t q = rp[i]; q < rp[i + 1]; ++q) {
    if (ci[q] == i) {
      d = abar<NC>(v, q);
      for (int c = 0; c < NC; ++c) dg[i * NC + c] = v[int64_t(q) * NC + c];
    } else {
      for (int c = 0; c < NC; ++c)
        if (v[int64_t(q) * NC + c] != 0.0) ex = 0;
    }
  }
  dgbar[i] = d;
  excl[i] = ex;
}

__device__ __forceinline__ int32_t find_col(const int32_t* __restrict__ ci, int32_t lo, int32_t hi, int32_t j) {
  while (lo < hi) {
    int32_t m = (lo + hi) >> 1;
    if (ci[m] < j) lo = m + 1;
    else hi = m;
  }
  return lo;
}

// symmetric strength graph: i~j if max(abar_ij, abar_ji) >= theta sqrt(abar_ii abar_jj); kStrLanes
// threads per row.  Both entries of a pair get the same bits (max and the product under the root are
// symmetric), so the lanes of row i decide the pairs of its entries above the diagonal and write both entries;
// an entry below the diagonal is decided by its own row only when its transposed entry is missing.  The
// columns of a row are sorted, so its entries above the diagonal are contiguous and the lanes stay busy.
constexpr int kStrLanes = 8;
template <int NC>
__device__ __forceinline__ void strength_pair(int64_t i, int32_t j, int32_t q, int32_t qt, bool has_t,
                                              const double* __restrict__ v, const double* __restrict__ dgbar,
                                              const uint8_t* __restrict__ excl, double theta,
                                              uint8_t* __restrict__ strong, double* __restrict__ wgt) {
  uint8_t s = 0;
  double w = 0.0;
  if (!excl[i] && !excl[j]) {
    const double aij = abar<NC>(v, q);
    const double aji = has_t ? abar<NC>(v, qt) : 0.0;
    const double t = aij > aji ? aij : aji;
    const double den = sqrt(dgbar[i] * dgbar[j]);
    if (t >= theta * den && t > 0.0) {
      s = 1;
      w = t / den;
    }
  }
  strong[q] = s;
  wgt[q] = w;
  if (has_t) {
    strong[qt] = s;
    wgt[qt] = w;
  }
}

template <int NC>
__global__ void k_strength(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const double* __restrict__ v, const double* __restrict__ dgbar,
                           const uint8_t* __restrict__ excl, double theta, uint8_t* __restrict__ strong,
                           double* __restrict__ wgt) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t i = t / kStrLanes;
  if (i >= n) return;
  const int sub = int(t % kStrLanes);
  const int32_t q0 = rp[i], q1 = rp[i + 1];
  const int32_t qd = find_col(ci, q0, q1, int32_t(i));  // first entry with column >= i
  const int32_t qu = (qd < q1 && ci[qd] == i) ? qd + 1 : qd;
  if (sub == 0 && qu != qd) {
    strong[qd] = 0;
    wgt[qd] = 0.0;
  }
  for (int32_t q = qu + sub; q < q1; q += kStrLanes) {
    const int32_t j = ci[q];
    const int32_t lo = rp[j], hi = rp[j + 1];
    const int32_t qt = find_col(ci, lo, hi, int32_t(i));
    strength_pair<NC>(i, j, q, qt, qt < hi && ci[qt] == i, v, dgbar, excl, theta, strong, wgt);
  }
  for (int32_t q = q0 + sub; q < qd; q += kStrLanes) {
    const int32_t j = ci[q];
    const int32_t lo = rp[j], hi = rp[j + 1];
    const int32_t qt = find_col(ci, lo, hi, int32_t(i));
    if (!(qt < hi && ci[qt] == i)) strength_pair<NC>(i, j, q, qt, false, v, dgbar, excl, theta, strong, wgt);
  }
}

// ---- distance-2 MIS rounds (state: 0 undecided, 1 root, 2 covered, 3 excluded) ----
// rows without a strong connection (identity rows included) are not aggregated:
// the smoother alone treats them (isolated-node rule of smoothed aggregation)
__global__ void k_mis_init(int64_t n, const int32_t* __restrict__ rp, const uint8_t* __restrict__ strong,
                           const uint8_t* __restrict__ excl, uint8_t* __restrict__ st) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  bool any = false;
  for (int32_t q = rp[i]; q < rp[i + 1]; ++q) any = any || strong[q];
  st[i] = (excl[i] || !any) ? 3 : 0;
}
// The four round kernels take kMisLanes threads per row: each lane scans a strided share of the row
// and the lanes combine by max (priorities) or by or (flags), which do not depend on the order, so the
// rounds decide exactly as one thread per row would.  Every lane reaches the shuffles; only lane 0
// of a row writes.
constexpr int kMisLanes = 8;
__device__ __forceinline__ int64_t group_max(int64_t v) {
#pragma unroll
  for (int o = kMisLanes / 2; o > 0; o >>= 1) {
    const int64_t u = __shfl_xor_sync(0xffffffffu, v, o, kMisLanes);
    v = u > v ? u : v;
  }
  return v;
}
__device__ __forceinline__ bool group_any(bool b) {
  const unsigned m = __ballot_sync(0xffffffffu, b);
  const int lane = int(threadIdx.x & 31);
  return ((m >> (lane & ~(kMisLanes - 1))) & ((1u << kMisLanes) - 1u)) != 0u;
}
// prev: the undecided flag of the previous round (null: none); a round after one that left no row
// undecided changes nothing, so its kernels return at once
#define MIS_ROW                                                      \
  if (prev && *prev == 0) return;                                    \
  const int64_t t_ = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; \
  const int64_t i = t_ / kMisLanes;                                  \
  const int sub = int(t_ % kMisLanes);                               \
  const bool act = i < n;

// the priority keys of a level, formed once per aggregation instead of per neighbour and round
__global__ void k_mis_keys(int64_t n, int level, int64_t* __restrict__ key) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) key[i] = mis_key(i, level);
}
__global__ void k_mis_m1(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                         const uint8_t* __restrict__ strong, const uint8_t* __restrict__ st,
                         const int64_t* __restrict__ key, int64_t* __restrict__ m1, const int32_t* __restrict__ prev) {
  MIS_ROW
  int64_t m = -1;
  if (act) {
    if (sub == 0 && st[i] == 0) m = key[i];
    for (int32_t q = rp[i] + sub; q < rp[i + 1]; q += kMisLanes)
      if (strong[q] && st[ci[q]] == 0) {
        const int64_t k = key[ci[q]];
        m = k > m ? k : m;
      }
  }
  m = group_max(m);
  if (act && sub == 0) m1[i] = m;
}
__global__ void k_mis_m2(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                         const uint8_t* __restrict__ strong, const int64_t* __restrict__ m1,
                         const int64_t* __restrict__ key, uint8_t* __restrict__ st, uint8_t* __restrict__ nr,
                         const int32_t* __restrict__ prev) {
  MIS_ROW
  int64_t m = -1;
  if (act) {
    if (sub == 0) m = m1[i];
    for (int32_t q = rp[i] + sub; q < rp[i + 1]; q += kMisLanes)
      if (strong[q]) {
        int64_t k = m1[ci[q]];
        m = k > m ? k : m;
      }
  }
  m = group_max(m);
  if (act && sub == 0) {
    uint8_t r = (st[i] == 0 && m == key[i]) ? 1 : 0;
    nr[i] = r;
    if (r) st[i] = 1;
  }
}
__global__ void k_mis_c1(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                         const uint8_t* __restrict__ strong, const uint8_t* __restrict__ nr,
                         uint8_t* __restrict__ c1, const int32_t* __restrict__ prev) {
  MIS_ROW
  bool c = false;
  if (act) {
    if (sub == 0) c = nr[i] != 0;
    for (int32_t q = rp[i] + sub; q < rp[i + 1]; q += kMisLanes)
      if (strong[q] && nr[ci[q]]) c = true;
  }
  c = group_any(c);
  if (act && sub == 0) c1[i] = c ? 1 : 0;
}
__global__ void k_mis_c2(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                         const uint8_t* __restrict__ strong, const uint8_t* __restrict__ c1,
                         uint8_t* __restrict__ st, int32_t* __restrict__ undecided, const int32_t* __restrict__ prev) {
  MIS_ROW
  const bool undec = act && st[i] == 0;
  bool c = false;
  if (undec) {
    if (sub == 0) c = c1[i] != 0;
    for (int32_t q = rp[i] + sub; q < rp[i + 1]; q += kMisLanes)
      if (strong[q] && c1[ci[q]]) c = true;
  }
  c = group_any(c);
  if (undec && sub == 0) {
    if (c) st[i] = 2;
    else *undecided = 1;  // the host only tests for zero: every writer stores the same value
  }
}
#undef MIS_ROW

__global__ void k_is_root(int64_t n, const uint8_t* __restrict__ st, int32_t* __restrict__ f) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) f[i] = st[i] == 1 ? 1 : 0;
}
// phase 1: roots take their id (roots in ascending node order); a strong
// neighbour of a root joins it (roots are >= 3 apart, so it is unique)
__global__ void k_agg_phase1(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             const uint8_t* __restrict__ strong, const uint8_t* __restrict__ st,
                             const int32_t* __restrict__ rootscan, int32_t* __restrict__ ph1) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t a = -1;
  if (st[i] == 1) a = rootscan[i];
  else if (st[i] == 2) {
    for (int32_t q = rp[i]; q < rp[i + 1]; ++q)
      if (strong[q] && st[ci[q]] == 1) { a = rootscan[ci[q]]; break; }
  }
  ph1[i] = a;
}
// phase 2: leftovers join the aggregate of their strongest phase-1 neighbour
// (largest weight, then smallest aggregate id)
__global__ void k_agg_phase2(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             const uint8_t* __restrict__ strong, const double* __restrict__ wgt,
                             const uint8_t* __restrict__ st, const int32_t* __restrict__ ph1,
                             int32_t* __restrict__ agg) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t a = ph1[i];
  if (st[i] == 2 && a < 0) {
    double bw = -1.0;
    int32_t ba = -1;
    for (int32_t q = rp[i]; q < rp[i + 1]; ++q) {
      if (!strong[q]) continue;
      int32_t aj = ph1[ci[q]];
      if (aj < 0) continue;
      if (wgt[q] > bw || (wgt[q] == bw && aj < ba)) { bw = wgt[q]; ba = aj; }
    }
    a = ba;
  }
  agg[i] = a;
}

// Gershgorin ratio sum_j |a_ij| / |a_ii| per row and component (component-major output)
template <int NC>
__global__ void k_gersh(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                        const double* __restrict__ v, double* __restrict__ out) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    double s = 0.0, d = 0.0;
    for (int32_t q = rp[i]; q < rp[i + 1]; ++q) {
      s = s + fabs(v[int64_t(q) * NC + c]);
      if (ci[q] == i) d = v[int64_t(q) * NC + c];
    }
    out[c * n + i] = s / fabs(d);
  }
}

template <int NC>
__global__ void k_l1(int64_t n, const int32_t* __restrict__ rp, const double* __restrict__ v,
                     double* __restrict__ out) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    double s = 0.0;
    for (int32_t q = rp[i]; q < rp[i + 1]; ++q) s = s + fabs(v[int64_t(q) * NC + c]);
    out[i * NC + c] = s;
  }
}

// tentative prolongator P_tent[i, agg(i)] = 1 (one entry per aggregated row)
__global__ void k_ptent_count(int64_t n, const int32_t* __restrict__ agg, int32_t* __restrict__ cnt) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) cnt[i] = agg[i] >= 0 ? 1 : 0;
}
template <int NC>
__global__ void k_ptent_fill(int64_t n, const int32_t* __restrict__ agg, const int32_t* __restrict__ rp,
                             int32_t* __restrict__ ci, double* __restrict__ v) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n || agg[i] < 0) return;
  ci[rp[i]] = agg[i];
  for (int c = 0; c < NC; ++c) v[int64_t(rp[i]) * NC + c] = 1.0;
}
// row lengths of P: those of T = A P_tent, except identity rows, which are empty
__global__ void k_p_rowlen(int64_t n, const int32_t* __restrict__ trp, const uint8_t* __restrict__ excl,
                           int32_t* __restrict__ cnt) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) cnt[i] = excl[i] ? 0 : trp[i + 1] - trp[i];
}
// P_ia = delta(a, agg(i)) - (omega / a_ii) * T_ia, T_ia = sum over the row's
// columns j of aggregate a of a_ij (ascending j)
template <int NC>
__global__ void k_p_finish(int64_t n, const int32_t* __restrict__ trp, const int32_t* __restrict__ tci,
                           const double* __restrict__ tv, const uint8_t* __restrict__ excl,
                           const int32_t* __restrict__ agg, const double* __restrict__ dg, double w0, double w1,
                           double w2, const int32_t* __restrict__ prp, int32_t* __restrict__ pci,
                           double* __restrict__ pv) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n || excl[i]) return;
  const double om[3] = {w0, w1, w2};
  int32_t o = prp[i];
  for (int32_t q = trp[i]; q < trp[i + 1]; ++q, ++o) {
    int32_t a = tci[q];
    pci[o] = a;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      double coef = om[c] / dg[i * NC + c];
      double delta = a == agg[i] ? 1.0 : 0.0;
      pv[int64_t(o) * NC + c] = delta - coef * tv[int64_t(q) * NC + c];
    }
  }
}

// ---- transpose (R = P^T) with rows sorted by fine index ----
__global__ void k_col_count(int64_t nnz, const int32_t* __restrict__ ci, int32_t* __restrict__ cnt) {
  int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q < nnz) atomicAdd(&cnt[ci[q]], 1);
}
template <int NC>
__global__ void k_transpose_fill(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                 const double* __restrict__ v, int32_t* __restrict__ cursor,
                                 int32_t* __restrict__ tci, double* __restrict__ tv) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int32_t q = rp[i]; q < rp[i + 1]; ++q) {
    int32_t pos = atomicAdd(&cursor[ci[q]], 1);
    tci[pos] = int32_t(i);
    for (int c = 0; c < NC; ++c) tv[int64_t(pos) * NC + c] = v[int64_t(q) * NC + c];
  }
}
// order each row by column: a warp per row ranks every entry by counting the
// smaller keys (keys in a row are distinct)
template <int NC>
__global__ void k_rank_rows(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci_in,
                            const double* __restrict__ v_in, int32_t* __restrict__ ci_out,
                            double* __restrict__ v_out) {
  int64_t row = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (row >= n) return;
  int32_t q0 = rp[row], q1 = rp[row + 1];
  for (int32_t q = q0 + lane; q < q1; q += 32) {
    int32_t k = ci_in[q];
    int32_t rank = 0;
    for (int32_t t = q0; t < q1; ++t) rank += ci_in[t] < k;
    ci_out[q0 + rank] = k;
    for (int c = 0; c < NC; ++c) v_out[int64_t(q0 + rank) * NC + c] = v_in[int64_t(q) * NC + c];
  }
}

// ---- SpGEMM C = X Y, one warp per row, shared-memory hash + sorted list ----
// Rows are binned by capacity class C (at most C distinct output columns, 2C hash
// slots) so that short rows -- most rows of A P on the fine levels -- use small
// tables and many warps per SM; rows above the largest class use the dense path.
constexpr int kUniq = 1024;   // largest class
constexpr int kEmpty = -1;
constexpr int kClasses = 4;
constexpr int64_t kDenseMaxCols = 1024;  // dense-accumulator path for long rows up to this many columns
__host__ __device__ constexpr int class_cap(int b) { return b == 0 ? 32 : b == 1 ? 128 : b == 2 ? 512 : 1024; }

template <int H>
__device__ __forceinline__ bool hash_insert(int32_t* tab, int32_t key, int* overflow) {
  uint32_t h = (uint32_t(key) * 2654435761u) & (H - 1);
  for (int probe = 0; probe < H; ++probe) {
    int32_t prev = atomicCAS(&tab[h], kEmpty, key);
    if (prev == kEmpty) return true;
    if (prev == key) return false;
    h = (h + 1) & (H - 1);
  }
  *overflow = 1;
  return false;
}

// Enumerates the products x_iq y_kr (k = xci[q]) of row i in (q, r) order, 32 at a time: each lane
// takes one product, found by a warp scan of the Y row lengths of 32 X entries and a shuffle search.
// f(valid, e, r) is called by every lane (it may shuffle); e is the lane that holds the product's X
// entry (its q, k and value), r the position of the Y entry.
template <class F>
__device__ __forceinline__ void for_products(int64_t i, const int32_t* __restrict__ xrp,
                                             const int32_t* __restrict__ xci, const int32_t* __restrict__ yrp,
                                             int lane, F&& f) {
  const int32_t q0 = xrp[i], q1 = xrp[i + 1];
  for (int32_t qc = q0; qc < q1; qc += 32) {
    const int32_t q = qc + lane;
    const bool v = q < q1;
    const int32_t k = v ? xci[q] : 0;
    const int32_t lo = v ? yrp[k] : 0;
    const int32_t len = v ? yrp[k + 1] - lo : 0;
    int32_t inc = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int32_t t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    const int32_t total = __shfl_sync(0xffffffffu, inc, 31);
    const int32_t excl = inc - len;
    for (int32_t p0 = 0; p0 < total; p0 += 32) {
      const int32_t p = p0 + lane;
      // the entry holding product p: the last lane whose first product is <= p
      int e = 0;
#pragma unroll
      for (int stp = 16; stp > 0; stp >>= 1) {
        int32_t ex = __shfl_sync(0xffffffffu, excl, e + stp);
        if (ex <= p) e += stp;
      }
      const int32_t lo_e = __shfl_sync(0xffffffffu, lo, e);
      const int32_t ex_e = __shfl_sync(0xffffffffu, excl, e);
      f(p < total, e, lo_e + (p - ex_e), qc);
    }
  }
}

// collect the distinct columns of row i into tab (H slots); returns their count (all lanes)
template <int H>
__device__ int spgemm_collect(int64_t i, const int32_t* __restrict__ xrp, const int32_t* __restrict__ xci,
                              const int32_t* __restrict__ yrp, const int32_t* __restrict__ yci, int32_t* tab,
                              int lane, int* overflow) {
  for (int t = lane; t < H; t += 32) tab[t] = kEmpty;
  __syncwarp();
  int cnt = 0;
  for_products(i, xrp, xci, yrp, lane, [&](bool valid, int, int32_t r, int32_t) {
    if (valid && hash_insert<H>(tab, yci[r], overflow)) ++cnt;
  });
  __syncwarp();
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  return cnt;
}

// upper bound of the distinct columns of each row (the number of products) and its count class
// slot of this lane in the list of class b (b < 0: none) with one atomic per warp and class; every
// lane of the warp must call it
template <int NCLS>
__device__ __forceinline__ int32_t warp_append(int b, int32_t* const (&ctr)[NCLS]) {
  const int lane = int(threadIdx.x & 31);
  int32_t slot = -1;
#pragma unroll
  for (int c = 0; c < NCLS; ++c) {
    const unsigned m = __ballot_sync(0xffffffffu, b == c);
    if (m == 0u) continue;
    const int leader = __ffs(int(m)) - 1;
    int32_t base = 0;
    if (lane == leader) base = atomicAdd(ctr[c], __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (b == c) slot = base + __popc(m & ((1u << lane) - 1u));
  }
  return slot;
}

// rows binned by their product bound (sum of the Y-row lengths over the X row)
__global__ void k_spgemm_bound(int64_t n, const int32_t* __restrict__ xrp, const int32_t* __restrict__ xci,
                               const int32_t* __restrict__ yrp, int32_t* __restrict__ lists,
                               int32_t* __restrict__ counts) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  int b = -1;
  if (i < n) {
    int64_t ub = 0;
    for (int32_t q = xrp[i]; q < xrp[i + 1]; ++q) ub += yrp[xci[q] + 1] - yrp[xci[q]];
    b = ub <= class_cap(0) ? 0 : ub <= class_cap(1) ? 1 : ub <= class_cap(2) ? 2 : 3;
  }
  int32_t* const ctr[4] = {counts, counts + 1, counts + 2, counts + 3};
  const int32_t slot = warp_append<4>(b, ctr);
  if (b >= 0) lists[int64_t(b) * n + slot] = int32_t(i);
}

// rows listed in rows[0..nrows): exact distinct-column count with a table of 2C slots; rows
// with more than kUniq columns (possible in the last class only) go to longrows[]
template <int C>
__global__ void k_spgemm_count(const int32_t* __restrict__ rows, int32_t nrows, const int32_t* __restrict__ xrp,
                               const int32_t* __restrict__ xci, const int32_t* __restrict__ yrp,
                               const int32_t* __restrict__ yci, int32_t* __restrict__ cnt,
                               uint8_t* __restrict__ islong, int32_t* __restrict__ longrows,
                               int32_t* __restrict__ nlong) {
  extern __shared__ int32_t smem[];
  int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t w = int64_t(blockIdx.x) * (blockDim.x >> 5) + wib;
  if (w >= nrows) return;
  int64_t i = rows[w];
  int32_t* tab = smem + wib * (2 * C);
  int ovf = 0;
  int c = spgemm_collect<2 * C>(i, xrp, xci, yrp, yci, tab, lane, &ovf);
  ovf = __any_sync(0xffffffffu, ovf);
  if (lane == 0) {
    bool lg = ovf || c > kUniq;
    cnt[i] = lg ? 0 : c;
    islong[i] = lg ? 1 : 0;
    if (lg) longrows[atomicAdd(nlong, 1)] = int32_t(i);
  }
}

// fill classes from the exact counts (long rows, cnt = 0 and listed apart, are skipped)
// With few output columns (dense_ok), rows with more than class_cap(1) distinct columns go to the
// dense-accumulator path, one CTA per row, instead of a warp with a large hash table: they are
// marked long and appended to longrows.  Long rows are not binned.
__global__ void k_spgemm_fill_bins(int64_t n, const int32_t* __restrict__ cnt, int32_t* __restrict__ lists,
                                   int32_t* __restrict__ counts, int dense_ok, uint8_t* __restrict__ islong,
                                   int32_t* __restrict__ longrows, int32_t* __restrict__ nlong) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  int b = -1;  // 0..3: capacity class, 4: the dense path
  if (i < n && !islong[i]) {
    const int32_t u = cnt[i];
    if (dense_ok && u > class_cap(1)) b = 4;
    else b = u <= class_cap(0) ? 0 : u <= class_cap(1) ? 1 : u <= class_cap(2) ? 2 : 3;
  }
  int32_t* const ctr[5] = {counts, counts + 1, counts + 2, counts + 3, nlong};
  const int32_t slot = warp_append<5>(b, ctr);
  if (b == 4) {
    islong[i] = 1;
    longrows[slot] = int32_t(i);
  } else if (b >= 0) {
    lists[int64_t(b) * n + slot] = int32_t(i);
  }
}

// rows of the largest product-bound class handled by the dense path from the count pass on
__global__ void k_spgemm_mark_long(const int32_t* __restrict__ rows, int32_t nr, uint8_t* __restrict__ islong,
                                   int32_t* __restrict__ longrows, int32_t* __restrict__ nlong) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nr) return;
  islong[rows[t]] = 1;
  longrows[atomicAdd(nlong, 1)] = rows[t];
}

// dense path, one CTA per long row: stamp[j] marks the columns seen for this row
// (stamps are row id + 1, so the scratch never needs clearing)
__global__ void k_spgemm_dense_count(const int32_t* __restrict__ rows, int32_t nrows, const int32_t* __restrict__ xrp,
                                     const int32_t* __restrict__ xci, const int32_t* __restrict__ yrp,
                                     const int32_t* __restrict__ yci, int32_t* __restrict__ stamp, int64_t m,
                                     int32_t* __restrict__ cnt) {
  int b = blockIdx.x;
  if (b >= nrows) return;
  int32_t i = rows[b];
  int32_t* mk = stamp + int64_t(b) * m;
  __shared__ int32_t c;
  if (threadIdx.x == 0) c = 0;
  __syncthreads();
  int32_t tag = i + 1;
  for (int32_t q = xrp[i]; q < xrp[i + 1]; ++q) {
    int32_t k = xci[q];
    for (int32_t r = yrp[k] + threadIdx.x; r < yrp[k + 1]; r += blockDim.x)
      if (atomicExch(&mk[yci[r]], tag) != tag) atomicAdd(&c, 1);
    __syncthreads();
  }
  if (threadIdx.x == 0) cnt[i] = c;
}

template <int NC>
__global__ void k_spgemm_dense_fill(const int32_t* __restrict__ rows, int32_t nrows, const int32_t* __restrict__ xrp,
                                    const int32_t* __restrict__ xci, const double* __restrict__ xv,
                                    const int32_t* __restrict__ yrp, const int32_t* __restrict__ yci,
                                    const double* __restrict__ yv, int32_t* __restrict__ stamp,
                                    double* __restrict__ acc_all, int64_t m, const int32_t* __restrict__ crp,
                                    int32_t* __restrict__ cci, double* __restrict__ cv) {
  int b = blockIdx.x;
  if (b >= nrows) return;
  int32_t i = rows[b];
  int32_t* mk = stamp + int64_t(b) * m;
  double* acc = acc_all + int64_t(b) * m * NC;
  // the stamp of the count pass is i + 1; mark this pass with -(i + 1) and zero the accumulators
  int32_t tag = -(i + 1);
  for (int32_t q = xrp[i]; q < xrp[i + 1]; ++q) {
    int32_t k = xci[q];
    for (int32_t r = yrp[k] + threadIdx.x; r < yrp[k + 1]; r += blockDim.x) {
      int32_t j = yci[r];
      if (atomicExch(&mk[j], tag) != tag)
        for (int c = 0; c < NC; ++c) acc[int64_t(j) * NC + c] = 0.0;
    }
    __syncthreads();
  }
  // products in ascending order of the inner index k (distinct j within one Y row)
  for (int32_t q = xrp[i]; q < xrp[i + 1]; ++q) {
    int32_t k = xci[q];
    double x[NC];
    for (int c = 0; c < NC; ++c) x[c] = xv[int64_t(q) * NC + c];
    for (int32_t r = yrp[k] + threadIdx.x; r < yrp[k + 1]; r += blockDim.x) {
      int32_t j = yci[r];
      for (int c = 0; c < NC; ++c)
        acc[int64_t(j) * NC + c] = fma(x[c], yv[int64_t(r) * NC + c], acc[int64_t(j) * NC + c]);
    }
    __syncthreads();
  }
  // emit in ascending column order: rank of each marked column by a block scan over j
  __shared__ int32_t base;
  if (threadIdx.x == 0) base = crp[i];
  __syncthreads();
  for (int64_t j0 = 0; j0 < m; j0 += blockDim.x) {
    int64_t j = j0 + threadIdx.x;
    int f = (j < m && mk[j] == tag) ? 1 : 0;
    // block-wide exclusive scan of f (blockDim.x <= 1024)
    __shared__ int32_t sc[1024];
    sc[threadIdx.x] = f;
    __syncthreads();
    for (int off = 1; off < blockDim.x; off <<= 1) {
      int32_t t = threadIdx.x >= off ? sc[threadIdx.x - off] : 0;
      __syncthreads();
      sc[threadIdx.x] += t;
      __syncthreads();
    }
    if (f) {
      int32_t pos = base + sc[threadIdx.x] - 1;
      cci[pos] = int32_t(j);
      for (int c = 0; c < NC; ++c) cv[int64_t(pos) * NC + c] = acc[j * NC + c];
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) base += sc[threadIdx.x];
    __syncthreads();
  }
}

// Dense path with few output columns (m <= kDenseMaxCols), one warp per row: the row's column set is a
// bitmap and its accumulators a dense array, both in the warp's shared memory.  The count pass marks the
// bitmap (in any order) and counts its bits.  The fill pass marks again, then adds the products one inner
// index at a time in ascending order (lanes take the entries of that Y row, whose columns are distinct, so
// no two lanes meet; a warp barrier separates consecutive inner indices), and emits the columns in
// ascending order from the bitmap.
__device__ __forceinline__ void dense_mark(int64_t i, const int32_t* __restrict__ xrp, const int32_t* __restrict__ xci,
                                           const int32_t* __restrict__ yrp, const int32_t* __restrict__ yci,
                                           uint32_t* bm, int32_t words, int lane) {
  for (int t = lane; t < words; t += 32) bm[t] = 0u;
  __syncwarp();
  for_products(i, xrp, xci, yrp, lane, [&](bool valid, int, int32_t r, int32_t) {
    if (valid) {
      const int32_t j = yci[r];
      atomicOr(&bm[j >> 5], 1u << (j & 31));
    }
  });
  __syncwarp();
}

__global__ void k_spgemm_dense_count_w(const int32_t* __restrict__ rows, int32_t nrows,
                                       const int32_t* __restrict__ xrp, const int32_t* __restrict__ xci,
                                       const int32_t* __restrict__ yrp, const int32_t* __restrict__ yci,
                                       int32_t words, int32_t* __restrict__ cnt) {
  extern __shared__ uint32_t bm_all[];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t w = int64_t(blockIdx.x) * (blockDim.x >> 5) + wib;
  if (w >= nrows) return;
  const int64_t i = rows[w];
  uint32_t* bm = bm_all + int64_t(wib) * words;
  dense_mark(i, xrp, xci, yrp, yci, bm, words, lane);
  int c = 0;
  for (int t = lane; t < words; t += 32) c += __popc(bm[t]);
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) cnt[i] = c;
}

template <int NC>
__global__ void k_spgemm_dense_fill_w(const int32_t* __restrict__ rows, int32_t nrows, const int32_t* __restrict__ xrp,
                                      const int32_t* __restrict__ xci, const double* __restrict__ xv,
                                      const int32_t* __restrict__ yrp, const int32_t* __restrict__ yci,
                                      const double* __restrict__ yv, int32_t m, int32_t words,
                                      const int32_t* __restrict__ crp, int32_t* __restrict__ cci,
                                      double* __restrict__ cv) {
  extern __shared__ double dsm[];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t w = int64_t(blockIdx.x) * (blockDim.x >> 5) + wib;
  if (w >= nrows) return;
  const int64_t i = rows[w];
  const int64_t per = int64_t(m) * NC + (words + 1) / 2;  // doubles per warp: accumulators, then the bitmap
  double* acc = dsm + int64_t(wib) * per;
  uint32_t* bm = reinterpret_cast<uint32_t*>(acc + int64_t(m) * NC);
  for (int64_t t = lane; t < int64_t(m) * NC; t += 32) acc[t] = 0.0;
  dense_mark(i, xrp, xci, yrp, yci, bm, words, lane);
  for (int32_t q = xrp[i]; q < xrp[i + 1]; ++q) {
    const int32_t k = xci[q];
    double x[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) x[c] = xv[int64_t(q) * NC + c];
    for (int32_t r = yrp[k] + lane; r < yrp[k + 1]; r += 32) {
      const int32_t j = yci[r];
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[int64_t(j) * NC + c] = fma(x[c], yv[int64_t(r) * NC + c], acc[int64_t(j) * NC + c]);
    }
    __syncwarp();
  }
  int32_t base = crp[i];
  for (int32_t w0 = 0; w0 < words; w0 += 32) {
    const int32_t t = w0 + lane;
    uint32_t bits = t < words ? bm[t] : 0u;
    const int32_t pc = __popc(bits);
    int32_t inc = pc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += v;
    }
    int32_t pos = base + inc - pc;
    while (bits) {
      const int b = __ffs(int(bits)) - 1;
      bits &= bits - 1u;
      const int32_t j = t * 32 + b;
      cci[pos] = j;
#pragma unroll
      for (int c = 0; c < NC; ++c) cv[int64_t(pos) * NC + c] = acc[int64_t(j) * NC + c];
      ++pos;
    }
    base += __shfl_sync(0xffffffffu, inc, 31);
  }
}

// ---- rows of the smallest class (at most 32 distinct columns) two to a warp ----
// The fill of a short row keeps few lanes busy in the in-order folds of same-column products, and on GB300 a
// warp's FP64 instruction costs the pipe a full issue whatever its active lanes.  Here each half-warp (16
// lanes) takes one row, so the folds of two rows share each instruction.  The two halves run the same
// sequence of warp-wide steps (loop counts are the larger of the two), and every result is formed as in
// k_spgemm_fill: products of a row in (q, r) order, a column's products folded in that order by fused
// multiply-adds, columns emitted sorted.
constexpr unsigned kFull = 0xffffffffu;
__device__ __forceinline__ int half_max(int v) { return max(v, __shfl_xor_sync(kFull, v, 16)); }

template <class F>
__device__ __forceinline__ void for_products_h(int64_t i, const int32_t* __restrict__ xrp,
                                               const int32_t* __restrict__ xci, const int32_t* __restrict__ yrp,
                                               int hl, F&& f) {
  const int32_t q0 = i >= 0 ? xrp[i] : 0, q1 = i >= 0 ? xrp[i + 1] : 0;
  const int nch = half_max((q1 - q0 + 15) / 16);
  for (int ch = 0; ch < nch; ++ch) {
    const int32_t qc = q0 + ch * 16;
    const int32_t q = qc + hl;
    const bool v = q < q1;
    const int32_t k = v ? xci[q] : 0;
    const int32_t lo = v ? yrp[k] : 0;
    const int32_t len = v ? yrp[k + 1] - lo : 0;
    int32_t inc = len;
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
      const int32_t t = __shfl_up_sync(kFull, inc, o, 16);
      if (hl >= o) inc += t;
    }
    const int32_t total = __shfl_sync(kFull, inc, 15, 16);
    const int32_t excl = inc - len;
    const int nr = half_max((total + 15) / 16);
    for (int rr = 0; rr < nr; ++rr) {
      const int32_t p = rr * 16 + hl;
      int e = 0;
#pragma unroll
      for (int stp = 8; stp > 0; stp >>= 1) {
        const int32_t ex = __shfl_sync(kFull, excl, e + stp, 16);
        if (ex <= p) e += stp;
      }
      const int32_t lo_e = __shfl_sync(kFull, lo, e, 16);
      const int32_t ex_e = __shfl_sync(kFull, excl, e, 16);
      f(p < total, e, lo_e + (p - ex_e), qc);
    }
  }
}

template <int NC, int C>
__global__ void k_spgemm_fill_h(const int32_t* __restrict__ rows, int32_t nrows, const int32_t* __restrict__ xrp,
                                const int32_t* __restrict__ xci, const double* __restrict__ xv,
                                const int32_t* __restrict__ yrp, const int32_t* __restrict__ yci,
                                const double* __restrict__ yv, const int32_t* __restrict__ crp,
                                int32_t* __restrict__ cci, double* __restrict__ cv,
                                const uint8_t* __restrict__ islong, int* __restrict__ err) {
  constexpr int H = 2 * C;
  constexpr int PER = H * 4 + C * 4 + C * NC * 8 + 16 * 2 * NC * 8;  // bytes per half-warp
  extern __shared__ unsigned char sraw[];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
  const int64_t w = int64_t(blockIdx.x) * (blockDim.x >> 5) + wib;
  if (w * 2 >= nrows) return;  // the whole warp
  const int64_t slot = w * 2 + half;
  int64_t i = slot < nrows ? rows[slot] : -1;
  if (i >= 0 && islong[i]) i = -1;
  unsigned char* base = sraw + size_t(PER) * (wib * 2 + half);
  int32_t* tab = reinterpret_cast<int32_t*>(base);
  int32_t* list = reinterpret_cast<int32_t*>(base + H * 4);
  double* acc = reinterpret_cast<double*>(base + H * 4 + C * 4);
  double* stg = acc + C * NC;
  // distinct columns into this half's hash table
  for (int t = hl; t < H; t += 16) tab[t] = kEmpty;
  __syncwarp();
  int ovf = 0, cnt = 0;
  for_products_h(i, xrp, xci, yrp, hl, [&](bool valid, int, int32_t r, int32_t) {
    if (valid && hash_insert<H>(tab, yci[r], &ovf)) ++cnt;
  });
  __syncwarp();
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) cnt += __shfl_xor_sync(kFull, cnt, o, 16);
  const int u = cnt;
  const int bad = __any_sync(kFull, ovf != 0 || u > C);
  if (bad) {
    if (lane == 0) atomicExch(err, 1);
    return;
  }
  // compact this half's table into list[0..u)
  int pos = 0;
  for (int t0 = 0; t0 < H; t0 += 16) {
    const int32_t key = tab[t0 + hl];
    const bool f = key != kEmpty;
    const unsigned mk = (__ballot_sync(kFull, f) >> (half * 16)) & 0xffffu;
    if (f) list[pos + __popc(mk & ((1u << hl) - 1u))] = key;
    pos += __popc(mk);
  }
  __syncwarp();
  // bitonic sort of list[0..P), P the larger of the two halves' next powers of two >= u (padding INT_MAX)
  int P = 1;
  while (P < u) P <<= 1;
  P = half_max(P);
  for (int t = u + hl; t < P; t += 16) list[t] = 0x7fffffff;
  __syncwarp();
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = hl; t < P; t += 16) {
        const int q = t ^ j;
        if (q > t) {
          const int32_t a = list[t], b = list[q];
          const bool up = (t & k) == 0;
          if ((a > b) == up) { list[t] = b; list[q] = a; }
        }
      }
      __syncwarp();
    }
  for (int t = hl; t < u * NC; t += 16) acc[t] = 0.0;
  __syncwarp();
  // numeric: a column's products folded in (q, r) order by the lowest lane of each same-column group
  const int32_t q1 = i >= 0 ? xrp[i + 1] : 0;
  for_products_h(i, xrp, xci, yrp, hl, [&](bool valid, int e, int32_t r, int32_t qc) {
    int pp = 0;
    if (valid) {
      const int32_t jj = yci[r];
      int lo = 0, hi = u;
      while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if (list[m] < jj) lo = m + 1;
        else hi = m;
      }
      pp = lo;
      const int32_t qe = qc + e;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        stg[hl * 2 * NC + c] = qe < q1 ? xv[int64_t(qe) * NC + c] : 0.0;
        stg[hl * 2 * NC + NC + c] = yv[int64_t(r) * NC + c];
      }
    }
    const unsigned peers = __match_any_sync(kFull, valid ? ((half << 30) | pp) : int(0x7fff0000 + lane));
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        double a = acc[pp * NC + c];
        for (unsigned m = peers; m; m &= m - 1) {
          const int pl = (__ffs(m) - 1) & 15;
          a = fma(stg[pl * 2 * NC + c], stg[pl * 2 * NC + NC + c], a);
        }
        acc[pp * NC + c] = a;
      }
    }
    __syncwarp();
  });
  if (i < 0) return;
  const int32_t o = crp[i];
  for (int t = hl; t < u; t += 16) {
    cci[o + t] = list[t];
#pragma unroll
    for (int c = 0; c < NC; ++c) cv[int64_t(o + t) * NC + c] = acc[t * NC + c];
  }
}

template <int NC, int C>
__global__ void k_spgemm_fill(const int32_t* __restrict__ rows, int32_t nrows, const int32_t* __restrict__ xrp,
                              const int32_t* __restrict__ xci, const double* __restrict__ xv,
                              const int32_t* __restrict__ yrp, const int32_t* __restrict__ yci,
                              const double* __restrict__ yv, const int32_t* __restrict__ crp,
                              int32_t* __restrict__ cci, double* __restrict__ cv, const uint8_t* __restrict__ islong,
                              int* __restrict__ err) {
  extern __shared__ unsigned char sraw[];
  constexpr int H = 2 * C;
  int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t w = int64_t(blockIdx.x) * (blockDim.x >> 5) + wib;
  if (w >= nrows) return;
  int64_t i = rows[w];
  if (islong[i]) return;
  constexpr size_t per = size_t(H) * 4 + size_t(C) * 4 + size_t(C) * NC * 8 + size_t(32) * NC * 16;
  unsigned char* base = sraw + per * wib;
  int32_t* tab = reinterpret_cast<int32_t*>(base);
  int32_t* list = reinterpret_cast<int32_t*>(base + H * 4);
  double* acc = reinterpret_cast<double*>(base + H * 4 + C * 4);
  double* stg = acc + C * NC;  // the two factors of one product per lane, staged for the in-order fold
  int ovf = 0;
  int u = spgemm_collect<H>(i, xrp, xci, yrp, yci, tab, lane, &ovf);
  if (u > C || __any_sync(0xffffffffu, ovf)) {
    if (lane == 0) atomicExch(err, 1);
    return;
  }
  // compact the table into list[0..u) (the order is fixed by the sort below)
  int pos = 0;
  for (int t0 = 0; t0 < H; t0 += 32) {
    int32_t key = tab[t0 + lane];
    bool f = key != kEmpty;
    unsigned mk = __ballot_sync(0xffffffffu, f);
    if (f) list[pos + __popc(mk & ((1u << lane) - 1u))] = key;
    pos += __popc(mk);
  }
  __syncwarp();
  // bitonic sort of list[0..P), P = next power of two >= u, padded with INT_MAX
  int P = 1;
  while (P < u) P <<= 1;
  for (int t = u + lane; t < P; t += 32) list[t] = 0x7fffffff;
  __syncwarp();
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = lane; t < P; t += 32) {
        int p = t ^ j;
        if (p > t) {
          int32_t a = list[t], b = list[p];
          bool up = (t & k) == 0;
          if ((a > b) == up) { list[t] = b; list[p] = a; }
        }
      }
      __syncwarp();
    }
  for (int t = lane; t < u * NC; t += 32) acc[t] = 0.0;
  __syncwarp();
  // numeric: for each output column, products added one at a time in ascending order of the inner
  // index k (products are enumerated q-major; within a round of 32, lanes that hit the same column
  // are folded in by the lowest of them in lane order)
  for_products(i, xrp, xci, yrp, lane, [&](bool valid, int e, int32_t r, int32_t qc) {
    double x[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int32_t qe = qc + e;
      double xl = 0.0;
      if (qe < xrp[i + 1]) xl = xv[int64_t(qe) * NC + c];
      x[c] = xl;
    }
    int pos = 0;
    if (valid) {
      const int32_t j = yci[r];
      int lo = 0, hi = u;
      while (lo < hi) {
        int m = (lo + hi) >> 1;
        if (list[m] < j) lo = m + 1;
        else hi = m;
      }
      pos = lo;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        stg[lane * 2 * NC + c] = x[c];
        stg[lane * 2 * NC + NC + c] = yv[int64_t(r) * NC + c];
      }
    }
    const unsigned peers = __match_any_sync(0xffffffffu, valid ? pos : (1 << 30) + lane);
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        double a = acc[pos * NC + c];
        for (unsigned m = peers; m; m &= m - 1) {
          const int pl = __ffs(m) - 1;
          a = fma(stg[pl * 2 * NC + c], stg[pl * 2 * NC + NC + c], a);
        }
        acc[pos * NC + c] = a;
      }
    }
    __syncwarp();
  });
  int32_t o = crp[i];
  for (int t = lane; t < u; t += 32) {
    cci[o + t] = list[t];
#pragma unroll
    for (int c = 0; c < NC; ++c) cv[int64_t(o + t) * NC + c] = acc[t * NC + c];
  }
}

// ---- coarsest level: Gauss-Jordan inverse with partial pivoting, per component ----
// M: [nc][n][n] row-major, I: [nc][n][n]; f: [nc][n] multipliers, piv scratch
__global__ void k_dense_unpack(int64_t n, int nc, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                               const double* __restrict__ v, double* __restrict__ M, double* __restrict__ I) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n) return;
  for (int c = 0; c < nc; ++c) {
    for (int32_t q = rp[t]; q < rp[t + 1]; ++q) M[(c * n + t) * n + ci[q]] = v[int64_t(q) * nc + c];
    I[(c * n + t) * n + t] = 1.0;
  }
}
__global__ void k_gj_pivot(int64_t n, int64_t k, double* __restrict__ M, double* __restrict__ I,
                           double* __restrict__ f) {
  int c = blockIdx.x;
  double* A = M + int64_t(c) * n * n;
  double* B = I + int64_t(c) * n * n;
  __shared__ double bv[256];
  __shared__ int64_t bi[256];
  double best = -1.0;
  int64_t arg = k;
  for (int64_t r = k + threadIdx.x; r < n; r += blockDim.x) {
    double a = fabs(A[r * n + k]);
    if (a > best) { best = a; arg = r; }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = arg;
  __syncthreads();
  for (int off = blockDim.x >> 1; off > 0; off >>= 1) {
    if (threadIdx.x < off) {
      double o = bv[threadIdx.x + off];
      int64_t oi = bi[threadIdx.x + off];
      if (o > bv[threadIdx.x] || (o == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
        bv[threadIdx.x] = o;
        bi[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  int64_t p = bi[0];
  if (p != k)
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
      double t = A[k * n + j]; A[k * n + j] = A[p * n + j]; A[p * n + j] = t;
      t = B[k * n + j]; B[k * n + j] = B[p * n + j]; B[p * n + j] = t;
    }
  __syncthreads();
  double piv = A[k * n + k];
  __syncthreads();
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    A[k * n + j] = A[k * n + j] / piv;
    B[k * n + j] = B[k * n + j] / piv;
  }
  __syncthreads();
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) f[int64_t(c) * n + r] = A[r * n + k];
}
__global__ void k_gj_elim(int64_t n, int64_t k, double* __restrict__ M, double* __restrict__ I,
                          const double* __restrict__ f) {
  int c = blockIdx.z;
  int64_t r = int64_t(blockIdx.y);
  int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r == k || j >= 2 * n) return;
  double m = f[int64_t(c) * n + r];
  if (m == 0.0) return;
  double* A = M + int64_t(c) * n * n;
  double* B = I + int64_t(c) * n * n;
  if (j < n) A[r * n + j] = A[r * n + j] - m * A[k * n + j];
  else B[r * n + j - n] = B[r * n + j - n] - m * B[k * n + j - n];
}

// The whole Gauss-Jordan inverse in one cooperative launch (every CTA co-resident): for each pivot k, CTA c
// (c < nc) finds, swaps and normalises the pivot row of component c exactly as k_gj_pivot does, then all
// CTAs eliminate column k from every other row of every component as k_gj_elim does, with a bounded grid
// barrier after each of the two steps (2 n barriers in place of 2 n launches).  Data written in an earlier
// step is loaded through L2 (ld.global.cg).
__global__ void __launch_bounds__(256) k_gj_all(int64_t n, int nc, double* __restrict__ M, double* __restrict__ I,
                                                double* __restrict__ f, unsigned long long* bar, int64_t limit,
                                                int* err) {
  const unsigned long long G = gridDim.x;
  unsigned long long phase = 0;
  __shared__ double bv[256];
  __shared__ int64_t bi[256];
  for (int64_t k = 0; k < n; ++k) {
    if (int(blockIdx.x) < nc) {
      const int c = blockIdx.x;
      double* A = M + int64_t(c) * n * n;
      double* B = I + int64_t(c) * n * n;
      double best = -1.0;
      int64_t arg = k;
      for (int64_t r = k + threadIdx.x; r < n; r += blockDim.x) {
        double a = fabs(__ldcg(A + r * n + k));
        if (a > best) { best = a; arg = r; }
      }
      bv[threadIdx.x] = best;
      bi[threadIdx.x] = arg;
      __syncthreads();
      for (int off = blockDim.x >> 1; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
          double o = bv[threadIdx.x + off];
          int64_t oi = bi[threadIdx.x + off];
          if (o > bv[threadIdx.x] || (o == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
            bv[threadIdx.x] = o;
            bi[threadIdx.x] = oi;
          }
        }
        __syncthreads();
      }
      const int64_t p = bi[0];
      if (p != k)
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
          double t = __ldcg(A + k * n + j); A[k * n + j] = __ldcg(A + p * n + j); A[p * n + j] = t;
          t = __ldcg(B + k * n + j); B[k * n + j] = __ldcg(B + p * n + j); B[p * n + j] = t;
        }
      __syncthreads();
      const double piv = A[k * n + k];
      __syncthreads();
      for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        A[k * n + j] = A[k * n + j] / piv;
        B[k * n + j] = B[k * n + j] / piv;
      }
      __syncthreads();
      for (int64_t r = threadIdx.x; r < n; r += blockDim.x) f[int64_t(c) * n + r] = A[r * n + k];
      __syncthreads();
    }
    if (!grid_barrier(bar, ++phase * G, limit, err)) return;
    // elimination, one row of one component per CTA at a time.  Columns j < k of A are skipped: there the
    // pivot row holds exact zeros (earlier pivots cleared them), so the update would leave the entry as it is.
    for (int64_t rc = blockIdx.x; rc < int64_t(nc) * n; rc += int64_t(G)) {
      const int c = int(rc / n);
      const int64_t r = rc - int64_t(c) * n;
      if (r == k) continue;
      const double m = __ldcg(f + int64_t(c) * n + r);
      if (m == 0.0) continue;
      double* A = M + int64_t(c) * n * n;
      double* B = I + int64_t(c) * n * n;
      for (int64_t j = k + threadIdx.x; j < n; j += blockDim.x)
        A[r * n + j] = __ldcg(A + r * n + j) - m * __ldcg(A + k * n + j);
      for (int64_t j = threadIdx.x; j < n; j += blockDim.x)
        B[r * n + j] = __ldcg(B + r * n + j) - m * __ldcg(B + k * n + j);
    }
    if (!grid_barrier(bar, ++phase * G, limit, err)) return;
  }
}

__global__ void k_fill_one(double* __restrict__ a, int64_t n) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < n) a[t] = 1.0;
}
__global__ void k_to_bf16(const double* __restrict__ a, __nv_bfloat16* __restrict__ b, int64_t n) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < n) b[t] = __double2bfloat16(a[t]);
}
__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < n) b[t] = float(a[t]);
}

// launch f<C>(warps per block, dynamic shared bytes) for capacity class b
template <class F>
void for_class(int b, F&& f) {
  switch (b) {
    case 0: f(std::integral_constant<int, 32>()); break;
    case 1: f(std::integral_constant<int, 128>()); break;
    case 2: f(std::integral_constant<int, 512>()); break;
    default: f(std::integral_constant<int, 1024>()); break;
  }
}

template <int NC>
ps_status spgemm(Arena& ar, int64_t n, int64_t m, const int32_t* xrp, const int32_t* xci, const double* xv,
                 const int32_t* yrp, const int32_t* yci, const double* yv, int32_t** crp, int32_t** cci, double** cv,
                 int64_t* cnnz, int* d_err, cudaStream_t st) {
  int32_t *cnt, *longrows, *nlong, *lists, *counts;
  uint8_t* islong;
  PS_TRY(ar.alloc(&cnt, n + 1));
  PS_TRY(ar.alloc(crp, n + 1));
  PS_TRY(ar.alloc(&islong, n + 1));
  PS_TRY(ar.alloc(&longrows, n + 1));
  PS_TRY(ar.alloc(&nlong, 1));
  PS_TRY(ar.alloc(&lists, size_t(kClasses) * n + 1));
  PS_TRY(ar.alloc(&counts, 2 * kClasses));
  PS_CUDA(cudaMemsetAsync(nlong, 0, sizeof(int32_t), st));
  PS_CUDA(cudaMemsetAsync(counts, 0, sizeof(int32_t) * 2 * kClasses, st));
  // count pass, binned by the product bound
  PS_TICK(); k_spgemm_bound<<<grid_for(n, 256), 256, 0, st>>>(n, xrp, xci, yrp, lists, counts);
  int32_t hc[2 * kClasses];
  PS_CUDA(cudaMemcpyAsync(hc, counts, sizeof(hc), cudaMemcpyDeviceToHost, st));
  PS_CUDA(cudaStreamSynchronize(st));
  // few output columns: the dense path (one CTA per row) takes the rows with the most products
  const bool dense_ok = m <= kDenseMaxCols;
  PS_CUDA(cudaMemsetAsync(islong, 0, size_t(n) + 1, st));
  for (int b = 0; b < kClasses; ++b) {
    int32_t nr = hc[b];
    if (nr == 0) continue;
    const int32_t* rows = lists + int64_t(b) * n;
    if (dense_ok && b == kClasses - 1) {
      PS_TICK(); k_spgemm_mark_long<<<grid_for(nr, 256), 256, 0, st>>>(rows, nr, islong, longrows, nlong);
      continue;
    }
    for_class(b, [&](auto cc) {
      constexpr int C = decltype(cc)::value;
      const int wpb = C <= 128 ? 8 : 4;
      size_t sm = size_t(wpb) * 2 * C * 4;
      PS_TICK(); k_spgemm_count<C><<<unsigned((nr + wpb - 1) / wpb), 32 * wpb, sm, st>>>(
          rows, nr, xrp, xci, yrp, yci, cnt, islong, longrows, nlong);
    });
  }
  PS_CUDA(cudaGetLastError());
  int32_t hl = 0;
  PS_CUDA(cudaMemcpyAsync(&hl, nlong, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  PS_CUDA(cudaStreamSynchronize(st));
  // dense-accumulator batches for the long rows
  int32_t* stamp = nullptr;
  double* acc = nullptr;
  int64_t B = 0;
  const int32_t words = int32_t((m + 31) / 32);
  // warps per CTA of the shared-memory dense path (m <= kDenseMaxCols)
  const size_t dense_per = (size_t(m) * NC + size_t(words + 1) / 2) * 8;
  const int dense_wpb = int(std::max<size_t>(1, std::min<size_t>(8, (96u << 10) / (dense_per > 0 ? dense_per : 1))));
  if (hl > 0 && dense_ok) {
    PS_TICK(); k_spgemm_dense_count_w<<<unsigned((hl + dense_wpb - 1) / dense_wpb), 32 * dense_wpb,
                                        size_t(dense_wpb) * words * 4, st>>>(longrows, hl, xrp, xci, yrp, yci, words,
                                                                             cnt);
  } else if (hl > 0) {
    int64_t per = m * (4 + 8 * NC);
    B = (int64_t(256) << 20) / (per > 0 ? per : 1);
    if (B < 1) B = 1;
    if (B > hl) B = hl;
    PS_TRY(ar.alloc(&stamp, size_t(B) * m + 1));
    PS_TRY(ar.alloc(&acc, (size_t(B) * m + 1) * NC));
    PS_CUDA(cudaMemsetAsync(stamp, 0, sizeof(int32_t) * (size_t(B) * m + 1), st));
    for (int64_t b0 = 0; b0 < hl; b0 += B) {
      int32_t nb = int32_t(hl - b0 < B ? hl - b0 : B);
      PS_TICK(); k_spgemm_dense_count<<<nb, 256, 0, st>>>(longrows + b0, nb, xrp, xci, yrp, yci, stamp, m, cnt);
    }
  }
  int32_t tot = 0;
  PS_TRY(scan_i32(ar, cnt, *crp, n, &tot, st));
  *cnnz = tot;
  PS_TRY(ar.alloc(cci, size_t(tot) + 1));
  PS_TRY(ar.alloc(cv, (size_t(tot) + 1) * NC));
  // fill pass, binned by the exact count; long rows (and, with few output columns, rows with many
  // distinct columns) take the dense path
  PS_CUDA(cudaMemsetAsync(counts + kClasses, 0, sizeof(int32_t) * kClasses, st));
  PS_TICK(); k_spgemm_fill_bins<<<grid_for(n, 256), 256, 0, st>>>(n, cnt, lists, counts + kClasses, dense_ok ? 1 : 0,
                                                                islong, longrows, nlong);
  PS_CUDA(cudaMemcpyAsync(hc, counts, sizeof(hc), cudaMemcpyDeviceToHost, st));
  PS_CUDA(cudaMemcpyAsync(&hl, nlong, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  PS_CUDA(cudaStreamSynchronize(st));
  if (!dense_ok && hl > B) {
    // more long rows than the count pass had: a larger batch of accumulators (tags are unique per
    // row, so fresh zeroed stamps serve any row)
    int64_t per = m * (4 + 8 * NC);
    int64_t Bmax = (int64_t(256) << 20) / (per > 0 ? per : 1);
    if (Bmax < 1) Bmax = 1;
    int64_t Bn = hl < Bmax ? hl : Bmax;
    if (Bn > B) {
      if (stamp) { ar.release(stamp); ar.release(acc); }
      B = Bn;
      PS_TRY(ar.alloc(&stamp, size_t(B) * m + 1));
      PS_TRY(ar.alloc(&acc, (size_t(B) * m + 1) * NC));
      PS_CUDA(cudaMemsetAsync(stamp, 0, sizeof(int32_t) * (size_t(B) * m + 1), st));
    }
  }
  for (int b = 0; b < kClasses; ++b) {
    int32_t nr = hc[kClasses + b];
    if (nr == 0) continue;
    const int32_t* rows = lists + int64_t(b) * n;
    if (b == 0) {
      // rows of at most 32 columns: two to a warp (the 128-column class measured slower this way: its rows
      // have enough products per round to keep the lanes busy, and half the lanes doubled its rounds)
      for_class(b, [&](auto cc) {
        constexpr int C = decltype(cc)::value;
        constexpr int wpb = 8;
        constexpr size_t per = size_t(2) * (2 * C * 4 + C * 4 + C * NC * 8 + 16 * 2 * NC * 8);
        static std::once_flag once;  // one size per instance: set once per process
        std::call_once(once, []() {
          cudaFuncSetAttribute(k_spgemm_fill_h<NC, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(per * wpb));
        });
        PS_TICK(); k_spgemm_fill_h<NC, C><<<unsigned((nr + 2 * wpb - 1) / (2 * wpb)), 32 * wpb, per * wpb, st>>>(
            rows, nr, xrp, xci, xv, yrp, yci, yv, *crp, *cci, *cv, islong, d_err);
      });
      continue;
    }
    for_class(b, [&](auto cc) {
      constexpr int C = decltype(cc)::value;
      const int wpb = C <= 128 ? 8 : (C <= 512 ? 4 : 2);
      size_t per = size_t(2 * C) * 4 + size_t(C) * 4 + size_t(C) * NC * 8 + size_t(32) * NC * 16;
      size_t sm = per * wpb;
      static std::once_flag once;  // one size per instance: set once per process
      std::call_once(once, [sm]() {
        cudaFuncSetAttribute(k_spgemm_fill<NC, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
      });
      PS_TICK(); k_spgemm_fill<NC, C><<<unsigned((nr + wpb - 1) / wpb), 32 * wpb, sm, st>>>(
          rows, nr, xrp, xci, xv, yrp, yci, yv, *crp, *cci, *cv, islong, d_err);
    });
  }
  PS_CUDA(cudaGetLastError());
  if (dense_ok && hl > 0) {
    const size_t sm = size_t(dense_wpb) * dense_per;
    // the largest allowed size, set once, the same for every caller (setups on several host threads)
    static std::once_flag once;
    std::call_once(once, []() {
      int dev = 0, maxsm = 0;
      cudaFuncAttributes fa;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      if (cudaFuncGetAttributes(&fa, k_spgemm_dense_fill_w<NC>) == cudaSuccess) maxsm -= int(fa.sharedSizeBytes);
      cudaFuncSetAttribute(k_spgemm_dense_fill_w<NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm);
      cudaGetLastError();
    });
    PS_TICK(); k_spgemm_dense_fill_w<NC><<<unsigned((hl + dense_wpb - 1) / dense_wpb), 32 * dense_wpb, sm, st>>>(
        longrows, hl, xrp, xci, xv, yrp, yci, yv, int32_t(m), words, *crp, *cci, *cv);
  }
  for (int64_t b0 = 0; !dense_ok && b0 < hl; b0 += B) {
    int32_t nb = int32_t(hl - b0 < B ? hl - b0 : B);
    PS_TICK(); k_spgemm_dense_fill<NC><<<nb, 256, 0, st>>>(longrows + b0, nb, xrp, xci, xv, yrp, yci, yv, stamp, acc, m,
                                                           *crp, *cci, *cv);
  }
  PS_CUDA(cudaGetLastError());
  if (stamp) { ar.release(stamp); ar.release(acc); }
  ar.release(cnt); ar.release(islong); ar.release(longrows); ar.release(nlong); ar.release(lists);
  ar.release(counts);
  return PS_OK;
}

// ---- Galerkin product R (A P) with few coarse columns, against a dense copy of A P ----
// A P (ny x m, m <= kDenseMaxCols) is scattered into a dense array Dn[k][j][c] that holds exact zeros off its
// pattern, and into one pattern bitmap per row.  Row i of the product takes as its pattern the union of the
// bitmaps of the A P rows that its R row touches, and each of its values is the sum over the R row, in
// ascending order, of r_ik (A P)_kj: the terms off the pattern of A P are exact zeros, which leave a running
// sum as it is, so the values equal those of the row-by-row sparse product.  All lanes work on outputs, where
// the sparse product of such short, dense rows is bound by the latency of its chain of inner indices.
__global__ void k_gal_densify(int64_t ny, int nc, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                              const double* __restrict__ v, int64_t m, int32_t words, double* __restrict__ Dn,
                              uint32_t* __restrict__ YB) {
  const int64_t k = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (k >= ny) return;
  for (int32_t q = rp[k] + lane; q < rp[k + 1]; q += 32) {
    const int32_t j = ci[q];
    for (int c = 0; c < nc; ++c) Dn[(k * m + j) * nc + c] = v[int64_t(q) * nc + c];
    atomicOr(&YB[k * words + (j >> 5)], 1u << (j & 31));
  }
}

__global__ void k_gal_count(int64_t n, const int32_t* __restrict__ xrp, const int32_t* __restrict__ xci,
                            const uint32_t* __restrict__ YB, int32_t words, uint32_t* __restrict__ XB,
                            int32_t* __restrict__ cnt) {
  const int64_t i = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  int c = 0;
  for (int32_t w0 = 0; w0 < words; w0 += 32) {
    const int32_t w = w0 + lane;
    uint32_t b = 0u;
    if (w < words)
      for (int32_t q = xrp[i]; q < xrp[i + 1]; ++q) b |= YB[int64_t(xci[q]) * words + w];
    if (w < words) XB[i * words + w] = b;
    c += __popc(b);
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) cnt[i] = c;
}

template <int NC>
__global__ void __launch_bounds__(256) k_gal_fill(int64_t n, const int32_t* __restrict__ xrp,
                                                  const int32_t* __restrict__ xci, const double* __restrict__ xv,
                                                  const double* __restrict__ Dn, int64_t m, int32_t words,
                                                  const uint32_t* __restrict__ XB, const int32_t* __restrict__ crp,
                                                  int32_t* __restrict__ cci, double* __restrict__ cv) {
  __shared__ int32_t cols[kDenseMaxCols];
  __shared__ int32_t wbase[33];
  const int64_t i = blockIdx.x;
  if (i >= n) return;
  // the row's columns in ascending order, from its bitmap (words <= 32: one warp scans the word counts)
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const uint32_t b = lane < words ? XB[i * words + lane] : 0u;
    const int32_t pc = __popc(b);
    int32_t inc = pc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += v;
    }
    wbase[lane] = inc - pc;
    if (lane == 31) wbase[32] = inc;
  }
  __syncthreads();
  for (int32_t w = threadIdx.x; w < words; w += blockDim.x) {
    uint32_t b = XB[i * words + w];
    int32_t pos = wbase[w];
    while (b) {
      const int t = __ffs(int(b)) - 1;
      b &= b - 1u;
      cols[pos++] = w * 32 + t;
    }
  }
  __syncthreads();
  const int32_t u = wbase[32], q0 = xrp[i], q1 = xrp[i + 1], o = crp[i];
  for (int32_t idx = threadIdx.x; idx < u * NC; idx += blockDim.x) {
    const int32_t slot = idx / NC, c = idx - slot * NC;
    const int64_t j = cols[slot];
    double acc = 0.0;
#pragma unroll 4
    for (int32_t q = q0; q < q1; ++q) acc = fma(xv[int64_t(q) * NC + c], Dn[(int64_t(xci[q]) * m + j) * NC + c], acc);
    cv[int64_t(o + slot) * NC + c] = acc;
    if (c == 0) cci[o + slot] = int32_t(j);
  }
}

// C = X Y with Y of m <= kDenseMaxCols columns by the dense-copy kernels above; *used = false (nothing done)
// when the dense copy of Y would exceed max_bytes
template <int NC>
ps_status galerkin_dense(Arena& ar, int64_t n, int64_t ny, int64_t m, const int32_t* xrp, const int32_t* xci,
                         const double* xv, const int32_t* yrp, const int32_t* yci, const double* yv, int32_t** crp,
                         int32_t** cci, double** cv, int64_t* cnnz, size_t max_bytes, bool* used, cudaStream_t st) {
  *used = false;
  const int32_t words = int32_t((m + 31) / 32);
  const size_t dbytes = size_t(ny) * size_t(m) * NC * 8;
  if (m > kDenseMaxCols || m < 1 || dbytes > max_bytes) return PS_OK;
  double* Dn;
  uint32_t *YB, *XB;
  int32_t* cnt;
  PS_TRY(ar.alloc(&Dn, size_t(ny) * m * NC));
  PS_TRY(ar.alloc(&YB, size_t(ny) * words + 1));
  PS_TRY(ar.alloc(&XB, size_t(n) * words + 1));
  PS_TRY(ar.alloc(&cnt, n + 1));
  PS_TRY(ar.alloc(crp, n + 1));
  PS_CUDA(cudaMemsetAsync(Dn, 0, dbytes, st));
  PS_CUDA(cudaMemsetAsync(YB, 0, sizeof(uint32_t) * (size_t(ny) * words + 1), st));
  PS_TICK(); k_gal_densify<<<grid_for(ny * 32, 256), 256, 0, st>>>(ny, NC, yrp, yci, yv, m, words, Dn, YB);
  PS_TICK(); k_gal_count<<<grid_for(n * 32, 256), 256, 0, st>>>(n, xrp, xci, YB, words, XB, cnt);
  PS_CUDA(cudaGetLastError());
  int32_t tot = 0;
  PS_TRY(scan_i32(ar, cnt, *crp, n, &tot, st));
  *cnnz = tot;
  PS_TRY(ar.alloc(cci, size_t(tot) + 1));
  PS_TRY(ar.alloc(cv, (size_t(tot) + 1) * NC));
  PS_TICK(); k_gal_fill<NC><<<unsigned(n), 256, 0, st>>>(n, xrp, xci, xv, Dn, m, words, XB, *crp, *cci, *cv);
  PS_CUDA(cudaGetLastError());
  ar.release(Dn); ar.release(YB); ar.release(XB); ar.release(cnt);
  *used = true;
  return PS_OK;
}

// The Gauss-Jordan inverse on one thread-block cluster per component, the matrix held in the cluster's
// distributed shared memory: CTA `rank` keeps physical rows [rank R, rank R + R) of A and of the inverse.  Row
// exchanges are a permutation (logical row r is physical row perm[r]).  The pivot is the largest |a| of
// column k over the logical rows >= k (ties: the smaller logical row); its row is divided by the pivot, and
// every other row subtracts its column-k entry times that row, with one fused multiply-add per entry.  In the
// inverse only the columns of the rows pivoted so far (perm[0..k]) can be nonzero in the pivot row, so only
// those are divided and updated.  Per pivot two hardware cluster barriers (no polling): one after the local
// column maxima, one after the division; then each CTA copies the pivot row and updates its own rows.
constexpr int kGjCluster = 16;
__global__ void __launch_bounds__(256) k_gj_cluster(int64_t n, int R, const double* __restrict__ M,
                                                    double* __restrict__ I) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ double gsm[];
  const int rank = int(cluster.block_rank());
  const int CS = int(cluster.num_blocks());
  const int c = int(blockIdx.x) / CS;
  const int nn = int(n);
  double* A = gsm;                         // [R][n]
  double* B = A + int64_t(R) * n;          // [R][n]
  double* prow = B + int64_t(R) * n;       // [2 n]: pivot row of A, then of B
  double* fv = prow + 2 * n;               // [R]: column-k entries of the own rows
  double* pval = fv + R;                   // [2]: local maximum, by pivot parity
  int* pidx = reinterpret_cast<int*>(pval + 2);  // [2]
  int* perm = pidx + 2;                    // [n]
  int* iperm = perm + n;                   // [n]
  __shared__ int sh_p;
  const int ph0 = rank * R;
  const int warp = int(threadIdx.x) >> 5, lane = int(threadIdx.x) & 31, nwarp = int(blockDim.x) >> 5;
  for (int lr = warp; lr < R; lr += nwarp) {
    const int ph = ph0 + lr;
    for (int j = lane; j < nn; j += 32) {
      A[int64_t(lr) * n + j] = ph < nn ? M[(int64_t(c) * n + ph) * n + j] : 0.0;
      B[int64_t(lr) * n + j] = (ph < nn && j == ph) ? 1.0 : 0.0;
    }
  }
  for (int r = threadIdx.x; r < nn; r += blockDim.x) {
    perm[r] = r;
    iperm[r] = r;
  }
  cluster.sync();
  for (int k = 0; k < nn; ++k) {
    const int par = k & 1;
    if (warp == 0) {
      double best = -1.0;
      int arg = INT_MAX;
      for (int lr = lane; lr < R; lr += 32) {
        const int ph = ph0 + lr;
        if (ph < nn && iperm[ph] >= k) {
          const double a = fabs(A[int64_t(lr) * n + k]);
          const int li = iperm[ph];
          if (a > best || (a == best && li < arg)) { best = a; arg = li; }
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
        if (ob > best || (ob == best && oa < arg)) { best = ob; arg = oa; }
      }
      if (lane == 0) { pval[par] = best; pidx[par] = arg; }
    }
    cluster.sync();
    if (warp == 0) {
      double best = -1.0;
      int arg = INT_MAX;
      if (lane < CS) {
        best = *cluster.map_shared_rank(pval + par, lane);
        arg = *cluster.map_shared_rank(pidx + par, lane);
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
        if (ob > best || (ob == best && oa < arg)) { best = ob; arg = oa; }
      }
      if (lane == 0) {
        const int p = arg == INT_MAX ? k : arg;
        const int rk = perm[k], rp = perm[p];
        perm[k] = rp; perm[p] = rk;
        iperm[rp] = k; iperm[rk] = p;
        sh_p = rp;
      }
    }
    __syncthreads();
    const int php = sh_p;  // physical row of the pivot
    const int owner = php / R, lp = php - owner * R;
    if (rank == owner) {
      const double piv = A[int64_t(lp) * n + k];
      __syncthreads();
      for (int j = k + threadIdx.x; j < nn; j += blockDim.x) A[int64_t(lp) * n + j] = A[int64_t(lp) * n + j] / piv;
      for (int jj = threadIdx.x; jj <= k; jj += blockDim.x) {
        const int j = perm[jj];
        B[int64_t(lp) * n + j] = B[int64_t(lp) * n + j] / piv;
      }
    }
    cluster.sync();
    {
      const double* rA = cluster.map_shared_rank(A, owner) + int64_t(lp) * n;
      const double* rB = cluster.map_shared_rank(B, owner) + int64_t(lp) * n;
      for (int j = k + threadIdx.x; j < nn; j += blockDim.x) prow[j] = rA[j];
      for (int jj = threadIdx.x; jj <= k; jj += blockDim.x) {
        const int j = perm[jj];
        prow[n + j] = rB[j];
      }
      for (int lr = threadIdx.x; lr < R; lr += blockDim.x) fv[lr] = A[int64_t(lr) * n + k];
    }
    __syncthreads();
    for (int lr = warp; lr < R; lr += nwarp) {
      const int ph = ph0 + lr;
      const double m = fv[lr];
      if (ph >= nn || ph == php || m == 0.0) continue;
      double* a = A + int64_t(lr) * n;
      double* b = B + int64_t(lr) * n;
      for (int j = k + lane; j < nn; j += 32) a[j] = fma(-m, prow[j], a[j]);
      for (int jj = lane; jj <= k; jj += 32) {
        const int j = perm[jj];
        b[j] = fma(-m, prow[n + j], b[j]);
      }
    }
    __syncthreads();
  }
  for (int lr = warp; lr < R; lr += nwarp) {
    const int ph = ph0 + lr;
    if (ph >= nn) continue;
    const int r = iperm[ph];
    for (int j = lane; j < nn; j += 32) I[(int64_t(c) * n + r) * n + j] = B[int64_t(lr) * n + j];
  }
  cluster.sync();  // no CTA leaves while another may still read its shared memory
}

// k_gj_cluster when the rows fit the clusters' shared memory: true when done
bool gj_cluster(int64_t n, int nc, const double* M, double* I, cudaStream_t st) {
  // device limits and kernel attributes, set once per process: the attributes take the largest allowed
  // shared-memory size, the same for every caller, so that setups on several host threads may launch at once
  static std::once_flag once;
  static int maxsm = 0;
  static bool nonportable = false;
  std::call_once(once, []() {
    int dev = 0;
    cudaFuncAttributes fa;
    // the dynamic limit is the opt-in maximum less the kernel's static shared memory
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, k_gj_cluster) != cudaSuccess ||
        (maxsm -= int(fa.sharedSizeBytes)) <= 0 ||
        cudaFuncSetAttribute(k_gj_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm) != cudaSuccess) {
      cudaGetLastError();
      maxsm = 0;
      return;
    }
    nonportable = cudaFuncSetAttribute(k_gj_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
    cudaGetLastError();
  });
  if (maxsm == 0) return false;
  // whether a cluster of cs CTAs with this much shared memory each can be resident: asked once per
  // (cluster size, 8 KB step of the size), the size rounded up
  static std::atomic<int8_t> fits[2][32];  // 0 unknown, 1 fits, 2 does not
  for (int t = 0; t < 2; ++t) {
    const int cs = t == 0 ? kGjCluster : 8;
    if (cs > 8 && !nonportable) continue;
    const int R = int((n + cs - 1) / cs);
    const size_t smem = (size_t(2) * R * n + 2 * n + R + 2) * 8 + size_t(2 + 2 * n) * 4;
    if (smem > size_t(maxsm) - 1024) continue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(cs * nc));
    cfg.blockDim = dim3(256);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = unsigned(cs);
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const int step = int(std::min<size_t>(31, (smem + 8191) / 8192));
    int8_t f = fits[t][step].load();
    if (f == 0) {
      cfg.dynamicSmemBytes = std::min<size_t>(size_t(step) * 8192, size_t(maxsm) - 1024);
      cfg.gridDim = dim3(unsigned(cs));
      int ncl = 0;
      f = (cudaOccupancyMaxActiveClusters(&ncl, k_gj_cluster, &cfg) == cudaSuccess && ncl >= 1) ? 1 : 2;
      cudaGetLastError();
      fits[t][step].store(f);
      cfg.gridDim = dim3(unsigned(cs * nc));
    }
    if (f != 1) continue;
    cfg.dynamicSmemBytes = smem;
    PS_TICK();
    if (cudaLaunchKernelEx(&cfg, k_gj_cluster, n, R, M, I) == cudaSuccess) return true;
    cudaGetLastError();
  }
  return false;
}

// The coarsest inverse by k_gj_all: 0 done, 1 not launched (no cooperative launch; the caller runs the
// launch-per-step path), 2 a grid barrier wait gave up (the inverse is incomplete)
// Cooperative launches of the inverse from setups on several host threads run one at a time (each waits for
// its kernel before releasing the lock): two grids that each wait for all their CTAs to be resident must not
// share the GPU.
std::mutex g_coop_gj;
int gj_cooperative(int64_t n, int nc, double* M, double* I, double* f, Arena& ar, cudaStream_t st) {
  std::lock_guard<std::mutex> lock(g_coop_gj);
  int dev = 0, coop = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gj_all, 256, 0) != cudaSuccess || !coop || occ < 1) {
    cudaGetLastError();
    return 1;
  }
  unsigned long long* bar;
  int* err;
  if (ar.alloc(&bar, 1) != PS_OK) return 1;
  if (ar.alloc(&err, 1) != PS_OK) { ar.release(bar); return 1; }
  cudaMemsetAsync(bar, 0, sizeof(unsigned long long), st);
  cudaMemsetAsync(err, 0, sizeof(int), st);
  int64_t limit = 20000000;
  const unsigned grid = unsigned(std::max(nc, sms));
  void* args[] = {&n, &nc, &M, &I, &f, &bar, &limit, &err};
  int result = 0;
  if (cudaLaunchCooperativeKernel((const void*)k_gj_all, grid, 256, args, 0, st) != cudaSuccess) {
    cudaGetLastError();
    result = 1;
  } else {
    PS_TICK();
    int h = 0;
    cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    if (h) result = 2;
  }
  ar.release(bar);
  ar.release(err);
  return result;
}

// Gauss-Jordan inverses of nc dense n x n matrices (M is overwritten, inv starts as the identity): one
// thread-block cluster per component when its rows fit the cluster's shared memory, else one cooperative
// launch, else one launch pair per pivot
ps_status gj_inverse(int64_t n, int nc, double* M, double* inv, double* f, Arena& ar, cudaStream_t st) {
  if (gj_cluster(n, nc, M, inv, st)) {
    PS_CUDA(cudaGetLastError());
    return PS_OK;
  }
  const int gj = gj_cooperative(n, nc, M, inv, f, ar, st);
  if (gj == 2) {
    set_reason("a bounded grid barrier wait of the coarsest-level Gauss-Jordan inverse gave up");
    return PS_ERR_TIMEOUT;
  }
  if (gj == 1) {
    for (int64_t k = 0; k < n; ++k) {
      PS_TICK(); k_gj_pivot<<<nc, 256, 0, st>>>(n, k, M, inv, f);
      dim3 g(unsigned(ceil_div(2 * n, 128)), unsigned(n), unsigned(nc));
      PS_TICK(); k_gj_elim<<<g, 128, 0, st>>>(n, k, M, inv, f);
    }
  }
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

// Aggregation of one level: symmetric strength graph, distance-2 MIS rounds under the priority key of the
// level, phase 1 (strong neighbours of a root join it), phase 2 (leftovers join their strongest phase-1
// neighbour).  dgbar and excl as k_diag_excl leaves them; *agg is allocated here (-1: not aggregated).
template <int NC>
ps_status aggregate_impl(Arena& ar, int64_t n, int64_t nnz, const int32_t* rp, const int32_t* ci, const double* v,
                         const double* dgbar, const uint8_t* excl, double theta, int l, int32_t** agg, int64_t* nagg,
                         cudaStream_t st) {
  uint8_t *strong = nullptr, *stt = nullptr;
  double* wgt = nullptr;
  PS_TRY(ar.alloc(&strong, nnz));
  PS_TRY(ar.alloc(&wgt, nnz));
  PS_TICK(); k_strength<NC><<<grid_for(n * kStrLanes, 256), 256, 0, st>>>(n, rp, ci, v, dgbar, excl, theta, strong,
                                                                         wgt);
  PS_TRY(ar.alloc(&stt, n));
  int64_t* m1;
  uint8_t *nr, *c1;
  int32_t* und;
  // rounds go in batches between host checks, two then kMisBatch (small levels often finish within two
  // rounds); und[b] is the undecided flag of round b of a batch
  constexpr int kMisBatch = 4;
  PS_TRY(ar.alloc(&m1, n)); PS_TRY(ar.alloc(&nr, n)); PS_TRY(ar.alloc(&c1, n)); PS_TRY(ar.alloc(&und, kMisBatch));
  int64_t* key;
  PS_TRY(ar.alloc(&key, n));
  PS_TICK(); k_mis_keys<<<grid_for(n, 256), 256, 0, st>>>(n, l, key);
  PS_TICK(); k_mis_init<<<grid_for(n, 256), 256, 0, st>>>(n, rp, strong, excl, stt);
  for (int round = 0, nbat = 2;; round += nbat, nbat = kMisBatch) {
    PS_CUDA(cudaMemsetAsync(und, 0, sizeof(int32_t) * kMisBatch, st));
    for (int b = 0; b < nbat; ++b) {
      const int32_t* prev = b > 0 ? und + b - 1 : nullptr;
      PS_TICK(); k_mis_m1<<<grid_for(n * kMisLanes, 256), 256, 0, st>>>(n, rp, ci, strong, stt, key, m1, prev);
      PS_TICK(); k_mis_m2<<<grid_for(n * kMisLanes, 256), 256, 0, st>>>(n, rp, ci, strong, m1, key, stt, nr, prev);
      PS_TICK(); k_mis_c1<<<grid_for(n * kMisLanes, 256), 256, 0, st>>>(n, rp, ci, strong, nr, c1, prev);
      PS_TICK(); k_mis_c2<<<grid_for(n * kMisLanes, 256), 256, 0, st>>>(n, rp, ci, strong, c1, stt, und + b, prev);
    }
    int32_t h_und = 0;
    PS_CUDA(cudaMemcpyAsync(&h_und, und + nbat - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    if (h_und == 0) break;
    if (round > 100000) {
      set_reason("aggregation did not terminate on level %d", l);
      return PS_ERR_INVALID;
    }
  }
  int32_t *isr, *rscan, *ph1;
  PS_TRY(ar.alloc(&isr, n)); PS_TRY(ar.alloc(&rscan, n + 1)); PS_TRY(ar.alloc(&ph1, n));
  PS_TRY(ar.alloc(agg, n));
  PS_TICK(); k_is_root<<<grid_for(n, 256), 256, 0, st>>>(n, stt, isr);
  int32_t na = 0;
  PS_TRY(scan_i32(ar, isr, rscan, n, &na, st));
  PS_TICK(); k_agg_phase1<<<grid_for(n, 256), 256, 0, st>>>(n, rp, ci, strong, stt, rscan, ph1);
  PS_TICK(); k_agg_phase2<<<grid_for(n, 256), 256, 0, st>>>(n, rp, ci, strong, wgt, stt, ph1, *agg);
  PS_CUDA(cudaGetLastError());
  *nagg = na;
  ar.release(m1); ar.release(nr); ar.release(c1); ar.release(und); ar.release(key); ar.release(isr); ar.release(rscan);
  ar.release(ph1); ar.release(strong); ar.release(wgt); ar.release(stt);
  return PS_OK;
}

template <int NC>
ps_status build_impl(Arena& ar, Amg& H, int64_t n0, int64_t nnz0, int32_t* rp0, int32_t* ci0, double* v0,
                     const AmgParams& prm, cudaStream_t st) {
  H.nc = NC;
  H.L.clear();
  H.L.emplace_back();
  H.L[0].n = n0; H.L[0].nnz = nnz0; H.L[0].rp = rp0; H.L[0].ci = ci0; H.L[0].v = v0;
  int* d_err;
  PS_TRY(ar.alloc(&d_err, 4));
  PS_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), st));
  double theta = prm.theta;
  for (int l = 0;; ++l) {
    AmgLevel& lev = H.L[l];
    int64_t n = lev.n, nnz = lev.nnz;
    lev.lanes = lanes_for(double(nnz) / double(n > 0 ? n : 1));
    double* dgbar;
    uint8_t* excl;
    PS_TRY(ar.alloc(&dgbar, n));
    PS_TRY(ar.alloc(&excl, n));
    PS_TRY(ar.alloc(&lev.dg, n * NC));
    PS_TICK(); k_diag_excl<NC><<<grid_for(n, 256), 256, 0, st>>>(n, lev.rp, lev.ci, lev.v, dgbar, excl, lev.dg);
    PS_CUDA(cudaGetLastError());
    bool coarsest = n <= prm.coarse_max || l + 1 >= prm.max_levels;
    if (!coarsest) {
      int64_t na = 0;
      PS_TRY(aggregate_impl<NC>(ar, n, nnz, lev.rp, lev.ci, lev.v, dgbar, excl, theta, l, &lev.agg, &na, st));
      lev.nagg = na;
      if (na == 0 || double(n) / double(na) < 1.2) coarsest = true;
    }
    if (coarsest) {
      if (n > 16384) {  // coarsening stalled on a large level
        set_reason("coarsening stalled: level %d has %lld rows (nc=%d)", l, (long long)n, NC);
        return PS_ERR_INVALID;
      }
      lev.coarsest = true;
      lev.nagg = 0;
      if (lev.agg) { ar.release(lev.agg); lev.agg = nullptr; }
      double *M, *f;
      PS_TRY(ar.alloc(&M, size_t(NC) * n * n));
      PS_TRY(ar.alloc(&lev.inv, size_t(NC) * n * n));
      PS_TRY(ar.alloc(&f, size_t(NC) * n));
      PS_CUDA(cudaMemsetAsync(M, 0, sizeof(double) * NC * n * n, st));
      PS_CUDA(cudaMemsetAsync(lev.inv, 0, sizeof(double) * NC * n * n, st));
      PS_TICK(); k_dense_unpack<<<grid_for(n, 128), 128, 0, st>>>(n, NC, lev.rp, lev.ci, lev.v, M, lev.inv);
      PS_TRY(gj_inverse(n, NC, M, lev.inv, f, ar, st));
      ar.release(M); ar.release(f);
    }
    if (coarsest) { ar.release(dgbar); ar.release(excl); }
    if (prm.mixed) {
      PS_TRY(ar.alloc(&lev.vf, nnz * NC));
      PS_TRY(ar.alloc(&lev.dgf, n * NC));
      PS_TICK(); k_to_f32<<<grid_for(nnz * NC, 256), 256, 0, st>>>(lev.v, lev.vf, nnz * NC);
      PS_TICK(); k_to_f32<<<grid_for(n * NC, 256), 256, 0, st>>>(lev.dg, lev.dgf, n * NC);
    }
    if (lev.coarsest) break;
    // Gershgorin bound, omega = (4/3) / lambda
    double* gr;
    PS_TRY(ar.alloc(&gr, n * NC));
    PS_TICK(); k_gersh<NC><<<grid_for(n, 256), 256, 0, st>>>(n, lev.rp, lev.ci, lev.v, gr);
    double* dmax;
    PS_TRY(ar.alloc(&dmax, NC));
    for (int c = 0; c < NC; ++c) PS_TRY(max_f64(ar, gr + c * n, n, dmax + c, st));
    PS_CUDA(cudaMemcpyAsync(lev.lam, dmax, sizeof(double) * NC, cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    ar.release(gr); ar.release(dmax);
    double om[3] = {0, 0, 0};
    for (int c = 0; c < NC; ++c) om[c] = (4.0 / 3.0) / lev.lam[c];
    // l1 row norms for the l1-Jacobi smoother
    if (prm.l1) {
      PS_TRY(ar.alloc(&lev.dl1, n * NC));
      PS_TICK(); k_l1<NC><<<grid_for(n, 256), 256, 0, st>>>(n, lev.rp, lev.v, lev.dl1);
      if (prm.mixed) {
        PS_TRY(ar.alloc(&lev.dl1f, n * NC));
        PS_TICK(); k_to_f32<<<grid_for(n * NC, 256), 256, 0, st>>>(lev.dl1, lev.dl1f, n * NC);
      }
    }
    // prolongator: T = A P_tent by the deterministic SpGEMM, then P = P_tent - omega D^{-1} T
    int64_t na = lev.nagg;
    int32_t *trp0, *tci0, *pc;
    double* tv0;
    PS_TRY(ar.alloc(&pc, n + 1));
    PS_TRY(ar.alloc(&trp0, n + 1));
    PS_TICK(); k_ptent_count<<<grid_for(n, 256), 256, 0, st>>>(n, lev.agg, pc);
    int32_t nt = 0;
    PS_TRY(scan_i32(ar, pc, trp0, n, &nt, st));
    PS_TRY(ar.alloc(&tci0, size_t(nt) + 1));
    PS_TRY(ar.alloc(&tv0, (size_t(nt) + 1) * NC));
    PS_TICK(); k_ptent_fill<NC><<<grid_for(n, 256), 256, 0, st>>>(n, lev.agg, trp0, tci0, tv0);
    int32_t *Trp, *Tci;
    double* Tv;
    int64_t Tnnz = 0;
    PS_TRY(spgemm<NC>(ar, n, na, lev.rp, lev.ci, lev.v, trp0, tci0, tv0, &Trp, &Tci, &Tv, &Tnnz, d_err, st));
    ar.release(trp0); ar.release(tci0); ar.release(tv0);
    PS_TRY(ar.alloc(&lev.prp, n + 1));
    PS_TICK(); k_p_rowlen<<<grid_for(n, 256), 256, 0, st>>>(n, Trp, excl, pc);
    int32_t pnnz = 0;
    PS_TRY(scan_i32(ar, pc, lev.prp, n, &pnnz, st));
    lev.pnnz = pnnz;
    PS_TRY(ar.alloc(&lev.pci, size_t(pnnz) + 1));
    PS_TRY(ar.alloc(&lev.pv, (size_t(pnnz) + 1) * NC));
    PS_TICK(); k_p_finish<NC><<<grid_for(n, 256), 256, 0, st>>>(n, Trp, Tci, Tv, excl, lev.agg, lev.dg, om[0], om[1],
                                                                 om[2], lev.prp, lev.pci, lev.pv);
    PS_CUDA(cudaGetLastError());
    ar.release(pc); ar.release(Trp); ar.release(Tci); ar.release(Tv);
    lev.plane = lanes_for(double(pnnz) / double(n));
    // restriction R = P^T
    int32_t *ccount, *cursor, *tci;
    double* tv;
    PS_TRY(ar.alloc(&ccount, na + 1));
    PS_TRY(ar.alloc(&lev.rrp, na + 1));
    PS_TRY(ar.alloc(&cursor, na + 1));
    PS_TRY(ar.alloc(&tci, size_t(pnnz) + 1));
    PS_TRY(ar.alloc(&tv, (size_t(pnnz) + 1) * NC));
    PS_TRY(ar.alloc(&lev.rci, size_t(pnnz) + 1));
    PS_TRY(ar.alloc(&lev.rv, (size_t(pnnz) + 1) * NC));
    PS_CUDA(cudaMemsetAsync(ccount, 0, sizeof(int32_t) * (na + 1), st));
    PS_TICK(); k_col_count<<<grid_for(pnnz, 256), 256, 0, st>>>(pnnz, lev.pci, ccount);
    PS_TRY(scan_i32(ar, ccount, lev.rrp, na, nullptr, st));
    PS_CUDA(cudaMemcpyAsync(cursor, lev.rrp, sizeof(int32_t) * na, cudaMemcpyDeviceToDevice, st));
    PS_TICK(); k_transpose_fill<NC><<<grid_for(n, 256), 256, 0, st>>>(n, lev.prp, lev.pci, lev.pv, cursor, tci, tv);
    PS_TICK(); k_rank_rows<NC><<<grid_for(na * 32, 256), 256, 0, st>>>(na, lev.rrp, tci, tv, lev.rci, lev.rv);
    PS_CUDA(cudaGetLastError());
    ar.release(ccount); ar.release(cursor); ar.release(tci); ar.release(tv);
    lev.rlane = lanes_for(double(pnnz) / double(na));
    if (prm.mixed) {
      PS_TRY(ar.alloc(&lev.pvf, size_t(pnnz) * NC + 1));
      PS_TRY(ar.alloc(&lev.rvf, size_t(pnnz) * NC + 1));
      PS_TICK(); k_to_f32<<<grid_for(pnnz * NC, 256), 256, 0, st>>>(lev.pv, lev.pvf, pnnz * NC);
      PS_TICK(); k_to_f32<<<grid_for(pnnz * NC, 256), 256, 0, st>>>(lev.rv, lev.rvf, pnnz * NC);
      if (prm.bf16p) {
        PS_TRY(ar.alloc(&lev.pvb, size_t(pnnz) * NC + 8));
        PS_TRY(ar.alloc(&lev.rvb, size_t(pnnz) * NC + 8));
        PS_TICK(); k_to_bf16<<<grid_for(pnnz * NC, 256), 256, 0, st>>>(lev.pv, lev.pvb, pnnz * NC);
        PS_TICK(); k_to_bf16<<<grid_for(pnnz * NC, 256), 256, 0, st>>>(lev.rv, lev.rvb, pnnz * NC);
      }
    }
    // Galerkin product A_c = R (A P)
    int32_t *aprp, *apci, *crp, *cci;
    double *apv, *cv;
    int64_t apnnz = 0, cnnz = 0;
    PS_TRY(spgemm<NC>(ar, n, na, lev.rp, lev.ci, lev.v, lev.prp, lev.pci, lev.pv, &aprp, &apci, &apv, &apnnz, d_err, st));
    bool dense_rap = false;
    PS_TRY(galerkin_dense<NC>(ar, na, n, na, lev.rrp, lev.rci, lev.rv, aprp, apci, apv, &crp, &cci, &cv, &cnnz,
                              size_t(512) << 20, &dense_rap, st));
    if (!dense_rap)
      PS_TRY(spgemm<NC>(ar, na, na, lev.rrp, lev.rci, lev.rv, aprp, apci, apv, &crp, &cci, &cv, &cnnz, d_err, st));
    int herr = 0;
    PS_CUDA(cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    if (herr) {
      set_reason("SpGEMM capacity exceeded on level %d", l);
      return PS_ERR_INVALID;
    }
    ar.release(aprp); ar.release(apci); ar.release(apv);
    ar.release(dgbar);
    ar.release(excl);
    H.L.emplace_back();
    AmgLevel& nx = H.L.back();
    nx.n = na; nx.nnz = cnnz; nx.rp = crp; nx.ci = cci; nx.v = cv;
    theta *= 0.5;
  }
  // Gershgorin bounds for the levels that did not compute one (coarsest)
  ar.release(d_err);
  return PS_OK;
}

}  // namespace

ps_status amg_build(Arena& ar, Amg& H, int nc, int64_t n, int64_t nnz, int32_t* rp, int32_t* ci, double* v,
                    const AmgParams& prm, cudaStream_t st) {
  if (nc == 3) return build_impl<3>(ar, H, n, nnz, rp, ci, v, prm, st);
  if (nc == 1) return build_impl<1>(ar, H, n, nnz, rp, ci, v, prm, st);
  return PS_ERR_INVALID;
}

ps_status amg_aggregate_scalar(Arena& ar, int64_t n, int64_t nnz, const int32_t* rp, const int32_t* ci,
                               const double* v, double theta, int level, int32_t** agg, int64_t* nagg,
                               uint8_t** excl, cudaStream_t st) {
  double *dgbar, *dg;
  PS_TRY(ar.alloc(&dgbar, n));
  PS_TRY(ar.alloc(&dg, n));
  PS_TRY(ar.alloc(excl, n));
  PS_TICK(); k_diag_excl<1><<<grid_for(n, 256), 256, 0, st>>>(n, rp, ci, v, dgbar, *excl, dg);
  PS_CUDA(cudaGetLastError());
  PS_TRY(aggregate_impl<1>(ar, n, nnz, rp, ci, v, dgbar, *excl, theta, level, agg, nagg, st));
  ar.release(dgbar);
  ar.release(dg);
  return PS_OK;
}

ps_status amg_spgemm_pattern(Arena& ar, int64_t n, int64_t m, const int32_t* xrp, const int32_t* xci, int64_t xnnz,
                             const int32_t* yrp, const int32_t* yci, int64_t ynnz, int32_t** crp, int32_t** cci,
                             int64_t* cnnz, cudaStream_t st) {
  double *xo, *yo, *cv;
  int* d_err;
  PS_TRY(ar.alloc(&xo, xnnz + 1));
  PS_TRY(ar.alloc(&yo, ynnz + 1));
  PS_TRY(ar.alloc(&d_err, 1));
  PS_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), st));
  PS_TICK(); k_fill_one<<<grid_for(xnnz + 1, 256), 256, 0, st>>>(xo, xnnz + 1);
  PS_TICK(); k_fill_one<<<grid_for(ynnz + 1, 256), 256, 0, st>>>(yo, ynnz + 1);
  PS_TRY(spgemm<1>(ar, n, m, xrp, xci, xo, yrp, yci, yo, crp, cci, &cv, cnnz, d_err, st));
  int herr = 0;
  PS_CUDA(cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  PS_CUDA(cudaStreamSynchronize(st));
  ar.release(xo); ar.release(yo); ar.release(cv); ar.release(d_err);
  if (herr) {
    set_reason("SpGEMM capacity exceeded in a block Galerkin product");
    return PS_ERR_INVALID;
  }
  return PS_OK;
}

ps_status amg_dense_inverse(Arena& ar, int64_t n, double* M, double* inv, cudaStream_t st) {
  double* f;
  PS_TRY(ar.alloc(&f, n));
  PS_TRY(gj_inverse(n, 1, M, inv, f, ar, st));
  ar.release(f);
  return PS_OK;
}

namespace {

// slot of the neighbour offset (dx, dy, dz) in the ns-point pattern, -1 if it is not one
__device__ __forceinline__ int stencil_slot(int ns, int dx, int dy, int dz) {
  if (dx < -1 || dx > 1 || dy < -1 || dy > 1 || dz < -1 || dz > 1) return -1;
  if (ns == 27) return (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
  int nz = (dx != 0) + (dy != 0) + (dz != 0);
  if (nz > 1) return -1;
  if (dz == -1) return 0;
  if (dy == -1) return 1;
  if (dx == -1) return 2;
  if (dx == 1) return 4;
  if (dy == 1) return 5;
  if (dz == 1) return 6;
  return 3;
}

template <class T>
__global__ void k_level_to_stencil(int64_t n, int gx, int gy, int ns, int nc, const int32_t* __restrict__ rp,
                                   const int32_t* __restrict__ ci, const double* __restrict__ v, T* __restrict__ sv,
                                   int* bad) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t gxy = int64_t(gx) * gy;
  const int iz = int(i / gxy);
  const int64_t rem = i - iz * gxy;
  const int iy = int(rem / gx), ix = int(rem - int64_t(iy) * gx);
  for (int32_t q = rp[i]; q < rp[i + 1]; ++q) {
    int64_t j = ci[q];
    const int jz = int(j / gxy);
    const int64_t jr = j - jz * gxy;
    const int jy = int(jr / gx), jx = int(jr - int64_t(jy) * gx);
    int s = stencil_slot(ns, jx - ix, jy - iy, jz - iz);
    if (s < 0) {
      atomicExch(bad, 1);
      continue;
    }
    for (int c = 0; c < nc; ++c) sv[(int64_t(s) * nc + c) * n + i] = T(v[int64_t(q) * nc + c]);
  }
}

}  // namespace

ps_status amg_stencil(Arena& ar, Amg& H, int gx, int gy, int gz, int ns, bool mixed, bool* ok, cudaStream_t st) {
  *ok = false;
  if (H.L.empty()) return PS_OK;
  AmgLevel& L = H.L[0];
  if (L.coarsest || int64_t(gx) * gy * gz != L.n || L.n >= int64_t(INT32_MAX) || (ns != 27 && ns != 7)) return PS_OK;
  int nc = H.nc;
  size_t cnt = size_t(ns) * nc * L.n;
  int* bad = nullptr;
  PS_TRY(ar.alloc(&bad, 1));
  PS_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
  if (mixed) {
    PS_TRY(ar.alloc(&L.sv_f, cnt));
    PS_CUDA(cudaMemsetAsync(L.sv_f, 0, cnt * sizeof(float), st));
    PS_TICK(); k_level_to_stencil<float><<<grid_for(L.n, 256), 256, 0, st>>>(L.n, gx, gy, ns, nc, L.rp, L.ci, L.v,
                                                                            L.sv_f, bad);
  } else {
    PS_TRY(ar.alloc(&L.sv_d, cnt));
    PS_CUDA(cudaMemsetAsync(L.sv_d, 0, cnt * sizeof(double), st));
    PS_TICK(); k_level_to_stencil<double><<<grid_for(L.n, 256), 256, 0, st>>>(L.n, gx, gy, ns, nc, L.rp, L.ci,
                                                                             L.v, L.sv_d, bad);
  }
  PS_CUDA(cudaGetLastError());
  int hb = 0;
  PS_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  PS_CUDA(cudaStreamSynchronize(st));
  ar.release(bad);
  if (hb) {
    if (L.sv_f) ar.release(L.sv_f);
    if (L.sv_d) ar.release(L.sv_d);
    L.sv_f = nullptr;
    L.sv_d = nullptr;
    return PS_OK;
  }
  L.sgx = gx; L.sgy = gy; L.sgz = gz; L.sns = ns;
  *ok = true;
  return PS_OK;
}

}  // namespace ps_internal
