// Algorithm 1, flow part: steps 2-4 (A_fu coupling, D_ss^{-1}, complete A_ps)
// and steps 6-8 (residual of S_ff^(FS), block ILU(0) forward / backward sweeps,
// correction), in the interleaved (s, p) cell ordering of §5.3.
#include "flow.cuh"

namespace ps_internal {
namespace {

template <class T>
struct FlowView {
  const T *fu, *sff, *aps, *dinv, *dss, *s28;
};
template <class T>
FlowView<T> fview(const FlowStage& F) {
  FlowView<T> o;
  if constexpr (sizeof(T) == 4) {
    o.fu = F.fu_vf; o.sff = F.sff_f; o.aps = F.aps_f; o.dinv = F.dinv_f; o.dss = F.dss_f; o.s28 = F.s28_f;
  } else {
    o.fu = F.fu_v; o.sff = F.sff; o.aps = F.aps; o.dinv = F.dinv; o.dss = F.dss; o.s28 = F.s28;
  }
  return o;
}

// steps 2-3: y_f = v_f - A_fu z_u ; z_s = D_ss^{-1} y_s   (8 lanes per cell, one 2x3 block each)
template <class T>
__global__ void k_step23(int64_t nc, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                         const T* __restrict__ fu, const T* __restrict__ vf, const T* __restrict__ zu,
                         const T* __restrict__ dss, T* __restrict__ y, T* __restrict__ zs) {
  int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  int64_t c = tid >> 3;
  int sub = int(tid & 7);
  bool active = c < nc;
  T a0 = T(0), a1 = T(0);
  if (active) {
    int32_t q = rp[c] + sub;
    if (q < rp[c + 1]) {
      int64_t J = ci[q];
      const T* b = fu + int64_t(q) * 6;
      T x0 = zu[3 * J], x1 = zu[3 * J + 1], x2 = zu[3 * J + 2];
      a0 = b[0] * x0 + b[1] * x1 + b[2] * x2;
      a1 = b[3] * x0 + b[4] * x1 + b[5] * x2;
    }
  }
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
  }
  if (active && sub == 0) {
    T ys = vf[2 * c] - a0, yp = vf[2 * c + 1] - a1;
    y[2 * c] = ys;
    y[2 * c + 1] = yp;
    zs[c] = ys / dss[c];
  }
}

// steps 2-3 with A_fu by cell corner (blocked by 32 cells), one thread per cell
template <class T>
__global__ void k_step23_st(int nx, int ny, int nz, const T* __restrict__ fu, const T* __restrict__ vf,
                            const T* __restrict__ zu, const T* __restrict__ dss, T* __restrict__ y,
                            T* __restrict__ zs) {
  int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t nc = int64_t(nx) * ny * nz;
  if (c >= nc) return;
  const int i = int(c % nx), j = int((c / nx) % ny), k = int(c / (int64_t(nx) * ny));
  const T* A = fu + (c >> 5) * int64_t(8 * 6 * 32) + (c & 31);
  T a0 = T(0), a1 = T(0);
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int64_t J = (i + (s & 1)) + int64_t(nx + 1) * ((j + ((s >> 1) & 1)) + int64_t(ny + 1) * (k + (s >> 2)));
    const T x0 = zu[3 * J], x1 = zu[3 * J + 1], x2 = zu[3 * J + 2];
    const T* b = A + s * 6 * 32;
    a0 = fma(b[0], x0, a0); a0 = fma(b[32], x1, a0); a0 = fma(b[64], x2, a0);
    a1 = fma(b[96], x0, a1); a1 = fma(b[128], x1, a1); a1 = fma(b[160], x2, a1);
  }
  const T ys = vf[2 * c] - a0, yp = vf[2 * c + 1] - a1;
  y[2 * c] = ys;
  y[2 * c + 1] = yp;
  zs[c] = ys / dss[c];
}

// step 4 with A_ps by 7-point slot (blocked by 32 cells), one thread per cell
template <class T>
__global__ void k_step4_st(int nx, int ny, int nz, const T* __restrict__ aps, const T* __restrict__ y,
                           const T* __restrict__ zs, T* __restrict__ wp) {
  int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t nc = int64_t(nx) * ny * nz, nxy = int64_t(nx) * ny;
  if (c >= nc) return;
  const int i = int(c % nx), j = int((c / nx) % ny), k = int(c / nxy);
  const int64_t nb[7] = {c - nxy, c - nx, c - 1, c, c + 1, c + nx, c + nxy};
  const bool in[7] = {k > 0, j > 0, i > 0, true, i + 1 < nx, j + 1 < ny, k + 1 < nz};
  const T* A = aps + (c >> 5) * int64_t(7 * 32) + (c & 31);
  T a = T(0);
#pragma unroll
  for (int q = 0; q < 7; ++q)
    if (in[q]) a = fma(A[q * 32], zs[nb[q]], a);
  wp[c] = y[2 * c + 1] - a;
}

// step 4: w_p = y_p - A_ps z_s with the complete A_ps (8 lanes per cell)
template <class T>
__global__ void k_step4(int64_t nc, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                        const T* __restrict__ aps, const T* __restrict__ y, const T* __restrict__ zs,
                        T* __restrict__ wp) {
  int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  int64_t c = tid >> 3;
  int sub = int(tid & 7);
  bool active = c < nc;
  T a = T(0);
  if (active) {
    int32_t q = rp[c] + sub;
    if (q < rp[c + 1]) a = aps[q] * zs[ci[q]];
  }
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if (active && sub == 0) wp[c] = y[2 * c + 1] - a;
}

// ILU forward sweep fused with step 6, one wavefront level:
//   w_i = y_i - sum_j S_ij z_j ; u_i = w_i - sum_{k<i} S_ik t_k ; t_i = inv(U_ii) u_i
// (processor-local scope: the sum over k leaves out cells of other tiles)
template <class T>
__global__ void k_ilu_fwd(const int32_t* __restrict__ cells, int32_t m, const int32_t* __restrict__ rp,
                          const int32_t* __restrict__ ci, const int32_t* __restrict__ diagpos,
                          const T* __restrict__ sff, const T* __restrict__ dinv, const T* __restrict__ y,
                          const T* __restrict__ zs, const T* __restrict__ zp, T* __restrict__ t, int nx, int ny,
                          int local) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m) return;
  int32_t i = cells[idx];
  int32_t qd = diagpos[i];
  T w0 = y[2 * i], w1 = y[2 * i + 1];
  for (int32_t q = rp[i]; q < rp[i + 1]; ++q) {
    int32_t j = ci[q];
    const T* S = sff + int64_t(q) * 4;
    T zsj = zs[j], zpj = zp[j];
    w0 -= S[0] * zsj + S[1] * zpj;
    w1 -= S[2] * zsj + S[3] * zpj;
    if (q < qd && !(local && cross_tile(i, j, nx, ny))) {
      T t0 = t[2 * j], t1 = t[2 * j + 1];
      w0 -= S[0] * t0 + S[1] * t1;
      w1 -= S[2] * t0 + S[3] * t1;
    }
  }
  const T* D = dinv + int64_t(i) * 4;
  t[2 * i] = D[0] * w0 + D[1] * w1;
  t[2 * i + 1] = D[2] * w0 + D[3] * w1;
}

// ILU backward sweep fused with step 8, one level:
//   dz_i = t_i - inv(U_ii) sum_{j>i} S_ij dz_j ; z_f = (z_s, z_p) + dz  -> FP64 output
template <class T>
__global__ void k_ilu_bwd(const int32_t* __restrict__ cells, int32_t m, const int32_t* __restrict__ rp,
                          const int32_t* __restrict__ ci, const int32_t* __restrict__ diagpos,
                          const T* __restrict__ sff, const T* __restrict__ dinv, const T* __restrict__ t,
                          const T* __restrict__ zs, const T* __restrict__ zp, T* __restrict__ dz,
                          double* __restrict__ zout, int nx, int ny, int local) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m) return;
  int32_t i = cells[idx];
  int32_t qd = diagpos[i];
  T a0 = T(0), a1 = T(0);
  for (int32_t q = qd + 1; q < rp[i + 1]; ++q) {
    int32_t j = ci[q];
    if (local && cross_tile(i, j, nx, ny)) continue;
    const T* S = sff + int64_t(q) * 4;
    T d0 = dz[2 * j], d1 = dz[2 * j + 1];
    a0 += S[0] * d0 + S[1] * d1;
    a1 += S[2] * d0 + S[3] * d1;
  }
  const T* D = dinv + int64_t(i) * 4;
  T e0 = t[2 * i] - (D[0] * a0 + D[1] * a1);
  T e1 = t[2 * i + 1] - (D[2] * a0 + D[3] * a1);
  dz[2 * i] = e0;
  dz[2 * i + 1] = e1;
  zout[2 * i] = double(zs[i] + e0);
  zout[2 * i + 1] = double(zp[i] + e1);
}

// ---------------------------------------------------------------------------
// Sync-free wavefront sweeps over the stencil-indexed S_ff^(FS).
// Thread (ly, lz) of CTA (BY, BZ) owns the x-pencil (y, z) = (BY*kTY + ly,
// BZ*kTZ + lz) and walks it sequentially: at CTA step s it handles position
// s - ry - rz (ry, rz = distance from the producing CTA boundary), so its y- and
// z-predecessors inside the CTA were computed at step s - 1 (double-buffered
// shared array, one barrier per step).  Values crossing a CTA boundary go
// through a halo buffer of 64-bit words that each carry a 32-bit payload and the
// 32-bit sweep tag (single-copy atomic stores, so no fence or flag is needed):
// consumers prefetch the words they need two steps ahead, at the start of a step,
// and re-read them only while the tag is not yet the current one; the wait is
// bounded and raises *err.
// The cell records, which do not depend on the wavefront, arrive by bulk copy
// one to two copy windows ahead (see k_ilu_pencil).
// ---------------------------------------------------------------------------

template <class T>
struct HaloWord {
  static constexpr int W = int(sizeof(T)) * 2 / 4;  // 32-bit chunks of a (v0, v1) pair
};

__device__ __forceinline__ void st_relaxed64(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_relaxed64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

template <class T>
__device__ __forceinline__ void halo_put(uint64_t* h, int64_t i, T v0, T v1, uint32_t tag) {
  constexpr int W = HaloWord<T>::W;
  uint32_t c[W];
  if constexpr (sizeof(T) == 4) {
    c[0] = __float_as_uint(v0);
    c[1] = __float_as_uint(v1);
  } else {
    uint64_t a = __double_as_longlong(v0), b = __double_as_longlong(v1);
    c[0] = uint32_t(a); c[1] = uint32_t(a >> 32); c[2] = uint32_t(b); c[3] = uint32_t(b >> 32);
  }
#pragma unroll
  for (int k = 0; k < W; ++k) st_relaxed64(h + i * W + k, (uint64_t(tag) << 32) | c[k]);
}

template <class T>
struct HaloVal {
  uint64_t w[HaloWord<T>::W];
};
template <class T>
__device__ __forceinline__ void halo_fetch(const uint64_t* h, int64_t i, HaloVal<T>& v) {
#pragma unroll
  for (int k = 0; k < HaloWord<T>::W; ++k) v.w[k] = ld_relaxed64(h + i * HaloWord<T>::W + k);
}
template <class T>
__device__ __forceinline__ bool halo_ready(const HaloVal<T>& v, uint32_t tag) {
  bool ok = true;
#pragma unroll
  for (int k = 0; k < HaloWord<T>::W; ++k) ok = ok && uint32_t(v.w[k] >> 32) == tag;
  return ok;
}
template <class T>
__device__ __forceinline__ void halo_decode(const HaloVal<T>& v, T& v0, T& v1) {
  if constexpr (sizeof(T) == 4) {
    v0 = __uint_as_float(uint32_t(v.w[0]));
    v1 = __uint_as_float(uint32_t(v.w[1]));
  } else {
    v0 = __longlong_as_double(int64_t(uint32_t(v.w[0]) | (uint64_t(uint32_t(v.w[1])) << 32)));
    v1 = __longlong_as_double(int64_t(uint32_t(v.w[2]) | (uint64_t(uint32_t(v.w[3])) << 32)));
  }
}
// bounded re-read until the word carries the current tag
template <class T>
__device__ __forceinline__ bool halo_wait(const uint64_t* h, int64_t i, uint32_t tag, HaloVal<T>& v, int64_t limit,
                                          const int* err) {
  int64_t it = 0;
  while (!halo_ready<T>(v, tag)) {
    if (++it > limit) return false;
    if ((it & 255) == 0 && *(volatile const int*)err) return false;
    halo_fetch<T>(h, i, v);
  }
  return true;
}

// step 6 of Algorithm 1 as a stencil sweep: w_i = y_i - sum_j S_ij z_j (fully parallel)
template <class T>
__global__ void k_ff_residual(int nx, int ny, int nz, const T* __restrict__ S28, const T* __restrict__ y,
                              const T* __restrict__ zs, const T* __restrict__ zp, T* __restrict__ w) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  int64_t nc = int64_t(nx) * ny * nz;
  if (i >= nc) return;
  int x = int(i % nx), yy = int((i / nx) % ny), zz = int(i / (int64_t(nx) * ny));
  const int64_t nxy = int64_t(nx) * ny;
  const int64_t nb[7] = {zz > 0 ? i - nxy : i, yy > 0 ? i - nx : i, x > 0 ? i - 1 : i, i,
                         x + 1 < nx ? i + 1 : i, yy + 1 < ny ? i + nx : i, zz + 1 < nz ? i + nxy : i};
  const T* S = S28 + i * 28;
  T w0 = y[2 * i], w1 = y[2 * i + 1];
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    T a = zs[nb[q]], b = zp[nb[q]];
    w0 -= S[q * 4] * a + S[q * 4 + 1] * b;
    w1 -= S[q * 4 + 2] * a + S[q * 4 + 3] * b;
  }
  w[2 * i] = w0;
  w[2 * i + 1] = w1;
}

// §5.3 option 1, block Gauss-Seidel on the interleaved S_ff^(FS): one colour of one sweep.  Thread p owns
// colour slot p (gs_index); the colour's cells share no face, so each is updated from the other colour's
// newest values: dz_i = inv(S_ii) (w_i - sum_j S_ij dz_j) over the face neighbours j, in slot order
// (z-1, y-1, x-1, x+1, y+1, z+1); neighbours outside the grid are skipped (their stored blocks are zero, and
// dz is not read there: the cell's own dz may still hold a previous apply's value).  ZERO: the first colour
// of the first sweep (every dz_j is still 0).  LAST: the last sweep also writes z_f + dz_f (FP64) for its
// cells to zout.
template <class T, bool ZERO, bool LAST>
__global__ void k_gs_colour(int nx, int ny, int nz, int col, int64_t ncp, const T* __restrict__ rec,
                            const T* __restrict__ w, T* __restrict__ dz, const T* __restrict__ zs,
                            const T* __restrict__ zp, double* __restrict__ zout) {
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= ncp) return;
  const int hx = gs_hx(nx);
  const int m = int(p % hx);
  const int64_t row = p / hx;
  const int y = int(row % ny), z = int(row / ny);
  const int x = 2 * m + ((col + y + z) & 1);
  if (x >= nx) return;
  const int64_t nxy = int64_t(nx) * ny;
  const int64_t i = x + nx * int64_t(y) + nxy * z;
  const T* R = rec + ((int64_t(col) * ((ncp + 31) / 32) + (p >> 5)) * 28) * 32 + (p & 31);
  T a0 = w[2 * i], a1 = w[2 * i + 1];
  if (!ZERO) {
    const int64_t nb[6] = {i - nxy, i - nx, i - 1, i + 1, i + nx, i + nxy};
    const bool in[6] = {z > 0, y > 0, x > 0, x + 1 < nx, y + 1 < ny, z + 1 < nz};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const T d0 = in[q] ? dz[2 * nb[q]] : T(0), d1 = in[q] ? dz[2 * nb[q] + 1] : T(0);
      a0 -= R[(4 * q) * 32] * d0 + R[(4 * q + 1) * 32] * d1;
      a1 -= R[(4 * q + 2) * 32] * d0 + R[(4 * q + 3) * 32] * d1;
    }
  }
  const T e0 = R[24 * 32] * a0 + R[25 * 32] * a1;
  const T e1 = R[26 * 32] * a0 + R[27 * 32] * a1;
  dz[2 * i] = e0;
  dz[2 * i + 1] = e1;
  if (LAST) {
    zout[2 * i] = double(zs[i] + e0);
    zout[2 * i + 1] = double(zp[i] + e1);
  }
}

// per-cell data of one sweep step: forward (w_i, lower blocks, inv(U_ii)),
// backward (t_i, upper blocks, inv(U_ii), z_i)
template <class T>
struct Cell {
  T a0, a1;
  T S[3][4];
  T D[4];
  T z0, z1;
};

// Per-cell records of a sweep, packed at setup and per apply in the order the CTAs consume them
// (sweep_rec): [3 blocks of the sweep's side (12) | inv(U_ii) (4) | right-hand side pair (2) | z pair (2)].
// Forward records hold the lower blocks (z-1, y-1, x-1) and w; backward records the upper blocks
// (x+1, y+1, z+1), t (written by the forward sweep) and z_s, z_p.
template <class T>
__host__ __device__ constexpr size_t win_bytes() {  // two window buffers for the CTA
  return size_t(2) * kTY * kTZ * win_cells<T>() * kRec * sizeof(T);
}

__device__ __forceinline__ void mbar_init(uint64_t* m, unsigned count) {
  unsigned a = unsigned(__cvta_generic_to_shared(m));
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* m, unsigned bytes) {
  unsigned a = unsigned(__cvta_generic_to_shared(m));
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* m, unsigned parity) {
  unsigned a = unsigned(__cvta_generic_to_shared(m));
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
// bulk copy of bytes (multiple of 16, both addresses 16-byte aligned) completing on mbarrier m
__device__ __forceinline__ void bulk_copy(void* sdst, const void* gsrc, unsigned bytes, uint64_t* m) {
  unsigned d = unsigned(__cvta_generic_to_shared(sdst));
  unsigned b = unsigned(__cvta_generic_to_shared(m));
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d),
               "l"(gsrc), "r"(bytes), "r"(b)
               : "memory");
}

// move one record from shared memory to registers (16-byte vector reads)
template <class T>
__device__ __forceinline__ void read_cell(const T* sv, Cell<T>& c) {
  T v[kRec];
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int k = 0; k < kRec; k += 4) {
      float4 f = *reinterpret_cast<const float4*>(sv + k);
      v[k] = f.x; v[k + 1] = f.y; v[k + 2] = f.z; v[k + 3] = f.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < kRec; k += 2) {
      double2 f = *reinterpret_cast<const double2*>(sv + k);
      v[k] = f.x; v[k + 1] = f.y;
    }
  }
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int e = 0; e < 4; ++e) c.S[r][e] = v[r * 4 + e];
#pragma unroll
  for (int e = 0; e < 4; ++e) c.D[e] = v[12 + e];
  c.a0 = v[16]; c.a1 = v[17]; c.z0 = v[18]; c.z1 = v[19];
}

template <class T>
__device__ __forceinline__ void store2(T* p, T a, T b) {
  if constexpr (sizeof(T) == 4) *reinterpret_cast<float2*>(p) = make_float2(a, b);
  else *reinterpret_cast<double2*>(p) = make_double2(a, b);
}

// step 6 for the pencil sweeps: w into the forward records, z_s and z_p into the backward records
template <class T>
__global__ void k_ff_residual_pack(int nx, int ny, int nz, int steps, const T* __restrict__ S28,
                                   const T* __restrict__ y, const T* __restrict__ zs, const T* __restrict__ zp,
                                   T* __restrict__ pf, T* __restrict__ pb) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  int64_t nc = int64_t(nx) * ny * nz;
  if (i >= nc) return;
  int x = int(i % nx), yy = int((i / nx) % ny), zz = int(i / (int64_t(nx) * ny));
  const int64_t nxy = int64_t(nx) * ny;
  const int64_t nb[7] = {zz > 0 ? i - nxy : i, yy > 0 ? i - nx : i, x > 0 ? i - 1 : i, i,
                         x + 1 < nx ? i + 1 : i, yy + 1 < ny ? i + nx : i, zz + 1 < nz ? i + nxy : i};
  const T* S = S28 + i * 28;
  T w0 = y[2 * i], w1 = y[2 * i + 1];
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    T a = zs[nb[q]], b = zp[nb[q]];
    w0 -= S[q * 4] * a + S[q * 4 + 1] * b;
    w1 -= S[q * 4 + 2] * a + S[q * 4 + 3] * b;
  }
  store2<T>(pf + sweep_rec(true, nx, ny, steps, x, yy, zz) + 16, w0, w1);
  store2<T>(pb + sweep_rec(false, nx, ny, steps, x, yy, zz) + 18, zs[i], zp[i]);
}

// Sync-free wavefront sweep over the packed records (see the block comment above).  A window of
// win_cells steps of a tile is one contiguous range of the records ([tile][step][thread]): thread 0
// moves it with one bulk copy into one of two window buffers, completing on that buffer's mbarrier
// (one arrival plus the copied bytes).  FWD writes t into the backward records; the backward sweep
// writes z_f.
template <class T, bool FWD>
__global__ void __launch_bounds__(kTY * kTZ) k_ilu_pencil(int nx, int ny, int nz, int steps, const T* __restrict__ rec,
                                                         T* __restrict__ rec_bwd, double* __restrict__ zout,
                                                         uint64_t* halo, int* err, uint32_t tag, int64_t limit,
                                                         int stall, int local) {
  constexpr int W = win_cells<T>();
  __shared__ __align__(16) T buf[2][kTZ][kTY][2];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ int abort_flag;
  extern __shared__ __align__(16) unsigned char win_raw[];
  T* win = reinterpret_cast<T*>(win_raw);
  const int nby = (ny + kTY - 1) / kTY;
  const int BY = blockIdx.x % nby, BZ = blockIdx.x / nby;
  // test hook: the CTA numbered stall - 1 never runs, so its halo words never get the current tag
  if (stall > 0 && int(blockIdx.x) == stall - 1) return;
  const int ly = threadIdx.x % kTY, lz = threadIdx.x / kTY;
  const int yy = BY * kTY + ly, zz = BZ * kTZ + lz;
  const bool valid = yy < ny && zz < nz;
  const int last = nx + kTY + kTZ - 3;
  const int64_t nxy = int64_t(nx) * ny;
  const int ry = FWD ? ly : kTY - 1 - ly, rz = FWD ? lz : kTZ - 1 - lz;
  // processor-local scope: a predecessor in another tile is not coupled, and no CTA waits on another
  const bool hy = valid && (FWD ? yy > 0 : yy + 1 < ny) && !(local && ry == 0),
             hz = valid && (FWD ? zz > 0 : zz + 1 < nz) && !(local && rz == 0);
  const bool gy = hy && ry == 0, gz = hz && rz == 0;  // predecessor lives in another CTA
  // this pencil feeds another CTA along y (z) when it sits on the far boundary
  const bool py = !local && valid && ry == kTY - 1 && (FWD ? yy + 1 < ny : yy > 0);
  const bool pz = !local && valid && rz == kTZ - 1 && (FWD ? zz + 1 < nz : zz > 0);
  const int64_t jy = FWD ? -int64_t(nx) : int64_t(nx), jz = FWD ? -nxy : nxy;
  const int64_t pbase = valid ? int64_t(nx) * (yy + int64_t(ny) * zz) : 0;
  const int off = ry + rz;  // step s handles pencil position xs = s - off
  // window k holds steps [k W, k W + W) of the whole tile: W * kTY * kTZ records, step-major
  constexpr unsigned kWinVals = unsigned(W) * kTY * kTZ * kRec;
  const T* trec = rec + size_t(blockIdx.x) * steps * (kTY * kTZ) * kRec;
  auto request = [&](int k) {  // thread 0 only; k * W < steps
    const int b = k & 1;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_tx(&mbar[b], kWinVals * unsigned(sizeof(T)));
    bulk_copy(win + size_t(b) * kWinVals, trec + size_t(k) * kWinVals, kWinVals * unsigned(sizeof(T)), &mbar[b]);
  };
  auto wait_window = [&](int k) -> bool {
    int64_t it = 0;
    while (!mbar_try_wait(&mbar[k & 1], unsigned((k >> 1) & 1))) {
      if (++it > limit) return false;
    }
    return true;
  };
  if (threadIdx.x == 0) {
    abort_flag = 0;
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    request(0);
    if (W <= last) request(1);
  }
  // Per-step state kept incrementally: xs = step - off is the pencil position and gi the cell index
  // (one step moves gi by +1 forward, -1 backward).  In the loop below the slot loop is unrolled over
  // two windows, so a step's window buffer and record position are compile-time constants.
  constexpr int64_t kStep = FWD ? 1 : -1;
  const unsigned unx = unsigned(nx);
  auto on = [&](int xs) { return valid && unsigned(xs) < unx; };
  const T* tbase = win + size_t(threadIdx.x) * kRec;
  auto rec_at = [&](int q2) -> const T* {  // record of the step whose unrolled index is q2 (mod 2W)
    const int b = (q2 / W) & 1, pos = q2 % W;
    return tbase + (size_t(b) * W + pos) * (kTY * kTZ) * kRec;
  };
  // forward sweep: t of the cell at pencil position xs goes to its backward record, backward step
  // nx - 1 - xs + (kTY - 1 - ly) + (kTZ - 1 - lz) of the same tile and thread
  T* tout = FWD ? rec_bwd + (size_t(blockIdx.x) * steps * (kTY * kTZ) + threadIdx.x) * kRec + 16 : nullptr;
  const int boff = (kTY - 1 - ly) + (kTZ - 1 - lz) + nx - 1;
  HaloVal<T> hyr[2], hzr[2];
  int xs = -off;                        // step 0
  int64_t gi = pbase + (FWD ? xs : nx - 1 - xs);
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (gy && on(xs + q)) halo_fetch<T>(halo, gi + q * kStep + jy, hyr[q]);
    if (gz && on(xs + q)) halo_fetch<T>(halo, gi + q * kStep + jz, hzr[q]);
  }
  Cell<T> cs[2];
  T p0[2], p1[2];  // x-neighbour part of step s: FWD w - S_x-1 t_x-1, BWD S_x+1 dz_x+1
  bool ok0 = wait_window(0);
  if (!ok0) { atomicExch(err, 1); abort_flag = 1; }
  if (on(xs)) read_cell<T>(rec_at(0), cs[0]);
  p0[0] = (FWD && on(xs)) ? cs[0].a0 : T(0);
  p1[0] = (FWD && on(xs)) ? cs[0].a1 : T(0);
  for (int s0 = 0; s0 <= last; s0 += 2 * W) {
#pragma unroll
    for (int q = 0; q < 2 * W; ++q) {
      const int step = s0 + q;
      if (step > last) break;  // the same in every thread of the CTA
      const int cur = q & 1, nxt = (q + 1) & 1;
      const Cell<T>& c0 = cs[cur];
      const bool act = on(xs);
      const int64_t i0 = gi;
      T r0 = T(0), r1 = T(0);
      T ny0 = T(0), ny1 = T(0), nz0 = T(0), nz1 = T(0);
      if (act) {
        bool ok = true;
        if (gy) {
          ok = ok && halo_wait<T>(halo, i0 + jy, tag, hyr[cur], limit, err);
          halo_decode<T>(hyr[cur], ny0, ny1);
        } else if (hy) {
          const T* qq = buf[(q + 1) & 1][lz][FWD ? ly - 1 : ly + 1];
          ny0 = qq[0]; ny1 = qq[1];
        }
        if (gz) {
          ok = ok && halo_wait<T>(halo, i0 + jz, tag, hzr[cur], limit, err);
          halo_decode<T>(hzr[cur], nz0, nz1);
        } else if (hz) {
          const T* qq = buf[(q + 1) & 1][FWD ? lz - 1 : lz + 1][ly];
          nz0 = qq[0]; nz1 = qq[1];
        }
        if (!ok) { abort_flag = 1; atomicExch(err, 1); }
      }
      // halo words of step + 2 into the slots just read: issued before this step's update, the loads
      // have the rest of this step and all of the next to arrive
      if (gy && on(xs + 2)) halo_fetch<T>(halo, gi + 2 * kStep + jy, hyr[cur]);
      if (gz && on(xs + 2)) halo_fetch<T>(halo, gi + 2 * kStep + jz, hzr[cur]);
      if (act) {
        if (FWD) {
          // u_i = w_i - sum_{k<i} S_ik t_k (blocks z-1, y-1, x-1) ; t_i = inv(U_ii) u_i
          T u0 = p0[cur] - (c0.S[0][0] * nz0 + c0.S[0][1] * nz1) - (c0.S[1][0] * ny0 + c0.S[1][1] * ny1);
          T u1 = p1[cur] - (c0.S[0][2] * nz0 + c0.S[0][3] * nz1) - (c0.S[1][2] * ny0 + c0.S[1][3] * ny1);
          r0 = c0.D[0] * u0 + c0.D[1] * u1;
          r1 = c0.D[2] * u0 + c0.D[3] * u1;
          store2<T>(tout + size_t(boff - xs) * (kTY * kTZ) * kRec, r0, r1);
        } else {
          // dz_i = t_i - inv(U_ii) sum_{j>i} S_ij dz_j (blocks x+1, y+1, z+1) ; z_f = z + dz
          T s0v = p0[cur] + (c0.S[1][0] * ny0 + c0.S[1][1] * ny1) + (c0.S[2][0] * nz0 + c0.S[2][1] * nz1);
          T s1v = p1[cur] + (c0.S[1][2] * ny0 + c0.S[1][3] * ny1) + (c0.S[2][2] * nz0 + c0.S[2][3] * nz1);
          r0 = c0.a0 - (c0.D[0] * s0v + c0.D[1] * s1v);
          r1 = c0.a1 - (c0.D[2] * s0v + c0.D[3] * s1v);
          // z_f may start at an odd multiple of 8 bytes (it follows the 3 * nodes displacement entries)
          zout[2 * i0] = double(c0.z0 + r0);
          zout[2 * i0 + 1] = double(c0.z1 + r1);
        }
        if (py || pz) halo_put<T>(halo, i0, r0, r1, tag);
        store2<T>(buf[q & 1][lz][ly], r0, r1);
      }
      // step + 1's record (its window is waited for when step + 1 starts a window)
      if ((q + 1) % W == 0 && step + 1 <= last) {
        if (!wait_window((step + 1) / W)) { abort_flag = 1; atomicExch(err, 1); }
      }
      const bool actn = on(xs + 1);
      if (actn) read_cell<T>(rec_at((q + 1) % (2 * W)), cs[nxt]);
      {
        // x-neighbour term of step + 1: this thread's result of step when both lie on the pencil
        const T x0 = act ? r0 : T(0), x1 = act ? r1 : T(0);
        const Cell<T>& cn = cs[nxt];
        if (FWD) {
          p0[nxt] = actn ? cn.a0 - (cn.S[2][0] * x0 + cn.S[2][1] * x1) : T(0);
          p1[nxt] = actn ? cn.a1 - (cn.S[2][2] * x0 + cn.S[2][3] * x1) : T(0);
        } else {
          p0[nxt] = actn ? cn.S[0][0] * x0 + cn.S[0][1] * x1 : T(0);
          p1[nxt] = actn ? cn.S[0][2] * x0 + cn.S[0][3] * x1 : T(0);
        }
      }
      ++xs;
      gi += kStep;
      __syncthreads();
      if ((q + 1) % W == 0) {
        // every thread has read its last record of window step / W: refill that buffer two windows on
        if (abort_flag) {
          // the next window may still be landing in shared memory: wait for it (bounded) before leaving
          if (step + 1 <= last) wait_window((step + 1) / W);
          return;
        }
        const int k = step / W + 2;
        if (k * W <= last && threadIdx.x == 0) request(k);
      }
    }
  }
}

}  // namespace

template <class T>
ps_status flow_alloc_work(Arena& ar, const FlowStage& F, FlowWork<T>& W) {
  int64_t nc = F.nc;
  PS_TRY(ar.alloc(&W.vf, 2 * nc)); PS_TRY(ar.alloc(&W.y, 2 * nc)); PS_TRY(ar.alloc(&W.zs, nc));
  PS_TRY(ar.alloc(&W.wp, nc)); PS_TRY(ar.alloc(&W.zp, nc)); PS_TRY(ar.alloc(&W.t, 2 * nc));
  PS_TRY(ar.alloc(&W.dz, 2 * nc));
  PS_TRY(ar.alloc(&W.wf, 2 * nc));
  return PS_OK;
}

template <class T>
void alg1_steps_2_4(const FlowStage& F, const FlowWork<T>& W, const T* zu, cudaStream_t st) {
  FlowView<T> V = fview<T>(F);
  const T* fu_st = sizeof(T) == 4 ? reinterpret_cast<const T*>(F.fu_st_f) : reinterpret_cast<const T*>(F.fu_st_d);
  const T* aps_st = sizeof(T) == 4 ? reinterpret_cast<const T*>(F.aps_st_f) : reinterpret_cast<const T*>(F.aps_st_d);
  if (fu_st) {
    PS_TICK(); k_step23_st<T><<<grid_for(F.nc, 256), 256, 0, st>>>(F.nx, F.ny, F.nz, fu_st, W.vf, zu, V.dss, W.y, W.zs);
  } else {
    PS_TICK(); k_step23<T><<<grid_for(F.nc * 8, 256), 256, 0, st>>>(F.nc, F.fu_rp, F.fu_ci, V.fu, W.vf, zu, V.dss, W.y,
                                                                  W.zs);
  }
  if (aps_st) {
    PS_TICK(); k_step4_st<T><<<grid_for(F.nc, 256), 256, 0, st>>>(F.nx, F.ny, F.nz, aps_st, W.y, W.zs, W.wp);
  } else {
    PS_TICK(); k_step4<T><<<grid_for(F.nc * 8, 256), 256, 0, st>>>(F.nc, F.rp, F.ci, V.aps, W.y, W.zs, W.wp);
  }
}

template <class T>
bool ilu_pencil(const FlowStage& F, const FlowWork<T>& W, double* zout, cudaStream_t st) {
  FlowView<T> V = fview<T>(F);
  T* pf = sizeof(T) == 4 ? reinterpret_cast<T*>(F.pk_fwd_f) : reinterpret_cast<T*>(F.pk_fwd_d);
  T* pb = sizeof(T) == 4 ? reinterpret_cast<T*>(F.pk_bwd_f) : reinterpret_cast<T*>(F.pk_bwd_d);
  if (!V.s28 || !F.halo || !pf || !pb) return false;
  int nby = (F.ny + kTY - 1) / kTY, nbz = (F.nz + kTZ - 1) / kTZ;
  unsigned grid = unsigned(nby * nbz);
  FlowStage& Fm = const_cast<FlowStage&>(F);
  if (F.pk_steps != sweep_steps(F.nx, win_cells<T>())) return false;
  PS_TICK(); k_ff_residual_pack<T><<<grid_for(F.nc, 256), 256, 0, st>>>(F.nx, F.ny, F.nz, F.pk_steps, V.s28, W.y, W.zs,
                                                                      W.zp, pf, pb);
  for (int dir = 0; dir < 2; ++dir) {
    uint32_t tag = uint32_t(++Fm.ilu_epoch);
    if (tag == 0) tag = uint32_t(++Fm.ilu_epoch);  // 0 marks never-written halo words
    int nx = F.nx, ny = F.ny, nz = F.nz;
    const T* rec = dir == 0 ? pf : pb;
    T* rec_bwd = pb;
    uint64_t* halo = F.halo;
    int* err = F.ilu_err;
    int64_t lim = F.spin_limit;
    int stall = F.test_stall;
    int steps = F.pk_steps;
    int local = F.ilu_local;
    void* args[] = {&nx, &ny, &nz, &steps, &rec, &rec_bwd, &zout, &halo, &err, &tag, &lim, &stall, &local};
    const void* fn = dir == 0 ? (const void*)k_ilu_pencil<T, true> : (const void*)k_ilu_pencil<T, false>;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(win_bytes<T>()));
    cudaError_t e = cudaLaunchCooperativeKernel(fn, grid, kTY * kTZ, args, win_bytes<T>(), st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    PS_TICK();
  }
  return true;
}

// steps 6-8 with the block Gauss-Seidel local stage: w_f = y_f - S_ff^(FS) z_f, then gs_sweeps sweeps of
// two colours from dz = 0, the last one adding z_f into zout
template <class T>
void gs_local(const FlowStage& F, const FlowWork<T>& W, double* zout, cudaStream_t st) {
  FlowView<T> V = fview<T>(F);
  const T* rec = sizeof(T) == 4 ? reinterpret_cast<const T*>(F.gs_rec_f) : reinterpret_cast<const T*>(F.gs_rec_d);
  PS_TICK(); k_ff_residual<T><<<grid_for(F.nc, 256), 256, 0, st>>>(F.nx, F.ny, F.nz, V.s28, W.y, W.zs, W.zp, W.wf);
  const unsigned g = grid_for(F.gs_ncp, 256);
  for (int sw = 0; sw < F.gs_sweeps; ++sw)
    for (int col = 0; col < 2; ++col) {
      const bool last = sw == F.gs_sweeps - 1;
      PS_TICK();
      if (sw == 0 && col == 0) {
        if (last) k_gs_colour<T, true, true><<<g, 256, 0, st>>>(F.nx, F.ny, F.nz, col, F.gs_ncp, rec, W.wf, W.dz, W.zs, W.zp, zout);
        else k_gs_colour<T, true, false><<<g, 256, 0, st>>>(F.nx, F.ny, F.nz, col, F.gs_ncp, rec, W.wf, W.dz, W.zs, W.zp, zout);
      } else if (last) {
        k_gs_colour<T, false, true><<<g, 256, 0, st>>>(F.nx, F.ny, F.nz, col, F.gs_ncp, rec, W.wf, W.dz, W.zs, W.zp, zout);
      } else {
        k_gs_colour<T, false, false><<<g, 256, 0, st>>>(F.nx, F.ny, F.nz, col, F.gs_ncp, rec, W.wf, W.dz, W.zs, W.zp, zout);
      }
    }
}

template <class T>
void alg1_steps_6_8(const FlowStage& F, const FlowWork<T>& W, double* zout, int ilu_mode, cudaStream_t st) {
  if (F.local == PS_LOCAL_HBGS) {
    gs_local<T>(F, W, zout, st);
    return;
  }
  if (ilu_mode == PS_ILU_PENCIL && F.halo && ilu_pencil<T>(F, W, zout, st)) return;
  FlowView<T> V = fview<T>(F);
  for (int l = 0; l < F.nlev; ++l) {
    int32_t m = F.lev_off[l + 1] - F.lev_off[l];
    PS_TICK(); k_ilu_fwd<T><<<grid_for(m, 128), 128, 0, st>>>(F.lev_cells + F.lev_off[l], m, F.rp, F.ci, F.diagpos, V.sff,
                                                   V.dinv, W.y, W.zs, W.zp, W.t, F.nx, F.ny, F.ilu_local);
  }
  for (int l = F.nlev - 1; l >= 0; --l) {
    int32_t m = F.lev_off[l + 1] - F.lev_off[l];
    PS_TICK(); k_ilu_bwd<T><<<grid_for(m, 128), 128, 0, st>>>(F.lev_cells + F.lev_off[l], m, F.rp, F.ci, F.diagpos, V.sff,
                                                   V.dinv, W.t, W.zs, W.zp, W.dz, zout, F.nx, F.ny, F.ilu_local);
  }
}

template ps_status flow_alloc_work<float>(Arena&, const FlowStage&, FlowWork<float>&);
template ps_status flow_alloc_work<double>(Arena&, const FlowStage&, FlowWork<double>&);
template void alg1_steps_2_4<float>(const FlowStage&, const FlowWork<float>&, const float*, cudaStream_t);
template void alg1_steps_2_4<double>(const FlowStage&, const FlowWork<double>&, const double*, cudaStream_t);
template void alg1_steps_6_8<float>(const FlowStage&, const FlowWork<float>&, double*, int, cudaStream_t);
template void alg1_steps_6_8<double>(const FlowStage&, const FlowWork<double>&, double*, int, cudaStream_t);

}  // namespace ps_internal
