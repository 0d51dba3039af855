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
template <class T>
__global__ void k_ilu_fwd(const int32_t* __restrict__ cells, int32_t m, const int32_t* __restrict__ rp,
                          const int32_t* __restrict__ ci, const int32_t* __restrict__ diagpos,
                          const T* __restrict__ sff, const T* __restrict__ dinv, const T* __restrict__ y,
                          const T* __restrict__ zs, const T* __restrict__ zp, T* __restrict__ t) {
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
    if (q < qd) {
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
                          double* __restrict__ zout) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m) return;
  int32_t i = cells[idx];
  int32_t qd = diagpos[i];
  T a0 = T(0), a1 = T(0);
  for (int32_t q = qd + 1; q < rp[i + 1]; ++q) {
    int32_t j = ci[q];
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
// shared array).  Everything that does not depend on the wavefront is loaded
// one step ahead.  Boundary pencils take their predecessors from global memory:
// before prefetching the value for step s + 1 each polls its producer CTA's
// progress with an acquire load (bounded; on timeout it raises *err); each CTA
// publishes its progress with a release store after the step's barrier.
// ---------------------------------------------------------------------------
constexpr int kTY = 16, kTZ = 8;
constexpr int64_t kEpochStride = 1 << 20;  // > steps per sweep

__device__ __forceinline__ int64_t ld_acquire(const int64_t* p) {
  int64_t v;
  asm volatile("ld.acquire.gpu.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int64_t* p, int64_t v) {
  asm volatile("st.release.gpu.global.s64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// bounded wait until *flag >= need; `seen` caches the last observed value
__device__ __forceinline__ bool wait_progress(const int64_t* flag, int64_t need, int64_t& seen, int64_t limit,
                                              const int* err) {
  int64_t it = 0;
  while (seen < need) {
    seen = ld_acquire(flag);
    if (seen >= need) break;
    if (++it > limit) return false;
    if ((it & 255) == 0 && *(volatile const int*)err) return false;
  }
  return true;
}

// per-cell data of one sweep step
template <class T, bool FWD>
struct StepData {
  T S[7][4];  // forward: all 7 blocks; backward: blocks 4..6 (upper) used
  T D[4];
  T a0, a1;   // forward: y_i ; backward: t_i
  T zs[7], zp[7];  // forward: neighbour z (s, p); backward: own z in zs[3], zp[3]
};

template <class T, bool FWD>
__device__ __forceinline__ void load_step(StepData<T, FWD>& d, int64_t i, int x, int yy, int zz, int nx, int ny,
                                          int nz, const T* __restrict__ S28, const T* __restrict__ dinv,
                                          const T* __restrict__ y, const T* __restrict__ t,
                                          const T* __restrict__ zs, const T* __restrict__ zp) {
  const int64_t nxy = int64_t(nx) * ny;
  const T* Si = S28 + i * 28;
#pragma unroll
  for (int q = 0; q < 7; ++q)
#pragma unroll
    for (int e = 0; e < 4; ++e) d.S[q][e] = (FWD || q >= 4) ? Si[q * 4 + e] : T(0);
#pragma unroll
  for (int e = 0; e < 4; ++e) d.D[e] = dinv[i * 4 + e];
  if (FWD) {
    d.a0 = y[2 * i]; d.a1 = y[2 * i + 1];
    const int64_t nb[7] = {zz > 0 ? i - nxy : i, yy > 0 ? i - nx : i, x > 0 ? i - 1 : i, i,
                           x + 1 < nx ? i + 1 : i, yy + 1 < ny ? i + nx : i, zz + 1 < nz ? i + nxy : i};
#pragma unroll
    for (int q = 0; q < 7; ++q) { d.zs[q] = zs[nb[q]]; d.zp[q] = zp[nb[q]]; }
  } else {
    d.a0 = t[2 * i]; d.a1 = t[2 * i + 1];
    d.zs[3] = zs[i]; d.zp[3] = zp[i];
  }
}

template <class T, bool FWD>
__global__ void __launch_bounds__(kTY * kTZ) k_ilu_pencil(
    int nx, int ny, int nz, const T* __restrict__ S28, const T* __restrict__ dinv, const T* __restrict__ y,
    const T* __restrict__ zs, const T* __restrict__ zp, T* t, T* dz, double* __restrict__ zout, int64_t* progress,
    int* err, int64_t epoch, int64_t limit, int stall) {
  __shared__ T buf[2][kTZ][kTY][2];
  __shared__ int abort_flag;
  const int nby = (ny + kTY - 1) / kTY;
  const int BY = blockIdx.x % nby, BZ = blockIdx.x / nby;
  // test hook: the CTA numbered stall - 1 never runs nor publishes progress
  if (stall > 0 && int(blockIdx.x) == stall - 1) return;
  const int ly = threadIdx.x % kTY, lz = threadIdx.x / kTY;
  const int yy = BY * kTY + ly, zz = BZ * kTZ + lz;
  const bool valid = yy < ny && zz < nz;
  const int64_t nxy = int64_t(nx) * ny;
  const int last = nx + kTY + kTZ - 3;
  const int64_t base = epoch * kEpochStride;
  const int ry = FWD ? ly : kTY - 1 - ly, rz = FWD ? lz : kTZ - 1 - lz;
  // boundary roles: take the y (z) predecessor from the producer CTA
  const bool hy = valid && (FWD ? yy > 0 : yy + 1 < ny), hz = valid && (FWD ? zz > 0 : zz + 1 < nz);
  const bool gy = hy && ry == 0, gz = hz && rz == 0;
  const int64_t* fy = progress + (int64_t(BZ) * nby + (FWD ? BY - 1 : BY + 1));
  const int64_t* fz = progress + (int64_t(FWD ? BZ - 1 : BZ + 1) * nby + BY);
  const T* src = FWD ? t : dz;
  const int64_t jy = FWD ? -int64_t(nx) : int64_t(nx), jz = FWD ? -nxy : nxy;
  int64_t seen_y = 0, seen_z = 0;
  if (threadIdx.x == 0) abort_flag = 0;
  __syncthreads();
  auto cell_at = [&](int s, int* xo) -> int64_t {
    int xs = s - ry - rz;
    if (!valid || xs < 0 || xs >= nx) return -1;
    int x = FWD ? xs : nx - 1 - xs;
    *xo = x;
    return x + int64_t(nx) * (yy + int64_t(ny) * zz);
  };
  // prefetch for step 0
  StepData<T, FWD> cur;
  int xc = 0;
  int64_t ic = cell_at(0, &xc);
  if (ic >= 0) load_step<T, FWD>(cur, ic, xc, yy, zz, nx, ny, nz, S28, dinv, y, t, zs, zp);
  T by0 = T(0), by1 = T(0), bz0 = T(0), bz1 = T(0);  // boundary predecessors for the current step
  bool ok = true;
  if (ic >= 0 && gy) {
    ok = ok && wait_progress(fy, base + min(0 + kTY - 1, last), seen_y, limit, err);
    if (ok) { by0 = __ldcg(src + 2 * (ic + jy)); by1 = __ldcg(src + 2 * (ic + jy) + 1); }
  }
  if (ic >= 0 && gz) {
    ok = ok && wait_progress(fz, base + min(0 + kTZ - 1, last), seen_z, limit, err);
    if (ok) { bz0 = __ldcg(src + 2 * (ic + jz)); bz1 = __ldcg(src + 2 * (ic + jz) + 1); }
  }
  if (!ok) { abort_flag = 1; atomicExch(err, 1); }
  T prev0 = T(0), prev1 = T(0);
  for (int step = 0; step <= last; ++step) {
    // compute the current cell
    if (ic >= 0) {
      T ny0 = by0, ny1 = by1, nz0 = bz0, nz1 = bz1;
      if (hy && !gy) {
        const T* b = buf[(step - 1) & 1][lz][FWD ? ly - 1 : ly + 1];
        ny0 = b[0]; ny1 = b[1];
      }
      if (hz && !gz) {
        const T* b = buf[(step - 1) & 1][FWD ? lz - 1 : lz + 1][ly];
        nz0 = b[0]; nz1 = b[1];
      }
      T r0, r1;
      if (FWD) {
        // w_i = y_i - sum_j S_ij z_j ; u_i = w_i - sum_{k<i} S_ik t_k ; t_i = inv(U_ii) u_i
        T w0 = cur.a0, w1 = cur.a1;
        const T l0[3] = {nz0, ny0, xc > 0 ? prev0 : T(0)}, l1[3] = {nz1, ny1, xc > 0 ? prev1 : T(0)};
#pragma unroll
        for (int q = 0; q < 7; ++q) {
          T a = cur.zs[q] + (q < 3 ? l0[q] : T(0)), b = cur.zp[q] + (q < 3 ? l1[q] : T(0));
          w0 -= cur.S[q][0] * a + cur.S[q][1] * b;
          w1 -= cur.S[q][2] * a + cur.S[q][3] * b;
        }
        r0 = cur.D[0] * w0 + cur.D[1] * w1;
        r1 = cur.D[2] * w0 + cur.D[3] * w1;
        t[2 * ic] = r0;
        t[2 * ic + 1] = r1;
      } else {
        // dz_i = t_i - inv(U_ii) sum_{j>i} S_ij dz_j ; z_f = (z_s, z_p) + dz
        const T u0[3] = {xc + 1 < nx ? prev0 : T(0), ny0, nz0}, u1[3] = {xc + 1 < nx ? prev1 : T(0), ny1, nz1};
        T a0 = T(0), a1 = T(0);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          a0 += cur.S[4 + q][0] * u0[q] + cur.S[4 + q][1] * u1[q];
          a1 += cur.S[4 + q][2] * u0[q] + cur.S[4 + q][3] * u1[q];
        }
        r0 = cur.a0 - (cur.D[0] * a0 + cur.D[1] * a1);
        r1 = cur.a1 - (cur.D[2] * a0 + cur.D[3] * a1);
        dz[2 * ic] = r0;
        dz[2 * ic + 1] = r1;
        zout[2 * ic] = double(cur.zs[3] + r0);
        zout[2 * ic + 1] = double(cur.zp[3] + r1);
      }
      prev0 = r0;
      prev1 = r1;
      buf[step & 1][lz][ly][0] = r0;
      buf[step & 1][lz][ly][1] = r1;
    }
    // prefetch the next step: own cell data, then boundary predecessors once published
    int xn = 0;
    int64_t in = step < last ? cell_at(step + 1, &xn) : -1;
    if (in >= 0) {
      load_step<T, FWD>(cur, in, xn, yy, zz, nx, ny, nz, S28, dinv, y, t, zs, zp);
      bool okn = true;
      if (gy) {
        okn = okn && wait_progress(fy, base + min(step + kTY, last), seen_y, limit, err);
        if (okn) { by0 = __ldcg(src + 2 * (in + jy)); by1 = __ldcg(src + 2 * (in + jy) + 1); }
      }
      if (gz) {
        okn = okn && wait_progress(fz, base + min(step + kTZ, last), seen_z, limit, err);
        if (okn) { bz0 = __ldcg(src + 2 * (in + jz)); bz1 = __ldcg(src + 2 * (in + jz) + 1); }
      }
      if (!okn) { abort_flag = 1; atomicExch(err, 1); }
    }
    ic = in;
    xc = xn;
    __syncthreads();
    if (abort_flag) return;
    if (threadIdx.x == 0) st_release(progress + blockIdx.x, base + step);
  }
}

}  // namespace

template <class T>
ps_status flow_alloc_work(Arena& ar, const FlowStage& F, FlowWork<T>& W) {
  int64_t nc = F.nc;
  PS_TRY(ar.alloc(&W.vf, 2 * nc)); PS_TRY(ar.alloc(&W.y, 2 * nc)); PS_TRY(ar.alloc(&W.zs, nc));
  PS_TRY(ar.alloc(&W.wp, nc)); PS_TRY(ar.alloc(&W.zp, nc)); PS_TRY(ar.alloc(&W.t, 2 * nc));
  PS_TRY(ar.alloc(&W.dz, 2 * nc));
  return PS_OK;
}

template <class T>
void alg1_steps_2_4(const FlowStage& F, const FlowWork<T>& W, const T* zu, cudaStream_t st) {
  FlowView<T> V = fview<T>(F);
  PS_TICK(); k_step23<T><<<grid_for(F.nc * 8, 256), 256, 0, st>>>(F.nc, F.fu_rp, F.fu_ci, V.fu, W.vf, zu, V.dss, W.y, W.zs);
  PS_TICK(); k_step4<T><<<grid_for(F.nc * 8, 256), 256, 0, st>>>(F.nc, F.rp, F.ci, V.aps, W.y, W.zs, W.wp);
}

template <class T>
bool ilu_pencil(const FlowStage& F, const FlowWork<T>& W, double* zout, cudaStream_t st) {
  FlowView<T> V = fview<T>(F);
  if (!V.s28) return false;
  int nby = (F.ny + kTY - 1) / kTY, nbz = (F.nz + kTZ - 1) / kTZ;
  unsigned grid = unsigned(nby * nbz);
  FlowStage& Fm = const_cast<FlowStage&>(F);
  for (int dir = 0; dir < 2; ++dir) {
    int64_t epoch = ++Fm.ilu_epoch;
    int nx = F.nx, ny = F.ny, nz = F.nz;
    const T *s28 = V.s28, *dinv = V.dinv, *y = W.y, *zs = W.zs, *zp = W.zp;
    T *t = W.t, *dz = W.dz;
    int64_t* prog = dir == 0 ? F.prog_fwd : F.prog_bwd;
    int* err = F.ilu_err;
    int64_t lim = F.spin_limit;
    int stall = F.test_stall;
    void* args[] = {&nx, &ny, &nz, &s28, &dinv, &y, &zs, &zp, &t, &dz, &zout, &prog, &err, &epoch, &lim, &stall};
    cudaError_t e = dir == 0
        ? cudaLaunchCooperativeKernel((const void*)k_ilu_pencil<T, true>, grid, kTY * kTZ, args, 0, st)
        : cudaLaunchCooperativeKernel((const void*)k_ilu_pencil<T, false>, grid, kTY * kTZ, args, 0, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    PS_TICK();
  }
  return true;
}

template <class T>
void alg1_steps_6_8(const FlowStage& F, const FlowWork<T>& W, double* zout, int ilu_mode, cudaStream_t st) {
  if (ilu_mode == PS_ILU_PENCIL && F.prog_fwd && ilu_pencil<T>(F, W, zout, st)) return;
  FlowView<T> V = fview<T>(F);
  for (int l = 0; l < F.nlev; ++l) {
    int32_t m = F.lev_off[l + 1] - F.lev_off[l];
    PS_TICK(); k_ilu_fwd<T><<<grid_for(m, 128), 128, 0, st>>>(F.lev_cells + F.lev_off[l], m, F.rp, F.ci, F.diagpos, V.sff,
                                                   V.dinv, W.y, W.zs, W.zp, W.t);
  }
  for (int l = F.nlev - 1; l >= 0; --l) {
    int32_t m = F.lev_off[l + 1] - F.lev_off[l];
    PS_TICK(); k_ilu_bwd<T><<<grid_for(m, 128), 128, 0, st>>>(F.lev_cells + F.lev_off[l], m, F.rp, F.ci, F.diagpos, V.sff,
                                                   V.dinv, W.t, W.zs, W.zp, W.dz, zout);
  }
}

template ps_status flow_alloc_work<float>(Arena&, const FlowStage&, FlowWork<float>&);
template ps_status flow_alloc_work<double>(Arena&, const FlowStage&, FlowWork<double>&);
template void alg1_steps_2_4<float>(const FlowStage&, const FlowWork<float>&, const float*, cudaStream_t);
template void alg1_steps_2_4<double>(const FlowStage&, const FlowWork<double>&, const double*, cudaStream_t);
template void alg1_steps_6_8<float>(const FlowStage&, const FlowWork<float>&, double*, int, cudaStream_t);
template void alg1_steps_6_8<double>(const FlowStage&, const FlowWork<double>&, double*, int, cudaStream_t);

}  // namespace ps_internal
