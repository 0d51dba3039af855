// Algorithm 1, flow part: steps 2-4 (A_fu coupling, D_ss^{-1}, complete A_ps)
// and steps 6-8 (residual of S_ff^(FS), block ILU(0) forward / backward sweeps,
// correction), in the interleaved (s, p) cell ordering of §5.3.
#include "flow.cuh"

namespace ps_internal {
namespace {

template <class T>
struct FlowView {
  const T *fu, *sff, *aps, *dinv, *dss;
};
template <class T>
FlowView<T> fview(const FlowStage& F) {
  FlowView<T> o;
  if constexpr (sizeof(T) == 4) {
    o.fu = F.fu_vf; o.sff = F.sff_f; o.aps = F.aps_f; o.dinv = F.dinv_f; o.dss = F.dss_f;
  } else {
    o.fu = F.fu_v; o.sff = F.sff; o.aps = F.aps; o.dinv = F.dinv; o.dss = F.dss;
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
void alg1_steps_6_8(const FlowStage& F, const FlowWork<T>& W, double* zout, int ilu_mode, cudaStream_t st) {
  (void)ilu_mode;
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
