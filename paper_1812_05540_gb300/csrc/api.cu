// C ABI: setup phase, Algorithm 1 and the flexible-GMRES iteration phase.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "amg.cuh"
#include "flow.cuh"
#include "krylov.cuh"
#include "rbm.cuh"

using namespace ps_internal;

namespace {

__global__ void k_sdc(int64_t nnzb, const double* __restrict__ uu, double* __restrict__ out) {
  int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= nnzb) return;
  out[q * 3 + 0] = uu[q * 9 + 0];
  out[q * 3 + 1] = uu[q * 9 + 4];
  out[q * 3 + 2] = uu[q * 9 + 8];
}
__global__ void k_d2f(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < n) b[t] = float(a[t]);
}
__global__ void k_f2d(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < n) b[t] = double(a[t]);
}
// row-sum lumping (§5.1 remark): A_up e per node (the p column of every 3x2 block of A_uf, summed over the row)
__global__ void k_rsl_aupe(int64_t nn, const int32_t* __restrict__ rp, const double* __restrict__ uf,
                           double* __restrict__ out) {
  int64_t I = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (I >= nn) return;
  double a[3] = {0.0, 0.0, 0.0};
  for (int32_t q = rp[I]; q < rp[I + 1]; ++q)
    for (int d = 0; d < 3; ++d) a[d] = a[d] + uf[int64_t(q) * 6 + d * 2 + 1];
  for (int d = 0; d < 3; ++d) out[3 * I + d] = a[d];
}
// D_sp = -(A_su w)_c, D_pp = -(A_pu w)_c per cell
__global__ void k_rsl_dfs(int64_t nc, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const double* __restrict__ fu, const double* __restrict__ w, double* __restrict__ dfs) {
  int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  for (int a = 0; a < 2; ++a) {
    double acc = 0.0;
    for (int32_t q = rp[c]; q < rp[c + 1]; ++q) {
      const int64_t J = ci[q];
      for (int e = 0; e < 3; ++e) acc += fu[int64_t(q) * 6 + a * 3 + e] * w[3 * J + e];
    }
    dfs[2 * c + a] = -acc;
  }
}
__global__ void k_i32_to_i64(const int32_t* __restrict__ a, int64_t* __restrict__ b, int64_t n) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < n) b[t] = a[t];
}

}  // namespace

struct ps_handle {
  Arena ar;   // Jacobian copies, mechanics AMG, Krylov workspace
  Arena arf;  // flow stage and pressure AMG (rebuilt by ps_setup_flow)
  cudaStream_t st = 0;
  ps_params prm;
  ps_grid grid;
  int64_t nn = 0, nc = 0, nu = 0, nf = 0, n = 0;
  int64_t nnzb_uu = 0, nnzb_uf = 0, nnzb_fu = 0;  // block patterns given to ps_setup
  bool mixed = false;
  bool bf16p = false;  // BF16 transfer operators (PS_MIXED_BF16P)
  JacDev J;
  double* dfs = nullptr;
  // row-sum-lumped fixed stress (PS_FS_RSL): w = M_uu^{-1} (A_up e) per node, and the (D_sp, D_pp) it gives
  double* rsl_w = nullptr;
  double* rsl_dfs = nullptr;
  Amg amg_u, amg_p;
  Rbm rbm_u;          // PS_MECH_RBM: the mechanics hierarchy in place of amg_u
  bool rbm = false;
  FlowStage F;
  FlowWork<float> w32;
  FlowWork<double> w64;
  float *vu32 = nullptr, *zu32 = nullptr;
  double* zu64 = nullptr;
  // Krylov
  int m = 100;
  int64_t ldv = 0;  // basis column stride: n rounded up to 32 rows, rows n..ldv-1 kept zero
  double *V = nullptr, *Z = nullptr, *r = nullptr, *b = nullptr, *x = nullptr, *part = nullptr, *mpart = nullptr;
  KrylovState K;
  double* hsc = nullptr;  // pinned: 8 scalars
  int* hflag = nullptr;   // pinned: Krylov flags [0..2], ILU error [3]
  // modified Gram-Schmidt launch: CTAs (0 = not possible), ticket barrier counter and its base
  int mgs_blocks[4] = {0, 0, 0, 0};
  double* mgs_part = nullptr;
  unsigned long long* mgs_bar = nullptr;
  unsigned long long mgs_base = 0;
  float ms_setup_u = 0, ms_setup_f = 0, ms_copy_in = 0;
  int64_t spmv_part = 0;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // per-iteration phase timers
  cudaEvent_t fe[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // Algorithm 1 sub-phase timers
  bool fine_pending = false;
  bool own_stream = false;  // the stream was created by ps_setup_batch and is destroyed by ps_free
};

namespace {

SmoothParams smooth_params(const ps_params& p) {
  SmoothParams s;
  s.kind = p.smoother; s.pre = p.pre; s.post = p.post; s.degree = p.cheb_degree; s.ratio = p.cheb_ratio;
  return s;
}

template <class T>
ps_status alg1(ps_handle* h, const double* v, double* z) {
  cudaStream_t st = h->st;
  SmoothParams sp = smooth_params(h->prm);
  FlowWork<T>* W;
  if constexpr (sizeof(T) == 4) W = &h->w32;
  else W = &h->w64;
  cudaEventRecord(h->fe[0], st);
  // step 1: z_u = M_uu^{-1} v_u
  if constexpr (sizeof(T) == 4) {
    PS_TICK(); k_d2f<<<grid_for(h->nu, 256), 256, 0, st>>>(v, h->vu32, h->nu);
    if (h->rbm) PS_TRY(rbm_vcycle<float>(h->rbm_u, sp, h->vu32, h->zu32, st));
    else PS_TRY(amg_vcycle<float>(h->amg_u, sp, h->vu32, h->zu32, st));
    cudaEventRecord(h->fe[1], st);
    PS_TICK(); k_f2d<<<grid_for(h->nu, 256), 256, 0, st>>>(h->zu32, z, h->nu);
    PS_TICK(); k_d2f<<<grid_for(h->nf, 256), 256, 0, st>>>(v + h->nu, W->vf, h->nf);
    // steps 2-4
    alg1_steps_2_4<float>(h->F, *W, h->zu32, st);
  } else {
    if (h->rbm) PS_TRY(rbm_vcycle<double>(h->rbm_u, sp, v, z, st));
    else PS_TRY(amg_vcycle<double>(h->amg_u, sp, v, z, st));
    cudaEventRecord(h->fe[1], st);
    PS_CUDA(cudaMemcpyAsync(W->vf, v + h->nu, sizeof(double) * h->nf, cudaMemcpyDeviceToDevice, st));
    alg1_steps_2_4<double>(h->F, *W, z, st);
  }
  cudaEventRecord(h->fe[2], st);
  // step 5: z_p = M_pp^{-1} w_p
  PS_TRY(amg_vcycle<T>(h->amg_p, sp, W->wp, W->zp, st));
  cudaEventRecord(h->fe[3], st);
  // steps 6-8
  alg1_steps_6_8<T>(h->F, *W, z + h->nu, h->prm.ilu_mode, st);  // ILU(0) or block Gauss-Seidel, per F.local
  cudaEventRecord(h->fe[4], st);
  h->fine_pending = true;
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

ps_status apply_prec(ps_handle* h, const double* v, double* z) {
  return h->mixed ? alg1<float>(h, v, z) : alg1<double>(h, v, z);
}

// streaming copy of n16 16-byte words, four independent loads in flight per thread
__global__ void __launch_bounds__(256) k_copy16(const uint4* __restrict__ src, uint4* __restrict__ dst, int64_t n16) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n16; i += 4 * stride) {
    const uint4 a = src[i], b = src[i + stride], c = src[i + 2 * stride], d = src[i + 3 * stride];
    dst[i] = a; dst[i + stride] = b; dst[i + 2 * stride] = c; dst[i + 3 * stride] = d;
  }
  for (; i < n16; i += stride) dst[i] = src[i];
}

// Copy of one input array into device memory the handle owns.  Host memory that CUDA has pinned is mapped
// into the device's address space: a streaming kernel reads it over the host link, the whole array in one
// launch, without a copy-engine transfer; pageable host memory, unaligned arrays and device memory use
// cudaMemcpyAsync.
ps_status copy_to(const void* src, size_t bytes, void* dst, bool host, cudaStream_t st) {
  if (bytes == 0) return PS_OK;
  if (host && bytes >= 16) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, src) == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer &&
        (reinterpret_cast<uintptr_t>(at.devicePointer) & 15) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
      static int sms = 0;
      if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
      }
      const int64_t n16 = int64_t(bytes / 16);
      const int64_t blocks = std::min<int64_t>(int64_t(sms) * 8, (n16 + 255) / 256);
      PS_TICK(); k_copy16<<<unsigned(blocks), 256, 0, st>>>(static_cast<const uint4*>(at.devicePointer),
                                                          static_cast<uint4*>(dst), n16);
      PS_CUDA(cudaGetLastError());
      const size_t tail = bytes - size_t(n16) * 16;
      if (tail)
        PS_CUDA(cudaMemcpyAsync(static_cast<char*>(dst) + n16 * 16, static_cast<const char*>(src) + n16 * 16, tail,
                                cudaMemcpyHostToDevice, st));
      return PS_OK;
    }
    cudaGetLastError();
  }
  PS_CUDA(cudaMemcpyAsync(dst, src, bytes, host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
  return PS_OK;
}

ps_status copy_in(Arena& ar, const void* src, size_t bytes, void** dst, bool host, cudaStream_t st) {
  PS_TRY(ar.alloc(dst, bytes));
  return copy_to(src, bytes, *dst, host, st);
}

ps_status copy_bsr(ps_handle* h, const ps_bsr& B, int32_t** rp, int32_t** ci, const double** v) {
  bool host = h->prm.host_ptrs != 0;
  int64_t* rp64;
  PS_TRY(copy_in(h->ar, B.rowptr, sizeof(int64_t) * (B.n_brow + 1), (void**)&rp64, host, h->st));
  PS_TRY(h->ar.alloc(rp, B.n_brow + 1));
  rowptr_to_i32(rp64, *rp, B.n_brow + 1, h->st);
  PS_TRY(h->ar.alloc(ci, B.nnzb + 1));
  PS_TRY(copy_to(B.colind, sizeof(int32_t) * B.nnzb, *ci, host, h->st));
  void* vv;
  PS_TRY(copy_in(h->ar, B.val, sizeof(double) * B.nnzb * B.br * B.bc, &vv, host, h->st));
  *v = static_cast<const double*>(vv);
  PS_CUDA(cudaStreamSynchronize(h->st));
  h->ar.release(rp64);
  return PS_OK;
}

bool bsr_ok(const ps_bsr& B, int64_t rows, int64_t cols, int br, int bc) {
  return B.n_brow == rows && B.n_bcol == cols && B.br == br && B.bc == bc && B.rowptr && B.colind && B.val &&
         B.nnzb >= 0 && B.nnzb < (int64_t(1) << 31) / 9;
}

ps_status build_flow(ps_handle* h, cudaStream_t st) {
  Arena& ar = h->arf;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  FlowStage& F = h->F;
  F.nx = h->grid.nx; F.ny = h->grid.ny; F.nz = h->grid.nz;
  F.nc = h->nc; F.nnzb = int64_t(0);
  int32_t tot = 0;
  PS_CUDA(cudaMemcpyAsync(&tot, h->J.ff_rp + h->nc, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  PS_CUDA(cudaStreamSynchronize(st));
  F.nnzb = tot;
  F.rp = h->J.ff_rp; F.ci = h->J.ff_ci;
  F.fu_rp = h->J.fu_rp; F.fu_ci = h->J.fu_ci; F.fu_v = h->J.fu_v;
  F.spin_limit = h->prm.spin_limit > 0 ? h->prm.spin_limit : 2000000;
  F.local = h->prm.local_stage;
  F.cpr = h->prm.cpr_reduction;
  F.gs_sweeps = h->prm.local_sweeps;
  F.ilu_local = h->prm.ilu_scope == PS_ILU_LOCAL ? 1 : 0;
  F.test_stall = h->prm.test_stall_wave;
  const double* dfs = h->dfs;
  if (h->prm.fs_mode == PS_FS_RSL) {
    PS_TRY(ar.alloc(&h->rsl_dfs, 2 * h->nc));
    PS_TICK(); k_rsl_dfs<<<grid_for(h->nc, 256), 256, 0, st>>>(h->nc, h->J.fu_rp, h->J.fu_ci, h->J.fu_v, h->rsl_w,
                                                              h->rsl_dfs);
    dfs = h->rsl_dfs;
  }
  PS_TRY(flow_setup(ar, F, h->J.ff_rp, h->J.ff_ci, h->J.ff_v, dfs, h->mixed, st));
  if (h->mixed) {
    int64_t nfu = 0;
    int32_t t2 = 0;
    PS_CUDA(cudaMemcpyAsync(&t2, h->J.fu_rp + h->nc, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    nfu = t2;
    PS_TRY(ar.alloc(&F.fu_vf, nfu * 6 + 1));
    PS_TICK(); k_d2f<<<grid_for(nfu * 6, 256), 256, 0, st>>>(h->J.fu_v, F.fu_vf, nfu * 6);
  }
  // steps 2 and 4 on the structured grid: A_fu from the Jacobian's stencil copy (FP32 copy in mixed mode)
  if (h->J.fu_s) {
    if (h->mixed) {
      const int64_t cnt = (h->nc + 31) / 32 * 32 * 8 * 6;
      PS_TRY(ar.alloc(&F.fu_st_f, cnt));
      PS_TICK(); k_d2f<<<grid_for(cnt, 256), 256, 0, st>>>(h->J.fu_s, F.fu_st_f, cnt);
    } else {
      F.fu_st_d = h->J.fu_s;
    }
  }
  AmgParams ap;
  ap.theta = h->prm.theta_p; ap.coarse_max = h->prm.coarse_max_p; ap.max_levels = h->prm.max_levels;
  ap.mixed = h->mixed;
  ap.bf16p = h->bf16p;
  ap.l1 = h->prm.smoother == PS_SMOOTH_L1JACOBI;
  PS_TRY(amg_build(ar, h->amg_p, 1, h->nc, F.nnzb, F.rp, F.ci, F.spp, ap, st));
  bool sp_ok = false;
  PS_TRY(amg_stencil(ar, h->amg_p, h->grid.nx, h->grid.ny, h->grid.nz, 7, h->mixed, &sp_ok, st));
  h->amg_p.tail_mode = h->prm.vcycle_tail;
  h->amg_p.autotune = h->prm.autotune;
  if (h->mixed) {
    PS_TRY(amg_alloc_work<float>(ar, h->amg_p, smooth_params(h->prm), st));
    PS_TRY(flow_alloc_work<float>(ar, F, h->w32));
  } else {
    PS_TRY(amg_alloc_work<double>(ar, h->amg_p, smooth_params(h->prm), st));
    PS_TRY(flow_alloc_work<double>(ar, F, h->w64));
  }
  cudaEventRecord(e1, st);
  PS_CUDA(cudaEventSynchronize(e1));
  cudaEventElapsedTime(&h->ms_setup_f, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return PS_OK;
}

ps_status build_mechanics(ps_handle* h, int64_t nnzb, cudaEvent_t e0, cudaEvent_t e1);
ps_status finish_setup(ps_handle* h);

ps_status setup_impl(ps_handle* h, const ps_jacobian* jac) {
  cudaStream_t st = h->st;
  Arena& ar = h->ar;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  JacDev& J = h->J;
  J.nn = h->nn; J.nc = h->nc;
  PS_TRY(copy_bsr(h, jac->A_uu, &J.uu_rp, &J.uu_ci, &J.uu_v));
  PS_TRY(copy_bsr(h, jac->A_uf, &J.uf_rp, &J.uf_ci, &J.uf_v));
  PS_TRY(copy_bsr(h, jac->A_fu, &J.fu_rp, &J.fu_ci, &J.fu_v));
  PS_TRY(copy_bsr(h, jac->A_ff, &J.ff_rp, &J.ff_ci, &J.ff_v));
  PS_TRY(copy_in(ar, jac->d_fs, sizeof(double) * 2 * h->nc, (void**)&h->dfs, h->prm.host_ptrs != 0, st));
  {
    cudaEvent_t ec;
    cudaEventCreate(&ec);
    cudaEventRecord(ec, st);
    PS_CUDA(cudaEventSynchronize(ec));
    cudaEventElapsedTime(&h->ms_copy_in, e0, ec);
    cudaEventDestroy(ec);
  }
  J.nx = h->grid.nx; J.ny = h->grid.ny; J.nz = h->grid.nz;
  bool structured = false;
  PS_TRY(jac_build_stencil(ar, J, &structured, st));
  if (flow_check_pattern(ar, h->grid, J.ff_rp, J.ff_ci, st) != PS_OK) {
    set_reason("A_ff is not the 7-point TPFA pattern of the %dx%dx%d grid", h->grid.nx, h->grid.ny, h->grid.nz);
    return PS_ERR_INVALID;
  }
  int64_t nnzb = jac->A_uu.nnzb;
  PS_TRY(build_mechanics(h, nnzb, e0, e1));
  // §5.3 flow stage
  PS_TRY(build_flow(h, st));
  return finish_setup(h);
}

// §5.2 mechanics preconditioner (and the row-sum-lumped fixed stress, which applies it), on the handle's stream
ps_status build_mechanics(ps_handle* h, int64_t nnzb, cudaEvent_t e0, cudaEvent_t e1) {
  cudaStream_t st = h->st;
  Arena& ar = h->ar;
  JacDev& J = h->J;
  if (h->rbm) {
    // rigid-body-mode smoothed aggregation on the full A_uu
    PS_TRY(rbm_build(ar, h->rbm_u, h->grid.nx, h->grid.ny, h->grid.nz, nnzb, J.uu_rp, J.uu_ci, J.uu_v,
                     h->prm.theta_u, h->prm.coarse_max_u, h->prm.max_levels, h->mixed, st));
    if (h->mixed) PS_TRY(rbm_alloc_work<float>(ar, h->rbm_u, st));
    else PS_TRY(rbm_alloc_work<double>(ar, h->rbm_u, st));
  } else {
    // §5.2 mechanics: amg(A_uu^(SDC)) on the three diagonal components of each 3x3 block
    double* sdc;
    PS_TRY(ar.alloc(&sdc, nnzb * 3));
    PS_TICK(); k_sdc<<<grid_for(nnzb, 256), 256, 0, st>>>(nnzb, J.uu_v, sdc);
    AmgParams ap;
    ap.theta = h->prm.theta_u; ap.coarse_max = h->prm.coarse_max_u; ap.max_levels = h->prm.max_levels;
    ap.mixed = h->mixed;
    ap.bf16p = h->bf16p;
    ap.l1 = h->prm.smoother == PS_SMOOTH_L1JACOBI;
    PS_TRY(amg_build(ar, h->amg_u, 3, h->nn, nnzb, J.uu_rp, J.uu_ci, sdc, ap, st));
    bool su_ok = false;
    PS_TRY(amg_stencil(ar, h->amg_u, h->grid.nx + 1, h->grid.ny + 1, h->grid.nz + 1, 27, h->mixed, &su_ok, st));
    h->amg_u.tail_mode = h->prm.vcycle_tail;
    h->amg_u.autotune = h->prm.autotune;
    if (h->mixed) PS_TRY(amg_alloc_work<float>(ar, h->amg_u, smooth_params(h->prm), st));
    else PS_TRY(amg_alloc_work<double>(ar, h->amg_u, smooth_params(h->prm), st));
  }
  if (h->mixed) {
    PS_TRY(ar.alloc(&h->vu32, h->nu));
    PS_TRY(ar.alloc(&h->zu32, h->nu));
  }
  if (h->prm.fs_mode == PS_FS_RSL) {
    // w = M_uu^{-1} (A_up e): one FP64 V-cycle on a view of the mechanics hierarchy with its own FP64 work
    // vectors (the fixed-stress diagonal is one of the FP64 parts of the mixed mode)
    double* aupe;
    PS_TRY(ar.alloc(&aupe, h->nu));
    PS_TRY(ar.alloc(&h->rsl_w, h->nu));
    PS_TICK(); k_rsl_aupe<<<grid_for(h->nn, 256), 256, 0, st>>>(h->nn, J.uf_rp, J.uf_v, aupe);
    Arena tmp;
    tmp.stream = st;
    ps_status rs = PS_OK;
    if (h->rbm) {
      Rbm S = h->rbm_u;
      S.gexec = nullptr;
      rs = rbm_alloc_work<double>(tmp, S, st);
      if (rs == PS_OK) rs = rbm_vcycle_direct<double>(S, smooth_params(h->prm), aupe, h->rsl_w, st);
    } else {
      Amg S = h->amg_u;
      S.gexec = nullptr;
      S.tail = nullptr;
      for (auto& L : S.L) {
        L.x = L.t = L.r = L.d = L.b = L.e = L.dsi = nullptr;
        L.sv_f = nullptr;
      }
      rs = amg_alloc_work<double>(tmp, S, smooth_params(h->prm), st);
      if (rs == PS_OK) rs = amg_vcycle_direct<double>(S, smooth_params(h->prm), aupe, h->rsl_w, st);
    }
    cudaStreamSynchronize(st);
    tmp.free_all();
    ar.release(aupe);
    PS_TRY(rs);
  }
  cudaEventRecord(e1, st);
  PS_CUDA(cudaEventSynchronize(e1));
  cudaEventElapsedTime(&h->ms_setup_u, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return PS_OK;
}

// what follows both stages: the V-cycles' flags and launch options, the Krylov workspace
ps_status finish_setup(ps_handle* h) {
  cudaStream_t st = h->st;
  Arena& ar = h->ar;
  // the V-cycles' bounded grid barriers report through the same flag as the wavefront waits
  h->amg_u.err = h->prm.vcycle_tail ? h->F.ilu_err : nullptr;
  h->amg_p.err = h->prm.vcycle_tail ? h->F.ilu_err : nullptr;
  h->amg_u.pdl = h->amg_p.pdl = h->prm.pdl ? 1 : 0;
  h->amg_u.spin_limit = h->amg_p.spin_limit = h->F.spin_limit;
  // Krylov workspace
  int m = h->m;
  int64_t n = h->n;
  h->ldv = (n + 31) / 32 * 32;
  PS_TRY(ar.alloc(&h->V, size_t(h->ldv) * (m + 1)));
  PS_TRY(ar.alloc(&h->Z, size_t(n) * m));
  PS_TRY(ar.alloc(&h->r, n));
  PS_TRY(ar.alloc(&h->b, n));
  PS_TRY(ar.alloc(&h->x, n));
  int64_t gu = ceil_div(h->nn * 32, 256), gf = ceil_div(h->nc * 32, 256);  // bound for both SpMV paths
  h->spmv_part = kRedBlocks + gu + gf;
  PS_TRY(ar.alloc(&h->part, h->spmv_part));
  PS_TRY(ar.alloc(&h->mpart, size_t(m + 2) * kRedBlocks));
  KrylovState& K = h->K;
  PS_TRY(ar.alloc(&K.H, size_t(m + 1) * m));
  PS_TRY(ar.alloc(&K.cs, m)); PS_TRY(ar.alloc(&K.sn, m)); PS_TRY(ar.alloc(&K.g, m + 1));
  PS_TRY(ar.alloc(&K.h1, m + 2)); PS_TRY(ar.alloc(&K.h2, m + 2)); PS_TRY(ar.alloc(&K.y, m + 1));
  PS_TRY(ar.alloc(&K.sc, 16)); PS_TRY(ar.alloc(&K.flag, 4));
  PS_CUDA(cudaMemsetAsync(K.flag, 0, 4 * sizeof(int), st));
  if (h->prm.ortho == PS_ORTHO_MGS) {
    PS_TRY(mgs_grid(h->mgs_blocks));
    int mb = std::max(std::max(h->mgs_blocks[0], h->mgs_blocks[1]), std::max(h->mgs_blocks[2], h->mgs_blocks[3]));
    if (mb > 0) {
      PS_TRY(ar.alloc(&h->mgs_part, size_t(mgs_partials()) * mb));
      PS_TRY(ar.alloc(&K.gram, size_t(m + 1) * mgs_gram_stride()));
      PS_TRY(ar.alloc(&h->mgs_bar, 1));
      PS_CUDA(cudaMemsetAsync(h->mgs_bar, 0, sizeof(unsigned long long), st));
      h->mgs_base = 0;
    }
  }
  for (int e = 0; e < 4; ++e) PS_CUDA(cudaEventCreate(&h->ev[e]));
  for (int e = 0; e < 5; ++e) PS_CUDA(cudaEventCreate(&h->fe[e]));
  PS_CUDA(cudaMallocHost(&h->hsc, 16 * sizeof(double)));
  PS_CUDA(cudaMallocHost(&h->hflag, 4 * sizeof(int)));
  PS_CUDA(cudaStreamSynchronize(st));
  return PS_OK;
}

}  // namespace

extern "C" {

void ps_params_default(ps_params* p) {
  std::memset(p, 0, sizeof(*p));
  p->precision = PS_FP64;
  p->restart = 100;
  p->max_iters = 1000;
  p->smoother = PS_SMOOTH_CHEBYSHEV;
  p->pre = 1; p->post = 1;
  p->cheb_degree = 2;
  p->cheb_ratio = 20.0;
  p->theta_u = 0.08; p->theta_p = 0.08;
  p->coarse_max_u = 500; p->coarse_max_p = 500;
  p->max_levels = 25;
  p->ilu_mode = PS_ILU_PENCIL;
  p->spin_limit = 2000000;
  p->ortho_sweep = 8;
  p->vcycle_tail = 0;
  p->pdl = 1;
  p->ilu_scope = PS_ILU_LOCAL;
  p->mech_amg = PS_MECH_SDC;
  p->local_stage = PS_LOCAL_ILU0;
  p->local_sweeps = 3;
}

ps_status ps_setup(const ps_jacobian* jac, const ps_grid* grid, const ps_params* params, ps_handle** out) {
  if (!jac || !grid || !params || !out) return PS_ERR_INVALID;
  *out = nullptr;
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return PS_ERR_INVALID;
  int64_t nn = int64_t(grid->nx + 1) * (grid->ny + 1) * (grid->nz + 1);
  int64_t nc = int64_t(grid->nx) * grid->ny * grid->nz;
  if (!bsr_ok(jac->A_uu, nn, nn, 3, 3) || !bsr_ok(jac->A_uf, nn, nc, 3, 2) || !bsr_ok(jac->A_fu, nc, nn, 2, 3) ||
      !bsr_ok(jac->A_ff, nc, nc, 2, 2) || !jac->d_fs)
    return PS_ERR_INVALID;
  if (params->restart < 1 || params->restart > 120 || params->max_iters < 1) return PS_ERR_INVALID;
  if (params->precision != PS_FP64 && params->precision != PS_MIXED_FP32 && params->precision != PS_MIXED_BF16P)
    return PS_ERR_INVALID;
  if (params->local_stage != PS_LOCAL_ILU0 && params->local_stage != PS_LOCAL_HBGS) return PS_ERR_INVALID;
  if (params->cpr_reduction != PS_CPR_QUASI_IMPES && params->cpr_reduction != PS_CPR_TRUE_IMPES)
    return PS_ERR_INVALID;
  if (params->solver != PS_SOLVER_FGMRES && params->solver != PS_SOLVER_RICHARDSON) return PS_ERR_INVALID;
  if (params->fs_mode != PS_FS_GIVEN && params->fs_mode != PS_FS_RSL) return PS_ERR_INVALID;
  if (params->vcycle_tail < 0 || params->vcycle_tail > 2) return PS_ERR_INVALID;
  if (params->autotune < 0 || params->autotune > 1) return PS_ERR_INVALID;
  if (params->mech_amg != PS_MECH_SDC && params->mech_amg != PS_MECH_RBM) return PS_ERR_INVALID;
  if (params->mech_amg == PS_MECH_RBM && params->smoother != PS_SMOOTH_CHEBYSHEV) {
    set_reason("the rigid-body-mode mechanics hierarchy smooths with Chebyshev only");
    return PS_ERR_INVALID;
  }
  if (params->local_stage == PS_LOCAL_HBGS && (params->local_sweeps < 1 || params->local_sweeps > 64)) {
    set_reason("local_sweeps must be 1..64 for the block Gauss-Seidel local stage");
    return PS_ERR_INVALID;
  }
  ps_handle* h = new ps_handle();
  h->prm = *params;
  h->rbm = params->mech_amg == PS_MECH_RBM;
  h->grid = *grid;
  h->st = (cudaStream_t)params->stream;
  h->ar.stream = h->st;
  h->arf.stream = h->st;
  h->ar.budget = params->hbm_budget;
  h->nn = nn; h->nc = nc; h->nu = 3 * nn; h->nf = 2 * nc; h->n = h->nu + h->nf;
  h->nnzb_uu = jac->A_uu.nnzb; h->nnzb_uf = jac->A_uf.nnzb; h->nnzb_fu = jac->A_fu.nnzb;
  h->mixed = params->precision == PS_MIXED_FP32 || params->precision == PS_MIXED_BF16P;
  h->bf16p = params->precision == PS_MIXED_BF16P;
  h->m = params->restart;
  ps_status s = setup_impl(h, jac);
  if (s != PS_OK) {
    ps_free(h);
    return s;
  }
  *out = h;
  return PS_OK;
}

ps_status ps_set_test_stall(ps_handle* h, int32_t wave_cta_plus_one) {
  if (!h || wave_cta_plus_one < 0) return PS_ERR_INVALID;
  h->prm.test_stall_wave = wave_cta_plus_one;
  h->F.test_stall = wave_cta_plus_one;
  return PS_OK;
}

ps_status ps_set_test_stall_gs(ps_handle* h, int32_t cta_plus_one) {
  if (!h || cta_plus_one < 0) return PS_ERR_INVALID;
  h->prm.test_stall_gs = cta_plus_one;
  return PS_OK;
}

ps_status ps_setup_flow(ps_handle* h, const ps_jacobian* jac) {
  if (!h || !jac) return PS_ERR_INVALID;
  if (!bsr_ok(jac->A_fu, h->nc, h->nn, 2, 3) || !bsr_ok(jac->A_ff, h->nc, h->nc, 2, 2) || !jac->d_fs ||
      jac->A_ff.nnzb != h->F.nnzb || jac->A_fu.nnzb != h->nnzb_fu) {
    set_reason("ps_setup_flow: A_fu, A_ff and d_fs must keep the patterns given to ps_setup");
    return PS_ERR_INVALID;
  }
  // new mechanics-row values are optional: A_uu and A_uf with the setup's patterns, used by the outer
  // Jacobian SpMV; the mechanics AMG built at ps_setup is kept either way
  const bool new_uu = jac->A_uu.val != nullptr, new_uf = jac->A_uf.val != nullptr;
  if ((new_uu && (!bsr_ok(jac->A_uu, h->nn, h->nn, 3, 3) || jac->A_uu.nnzb != h->nnzb_uu)) ||
      (new_uf && (!bsr_ok(jac->A_uf, h->nn, h->nc, 3, 2) || jac->A_uf.nnzb != h->nnzb_uf))) {
    set_reason("ps_setup_flow: A_uu and A_uf, when given, must keep the patterns given to ps_setup");
    return PS_ERR_INVALID;
  }
  cudaStream_t st = h->st;
  bool host = h->prm.host_ptrs != 0;
  if (new_uu) PS_TRY(copy_to(jac->A_uu.val, sizeof(double) * h->nnzb_uu * 9, const_cast<double*>(h->J.uu_v), host, st));
  if (new_uf) PS_TRY(copy_to(jac->A_uf.val, sizeof(double) * h->nnzb_uf * 6, const_cast<double*>(h->J.uf_v), host, st));
  PS_TRY(copy_to(jac->A_fu.val, sizeof(double) * jac->A_fu.nnzb * 6, const_cast<double*>(h->J.fu_v), host, st));
  PS_TRY(copy_to(jac->A_ff.val, sizeof(double) * jac->A_ff.nnzb * 4, const_cast<double*>(h->J.ff_v), host, st));
  PS_TRY(copy_to(jac->d_fs, sizeof(double) * 2 * h->nc, h->dfs, host, st));
  // the outer SpMV reads the stencil-indexed copies: refill them from the new values
  PS_TRY(jac_refresh_stencil(h->ar, h->J, (new_uu ? 1 : 0) | (new_uf ? 2 : 0) | 4 | 8, st));
  cudaStreamSynchronize(st);
  amg_release_graph(h->amg_p);
  h->arf.free_all();
  h->F = FlowStage();
  h->amg_p = Amg();
  h->w32 = FlowWork<float>();
  h->w64 = FlowWork<double>();
  PS_TRY(build_flow(h, st));
  // the mechanics V-cycle graph holds the old flag's address: capture it again with the new one
  amg_release_graph(h->amg_u);
  rbm_release_graph(h->rbm_u);
  h->amg_u.err = h->prm.vcycle_tail ? h->F.ilu_err : nullptr;
  h->amg_p.err = h->prm.vcycle_tail ? h->F.ilu_err : nullptr;
  h->amg_u.pdl = h->amg_p.pdl = h->prm.pdl ? 1 : 0;
  h->amg_u.spin_limit = h->amg_p.spin_limit = h->F.spin_limit;
  return PS_OK;
}

ps_status ps_spmv(ps_handle* h, const double* x, double* y) {
  if (!h || !x || !y) return PS_ERR_INVALID;
  jac_spmv(h->J, x, y, nullptr, nullptr, h->st);
  PS_CUDA(cudaGetLastError());
  PS_CUDA(cudaStreamSynchronize(h->st));
  return PS_OK;
}

ps_status ps_apply_prec(ps_handle* h, const double* v, double* z) {
  if (!h || !v || !z) return PS_ERR_INVALID;
  PS_TRY(apply_prec(h, v, z));
  PS_CUDA(cudaStreamSynchronize(h->st));
  return PS_OK;
}

namespace {

// Sequential fixed-stress strategy (§5.4 remark): x_{k+1} = x_k + M^{-1}(b - A x_k) from x_0 = 0, with the
// true FP64 residual checked before every pass.  Work vectors: r (residual), Z's first column (M^{-1} r).
ps_status solve_richardson(ps_handle* h, const double* rhs, double* x, double tol, ps_stats* stats) {
  cudaStream_t st = h->st;
  const int64_t n = h->n;
  KrylovState& K = h->K;
  const bool host = h->prm.host_ptrs != 0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  PS_TRY(copy_to(rhs, sizeof(double) * n, h->b, host, st));
  double* xk = h->x;
  double* z = h->Z;
  fill_zero(xk, n, st);
  const double one = 1.0;
  PS_CUDA(cudaMemcpyAsync(K.y, &one, sizeof(double), cudaMemcpyHostToDevice, st));
  multidot(h->V, n, 0, h->b, n, h->mpart, K.sc + 7, 1, nullptr, st);
  PS_CUDA(cudaMemcpyAsync(h->hsc, K.sc, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
  PS_CUDA(cudaStreamSynchronize(st));
  const double bn2 = h->hsc[7];
  ps_stats S;
  std::memset(&S, 0, sizeof(S));
  ps_status result = PS_OK;
  if (std::isnan(bn2)) {
    result = PS_ERR_NAN;
  } else if (bn2 > 0.0) {
    const double bnorm = std::sqrt(bn2);
    for (;;) {
      jac_spmv(h->J, xk, h->r, h->b, h->part, st);
      finish_sum(h->part, K.sc + 3, st);
      PS_CUDA(cudaMemcpyAsync(h->hsc, K.sc, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
      PS_CUDA(cudaMemcpyAsync(h->hflag + 3, h->F.ilu_err, sizeof(int), cudaMemcpyDeviceToHost, st));
      PS_CUDA(cudaStreamSynchronize(st));
      if (h->hflag[3]) {
        PS_CUDA(cudaMemsetAsync(h->F.ilu_err, 0, sizeof(int), st));
        set_reason("a bounded wait of the wavefront ILU(0) sweep or of a V-cycle grid barrier gave up");
        result = PS_ERR_TIMEOUT;
        break;
      }
      const double rr = std::sqrt(h->hsc[3]) / bnorm;
      S.true_relres = rr;
      S.est_relres = rr;
      if (std::isnan(rr)) { result = PS_ERR_NAN; break; }
      if (rr <= tol) break;
      if (S.iters >= h->prm.max_iters) { result = PS_ERR_NOT_CONVERGED; break; }
      cudaEventRecord(h->ev[0], st);
      PS_TRY(apply_prec(h, h->r, z));
      cudaEventRecord(h->ev[1], st);
      maxpy(z, n, 1, K.y, xk, n, st);
      S.iters++;
      {
        // phase times of the previous pass (its events completed with the synchronisation above)
        float a = 0;
        PS_CUDA(cudaEventSynchronize(h->ev[1]));
        cudaEventElapsedTime(&a, h->ev[0], h->ev[1]);
        S.ms_prec += a;
        float f[4] = {0, 0, 0, 0};
        for (int q = 0; q < 4; ++q) cudaEventElapsedTime(&f[q], h->fe[q], h->fe[q + 1]);
        S.ms_vcycle_u += f[0]; S.ms_flow24 += f[1]; S.ms_vcycle_p += f[2]; S.ms_ilu += f[3];
      }
    }
  }
  PS_CUDA(cudaMemcpyAsync(x, xk, sizeof(double) * n, host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
  cudaEventRecord(e1, st);
  PS_CUDA(cudaEventSynchronize(e1));
  cudaEventElapsedTime(&S.ms_solve, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  S.ms_setup_u = h->ms_setup_u;
  S.ms_setup_f = h->ms_setup_f;
  S.ms_copy_in = h->ms_copy_in;
  S.handle_bytes = h->ar.bytes + h->arf.bytes;
  S.levels_u = int32_t(h->rbm ? h->rbm_u.L.size() : h->amg_u.L.size());
  S.levels_p = int32_t(h->amg_p.L.size());
  if (stats) *stats = S;
  return result;
}

}  // namespace

}  // extern "C"

namespace {

// One FGMRES(m) solve (§4, flexible right preconditioning) as a resumable sequence of device steps, so
// that ps_solve runs one and ps_solve_batch runs many in lockstep on their own streams with one host
// synchronisation per step for all of them.  A step is either one Arnoldi iteration (Algorithm 1, the
// FP64 Jacobian SpMV, Gram-Schmidt, Givens update, status copy) or the end of a cycle (Hessenberg solve,
// x += Z y, true residual).  Each system runs the same kernels in the same order either way.
struct FgmresRun {
  ps_handle* h = nullptr;
  const double* rhs = nullptr;
  double* x = nullptr;
  double tol = 0.0;
  ps_stats S;
  ps_status result = PS_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double bnorm = 0.0;
  int total = 0, j = 0, jend = -1;
  bool brk = false;
  bool done = false;
  bool cycle_end = false;  // the next step closes the cycle
  bool fresh_cycle = true; // the next Arnoldi iteration opens a cycle

  // ||b|| and the start of the first cycle (one synchronisation)
  ps_status start(ps_handle* hh, const double* b_in, double* x_out, double t) {
    h = hh; rhs = b_in; x = x_out; tol = t;
    std::memset(&S, 0, sizeof(S));
    cudaStream_t st = h->st;
    const int64_t n = h->n;
    KrylovState& K = h->K;
    const bool host = h->prm.host_ptrs != 0;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    PS_TRY(copy_to(rhs, sizeof(double) * n, h->b, host, st));
    fill_zero(h->x, n, st);
    const int64_t ldv = h->ldv;
    if (ldv > n)  // padding rows of the basis (a failed solve may have left a NaN there)
      PS_CUDA(cudaMemset2DAsync(h->V + n, size_t(ldv) * sizeof(double), 0, size_t(ldv - n) * sizeof(double), h->m + 1,
                                st));
    multidot(h->V, n, 0, h->b, n, h->mpart, K.sc + 7, 1, nullptr, st);
    PS_CUDA(cudaMemcpyAsync(h->hsc, K.sc, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    const double bn2 = h->hsc[7];
    if (!(bn2 > 0.0)) {
      if (std::isnan(bn2)) result = PS_ERR_NAN;
      done = true;
      return PS_OK;
    }
    bnorm = std::sqrt(bn2);
    h->hsc[8] = bn2;
    h->hsc[9] = bnorm;
    PS_CUDA(cudaMemcpyAsync(K.sc + 3, &h->hsc[8], sizeof(double), cudaMemcpyHostToDevice, st));
    PS_CUDA(cudaMemcpyAsync(K.sc + 7, &h->hsc[9], sizeof(double), cudaMemcpyHostToDevice, st));
    PS_CUDA(cudaMemcpyAsync(h->r, h->b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    return PS_OK;
  }

  // enqueue the next step (no synchronisation)
  ps_status enqueue() {
    cudaStream_t st = h->st;
    const int64_t n = h->n, ldv = h->ldv;
    const int m = h->m;
    KrylovState& K = h->K;
    if (cycle_end) {
      hessenberg_solve(K, m, jend, st);
      maxpy(h->Z, n, jend + 1, K.y, h->x, n, st);
      jac_spmv(h->J, h->x, h->r, h->b, h->part, st);
      finish_sum(h->part, K.sc + 3, st);
      PS_CUDA(cudaMemcpyAsync(h->hsc, K.sc, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
      return PS_OK;
    }
    if (fresh_cycle) {
      cycle_start(K, m, st);
      scale_vec(h->r, h->V, n, K.sc + 4, st);
      j = 0;
      jend = -1;
      brk = false;
      fresh_cycle = false;
    }
    double* vj = h->V + j * ldv;
    double* zj = h->Z + int64_t(j) * n;
    double* w = h->V + (j + 1) * ldv;
    cudaEventRecord(h->ev[0], st);
    PS_TRY(apply_prec(h, vj, zj));
    cudaEventRecord(h->ev[1], st);
    jac_spmv(h->J, zj, w, nullptr, nullptr, st);
    cudaEventRecord(h->ev[2], st);
    if (h->prm.ortho == PS_ORTHO_MGS &&
        mgs_step(h->V, ldv, j, w, n, K, h->mgs_part, h->mgs_blocks, h->mgs_bar, &h->mgs_base, h->prm.spin_limit,
                 h->prm.test_stall_gs, h->prm.ortho_sweep, st)) {
      // modified Gram-Schmidt (w normalised in the same launch)
      arnoldi_finish(K, m, j, st);
    } else {
      // classical Gram-Schmidt with selective reorthogonalisation
      multidot(h->V, ldv, j + 1, w, n, h->mpart, K.h1, 1, nullptr, st);
      PS_CUDA(cudaMemcpyAsync(K.sc + 0, K.h1 + j + 1, sizeof(double), cudaMemcpyDeviceToDevice, st));
      mupdate(h->V, ldv, j + 1, K.h1, w, n, h->mpart, K.sc + 1, nullptr, st);
      arnoldi_check(K, st);
      multidot(h->V, ldv, j + 1, w, n, h->mpart, K.h2, 0, K.flag, st);
      mupdate(h->V, ldv, j + 1, K.h2, w, n, h->mpart, K.sc + 2, K.flag, st);
      arnoldi_finish(K, m, j, st);
      scale_vec(w, w, n, K.sc + 4, st);
    }
    cudaEventRecord(h->ev[3], st);
    PS_CUDA(cudaMemcpyAsync(h->hsc, K.sc, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaMemcpyAsync(h->hflag, K.flag, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaMemcpyAsync(h->hflag + 3, h->F.ilu_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    return PS_OK;
  }

  // after the stream has reached the end of the enqueued step: read its status and choose the next one
  ps_status after_sync() {
    cudaStream_t st = h->st;
    KrylovState& K = h->K;
    if (cycle_end) {
      cycle_end = false;
      const double rr = std::sqrt(h->hsc[3]) / bnorm;
      S.true_relres = rr;
      S.iters = total;
      if (std::isnan(rr)) { result = PS_ERR_NAN; done = true; }
      else if (rr <= tol) { result = PS_OK; done = true; }
      else if (brk) { result = PS_ERR_BREAKDOWN; done = true; }
      else if (total >= h->prm.max_iters) { result = PS_ERR_NOT_CONVERGED; done = true; }
      else { S.restarts++; fresh_cycle = true; }
      return PS_OK;
    }
    ++total;
    const double est = h->hsc[5], hn = h->hsc[6];
    {
      float a = 0, b = 0, c = 0;
      cudaEventElapsedTime(&a, h->ev[0], h->ev[1]);
      cudaEventElapsedTime(&b, h->ev[1], h->ev[2]);
      cudaEventElapsedTime(&c, h->ev[2], h->ev[3]);
      S.ms_prec += a; S.ms_spmv += b; S.ms_orth += c;
      float f[4] = {0, 0, 0, 0};
      for (int q = 0; q < 4; ++q) cudaEventElapsedTime(&f[q], h->fe[q], h->fe[q + 1]);
      S.ms_vcycle_u += f[0]; S.ms_flow24 += f[1]; S.ms_vcycle_p += f[2]; S.ms_ilu += f[3];
    }
    S.est_relres = est;
    jend = j;
    S.reorth += h->hflag[0];
    if (h->hflag[3] || h->hflag[2]) {
      const bool wave = h->hflag[3] != 0;
      if (h->hflag[3]) PS_CUDA(cudaMemsetAsync(h->F.ilu_err, 0, sizeof(int), st));
      if (h->hflag[2]) {
        // the barrier counter is left mid-count: start it again from zero
        PS_CUDA(cudaMemsetAsync(K.flag + 2, 0, sizeof(int), st));
        PS_CUDA(cudaMemsetAsync(h->mgs_bar, 0, sizeof(unsigned long long), st));
        h->mgs_base = 0;
      }
      set_reason(wave ? "a bounded wait of the wavefront ILU(0) sweep or of a V-cycle grid barrier gave up"
                      : "a bounded grid barrier wait of the Gram-Schmidt step gave up");
      result = PS_ERR_TIMEOUT;
      S.iters = total;
      done = true;
      return PS_OK;
    }
    if (h->hflag[1]) { result = PS_ERR_NAN; S.iters = total; done = true; return PS_OK; }
    if (!(hn > 1e-300 * bnorm)) brk = true;
    if (est <= tol || brk || total >= h->prm.max_iters || j == h->m - 1) cycle_end = true;
    else ++j;
    return PS_OK;
  }

  // x out, timings, stats (synchronises the stream)
  ps_status finish(ps_stats* stats) {
    cudaStream_t st = h->st;
    const bool host = h->prm.host_ptrs != 0;
    PS_CUDA(cudaMemcpyAsync(x, h->x, sizeof(double) * h->n, host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                            st));
    cudaEventRecord(e1, st);
    PS_CUDA(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&S.ms_solve, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    e0 = e1 = nullptr;
    S.ms_setup_u = h->ms_setup_u;
    S.ms_setup_f = h->ms_setup_f;
    S.ms_copy_in = h->ms_copy_in;
  S.ms_copy_in = h->ms_copy_in;
    S.handle_bytes = h->ar.bytes + h->arf.bytes;
    S.levels_u = int32_t(h->rbm ? h->rbm_u.L.size() : h->amg_u.L.size());
    S.levels_p = int32_t(h->amg_p.L.size());
    if (stats) *stats = S;
    return result;
  }
};

}  // namespace

extern "C" {

ps_status ps_solve(ps_handle* h, const double* rhs, double* x, double tol, ps_stats* stats) {
  if (!h || !rhs || !x || !(tol > 0.0)) return PS_ERR_INVALID;
  if (h->prm.solver == PS_SOLVER_RICHARDSON) return solve_richardson(h, rhs, x, tol, stats);
  FgmresRun run;
  PS_TRY(run.start(h, rhs, x, tol));
  while (!run.done) {
    PS_TRY(run.enqueue());
    PS_CUDA(cudaStreamSynchronize(h->st));
    PS_TRY(run.after_sync());
  }
  return run.finish(stats);
}

int32_t ps_amg_nlevels(ps_handle* h, int32_t which) {
  if (!h) return 0;
  return int32_t((which == 0 ? h->amg_u : h->amg_p).L.size());
}

ps_status ps_amg_level_info(ps_handle* h, int32_t which, int32_t level, int64_t* n, int64_t* nnz, int64_t* nagg) {
  if (!h) return PS_ERR_INVALID;
  Amg& A = which == 0 ? h->amg_u : h->amg_p;
  if (level < 0 || level >= int32_t(A.L.size())) return PS_ERR_INVALID;
  if (n) *n = A.L[level].n;
  if (nnz) *nnz = A.L[level].nnz;
  if (nagg) *nagg = A.L[level].nagg;
  return PS_OK;
}

ps_status ps_amg_level_shape(ps_handle* h, int32_t which, int32_t level, int64_t* shape) {
  if (!h || !shape) return PS_ERR_INVALID;
  Amg& A = which == 0 ? h->amg_u : h->amg_p;
  if (level < 0 || level >= int32_t(A.L.size())) return PS_ERR_INVALID;
  const AmgLevel& L = A.L[level];
  const bool st = h->mixed ? L.sv_f != nullptr : L.sv_d != nullptr;
  shape[0] = L.n;
  shape[1] = L.nnz;
  shape[2] = L.coarsest ? 0 : L.nagg;
  shape[3] = L.coarsest ? 0 : L.pnnz;
  shape[4] = st ? L.sns : 0;
  shape[5] = h->mixed ? 4 : 8;
  shape[6] = h->bf16p && L.pvb ? 2 : (h->mixed ? 4 : 8);
  shape[7] = L.coarsest ? 1 : 0;
  return PS_OK;
}

ps_status ps_amg_level_copy(ps_handle* h, int32_t which, int32_t level, int64_t* rowptr, int32_t* colind,
                            double* val, int32_t* agg) {
  if (!h) return PS_ERR_INVALID;
  Amg& A = which == 0 ? h->amg_u : h->amg_p;
  if (level < 0 || level >= int32_t(A.L.size())) return PS_ERR_INVALID;
  AmgLevel& L = A.L[level];
  cudaStream_t st = h->st;
  if (rowptr) {
    int64_t* tmp;
    PS_TRY(h->ar.alloc(&tmp, L.n + 1));
    PS_TICK(); k_i32_to_i64<<<grid_for(L.n + 1, 256), 256, 0, st>>>(L.rp, tmp, L.n + 1);
    PS_CUDA(cudaMemcpyAsync(rowptr, tmp, sizeof(int64_t) * (L.n + 1), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    h->ar.release(tmp);
  }
  if (colind) PS_CUDA(cudaMemcpyAsync(colind, L.ci, sizeof(int32_t) * L.nnz, cudaMemcpyDeviceToHost, st));
  if (val) PS_CUDA(cudaMemcpyAsync(val, L.v, sizeof(double) * L.nnz * A.nc, cudaMemcpyDeviceToHost, st));
  if (agg) {
    if (L.agg) PS_CUDA(cudaMemcpyAsync(agg, L.agg, sizeof(int32_t) * L.n, cudaMemcpyDeviceToHost, st));
    else for (int64_t i = 0; i < L.n; ++i) agg[i] = -1;
  }
  PS_CUDA(cudaStreamSynchronize(st));
  return PS_OK;
}

int32_t ps_rbm_nlevels(ps_handle* h) { return h && h->rbm ? int32_t(h->rbm_u.L.size()) : 0; }

ps_status ps_rbm_level_shape(ps_handle* h, int32_t level, int64_t* shape) {
  if (!h || !h->rbm || !shape || level < 0 || level >= int32_t(h->rbm_u.L.size())) return PS_ERR_INVALID;
  const RbmLevel& L = h->rbm_u.L[level];
  shape[0] = L.n; shape[1] = L.b; shape[2] = L.nnzb; shape[3] = L.coarsest ? 0 : L.nagg;
  shape[4] = L.coarsest ? 0 : L.pnnzb; shape[5] = L.coarsest ? 1 : 0;
  return PS_OK;
}

namespace {
ps_status copy_rowptr(ps_handle* h, const int32_t* rp, int64_t n, int64_t* out) {
  int64_t* tmp;
  PS_TRY(h->ar.alloc(&tmp, n + 1));
  PS_TICK(); k_i32_to_i64<<<grid_for(n + 1, 256), 256, 0, h->st>>>(rp, tmp, n + 1);
  PS_CUDA(cudaMemcpyAsync(out, tmp, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, h->st));
  PS_CUDA(cudaStreamSynchronize(h->st));
  h->ar.release(tmp);
  return PS_OK;
}
}  // namespace

ps_status ps_rbm_level_copy(ps_handle* h, int32_t level, int64_t* rowptr, int32_t* colind, double* val,
                            int32_t* agg) {
  if (!h || !h->rbm || level < 0 || level >= int32_t(h->rbm_u.L.size())) return PS_ERR_INVALID;
  const RbmLevel& L = h->rbm_u.L[level];
  cudaStream_t st = h->st;
  if (rowptr) PS_TRY(copy_rowptr(h, L.rp, L.n, rowptr));
  if (colind) PS_CUDA(cudaMemcpyAsync(colind, L.ci, sizeof(int32_t) * L.nnzb, cudaMemcpyDeviceToHost, st));
  if (val) PS_CUDA(cudaMemcpyAsync(val, L.v, sizeof(double) * L.nnzb * L.b * L.b, cudaMemcpyDeviceToHost, st));
  if (agg) {
    if (L.agg && !L.coarsest) PS_CUDA(cudaMemcpyAsync(agg, L.agg, sizeof(int32_t) * L.n, cudaMemcpyDeviceToHost, st));
    else for (int64_t i = 0; i < L.n; ++i) agg[i] = -1;
  }
  PS_CUDA(cudaStreamSynchronize(st));
  return PS_OK;
}

ps_status ps_rbm_prolongator_copy(ps_handle* h, int32_t level, int64_t* rowptr, int32_t* colind, double* val) {
  if (!h || !h->rbm || level < 0 || level >= int32_t(h->rbm_u.L.size()) || h->rbm_u.L[level].coarsest)
    return PS_ERR_INVALID;
  const RbmLevel& L = h->rbm_u.L[level];
  cudaStream_t st = h->st;
  if (rowptr) PS_TRY(copy_rowptr(h, L.prp, L.n, rowptr));
  if (colind) PS_CUDA(cudaMemcpyAsync(colind, L.pci, sizeof(int32_t) * L.pnnzb, cudaMemcpyDeviceToHost, st));
  if (val)
    PS_CUDA(cudaMemcpyAsync(val, L.pv, sizeof(double) * L.pnnzb * L.b * kRbmModes, cudaMemcpyDeviceToHost, st));
  PS_CUDA(cudaStreamSynchronize(st));
  return PS_OK;
}

ps_status ps_flow_copy(ps_handle* h, double* spp, double* dinv) {
  if (!h) return PS_ERR_INVALID;
  if (spp) PS_CUDA(cudaMemcpyAsync(spp, h->F.spp, sizeof(double) * h->F.nnzb, cudaMemcpyDeviceToHost, h->st));
  if (dinv) PS_CUDA(cudaMemcpyAsync(dinv, h->F.dinv, sizeof(double) * 4 * h->nc, cudaMemcpyDeviceToHost, h->st));
  PS_CUDA(cudaStreamSynchronize(h->st));
  return PS_OK;
}

void ps_free(ps_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  amg_release_graph(h->amg_u);
  amg_release_graph(h->amg_p);
  rbm_release_graph(h->rbm_u);
  h->arf.free_all();
  h->ar.free_all();
  cudaStreamSynchronize(h->st);
  for (int e = 0; e < 4; ++e)
    if (h->ev[e]) cudaEventDestroy(h->ev[e]);
  for (int e = 0; e < 5; ++e)
    if (h->fe[e]) cudaEventDestroy(h->fe[e]);
  if (h->hsc) cudaFreeHost(h->hsc);
  if (h->hflag) cudaFreeHost(h->hflag);
  if (h->own_stream && h->st) cudaStreamDestroy(h->st);
  delete h;
}

ps_status ps_setup_batch(int32_t n, const ps_jacobian* jac, const ps_grid* grid, const ps_params* params,
                         ps_handle** out) {
  if (n < 0 || (n > 0 && (!jac || !grid || !params || !out))) return PS_ERR_INVALID;
  for (int32_t i = 0; i < n; ++i) out[i] = nullptr;
  std::vector<ps_status> st(n, PS_OK);
  std::atomic<int32_t> next{0};
  auto worker = [&]() {
    int dev = 0;
    cudaGetDevice(&dev);
    for (;;) {
      const int32_t i = next.fetch_add(1);
      if (i >= n) return;
      cudaStream_t s = nullptr;
      if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        st[i] = PS_ERR_CUDA;
        continue;
      }
      ps_params p = *params;
      p.stream = s;
      st[i] = ps_setup(&jac[i], &grid[i], &p, &out[i]);
      if (st[i] == PS_OK) out[i]->own_stream = true;
      else cudaStreamDestroy(s);
    }
  };
  int dev = 0;
  PS_CUDA(cudaGetDevice(&dev));
  const int nthreads = std::min<int32_t>(n, 8);
  std::vector<std::thread> pool;
  for (int t = 0; t < nthreads; ++t)
    pool.emplace_back([&, dev]() {
      cudaSetDevice(dev);
      worker();
    });
  for (auto& t : pool) t.join();
  for (int32_t i = 0; i < n; ++i)
    if (st[i] != PS_OK) {
      for (int32_t k = 0; k < n; ++k) {
        ps_free(out[k]);
        out[k] = nullptr;
      }
      return st[i];
    }
  return PS_OK;
}

ps_status ps_solve_batch(int32_t n, ps_handle* const* h, const double* const* rhs, double* const* x, double tol,
                         ps_stats* stats) {
  if (n < 0 || (n > 0 && (!h || !rhs || !x)) || !(tol > 0.0)) return PS_ERR_INVALID;
  for (int32_t i = 0; i < n; ++i)
    if (!h[i] || !rhs[i] || !x[i]) return PS_ERR_INVALID;
  std::vector<ps_status> res(n, PS_OK);
  std::vector<FgmresRun> runs(n);
  // systems are dealt round-robin to up to eight host threads; each thread advances its group in lockstep,
  // one step of every unfinished system per round and one synchronisation per round, so the launch work of
  // the groups proceeds in parallel
  const int nthreads = std::min<int32_t>(n, 8);
  int dev = 0;
  PS_CUDA(cudaGetDevice(&dev));
  auto group = [&](int t) -> void {
    cudaSetDevice(dev);
    std::vector<int32_t> mine;
    for (int32_t i = t; i < n; i += nthreads) {
      if (h[i]->prm.solver == PS_SOLVER_RICHARDSON) {
        res[i] = ps_solve(h[i], rhs[i], x[i], tol, stats ? &stats[i] : nullptr);
        continue;
      }
      res[i] = runs[i].start(h[i], rhs[i], x[i], tol);
      if (res[i] == PS_OK) mine.push_back(i);
    }
    std::vector<char> failed(n, 0);
    for (;;) {
      bool any = false;
      for (int32_t i : mine)
        if (!runs[i].done && !failed[i]) {
          ps_status e = runs[i].enqueue();
          if (e != PS_OK) { res[i] = e; failed[i] = 1; continue; }
          any = true;
        }
      if (!any) break;
      for (int32_t i : mine)
        if (!runs[i].done && !failed[i]) {
          cudaError_t ce = cudaStreamSynchronize(h[i]->st);
          if (ce != cudaSuccess) { set_last_error(ce, "cudaStreamSynchronize", __FILE__, __LINE__); res[i] = PS_ERR_CUDA; failed[i] = 1; continue; }
          ps_status e = runs[i].after_sync();
          if (e != PS_OK) { res[i] = e; failed[i] = 1; }
        }
    }
    for (int32_t i : mine) {
      ps_status e = runs[i].finish(stats ? &stats[i] : nullptr);
      if (!failed[i]) res[i] = e;
    }
  };
  std::vector<std::thread> pool;
  for (int t = 0; t < nthreads; ++t) pool.emplace_back(group, t);
  for (auto& th : pool) th.join();
  for (int32_t i = 0; i < n; ++i)
    if (res[i] != PS_OK) return res[i];
  return PS_OK;
}

const char* ps_strerror(ps_status s) {
  switch (s) {
    case PS_OK: return "ok";
    case PS_ERR_INVALID:
      return ps_internal::last_reason().empty() ? "invalid argument, shape or pattern" : ps_internal::last_reason().c_str();
    case PS_ERR_OOM: return "device out of memory";
    case PS_ERR_CUDA: return ps_internal::last_error().empty() ? "CUDA error" : ps_internal::last_error().c_str();
    case PS_ERR_NOT_CONVERGED: return "not converged within max_iters";
    case PS_ERR_BREAKDOWN: return "Krylov breakdown before convergence";
    case PS_ERR_NAN: return "NaN or Inf encountered";
    case PS_ERR_TIMEOUT:
      return ps_internal::last_reason().empty() ? "bounded device wait timed out" : ps_internal::last_reason().c_str();
    case PS_ERR_BUDGET: return "HBM budget exceeded";
  }
  return "unknown status";
}

}  // extern "C"
