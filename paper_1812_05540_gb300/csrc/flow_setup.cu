// Flow-stage setup.  Compiled without floating-point contraction: S_pp feeds
// the pressure aggregation, so its entries are formed with exactly the
// operations of the reduction formula, in that order.
#include "flow.cuh"

namespace ps_internal {
namespace {

__device__ __forceinline__ void mul22(const double* a, const double* b, double* c) {
  double c0 = a[0] * b[0] + a[1] * b[2], c1 = a[0] * b[1] + a[1] * b[3];
  double c2 = a[2] * b[0] + a[3] * b[2], c3 = a[2] * b[1] + a[3] * b[3];
  c[0] = c0; c[1] = c1; c[2] = c2; c[3] = c3;
}
__device__ __forceinline__ void inv22(const double* a, double* r) {
  double det = a[0] * a[3] - a[1] * a[2];
  r[0] = a[3] / det; r[1] = -a[1] / det; r[2] = -a[2] / det; r[3] = a[0] / det;
}

// the A_ff pattern must be the 7-point TPFA stencil of the grid in natural order
__global__ void k_check7(int nx, int ny, int nz, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                         int* __restrict__ bad) {
  int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  int64_t nc = int64_t(nx) * ny * nz;
  if (c >= nc) return;
  int i = int(c % nx), j = int((c / nx) % ny), k = int(c / (int64_t(nx) * ny));
  int64_t nxy = int64_t(nx) * ny;
  int64_t want[7];
  int m = 0;
  if (k > 0) want[m++] = c - nxy;
  if (j > 0) want[m++] = c - nx;
  if (i > 0) want[m++] = c - 1;
  want[m++] = c;
  if (i + 1 < nx) want[m++] = c + 1;
  if (j + 1 < ny) want[m++] = c + nx;
  if (k + 1 < nz) want[m++] = c + nxy;
  if (rp[c + 1] - rp[c] != m) { atomicExch(bad, 1); return; }
  for (int t = 0; t < m; ++t)
    if (ci[rp[c] + t] != want[t]) { atomicExch(bad, 1); return; }
}

// S_ff^(FS) = A_ff + [[0 D_sp] [0 D_pp]] on the diagonal (§5.1);
// quasi-IMPES: d_ss = (A_ss)_ii, d_ps = (A_ps)_ii; true-IMPES: d_ss = (A_ss^T e)_i, d_ps = (A_ps^T e)_i, the
// column sums taken over the rows in ascending order (the 7-point pattern is structurally symmetric, so
// the rows of column c are the columns of row c); S_pp = A_pp^(FS) - (d_ps/d_ss) A_sp^(FS) (§5.3)
__global__ void k_sff_spp(int64_t nc, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const double* __restrict__ aff, const double* __restrict__ dfs, double* __restrict__ sff,
                          double* __restrict__ spp, double* __restrict__ dss, double* __restrict__ dps,
                          double* __restrict__ aps, int32_t* __restrict__ diagpos, int true_impes) {
  int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  int32_t qd = rp[c];
  while (ci[qd] != c) ++qd;
  diagpos[c] = qd;
  double s = aff[int64_t(qd) * 4 + 0], ps = aff[int64_t(qd) * 4 + 2];
  if (true_impes) {
    s = 0.0;
    ps = 0.0;
    for (int32_t q = rp[c]; q < rp[c + 1]; ++q) {
      const int32_t r = ci[q];
      int32_t qr = rp[r];
      while (ci[qr] != c) ++qr;
      s = s + aff[int64_t(qr) * 4 + 0];
      ps = ps + aff[int64_t(qr) * 4 + 2];
    }
  }
  dss[c] = s;
  dps[c] = ps;
  double ratio = ps / s;
  for (int32_t q = rp[c]; q < rp[c + 1]; ++q) {
    double b0 = aff[int64_t(q) * 4 + 0], b1 = aff[int64_t(q) * 4 + 1];
    double b2 = aff[int64_t(q) * 4 + 2], b3 = aff[int64_t(q) * 4 + 3];
    if (q == qd) {
      b1 = b1 + dfs[2 * c];
      b3 = b3 + dfs[2 * c + 1];
    }
    sff[int64_t(q) * 4 + 0] = b0; sff[int64_t(q) * 4 + 1] = b1;
    sff[int64_t(q) * 4 + 2] = b2; sff[int64_t(q) * 4 + 3] = b3;
    spp[q] = b3 - ratio * b1;
    aps[q] = b2;
  }
}

__global__ void k_level_count(int nx, int ny, int nz, int32_t* __restrict__ cnt) {
  int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  int64_t nc = int64_t(nx) * ny * nz;
  if (c >= nc) return;
  int i = int(c % nx), j = int((c / nx) % ny), k = int(c / (int64_t(nx) * ny));
  atomicAdd(&cnt[i + j + k], 1);
}
__global__ void k_level_fill(int nx, int ny, int nz, int32_t* __restrict__ cursor, int32_t* __restrict__ cells) {
  int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  int64_t nc = int64_t(nx) * ny * nz;
  if (c >= nc) return;
  int i = int(c % nx), j = int((c / nx) % ny), k = int(c / (int64_t(nx) * ny));
  cells[atomicAdd(&cursor[i + j + k], 1)] = int32_t(c);
}

// Block ILU(0) of S_ff^(FS) in natural order, one wavefront level: with the
// 7-point stencil no two lower neighbours of a cell are coupled, so the IKJ
// elimination only updates the diagonal block:
//   U_ii = S_ii - sum_{k<i} (S_ik inv(U_kk)) S_ki   (k ascending)
// Processor-local scope (local != 0): lower neighbours in another sweep tile are left out, which is the
// ILU(0) of S_ff^(FS) without the blocks that couple different tiles.
__global__ void k_ilu_factor(const int32_t* __restrict__ cells, int32_t ncell_lev, const int32_t* __restrict__ rp,
                             const int32_t* __restrict__ ci, const int32_t* __restrict__ diagpos,
                             const double* __restrict__ sff, double* __restrict__ dinv, int nx, int ny, int local) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ncell_lev) return;
  int32_t i = cells[t];
  int32_t qd = diagpos[i];
  double D[4] = {sff[int64_t(qd) * 4], sff[int64_t(qd) * 4 + 1], sff[int64_t(qd) * 4 + 2], sff[int64_t(qd) * 4 + 3]};
  for (int32_t q = rp[i]; q < qd; ++q) {
    int32_t k = ci[q];
    if (local && cross_tile(i, k, nx, ny)) continue;
    double L[4], U[4];
    mul22(&sff[int64_t(q) * 4], &dinv[int64_t(k) * 4], L);
    // (k, i) is the upper block of row k
    int32_t qk = diagpos[k] + 1;
    while (ci[qk] != i) ++qk;
    mul22(L, &sff[int64_t(qk) * 4], U);
    for (int e = 0; e < 4; ++e) D[e] -= U[e];
  }
  inv22(D, &dinv[int64_t(i) * 4]);
}

// Processor-local ILU(0) factor in one launch: CTA t factors the cells of sweep tile t (its own subdomain) in
// the forward sweep's wavefront order, thread (ly, lz) taking pencil position x = s - ly - lz at step s, so a
// cell's lower neighbours in the tile were factored at earlier steps; one barrier per step.  Each cell runs
// the arithmetic of k_ilu_factor with local != 0, so the factors are the same bits.
__global__ void __launch_bounds__(kTY * kTZ) k_ilu_factor_tiles(int nx, int ny, int nz, const int32_t* __restrict__ rp,
                                                                const int32_t* __restrict__ ci,
                                                                const int32_t* __restrict__ diagpos,
                                                                const double* __restrict__ sff, double* __restrict__ dinv) {
  const int nby = (ny + kTY - 1) / kTY;
  const int ly = threadIdx.x % kTY, lz = threadIdx.x / kTY;
  const int yy = (blockIdx.x % nby) * kTY + ly, zz = (blockIdx.x / nby) * kTZ + lz;
  const bool valid = yy < ny && zz < nz;
  const int last = nx + kTY + kTZ - 3;
  for (int s = 0; s <= last; ++s) {
    const int x = s - ly - lz;
    if (valid && x >= 0 && x < nx) {
      const int32_t i = int32_t(x + int64_t(nx) * (yy + int64_t(ny) * zz));
      const int32_t qd = diagpos[i];
      double D[4] = {sff[int64_t(qd) * 4], sff[int64_t(qd) * 4 + 1], sff[int64_t(qd) * 4 + 2], sff[int64_t(qd) * 4 + 3]};
      for (int32_t q = rp[i]; q < qd; ++q) {
        const int32_t k = ci[q];
        if (cross_tile(i, k, nx, ny)) continue;
        double L[4], U[4];
        mul22(&sff[int64_t(q) * 4], &dinv[int64_t(k) * 4], L);
        int32_t qk = diagpos[k] + 1;
        while (ci[qk] != i) ++qk;
        mul22(L, &sff[int64_t(qk) * 4], U);
        for (int e = 0; e < 4; ++e) D[e] -= U[e];
      }
      inv22(D, &dinv[int64_t(i) * 4]);
    }
    __syncthreads();
  }
}

// S_ff^(FS) by stencil slot (the row of a 7-point pattern is z-1, y-1, x-1, self, x+1, y+1, z+1 with
// the missing neighbours left out), 28 entries per cell
__global__ void k_s28(int nx, int ny, int nz, const int32_t* __restrict__ rp, const double* __restrict__ sff,
                      double* __restrict__ out) {
  int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  int64_t nc = int64_t(nx) * ny * nz;
  if (c >= nc) return;
  int i = int(c % nx), j = int((c / nx) % ny), k = int(c / (int64_t(nx) * ny));
  const bool have[7] = {k > 0, j > 0, i > 0, true, i + 1 < nx, j + 1 < ny, k + 1 < nz};
  int32_t q = rp[c];
  for (int s = 0; s < 7; ++s) {
    for (int e = 0; e < 4; ++e) out[c * 28 + s * 4 + e] = have[s] ? sff[int64_t(q) * 4 + e] : 0.0;
    if (have[s]) ++q;
  }
}

// Block Gauss-Seidel records (§5.3 option 1): per colour slot p, the face blocks of S_ff^(FS) in slot order
// (z-1, y-1, x-1, x+1, y+1, z+1; zero outside the grid) and inv(S_ii), 28 values, blocked by 32 slots.
// Empty slots (odd nx) keep zeros.
template <class T>
__global__ void k_gs_pack(int nx, int ny, int nz, int col, const double* __restrict__ s28, T* __restrict__ rec) {
  const int hx = gs_hx(nx);
  const int64_t ncp = int64_t(nz) * ny * hx;
  int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= ncp) return;
  const int m = int(p % hx);
  const int64_t row = p / hx;
  const int y = int(row % ny), z = int(row / ny);
  const int x = 2 * m + ((col + y + z) & 1);
  T* R = rec + (((int64_t(col) * ((ncp + 31) / 32)) + (p >> 5)) * 28) * 32 + (p & 31);
  if (x >= nx) {
    for (int v = 0; v < 28; ++v) R[v * 32] = T(0);
    return;
  }
  const int64_t c = x + int64_t(nx) * (y + int64_t(ny) * z);
  const double* S = s28 + c * 28;
  const int slot[6] = {0, 1, 2, 4, 5, 6};
  for (int q = 0; q < 6; ++q)
    for (int e = 0; e < 4; ++e) R[(q * 4 + e) * 32] = T(S[slot[q] * 4 + e]);
  double D[4];
  inv22(S + 12, D);
  for (int e = 0; e < 4; ++e) R[(24 + e) * 32] = T(D[e]);
}

// A_ps by 7-point slot, blocked by 32 cells, from the stencil blocks of S_ff^(FS) (the fixed-stress
// terms change only the (s, p) and (p, p) entries, so entry (p, s) is A_ps)
template <class T>
__global__ void k_aps_st(int64_t nc, const T* __restrict__ s28, T* __restrict__ out) {
  int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  for (int q = 0; q < 7; ++q) out[((c >> 5) * 7 + q) * 32 + (c & 31)] = s28[c * 28 + q * 4 + 2];
}

// S/inv(U_ii) part of the sweep records (see FlowStage): forward lower blocks, backward upper blocks; with
// the processor-local scope the blocks towards another tile are zero
template <class T>
__global__ void k_pack_sd(int nx, int ny, int nz, int steps, const T* __restrict__ s28, const T* __restrict__ dinv,
                          T* __restrict__ pf, T* __restrict__ pb, int local) {
  int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (c >= int64_t(nx) * ny * nz) return;
  const int x = int(c % nx), y = int((c / nx) % ny), z = int(c / (int64_t(nx) * ny));
  T* f = pf + sweep_rec(true, nx, ny, steps, x, y, z);
  T* b = pb + sweep_rec(false, nx, ny, steps, x, y, z);
  // forward slots z-1, y-1, x-1; backward slots x+1, y+1, z+1
  const bool fkeep[3] = {!local || z % kTZ != 0, !local || y % kTY != 0, true};
  const bool bkeep[3] = {true, !local || y % kTY != kTY - 1, !local || z % kTZ != kTZ - 1};
  for (int e = 0; e < 12; ++e) {
    f[e] = fkeep[e / 4] ? s28[c * 28 + e] : T(0);
    b[e] = bkeep[e / 4] ? s28[c * 28 + 16 + e] : T(0);
  }
  for (int e = 0; e < 4; ++e) {
    f[12 + e] = dinv[c * 4 + e];
    b[12 + e] = dinv[c * 4 + e];
  }
}

__global__ void k_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < n) b[t] = float(a[t]);
}

}  // namespace

ps_status flow_check_pattern(Arena& ar, const ps_grid& g, const int32_t* ff_rp, const int32_t* ff_ci,
                             cudaStream_t st) {
  int* bad;
  PS_TRY(ar.alloc(&bad, 1));
  PS_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
  int64_t nc = int64_t(g.nx) * g.ny * g.nz;
  PS_TICK(); k_check7<<<grid_for(nc, 256), 256, 0, st>>>(g.nx, g.ny, g.nz, ff_rp, ff_ci, bad);
  int h = 0;
  PS_CUDA(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  PS_CUDA(cudaStreamSynchronize(st));
  ar.release(bad);
  return h ? PS_ERR_INVALID : PS_OK;
}

ps_status flow_setup(Arena& ar, FlowStage& F, const int32_t* ff_rp, const int32_t* ff_ci, const double* ff_v,
                     const double* d_fs, bool mixed, cudaStream_t st) {
  int64_t nc = F.nc, nnzb = F.nnzb;
  if (!F.sff) {
    PS_TRY(ar.alloc(&F.sff, nnzb * 4));
    PS_TRY(ar.alloc(&F.spp, nnzb));
    PS_TRY(ar.alloc(&F.aps, nnzb));
    PS_TRY(ar.alloc(&F.dss, nc));
    PS_TRY(ar.alloc(&F.dps, nc));
    PS_TRY(ar.alloc(&F.dinv, nc * 4));
    PS_TRY(ar.alloc(&F.diagpos, nc));
    PS_TRY(ar.alloc(&F.s28, nc * 28));
    PS_TRY(ar.alloc(&F.ilu_err, 4));  // bounded-wait error flag, read after every iteration in both local modes
    PS_CUDA(cudaMemsetAsync(F.ilu_err, 0, 4 * sizeof(int), st));
    if (mixed) {
      PS_TRY(ar.alloc(&F.s28_f, nc * 28));
      PS_TRY(ar.alloc(&F.sff_f, nnzb * 4));
      PS_TRY(ar.alloc(&F.aps_f, nnzb));
      PS_TRY(ar.alloc(&F.dinv_f, nc * 4));
      PS_TRY(ar.alloc(&F.dss_f, nc));
    }
    if (F.local == PS_LOCAL_HBGS) {
      F.gs_ncp = int64_t(F.nz) * F.ny * gs_hx(F.nx);
      const size_t nrec = size_t(2) * ((F.gs_ncp + 31) / 32) * 28 * 32;
      if (mixed) PS_TRY(ar.alloc(&F.gs_rec_f, nrec));
      else PS_TRY(ar.alloc(&F.gs_rec_d, nrec));
    }
  }
  if (F.local != PS_LOCAL_HBGS && !F.halo) {
    // wavefront levels
    F.nlev = F.nx + F.ny + F.nz - 2;
    int32_t *cnt, *off, *cursor;
    PS_TRY(ar.alloc(&cnt, F.nlev + 1));
    PS_TRY(ar.alloc(&off, F.nlev + 1));
    PS_TRY(ar.alloc(&cursor, F.nlev + 1));
    PS_TRY(ar.alloc(&F.lev_cells, nc));
    PS_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (F.nlev + 1), st));
    PS_TICK(); k_level_count<<<grid_for(nc, 256), 256, 0, st>>>(F.nx, F.ny, F.nz, cnt);
    PS_TRY(scan_i32(ar, cnt, off, F.nlev, nullptr, st));
    PS_CUDA(cudaMemcpyAsync(cursor, off, sizeof(int32_t) * F.nlev, cudaMemcpyDeviceToDevice, st));
    PS_TICK(); k_level_fill<<<grid_for(nc, 256), 256, 0, st>>>(F.nx, F.ny, F.nz, cursor, F.lev_cells);
    // sweep records, [tile][step][thread][kRec]; slots of cells outside the grid stay zero
    F.pk_steps = sweep_steps(F.nx, mixed ? win_cells<float>() : win_cells<double>());
    const size_t nrec = size_t(sweep_tiles(F.ny, F.nz)) * F.pk_steps * (kTY * kTZ) * kRec;
    if (mixed) {
      PS_TRY(ar.alloc(&F.pk_fwd_f, nrec));
      PS_TRY(ar.alloc(&F.pk_bwd_f, nrec));
      PS_CUDA(cudaMemsetAsync(F.pk_fwd_f, 0, sizeof(float) * nrec, st));
      PS_CUDA(cudaMemsetAsync(F.pk_bwd_f, 0, sizeof(float) * nrec, st));
    } else {
      PS_TRY(ar.alloc(&F.pk_fwd_d, nrec));
      PS_TRY(ar.alloc(&F.pk_bwd_d, nrec));
      PS_CUDA(cudaMemsetAsync(F.pk_fwd_d, 0, sizeof(double) * nrec, st));
      PS_CUDA(cudaMemsetAsync(F.pk_bwd_d, 0, sizeof(double) * nrec, st));
    }
    PS_TRY(ar.alloc(&F.halo, size_t(nc) * 4));
    PS_CUDA(cudaMemsetAsync(F.halo, 0, sizeof(uint64_t) * nc * 4, st));
    F.lev_off.resize(F.nlev + 1);
    PS_CUDA(cudaMemcpyAsync(F.lev_off.data(), off, sizeof(int32_t) * (F.nlev + 1), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    ar.release(cnt); ar.release(off); ar.release(cursor);
  }
  PS_TICK(); k_sff_spp<<<grid_for(nc, 256), 256, 0, st>>>(nc, ff_rp, ff_ci, ff_v, d_fs, F.sff, F.spp, F.dss, F.dps, F.aps,
                                               F.diagpos, F.cpr == PS_CPR_TRUE_IMPES);
  if (F.local != PS_LOCAL_HBGS && F.ilu_local) {
    // processor-local: the tiles are independent, one CTA each
    PS_TICK(); k_ilu_factor_tiles<<<unsigned(sweep_tiles(F.ny, F.nz)), kTY * kTZ, 0, st>>>(F.nx, F.ny, F.nz, F.rp, F.ci,
                                                                                         F.diagpos, F.sff, F.dinv);
  } else {
    for (int l = 0; l < (F.local == PS_LOCAL_HBGS ? 0 : F.nlev); ++l) {
      int32_t m = F.lev_off[l + 1] - F.lev_off[l];
      PS_TICK(); k_ilu_factor<<<grid_for(m, 128), 128, 0, st>>>(F.lev_cells + F.lev_off[l], m, F.rp, F.ci, F.diagpos,
                                                                 F.sff, F.dinv, F.nx, F.ny, F.ilu_local);
    }
  }
  PS_TICK(); k_s28<<<grid_for(nc, 256), 256, 0, st>>>(F.nx, F.ny, F.nz, F.rp, F.sff, F.s28);
  PS_CUDA(cudaGetLastError());
  if (F.local == PS_LOCAL_HBGS) {
    for (int col = 0; col < 2; ++col) {
      if (mixed) { PS_TICK(); k_gs_pack<float><<<grid_for(F.gs_ncp, 256), 256, 0, st>>>(F.nx, F.ny, F.nz, col, F.s28, F.gs_rec_f); }
      else { PS_TICK(); k_gs_pack<double><<<grid_for(F.gs_ncp, 256), 256, 0, st>>>(F.nx, F.ny, F.nz, col, F.s28, F.gs_rec_d); }
    }
    PS_CUDA(cudaGetLastError());
  }
  if (mixed) {
    PS_TICK(); k_f32<<<grid_for(nc * 28, 256), 256, 0, st>>>(F.s28, F.s28_f, nc * 28);
    PS_TICK(); k_f32<<<grid_for(nnzb * 4, 256), 256, 0, st>>>(F.sff, F.sff_f, nnzb * 4);
    PS_TICK(); k_f32<<<grid_for(nnzb, 256), 256, 0, st>>>(F.aps, F.aps_f, nnzb);
    PS_TICK(); k_f32<<<grid_for(nc * 4, 256), 256, 0, st>>>(F.dinv, F.dinv_f, nc * 4);
    PS_TICK(); k_f32<<<grid_for(nc, 256), 256, 0, st>>>(F.dss, F.dss_f, nc);
    PS_CUDA(cudaGetLastError());
    if (F.pk_fwd_f) {
      PS_TICK(); k_pack_sd<float><<<grid_for(nc, 256), 256, 0, st>>>(F.nx, F.ny, F.nz, F.pk_steps, F.s28_f, F.dinv_f,
                                                                    F.pk_fwd_f, F.pk_bwd_f, F.ilu_local);
    }
    if (!F.aps_st_f) PS_TRY(ar.alloc(&F.aps_st_f, size_t((nc + 31) / 32) * 32 * 7));
    PS_TICK(); k_aps_st<float><<<grid_for(nc, 256), 256, 0, st>>>(nc, F.s28_f, F.aps_st_f);
  } else {
    if (F.pk_fwd_d) {
      PS_TICK(); k_pack_sd<double><<<grid_for(nc, 256), 256, 0, st>>>(F.nx, F.ny, F.nz, F.pk_steps, F.s28, F.dinv,
                                                                     F.pk_fwd_d, F.pk_bwd_d, F.ilu_local);
    }
    if (!F.aps_st_d) PS_TRY(ar.alloc(&F.aps_st_d, size_t((nc + 31) / 32) * 32 * 7));
    PS_TICK(); k_aps_st<double><<<grid_for(nc, 256), 256, 0, st>>>(nc, F.s28, F.aps_st_d);
  }
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

}  // namespace ps_internal
