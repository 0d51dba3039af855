// Flow stage of the preconditioner: the fixed-stress Schur approximation
// S_ff^(FS) (§5.1), the quasi-IMPES reduction to S_pp (§5.3) and block ILU(0)
// of S_ff^(FS) in the interleaved (s, p) ordering (§5.3, option 2).
#pragma once
#include "internal.cuh"

namespace ps_internal {

// Tiles of the sync-free ILU(0) sweeps: CTA (BY, BZ) owns the x-pencils of a kTY x kTZ tile of (y, z),
// thread ly + kTY * lz the pencil (BY * kTY + ly, BZ * kTZ + lz).  At CTA step s a thread handles pencil
// position s - ry - rz, with (ry, rz) = (ly, lz) in the forward sweep and (kTY-1-ly, kTZ-1-lz) in the
// backward one (position p is x = p forward and x = nx - 1 - p backward), so a sweep takes
// nx + kTY + kTZ - 2 steps.  Each cell has one record of kRec values per sweep.  The records are stored
// in the order a CTA consumes them, [tile][step][thread][kRec], steps padded to whole copy windows, so
// that one bulk copy moves a whole window of a tile.
constexpr int kTY = PS_ILU_TILE_Y, kTZ = PS_ILU_TILE_Z, kRec = 20;
// processor-local ILU(0): face neighbours i and j lie in different subdomains (the sweep tiles above)
__host__ __device__ inline bool cross_tile(int64_t i, int64_t j, int nx, int ny) {
  const int64_t yi = (i / nx) % ny, zi = i / (int64_t(nx) * ny), yj = (j / nx) % ny, zj = j / (int64_t(nx) * ny);
  return yi / kTY != yj / kTY || zi / kTZ != zj / kTZ;
}
template <class T>
__host__ __device__ constexpr int win_cells() { return sizeof(T) == 4 ? 4 : 2; }  // steps per copy window
// records per thread and tile of one sweep (a whole number of windows)
__host__ __device__ inline int sweep_steps(int nx, int W) { return (nx + kTY + kTZ - 2 + W - 1) / W * W; }
__host__ __device__ inline int64_t sweep_tiles(int ny, int nz) {
  return int64_t((ny + kTY - 1) / kTY) * ((nz + kTZ - 1) / kTZ);
}
// offset (in values) of the record of cell (x, y, z) in the forward (fwd) or backward sweep
__host__ __device__ inline int64_t sweep_rec(bool fwd, int nx, int ny, int steps, int x, int y, int z) {
  const int nby = (ny + kTY - 1) / kTY;
  const int ly = y % kTY, lz = z % kTZ;
  const int s = fwd ? x + ly + lz : (nx - 1 - x) + (kTY - 1 - ly) + (kTZ - 1 - lz);
  const int64_t tile = (y / kTY) + int64_t(nby) * (z / kTZ);
  return ((tile * steps + s) * (kTY * kTZ) + ly + kTY * lz) * kRec;
}

// Block Gauss-Seidel colour slots: slot p of colour col is the cell (x, y, z) with
// x = 2 (p % hx) + ((col + y + z) & 1), y = (p / hx) % ny, z = p / (hx ny), hx = ceil(nx / 2); slots with
// x >= nx (odd nx) are empty.  Face neighbours always have the other colour.
__host__ __device__ inline int gs_hx(int nx) { return (nx + 1) / 2; }

struct FlowStage {
  int nx = 0, ny = 0, nz = 0;
  int64_t nc = 0, nnzb = 0;
  int32_t *rp = nullptr, *ci = nullptr;  // A_ff pattern (7-point), int32
  int32_t* diagpos = nullptr;            // position of the diagonal block per row
  double* sff = nullptr;                 // S_ff^(FS) blocks, 4 per entry, FP64
  double* spp = nullptr;                 // S_pp^(cpr-fs), 1 per entry, FP64
  double *dss = nullptr, *dps = nullptr; // quasi-IMPES diagonals
  double* dinv = nullptr;                // inv(U_ii) of block ILU(0), 4 per cell
  float *sff_f = nullptr, *aps_f = nullptr, *dinv_f = nullptr, *dss_f = nullptr;
  double* aps = nullptr;                 // A_ps entries (lower-left of each block), FP64
  // wavefront levels of the natural ordering (level = i + j + k)
  int nlev = 0;
  int32_t* lev_cells = nullptr;
  std::vector<int32_t> lev_off;          // host copy, nlev + 1
  // S_ff^(FS) indexed by stencil slot, 28 entries per cell (z-1, y-1, x-1, self, x+1, y+1, z+1; 2x2
  // row-major each), zero blocks outside the grid
  double* s28 = nullptr;
  float* s28_f = nullptr;
  // local stage: PS_LOCAL_ILU0 (the ILU(0) factors, sweep records and halo words below) or PS_LOCAL_HBGS
  // (block Gauss-Seidel: per colour, the six face blocks and inv(S_ii) of each cell, 28 values, blocked
  // by 32 cells, [colour][p / 32][28][p % 32] with p the cell's index within its colour; see gs_index)
  int local = 0;
  int ilu_local = 0;  // PS_ILU_LOCAL: no ILU(0) coupling between cells of different sweep tiles
  int cpr = 0;  // PS_CPR_QUASI_IMPES or PS_CPR_TRUE_IMPES
  int gs_sweeps = 3;
  int64_t gs_ncp = 0;  // slots per colour: nz * ny * ceil(nx / 2)
  float* gs_rec_f = nullptr;
  double* gs_rec_d = nullptr;
  // records of the sync-free sweeps, kRec values per cell (forward: lower blocks, inv(U_ii), w; backward:
  // upper blocks, inv(U_ii), t, z_s, z_p), in the apply precision, at sweep_rec(...) with
  // pk_steps = sweep_steps(nx, win_cells<T>())
  int pk_steps = 0;
  float *pk_fwd_f = nullptr, *pk_bwd_f = nullptr;
  double *pk_fwd_d = nullptr, *pk_bwd_d = nullptr;
  // sync-free wavefront sweeps: tagged halo words (4 per cell) and error flag
  uint64_t* halo = nullptr;
  int* ilu_err = nullptr;
  int64_t ilu_epoch = 0;
  int64_t spin_limit = 2000000;
  int test_stall = 0;
  // A_fu for Algorithm 1 step 2
  int32_t *fu_rp = nullptr, *fu_ci = nullptr;
  const double* fu_v = nullptr;
  float* fu_vf = nullptr;
  // stencil-slot copies for steps 2 and 4 (null when the patterns are not the structured ones): A_fu
  // by cell corner, blocked by 32 cells [cell / 32][8 corners][6][cell % 32]; A_ps by 7-point slot,
  // [cell / 32][7][cell % 32]; FP64 (the Jacobian's own stencil copy) and FP32
  const double* fu_st_d = nullptr;
  float* fu_st_f = nullptr;
  double* aps_st_d = nullptr;
  float* aps_st_f = nullptr;
};

// Build S_ff^(FS), S_pp, the level lists and the ILU(0) factors from the
// caller's FP64 A_ff / d_fs (device pointers, already int32 row pointers).
ps_status flow_setup(Arena& ar, FlowStage& F, const int32_t* ff_rp, const int32_t* ff_ci, const double* ff_v,
                     const double* d_fs, bool mixed, cudaStream_t st);
ps_status flow_check_pattern(Arena& ar, const ps_grid& g, const int32_t* ff_rp, const int32_t* ff_ci,
                             cudaStream_t st);

// Algorithm 1 steps 2-4 and 6-8 for precision T (pressure V-cycle in between,
// called by the driver).  v_f, y, z_s, w_p, t, dz are per-cell work vectors.
template <class T>
struct FlowWork {
  T *vf, *y, *zs, *wp, *zp, *t, *dz, *wf;
};
template <class T>
ps_status flow_alloc_work(Arena& ar, const FlowStage& F, FlowWork<T>& W);
template <class T>
void alg1_steps_2_4(const FlowStage& F, const FlowWork<T>& W, const T* zu, cudaStream_t st);
// steps 6-8: ILU(0) sweeps; writes z_f (interleaved, FP64) to zout
template <class T>
void alg1_steps_6_8(const FlowStage& F, const FlowWork<T>& W, double* zout, int ilu_mode, cudaStream_t st);

}  // namespace ps_internal
