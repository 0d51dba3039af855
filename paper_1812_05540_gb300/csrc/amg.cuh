// Smoothed-aggregation AMG hierarchy on the device: the amg(.) operator of
// §5.2 (three SDC displacement components on shared nodal aggregates, nc = 3)
// and §5.3 (pressure, nc = 1).
#pragma once
#include <cuda_bf16.h>

#include <vector>

#include "internal.cuh"

namespace ps_internal {

struct AmgLevel {
  int64_t n = 0, nnz = 0;
  int32_t* rp = nullptr;  // n+1
  int32_t* ci = nullptr;  // nnz
  double* v = nullptr;    // nnz*nc, entry-major
  float* vf = nullptr;    // FP32 copy (mixed precision)
  double* dg = nullptr;   // diagonal, n*nc
  float* dgf = nullptr;
  double* dl1 = nullptr;  // l1 row norms, n*nc
  float* dl1f = nullptr;
  double lam[3] = {0, 0, 0};  // Gershgorin bound of rho(D^{-1}A) per component
  int lanes = 32;             // threads per row in SpMV kernels
  // level 0 on the structured grid (gx x gy x gz rows, x fastest): values by stencil slot,
  // [slot][component][row], zero outside the grid; sns = 27 (box) or 7 (star), 0 = CSR only.
  // One copy in the apply precision (sv_d for FP64, sv_f for mixed).
  int sgx = 0, sgy = 0, sgz = 0, sns = 0;
  double* sv_d = nullptr;
  float* sv_f = nullptr;
  // transfer to level+1
  int64_t nagg = 0;
  int32_t* agg = nullptr;
  int64_t pnnz = 0;
  int32_t *prp = nullptr, *pci = nullptr;
  double* pv = nullptr;
  float* pvf = nullptr;
  int plane = 8;
  int32_t *rrp = nullptr, *rci = nullptr;
  double* rv = nullptr;
  float* rvf = nullptr;
  // BF16 copies of P and R for the BF16-prolongator variant of the mixed mode (null otherwise)
  __nv_bfloat16 *pvb = nullptr, *rvb = nullptr;
  int rlane = 8;
  // coarsest level: dense FP64 inverse per component (row-major n x n), used in both precisions
  bool coarsest = false;
  double* inv = nullptr;
  // V-cycle work vectors (n*nc entries of the apply precision): iterate x and
  // its ping-pong partner t, residual r, Chebyshev direction d, right-hand
  // side b (written by the finer level's restriction) and result e (read by
  // the finer level's prolongation)
  void *x = nullptr, *t = nullptr, *r = nullptr, *d = nullptr, *b = nullptr, *e = nullptr;
  // Chebyshev smoothing: D^{-1} / theta per row and component (n*nc, apply precision), the scaling of
  // the first step from x = 0
  void* dsi = nullptr;
};

struct Amg {
  int nc = 1;
  std::vector<AmgLevel> L;
  // the V-cycle captured as a CUDA graph for one (input, output, stream) triple, replayed while the
  // triple stays the same; gnodes kernel launches per replay
  cudaGraphExec_t gexec = nullptr;
  const void* gb = nullptr;
  void* gx = nullptr;
  cudaStream_t gst = nullptr;
  int64_t gnodes = 0;
  // the levels from tail_l0 down run as one cooperative launch with bounded grid barriers between their
  // steps (k_vcycle_tail), when set up: tail points to the device array of their descriptors, tail_bar to
  // the barrier counter (zeroed before every launch); err is the handle's bounded-wait error flag
  // tail_mode: 0 none, 1 the cooperative launch from level 1, 2 one thread-block cluster from the first small
  // level (tail_grid is then the cluster's CTA count)
  void* tail = nullptr;
  int tail_mode = 0, tail_l0 = 0, tail_levels = 0, tail_grid = 0;
  // 1: the lanes per row of the coarse levels' CSR kernels are picked by timing (amg_alloc_work)
  int autotune = 0;
  unsigned long long* tail_bar = nullptr;
  int* err = nullptr;
  int64_t spin_limit = 2000000;
  // 1: the V-cycle's kernels after its first use programmatic dependent launch
  int pdl = 1;
};
// destroys the captured V-cycle graph, if any
void amg_release_graph(Amg& H);

struct AmgParams {
  double theta;
  int coarse_max, max_levels;
  bool mixed;
  bool bf16p;  // also keep BF16 copies of P and R (transfer operators read in BF16, summed in FP32)
  bool l1 = true;  // form the l1 row norms (read only by the l1-Jacobi smoother)
};

// Build the hierarchy from the level-0 operator (rp/ci/v are adopted: the
// arena must own them).  Bit-for-bit deterministic: aggregates and Galerkin
// operators do not depend on thread scheduling.
ps_status amg_build(Arena& ar, Amg& H, int nc, int64_t n, int64_t nnz, int32_t* rp, int32_t* ci, double* v,
                    const AmgParams& prm, cudaStream_t st);

// Stencil-slot copy of the level-0 operator of a hierarchy on a gx x gy x gz grid with an ns-point
// pattern (27 or 7).  Sets *ok = false (and leaves the level CSR-only) when some entry is not
// one of the pattern's slots.
ps_status amg_stencil(Arena& ar, Amg& H, int gx, int gy, int gz, int ns, bool mixed, bool* ok, cudaStream_t st);

// Smoothing schedule
struct SmoothParams {
  int kind;    // PS_SMOOTH_*
  int pre, post, degree;
  double ratio;
};

// x = V-cycle(b) on the level-0 vectors (interleaved nc components), T = float or double
template <class T>
ps_status amg_vcycle(Amg& H, const SmoothParams& sp, const T* b, T* x, cudaStream_t st);
// x = V-cycle(b) launched directly (no graph capture), for one-off applications during setup
template <class T>
ps_status amg_vcycle_direct(Amg& H, const SmoothParams& sp, const T* b, T* x, cudaStream_t st);
// allocate the per-level work vectors for precision T (and the Chebyshev first-step scaling of sp)
template <class T>
ps_status amg_alloc_work(Arena& ar, Amg& H, const SmoothParams& sp, cudaStream_t st);

// Aggregation of a scalar operator (one value per entry, sorted columns): the strength graph, distance-2 MIS
// and joining phases of the SDC hierarchy's levels.  *agg (n, -1 = not aggregated) and *excl (n, 1 = row
// without off-diagonal entries) are allocated in ar.
ps_status amg_aggregate_scalar(Arena& ar, int64_t n, int64_t nnz, const int32_t* rp, const int32_t* ci,
                               const double* v, double theta, int level, int32_t** agg, int64_t* nagg,
                               uint8_t** excl, cudaStream_t st);
// sorted column pattern of the product X Y of two CSR patterns (n rows of X, m columns of Y), by the
// SDC hierarchy's SpGEMM run on unit values; *crp (n + 1) and *cci are allocated in ar
ps_status amg_spgemm_pattern(Arena& ar, int64_t n, int64_t m, const int32_t* xrp, const int32_t* xci, int64_t xnnz,
                             const int32_t* yrp, const int32_t* yci, int64_t ynnz, int32_t** crp, int32_t** cci,
                             int64_t* cnnz, cudaStream_t st);
// inverse of a dense n x n FP64 matrix by Gauss-Jordan with partial pivoting: M (row-major) is destroyed,
// inv must hold the identity on entry
ps_status amg_dense_inverse(Arena& ar, int64_t n, double* M, double* inv, cudaStream_t st);

// SpMV lane choice from the mean row length (rows of a few entries, as in the level-0 prolongators, take
// one or two threads each)
inline int lanes_for(double mean_row) {
  if (mean_row <= 4) return 1;
  if (mean_row <= 8) return 2;
  if (mean_row <= 16) return 4;
  if (mean_row <= 48) return 8;
  if (mean_row <= 192) return 16;
  return 32;
}

}  // namespace ps_internal
