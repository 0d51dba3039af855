// Rigid-body-mode smoothed aggregation on the full A_uu: the usual AMG for elasticity, the alternative to the
// separate-displacement-component approximation that §5.2 takes.  Block levels (3 x 3 blocks on the nodes,
// 6 x 6 blocks on the aggregates below), the six rigid-body modes as near-nullspace, a tentative prolongator
// from a modified Gram-Schmidt QR of the modes on each aggregate, P = (I - omega D^{-1} A) P_tent with the
// point diagonal D, Galerkin coarse operators, Chebyshev smoothing on D^{-1} A and a dense FP64 inverse on
// the coarsest level.
#pragma once
#include "amg.cuh"

namespace ps_internal {

constexpr int kRbmModes = 6;

struct RbmLevel {
  int64_t n = 0;  // block rows: nodes on the finest level, aggregates below
  int b = 3;      // block size
  int64_t nnzb = 0;
  int32_t *rp = nullptr, *ci = nullptr;
  double* v = nullptr;  // b x b per block, row-major
  float* vf = nullptr;
  double* dg = nullptr;  // point diagonal, n b
  float* dgf = nullptr;
  double lam = 0.0;      // Gershgorin bound of rho(D^{-1} A) over the point rows
  int lanes = 8;         // threads per block row in the apply kernels
  int32_t* agg = nullptr;
  int64_t nagg = 0;
  double* B = nullptr;   // near-nullspace, n b rows of 6
  double* Pt = nullptr;  // tentative prolongator, n b rows of 6 (zero outside the aggregates)
  int32_t *prp = nullptr, *pci = nullptr;  // P: b x 6 blocks
  int64_t pnnzb = 0;
  double* pv = nullptr;
  float* pvf = nullptr;
  int plane = 4;
  int32_t *rrp = nullptr, *rci = nullptr;  // R = P^T: 6 x b blocks
  double* rv = nullptr;
  float* rvf = nullptr;
  int rlane = 8;
  double* inv = nullptr;  // coarsest: dense inverse, (n b)^2
  bool coarsest = false;
  void *x = nullptr, *t = nullptr, *r = nullptr, *d = nullptr, *bv = nullptr, *e = nullptr;  // work vectors
};

struct Rbm {
  std::vector<RbmLevel> L;
  cudaGraphExec_t gexec = nullptr;  // the V-cycle captured for one (input, output, stream) triple
  const void* gb = nullptr;
  void* gx = nullptr;
  cudaStream_t gst = nullptr;
  int64_t gnodes = 0;
};

// Hierarchy of the nn x nn block operator A_uu (3 x 3 blocks, int32 row pointers, sorted columns) on the
// (nx+1) x (ny+1) x (nz+1) node grid; Chebyshev smoothing only (PS_ERR_INVALID otherwise)
ps_status rbm_build(Arena& ar, Rbm& H, int nx, int ny, int nz, int64_t nnzb, const int32_t* rp, const int32_t* ci,
                    const double* v, double theta, int coarse_max, int max_levels, bool mixed, cudaStream_t st);
template <class T>
ps_status rbm_alloc_work(Arena& ar, Rbm& H, cudaStream_t st);
// x = V-cycle(b) on node-major displacement vectors; replayed as a CUDA graph on capturable streams
template <class T>
ps_status rbm_vcycle(Rbm& H, const SmoothParams& sp, const T* b, T* x, cudaStream_t st);
// the same without a graph
template <class T>
ps_status rbm_vcycle_direct(Rbm& H, const SmoothParams& sp, const T* b, T* x, cudaStream_t st);
void rbm_release_graph(Rbm& H);

}  // namespace ps_internal
