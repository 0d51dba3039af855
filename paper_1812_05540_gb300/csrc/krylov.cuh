// Outer FP64 operator and flexible-GMRES building blocks (§4, right
// preconditioning; flexible variant so that the FP32 preconditioner need not
// be a fixed linear operator).
#pragma once
#include "internal.cuh"

namespace ps_internal {

struct JacDev {
  int64_t nn = 0, nc = 0;
  int nx = 0, ny = 0, nz = 0;
  // stencil-indexed copies of the four blocks, zero padded at the boundary, blocked by 32 rows:
  // [row / 32][slot][entry][row % 32] (null when a pattern is not the structured one; the CSR
  // kernels are used then)
  double *uu_s = nullptr, *uf_s = nullptr, *fu_s = nullptr, *ff_s = nullptr;
  int32_t *uu_rp = nullptr, *uu_ci = nullptr, *uf_rp = nullptr, *uf_ci = nullptr;
  int32_t *fu_rp = nullptr, *fu_ci = nullptr, *ff_rp = nullptr, *ff_ci = nullptr;
  const double *uu_v = nullptr, *uf_v = nullptr, *fu_v = nullptr, *ff_v = nullptr;
};

// y = A x; when b != nullptr also r = b - A x (written to y) and per-block
// partial sums of r^2 into part[0..kRedBlocks)
constexpr int kRedBlocks = 1024;
void jac_spmv(const JacDev& J, const double* x, double* y, const double* b, double* part, cudaStream_t st);
// build the stencil-indexed copies; returns false (and leaves them null) if a pattern is not structured
ps_status jac_build_stencil(Arena& ar, JacDev& J, bool* ok, cudaStream_t st);
// refill existing stencil-indexed copies from the CSR values (same patterns); mask bit k = block k of
// (A_uu, A_uf, A_fu, A_ff)
ps_status jac_refresh_stencil(Arena& ar, JacDev& J, int mask, cudaStream_t st);

// h[c] = V[:,c] . w for c < m (V column-major, leading dimension ldv); also
// ||w||^2 into h[m] when with_norm.  Partials in part (m+1 x kRedBlocks), result in h.
void multidot(const double* V, int64_t ldv, int m, const double* w, int64_t n, double* part, double* h,
              int with_norm, const int* gate, cudaStream_t st);
// w -= V[:, :m] h and ||w||^2 into *norm2 (via partials)
void mupdate(const double* V, int64_t ldv, int m, const double* h, double* w, int64_t n, double* part,
             double* norm2, const int* gate, cudaStream_t st);
// x += Z[:, :m] y
void maxpy(const double* Z, int64_t ldz, int m, const double* y, double* x, int64_t n, cudaStream_t st);
// sum of kRedBlocks partials -> *out
void finish_sum(const double* part, double* out, cudaStream_t st);
// y = x * (*scale)
void scale_vec(const double* x, double* y, int64_t n, const double* scale, cudaStream_t st);
void fill_zero(double* x, int64_t n, cudaStream_t st);

// small dense FGMRES state on the device (declared below); modified Gram-Schmidt step in one
// cooperative launch: h1[0..j] = coefficients, sc[1] = ||w||^2 after projection, w normalised in
// place, flag[0] = 0; a grid barrier that gives up sets flag[2].  Returns false when the launch is
// not possible (blocks = 0 or a cooperative-launch error): the caller falls back to CGS2.  Rows are
// read in pairs: V and w 16-byte aligned, ldv even, and when n is odd row n of every column is zero.
// K.gram holds (m + 1) x mgs_gram_stride() in-block Gram entries; part holds mgs_partials() x blocks.
struct KrylovState;
ps_status mgs_grid(int* blocks);  // four entries: sweeps of 1, 2, 4, 8 vectors
int mgs_gram_stride();
int mgs_partials();
bool mgs_step(const double* V, int64_t ldv, int j, double* w, int64_t n, KrylovState& K, double* part,
              const int* blocks_by_sweep,
              unsigned long long* bar, unsigned long long* base, int64_t limit, int stall, int sweep,
              cudaStream_t st);

// small dense FGMRES state on the device
struct KrylovState {
  double* H;    // (m+1) x m column-major
  double *cs, *sn, *g, *h1, *h2, *y;
  double* gram;  // in-block Gram entries of the basis (modified Gram-Schmidt sweeps)
  double* sc;   // scalars: [0] ||w||^2, [1] ||w'||^2, [2] ||w''||^2, [3] beta, [4] 1/hn, [5] est, [6] hn, [7] bnorm
  int* flag;    // [0] reorthogonalise, [1] nan, [2] a Gram-Schmidt grid barrier gave up
};
// after the first Gram-Schmidt pass: decide on reorthogonalisation (DGKS)
void arnoldi_check(KrylovState& K, cudaStream_t st);
// finish column j: H[:,j], Givens, residual estimate, 1/hn
void arnoldi_finish(KrylovState& K, int m, int j, cudaStream_t st);
// start a cycle from ||r||^2 in sc[3]: g = (beta, 0, ...), 1/beta into sc[4]
void cycle_start(KrylovState& K, int m, cudaStream_t st);
// y = H(0:k,0:k)^{-1} g(0:k)
void hessenberg_solve(KrylovState& K, int m, int k, cudaStream_t st);

// status copied to the host once per iteration
struct IterStatus {
  double est, hn, norm2;
  int nan;
};

}  // namespace ps_internal
