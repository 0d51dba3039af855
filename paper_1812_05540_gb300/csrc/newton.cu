// Newton's method for one time step of the generated problem (§4 and its remarks on inexact Newton): the
// step either side of the linear solve.  The previous time level is the generator's base state (zero
// displacement, its saturation and pressure fields) and is also the first iterate.  Each Newton step assembles
// the residual and the Jacobian at the current state on the device (ps_assemble_at), solves J y = -R r with
// FGMRES under the two-stage preconditioner to the relative tolerance eta_k, the mechanics hierarchy of the
// first step kept (§5.4: ps_setup once, ps_setup_flow afterwards), and updates x += lambda C y, C scaling the
// pressure unknowns from MPa to Pa, lambda halved while the residual does not decrease enough.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "internal.cuh"

namespace ps_internal {
namespace {

// squares of the R-scaled residual entries (Dirichlet rows are zero in r)
__global__ void k_scaled_sq(int64_t n, int64_t nu, const double* __restrict__ r, double au, double af,
                            double* __restrict__ out) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = r[i] / (i < nu ? au : af);
  out[i] = v * v;
}
// rhs = -R r
__global__ void k_newton_rhs(int64_t n, int64_t nu, const double* __restrict__ r, double au, double af,
                             double* __restrict__ rhs) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) rhs[i] = -r[i] / (i < nu ? au : af);
}
// xt = x + lambda C y, C = 1e6 on the pressure unknowns
__global__ void k_newton_step(int64_t n, int64_t nu, const double* __restrict__ x, const double* __restrict__ y,
                              double lam, double* __restrict__ xt) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool pcol = i >= nu && ((i - nu) & 1);
  xt[i] = x[i] + lam * (pcol ? 1e6 * y[i] : y[i]);
}

ps_status scaled_norm(Arena& ar, int64_t n, int64_t nu, const double* r, double au, double af, double* sq,
                      double* dsum, double* out, cudaStream_t st) {
  PS_TICK(); k_scaled_sq<<<grid_for(n, 256), 256, 0, st>>>(n, nu, r, au, af, sq);
  PS_TRY(sum_f64(ar, sq, n, dsum, st));
  double h = 0.0;
  PS_CUDA(cudaMemcpyAsync(&h, dsum, sizeof(double), cudaMemcpyDeviceToHost, st));
  PS_CUDA(cudaStreamSynchronize(st));
  *out = std::sqrt(h);
  return PS_OK;
}

float elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, a, b);
  return ms;
}

}  // namespace
}  // namespace ps_internal

using namespace ps_internal;

extern "C" {

void ps_newton_params_default(ps_newton_params* np) {
  std::memset(np, 0, sizeof(*np));
  np->rtol = 1e-5;  // the Newton tolerance of the paper's runs (Table 1)
  np->max_newton = 12;
  np->forcing = PS_FORCING_EW;
  np->eta_fixed = 1e-6;
  np->ew_gamma = 0.9;
  np->ew_omega = 2.0;
  np->ew_eta0 = 0.1;
  np->ew_eta_max = 0.1;
  np->max_backtracks = 4;
}

double ps_newton_eta(const ps_newton_params* np, int32_t k, double rk, double rkm1, double eta_prev, double r0) {
  if (np->forcing == PS_FORCING_FIXED) return np->eta_fixed;
  double eta;
  if (k == 0) {
    eta = np->ew_eta0;
  } else {
    eta = np->ew_gamma * std::pow(rk / rkm1, np->ew_omega);
    const double safe = np->ew_gamma * std::pow(eta_prev, np->ew_omega);
    if (safe > 0.1) eta = std::max(eta, safe);
  }
  eta = std::min(eta, np->ew_eta_max);
  eta = std::max(eta, 0.5 * np->rtol * r0 / rk);
  return eta;
}

ps_status ps_newton(const ps_gen_params* gp, const ps_params* lin, const ps_newton_params* np, double* x_out,
                    ps_newton_stats* stats) {
  if (!gp || !lin || !np || !x_out || !stats) return PS_ERR_INVALID;
  if (!(np->rtol > 0.0) || np->max_newton < 1 || np->max_backtracks < 0) return PS_ERR_INVALID;
  std::memset(stats, 0, sizeof(*stats));
  cudaStream_t st = static_cast<cudaStream_t>(lin->stream);
  ps_system* sys = nullptr;
  PS_TRY(ps_generate(gp, st, &sys));
  const int64_t n = sys->n, nu = sys->n_u;
  Arena ar;
  ar.stream = st;
  ps_handle* h = nullptr;
  cudaEvent_t ev[2];
  cudaEventCreate(&ev[0]);
  cudaEventCreate(&ev[1]);
  auto done = [&](ps_status s) {
    if (h) ps_free(h);
    cudaStreamSynchronize(st);
    ar.free_all();
    ps_system_free(sys);
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    return s;
  };
  double *x, *xt, *r, *rt, *y, *rhs, *sq, *dsum;
  ps_status s = PS_OK;
  if ((s = ar.alloc(&x, n)) || (s = ar.alloc(&xt, n)) || (s = ar.alloc(&r, n)) || (s = ar.alloc(&rt, n)) ||
      (s = ar.alloc(&y, n)) || (s = ar.alloc(&rhs, n)) || (s = ar.alloc(&sq, n)) || (s = ar.alloc(&dsum, 1)))
    return done(s);
  cudaMemsetAsync(x, 0, sizeof(double) * n, st);
  auto t0 = std::chrono::steady_clock::now();
  cudaEventRecord(ev[0], st);
  if ((s = ps_assemble_at(gp, sys, x, r, st)) != PS_OK) return done(s);
  cudaEventRecord(ev[1], st);
  cudaEventSynchronize(ev[1]);
  stats->ms_assemble += elapsed(ev[0], ev[1]);
  const double au0 = sys->alpha_u, af0 = sys->alpha_f;
  double rk = 0.0;
  if ((s = scaled_norm(ar, n, nu, r, au0, af0, sq, dsum, &rk, st)) != PS_OK) return done(s);
  const double r0 = rk;
  stats->rnorm[0] = rk;
  double rkm1 = rk, eta_prev = np->ew_eta0;
  const int kmax = std::min(np->max_newton, 32);
  for (int k = 0; k < kmax; ++k) {
    if (rk <= np->rtol * r0) break;
    if (k > 0) {  // the Jacobian at the current state (the residual there is already in r)
      cudaEventRecord(ev[0], st);
      if ((s = ps_assemble_at(gp, sys, x, nullptr, st)) != PS_OK) return done(s);
      cudaEventRecord(ev[1], st);
      cudaEventSynchronize(ev[1]);
      stats->ms_assemble += elapsed(ev[0], ev[1]);
    }
    const double eta = ps_newton_eta(np, k, rk, rkm1, eta_prev, r0);
    PS_TICK(); k_newton_rhs<<<grid_for(n, 256), 256, 0, st>>>(n, nu, r, sys->alpha_u, sys->alpha_f, rhs);
    cudaMemsetAsync(y, 0, sizeof(double) * n, st);
    cudaEventRecord(ev[0], st);
    if (!h) {
      ps_params p = *lin;
      p.host_ptrs = 0;
      if ((s = ps_setup(&sys->jac, &sys->grid, &p, &h)) != PS_OK) return done(s);
    } else if ((s = ps_setup_flow(h, &sys->jac)) != PS_OK) {
      return done(s);
    }
    ps_stats ls;
    s = ps_solve(h, rhs, y, eta, &ls);
    cudaEventRecord(ev[1], st);
    cudaEventSynchronize(ev[1]);
    stats->ms_linear += elapsed(ev[0], ev[1]);
    if (s != PS_OK && s != PS_ERR_NOT_CONVERGED) return done(s);
    stats->eta[k] = eta;
    stats->lin_iters[k] = ls.iters;
    stats->linear_iters += ls.iters;
    // backtracking on the base-state scaled residual norm
    double lam = 1.0, rt_norm = 0.0;
    for (int bt = 0;; ++bt) {
      PS_TICK(); k_newton_step<<<grid_for(n, 256), 256, 0, st>>>(n, nu, x, y, lam, xt);
      cudaEventRecord(ev[0], st);
      if ((s = ps_residual_at(gp, sys, xt, rt, st)) != PS_OK) return done(s);
      cudaEventRecord(ev[1], st);
      cudaEventSynchronize(ev[1]);
      stats->ms_assemble += elapsed(ev[0], ev[1]);
      if ((s = scaled_norm(ar, n, nu, rt, au0, af0, sq, dsum, &rt_norm, st)) != PS_OK) return done(s);
      if (rt_norm <= (1.0 - 1e-4 * lam) * rk || bt >= np->max_backtracks) break;
      lam *= 0.5;
      ++stats->backtracks;
    }
    std::swap(x, xt);
    std::swap(r, rt);
    rkm1 = rk;
    rk = rt_norm;
    eta_prev = eta;
    stats->newton_iters = k + 1;
    stats->rnorm[k + 1] = rk;
  }
  stats->converged = rk <= np->rtol * r0 ? 1 : 0;
  cudaMemcpyAsync(x_out, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
  cudaStreamSynchronize(st);
  stats->ms_total =
      float(std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count());
  return done(stats->converged ? PS_OK : PS_ERR_NOT_CONVERGED);
}

}  // extern "C"
