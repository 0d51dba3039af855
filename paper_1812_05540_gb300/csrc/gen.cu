// Seeded synthetic Jacobian generator on the device (test input of the solve).
//
// Physics: quasi-static Biot poroelasticity + two-phase immiscible flow (§2),
// Q1 displacements / P0 saturation and pressure (§3), TPFA fluxes with
// single-point upwinding and face-averaged densities (Eq. (8)-(12)), harmonic
// transmissibilities (App. A), the element and face Jacobian blocks of App. B,
// the fixed-stress diagonals of §5.1 and the block-row scaling remark of §4.
// Fields are synthetic stand-ins for the paper's staircase / SPE10 inputs,
// drawn from a counter-based splitmix64 stream so that every cell can be
// generated independently.
#include <cmath>
#include <cstring>

#include "internal.cuh"

using namespace ps_internal;

namespace {

const double kMD = 9.869233e-16;  // one millidarcy in m^2
const double kPiG = 3.14159265358979323846;

// ---- counter-based random numbers (splitmix64 finaliser, Vigna) ----
__host__ __device__ inline uint64_t mix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ inline uint64_t lat3(int64_t i, int64_t j, int64_t k) {
  const int64_t o = int64_t(1) << 17;
  return uint64_t(i + o) | (uint64_t(j + o) << 18) | (uint64_t(k + o) << 36);
}
__host__ __device__ inline double u01(uint64_t seed, int field, int sub, uint64_t idx) {
  uint64_t r = mix64(mix64(seed) ^ (uint64_t(field) << 55) ^ (uint64_t(sub) << 54) ^ idx);
  return double(r >> 11) * 0x1.0p-53;
}
__device__ inline double normal01(uint64_t seed, int field, uint64_t idx) {
  double a = u01(seed, field, 0, idx), b = u01(seed, field, 1, idx);
  return sqrt(-2.0 * log(1.0 - a)) * cos(2.0 * kPiG * b);
}
enum { FE = 1, FNU = 2, FKAP = 3, FPHI = 4, FSW = 5, FDP = 6, FELAY = 7, FCHAN = 8, FRHS = 9 };

// ---- Gaussian-correlated unit-variance fields ----
__global__ void k_white(double* __restrict__ W, int px, int py, int pz, int Rx, int Ry, int Rz, uint64_t seed,
                        int field) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  int64_t n = int64_t(px) * py * pz;
  if (t >= n) return;
  int i = int(t % px), j = int((t / px) % py), k = int(t / (int64_t(px) * py));
  W[t] = normal01(seed, field, lat3(i - Rx, j - Ry, k - Rz));
}

// out(i, j, k) = sum_d w[d] in(i + R - d, j, k) along axis `ax` (in has the
// padded extent along that axis)
__global__ void k_conv(const double* __restrict__ in, double* __restrict__ out, const double* __restrict__ w, int R,
                       int ox, int oy, int oz, int ax, double scale) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  int64_t n = int64_t(ox) * oy * oz;
  if (t >= n) return;
  int i = int(t % ox), j = int((t / ox) % oy), k = int(t / (int64_t(ox) * oy));
  int ix = ox + (ax == 0 ? 2 * R : 0), iy = oy + (ax == 1 ? 2 * R : 0);
  double s = 0.0;
  for (int d = -R; d <= R; ++d) {
    int a = i, b = j, c = k;
    if (ax == 0) a += R - d;
    if (ax == 1) b += R - d;
    if (ax == 2) c += R - d;
    s += w[d + R] * in[(int64_t(c) * iy + b) * ix + a];
  }
  out[t] = scale == 1.0 ? s : s / scale;
}

ps_status correlated(Arena& ar, uint64_t seed, int field, int nx, int ny, int nz, int Lx, int Ly, int Lz,
                     double* out, cudaStream_t st) {
  int L[3] = {Lx, Ly, Lz}, R[3] = {3 * Lx, 3 * Ly, 3 * Lz};
  std::vector<double> hw[3];
  double norm = 1.0;
  for (int a = 0; a < 3; ++a) {
    double s2 = 0.0;
    for (int d = -R[a]; d <= R[a]; ++d) {
      double q = double(d) / double(L[a]);
      double v = std::exp(-0.5 * q * q);
      hw[a].push_back(v);
      s2 += v * v;
    }
    norm *= std::sqrt(s2);
  }
  int px = nx + 2 * R[0], py = ny + 2 * R[1], pz = nz + 2 * R[2];
  double *W, *X, *Y, *dw[3];
  PS_TRY(ar.alloc(&W, size_t(px) * py * pz));
  PS_TRY(ar.alloc(&X, size_t(nx) * py * pz));
  PS_TRY(ar.alloc(&Y, size_t(nx) * ny * pz));
  for (int a = 0; a < 3; ++a) {
    PS_TRY(ar.alloc(&dw[a], hw[a].size()));
    PS_CUDA(cudaMemcpyAsync(dw[a], hw[a].data(), hw[a].size() * sizeof(double), cudaMemcpyHostToDevice, st));
  }
  int64_t n0 = int64_t(px) * py * pz;
  PS_TICK(); k_white<<<grid_for(n0, 256), 256, 0, st>>>(W, px, py, pz, R[0], R[1], R[2], seed, field);
  PS_TICK(); k_conv<<<grid_for(int64_t(nx) * py * pz, 256), 256, 0, st>>>(W, X, dw[0], R[0], nx, py, pz, 0, 1.0);
  PS_TICK(); k_conv<<<grid_for(int64_t(nx) * ny * pz, 256), 256, 0, st>>>(X, Y, dw[1], R[1], nx, ny, pz, 1, 1.0);
  PS_TICK(); k_conv<<<grid_for(int64_t(nx) * ny * nz, 256), 256, 0, st>>>(Y, out, dw[2], R[2], nx, ny, nz, 2, norm);
  PS_CUDA(cudaGetLastError());
  PS_CUDA(cudaStreamSynchronize(st));  // host weight buffers go out of scope
  ar.release(W); ar.release(X); ar.release(Y);
  for (int a = 0; a < 3; ++a) ar.release(dw[a]);
  return PS_OK;
}

struct Channel {
  double x0, A, lam, ph, halfw, logk;
  int k0, thick;
};

struct FieldArgs {
  int nx, ny, nz, kind, n_low, nch;
  uint64_t seed;
  double h, grav, rho_w0, p_ref, dp_amp, E0, nu0, kappa0, phi0, sw0;
  Channel ch[12];
};

__global__ void k_fields(FieldArgs fa, const double* __restrict__ ghat, const double* __restrict__ ksm,
                         const double* __restrict__ swsm, double* E, double* nu, double* kh, double* kv, double* phi,
                         double* sw, double* p) {
  int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  int64_t nc = int64_t(fa.nx) * fa.ny * fa.nz;
  if (c >= nc) return;
  int i = int(c % fa.nx), j = int((c / fa.nx) % fa.ny), k = int(c / (int64_t(fa.nx) * fa.ny));
  uint64_t L = lat3(i, j, k);
  uint64_t sd = fa.seed;
  double e_, n_, kh_, kv_, ph_, s_;
  if (fa.kind == PS_FIELDS_LOGNORMAL) {
    e_ = exp(log(1e10) - 0.5 * 0.25 + 0.5 * normal01(sd, FE, L));
    n_ = 0.2 + 0.1 * u01(sd, FNU, 0, L);
    kh_ = exp(log(100.0 * kMD) - 0.5 + normal01(sd, FKAP, L));
    kv_ = kh_;
    ph_ = 0.15 + 0.1 * u01(sd, FPHI, 0, L);
    s_ = 0.2 + 0.6 * u01(sd, FSW, 0, L);
  } else if (fa.kind == PS_FIELDS_LAYERED || fa.kind == PS_FIELDS_CHANNELS) {
    if (fa.kind == PS_FIELDS_LAYERED) {
      e_ = exp(log(1e9) + log(50.0) * u01(sd, FELAY, 0, lat3(0, 0, k)));
      kh_ = 100.0 * kMD * exp(2.0 * ksm[c]);
    } else {
      e_ = exp(log(0.5e9) + log(100.0) * u01(sd, FE, 0, L));
      if (k < fa.n_low) {
        double best = log(1e-2);
        for (int q = 0; q < fa.nch; ++q) {
          const Channel& C = fa.ch[q];
          if (k < C.k0 || k >= C.k0 + C.thick) continue;
          double xc = C.x0 + C.A * sin(2.0 * kPiG * (j + 0.5) / C.lam + C.ph);
          if (fabs((i + 0.5) - xc) <= C.halfw) best = fmax(best, C.logk);
        }
        kh_ = exp(best) * kMD;
      } else {
        kh_ = 100.0 * kMD * exp(2.5 * ksm[c]);
      }
    }
    kv_ = 0.1 * kh_;
    n_ = 0.2 + 0.1 * u01(sd, FNU, 0, L);
    ph_ = 0.15 + 0.1 * u01(sd, FPHI, 0, L);
    s_ = 0.2 + 0.6 * (0.5 * erfc(-swsm[c] / sqrt(2.0)));
  } else {
    e_ = fa.E0; n_ = fa.nu0; kh_ = fa.kappa0; kv_ = fa.kappa0; ph_ = fa.phi0; s_ = fa.sw0;
  }
  E[c] = e_; nu[c] = n_; kh[c] = kh_; kv[c] = kv_; phi[c] = ph_; sw[c] = s_;
  double zc = (k + 0.5) * fa.h, ztop = fa.nz * fa.h;
  p[c] = fa.p_ref + fa.rho_w0 * fa.grav * (ztop - zc) + fa.dp_amp * tanh(ghat[c]);
}

// ---- constitutive state per cell (§2 porosity law Eq. (4), §6 density law,
// App. B density derivatives) ----
struct Phys {
  double dt, b, c_w, c_nw, c_r, mu_w, mu_nw, rho_w0, rho_nw0, rho_s0, s_wr, s_nwr, grav, p_ref, corey, h;
  double inv_den, inv_mu_w, inv_mu_nw;  // 1 / (1 - s_wr - s_nwr), 1 / mu_w, 1 / mu_nw
  uint32_t flags;
  int fs_modulus;  // 0: K_dr in the fixed-stress diagonal, 1: uniaxial modulus K_dr + 4G/3
};
struct CellMat {
  double lam, G, Kdr, dphidp, phi, rw, rnw, rs, drho_deps, drho_dp, drho_ds;
};

// material state of a cell (App. B): moduli, porosity at mean volumetric strain ev, densities and their
// derivatives
__device__ inline CellMat cell_mat(const Phys& P, double E, double nu, double phi0, double s, double p,
                                   double ev = 0.0) {
  CellMat m;
  m.lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  m.G = E / (2.0 * (1.0 + nu));
  m.Kdr = E / (3.0 * (1.0 - 2.0 * nu));
  m.dphidp = (P.b - phi0) * (1.0 - P.b) / m.Kdr;
  double dp = p - P.p_ref;
  m.phi = phi0 + P.b * ev + m.dphidp * dp;
  m.rw = P.rho_w0 * (1.0 + P.c_w * dp);
  m.rnw = P.rho_nw0 * (1.0 + P.c_nw * dp);
  m.rs = P.rho_s0 * (1.0 + P.c_r * dp);
  double B = -m.rs + s * m.rw + (1.0 - s) * m.rnw;
  m.drho_deps = B * P.b;
  m.drho_dp = B * m.dphidp + (1.0 - m.phi) * P.rho_s0 * P.c_r + s * m.phi * P.rho_w0 * P.c_w +
              (1.0 - s) * m.phi * P.rho_nw0 * P.c_nw;
  m.drho_ds = m.phi * (m.rw - m.rnw);
  return m;
}

// Corey relative permeabilities of §6 (exponent P.corey) and their s-derivatives
__device__ inline void corey(const Phys& P, double s, double* krw, double* krnw, double* dkrw, double* dkrnw) {
  // the scaled saturation is divided as written: whether it lies inside (0, 1) decides the derivatives
  const double den = 1.0 - P.s_wr - P.s_nwr, rden = P.inv_den;
  double sh = (s - P.s_wr) / den;
  bool in = sh > 0.0 && sh < 1.0;
  sh = fmin(1.0, fmax(0.0, sh));
  double n = P.corey;
  if (n == 2.0) {
    *krw = sh * sh; *krnw = (1.0 - sh) * (1.0 - sh);
    *dkrw = in ? 2.0 * sh * rden : 0.0; *dkrnw = in ? -2.0 * (1.0 - sh) * rden : 0.0;
  } else if (n == 1.0) {
    *krw = sh; *krnw = 1.0 - sh;
    *dkrw = in ? rden : 0.0; *dkrnw = in ? -rden : 0.0;
  } else {
    *krw = pow(sh, n); *krnw = pow(1.0 - sh, n);
    *dkrw = in ? n * pow(sh, n - 1.0) / den : 0.0; *dkrnw = in ? -n * pow(1.0 - sh, n - 1.0) / den : 0.0;
  }
}

struct Ref {  // Q1 integrals on the cube of edge h, and the shape functions at the 8 Gauss points
  double G[8][8][3][3], IN[8], IdN[8][3], INdN[8][8][3];
  double H[8][8][3][3];  // the shear part of the element block: H_ab[d][e] = G_ab[e][d] + delta_de tr G_ab
  double B1[2][2];       // 1-D linear shape functions at the two Gauss abscissae: B1[q][a]
  double gN[8][8], gdN[8][8][3], gw;  // [Gauss point][node]
};

// 2x2x2 Gauss on [0,h]^3; node a has coordinates ((a>>d)&1) h along axis d
void build_ref(double h, Ref* R) {
  std::memset(R, 0, sizeof(Ref));
  const double q[2] = {0.5 - 0.5 / std::sqrt(3.0), 0.5 + 0.5 / std::sqrt(3.0)};
  const double w = h * h * h / 8.0;
  for (int g = 0; g < 8; ++g) {
    double xi[3] = {q[g & 1], q[(g >> 1) & 1], q[(g >> 2) & 1]};
    double N[8], dN[8][3];
    for (int a = 0; a < 8; ++a) {
      double f[3], df[3];
      for (int d = 0; d < 3; ++d) {
        int bit = (a >> d) & 1;
        f[d] = bit ? xi[d] : 1.0 - xi[d];
        df[d] = (bit ? 1.0 : -1.0) / h;
      }
      N[a] = f[0] * f[1] * f[2];
      dN[a][0] = df[0] * f[1] * f[2];
      dN[a][1] = f[0] * df[1] * f[2];
      dN[a][2] = f[0] * f[1] * df[2];
    }
    R->gw = w;
    for (int qq = 0; qq < 2; ++qq) {
      R->B1[qq][0] = 1.0 - q[qq];
      R->B1[qq][1] = q[qq];
    }
    for (int a = 0; a < 8; ++a) {
      R->gN[g][a] = N[a];
      for (int d = 0; d < 3; ++d) R->gdN[g][a][d] = dN[a][d];
    }
    for (int a = 0; a < 8; ++a) {
      R->IN[a] += w * N[a];
      for (int d = 0; d < 3; ++d) R->IdN[a][d] += w * dN[a][d];
      for (int b = 0; b < 8; ++b)
        for (int d = 0; d < 3; ++d) {
          R->INdN[a][b][d] += w * N[a] * dN[b][d];
          for (int e = 0; e < 3; ++e) R->G[a][b][d][e] += w * dN[a][d] * dN[b][e];
        }
    }
  }
  for (int a = 0; a < 8; ++a)
    for (int b = 0; b < 8; ++b) {
      const double tr = R->G[a][b][0][0] + R->G[a][b][1][1] + R->G[a][b][2][2];
      for (int d = 0; d < 3; ++d)
        for (int e = 0; e < 3; ++e) R->H[a][b][d][e] = R->G[a][b][e][d] + (d == e ? tr : 0.0);
    }
}

struct Grid3 {
  int nx, ny, nz;
  __host__ __device__ int64_t node(int i, int j, int k) const { return i + int64_t(nx + 1) * (j + int64_t(ny + 1) * k); }
  __host__ __device__ int64_t cell(int i, int j, int k) const { return i + int64_t(nx) * (j + int64_t(ny) * k); }
};

// ---- patterns (structured; columns ascending) ----
// kind 0: A_uu (node -> 27 nodes), 1: A_uf (node -> <=8 cells), 2: A_fu (cell -> 8 nodes), 3: A_ff (cell -> 7 cells)
__device__ inline int pattern_row(const Grid3& g, int kind, int64_t r, int32_t* cols) {
  int n = 0;
  if (kind == 0 || kind == 1) {
    int i = int(r % (g.nx + 1)), j = int((r / (g.nx + 1)) % (g.ny + 1)), k = int(r / (int64_t(g.nx + 1) * (g.ny + 1)));
    if (kind == 0) {
      for (int dk = -1; dk <= 1; ++dk)
        for (int dj = -1; dj <= 1; ++dj)
          for (int di = -1; di <= 1; ++di) {
            int a = i + di, b = j + dj, c = k + dk;
            if (a < 0 || b < 0 || c < 0 || a > g.nx || b > g.ny || c > g.nz) continue;
            if (cols) cols[n] = int32_t(g.node(a, b, c));
            ++n;
          }
    } else {
      for (int dk = -1; dk <= 0; ++dk)
        for (int dj = -1; dj <= 0; ++dj)
          for (int di = -1; di <= 0; ++di) {
            int a = i + di, b = j + dj, c = k + dk;
            if (a < 0 || b < 0 || c < 0 || a >= g.nx || b >= g.ny || c >= g.nz) continue;
            if (cols) cols[n] = int32_t(g.cell(a, b, c));
            ++n;
          }
    }
  } else {
    int i = int(r % g.nx), j = int((r / g.nx) % g.ny), k = int(r / (int64_t(g.nx) * g.ny));
    if (kind == 2) {
      for (int dk = 0; dk <= 1; ++dk)
        for (int dj = 0; dj <= 1; ++dj)
          for (int di = 0; di <= 1; ++di) {
            if (cols) cols[n] = int32_t(g.node(i + di, j + dj, k + dk));
            ++n;
          }
    } else {
      int64_t nxy = int64_t(g.nx) * g.ny;
      if (k > 0) { if (cols) cols[n] = int32_t(r - nxy); ++n; }
      if (j > 0) { if (cols) cols[n] = int32_t(r - g.nx); ++n; }
      if (i > 0) { if (cols) cols[n] = int32_t(r - 1); ++n; }
      if (cols) cols[n] = int32_t(r);
      ++n;
      if (i + 1 < g.nx) { if (cols) cols[n] = int32_t(r + 1); ++n; }
      if (j + 1 < g.ny) { if (cols) cols[n] = int32_t(r + g.nx); ++n; }
      if (k + 1 < g.nz) { if (cols) cols[n] = int32_t(r + nxy); ++n; }
    }
  }
  return n;
}

__global__ void k_pattern_count(Grid3 g, int kind, int64_t nrows, int32_t* __restrict__ cnt) {
  int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r < nrows) cnt[r] = pattern_row(g, kind, r, nullptr);
}
__global__ void k_pattern_fill(Grid3 g, int kind, int64_t nrows, const int64_t* __restrict__ rp,
                               int32_t* __restrict__ ci) {
  int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r < nrows) pattern_row(g, kind, r, ci + rp[r]);
}

// ---- material table per cell ----
__global__ void k_material(Phys P, int64_t nc, const double* __restrict__ E, const double* __restrict__ nu,
                           const double* __restrict__ phi0, const double* __restrict__ sw,
                           const double* __restrict__ p, const double* __restrict__ ev, CellMat* __restrict__ out) {
  int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (c < nc) out[c] = cell_mat(P, E[c], nu[c], phi0[c], sw[c], p[c], ev ? ev[c] : 0.0);
}

// A_uu block (I, J): sum over the elements shared by nodes I and J (ascending element id) of the App. B
// element block, lam G_ab + mu H_ab (elasticity) plus the gravity term drho/deps_v g IN_a dN_b in the z row.
// The neighbours J are walked in the pattern's order (27-point box, ascending id), so no column is decoded.
__global__ void k_values_uu(Grid3 g, Phys P, const Ref* __restrict__ R, const CellMat* __restrict__ M,
                            const int64_t* __restrict__ rp, int64_t nn, double* __restrict__ val) {
  const int64_t I = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (I >= nn) return;
  const int ix = int(I % (g.nx + 1)), iy = int((I / (g.nx + 1)) % (g.ny + 1)),
            iz = int(I / (int64_t(g.nx + 1) * (g.ny + 1)));
  const double grav = (P.flags & PS_GEN_GRAVITY) ? P.grav : 0.0;
  int64_t q = rp[I];
  for (int jz = max(iz - 1, 0); jz <= min(iz + 1, g.nz); ++jz)
    for (int jy = max(iy - 1, 0); jy <= min(iy + 1, g.ny); ++jy)
      for (int jx = max(ix - 1, 0); jx <= min(ix + 1, g.nx); ++jx, ++q) {
        double blk[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        const int ex0 = max(max(ix, jx) - 1, 0), ex1 = min(min(ix, jx), g.nx - 1);
        const int ey0 = max(max(iy, jy) - 1, 0), ey1 = min(min(iy, jy), g.ny - 1);
        const int ez0 = max(max(iz, jz) - 1, 0), ez1 = min(min(iz, jz), g.nz - 1);
        for (int ez = ez0; ez <= ez1; ++ez)
          for (int ey = ey0; ey <= ey1; ++ey)
            for (int ex = ex0; ex <= ex1; ++ex) {
              const CellMat& m = M[g.cell(ex, ey, ez)];
              const int a = (ix - ex) | ((iy - ey) << 1) | ((iz - ez) << 2);
              const int b = (jx - ex) | ((jy - ey) << 1) | ((jz - ez) << 2);
              const double lam = m.lam, mu = m.G;
              const double* Gab = &R->G[a][b][0][0];
              const double* Hab = &R->H[a][b][0][0];
#pragma unroll
              for (int t = 0; t < 9; ++t) blk[t] = fma(lam, Gab[t], fma(mu, Hab[t], blk[t]));
              if (grav != 0.0) {
                const double cg = m.drho_deps * grav;
#pragma unroll
                for (int e = 0; e < 3; ++e) blk[6 + e] = fma(cg, R->INdN[a][b][e], blk[6 + e]);
              }
            }
#pragma unroll
        for (int t = 0; t < 9; ++t) val[q * 9 + t] = blk[t];
      }
}

// A_uf (node I, cell c) = [A_us A_up] and A_fu (cell c, node J) = [A_su; A_pu]
__global__ void k_values_uf(Grid3 g, Phys P, const Ref* __restrict__ R, const CellMat* __restrict__ M,
                            const int64_t* __restrict__ rp, const int32_t* __restrict__ ci, int64_t nn,
                            double* __restrict__ val) {
  int64_t I = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (I >= nn) return;
  int ix = int(I % (g.nx + 1)), iy = int((I / (g.nx + 1)) % (g.ny + 1)), iz = int(I / (int64_t(g.nx + 1) * (g.ny + 1)));
  double grav = (P.flags & PS_GEN_GRAVITY) ? P.grav : 0.0;
  bool coup = (P.flags & PS_GEN_COUPLING) != 0;
  for (int64_t q = rp[I]; q < rp[I + 1]; ++q) {
    int64_t c = ci[q];
    int ex = int(c % g.nx), ey = int((c / g.nx) % g.ny), ez = int(c / (int64_t(g.nx) * g.ny));
    int a = (ix - ex) | ((iy - ey) << 1) | ((iz - ez) << 2);
    const CellMat& m = M[c];
    for (int d = 0; d < 3; ++d) {
      double gd = d == 2 ? -grav : 0.0;
      double us = -R->IN[a] * m.drho_ds * gd;
      double up = -P.b * R->IdN[a][d] - R->IN[a] * m.drho_dp * gd;
      val[q * 6 + d * 2 + 0] = coup ? 0.0 + us : 0.0;
      val[q * 6 + d * 2 + 1] = coup ? 0.0 + up : 0.0;
    }
  }
}

__global__ void k_values_fu(Grid3 g, Phys P, const Ref* __restrict__ R, const CellMat* __restrict__ M,
                            const double* __restrict__ sw, const int64_t* __restrict__ rp,
                            const int32_t* __restrict__ ci, int64_t nc, double* __restrict__ val) {
  int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  int ex = int(c % g.nx), ey = int((c / g.nx) % g.ny), ez = int(c / (int64_t(g.nx) * g.ny));
  bool coup = (P.flags & PS_GEN_COUPLING) != 0;
  const CellMat& m = M[c];
  double s = sw[c];
  for (int64_t q = rp[c]; q < rp[c + 1]; ++q) {
    int64_t J = ci[q];
    int jx = int(J % (g.nx + 1)), jy = int((J / (g.nx + 1)) % (g.ny + 1)), jz = int(J / (int64_t(g.nx + 1) * (g.ny + 1)));
    int b = (jx - ex) | ((jy - ey) << 1) | ((jz - ez) << 2);
    for (int e = 0; e < 3; ++e) {
      double su = s * m.rw * P.b * R->IdN[b][e];
      double pu = (1.0 - s) * m.rnw * P.b * R->IdN[b][e];
      val[q * 6 + e] = coup ? 0.0 + su : 0.0;
      val[q * 6 + 3 + e] = coup ? 0.0 + pu : 0.0;
    }
  }
}

// TPFA face between K < L (App. A transmissibility, Eq. (8), Eq. (12), App. B
// face derivatives); phase 0 = wetting, 1 = non-wetting.
struct FaceD {
  double dsK, dsL, dpK, dpL;
};
__device__ inline FaceD face_deriv(const Phys& P, double Ups, double dz, int ph, double sK, double pK, double sL,
                                   double pL) {
  double grav = (P.flags & PS_GEN_GRAVITY) ? P.grav : 0.0;
  double r0 = ph == 0 ? P.rho_w0 : P.rho_nw0;
  double c = ph == 0 ? P.c_w : P.c_nw;
  double rmu = ph == 0 ? P.inv_mu_w : P.inv_mu_nw;
  double rK = r0 * (1.0 + c * (pK - P.p_ref)), rL = r0 * (1.0 + c * (pL - P.p_ref));
  double aK = ph == 0 ? sK : 1.0 - sK, aL = ph == 0 ? sL : 1.0 - sL;
  double vr, dvK, dvL;
  if (aK > 0.0 && aL > 0.0) { vr = 0.5 * (rK + rL); dvK = 0.5 * r0 * c; dvL = 0.5 * r0 * c; }
  else if (aK > 0.0) { vr = rK; dvK = r0 * c; dvL = 0.0; }
  else if (aL > 0.0) { vr = rL; dvK = 0.0; dvL = r0 * c; }
  else { vr = 0.0; dvK = 0.0; dvL = 0.0; }
  double Phi = Ups * ((pL - pK) + vr * grav * dz);
  bool upL = Phi > 0.0;
  double sU = upL ? sL : sK, pU = upL ? pL : pK;
  double krw, krnw, dkrw, dkrnw;
  corey(P, sU, &krw, &krnw, &dkrw, &dkrnw);
  double kr = ph == 0 ? krw : krnw, dkr = ph == 0 ? dkrw : dkrnw;
  double rU = r0 * (1.0 + c * (pU - P.p_ref));
  double lamU = kr * rmu;
  double dsU = rU * rmu * Phi * dkr;
  FaceD f;
  bool sat = (P.flags & PS_GEN_FLUX_SAT) != 0;
  f.dsK = sat ? (upL ? 0.0 : dsU) : 0.0;
  f.dsL = sat ? (upL ? dsU : 0.0) : 0.0;
  double drU = r0 * c;
  f.dpK = (upL ? 0.0 : drU * lamU * Phi) + rU * lamU * Ups * (-1.0 + dvK * grav * dz);
  f.dpL = (upL ? drU * lamU * Phi : 0.0) + rU * lamU * Ups * (1.0 + dvL * grav * dz);
  return f;
}

// harmonic mean of the two half transmissibilities |f| kappa / (h/2) = 2 h kappa (App. A)
__device__ inline double face_ups(double h, double kK, double kL) {
  const double UK = 2.0 * h * kK, UL = 2.0 * h * kL;
  return UK * UL / (UK + UL);
}

// Peaceman well of the cell column (i, j) under bottom-hole pressure control (§3 well model, Eq. (peaceman),
// Eq. (well_index); Table 1): 1 the water injector (column (0, 0)), 2 the producer (column (nx-1, ny-1)), 0 none.
// Both perforate every layer; the bottom-hole pressure is referred to the top perforation's centroid and set
// 5 MPa above (injector) or below (producer) the hydrostatic formation pressure there, built up linearly over
// one day (a step of dt from the start reaches the fraction min(dt / 1 day, 1)).  For the cube cell of
// edge h, WI = 2 pi h kappa_h / ln(r / r_w), r = 0.28 sqrt(2) h / 2, r_w = 0.1524 m, no skin.  The cell's
// mass-balance rows get -dt (q^I_l - q^P_l): injector q^I_w = rho_w (lambda_w + lambda_nw) Phi_w (no
// non-wetting injection), producer q^P_l = -rho_l lambda_l Phi_l, Phi_l = WI [(p_bh - p) + rho_l g (z_bh - z)];
// wr gets the two terms and wd their (s, p) derivatives.
__device__ inline int well_kind(const Grid3& g, int i, int j) {
  if (i == 0 && j == 0) return 1;
  if (i == g.nx - 1 && j == g.ny - 1) return 2;
  return 0;
}
__device__ void well_terms(const Phys& P, const Grid3& g, int kind, int k, double kh, double s, double p,
                           double wr[2], double wd[2][2]) {
  const double grav = (P.flags & PS_GEN_GRAVITY) ? P.grav : 0.0;
  const double h = P.h, zbh = (g.nz - 0.5) * h, zK = (k + 0.5) * h;
  const double pform = P.p_ref + P.rho_w0 * grav * (g.nz * h - zbh);
  const double dbhp = 5.0e6 * fmin(P.dt / 86400.0, 1.0);  // one-day linear build-up of the offsets
  const double pbh = kind == 1 ? pform + dbhp : pform - dbhp;
  const double WI = 2.0 * kPiG * h * kh / log(0.28 * sqrt(2.0) * h / 2.0 / 0.1524);
  double krw, krnw, dkrw, dkrnw;
  corey(P, s, &krw, &krnw, &dkrw, &dkrnw);
  const double lam[2] = {krw * P.inv_mu_w, krnw * P.inv_mu_nw};
  const double dlam[2] = {dkrw * P.inv_mu_w, dkrnw * P.inv_mu_nw};
  const double dp = p - P.p_ref;
  const double rho[2] = {P.rho_w0 * (1.0 + P.c_w * dp), P.rho_nw0 * (1.0 + P.c_nw * dp)};
  const double drho[2] = {P.rho_w0 * P.c_w, P.rho_nw0 * P.c_nw};
  for (int l = 0; l < 2; ++l) {
    const double Phi = WI * ((pbh - p) + rho[l] * grav * (zbh - zK));
    const double dPhi = WI * (-1.0 + drho[l] * grav * (zbh - zK));
    double q = 0.0, dqs = 0.0, dqp = 0.0;
    if (kind == 1) {
      if (l == 0) {
        const double lt = lam[0] + lam[1];
        q = rho[0] * lt * Phi;
        dqs = rho[0] * (dlam[0] + dlam[1]) * Phi;
        dqp = drho[0] * lt * Phi + rho[0] * lt * dPhi;
      }
    } else {
      q = rho[l] * lam[l] * Phi;
      dqs = rho[l] * dlam[l] * Phi;
      dqp = drho[l] * lam[l] * Phi + rho[l] * lam[l] * dPhi;
    }
    wr[l] = -P.dt * q;
    wd[l][0] = -P.dt * dqs;
    wd[l][1] = -P.dt * dqp;
  }
}

// A_ff row of cell c: accumulation (App. B element blocks), then the faces in
// which c is the upper cell L (lower cells ascending), then those in which c is
// the lower cell K (x, y, z).  Row K gets -dt dF, row L gets +dt dF.
__global__ void k_values_ff(Grid3 g, Phys P, const CellMat* __restrict__ M, const double* __restrict__ sw,
                            const double* __restrict__ p, const double* __restrict__ kh,
                            const double* __restrict__ kv, const int64_t* __restrict__ rp,
                            const int32_t* __restrict__ ci, int64_t nc, double* __restrict__ val,
                            double* __restrict__ dfs) {
  int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  int i = int(c % g.nx), j = int((c / g.nx) % g.ny), k = int(c / (int64_t(g.nx) * g.ny));
  int64_t nxy = int64_t(g.nx) * g.ny;
  double V = P.h * P.h * P.h;
  const CellMat& m = M[c];
  double s = sw[c];
  int64_t q0 = rp[c], q1 = rp[c + 1], qd = q0;
  for (int64_t q = q0; q < q1; ++q) {
    if (ci[q] == c) qd = q;
    for (int t = 0; t < 4; ++t) val[q * 4 + t] = 0.0;
  }
  double dg[4] = {0, 0, 0, 0};
  if (P.flags & PS_GEN_ACCUM) {
    dg[0] += V * m.phi * m.rw;
    dg[1] += V * (s * m.rw * m.dphidp + m.phi * s * P.rho_w0 * P.c_w);
    dg[2] += -V * m.phi * m.rnw;
    dg[3] += V * ((1.0 - s) * m.rnw * m.dphidp + m.phi * (1.0 - s) * P.rho_nw0 * P.c_nw);
  }
  if (P.flags & PS_GEN_FLUX) {
    // faces where c is the upper cell L: neighbours below in z, y, x (ascending id)
    for (int dir = 2; dir >= 0; --dir) {
      int a = i - (dir == 0), b = j - (dir == 1), cc = k - (dir == 2);
      if (a < 0 || b < 0 || cc < 0) continue;
      int64_t K = c - (dir == 0 ? 1 : dir == 1 ? g.nx : nxy);
      double Ups = dir == 2 ? face_ups(P.h, kv[K], kv[c]) : face_ups(P.h, kh[K], kh[c]);
      double dz = dir == 2 ? P.h : 0.0;
      int64_t qK = q0;
      while (ci[qK] != K) ++qK;
      for (int ph = 0; ph < 2; ++ph) {
        FaceD f = face_deriv(P, Ups, dz, ph, sw[K], p[K], s, p[c]);
        dg[ph * 2 + 0] += P.dt * f.dsL;
        dg[ph * 2 + 1] += P.dt * f.dpL;
        val[qK * 4 + ph * 2 + 0] = 0.0 + P.dt * f.dsK;
        val[qK * 4 + ph * 2 + 1] = 0.0 + P.dt * f.dpK;
      }
    }
    // faces where c is the lower cell K: neighbours above in x, y, z
    for (int dir = 0; dir < 3; ++dir) {
      int a = i + (dir == 0), b = j + (dir == 1), cc = k + (dir == 2);
      if (a >= g.nx || b >= g.ny || cc >= g.nz) continue;
      int64_t L = c + (dir == 0 ? 1 : dir == 1 ? g.nx : nxy);
      double Ups = dir == 2 ? face_ups(P.h, kv[c], kv[L]) : face_ups(P.h, kh[c], kh[L]);
      double dz = dir == 2 ? P.h : 0.0;
      int64_t qL = q0;
      while (ci[qL] != L) ++qL;
      for (int ph = 0; ph < 2; ++ph) {
        FaceD f = face_deriv(P, Ups, dz, ph, s, p[c], sw[L], p[L]);
        dg[ph * 2 + 0] += -P.dt * f.dsK;
        dg[ph * 2 + 1] += -P.dt * f.dpK;
        val[qL * 4 + ph * 2 + 0] = 0.0 + -P.dt * f.dsL;
        val[qL * 4 + ph * 2 + 1] = 0.0 + -P.dt * f.dpL;
      }
    }
  }
  if (P.flags & PS_GEN_WELLS) {
    const int kind = well_kind(g, i, j);
    if (kind) {
      double wr[2], wd[2][2];
      well_terms(P, g, kind, k, kh[c], s, p[c], wr, wd);
      for (int l = 0; l < 2; ++l)
        for (int e = 0; e < 2; ++e) dg[l * 2 + e] += wd[l][e];
    }
  }
  for (int t = 0; t < 4; ++t) val[qd * 4 + t] = dg[t];
  // §5.1 fixed-stress diagonal entries (K_dr, or the uniaxial modulus of the §5.1 remark)
  const double Kfs = P.fs_modulus == 1 ? m.Kdr + 4.0 * m.G / 3.0 : m.Kdr;
  dfs[2 * c + 0] = V * P.b * P.b / Kfs * s * m.rw;
  dfs[2 * c + 1] = V * P.b * P.b / Kfs * (1.0 - s) * m.rnw;
}

// ---- residual of the discrete equations at a state (§3, App. B), for Newton's method ----
// Element-mean volumetric strain of each cell from the nodal displacements: (1/|K|) sum_a sum_d IdN_a,d u_a,d.
__global__ void k_mean_epsv(Grid3 g, const Ref* __restrict__ R, const double* __restrict__ u, double h,
                            double* __restrict__ ev) {
  const int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t nc = int64_t(g.nx) * g.ny * g.nz;
  if (c >= nc) return;
  const int i = int(c % g.nx), j = int((c / g.nx) % g.ny), k = int(c / (int64_t(g.nx) * g.ny));
  double s = 0.0;
  for (int a = 0; a < 8; ++a) {
    const int64_t I = g.node(i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
    for (int d = 0; d < 3; ++d) s += R->IdN[a][d] * u[3 * I + d];
  }
  ev[c] = s / (h * h * h);
}

// Two-axis tensor contractions of the trilinear element (node a = ax | ay << 1 | az << 2, Gauss point
// q = qx | qy << 1 | qz << 2).  interp2: values at the 2 x 2 Gauss abscissae of a bilinear field given at the
// 2 x 2 nodes, out[p][r] = sum_ij B[p][i] B[r][j] in[i][j]; project2 is its transpose,
// out[i][j] = sum_pr B[p][i] B[r][j] in[p][r].
__device__ __forceinline__ void interp2(const double (&B)[2][2], const double (&in)[2][2], double (&out)[2][2]) {
  double t[2][2];
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int j = 0; j < 2; ++j) t[p][j] = fma(B[p][0], in[0][j], B[p][1] * in[1][j]);
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int r = 0; r < 2; ++r) out[p][r] = fma(B[r][0], t[p][0], B[r][1] * t[p][1]);
}
__device__ __forceinline__ void project2(const double (&B)[2][2], const double (&in)[2][2], double (&out)[2][2]) {
  double t[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int r = 0; r < 2; ++r) t[i][r] = fma(B[0][i], in[0][r], B[1][i] * in[1][r]);
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) out[i][j] = fma(B[0][j], t[i][0], B[1][j] * t[i][1]);
}

// Element part of the mechanics residual and the cell's flow accumulation (App. B, Eq. (5) weak form, 2 x 2 x 2
// Gauss).  Per cell: at each Gauss point the displacement gradient, the effective stress
// lam eps_v I + G (grad u + grad u^T) and the bulk density at the pointwise strain; the nodal terms
// int (sigma' : grad eta - b p div eta - rho g . eta) go to er[c][a][d].  The Q1 element is a tensor product,
// so the gradients at the Gauss points and the projections onto the test functions are taken axis by axis
// (sum factorisation): the x-derivative of a trilinear field is bilinear in (y, z) and the same at both x
// abscissae, and so on.  The pressure term is b p times the integral of grad N_a; the density is affine in
// the pointwise strain, rho = rho(phi_bar) + b (rho_f - rho_s) eps_v.  The accumulation change of both
// phases against the previous time level (the base state: zero displacement, saturation s0, pressure p0)
// goes to rf[2 c], rf[2 c + 1].
__global__ void __launch_bounds__(128) k_res_elem(Grid3 g, Phys P, const Ref* __restrict__ R,
                                                  const double* __restrict__ E, const double* __restrict__ nu,
                                                  const double* __restrict__ phi0, const double* __restrict__ u,
                                                  const double* __restrict__ s, const double* __restrict__ p,
                                                  const double* __restrict__ s0, const double* __restrict__ p0,
                                                  double* __restrict__ er, double* __restrict__ rf) {
  const int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t nc = int64_t(g.nx) * g.ny * g.nz;
  if (c >= nc) return;
  const int i = int(c % g.nx), j = int((c / g.nx) % g.ny), k = int(c / (int64_t(g.nx) * g.ny));
  double B[2][2];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int a = 0; a < 2; ++a) B[q][a] = R->B1[q][a];
  const double rh = 1.0 / P.h, w = R->gw;
  // gradients at the Gauss points: gr[d][e][.][.] = d u_d / d x_e over the two abscissae of the other axes
  // (e = x: [qy][qz], e = y: [qx][qz], e = z: [qx][qy])
  double gr[3][3][2][2];
  {
    double un[3][8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int64_t I = g.node(i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
#pragma unroll
      for (int d = 0; d < 3; ++d) un[d][a] = u[3 * I + d];
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      double dl[2][2];
#pragma unroll
      for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int n = 0; n < 2; ++n) dl[m][n] = (un[d][1 | (m << 1) | (n << 2)] - un[d][0 | (m << 1) | (n << 2)]) * rh;
      interp2(B, dl, gr[d][0]);
#pragma unroll
      for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int n = 0; n < 2; ++n) dl[m][n] = (un[d][m | (1 << 1) | (n << 2)] - un[d][m | (0 << 1) | (n << 2)]) * rh;
      interp2(B, dl, gr[d][1]);
#pragma unroll
      for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int n = 0; n < 2; ++n) dl[m][n] = (un[d][m | (n << 1) | (1 << 2)] - un[d][m | (n << 1) | (0 << 2)]) * rh;
      interp2(B, dl, gr[d][2]);
    }
  }
  const double grav = (P.flags & PS_GEN_GRAVITY) ? P.grav : 0.0;
  const CellMat m0 = cell_mat(P, E[c], nu[c], phi0[c], s[c], p[c]);
  const double sc = s[c], pc = p[c], b = P.b;
  const double lam = m0.lam, mu = m0.G;
  // stresses summed over the abscissa of their derivative's axis: S[d][e][.][.] indexed like gr[d][e]
  double S[3][3][2][2];
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int e = 0; e < 3; ++e)
#pragma unroll
      for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int n = 0; n < 2; ++n) S[d][e][m][n] = 0.0;
  double evq[2][2][2];  // [qx][qy][qz]
#pragma unroll
  for (int qz = 0; qz < 2; ++qz)
#pragma unroll
    for (int qy = 0; qy < 2; ++qy)
#pragma unroll
      for (int qx = 0; qx < 2; ++qx) {
        double G[3][3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          G[d][0] = gr[d][0][qy][qz];
          G[d][1] = gr[d][1][qx][qz];
          G[d][2] = gr[d][2][qx][qy];
        }
        const double ev = G[0][0] + G[1][1] + G[2][2];
        evq[qx][qy][qz] = ev;
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int e = 0; e < 3; ++e) {
            const double sig = (d == e) ? fma(lam, ev, 2.0 * mu * G[d][d]) : mu * (G[d][e] + G[e][d]);
            if (e == 0) S[d][0][qy][qz] += sig;
            else if (e == 1) S[d][1][qx][qz] += sig;
            else S[d][2][qx][qy] += sig;
          }
      }
  // projections onto the test-function gradients: f[a][d] = w sum_e D_e(a) (B B)^T S[d][e]
  double f[8][3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double T[2][2];
    project2(B, S[d][0], T);  // T[ay][az]
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const double v = w * rh * T[(a >> 1) & 1][(a >> 2) & 1];
      f[a][d] = (a & 1) ? v : -v;
    }
    project2(B, S[d][1], T);  // T[ax][az]
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const double v = w * rh * T[a & 1][(a >> 2) & 1];
      f[a][d] += ((a >> 1) & 1) ? v : -v;
    }
    project2(B, S[d][2], T);  // T[ax][ay]
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const double v = w * rh * T[a & 1][(a >> 1) & 1];
      f[a][d] += ((a >> 2) & 1) ? v : -v;
    }
  }
  // pressure: - b p int dN_a / dx_d
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int d = 0; d < 3; ++d) f[a][d] = fma(-b * pc, R->IdN[a][d], f[a][d]);
  // integral of the strain and, for gravity, of N_a times the strain: w sum_q N_a(q) eps_v(q), axis by axis
  double int_ev = 0.0;
#pragma unroll
  for (int qz = 0; qz < 2; ++qz)
#pragma unroll
    for (int qy = 0; qy < 2; ++qy)
#pragma unroll
      for (int qx = 0; qx < 2; ++qx) int_ev += evq[qx][qy][qz];
  int_ev *= w;
  const double phibar = phi0[c] + m0.dphidp * (pc - P.p_ref);
  if (grav != 0.0) {
    const double rf_ = sc * m0.rw + (1.0 - sc) * m0.rnw;
    const double rho0 = m0.rs + phibar * (rf_ - m0.rs), kap = b * (rf_ - m0.rs);
    double t1[2][2][2], t2[2][2][2];  // contract qx, then qy, then qz
#pragma unroll
    for (int ax = 0; ax < 2; ++ax)
#pragma unroll
      for (int qy = 0; qy < 2; ++qy)
#pragma unroll
        for (int qz = 0; qz < 2; ++qz) t1[ax][qy][qz] = fma(B[0][ax], evq[0][qy][qz], B[1][ax] * evq[1][qy][qz]);
#pragma unroll
    for (int ax = 0; ax < 2; ++ax)
#pragma unroll
      for (int ay = 0; ay < 2; ++ay)
#pragma unroll
        for (int qz = 0; qz < 2; ++qz) t2[ax][ay][qz] = fma(B[0][ay], t1[ax][0][qz], B[1][ay] * t1[ax][1][qz]);
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
      const double Ne = w * fma(B[0][az], t2[ax][ay][0], B[1][az] * t2[ax][ay][1]);
      f[a][2] = fma(grav, fma(rho0, R->IN[a], kap * Ne), f[a][2]);
    }
  }
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int d = 0; d < 3; ++d) er[(c * 8 + a) * 3 + d] = f[a][d];
  double r0 = 0.0, r1 = 0.0;
  if (P.flags & PS_GEN_ACCUM) {
    const double V = P.h * P.h * P.h;
    const double phiV = V * phibar + b * int_ev;
    const CellMat mp = cell_mat(P, E[c], nu[c], phi0[c], s0[c], p0[c]);
    const double phiVp = V * (phi0[c] + mp.dphidp * (p0[c] - P.p_ref));
    r0 = phiV * m0.rw * sc - phiVp * mp.rw * s0[c];
    r1 = phiV * m0.rnw * (1.0 - sc) - phiVp * mp.rnw * (1.0 - s0[c]);
  }
  rf[2 * c] = r0;
  rf[2 * c + 1] = r1;
}

// mass flux of one phase through the face K -> L (Eq. (8), Eq. (12)): face density, upwind mobility
__device__ inline double face_value(const Phys& P, double Ups, double dz, int ph, double sK, double pK, double sL,
                                    double pL) {
  const double grav = (P.flags & PS_GEN_GRAVITY) ? P.grav : 0.0;
  const double r0 = ph == 0 ? P.rho_w0 : P.rho_nw0;
  const double c = ph == 0 ? P.c_w : P.c_nw;
  const double rmu = ph == 0 ? P.inv_mu_w : P.inv_mu_nw;
  const double rK = r0 * (1.0 + c * (pK - P.p_ref)), rL = r0 * (1.0 + c * (pL - P.p_ref));
  const double aK = ph == 0 ? sK : 1.0 - sK, aL = ph == 0 ? sL : 1.0 - sL;
  double vr;
  if (aK > 0.0 && aL > 0.0) vr = 0.5 * (rK + rL);
  else if (aK > 0.0) vr = rK;
  else if (aL > 0.0) vr = rL;
  else vr = 0.0;
  const double Phi = Ups * ((pL - pK) + vr * grav * dz);
  const bool upL = Phi > 0.0;
  const double sU = upL ? sL : sK, pU = upL ? pL : pK;
  double krw, krnw, dkrw, dkrnw;
  corey(P, sU, &krw, &krnw, &dkrw, &dkrnw);
  const double kr = ph == 0 ? krw : krnw;
  const double rU = r0 * (1.0 + c * (pU - P.p_ref));
  return rU * (kr * rmu) * Phi;
}

// Residual rows: mechanics rows gather the element terms of the node's elements (ascending element id);
// flow rows add the face fluxes to the accumulation in face order (below in z, y, x, then above in x, y, z),
// -dt F on the lower cell and +dt F on the upper one.  Dirichlet rows are zero.
__global__ void k_res_nodes(Grid3 g, const double* __restrict__ er, const uint8_t* __restrict__ dir,
                            double* __restrict__ r) {
  const int64_t I = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t nn = int64_t(g.nx + 1) * (g.ny + 1) * (g.nz + 1);
  if (I >= nn) return;
  const int ix = int(I % (g.nx + 1)), iy = int((I / (g.nx + 1)) % (g.ny + 1)), iz = int(I / (int64_t(g.nx + 1) * (g.ny + 1)));
  double v[3] = {0.0, 0.0, 0.0};
  for (int ez = max(iz - 1, 0); ez <= min(iz, g.nz - 1); ++ez)
    for (int ey = max(iy - 1, 0); ey <= min(iy, g.ny - 1); ++ey)
      for (int ex = max(ix - 1, 0); ex <= min(ix, g.nx - 1); ++ex) {
        const int64_t c = g.cell(ex, ey, ez);
        const int a = (ix - ex) | ((iy - ey) << 1) | ((iz - ez) << 2);
        for (int d = 0; d < 3; ++d) v[d] += er[(c * 8 + a) * 3 + d];
      }
  for (int d = 0; d < 3; ++d) r[3 * I + d] = dir[3 * I + d] ? 0.0 : v[d];
}

__global__ void k_res_cells(Grid3 g, Phys P, const double* __restrict__ kh, const double* __restrict__ kv,
                            const double* __restrict__ s, const double* __restrict__ p, const double* __restrict__ rf,
                            double* __restrict__ r) {
  const int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t nc = int64_t(g.nx) * g.ny * g.nz;
  if (c >= nc) return;
  const int i = int(c % g.nx), j = int((c / g.nx) % g.ny), k = int(c / (int64_t(g.nx) * g.ny));
  const int64_t nxy = int64_t(g.nx) * g.ny;
  double v[2] = {rf[2 * c], rf[2 * c + 1]};
  if (P.flags & PS_GEN_FLUX) {
    for (int dir = 2; dir >= 0; --dir) {  // c is the upper cell L
      if ((dir == 0 && i == 0) || (dir == 1 && j == 0) || (dir == 2 && k == 0)) continue;
      const int64_t K = c - (dir == 0 ? 1 : dir == 1 ? g.nx : nxy);
      const double Ups = dir == 2 ? face_ups(P.h, kv[K], kv[c]) : face_ups(P.h, kh[K], kh[c]);
      const double dz = dir == 2 ? P.h : 0.0;
      for (int ph = 0; ph < 2; ++ph) v[ph] += P.dt * face_value(P, Ups, dz, ph, s[K], p[K], s[c], p[c]);
    }
    for (int dir = 0; dir < 3; ++dir) {  // c is the lower cell K
      if ((dir == 0 && i + 1 >= g.nx) || (dir == 1 && j + 1 >= g.ny) || (dir == 2 && k + 1 >= g.nz)) continue;
      const int64_t L = c + (dir == 0 ? 1 : dir == 1 ? g.nx : nxy);
      const double Ups = dir == 2 ? face_ups(P.h, kv[c], kv[L]) : face_ups(P.h, kh[c], kh[L]);
      const double dz = dir == 2 ? P.h : 0.0;
      for (int ph = 0; ph < 2; ++ph) v[ph] += -P.dt * face_value(P, Ups, dz, ph, s[c], p[c], s[L], p[L]);
    }
  }
  if (P.flags & PS_GEN_WELLS) {
    const int kind = well_kind(g, i, j);
    if (kind) {
      double wr[2], wd[2][2];
      well_terms(P, g, kind, k, kh[c], s[c], p[c], wr, wd);
      v[0] += wr[0];
      v[1] += wr[1];
    }
  }
  r[2 * c] = v[0];
  r[2 * c + 1] = v[1];
}

// state arrays of base + dx: s = s0 + dx_s, p = p0 + dx_p per cell
__global__ void k_state(int64_t nc, int64_t nu, const double* __restrict__ dx, const double* __restrict__ s0,
                        const double* __restrict__ p0, double* __restrict__ s, double* __restrict__ p) {
  const int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  s[c] = s0[c] + dx[nu + 2 * c];
  p[c] = p0[c] + dx[nu + 2 * c + 1];
}

// ---- Dirichlet elimination and scaling ----
__global__ void k_dirichlet_flags(Grid3 g, int64_t nn, uint8_t* __restrict__ dir, int on) {
  int64_t I = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (I >= nn) return;
  int64_t k = I / (int64_t(g.nx + 1) * (g.ny + 1));
  uint8_t f = (on && k == 0) ? 1 : 0;
  dir[3 * I] = f; dir[3 * I + 1] = f; dir[3 * I + 2] = f;
}

__global__ void k_zero_uu(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci, int64_t nn,
                          const uint8_t* __restrict__ dir, double* __restrict__ v) {
  int64_t I = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (I >= nn) return;
  for (int64_t q = rp[I]; q < rp[I + 1]; ++q) {
    int64_t J = ci[q];
    for (int d = 0; d < 3; ++d)
      for (int e = 0; e < 3; ++e)
        if (dir[3 * I + d] || dir[3 * J + e]) v[q * 9 + d * 3 + e] = 0.0;
  }
}
__global__ void k_zero_uf(const int64_t* __restrict__ rp, int64_t nn, const uint8_t* __restrict__ dir,
                          double* __restrict__ v) {
  int64_t I = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (I >= nn) return;
  for (int64_t q = rp[I]; q < rp[I + 1]; ++q)
    for (int d = 0; d < 3; ++d)
      if (dir[3 * I + d]) { v[q * 6 + d * 2] = 0.0; v[q * 6 + d * 2 + 1] = 0.0; }
}
__global__ void k_zero_fu(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci, int64_t nc,
                          const uint8_t* __restrict__ dir, double* __restrict__ v) {
  int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  for (int64_t q = rp[c]; q < rp[c + 1]; ++q) {
    int64_t J = ci[q];
    for (int e = 0; e < 3; ++e)
      if (dir[3 * J + e]) { v[q * 6 + e] = 0.0; v[q * 6 + 3 + e] = 0.0; }
  }
}

// per-dof diagonal of A_uu over free dofs (value, 1) or (0, 0)
__global__ void k_diag_uu(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci, int64_t nn,
                          const uint8_t* __restrict__ dir, const double* __restrict__ v, double* __restrict__ dv,
                          double* __restrict__ cnt) {
  int64_t I = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (I >= nn) return;
  int64_t q = rp[I];
  while (ci[q] != I) ++q;
  for (int d = 0; d < 3; ++d) {
    bool f = !dir[3 * I + d];
    dv[3 * I + d] = f ? v[q * 9 + d * 4] : 0.0;
    cnt[3 * I + d] = f ? 1.0 : 0.0;
  }
}
__global__ void k_diag_pp(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci, int64_t nc,
                          const double* __restrict__ v, double pcol, double* __restrict__ dv) {
  int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  int64_t q = rp[c];
  while (ci[q] != c) ++q;
  dv[c] = fabs(v[q * 4 + 3] * pcol);
}

// p-columns in MPa (x 1e6), then mechanics rows / alpha_u and flow rows / alpha_f: each value is multiplied
// once by the factor of its kind, fac[f_even] at even positions and fac[f_odd] at odd ones (every block's
// row length is even where the two differ)
__global__ void k_scale(double* __restrict__ v, int64_t nvals, const double* __restrict__ fac, int f_even,
                        int f_odd) {
  const double fe = fac[f_even], fo = fac[f_odd];
  const int64_t npair = nvals >> 1;
  double2* __restrict__ v2 = reinterpret_cast<double2*>(v);
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < npair; t += int64_t(gridDim.x) * blockDim.x) {
    double2 x = v2[t];
    x.x *= fe;
    x.y *= fo;
    v2[t] = x;
  }
  if ((nvals & 1) && blockIdx.x == 0 && threadIdx.x == 0) v[nvals - 1] *= fe;
}

__global__ void k_unit_diag(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci, int64_t nn,
                            const uint8_t* __restrict__ dir, double* __restrict__ v) {
  int64_t I = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (I >= nn) return;
  int64_t q = rp[I];
  while (ci[q] != I) ++q;
  for (int d = 0; d < 3; ++d)
    if (dir[3 * I + d]) v[q * 9 + d * 4] = 1.0;
}

__global__ void k_rhs(uint64_t seed, int64_t n, int64_t nu, const uint8_t* __restrict__ dir, double* __restrict__ b) {
  int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= n) return;
  b[r] = (r < nu && dir[r]) ? 0.0 : 2.0 * u01(seed, FRHS, 0, uint64_t(r)) - 1.0;
}

__global__ void k_alpha(const double* __restrict__ sums, double* __restrict__ alpha, double nc, double pcol) {
  // sums: [sum diag_u, count_u, sum |diag_pp|]; alpha[2..5]: the scaling factors 1/alpha_u, pcol/alpha_u,
  // 1/alpha_f, pcol/alpha_f
  alpha[0] = sums[1] > 0.0 ? sums[0] / sums[1] : 1.0;
  alpha[1] = sums[2] / nc;
  alpha[2] = 1.0 / alpha[0];
  alpha[3] = pcol / alpha[0];
  alpha[4] = 1.0 / alpha[1];
  alpha[5] = pcol / alpha[1];
}

}  // namespace

// ---------------------------------------------------------------------------
struct ps_system_impl {
  ps_system pub;
  Arena ar;
};

extern "C" {

void ps_gen_default(ps_gen_params* gp, int32_t config) {
  std::memset(gp, 0, sizeof(*gp));
  gp->h = 10.0;
  gp->seed = 1000 + uint64_t(config);
  gp->field_kind = config == 0 ? PS_FIELDS_LOGNORMAL : config == 2 ? PS_FIELDS_CHANNELS : PS_FIELDS_LAYERED;
  if (config == 0) { gp->nx = 8; gp->ny = 8; gp->nz = 4; }
  else if (config == 1) { gp->nx = 64; gp->ny = 64; gp->nz = 32; }
  else if (config == 2) { gp->nx = 60; gp->ny = 220; gp->nz = 85; }
  else { gp->nx = 16; gp->ny = 16; gp->nz = 8; }
  gp->flags = PS_GEN_ALL;
  gp->dt = 86400.0; gp->biot = 0.8;
  gp->c_w = gp->c_nw = gp->c_r = 1e-9;
  gp->mu_w = 1e-3; gp->mu_nw = 5e-3;
  gp->rho_w0 = 1035.0; gp->rho_nw0 = 863.0; gp->rho_s0 = 2650.0;
  gp->s_wr = 0.2; gp->s_nwr = 0.2;
  gp->grav = 9.81; gp->p_ref = 20e6; gp->dp_amp = 5e6; gp->corey = 2.0;
  gp->E0 = 1e10; gp->nu0 = 0.25; gp->kappa0 = 100.0 * kMD; gp->phi0 = 0.2; gp->sw0 = 0.5;
}

// Phys of the generator's parameters
// streaming multiprocessors of the current device (grid sizes of the grid-stride kernels)
static int num_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms < 1)
    sms = 1;
  return sms;
}

static Phys phys_of(const ps_gen_params* gp) {
  Phys P;
  P.dt = gp->dt; P.b = gp->biot; P.c_w = gp->c_w; P.c_nw = gp->c_nw; P.c_r = gp->c_r; P.mu_w = gp->mu_w;
  P.mu_nw = gp->mu_nw; P.rho_w0 = gp->rho_w0; P.rho_nw0 = gp->rho_nw0; P.rho_s0 = gp->rho_s0; P.s_wr = gp->s_wr;
  P.s_nwr = gp->s_nwr; P.grav = gp->grav; P.p_ref = gp->p_ref; P.corey = gp->corey; P.h = gp->h; P.flags = gp->flags;
  P.fs_modulus = gp->fs_modulus;
  P.inv_den = 1.0 / (1.0 - gp->s_wr - gp->s_nwr);
  P.inv_mu_w = 1.0 / gp->mu_w;
  P.inv_mu_nw = 1.0 / gp->mu_nw;
  return P;
}

// block patterns of the four Jacobian blocks and the Dirichlet flags (base nodes)
static ps_status alloc_patterns(ps_system_impl* S, cudaStream_t st) {
  Arena& ar = S->ar;
  ps_system& o = S->pub;
  Grid3 g{o.grid.nx, o.grid.ny, o.grid.nz};
  const int64_t nn = o.n_nodes, nc = o.n_cells;
  ps_bsr* blocks[4] = {&o.jac.A_uu, &o.jac.A_uf, &o.jac.A_fu, &o.jac.A_ff};
  int64_t rows[4] = {nn, nn, nc, nc}, cols[4] = {nn, nc, nn, nc};
  int br[4] = {3, 3, 2, 2}, bc[4] = {3, 2, 3, 2};
  int32_t* cnt;
  PS_TRY(ar.alloc(&cnt, nn > nc ? nn : nc));
  for (int kind = 0; kind < 4; ++kind) {
    ps_bsr& B = *blocks[kind];
    int64_t* rp;
    int32_t* ci;
    double* v;
    PS_TRY(ar.alloc(&rp, rows[kind] + 1));
    PS_TICK(); k_pattern_count<<<grid_for(rows[kind], 256), 256, 0, st>>>(g, kind, rows[kind], cnt);
    int64_t nnzb = 0;
    PS_TRY(scan_i64(ar, cnt, rp, rows[kind], &nnzb, st));
    PS_TRY(ar.alloc(&ci, nnzb));
    PS_TRY(ar.alloc(&v, nnzb * br[kind] * bc[kind]));
    PS_TICK(); k_pattern_fill<<<grid_for(rows[kind], 256), 256, 0, st>>>(g, kind, rows[kind], rp, ci);
    B.n_brow = rows[kind]; B.n_bcol = cols[kind]; B.nnzb = nnzb; B.br = br[kind]; B.bc = bc[kind];
    B.rowptr = rp; B.colind = ci; B.val = v;
  }
  ar.release(cnt);
  double* dfs;
  PS_TRY(ar.alloc(&dfs, 2 * nc));
  o.jac.d_fs = dfs;
  uint8_t* dir;
  PS_TRY(ar.alloc(&dir, 3 * nn));
  o.jac.dirichlet_u = dir;
  return PS_OK;
}

// The Jacobian values of the system's patterns at the state (cell saturation s, pressure p, element-mean
// volumetric strain ev; ev = NULL: zero strain): App. B blocks, Dirichlet elimination of the base nodes,
// block-row scaling (alpha_u, alpha_f from these values; pressure columns in MPa), unit Dirichlet diagonal.
static ps_status assemble_values(const ps_gen_params* gp, cudaStream_t st, ps_system_impl* S, const double* s_state,
                                 const double* p_state, const double* ev) {
  Arena& ar = S->ar;
  ps_system& o = S->pub;
  Grid3 g{o.grid.nx, o.grid.ny, o.grid.nz};
  const int64_t nn = o.n_nodes, nc = o.n_cells;
  const Phys P = phys_of(gp);
  CellMat* M;
  PS_TRY(ar.alloc(&M, nc));
  PS_TICK(); k_material<<<grid_for(nc, 256), 256, 0, st>>>(P, nc, o.E, o.nu, o.phi0, s_state, p_state, ev, M);
  Ref hR;
  build_ref(gp->h, &hR);
  Ref* dR;
  PS_TRY(ar.alloc(&dR, 1));
  PS_CUDA(cudaMemcpyAsync(dR, &hR, sizeof(Ref), cudaMemcpyHostToDevice, st));
  double* vuu = const_cast<double*>(o.jac.A_uu.val);
  double* vuf = const_cast<double*>(o.jac.A_uf.val);
  double* vfu = const_cast<double*>(o.jac.A_fu.val);
  double* vff = const_cast<double*>(o.jac.A_ff.val);
  double* dfs = const_cast<double*>(o.jac.d_fs);
  uint8_t* dir = const_cast<uint8_t*>(o.jac.dirichlet_u);
  PS_TICK(); k_values_uu<<<grid_for(nn, 128), 128, 0, st>>>(g, P, dR, M, o.jac.A_uu.rowptr, nn, vuu);
  PS_TICK(); k_values_uf<<<grid_for(nn, 128), 128, 0, st>>>(g, P, dR, M, o.jac.A_uf.rowptr, o.jac.A_uf.colind, nn, vuf);
  PS_TICK(); k_values_fu<<<grid_for(nc, 128), 128, 0, st>>>(g, P, dR, M, s_state, o.jac.A_fu.rowptr, o.jac.A_fu.colind,
                                                         nc, vfu);
  PS_TICK(); k_values_ff<<<grid_for(nc, 128), 128, 0, st>>>(g, P, M, s_state, p_state, o.kh, o.kv, o.jac.A_ff.rowptr,
                                                         o.jac.A_ff.colind, nc, vff, dfs);
  PS_CUDA(cudaGetLastError());
  // Dirichlet elimination (base nodes)
  PS_TICK(); k_dirichlet_flags<<<grid_for(nn, 256), 256, 0, st>>>(g, nn, dir, (gp->flags & PS_GEN_DIRICHLET) ? 1 : 0);
  PS_TICK(); k_zero_uu<<<grid_for(nn, 128), 128, 0, st>>>(o.jac.A_uu.rowptr, o.jac.A_uu.colind, nn, dir, vuu);
  PS_TICK(); k_zero_uf<<<grid_for(nn, 256), 256, 0, st>>>(o.jac.A_uf.rowptr, nn, dir, vuf);
  PS_TICK(); k_zero_fu<<<grid_for(nc, 256), 256, 0, st>>>(o.jac.A_fu.rowptr, o.jac.A_fu.colind, nc, dir, vfu);
  double* alpha;  // [alpha_u, alpha_f, then the four scaling factors of k_alpha]
  PS_TRY(ar.alloc(&alpha, 6));
  double one2[2] = {1.0, 1.0};
  PS_CUDA(cudaMemcpyAsync(alpha, one2, sizeof(one2), cudaMemcpyHostToDevice, st));
  if (gp->flags & PS_GEN_SCALE) {
    double *dv, *cv, *sums;
    PS_TRY(ar.alloc(&dv, 3 * nn)); PS_TRY(ar.alloc(&cv, 3 * nn)); PS_TRY(ar.alloc(&sums, 3));
    PS_TICK(); k_diag_uu<<<grid_for(nn, 256), 256, 0, st>>>(o.jac.A_uu.rowptr, o.jac.A_uu.colind, nn, dir, vuu, dv, cv);
    PS_TRY(sum_f64(ar, dv, 3 * nn, sums + 0, st));
    PS_TRY(sum_f64(ar, cv, 3 * nn, sums + 1, st));
    PS_TICK(); k_diag_pp<<<grid_for(nc, 256), 256, 0, st>>>(o.jac.A_ff.rowptr, o.jac.A_ff.colind, nc, vff, 1e6, dv);
    PS_TRY(sum_f64(ar, dv, nc, sums + 2, st));
    PS_TICK(); k_alpha<<<1, 1, 0, st>>>(sums, alpha, double(nc), 1e6);
    // A_uu: mechanics rows; A_uf: mechanics rows, columns (s, p); A_fu: flow rows; A_ff: flow rows, columns
    // (s, p); d_fs: flow rows, p columns
    const int sgrid = 4 * num_sms();
    PS_TICK(); k_scale<<<sgrid, 256, 0, st>>>(vuu, o.jac.A_uu.nnzb * 9, alpha + 2, 0, 0);
    PS_TICK(); k_scale<<<sgrid, 256, 0, st>>>(vuf, o.jac.A_uf.nnzb * 6, alpha + 2, 0, 1);
    PS_TICK(); k_scale<<<sgrid, 256, 0, st>>>(vfu, o.jac.A_fu.nnzb * 6, alpha + 2, 2, 2);
    PS_TICK(); k_scale<<<sgrid, 256, 0, st>>>(vff, o.jac.A_ff.nnzb * 4, alpha + 2, 2, 3);
    PS_TICK(); k_scale<<<sgrid, 256, 0, st>>>(dfs, 2 * nc, alpha + 2, 3, 3);
    PS_CUDA(cudaGetLastError());
    ar.release(dv); ar.release(cv); ar.release(sums);
  }
  PS_TICK(); k_unit_diag<<<grid_for(nn, 256), 256, 0, st>>>(o.jac.A_uu.rowptr, o.jac.A_uu.colind, nn, dir, vuu);
  PS_CUDA(cudaGetLastError());
  double ha[2];
  PS_CUDA(cudaMemcpyAsync(ha, alpha, sizeof(ha), cudaMemcpyDeviceToHost, st));
  PS_CUDA(cudaStreamSynchronize(st));
  o.alpha_u = ha[0]; o.alpha_f = ha[1];
  ar.release(M); ar.release(dR); ar.release(alpha);
  return PS_OK;
}

static ps_status generate_impl(const ps_gen_params* gp, cudaStream_t st, ps_system_impl* S) {
  Arena& ar = S->ar;
  ar.stream = st;
  ps_system& o = S->pub;
  int64_t nn = int64_t(gp->nx + 1) * (gp->ny + 1) * (gp->nz + 1);
  int64_t nc = int64_t(gp->nx) * gp->ny * gp->nz;
  o.grid.nx = gp->nx; o.grid.ny = gp->ny; o.grid.nz = gp->nz;
  o.grid.hx = o.grid.hy = o.grid.hz = gp->h;
  o.n_nodes = nn; o.n_cells = nc; o.n_u = 3 * nn; o.n_f = 2 * nc; o.n = o.n_u + o.n_f;
  // fields
  double *E, *nu, *kh, *kv, *phi, *sw, *p;
  PS_TRY(ar.alloc(&E, nc)); PS_TRY(ar.alloc(&nu, nc)); PS_TRY(ar.alloc(&kh, nc)); PS_TRY(ar.alloc(&kv, nc));
  PS_TRY(ar.alloc(&phi, nc)); PS_TRY(ar.alloc(&sw, nc)); PS_TRY(ar.alloc(&p, nc));
  double *ghat, *ksm = nullptr, *swsm = nullptr;
  PS_TRY(ar.alloc(&ghat, nc));
  PS_TRY(correlated(ar, gp->seed, FDP, gp->nx, gp->ny, gp->nz, 10, 10, 3, ghat, st));
  if (gp->field_kind == PS_FIELDS_LAYERED || gp->field_kind == PS_FIELDS_CHANNELS) {
    PS_TRY(ar.alloc(&ksm, nc)); PS_TRY(ar.alloc(&swsm, nc));
    PS_TRY(correlated(ar, gp->seed, FKAP, gp->nx, gp->ny, gp->nz, 20, 20, 2, ksm, st));
    PS_TRY(correlated(ar, gp->seed, FSW, gp->nx, gp->ny, gp->nz, 10, 10, 3, swsm, st));
  }
  FieldArgs fa;
  std::memset(&fa, 0, sizeof(fa));
  fa.nx = gp->nx; fa.ny = gp->ny; fa.nz = gp->nz; fa.kind = gp->field_kind; fa.seed = gp->seed;
  fa.h = gp->h; fa.grav = (gp->flags & PS_GEN_GRAVITY) ? gp->grav : 0.0; fa.rho_w0 = gp->rho_w0;
  fa.p_ref = gp->p_ref; fa.dp_amp = gp->dp_amp;
  fa.E0 = gp->E0; fa.nu0 = gp->nu0; fa.kappa0 = gp->kappa0; fa.phi0 = gp->phi0; fa.sw0 = gp->sw0;
  fa.n_low = (gp->nz * 50 + 42) / 85;
  if (gp->field_kind == PS_FIELDS_CHANNELS) {
    fa.nch = 12;
    for (int c = 0; c < 12; ++c) {
      Channel& C = fa.ch[c];
      C.x0 = double(gp->nx) * u01(gp->seed, FCHAN, 0, lat3(c, 0, 0));
      C.A = 5.0 + 10.0 * u01(gp->seed, FCHAN, 0, lat3(c, 1, 0));
      C.lam = 40.0 + 70.0 * u01(gp->seed, FCHAN, 0, lat3(c, 2, 0));
      C.ph = 2.0 * kPiG * u01(gp->seed, FCHAN, 0, lat3(c, 3, 0));
      int width = 4 + int(std::floor(5.0 * u01(gp->seed, FCHAN, 0, lat3(c, 4, 0))));
      C.halfw = 0.5 * width;
      C.thick = 5 + int(std::floor(6.0 * u01(gp->seed, FCHAN, 0, lat3(c, 5, 0))));
      int room = fa.n_low - C.thick + 1;
      C.k0 = room > 0 ? int(std::floor(double(room) * u01(gp->seed, FCHAN, 0, lat3(c, 6, 0)))) : 0;
      C.logk = std::log(1e3) + std::log(10.0) * u01(gp->seed, FCHAN, 0, lat3(c, 7, 0));
    }
  }
  PS_TICK(); k_fields<<<grid_for(nc, 256), 256, 0, st>>>(fa, ghat, ksm, swsm, E, nu, kh, kv, phi, sw, p);
  PS_CUDA(cudaGetLastError());
  o.E = E; o.nu = nu; o.kh = kh; o.kv = kv; o.phi0 = phi; o.sw = sw; o.p = p;
  PS_TRY(alloc_patterns(S, st));
  PS_TRY(assemble_values(gp, st, S, sw, p, nullptr));
  double* rhs;
  PS_TRY(ar.alloc(&rhs, o.n));
  PS_TICK(); k_rhs<<<grid_for(o.n, 256), 256, 0, st>>>(gp->seed, o.n, o.n_u, o.jac.dirichlet_u, rhs);
  PS_CUDA(cudaGetLastError());
  o.rhs = rhs;
  ar.release(ghat);
  if (ksm) ar.release(ksm);
  if (swsm) ar.release(swsm);
  PS_CUDA(cudaStreamSynchronize(st));
  return PS_OK;
}

// the well index needs a cell wider than the wellbore: Peaceman's radius 0.28 sqrt(2) h / 2 above 0.1524 m
static bool wells_ok(const ps_gen_params* gp) {
  if (!(gp->flags & PS_GEN_WELLS) || 0.28 * std::sqrt(2.0) * gp->h / 2.0 > 0.1524) return true;
  set_reason("Peaceman wells need cells wider than the wellbore (h > 0.77 m), h = %g", gp->h);
  return false;
}

ps_status ps_generate(const ps_gen_params* gp, void* stream, ps_system** out) {
  if (!gp || !out || gp->nx < 1 || gp->ny < 1 || gp->nz < 1 || !(gp->h > 0.0)) return PS_ERR_INVALID;
  if (!wells_ok(gp)) return PS_ERR_INVALID;
  if (int64_t(gp->nx + 1) * (gp->ny + 1) * (gp->nz + 1) * 27 >= (int64_t(1) << 31)) return PS_ERR_INVALID;
  ps_system_impl* S = new ps_system_impl();
  std::memset(&S->pub, 0, sizeof(S->pub));
  ps_status st = generate_impl(gp, (cudaStream_t)stream, S);
  if (st != PS_OK) {
    S->ar.free_all();
    cudaStreamSynchronize((cudaStream_t)stream);
    delete S;
    *out = nullptr;
    return st;
  }
  *out = &S->pub;
  return PS_OK;
}

// residual (and with jac != 0 the Jacobian values) of a generated system at the state base + dx
static ps_status state_impl(const ps_gen_params* gp, ps_system* sys, const double* dx, double* r, bool jac,
                            cudaStream_t st) {
  if (!gp || !sys || !dx || (!r && !jac)) return PS_ERR_INVALID;
  if (!wells_ok(gp)) return PS_ERR_INVALID;
  ps_system_impl* S = reinterpret_cast<ps_system_impl*>(sys);
  ps_system& o = S->pub;
  if (o.grid.nx != gp->nx || o.grid.ny != gp->ny || o.grid.nz != gp->nz || o.grid.hx != gp->h) {
    set_reason("ps_assemble_at: the system was not generated with these parameters");
    return PS_ERR_INVALID;
  }
  Arena& ar = S->ar;
  ar.stream = st;
  const Grid3 g{o.grid.nx, o.grid.ny, o.grid.nz};
  const int64_t nc = o.n_cells, nn = o.n_nodes;
  double *s_st, *p_st, *ev;
  PS_TRY(ar.alloc(&s_st, nc)); PS_TRY(ar.alloc(&p_st, nc)); PS_TRY(ar.alloc(&ev, nc));
  Ref hR;
  build_ref(gp->h, &hR);
  Ref* dR;
  PS_TRY(ar.alloc(&dR, 1));
  PS_CUDA(cudaMemcpyAsync(dR, &hR, sizeof(Ref), cudaMemcpyHostToDevice, st));
  PS_TICK(); k_state<<<grid_for(nc, 256), 256, 0, st>>>(nc, 3 * nn, dx, o.sw, o.p, s_st, p_st);
  PS_TICK(); k_mean_epsv<<<grid_for(nc, 256), 256, 0, st>>>(g, dR, dx, gp->h, ev);
  PS_CUDA(cudaGetLastError());
  if (jac) PS_TRY(assemble_values(gp, st, S, s_st, p_st, ev));
  if (r) {
    const Phys P = phys_of(gp);
    double *er, *rf;
    PS_TRY(ar.alloc(&er, nc * 24)); PS_TRY(ar.alloc(&rf, 2 * nc));
    PS_TICK(); k_res_elem<<<grid_for(nc, 128), 128, 0, st>>>(g, P, dR, o.E, o.nu, o.phi0, dx, s_st, p_st, o.sw, o.p, er,
                                                          rf);
    PS_TICK(); k_res_nodes<<<grid_for(nn, 256), 256, 0, st>>>(g, er, o.jac.dirichlet_u, r);
    PS_TICK(); k_res_cells<<<grid_for(nc, 256), 256, 0, st>>>(g, P, o.kh, o.kv, s_st, p_st, rf, r + 3 * nn);
    PS_CUDA(cudaGetLastError());
    ar.release(er); ar.release(rf);
  }
  ar.release(s_st); ar.release(p_st); ar.release(ev); ar.release(dR);
  PS_CUDA(cudaStreamSynchronize(st));
  return PS_OK;
}

ps_status ps_assemble_at(const ps_gen_params* gp, ps_system* sys, const double* dx, double* r, void* stream) {
  return state_impl(gp, sys, dx, r, true, (cudaStream_t)stream);
}

ps_status ps_residual_at(const ps_gen_params* gp, ps_system* sys, const double* dx, double* r, void* stream) {
  return state_impl(gp, sys, dx, r, false, (cudaStream_t)stream);
}

void ps_system_free(ps_system* s) {
  if (!s) return;
  ps_system_impl* S = reinterpret_cast<ps_system_impl*>(s);
  S->ar.free_all();
  cudaStreamSynchronize(S->ar.stream);
  delete S;
}

}  // extern "C"
