// Plain FP64 CPU oracle for arXiv 1812.05540 (two-stage fixed-stress / CPR
// preconditioner for multiphase poromechanics).
//
// TEST INFRASTRUCTURE ONLY: the product (the CUDA library and its binding)
// never includes, links or calls this file.  It is deliberately slow and
// literal: every routine restates one passage of the paper (cited inline) in
// the order the paper states it, with no blocking, fusion or reordering.
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -fPIC -shared (see __init__.py), and
// a second build of the same source with -fopenmp, whose row loops run on all
// host cores.  Every sum over a vector is taken in fixed chunks (dot below) and
// every row's arithmetic is done by one thread in the order written, so the
// two builds return bit-identical results.
// -ffp-contract=off keeps every a*b+c as two roundings so that the integer
// decisions taken from floating point (strength of connection, aggregation)
// are reproducible on x86 and Arm hosts.
#include "oracle.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

typedef std::vector<double> vec;
const double kMilliDarcy = 9.869233e-16;  // m^2
const double kPi = 3.14159265358979323846;

// Inner product sum_e a[e] b[e] taken in fixed chunks of kChunk entries: each chunk is summed in index
// order, then the chunk sums are added in chunk order.  The chunking does not depend on the thread count.
const int64_t kChunk = 4096;
double dot(const double* a, const double* b, int64_t n) {
  const int64_t nch = (n + kChunk - 1) / kChunk;
  vec part(size_t(nch), 0.0);
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < nch; ++k) {
    double s = 0.0;
    const int64_t e1 = std::min(n, (k + 1) * kChunk);
    for (int64_t e = k * kChunk; e < e1; ++e) s += a[e] * b[e];
    part[k] = s;
  }
  double s = 0.0;
  for (int64_t k = 0; k < nch; ++k) s += part[k];
  return s;
}

// Row ranges for loops whose rows produce a variable number of outputs: rows [lo(t), lo(t+1)) form task t.
// Tasks are filled independently and concatenated in task order, so the result does not depend on how
// tasks are spread over threads.
const int kTasks = 64;
inline int64_t task_lo(int64_t n, int t) { return n * t / kTasks; }

// ---------------------------------------------------------------------------
// Counter-based random numbers: splitmix64 (S. Vigna), used as a pure
// function of a 64-bit counter so that any lattice point can be drawn alone.
// ---------------------------------------------------------------------------
inline uint64_t sm64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
inline uint64_t lattice(int64_t i, int64_t j, int64_t k) {
  const int64_t off = int64_t(1) << 17;
  return uint64_t(i + off) | (uint64_t(j + off) << 18) | (uint64_t(k + off) << 36);
}
inline uint64_t rbits(uint64_t seed, int field, int sub, uint64_t idx) {
  return sm64(sm64(seed) ^ (uint64_t(field) << 55) ^ (uint64_t(sub) << 54) ^ idx);
}
inline double unif(uint64_t seed, int field, int sub, uint64_t idx) {
  return double(rbits(seed, field, sub, idx) >> 11) * 0x1.0p-53;
}
// Box-Muller from two independent uniforms of the same counter
inline double gauss(uint64_t seed, int field, uint64_t idx) {
  double u0 = unif(seed, field, 0, idx), u1 = unif(seed, field, 1, idx);
  return std::sqrt(-2.0 * std::log(1.0 - u0)) * std::cos(2.0 * kPi * u1);
}
enum { F_E = 1, F_NU = 2, F_KAPPA = 3, F_PHI = 4, F_SW = 5, F_DP = 6, F_ELAYER = 7,
       F_CHANNEL = 8, F_RHS = 9 };

// Unit-variance Gaussian random field on the cells: white noise on the integer
// lattice (padded by the kernel radius) convolved separably with
// exp(-(d/L)^2/2), |d| <= 3L, then divided by the kernel's L2 norm.
vec correlated_field(uint64_t seed, int field, int nx, int ny, int nz, int Lx, int Ly, int Lz) {
  int R[3] = {3 * Lx, 3 * Ly, 3 * Lz};
  int L[3] = {Lx, Ly, Lz};
  std::vector<vec> w(3);
  double norm = 1.0;
  for (int a = 0; a < 3; ++a) {
    double s2 = 0.0;
    for (int d = -R[a]; d <= R[a]; ++d) {
      double t = double(d) / double(L[a]);
      w[a].push_back(std::exp(-0.5 * t * t));
      s2 += w[a].back() * w[a].back();
    }
    norm *= std::sqrt(s2);
  }
  int px = nx + 2 * R[0], py = ny + 2 * R[1], pz = nz + 2 * R[2];
  vec W(size_t(px) * py * pz);
  for (int k = 0; k < pz; ++k)
    for (int j = 0; j < py; ++j)
      for (int i = 0; i < px; ++i)
        W[(size_t(k) * py + j) * px + i] = gauss(seed, field, lattice(i - R[0], j - R[1], k - R[2]));
  // x pass: output i in [0,nx), padded j,k
  vec X(size_t(nx) * py * pz, 0.0);
  for (int k = 0; k < pz; ++k)
    for (int j = 0; j < py; ++j)
      for (int i = 0; i < nx; ++i) {
        double s = 0.0;
        for (int d = -R[0]; d <= R[0]; ++d)
          s += w[0][d + R[0]] * W[(size_t(k) * py + j) * px + (i + R[0] - d)];
        X[(size_t(k) * py + j) * nx + i] = s;
      }
  vec Y(size_t(nx) * ny * pz, 0.0);
  for (int k = 0; k < pz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double s = 0.0;
        for (int d = -R[1]; d <= R[1]; ++d)
          s += w[1][d + R[1]] * X[(size_t(k) * py + (j + R[1] - d)) * nx + i];
        Y[(size_t(k) * ny + j) * nx + i] = s;
      }
  vec Z(size_t(nx) * ny * nz, 0.0);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double s = 0.0;
        for (int d = -R[2]; d <= R[2]; ++d)
          s += w[2][d + R[2]] * Y[(size_t(k + R[2] - d) * ny + j) * nx + i];
        Z[(size_t(k) * ny + j) * nx + i] = s / norm;
      }
  return Z;
}

// ---------------------------------------------------------------------------
// Cell fields and the linearisation state (§6 constitutive models; the
// synthetic statistics stand in for the paper's staircase / SPE10 inputs).
// ---------------------------------------------------------------------------
struct Fields {
  int nx, ny, nz;
  vec E, nu, kh, kv, phi0, sw, p;
};

Fields make_fields(const or_gen_params& gp) {
  Fields f;
  f.nx = gp.nx; f.ny = gp.ny; f.nz = gp.nz;
  int nx = gp.nx, ny = gp.ny, nz = gp.nz;
  size_t nc = size_t(nx) * ny * nz;
  f.E.resize(nc); f.nu.resize(nc); f.kh.resize(nc); f.kv.resize(nc);
  f.phi0.resize(nc); f.sw.resize(nc); f.p.resize(nc);
  uint64_t sd = gp.seed;
  vec ghat = correlated_field(sd, F_DP, nx, ny, nz, 10, 10, 3);
  vec ksm, swsm;
  if (gp.field_kind == OR_FIELDS_LAYERED || gp.field_kind == OR_FIELDS_CHANNELS) {
    ksm = correlated_field(sd, F_KAPPA, nx, ny, nz, 20, 20, 2);
    swsm = correlated_field(sd, F_SW, nx, ny, nz, 10, 10, 3);
  }
  // channel geometry (channelised lower layers)
  int n_low = (nz * 50 + 42) / 85;
  struct Ch { double x0, A, lam, ph, halfw, logk; int k0, thick; };
  std::vector<Ch> ch;
  if (gp.field_kind == OR_FIELDS_CHANNELS) {
    for (int c = 0; c < 12; ++c) {
      Ch q;
      q.x0 = double(nx) * unif(sd, F_CHANNEL, 0, lattice(c, 0, 0));
      q.A = 5.0 + 10.0 * unif(sd, F_CHANNEL, 0, lattice(c, 1, 0));
      q.lam = 40.0 + 70.0 * unif(sd, F_CHANNEL, 0, lattice(c, 2, 0));
      q.ph = 2.0 * kPi * unif(sd, F_CHANNEL, 0, lattice(c, 3, 0));
      int width = 4 + int(std::floor(5.0 * unif(sd, F_CHANNEL, 0, lattice(c, 4, 0))));
      q.halfw = 0.5 * width;
      q.thick = 5 + int(std::floor(6.0 * unif(sd, F_CHANNEL, 0, lattice(c, 5, 0))));
      int room = n_low - q.thick + 1;
      q.k0 = room > 0 ? int(std::floor(double(room) * unif(sd, F_CHANNEL, 0, lattice(c, 6, 0)))) : 0;
      q.logk = std::log(1e3) + std::log(10.0) * unif(sd, F_CHANNEL, 0, lattice(c, 7, 0));
      ch.push_back(q);
    }
  }
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t c = (size_t(k) * ny + j) * nx + i;
        uint64_t L = lattice(i, j, k);
        double E, nu, kh, kv, phi, sw;
        switch (gp.field_kind) {
          case OR_FIELDS_LOGNORMAL: {
            E = std::exp(std::log(1e10) - 0.5 * 0.25 + 0.5 * gauss(sd, F_E, L));
            nu = 0.2 + 0.1 * unif(sd, F_NU, 0, L);
            kh = std::exp(std::log(100.0 * kMilliDarcy) - 0.5 + gauss(sd, F_KAPPA, L));
            kv = kh;
            phi = 0.15 + 0.1 * unif(sd, F_PHI, 0, L);
            sw = 0.2 + 0.6 * unif(sd, F_SW, 0, L);
            break;
          }
          case OR_FIELDS_LAYERED:
          case OR_FIELDS_CHANNELS: {
            if (gp.field_kind == OR_FIELDS_LAYERED) {
              E = std::exp(std::log(1e9) + std::log(50.0) * unif(sd, F_ELAYER, 0, lattice(0, 0, k)));
              kh = 100.0 * kMilliDarcy * std::exp(2.0 * ksm[c]);
            } else {
              E = std::exp(std::log(0.5e9) + std::log(100.0) * unif(sd, F_E, 0, L));
              if (k < n_low) {
                double best = std::log(1e-2);
                for (const Ch& q : ch) {
                  if (k < q.k0 || k >= q.k0 + q.thick) continue;
                  double xc = q.x0 + q.A * std::sin(2.0 * kPi * (j + 0.5) / q.lam + q.ph);
                  if (std::fabs((i + 0.5) - xc) <= q.halfw) best = std::max(best, q.logk);
                }
                kh = std::exp(best) * kMilliDarcy;
              } else {
                kh = 100.0 * kMilliDarcy * std::exp(2.5 * ksm[c]);
              }
            }
            kv = 0.1 * kh;
            nu = 0.2 + 0.1 * unif(sd, F_NU, 0, L);
            phi = 0.15 + 0.1 * unif(sd, F_PHI, 0, L);
            sw = 0.2 + 0.6 * (0.5 * std::erfc(-swsm[c] / std::sqrt(2.0)));
            break;
          }
          default: {
            E = gp.E0; nu = gp.nu0; kh = gp.kappa0; kv = gp.kappa0; phi = gp.phi0; sw = gp.sw0;
          }
        }
        f.E[c] = E; f.nu[c] = nu; f.kh[c] = kh; f.kv[c] = kv; f.phi0[c] = phi; f.sw[c] = sw;
        double g = (gp.flags & OR_GRAVITY) ? gp.grav : 0.0;
        double zc = (k + 0.5) * gp.h, ztop = nz * gp.h;
        f.p[c] = gp.p_ref + gp.rho_w0 * g * (ztop - zc) + gp.dp_amp * std::tanh(ghat[c]);
      }
  return f;
}

// Constitutive quantities of one cell at state (s, p, mean volumetric strain).
struct Mat {
  double lam, G, Kdr, dphidp, phi, rw, rnw, rs, drho_deps, drho_dp, drho_ds;
  double krw, krnw, dkrw, dkrnw;  // relative permeabilities and d/ds
};

void relperm(const or_gen_params& gp, double s, double* krw, double* krnw, double* dkrw, double* dkrnw) {
  double den = 1.0 - gp.s_wr - gp.s_nwr;
  double sh = (s - gp.s_wr) / den;
  bool inside = sh > 0.0 && sh < 1.0;
  sh = std::min(1.0, std::max(0.0, sh));
  double n = gp.corey;
  if (n == 2.0) {
    *krw = sh * sh; *krnw = (1.0 - sh) * (1.0 - sh);
    *dkrw = inside ? 2.0 * sh / den : 0.0;
    *dkrnw = inside ? -2.0 * (1.0 - sh) / den : 0.0;
  } else if (n == 1.0) {
    *krw = sh; *krnw = 1.0 - sh;
    *dkrw = inside ? 1.0 / den : 0.0;
    *dkrnw = inside ? -1.0 / den : 0.0;
  } else {
    *krw = std::pow(sh, n); *krnw = std::pow(1.0 - sh, n);
    *dkrw = inside ? n * std::pow(sh, n - 1.0) / den : 0.0;
    *dkrnw = inside ? -n * std::pow(1.0 - sh, n - 1.0) / den : 0.0;
  }
}

// Eq. (4) porosity law, §6 density law, §2 mixture density and App. B
// derivatives of the mixture density.
Mat material(const or_gen_params& gp, double E, double nu, double phi0, double s, double p,
             double epsv_mean) {
  Mat m;
  double b = gp.biot;
  m.lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  m.G = E / (2.0 * (1.0 + nu));
  m.Kdr = E / (3.0 * (1.0 - 2.0 * nu));
  m.dphidp = (b - phi0) * (1.0 - b) / m.Kdr;
  double dp = p - gp.p_ref;
  m.phi = phi0 + b * epsv_mean + m.dphidp * dp;
  m.rw = gp.rho_w0 * (1.0 + gp.c_w * dp);
  m.rnw = gp.rho_nw0 * (1.0 + gp.c_nw * dp);
  m.rs = gp.rho_s0 * (1.0 + gp.c_r * dp);
  double B = -m.rs + s * m.rw + (1.0 - s) * m.rnw;
  m.drho_deps = B * b;
  m.drho_dp = B * m.dphidp + (1.0 - m.phi) * gp.rho_s0 * gp.c_r + s * m.phi * gp.rho_w0 * gp.c_w +
              (1.0 - s) * m.phi * gp.rho_nw0 * gp.c_nw;
  m.drho_ds = m.phi * (m.rw - m.rnw);
  relperm(gp, s, &m.krw, &m.krnw, &m.dkrw, &m.dkrnw);
  return m;
}

// ---------------------------------------------------------------------------
// Q1 reference integrals on a cube of edge h, 2x2x2 Gauss (exact here).
// Local node a = (ax, ay, az) with ax = a&1, ay = (a>>1)&1, az = (a>>2)&1.
// ---------------------------------------------------------------------------
struct RefInt {
  double G[8][8][3][3], IN[8], IdN[8][3], INdN[8][8][3];
  double gp_N[8][8], gp_dN[8][8][3], gp_w;  // [gauss pt][node]
};
RefInt ref_integrals(double h) {
  RefInt R;
  std::memset(&R, 0, sizeof(R));
  double g[2] = {0.5 - 0.5 / std::sqrt(3.0), 0.5 + 0.5 / std::sqrt(3.0)};
  R.gp_w = h * h * h / 8.0;
  for (int q = 0; q < 8; ++q) {
    double xi[3] = {g[q & 1], g[(q >> 1) & 1], g[(q >> 2) & 1]};
    for (int a = 0; a < 8; ++a) {
      int ad[3] = {a & 1, (a >> 1) & 1, (a >> 2) & 1};
      double f[3], df[3];
      for (int d = 0; d < 3; ++d) {
        f[d] = ad[d] ? xi[d] : 1.0 - xi[d];
        df[d] = (ad[d] ? 1.0 : -1.0) / h;
      }
      R.gp_N[q][a] = f[0] * f[1] * f[2];
      R.gp_dN[q][a][0] = df[0] * f[1] * f[2];
      R.gp_dN[q][a][1] = f[0] * df[1] * f[2];
      R.gp_dN[q][a][2] = f[0] * f[1] * df[2];
    }
  }
  for (int q = 0; q < 8; ++q)
    for (int a = 0; a < 8; ++a) {
      R.IN[a] += R.gp_w * R.gp_N[q][a];
      for (int d = 0; d < 3; ++d) R.IdN[a][d] += R.gp_w * R.gp_dN[q][a][d];
      for (int b = 0; b < 8; ++b)
        for (int d = 0; d < 3; ++d) {
          R.INdN[a][b][d] += R.gp_w * R.gp_N[q][a] * R.gp_dN[q][b][d];
          for (int e = 0; e < 3; ++e) R.G[a][b][d][e] += R.gp_w * R.gp_dN[q][a][d] * R.gp_dN[q][b][e];
        }
    }
  return R;
}

// ---------------------------------------------------------------------------
// Block sparse storage and the structured patterns of §3 (Q1 nodes, P0 cells)
// ---------------------------------------------------------------------------
struct BSR {
  int64_t nbr = 0, nbc = 0;
  int br = 1, bc = 1;
  std::vector<int64_t> rp;
  std::vector<int32_t> ci;
  vec v;
  int64_t find(int64_t i, int64_t j) const {
    auto b = ci.begin() + rp[i], e = ci.begin() + rp[i + 1];
    auto it = std::lower_bound(b, e, int32_t(j));
    if (it == e || *it != j) return -1;
    return it - ci.begin();
  }
};

struct Grid {
  int nx, ny, nz;
  double h;
  int64_t nn() const { return int64_t(nx + 1) * (ny + 1) * (nz + 1); }
  int64_t ncell() const { return int64_t(nx) * ny * nz; }
  int64_t node(int i, int j, int k) const { return i + int64_t(nx + 1) * (j + int64_t(ny + 1) * k); }
  int64_t cell(int i, int j, int k) const { return i + int64_t(nx) * (j + int64_t(ny) * k); }
};

BSR pattern_uu(const Grid& g) {
  BSR A; A.nbr = A.nbc = g.nn(); A.br = A.bc = 3;
  A.rp.push_back(0);
  for (int k = 0; k <= g.nz; ++k)
    for (int j = 0; j <= g.ny; ++j)
      for (int i = 0; i <= g.nx; ++i) {
        for (int dk = -1; dk <= 1; ++dk)
          for (int dj = -1; dj <= 1; ++dj)
            for (int di = -1; di <= 1; ++di) {
              int a = i + di, b = j + dj, c = k + dk;
              if (a < 0 || b < 0 || c < 0 || a > g.nx || b > g.ny || c > g.nz) continue;
              A.ci.push_back(int32_t(g.node(a, b, c)));
            }
        A.rp.push_back(int64_t(A.ci.size()));
      }
  A.v.assign(A.ci.size() * 9, 0.0);
  return A;
}
BSR pattern_uf(const Grid& g) {
  BSR A; A.nbr = g.nn(); A.nbc = g.ncell(); A.br = 3; A.bc = 2;
  A.rp.push_back(0);
  for (int k = 0; k <= g.nz; ++k)
    for (int j = 0; j <= g.ny; ++j)
      for (int i = 0; i <= g.nx; ++i) {
        for (int dk = -1; dk <= 0; ++dk)
          for (int dj = -1; dj <= 0; ++dj)
            for (int di = -1; di <= 0; ++di) {
              int a = i + di, b = j + dj, c = k + dk;
              if (a < 0 || b < 0 || c < 0 || a >= g.nx || b >= g.ny || c >= g.nz) continue;
              A.ci.push_back(int32_t(g.cell(a, b, c)));
            }
        A.rp.push_back(int64_t(A.ci.size()));
      }
  A.v.assign(A.ci.size() * 6, 0.0);
  return A;
}
BSR pattern_fu(const Grid& g) {
  BSR A; A.nbr = g.ncell(); A.nbc = g.nn(); A.br = 2; A.bc = 3;
  A.rp.push_back(0);
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        for (int dk = 0; dk <= 1; ++dk)
          for (int dj = 0; dj <= 1; ++dj)
            for (int di = 0; di <= 1; ++di) A.ci.push_back(int32_t(g.node(i + di, j + dj, k + dk)));
        A.rp.push_back(int64_t(A.ci.size()));
      }
  A.v.assign(A.ci.size() * 6, 0.0);
  return A;
}
BSR pattern_ff(const Grid& g) {
  BSR A; A.nbr = A.nbc = g.ncell(); A.br = A.bc = 2;
  A.rp.push_back(0);
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        if (k > 0) A.ci.push_back(int32_t(g.cell(i, j, k - 1)));
        if (j > 0) A.ci.push_back(int32_t(g.cell(i, j - 1, k)));
        if (i > 0) A.ci.push_back(int32_t(g.cell(i - 1, j, k)));
        A.ci.push_back(int32_t(g.cell(i, j, k)));
        if (i + 1 < g.nx) A.ci.push_back(int32_t(g.cell(i + 1, j, k)));
        if (j + 1 < g.ny) A.ci.push_back(int32_t(g.cell(i, j + 1, k)));
        if (k + 1 < g.nz) A.ci.push_back(int32_t(g.cell(i, j, k + 1)));
        A.rp.push_back(int64_t(A.ci.size()));
      }
  A.v.assign(A.ci.size() * 4, 0.0);
  return A;
}

// Extra boundary conditions used only by the Terzaghi column.
struct ExtraBC {
  bool active = false;
  std::vector<uint8_t> dir_u;  // per displacement dof
  double sigma_top = 0.0;      // compressive load on the top face
  bool top_drained = false;    // Dirichlet flow face on top of the top cells
  double p_top = 0.0, s_top = 0.0;
};

struct State {  // linearisation point
  vec u;        // nodal displacement, 3 per node
  vec s, p;     // per cell
};

// mean volumetric strain of each element from nodal u (Q1, Gauss average)
vec mean_epsv(const Grid& g, const RefInt& R, const vec& u) {
  vec ev(g.ncell(), 0.0);
  if (u.empty()) return ev;
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        double s = 0.0;
        for (int a = 0; a < 8; ++a) {
          int64_t I = g.node(i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
          for (int d = 0; d < 3; ++d) s += R.IdN[a][d] * u[3 * I + d];
        }
        ev[g.cell(i, j, k)] = s / (g.h * g.h * g.h);
      }
  return ev;
}

struct Jac {
  BSR uu, uf, fu, ff;
  vec dfs;
  std::vector<uint8_t> dir;
  double alpha_u = 1.0, alpha_f = 1.0;
};

// Two-point flux of phase l across one interior face K|L (Eq. (8), Eq. (12),
// App. A transmissibility) and its derivatives (App. B, face Jacobian).
struct FaceFlux {
  double F, dF_dsK, dF_dsL, dF_dpK, dF_dpL;
};
FaceFlux face_flux(const or_gen_params& gp, double Ups, double dz, double g, int phase,
                   double sK, double pK, double sL, double pL, bool boundaryL) {
  double rho0 = phase == 0 ? gp.rho_w0 : gp.rho_nw0;
  double c = phase == 0 ? gp.c_w : gp.c_nw;
  double mu = phase == 0 ? gp.mu_w : gp.mu_nw;
  double rK = rho0 * (1.0 + c * (pK - gp.p_ref));
  double rL = rho0 * (1.0 + c * (pL - gp.p_ref));
  double satK = phase == 0 ? sK : 1.0 - sK;
  double satL = phase == 0 ? sL : 1.0 - sL;
  // Eq. (12): face density
  double varrho, dvK, dvL;
  if (satK > 0.0 && satL > 0.0) { varrho = 0.5 * (rK + rL); dvK = 0.5 * rho0 * c; dvL = 0.5 * rho0 * c; }
  else if (satK > 0.0) { varrho = rK; dvK = rho0 * c; dvL = 0.0; }
  else if (satL > 0.0) { varrho = rL; dvK = 0.0; dvL = rho0 * c; }
  else { varrho = 0.0; dvK = dvL = 0.0; }
  (void)boundaryL;
  double Phi = Ups * ((pL - pK) + varrho * g * dz);
  bool upL = Phi > 0.0;  // ties: K upstream
  double sU = upL ? sL : sK, pU = upL ? pL : pK;
  double krw, krnw, dkrw, dkrnw;
  relperm(gp, sU, &krw, &krnw, &dkrw, &dkrnw);
  double kr = phase == 0 ? krw : krnw, dkr = phase == 0 ? dkrw : dkrnw;
  double rU = rho0 * (1.0 + c * (pU - gp.p_ref));
  double lamU = kr / mu;
  FaceFlux f;
  f.F = rU * lamU * Phi;
  double dF_dsU = rU / mu * Phi * dkr;
  f.dF_dsK = upL ? 0.0 : dF_dsU;
  f.dF_dsL = upL ? dF_dsU : 0.0;
  double drU = rho0 * c;
  f.dF_dpK = (upL ? 0.0 : drU * lamU * Phi) + rU * lamU * Ups * (-1.0 + dvK * g * dz);
  f.dF_dpL = (upL ? drU * lamU * Phi : 0.0) + rU * lamU * Ups * (1.0 + dvL * g * dz);
  return f;
}

// Jacobian blocks of App. B at the given state, before scaling and Dirichlet.
// ---------------------------------------------------------------------------
// Peaceman wells under bottom-hole pressure control (§3 well model: Eq. (peaceman), Eq. (well_index);
// Table 1 well control).  Two vertical wells perforate every layer at opposite ends of the grid: the water
// injector in the cell column (0, 0), the producer in the column (nx - 1, ny - 1); each perforation connects
// the well to the centroid of its cell.  The bottom-hole pressure is referred to the top perforation's
// centroid z_bh and set 5 MPa above (injector) or below (producer) the formation pressure there, the
// hydrostatic part of the initial pressure field, after a linear build-up over one day (a step of dt from the
// start reaches the fraction min(dt / 1 day, 1) of it); well radius 0.1524 m, skin 0.  For the isotropic cube cell
// of edge h, WI = 2 pi h kappa_h / (ln(r / r_w) + s_k) with r = 0.28 sqrt(2) h / 2.  Phase potential
// Phi_l = WI [(p_bh - p_K) + rho_l g (z_bh - z_K)]; injector q^I_w = rho_w (lambda_w + lambda_nw) Phi_w and no
// non-wetting injection; producer q^P_l = -rho_l lambda_l Phi_l for both phases.  The cell's mass balances
// get -dt (q^I_l - q^P_l) and their derivatives (App. B, viscosities constant).
// ---------------------------------------------------------------------------
const double kWellRadius = 0.1524, kWellSkin = 0.0, kWellDeltaBHP = 5.0e6;

// the well index needs a cell wider than the wellbore: Peaceman's radius r = 0.28 sqrt(2) h / 2 above r_w
bool wells_ok(const or_gen_params& gp) {
  return !(gp.flags & OR_WELLS) || 0.28 * std::sqrt(2.0) * gp.h / 2.0 > kWellRadius;
}

// 1: injector, 2: producer, 0: no well in the cell column (i, j)
int well_kind(const Grid& g, int i, int j) {
  if (i == 0 && j == 0) return 1;
  if (i == g.nx - 1 && j == g.ny - 1) return 2;
  return 0;
}

struct WellTerm {
  double r[2];     // residual terms of the wetting (s) and non-wetting (p) rows
  double d[2][2];  // their derivatives by (s, p) of the cell
};

WellTerm well_term(const or_gen_params& gp, const Grid& g, const Fields& F, int kind, int64_t c, int k, double s,
                   double p) {
  WellTerm w;
  std::memset(&w, 0, sizeof(w));
  const double grav = (gp.flags & OR_GRAVITY) ? gp.grav : 0.0;
  const double h = g.h;
  const double ztop = g.nz * h, zbh = (g.nz - 0.5) * h, zK = (k + 0.5) * h;
  const double pform = gp.p_ref + gp.rho_w0 * grav * (ztop - zbh);
  // the offsets build up linearly over one day (Table 1 ramp time): at the end of a step of dt from the start
  const double dbhp = kWellDeltaBHP * std::min(gp.dt / 86400.0, 1.0);
  const double pbh = kind == 1 ? pform + dbhp : pform - dbhp;
  const double re = 0.28 * std::sqrt(2.0 * h * h) / 2.0;
  const double WI = 2.0 * kPi * h * F.kh[c] / (std::log(re / kWellRadius) + kWellSkin);
  double krw, krnw, dkrw, dkrnw;
  relperm(gp, s, &krw, &krnw, &dkrw, &dkrnw);
  const double lam[2] = {krw / gp.mu_w, krnw / gp.mu_nw}, dlam[2] = {dkrw / gp.mu_w, dkrnw / gp.mu_nw};
  const double dp = p - gp.p_ref;
  const double rho[2] = {gp.rho_w0 * (1.0 + gp.c_w * dp), gp.rho_nw0 * (1.0 + gp.c_nw * dp)};
  const double drho[2] = {gp.rho_w0 * gp.c_w, gp.rho_nw0 * gp.c_nw};
  for (int l = 0; l < 2; ++l) {
    const double Phi = WI * ((pbh - p) + rho[l] * grav * (zbh - zK));
    const double dPhi = WI * (-1.0 + drho[l] * grav * (zbh - zK));
    double q = 0.0, dqs = 0.0, dqp = 0.0;  // q^I_l - q^P_l and its derivatives
    if (kind == 1) {
      if (l == 0) {
        const double lt = lam[0] + lam[1];
        q = rho[0] * lt * Phi;
        dqs = rho[0] * (dlam[0] + dlam[1]) * Phi;
        dqp = drho[0] * lt * Phi + rho[0] * lt * dPhi;
      }
    } else {
      // -q^P_l = rho_l lambda_l Phi_l
      q = rho[l] * lam[l] * Phi;
      dqs = rho[l] * dlam[l] * Phi;
      dqp = drho[l] * lam[l] * Phi + rho[l] * lam[l] * dPhi;
    }
    w.r[l] = -gp.dt * q;
    w.d[l][0] = -gp.dt * dqs;
    w.d[l][1] = -gp.dt * dqp;
  }
  return w;
}

void assemble(const or_gen_params& gp, const Grid& g, const Fields& F, const State& st,
              const ExtraBC& bc, Jac& J) {
  RefInt R = ref_integrals(g.h);
  J.uu = pattern_uu(g); J.uf = pattern_uf(g); J.fu = pattern_fu(g); J.ff = pattern_ff(g);
  int64_t nc = g.ncell();
  J.dfs.assign(2 * nc, 0.0);
  double grav = (gp.flags & OR_GRAVITY) ? gp.grav : 0.0;
  vec ev = mean_epsv(g, R, st.u);
  double V = g.h * g.h * g.h;
  bool coupling = (gp.flags & OR_COUPLING) != 0;
  // element loop: mechanics and coupling blocks (App. B, element blocks)
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        int64_t c = g.cell(i, j, k);
        double s = st.s[c];
        Mat m = material(gp, F.E[c], F.nu[c], F.phi0[c], s, st.p[c], ev[c]);
        double b = gp.biot;
        int64_t nodes[8];
        for (int a = 0; a < 8; ++a) nodes[a] = g.node(i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
        for (int a = 0; a < 8; ++a) {
          for (int bb = 0; bb < 8; ++bb) {
            int64_t pos = J.uu.find(nodes[a], nodes[bb]);
            double* blk = &J.uu.v[pos * 9];
            double trG = R.G[a][bb][0][0] + R.G[a][bb][1][1] + R.G[a][bb][2][2];
            for (int d = 0; d < 3; ++d)
              for (int e = 0; e < 3; ++e) {
                // int grad^s eta_i : C_dr : grad^s eta_j
                double kel = m.lam * R.G[a][bb][d][e] + m.G * R.G[a][bb][e][d] + (d == e ? m.G * trG : 0.0);
                // - int eta_i . (drho/deps_v g) div eta_j, g = (0,0,-grav)
                double gd = d == 2 ? -grav : 0.0;
                double kg = -m.drho_deps * gd * R.INdN[a][bb][e];
                blk[d * 3 + e] += kel + kg;
              }
          }
          // A_us, A_up (node a, cell c): 3x2 block, columns (s, p)
          int64_t pos = J.uf.find(nodes[a], c);
          double* blk = &J.uf.v[pos * 6];
          for (int d = 0; d < 3; ++d) {
            double gd = d == 2 ? -grav : 0.0;
            double us = -R.IN[a] * m.drho_ds * gd;
            double up = -b * R.IdN[a][d] - R.IN[a] * m.drho_dp * gd;
            if (coupling) { blk[d * 2 + 0] += us; blk[d * 2 + 1] += up; }
          }
          // A_su, A_pu (cell c, node a): 2x3 block
          int64_t pos2 = J.fu.find(c, nodes[a]);
          double* blk2 = &J.fu.v[pos2 * 6];
          for (int e = 0; e < 3; ++e) {
            double su = s * m.rw * b * R.IdN[a][e];
            double pu = (1.0 - s) * m.rnw * b * R.IdN[a][e];
            if (coupling) { blk2[0 * 3 + e] += su; blk2[1 * 3 + e] += pu; }
          }
        }
        // accumulation (App. B element blocks A_ss, A_sp, A_ps, A_pp; the well terms follow the face loop)
        if (gp.flags & OR_ACCUM) {
          int64_t pos = J.ff.find(c, c);
          double* blk = &J.ff.v[pos * 4];
          blk[0] += V * m.phi * m.rw;
          blk[1] += V * (s * m.rw * m.dphidp + m.phi * s * gp.rho_w0 * gp.c_w);
          blk[2] += -V * m.phi * m.rnw;
          blk[3] += V * ((1.0 - s) * m.rnw * m.dphidp + m.phi * (1.0 - s) * gp.rho_nw0 * gp.c_nw);
        }
        // §5.1 fixed-stress diagonals, with K_dr or (remark on one-dimensional loading) the uniaxial modulus
        const double Kfs = gp.fs_modulus == 1 ? m.Kdr + 4.0 * m.G / 3.0 : m.Kdr;
        J.dfs[2 * c + 0] = V * b * b / Kfs * s * m.rw;
        J.dfs[2 * c + 1] = V * b * b / Kfs * (1.0 - s) * m.rnw;
      }
  // face loop: TPFA Jacobian (App. B face blocks, with the Jacobian's sign:
  // row K gets -dt dF, row L gets +dt dF)
  if (gp.flags & OR_FLUX) {
    for (int k = 0; k < g.nz; ++k)
      for (int j = 0; j < g.ny; ++j)
        for (int i = 0; i < g.nx; ++i) {
          int64_t K = g.cell(i, j, k);
          for (int dir = 0; dir < 3; ++dir) {
            int a = i + (dir == 0), b2 = j + (dir == 1), c2 = k + (dir == 2);
            if (a >= g.nx || b2 >= g.ny || c2 >= g.nz) continue;
            int64_t L = g.cell(a, b2, c2);
            double kK = dir == 2 ? F.kv[K] : F.kh[K];
            double kL = dir == 2 ? F.kv[L] : F.kh[L];
            double area = g.h * g.h;
            double UK = area * kK / (0.5 * g.h), UL = area * kL / (0.5 * g.h);
            double Ups = UK * UL / (UK + UL);
            double dz = dir == 2 ? g.h : 0.0;
            int64_t pKK = J.ff.find(K, K), pKL = J.ff.find(K, L), pLK = J.ff.find(L, K), pLL = J.ff.find(L, L);
            for (int ph = 0; ph < 2; ++ph) {
              FaceFlux f = face_flux(gp, Ups, dz, grav, ph, st.s[K], st.p[K], st.s[L], st.p[L], false);
              double dsK = (gp.flags & OR_FLUX_SAT) ? f.dF_dsK : 0.0;
              double dsL = (gp.flags & OR_FLUX_SAT) ? f.dF_dsL : 0.0;
              double dt = gp.dt;
              J.ff.v[pKK * 4 + ph * 2 + 0] += -dt * dsK;
              J.ff.v[pKK * 4 + ph * 2 + 1] += -dt * f.dF_dpK;
              J.ff.v[pKL * 4 + ph * 2 + 0] += -dt * dsL;
              J.ff.v[pKL * 4 + ph * 2 + 1] += -dt * f.dF_dpL;
              J.ff.v[pLK * 4 + ph * 2 + 0] += dt * dsK;
              J.ff.v[pLK * 4 + ph * 2 + 1] += dt * f.dF_dpK;
              J.ff.v[pLL * 4 + ph * 2 + 0] += dt * dsL;
              J.ff.v[pLL * 4 + ph * 2 + 1] += dt * f.dF_dpL;
            }
          }
        }
    if (bc.active && bc.top_drained) {
      // Dirichlet flow face on top of each top cell: Upsilon^f = Upsilon^{f,K}
      for (int j = 0; j < g.ny; ++j)
        for (int i = 0; i < g.nx; ++i) {
          int64_t K = g.cell(i, j, g.nz - 1);
          double Ups = g.h * g.h * F.kv[K] / (0.5 * g.h);
          int64_t pKK = J.ff.find(K, K);
          for (int ph = 0; ph < 2; ++ph) {
            // the face plays the role of L; jump of psi is -psi_K
            FaceFlux f = face_flux(gp, Ups, 0.5 * g.h, grav, ph, st.s[K], st.p[K], bc.s_top, bc.p_top, true);
            double dsK = (gp.flags & OR_FLUX_SAT) ? f.dF_dsK : 0.0;
            J.ff.v[pKK * 4 + ph * 2 + 0] += -gp.dt * dsK;
            J.ff.v[pKK * 4 + ph * 2 + 1] += -gp.dt * f.dF_dpK;
          }
        }
    }
  }
  // wells: cell-diagonal terms
  if (gp.flags & OR_WELLS)
    for (int k = 0; k < g.nz; ++k)
      for (int j = 0; j < g.ny; ++j)
        for (int i = 0; i < g.nx; ++i) {
          const int kind = well_kind(g, i, j);
          if (!kind) continue;
          const int64_t K = g.cell(i, j, k);
          const WellTerm w = well_term(gp, g, F, kind, K, k, st.s[K], st.p[K]);
          const int64_t pKK = J.ff.find(K, K);
          for (int l = 0; l < 2; ++l)
            for (int e = 0; e < 2; ++e) J.ff.v[pKK * 4 + l * 2 + e] += w.d[l][e];
        }
  // Dirichlet dofs
  int64_t nu = 3 * g.nn();
  J.dir.assign(nu, 0);
  if (bc.active) {
    J.dir = bc.dir_u;
  } else if (gp.flags & OR_DIRICHLET) {
    for (int j = 0; j <= g.ny; ++j)
      for (int i = 0; i <= g.nx; ++i) {
        int64_t I = g.node(i, j, 0);
        for (int d = 0; d < 3; ++d) J.dir[3 * I + d] = 1;
      }
  }
}

// Dirichlet elimination (zero rows and columns of the constrained dofs),
// block-row scaling (§4 remark) and unit diagonal for constrained dofs.
void finalize(const or_gen_params& gp, const Grid& g, Jac& J, bool scale) {
  int64_t nn = g.nn(), nc = g.ncell();
  for (int64_t I = 0; I < nn; ++I)
    for (int64_t q = J.uu.rp[I]; q < J.uu.rp[I + 1]; ++q) {
      int64_t Jn = J.uu.ci[q];
      for (int d = 0; d < 3; ++d)
        for (int e = 0; e < 3; ++e)
          if (J.dir[3 * I + d] || J.dir[3 * Jn + e]) J.uu.v[q * 9 + d * 3 + e] = 0.0;
    }
  for (int64_t I = 0; I < nn; ++I)
    for (int64_t q = J.uf.rp[I]; q < J.uf.rp[I + 1]; ++q)
      for (int d = 0; d < 3; ++d)
        if (J.dir[3 * I + d]) { J.uf.v[q * 6 + d * 2] = 0.0; J.uf.v[q * 6 + d * 2 + 1] = 0.0; }
  for (int64_t c = 0; c < nc; ++c)
    for (int64_t q = J.fu.rp[c]; q < J.fu.rp[c + 1]; ++q) {
      int64_t I = J.fu.ci[q];
      for (int e = 0; e < 3; ++e)
        if (J.dir[3 * I + e]) { J.fu.v[q * 6 + e] = 0.0; J.fu.v[q * 6 + 3 + e] = 0.0; }
    }
  J.alpha_u = 1.0; J.alpha_f = 1.0;
  if (scale) {
    const double pcol = 1e6;  // pressure unknown in MPa
    for (size_t q = 0; q < J.uf.ci.size(); ++q)
      for (int d = 0; d < 3; ++d) J.uf.v[q * 6 + d * 2 + 1] *= pcol;
    for (size_t q = 0; q < J.ff.ci.size(); ++q) { J.ff.v[q * 4 + 1] *= pcol; J.ff.v[q * 4 + 3] *= pcol; }
    for (int64_t c = 0; c < nc; ++c) { J.dfs[2 * c] *= pcol; J.dfs[2 * c + 1] *= pcol; }
    double su = 0.0; int64_t cnt = 0;
    for (int64_t I = 0; I < nn; ++I) {
      int64_t q = J.uu.find(I, I);
      for (int d = 0; d < 3; ++d)
        if (!J.dir[3 * I + d]) { su += J.uu.v[q * 9 + d * 4]; ++cnt; }
    }
    J.alpha_u = cnt ? su / double(cnt) : 1.0;
    double sf = 0.0;
    for (int64_t c = 0; c < nc; ++c) sf += std::fabs(J.ff.v[J.ff.find(c, c) * 4 + 3]);
    J.alpha_f = sf / double(nc);
    for (double& x : J.uu.v) x /= J.alpha_u;
    for (double& x : J.uf.v) x /= J.alpha_u;
    for (double& x : J.fu.v) x /= J.alpha_f;
    for (double& x : J.ff.v) x /= J.alpha_f;
    for (double& x : J.dfs) x /= J.alpha_f;
  }
  for (int64_t I = 0; I < nn; ++I) {
    int64_t q = J.uu.find(I, I);
    for (int d = 0; d < 3; ++d)
      if (J.dir[3 * I + d]) J.uu.v[q * 9 + d * 4] = 1.0;
  }
}

template <class T>
T* dup(const std::vector<T>& v) {
  T* p = (T*)std::malloc(std::max<size_t>(1, v.size()) * sizeof(T));
  if (!v.empty()) std::memcpy(p, v.data(), v.size() * sizeof(T));
  return p;
}

// ---------------------------------------------------------------------------
// Dense LU with partial pivoting (textbook Doolittle, row-major)
// ---------------------------------------------------------------------------
struct DenseLU {
  int64_t n = 0;
  vec a;
  std::vector<int64_t> piv;
  bool ok = false;
  void factor(int64_t n_, vec m) {
    n = n_; a = std::move(m); piv.resize(n);
    ok = true;
    for (int64_t k = 0; k < n; ++k) {
      int64_t p = k;
      double best = std::fabs(a[k * n + k]);
      for (int64_t i = k + 1; i < n; ++i)
        if (std::fabs(a[i * n + k]) > best) { best = std::fabs(a[i * n + k]); p = i; }
      piv[k] = p;
      if (best == 0.0) { ok = false; continue; }
      if (p != k)
        for (int64_t j = 0; j < n; ++j) std::swap(a[k * n + j], a[p * n + j]);
      for (int64_t i = k + 1; i < n; ++i) {
        double l = a[i * n + k] / a[k * n + k];
        a[i * n + k] = l;
        if (l == 0.0) continue;
        for (int64_t j = k + 1; j < n; ++j) a[i * n + j] -= l * a[k * n + j];
      }
    }
  }
  void solve(const double* b, double* x) const {
    vec y(b, b + n);
    for (int64_t k = 0; k < n; ++k) std::swap(y[k], y[piv[k]]);
    for (int64_t i = 0; i < n; ++i) {
      double s = y[i];
      for (int64_t j = 0; j < i; ++j) s -= a[i * n + j] * y[j];
      y[i] = s;
    }
    for (int64_t i = n - 1; i >= 0; --i) {
      double s = y[i];
      for (int64_t j = i + 1; j < n; ++j) s -= a[i * n + j] * y[j];
      y[i] = s / a[i * n + i];
    }
    for (int64_t i = 0; i < n; ++i) x[i] = y[i];
  }
};

// ---------------------------------------------------------------------------
// Scalar CSR with nc values per entry (shared pattern for the three SDC
// displacement components of §5.2)
// ---------------------------------------------------------------------------
struct CSR {
  int64_t n = 0, m = 0;
  int nc = 1;
  std::vector<int64_t> rp;
  std::vector<int32_t> ci;
  vec v;  // v[e*nc + comp]
  int64_t nnz() const { return int64_t(ci.size()); }
  int64_t find(int64_t i, int64_t j) const {
    auto b = ci.begin() + rp[i], e = ci.begin() + rp[i + 1];
    auto it = std::lower_bound(b, e, int32_t(j));
    if (it == e || *it != j) return -1;
    return it - ci.begin();
  }
};

void csr_spmv(const CSR& A, int comp, const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < A.n; ++i) {
    double s = 0.0;
    for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q) s += A.v[q * A.nc + comp] * x[A.ci[q]];
    y[i] = s;
  }
}

// transpose; entries of each output row appear in ascending input-row order
CSR transpose(const CSR& A) {
  CSR T; T.n = A.m; T.m = A.n; T.nc = A.nc;
  T.rp.assign(T.n + 1, 0);
  for (int32_t c : A.ci) T.rp[c + 1]++;
  for (int64_t i = 0; i < T.n; ++i) T.rp[i + 1] += T.rp[i];
  T.ci.resize(A.ci.size()); T.v.resize(A.v.size());
  std::vector<int64_t> fill(T.rp.begin(), T.rp.end() - 1);
  for (int64_t i = 0; i < A.n; ++i)
    for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q) {
      int64_t pos = fill[A.ci[q]]++;
      T.ci[pos] = int32_t(i);
      for (int c = 0; c < A.nc; ++c) T.v[pos * A.nc + c] = A.v[q * A.nc + c];
    }
  return T;
}

// C = X Y (row-wise Gustavson).  For each output entry the products are added
// in ascending order of the inner index k, starting from 0, each by one fused multiply-add.
CSR spgemm(const CSR& X, const CSR& Y) {
  CSR C; C.n = X.n; C.m = Y.m; C.nc = X.nc;
  C.rp.assign(C.n + 1, 0);
  std::vector<std::vector<int32_t>> tci(kTasks);
  std::vector<vec> tv(kTasks);
#pragma omp parallel for schedule(dynamic, 1)
  for (int t = 0; t < kTasks; ++t) {
    std::vector<int64_t> mark(Y.m, -1);
    vec acc(size_t(Y.m) * X.nc, 0.0);
    std::vector<int32_t> cols;
    for (int64_t i = task_lo(X.n, t); i < task_lo(X.n, t + 1); ++i) {
      cols.clear();
      for (int64_t q = X.rp[i]; q < X.rp[i + 1]; ++q) {
        int64_t k = X.ci[q];
        for (int64_t r = Y.rp[k]; r < Y.rp[k + 1]; ++r) {
          int64_t j = Y.ci[r];
          if (mark[j] != i) {
            mark[j] = i;
            cols.push_back(int32_t(j));
            for (int c = 0; c < X.nc; ++c) acc[j * X.nc + c] = 0.0;
          }
          for (int c = 0; c < X.nc; ++c) acc[j * X.nc + c] = std::fma(X.v[q * X.nc + c], Y.v[r * X.nc + c], acc[j * X.nc + c]);
        }
      }
      std::sort(cols.begin(), cols.end());
      for (int32_t j : cols) {
        tci[t].push_back(j);
        for (int c = 0; c < X.nc; ++c) tv[t].push_back(acc[j * X.nc + c]);
      }
      C.rp[i + 1] = int64_t(cols.size());
    }
  }
  for (int64_t i = 0; i < C.n; ++i) C.rp[i + 1] += C.rp[i];
  for (int t = 0; t < kTasks; ++t) {
    C.ci.insert(C.ci.end(), tci[t].begin(), tci[t].end());
    C.v.insert(C.v.end(), tv[t].begin(), tv[t].end());
  }
  return C;
}

// ---------------------------------------------------------------------------
// Smoothed-aggregation AMG (the amg(.) of §5.2 and §5.3; the paper uses Hypre
// BoomerAMG, this restates a deterministic smoothed aggregation)
// ---------------------------------------------------------------------------
struct Level {
  CSR A, P, R;
  std::vector<int32_t> agg;
  int64_t nagg = 0;
  vec dl1;  // n*nc, l1 row norms
  vec dg;   // n*nc, diagonal
  vec lam;  // nc, Gershgorin bound of rho(D^{-1}A)
  std::vector<uint8_t> root;  // distance-2 MIS roots
  std::vector<uint8_t> excl;  // rows whose off-diagonal entries are all zero
  std::vector<DenseLU> lu;  // coarsest only, per component
};
struct AMG {
  int nc = 1;
  std::vector<Level> L;
};

// node-level strength value: sum over components of |a_ij|
inline double abar(const CSR& A, int64_t q) {
  double s = 0.0;
  for (int c = 0; c < A.nc; ++c) s = s + std::fabs(A.v[q * A.nc + c]);
  return s;
}

inline int64_t mis_key(int64_t i, int level) {
  uint64_t h = sm64((uint64_t(level) << 32) | uint64_t(i));
  return (int64_t(h >> 33) << 32) | i;
}

// Strength graph, distance-2 maximal independent set, aggregates.
void aggregate(Level& lev, double theta, int level) {
  const CSR& A = lev.A;
  int64_t n = A.n;
  vec dg(n, 0.0);
  std::vector<uint8_t> excluded(n, 1);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i)
    for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q) {
      if (A.ci[q] == i) dg[i] = abar(A, q);
      else
        for (int c = 0; c < A.nc; ++c)
          if (A.v[q * A.nc + c] != 0.0) excluded[i] = 0;
    }
  // symmetric strength graph: edge i~j if max(abar_ij, abar_ji) >= theta*sqrt(abar_ii*abar_jj)
  std::vector<uint8_t> strong(A.nnz(), 0);
  vec wgt(A.nnz(), 0.0);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    if (excluded[i]) continue;
    for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q) {
      int64_t j = A.ci[q];
      if (j == i || excluded[j]) continue;
      int64_t qt = A.find(j, i);
      double aij = abar(A, q), aji = qt >= 0 ? abar(A, qt) : 0.0;
      double t = std::max(aij, aji);
      double den = std::sqrt(dg[i] * dg[j]);
      if (t >= theta * den && t > 0.0) { strong[q] = 1; wgt[q] = t / den; }
    }
  }
  // Rows without any strong connection (identity rows included) stay out of the
  // coarse space: the smoother alone treats them (the isolated-node rule of
  // smoothed aggregation).  Their prolongator rows still follow (I - w D^{-1} A) P_tent.
  lev.excl = excluded;
  std::vector<uint8_t> st(n, 0);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    bool any = false;
    for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q) any = any || strong[q];
    if (excluded[i] || !any) st[i] = 3;
  }
  // synchronous distance-2 MIS rounds: 0 undecided, 1 root, 2 covered, 3 not aggregated
  std::vector<int64_t> m1(n), m2(n);
  std::vector<uint8_t> nr(n), c1(n);
  for (;;) {
    bool any = false;
    for (int64_t i = 0; i < n; ++i) if (st[i] == 0) { any = true; break; }
    if (!any) break;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      int64_t m = st[i] == 0 ? mis_key(i, level) : -1;
      for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q)
        if (strong[q] && st[A.ci[q]] == 0) m = std::max(m, mis_key(A.ci[q], level));
      m1[i] = m;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      int64_t m = m1[i];
      for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q)
        if (strong[q]) m = std::max(m, m1[A.ci[q]]);
      m2[i] = m;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) nr[i] = (st[i] == 0 && m2[i] == mis_key(i, level));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) if (nr[i]) st[i] = 1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      uint8_t c = nr[i];
      for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q)
        if (strong[q] && nr[A.ci[q]]) c = 1;
      c1[i] = c;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      if (st[i] != 0) continue;
      uint8_t c = c1[i];
      for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q)
        if (strong[q] && c1[A.ci[q]]) c = 1;
      if (c) st[i] = 2;
    }
  }
  lev.agg.assign(n, -1);
  lev.root.assign(n, 0);
  for (int64_t i = 0; i < n; ++i) lev.root[i] = st[i] == 1;
  int64_t na = 0;
  for (int64_t i = 0; i < n; ++i) if (st[i] == 1) lev.agg[i] = int32_t(na++);
  lev.nagg = na;
  // phase 1: strong neighbours of a root join it
  std::vector<int32_t> ph1 = lev.agg;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    if (st[i] != 2) continue;
    for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q)
      if (strong[q] && st[A.ci[q]] == 1) { ph1[i] = lev.agg[A.ci[q]]; break; }
  }
  // phase 2: leftovers join the aggregate of their strongest phase-1 neighbour
  lev.agg = ph1;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    if (st[i] != 2 || ph1[i] >= 0) continue;
    double bw = -1.0; int32_t ba = -1;
    for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q) {
      if (!strong[q]) continue;
      int32_t a = ph1[A.ci[q]];
      if (a < 0) continue;
      if (wgt[q] > bw || (wgt[q] == bw && a < ba)) { bw = wgt[q]; ba = a; }
    }
    lev.agg[i] = ba;
  }
}

// Gershgorin bound lambda_hat = max_i sum_j |a_ij| / |a_ii| per component
vec gershgorin(const CSR& A) {
  vec lam(A.nc, 0.0);
  for (int c = 0; c < A.nc; ++c) {
    vec ratio(A.n);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < A.n; ++i) {
      double s = 0.0, d = 0.0;
      for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q) {
        s = s + std::fabs(A.v[q * A.nc + c]);
        if (A.ci[q] == i) d = A.v[q * A.nc + c];
      }
      ratio[i] = s / std::fabs(d);
    }
    for (int64_t i = 0; i < A.n; ++i) lam[c] = std::max(lam[c], ratio[i]);
  }
  return lam;
}

// P = (I - omega D^{-1} A) P_tent, omega = (4/3)/lambda_hat (Gershgorin)
CSR smoothed_prolongator(const Level& lev) {
  const CSR& A = lev.A;
  int nc = A.nc;
  int64_t n = A.n;
  vec lam = gershgorin(A), omega(nc);
  for (int c = 0; c < nc; ++c) omega[c] = (4.0 / 3.0) / lam[c];
  CSR P; P.n = n; P.m = lev.nagg; P.nc = nc; P.rp.assign(n + 1, 0);
  std::vector<std::vector<int32_t>> tci(kTasks);
  std::vector<vec> tv(kTasks);
#pragma omp parallel for schedule(dynamic, 1)
  for (int t = 0; t < kTasks; ++t) {
    std::vector<int32_t> aggs;
    for (int64_t i = task_lo(n, t); i < task_lo(n, t + 1); ++i) {
      if (lev.excl[i]) continue;
      aggs.clear();
      for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q)
        if (lev.agg[A.ci[q]] >= 0) aggs.push_back(lev.agg[A.ci[q]]);
      std::sort(aggs.begin(), aggs.end());
      aggs.erase(std::unique(aggs.begin(), aggs.end()), aggs.end());
      int64_t qd = A.find(i, i);
      for (int32_t a : aggs) {
        tci[t].push_back(a);
        for (int c = 0; c < nc; ++c) {
          double S = 0.0;
          for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q)
            if (lev.agg[A.ci[q]] == a) S = S + A.v[q * nc + c];
          double coef = omega[c] / A.v[qd * nc + c];
          double delta = a == lev.agg[i] ? 1.0 : 0.0;
          tv[t].push_back(delta - coef * S);
        }
      }
      P.rp[i + 1] = int64_t(aggs.size());
    }
  }
  for (int64_t i = 0; i < n; ++i) P.rp[i + 1] += P.rp[i];
  for (int t = 0; t < kTasks; ++t) {
    P.ci.insert(P.ci.end(), tci[t].begin(), tci[t].end());
    P.v.insert(P.v.end(), tv[t].begin(), tv[t].end());
  }
  return P;
}

vec l1_diag(const CSR& A) {
  vec d(A.n * A.nc, 0.0);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < A.n; ++i)
    for (int c = 0; c < A.nc; ++c) {
      double s = 0.0;
      for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q) s = s + std::fabs(A.v[q * A.nc + c]);
      d[i * A.nc + c] = s;
    }
  return d;
}

bool build_amg(AMG& H, CSR A0, double theta0, int coarse_max, int max_levels) {
  H.nc = A0.nc;
  H.L.clear();
  H.L.emplace_back();
  H.L[0].A = std::move(A0);
  double theta = theta0;
  for (int l = 0;; ++l) {
    Level& lev = H.L[l];
    bool coarsest = lev.A.n <= coarse_max || l + 1 >= max_levels;
    if (!coarsest) {
      aggregate(lev, theta, l);
      if (lev.nagg == 0 || double(lev.A.n) / double(lev.nagg) < 1.2) coarsest = true;
    }
    if (coarsest) {
      if (lev.A.n > 12000) return false;
      lev.agg.clear(); lev.nagg = 0;
      lev.lu.resize(H.nc);
      for (int c = 0; c < H.nc; ++c) {
        int64_t n = lev.A.n;
        vec d(size_t(n) * n, 0.0);
        for (int64_t i = 0; i < n; ++i)
          for (int64_t q = lev.A.rp[i]; q < lev.A.rp[i + 1]; ++q) d[i * n + lev.A.ci[q]] = lev.A.v[q * H.nc + c];
        lev.lu[c].factor(n, std::move(d));
      }
      break;
    }
    lev.P = smoothed_prolongator(lev);
    lev.R = transpose(lev.P);
    lev.dl1 = l1_diag(lev.A);
    lev.lam = gershgorin(lev.A);
    lev.dg.assign(lev.A.n * H.nc, 0.0);
    for (int64_t i = 0; i < lev.A.n; ++i) {
      int64_t q = lev.A.find(i, i);
      for (int c = 0; c < H.nc; ++c) lev.dg[i * H.nc + c] = lev.A.v[q * H.nc + c];
    }
    CSR AP = spgemm(lev.A, lev.P);
    CSR Ac = spgemm(lev.R, AP);
    H.L.emplace_back();
    H.L[l + 1].A = std::move(Ac);
    theta *= 0.5;
  }
  return true;
}

struct Smooth {
  int kind, pre, post, degree;
  double ratio;
};

// Chebyshev smoother on D^{-1}A over [lambda_hat/ratio, lambda_hat]
// (three-term recurrence of Adams, Brezina, Hu, Tuminaro 2003)
void chebyshev(const Level& lev, int nc, int c, const vec& b, vec& x, int degree, double ratio, bool zero) {
  int64_t n = lev.A.n;
  double lmax = lev.lam[c], lmin = lmax / ratio;
  double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
  double sigma = theta / delta, rho = 1.0 / sigma;
  vec r(n), d(n), Ax(n);
  if (zero) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] / lev.dg[i * nc + c];
  } else {
    csr_spmv(lev.A, c, x.data(), Ax.data());
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) r[i] = (b[i] - Ax[i]) / lev.dg[i * nc + c];
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) d[i] = r[i] / theta;
  for (int k = 0; k < degree; ++k) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) x[i] = x[i] + d[i];
    if (k == degree - 1) break;
    csr_spmv(lev.A, c, x.data(), Ax.data());
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) r[i] = (b[i] - Ax[i]) / lev.dg[i * nc + c];
    double rn = 1.0 / (2.0 * sigma - rho);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) d[i] = rn * rho * d[i] + 2.0 * rn / delta * r[i];
    rho = rn;
  }
}

void l1_jacobi(const Level& lev, int nc, int c, const vec& b, vec& x, int sweeps) {
  int64_t n = lev.A.n;
  vec Ax(n);
  for (int it = 0; it < sweeps; ++it) {
    csr_spmv(lev.A, c, x.data(), Ax.data());
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) x[i] = x[i] + (b[i] - Ax[i]) / lev.dl1[i * nc + c];
  }
}

// V-cycle: pre-smoothing from x = 0, coarse correction x += P V(R r), post-smoothing
void vcycle(const AMG& H, int l, int c, const vec& b, vec& x, const Smooth& sm) {
  const Level& lev = H.L[l];
  int64_t n = lev.A.n;
  x.assign(n, 0.0);
  if (lev.lu.size()) { lev.lu[c].solve(b.data(), x.data()); return; }
  if (sm.kind == 0) l1_jacobi(lev, H.nc, c, b, x, sm.pre);
  else chebyshev(lev, H.nc, c, b, x, sm.degree, sm.ratio, true);
  vec Ax(n);
  csr_spmv(lev.A, c, x.data(), Ax.data());
  vec r(n);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - Ax[i];
  vec bc(lev.R.n), xc;
  csr_spmv(lev.R, c, r.data(), bc.data());
  vcycle(H, l + 1, c, bc, xc, sm);
  vec Pe(n);
  csr_spmv(lev.P, c, xc.data(), Pe.data());
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) x[i] = x[i] + Pe[i];
  if (sm.kind == 0) l1_jacobi(lev, H.nc, c, b, x, sm.post);
  else chebyshev(lev, H.nc, c, b, x, sm.degree, sm.ratio, false);
}

inline void mul22(const double* a, const double* b, double* c) {
  double c0 = a[0] * b[0] + a[1] * b[2], c1 = a[0] * b[1] + a[1] * b[3];
  double c2 = a[2] * b[0] + a[3] * b[2], c3 = a[2] * b[1] + a[3] * b[3];
  c[0] = c0; c[1] = c1; c[2] = c2; c[3] = c3;
}
inline void inv22(const double* a, double* r) {
  double det = a[0] * a[3] - a[1] * a[2];
  r[0] = a[3] / det; r[1] = -a[1] / det; r[2] = -a[2] / det; r[3] = a[0] / det;
}

BSR to_bsr(const or_system* s, int which) {
  BSR A;
  if (which == 0) { A.nbr = s->n_nodes; A.nbc = s->n_nodes; A.br = 3; A.bc = 3; }
  if (which == 1) { A.nbr = s->n_nodes; A.nbc = s->n_cells; A.br = 3; A.bc = 2; }
  if (which == 2) { A.nbr = s->n_cells; A.nbc = s->n_nodes; A.br = 2; A.bc = 3; }
  if (which == 3) { A.nbr = s->n_cells; A.nbc = s->n_cells; A.br = 2; A.bc = 2; }
  const int64_t* rp = which == 0 ? s->uu_rp : which == 1 ? s->uf_rp : which == 2 ? s->fu_rp : s->ff_rp;
  const int32_t* ci = which == 0 ? s->uu_ci : which == 1 ? s->uf_ci : which == 2 ? s->fu_ci : s->ff_ci;
  const double* v = which == 0 ? s->uu_v : which == 1 ? s->uf_v : which == 2 ? s->fu_v : s->ff_v;
  A.rp.assign(rp, rp + A.nbr + 1);
  A.ci.assign(ci, ci + A.rp[A.nbr]);
  A.v.assign(v, v + A.rp[A.nbr] * A.br * A.bc);
  return A;
}

void bsr_dense(const BSR& A, vec& d, int64_t r0, int64_t c0, int64_t ld) {
  for (int64_t I = 0; I < A.nbr; ++I)
    for (int64_t q = A.rp[I]; q < A.rp[I + 1]; ++q)
      for (int a = 0; a < A.br; ++a)
        for (int b = 0; b < A.bc; ++b)
          d[(r0 + I * A.br + a) * ld + c0 + int64_t(A.ci[q]) * A.bc + b] = A.v[(q * A.br + a) * A.bc + b];
}


// ---------------------------------------------------------------------------
// Rigid-body-mode smoothed aggregation on the full A_uu: the usual AMG for elasticity, the alternative to the
// separate-displacement-component approximation that §5.2 takes.  Block operators (3 x 3 at the finest
// level, 6 x 6 below), a near-nullspace of the six rigid-body modes, a tentative prolongator from a modified
// Gram-Schmidt QR of the modes restricted to each aggregate, P = (I - omega D^{-1} A) P_tent with the point
// diagonal D, Galerkin coarse operators, Chebyshev smoothing on D^{-1} A and dense LU on the coarsest level.
// ---------------------------------------------------------------------------
constexpr int kModes = 6;

struct BLevel {
  BSR A, P, R;               // A: b x b blocks, P: b x 6, R = P^T: 6 x b
  int b = 3;
  std::vector<int32_t> agg;  // aggregate of each node (-1: not aggregated)
  int64_t nagg = 0;
  vec B;                     // near-nullspace, n b rows of 6
  vec Pt;                    // tentative prolongator, n b rows of 6 (zero rows for nodes outside aggregates)
  vec dg;                    // point diagonal, n b
  double lam = 0.0;          // Gershgorin bound of rho(D^{-1} A) over the point rows
  DenseLU lu;                // coarsest level
  bool coarsest = false;
};
struct BAMG {
  std::vector<BLevel> L;
};

// y = A x over point rows; each point row sums its blocks in column order, a block's entries in column order
void bsr_apply(const BSR& A, const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < A.nbr; ++i)
    for (int a = 0; a < A.br; ++a) {
      double s = 0.0;
      for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q)
        for (int e = 0; e < A.bc; ++e) s = s + A.v[(q * A.br + a) * A.bc + e] * x[int64_t(A.ci[q]) * A.bc + e];
      y[i * A.br + a] = s;
    }
}

// transpose with transposed blocks; entries of each output row in ascending input-row order
BSR bsr_transpose(const BSR& A) {
  BSR T; T.nbr = A.nbc; T.nbc = A.nbr; T.br = A.bc; T.bc = A.br;
  T.rp.assign(T.nbr + 1, 0);
  for (int32_t c : A.ci) T.rp[c + 1]++;
  for (int64_t i = 0; i < T.nbr; ++i) T.rp[i + 1] += T.rp[i];
  T.ci.resize(A.ci.size()); T.v.resize(A.v.size());
  std::vector<int64_t> fill(T.rp.begin(), T.rp.end() - 1);
  for (int64_t i = 0; i < A.nbr; ++i)
    for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q) {
      int64_t pos = fill[A.ci[q]]++;
      T.ci[pos] = int32_t(i);
      for (int a = 0; a < A.br; ++a)
        for (int e = 0; e < A.bc; ++e) T.v[(pos * T.br + e) * T.bc + a] = A.v[(q * A.br + a) * A.bc + e];
    }
  return T;
}

// C = X Y with block products.  For each output block the block products X_ik Y_kj are added in ascending
// order of k, starting from zero; each entry of a block product sums its inner index in ascending order, one
// fused multiply-add per term.
BSR bsr_spgemm(const BSR& X, const BSR& Y) {
  BSR C; C.nbr = X.nbr; C.nbc = Y.nbc; C.br = X.br; C.bc = Y.bc;
  const int br = X.br, bk = X.bc, bc = Y.bc, bs = br * bc;
  C.rp.assign(C.nbr + 1, 0);
  std::vector<std::vector<int32_t>> tci(kTasks);
  std::vector<vec> tv(kTasks);
#pragma omp parallel for schedule(dynamic, 1)
  for (int t = 0; t < kTasks; ++t) {
    std::vector<int64_t> mark(Y.nbc, -1);
    vec acc(size_t(Y.nbc) * bs, 0.0);
    std::vector<int32_t> cols;
    for (int64_t i = task_lo(X.nbr, t); i < task_lo(X.nbr, t + 1); ++i) {
      cols.clear();
      for (int64_t q = X.rp[i]; q < X.rp[i + 1]; ++q) {
        const int64_t k = X.ci[q];
        const double* xb = &X.v[q * br * bk];
        for (int64_t r = Y.rp[k]; r < Y.rp[k + 1]; ++r) {
          const int64_t j = Y.ci[r];
          const double* yb = &Y.v[r * bk * bc];
          if (mark[j] != i) {
            mark[j] = i;
            cols.push_back(int32_t(j));
            for (int e = 0; e < bs; ++e) acc[j * bs + e] = 0.0;
          }
          for (int a = 0; a < br; ++a)
            for (int c = 0; c < bc; ++c) {
              double p = 0.0;
              for (int e = 0; e < bk; ++e) p = std::fma(xb[a * bk + e], yb[e * bc + c], p);
              acc[j * bs + a * bc + c] = acc[j * bs + a * bc + c] + p;
            }
        }
      }
      std::sort(cols.begin(), cols.end());
      for (int32_t j : cols) {
        tci[t].push_back(j);
        for (int e = 0; e < bs; ++e) tv[t].push_back(acc[j * bs + e]);
      }
      C.rp[i + 1] = int64_t(cols.size());
    }
  }
  for (int64_t i = 0; i < C.nbr; ++i) C.rp[i + 1] += C.rp[i];
  for (int t = 0; t < kTasks; ++t) {
    C.ci.insert(C.ci.end(), tci[t].begin(), tci[t].end());
    C.v.insert(C.v.end(), tv[t].begin(), tv[t].end());
  }
  return C;
}

// the six rigid-body modes at the nodes of the grid: translations along x, y, z and rotations about the
// axes through the grid's centre, (0, -z, y), (z, 0, -x), (-y, x, 0), coordinates in cell widths
vec rigid_body_modes(int nx, int ny, int nz) {
  const int64_t nn = int64_t(nx + 1) * (ny + 1) * (nz + 1);
  vec B(size_t(nn) * 3 * kModes, 0.0);
  for (int64_t I = 0; I < nn; ++I) {
    const int64_t i = I % (nx + 1), j = (I / (nx + 1)) % (ny + 1), k = I / (int64_t(nx + 1) * (ny + 1));
    const double x = double(i) - 0.5 * nx, y = double(j) - 0.5 * ny, z = double(k) - 0.5 * nz;
    double* r = &B[I * 3 * kModes];
    // row d of node I: r[d * 6 + mode]
    r[0 * 6 + 0] = 1.0; r[1 * 6 + 1] = 1.0; r[2 * 6 + 2] = 1.0;
    r[1 * 6 + 3] = -z; r[2 * 6 + 3] = y;
    r[0 * 6 + 4] = z;  r[2 * 6 + 4] = -x;
    r[0 * 6 + 5] = -y; r[1 * 6 + 5] = x;
  }
  return B;
}

// strength matrix of a block operator: one value per block, its Frobenius norm (entries summed row by row)
CSR block_strength(const BSR& A) {
  CSR S; S.n = A.nbr; S.m = A.nbc; S.nc = 1; S.rp = A.rp; S.ci = A.ci;
  const int bs = A.br * A.bc;
  S.v.resize(A.ci.size());
#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < int64_t(A.ci.size()); ++q) {
    double s = 0.0;
    for (int e = 0; e < bs; ++e) s = s + A.v[q * bs + e] * A.v[q * bs + e];
    S.v[q] = std::sqrt(s);
  }
  return S;
}

// lambda_hat = max over point rows of sum_j |a_ij| / |a_ii| (blocks in column order, entries in column order)
double block_gershgorin(const BSR& A) {
  const int b = A.br;
  vec ratio(A.nbr * b, 0.0);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < A.nbr; ++i)
    for (int a = 0; a < b; ++a) {
      double s = 0.0, d = 0.0;
      for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q)
        for (int e = 0; e < A.bc; ++e) {
          const double v = A.v[(q * b + a) * A.bc + e];
          s = s + std::fabs(v);
          if (A.ci[q] == i && e == a) d = v;
        }
      ratio[i * b + a] = s / std::fabs(d);
    }
  double lam = 0.0;
  for (double r : ratio) lam = std::max(lam, r);
  return lam;
}

// Tentative prolongator and coarse near-nullspace: per aggregate (nodes in ascending order, b rows each) the
// modes restricted to the aggregate, B_a = Q_a R_a by modified Gram-Schmidt (columns in order; a column whose
// remainder is at most 1e-10 of its norm is dependent on the earlier ones: zero column of Q_a, zero row of
// R_a).  P_tent has one b x 6 block per aggregated node, Q_a's rows of that node; the coarse modes are R_a.
void tentative(BLevel& lev, vec& Bc) {
  const int b = lev.b;
  const int64_t n = lev.A.nbr;
  std::vector<std::vector<int64_t>> mem(lev.nagg);
  for (int64_t i = 0; i < n; ++i)
    if (lev.agg[i] >= 0) mem[lev.agg[i]].push_back(i);
  lev.Pt.assign(size_t(n) * b * kModes, 0.0);
  Bc.assign(size_t(lev.nagg) * kModes * kModes, 0.0);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t a = 0; a < lev.nagg; ++a) {
    const int64_t m = int64_t(mem[a].size()) * b;
    vec Q(size_t(m) * kModes);
    for (size_t t = 0; t < mem[a].size(); ++t)
      for (int d = 0; d < b; ++d)
        for (int k = 0; k < kModes; ++k) Q[(t * b + d) * kModes + k] = lev.B[(mem[a][t] * b + d) * kModes + k];
    double R[kModes][kModes] = {{0.0}};
    for (int k = 0; k < kModes; ++k) {
      double n0 = 0.0;
      for (int64_t r = 0; r < m; ++r) n0 = n0 + Q[r * kModes + k] * Q[r * kModes + k];
      n0 = std::sqrt(n0);
      for (int j = 0; j < k; ++j) {
        double c = 0.0;
        for (int64_t r = 0; r < m; ++r) c = c + Q[r * kModes + j] * Q[r * kModes + k];
        R[j][k] = c;
        for (int64_t r = 0; r < m; ++r) Q[r * kModes + k] = Q[r * kModes + k] - c * Q[r * kModes + j];
      }
      double nk = 0.0;
      for (int64_t r = 0; r < m; ++r) nk = nk + Q[r * kModes + k] * Q[r * kModes + k];
      nk = std::sqrt(nk);
      if (nk > 1e-10 * n0 && nk > 0.0) {
        R[k][k] = nk;
        for (int64_t r = 0; r < m; ++r) Q[r * kModes + k] = Q[r * kModes + k] / nk;
      } else {
        for (int64_t r = 0; r < m; ++r) Q[r * kModes + k] = 0.0;
      }
    }
    for (size_t t = 0; t < mem[a].size(); ++t)
      for (int d = 0; d < b; ++d)
        for (int k = 0; k < kModes; ++k) lev.Pt[(mem[a][t] * b + d) * kModes + k] = Q[(t * b + d) * kModes + k];
    for (int r = 0; r < kModes; ++r)
      for (int k = 0; k < kModes; ++k) Bc[(a * kModes + r) * kModes + k] = R[r][k];
  }
}

// P = (I - omega D^{-1} A) P_tent, omega = (4/3) / lambda_hat.  Row of node i (none for nodes that aggregation
// left out): a block for every aggregate among the nodes of A's row, in ascending order;
// block(i, a) = [a == agg(i)] P_tent(i) - omega D_i^{-1} S, S = sum over the row's nodes j in aggregate a
// (ascending) of A_ij P_tent(j).
BSR rbm_prolongator(const BLevel& lev) {
  const BSR& A = lev.A;
  const int b = lev.b;
  const int64_t n = A.nbr;
  const double omega = (4.0 / 3.0) / lev.lam;
  BSR P; P.nbr = n; P.nbc = lev.nagg; P.br = b; P.bc = kModes; P.rp.assign(n + 1, 0);
  const int bs = b * kModes;
  std::vector<std::vector<int32_t>> tci(kTasks);
  std::vector<vec> tv(kTasks);
  std::vector<uint8_t> excl(n, 1);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q)
      if (A.ci[q] != i)
        for (int e = 0; e < b * b; ++e)
          if (A.v[q * b * b + e] != 0.0) excl[i] = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int t = 0; t < kTasks; ++t) {
    std::vector<int32_t> aggs;
    for (int64_t i = task_lo(n, t); i < task_lo(n, t + 1); ++i) {
      if (excl[i]) continue;
      aggs.clear();
      for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q)
        if (lev.agg[A.ci[q]] >= 0) aggs.push_back(lev.agg[A.ci[q]]);
      std::sort(aggs.begin(), aggs.end());
      aggs.erase(std::unique(aggs.begin(), aggs.end()), aggs.end());
      for (int32_t a : aggs) {
        double S[6][kModes] = {{0.0}};
        for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q) {
          const int64_t j = A.ci[q];
          if (lev.agg[j] != a) continue;
          for (int r = 0; r < b; ++r)
            for (int c = 0; c < kModes; ++c) {
              double p = 0.0;
              for (int e = 0; e < b; ++e) p = p + A.v[(q * b + r) * b + e] * lev.Pt[(j * b + e) * kModes + c];
              S[r][c] = S[r][c] + p;
            }
        }
        tci[t].push_back(a);
        for (int r = 0; r < b; ++r)
          for (int c = 0; c < kModes; ++c) {
            const double delta = a == lev.agg[i] ? lev.Pt[(i * b + r) * kModes + c] : 0.0;
            tv[t].push_back(delta - (omega / lev.dg[i * b + r]) * S[r][c]);
          }
      }
      P.rp[i + 1] = int64_t(aggs.size());
    }
  }
  for (int64_t i = 0; i < n; ++i) P.rp[i + 1] += P.rp[i];
  for (int t = 0; t < kTasks; ++t) {
    P.ci.insert(P.ci.end(), tci[t].begin(), tci[t].end());
    P.v.insert(P.v.end(), tv[t].begin(), tv[t].end());
  }
  (void)bs;
  return P;
}

bool build_rbm(BAMG& H, BSR A0, vec B0, double theta0, int coarse_max, int max_levels) {
  H.L.clear();
  H.L.emplace_back();
  H.L[0].A = std::move(A0);
  H.L[0].b = 3;
  H.L[0].B = std::move(B0);
  double theta = theta0;
  for (int l = 0;; ++l) {
    BLevel& lev = H.L[l];
    const int b = lev.b;
    const int64_t n = lev.A.nbr;
    // coarse_max counts nodes: a level is coarsest at 3 coarse_max unknowns, as many as coarse_max nodes carry
    bool coarsest = n * b <= int64_t(3) * coarse_max || l + 1 >= max_levels;
    if (!coarsest) {
      Level sl;
      sl.A = block_strength(lev.A);
      aggregate(sl, theta, l);
      lev.agg = sl.agg;
      lev.nagg = sl.nagg;
      if (lev.nagg == 0 || double(n) / double(lev.nagg) < 1.2) coarsest = true;
    }
    lev.dg.assign(n * b, 0.0);
    for (int64_t i = 0; i < n; ++i) {
      const int64_t q = lev.A.find(i, i);
      for (int a = 0; a < b; ++a) lev.dg[i * b + a] = lev.A.v[(q * b + a) * b + a];
    }
    if (coarsest) {
      if (n * b > 12000) return false;
      lev.coarsest = true;
      lev.agg.clear(); lev.nagg = 0;
      vec d(size_t(n * b) * (n * b), 0.0);
      bsr_dense(lev.A, d, 0, 0, n * b);
      lev.lu.factor(n * b, std::move(d));
      break;
    }
    lev.lam = block_gershgorin(lev.A);
    vec Bc;
    tentative(lev, Bc);
    lev.P = rbm_prolongator(lev);
    lev.R = bsr_transpose(lev.P);
    BSR AP = bsr_spgemm(lev.A, lev.P);
    BSR Ac = bsr_spgemm(lev.R, AP);
    // a mode that an aggregate cannot represent (dependent column of its QR) gives a zero prolongator column,
    // hence a zero row and column of A_c: its diagonal entry is set to one, which decouples that coarse unknown
    for (int64_t I = 0; I < Ac.nbr; ++I) {
      const int64_t q = Ac.find(I, I);
      for (int k = 0; k < kModes; ++k)
        if (Ac.v[(q * kModes + k) * kModes + k] == 0.0) Ac.v[(q * kModes + k) * kModes + k] = 1.0;
    }
    H.L.emplace_back();
    BLevel& nx = H.L[l + 1];
    nx.A = std::move(Ac);
    nx.b = kModes;
    nx.B = std::move(Bc);
    theta *= 0.5;
  }
  return true;
}

// Chebyshev smoother on D^{-1} A over [lambda_hat/ratio, lambda_hat], the recurrence of chebyshev() above
void block_chebyshev(const BLevel& lev, const vec& b, vec& x, int degree, double ratio, bool zero) {
  const int64_t n = lev.A.nbr * lev.b;
  double lmax = lev.lam, lmin = lmax / ratio;
  double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
  double sigma = theta / delta, rho = 1.0 / sigma;
  vec r(n), d(n), Ax(n);
  if (zero) {
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] / lev.dg[i];
  } else {
    bsr_apply(lev.A, x.data(), Ax.data());
    for (int64_t i = 0; i < n; ++i) r[i] = (b[i] - Ax[i]) / lev.dg[i];
  }
  for (int64_t i = 0; i < n; ++i) d[i] = r[i] / theta;
  for (int k = 0; k < degree; ++k) {
    for (int64_t i = 0; i < n; ++i) x[i] = x[i] + d[i];
    if (k == degree - 1) break;
    bsr_apply(lev.A, x.data(), Ax.data());
    for (int64_t i = 0; i < n; ++i) r[i] = (b[i] - Ax[i]) / lev.dg[i];
    double rn = 1.0 / (2.0 * sigma - rho);
    for (int64_t i = 0; i < n; ++i) d[i] = rn * rho * d[i] + 2.0 * rn / delta * r[i];
    rho = rn;
  }
}

// V-cycle on the block hierarchy: pre-smoothing from x = 0, x += P V(R (b - A x)), post-smoothing
void block_vcycle(const BAMG& H, int l, const vec& b, vec& x, const Smooth& sm) {
  const BLevel& lev = H.L[l];
  const int64_t n = lev.A.nbr * lev.b;
  x.assign(n, 0.0);
  if (lev.coarsest) { lev.lu.solve(b.data(), x.data()); return; }
  block_chebyshev(lev, b, x, sm.degree, sm.ratio, true);
  vec Ax(n), r(n);
  bsr_apply(lev.A, x.data(), Ax.data());
  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - Ax[i];
  vec bc(lev.R.nbr * kModes), xc;
  bsr_apply(lev.R, r.data(), bc.data());
  block_vcycle(H, l + 1, bc, xc, sm);
  vec Pe(n);
  bsr_apply(lev.P, xc.data(), Pe.data());
  for (int64_t i = 0; i < n; ++i) x[i] = x[i] + Pe[i];
  block_chebyshev(lev, b, x, sm.degree, sm.ratio, false);
}

}  // namespace

// ---------------------------------------------------------------------------
// Preconditioner state
// ---------------------------------------------------------------------------
static Smooth smooth_of(const or_prec_params& pp) {
  Smooth s;
  s.kind = pp.smoother; s.pre = pp.pre; s.post = pp.post; s.degree = pp.cheb_degree; s.ratio = pp.cheb_ratio;
  return s;
}

// M_uu^{-1} of §5.2 on a node-major displacement vector: one V-cycle per component on the shared hierarchy
static void mech_apply(const AMG& H, const Smooth& sm, int64_t nn, const double* vu, double* zu) {
  for (int c = 0; c < 3; ++c) {
    vec b(nn), x;
#pragma omp parallel for schedule(static)
    for (int64_t I = 0; I < nn; ++I) b[I] = vu[3 * I + c];
    vcycle(H, 0, c, b, x, sm);
#pragma omp parallel for schedule(static)
    for (int64_t I = 0; I < nn; ++I) zu[3 * I + c] = x[I];
  }
}

struct or_prec {
  const or_system* s = nullptr;
  or_prec_params pp;
  BSR A_fu, A_ff, Sff;  // Sff = S_ff^(FS), §5.1
  vec dss, dps;         // quasi-IMPES diagonals, §5.3
  CSR spp;
  AMG amg_u, amg_p;
  BAMG amg_rbm;         // OR_MECH_AMG_RBM: rigid-body-mode smoothed aggregation on the full A_uu
  BSR ilu;              // L (unit, strictly lower) and U (upper) blocks in the S_ff pattern
  vec dinv;             // inv(U_ii)
  vec gs_dinv;          // inv of the diagonal blocks of S_ff^(FS) (block Gauss-Seidel)
  vec dfs;              // (D_sp, D_pp) per cell added to S_ff: the system's d_fs or the row-sum lumping
  DenseLU lu_uu, lu_flow, lu_local, lu_pp, lu_full;
};

extern "C" {

uint64_t or_splitmix64(uint64_t state) { return sm64(state); }

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_correlated_field(uint64_t seed, int field, int nx, int ny, int nz, int Lx, int Ly, int Lz, double* out) {
  vec f = correlated_field(seed, field, nx, ny, nz, Lx, Ly, Lz);
  std::memcpy(out, f.data(), f.size() * sizeof(double));
}

void or_default_params(or_gen_params* gp, int config) {
  std::memset(gp, 0, sizeof(*gp));
  gp->h = 10.0;
  gp->seed = 1000 + config;
  gp->field_kind = config == 0 ? OR_FIELDS_LOGNORMAL : config == 2 ? OR_FIELDS_CHANNELS : OR_FIELDS_LAYERED;
  if (config == 0) { gp->nx = 8; gp->ny = 8; gp->nz = 4; }
  else if (config == 1) { gp->nx = 64; gp->ny = 64; gp->nz = 32; }
  else if (config == 2) { gp->nx = 60; gp->ny = 220; gp->nz = 85; }
  else { gp->nx = 16; gp->ny = 16; gp->nz = 8; }
  gp->flags = OR_ALL;
  gp->dt = 86400.0;
  gp->biot = 0.8;
  gp->c_w = gp->c_nw = gp->c_r = 1e-9;
  gp->mu_w = 1e-3; gp->mu_nw = 5e-3;
  gp->rho_w0 = 1035.0; gp->rho_nw0 = 863.0; gp->rho_s0 = 2650.0;
  gp->s_wr = 0.2; gp->s_nwr = 0.2;
  gp->grav = 9.81;
  gp->p_ref = 20e6;
  gp->dp_amp = 5e6;
  gp->corey = 2.0;
  gp->E0 = 1e10; gp->nu0 = 0.25; gp->kappa0 = 100.0 * kMilliDarcy; gp->phi0 = 0.2; gp->sw0 = 0.5;
}

// the Jacobian at the state base + dx (dx = NULL: the base state u = 0, s = S_w, p of the fields), the base
// state being the previous time level
static int generate_at(const or_gen_params* gp, const double* dx, or_system** out) {
  if (gp->nx < 1 || gp->ny < 1 || gp->nz < 1 || !wells_ok(*gp)) return 1;
  Grid g{gp->nx, gp->ny, gp->nz, gp->h};
  Fields F = make_fields(*gp);
  State st;
  st.s = F.sw; st.p = F.p;
  if (dx) {
    const int64_t nu = 3 * g.nn();
    st.u.assign(dx, dx + nu);
    for (int64_t c = 0; c < g.ncell(); ++c) { st.s[c] += dx[nu + 2 * c]; st.p[c] += dx[nu + 2 * c + 1]; }
  }
  Jac J;
  ExtraBC bc;
  assemble(*gp, g, F, st, bc, J);
  finalize(*gp, g, J, (gp->flags & OR_SCALE) != 0);
  or_system* s = (or_system*)std::calloc(1, sizeof(or_system));
  s->nx = g.nx; s->ny = g.ny; s->nz = g.nz; s->h = g.h;
  s->n_nodes = g.nn(); s->n_cells = g.ncell();
  s->n_u = 3 * s->n_nodes; s->n_f = 2 * s->n_cells; s->n = s->n_u + s->n_f;
  s->nnzb_uu = J.uu.ci.size(); s->nnzb_uf = J.uf.ci.size(); s->nnzb_fu = J.fu.ci.size(); s->nnzb_ff = J.ff.ci.size();
  s->uu_rp = dup(J.uu.rp); s->uu_ci = dup(J.uu.ci); s->uu_v = dup(J.uu.v);
  s->uf_rp = dup(J.uf.rp); s->uf_ci = dup(J.uf.ci); s->uf_v = dup(J.uf.v);
  s->fu_rp = dup(J.fu.rp); s->fu_ci = dup(J.fu.ci); s->fu_v = dup(J.fu.v);
  s->ff_rp = dup(J.ff.rp); s->ff_ci = dup(J.ff.ci); s->ff_v = dup(J.ff.v);
  s->d_fs = dup(J.dfs);
  s->dirichlet = dup(J.dir);
  vec rhs(s->n, 0.0);
  for (int64_t r = 0; r < s->n; ++r) {
    if (r < s->n_u && J.dir[r]) continue;
    rhs[r] = 2.0 * unif(gp->seed, F_RHS, 0, uint64_t(r)) - 1.0;
  }
  s->rhs = dup(rhs);
  s->alpha_u = J.alpha_u; s->alpha_f = J.alpha_f;
  s->E = dup(F.E); s->nu = dup(F.nu); s->kh = dup(F.kh); s->kv = dup(F.kv);
  s->phi0 = dup(F.phi0); s->sw = dup(F.sw); s->p = dup(F.p);
  *out = s;
  return 0;
}

int or_generate(const or_gen_params* gp, or_system** out) { return generate_at(gp, nullptr, out); }
int or_generate_at(const or_gen_params* gp, const double* dx, or_system** out) { return generate_at(gp, dx, out); }

void or_system_free(or_system* s) {
  if (!s) return;
  void* ptrs[] = {s->uu_rp, s->uu_ci, s->uu_v, s->uf_rp, s->uf_ci, s->uf_v, s->fu_rp, s->fu_ci, s->fu_v,
                  s->ff_rp, s->ff_ci, s->ff_v, s->d_fs, s->dirichlet, s->rhs, s->E, s->nu, s->kh, s->kv,
                  s->phi0, s->sw, s->p};
  for (void* p : ptrs) std::free(p);
  std::free(s);
}

void or_spmv(const or_system* s, const double* x, double* y) {
  const double* xu = x;
  const double* xf = x + s->n_u;
#pragma omp parallel for schedule(static)
  for (int64_t I = 0; I < s->n_nodes; ++I) {
    double acc[3] = {0, 0, 0};
    for (int64_t q = s->uu_rp[I]; q < s->uu_rp[I + 1]; ++q)
      for (int d = 0; d < 3; ++d)
        for (int e = 0; e < 3; ++e) acc[d] += s->uu_v[q * 9 + d * 3 + e] * xu[3 * int64_t(s->uu_ci[q]) + e];
    for (int64_t q = s->uf_rp[I]; q < s->uf_rp[I + 1]; ++q)
      for (int d = 0; d < 3; ++d)
        for (int e = 0; e < 2; ++e) acc[d] += s->uf_v[q * 6 + d * 2 + e] * xf[2 * int64_t(s->uf_ci[q]) + e];
    for (int d = 0; d < 3; ++d) y[3 * I + d] = acc[d];
  }
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < s->n_cells; ++c) {
    double acc[2] = {0, 0};
    for (int64_t q = s->fu_rp[c]; q < s->fu_rp[c + 1]; ++q)
      for (int a = 0; a < 2; ++a)
        for (int e = 0; e < 3; ++e) acc[a] += s->fu_v[q * 6 + a * 3 + e] * xu[3 * int64_t(s->fu_ci[q]) + e];
    for (int64_t q = s->ff_rp[c]; q < s->ff_rp[c + 1]; ++q)
      for (int a = 0; a < 2; ++a)
        for (int e = 0; e < 2; ++e) acc[a] += s->ff_v[q * 4 + a * 2 + e] * xf[2 * int64_t(s->ff_ci[q]) + e];
    y[s->n_u + 2 * c] = acc[0];
    y[s->n_u + 2 * c + 1] = acc[1];
  }
}

void or_ref_integrals(double h, double* G, double* IN, double* IdN, double* INdN) {
  RefInt R = ref_integrals(h);
  std::memcpy(G, R.G, sizeof(R.G));
  std::memcpy(IN, R.IN, sizeof(R.IN));
  std::memcpy(IdN, R.IdN, sizeof(R.IdN));
  std::memcpy(INdN, R.INdN, sizeof(R.INdN));
}

}  // extern "C"

namespace {
// Residual of the discrete weak form, Eq. (5a)-(5c) with the App. B element and
// face contributions, at x_n = (u, s, p); the previous level is `prev`.  The
// face term carries the sign under which its derivative is the App. B face
// Jacobian (Dt sum_f [[psi]] F).
void residual(const or_gen_params& gp, const Grid& g, const Fields& F, const State& prev, const State& x,
              const ExtraBC& bc, vec& r) {
  RefInt R = ref_integrals(g.h);
  int64_t nn = g.nn(), nc = g.ncell();
  r.assign(3 * nn + 2 * nc, 0.0);
  double grav = (gp.flags & OR_GRAVITY) ? gp.grav : 0.0;
  double V = g.h * g.h * g.h;
  double b = gp.biot;
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        int64_t c = g.cell(i, j, k);
        int64_t nodes[8];
        for (int a = 0; a < 8; ++a) nodes[a] = g.node(i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
        Mat m0 = material(gp, F.E[c], F.nu[c], F.phi0[c], x.s[c], x.p[c], 0.0);
        double s = x.s[c], p = x.p[c];
        double int_ev = 0.0;
        for (int q = 0; q < 8; ++q) {
          double gu[3][3] = {{0}};
          for (int a = 0; a < 8; ++a)
            for (int d = 0; d < 3; ++d)
              for (int e = 0; e < 3; ++e) gu[d][e] += x.u[3 * nodes[a] + d] * R.gp_dN[q][a][e];
          double ev = gu[0][0] + gu[1][1] + gu[2][2];
          int_ev += R.gp_w * ev;
          double sig[3][3];
          for (int d = 0; d < 3; ++d)
            for (int e = 0; e < 3; ++e)
              sig[d][e] = m0.lam * ev * (d == e) + m0.G * (gu[d][e] + gu[e][d]);
          double phi = F.phi0[c] + b * ev + m0.dphidp * (p - gp.p_ref);
          double rho = (1.0 - phi) * m0.rs + phi * (s * m0.rw + (1.0 - s) * m0.rnw);
          for (int a = 0; a < 8; ++a)
            for (int d = 0; d < 3; ++d) {
              double v = 0.0;
              for (int e = 0; e < 3; ++e) v += sig[d][e] * R.gp_dN[q][a][e];
              v -= R.gp_dN[q][a][d] * b * p;
              double gd = d == 2 ? -grav : 0.0;
              v -= R.gp_N[q][a] * rho * gd;
              r[3 * nodes[a] + d] += R.gp_w * v;
            }
        }
        if (gp.flags & OR_ACCUM) {
          // int_K phi rho_l s_l, phi linear in the pointwise volumetric strain
          double phiV = V * (F.phi0[c] + m0.dphidp * (p - gp.p_ref)) + b * int_ev;
          Mat mp = material(gp, F.E[c], F.nu[c], F.phi0[c], prev.s[c], prev.p[c], 0.0);
          double int_evp = 0.0;  // int_K eps_v of the previous displacement
          for (int a = 0; a < 8; ++a)
            for (int d = 0; d < 3; ++d) int_evp += R.IdN[a][d] * prev.u[3 * nodes[a] + d];
          double phiVp = V * (F.phi0[c] + mp.dphidp * (prev.p[c] - gp.p_ref)) + b * int_evp;
          r[3 * nn + 2 * c] += phiV * m0.rw * s - phiVp * mp.rw * prev.s[c];
          r[3 * nn + 2 * c + 1] += phiV * m0.rnw * (1.0 - s) - phiVp * mp.rnw * (1.0 - prev.s[c]);
        }
      }
  if (bc.active && bc.sigma_top != 0.0) {
    // - int eta . tbar, tbar = (0,0,-sigma) on the top face: +sigma h^2/4 per node
    // each top face contributes sigma * h^2/4 to each of its four nodes
    for (int j = 0; j <= g.ny; ++j)
      for (int i = 0; i <= g.nx; ++i) {
        double fx = (i == 0 || i == g.nx) ? 1.0 : 2.0, fy = (j == 0 || j == g.ny) ? 1.0 : 2.0;
        r[3 * g.node(i, j, g.nz) + 2] += bc.sigma_top * g.h * g.h / 4.0 * fx * fy;
      }
  }
  if (gp.flags & OR_FLUX) {
    for (int k = 0; k < g.nz; ++k)
      for (int j = 0; j < g.ny; ++j)
        for (int i = 0; i < g.nx; ++i) {
          int64_t K = g.cell(i, j, k);
          for (int dir = 0; dir < 3; ++dir) {
            int a = i + (dir == 0), b2 = j + (dir == 1), c2 = k + (dir == 2);
            if (a >= g.nx || b2 >= g.ny || c2 >= g.nz) continue;
            int64_t L = g.cell(a, b2, c2);
            double kK = dir == 2 ? F.kv[K] : F.kh[K], kL = dir == 2 ? F.kv[L] : F.kh[L];
            double UK = g.h * g.h * kK / (0.5 * g.h), UL = g.h * g.h * kL / (0.5 * g.h);
            double Ups = UK * UL / (UK + UL);
            double dz = dir == 2 ? g.h : 0.0;
            for (int ph = 0; ph < 2; ++ph) {
              FaceFlux f = face_flux(gp, Ups, dz, grav, ph, x.s[K], x.p[K], x.s[L], x.p[L], false);
              r[3 * nn + 2 * K + ph] += -gp.dt * f.F;
              r[3 * nn + 2 * L + ph] += gp.dt * f.F;
            }
          }
        }
    if (bc.active && bc.top_drained)
      for (int j = 0; j < g.ny; ++j)
        for (int i = 0; i < g.nx; ++i) {
          int64_t K = g.cell(i, j, g.nz - 1);
          double Ups = g.h * g.h * F.kv[K] / (0.5 * g.h);
          for (int ph = 0; ph < 2; ++ph) {
            FaceFlux f = face_flux(gp, Ups, 0.5 * g.h, grav, ph, x.s[K], x.p[K], bc.s_top, bc.p_top, true);
            r[3 * nn + 2 * K + ph] += -gp.dt * f.F;
          }
        }
  }
  if (gp.flags & OR_WELLS)
    for (int k = 0; k < g.nz; ++k)
      for (int j = 0; j < g.ny; ++j)
        for (int i = 0; i < g.nx; ++i) {
          const int kind = well_kind(g, i, j);
          if (!kind) continue;
          const int64_t K = g.cell(i, j, k);
          const WellTerm w = well_term(gp, g, F, kind, K, k, x.s[K], x.p[K]);
          r[3 * nn + 2 * K] += w.r[0];
          r[3 * nn + 2 * K + 1] += w.r[1];
        }
}

void full_dense(const or_system* s, vec& d) {
  int64_t n = s->n;
  d.assign(size_t(n) * n, 0.0);
  bsr_dense(to_bsr(s, 0), d, 0, 0, n);
  bsr_dense(to_bsr(s, 1), d, 0, s->n_u, n);
  bsr_dense(to_bsr(s, 2), d, s->n_u, 0, n);
  bsr_dense(to_bsr(s, 3), d, s->n_u, s->n_u, n);
}

typedef std::function<void(const double*, double*)> Op;

// Flexible GMRES(m), right preconditioned (§4), modified Gram-Schmidt,
// Givens rotations, restart from the current iterate, x0 = 0.
void fgmres(int64_t n, const Op& A, const Op& M, const double* b, double* x, double tol, int m, int maxit,
            or_stats* st) {
  std::memset(st, 0, sizeof(*st));
  double bn = std::sqrt(dot(b, b, n));
  for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
  if (bn == 0.0) { st->converged = 1; return; }
  vec r(b, b + n), w(n);
  int total = 0;
  for (;;) {
    double beta = std::sqrt(dot(r.data(), r.data(), n));
    std::vector<vec> V, Z;
    V.emplace_back(n);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) V[0][i] = r[i] / beta;
    vec H(size_t(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1, 0.0);
    g[0] = beta;
    int jend = -1;
    bool brk = false;
    for (int j = 0; j < m; ++j) {
      Z.emplace_back(n);
      M(V[j].data(), Z[j].data());
      A(Z[j].data(), w.data());
      for (int i = 0; i <= j; ++i) {
        double h = dot(w.data(), V[i].data(), n);
        H[i * m + j] = h;
#pragma omp parallel for schedule(static)
        for (int64_t e = 0; e < n; ++e) w[e] -= h * V[i][e];
      }
      double hn = std::sqrt(dot(w.data(), w.data(), n));
      H[(j + 1) * m + j] = hn;
      for (int i = 0; i < j; ++i) {
        double a = H[i * m + j], c = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * c;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      double a = H[j * m + j], c = H[(j + 1) * m + j];
      double rr = std::hypot(a, c);
      cs[j] = a / rr; sn[j] = c / rr;
      H[j * m + j] = rr; H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++total;
      st->est_relres = std::fabs(g[j + 1]) / bn;
      jend = j;
      if (!(hn > 1e-300)) brk = true;
      if (st->est_relres <= tol || brk || total >= maxit || j == m - 1) break;
      V.emplace_back(n);
#pragma omp parallel for schedule(static)
      for (int64_t e = 0; e < n; ++e) V[j + 1][e] = w[e] / hn;
    }
    vec y(jend + 1);
    for (int i = jend; i >= 0; --i) {
      double s = g[i];
      for (int k2 = i + 1; k2 <= jend; ++k2) s -= H[i * m + k2] * y[k2];
      y[i] = s / H[i * m + i];
    }
    for (int i = 0; i <= jend; ++i) {
#pragma omp parallel for schedule(static)
      for (int64_t e = 0; e < n; ++e) x[e] += y[i] * Z[i][e];
    }
    A(x, w.data());
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < n; ++e) r[e] = b[e] - w[e];
    double rn = dot(r.data(), r.data(), n);
    st->true_relres = std::sqrt(rn) / bn;
    st->iters = total;
    if (std::isnan(st->true_relres)) return;
    if (st->true_relres <= tol) { st->converged = 1; return; }
    if (brk) { st->breakdown = 1; return; }
    if (total >= maxit) return;
    st->restarts++;
  }
}

}  // namespace

extern "C" {

int or_residual(const or_gen_params* gp, const double* dx, double* r) {
  if (!wells_ok(*gp)) return 1;
  Grid g{gp->nx, gp->ny, gp->nz, gp->h};
  Fields F = make_fields(*gp);
  State prev;
  prev.u.assign(3 * g.nn(), 0.0); prev.s = F.sw; prev.p = F.p;
  State x = prev;
  int64_t nu = 3 * g.nn();
  for (int64_t i = 0; i < nu; ++i) x.u[i] += dx[i];
  for (int64_t c = 0; c < g.ncell(); ++c) { x.s[c] += dx[nu + 2 * c]; x.p[c] += dx[nu + 2 * c + 1]; }
  vec rv;
  ExtraBC bc;
  residual(*gp, g, F, prev, x, bc, rv);
  std::memcpy(r, rv.data(), rv.size() * sizeof(double));
  return 0;
}

void or_default_prec_params(or_prec_params* pp) {
  std::memset(pp, 0, sizeof(*pp));
  pp->theta_u = 0.08; pp->theta_p = 0.08;
  pp->coarse_max_u = 500; pp->coarse_max_p = 500;
  pp->max_levels = 25;
  pp->pre = 1; pp->post = 1;
  pp->smoother = 1; pp->cheb_degree = 2; pp->cheb_ratio = 20.0;
  pp->local_sweeps = 3;
  pp->ilu_tile_y = 16;
  pp->ilu_tile_z = 8;
}

int or_prec_setup(const or_system* s, const or_prec_params* pp, or_prec** out) {
  return or_prec_setup_reuse(s, s, pp, out);
}

int or_prec_setup_reuse(const or_system* s, const or_system* mech, const or_prec_params* pp, or_prec** out) {
  if (mech->n_nodes != s->n_nodes || mech->nnzb_uu != s->nnzb_uu) return 4;
  or_prec* P = new or_prec();
  P->s = s; P->pp = *pp;
  int64_t nc = s->n_cells, nn = s->n_nodes;
  P->A_fu = to_bsr(s, 2);
  P->A_ff = to_bsr(s, 3);
  BSR Auu = to_bsr(s, 0);
  // §5.2: M_uu = amg(A_uu^(SDC)), three displacement components, shared aggregates
  if (pp->mech_mode == OR_MECH_AMG) {
    BSR AuuM = to_bsr(mech, 0);
    CSR A0; A0.n = A0.m = nn; A0.nc = 3; A0.rp = AuuM.rp; A0.ci = AuuM.ci;
    A0.v.resize(AuuM.ci.size() * 3);
    for (size_t q = 0; q < AuuM.ci.size(); ++q)
      for (int d = 0; d < 3; ++d) A0.v[q * 3 + d] = AuuM.v[q * 9 + d * 4];
    if (!build_amg(P->amg_u, std::move(A0), pp->theta_u, pp->coarse_max_u, pp->max_levels)) { delete P; return 2; }
  } else if (pp->mech_mode == OR_MECH_AMG_RBM) {
    if (pp->smoother != 1) { delete P; return 4; }
    if (!build_rbm(P->amg_rbm, to_bsr(mech, 0), rigid_body_modes(s->nx, s->ny, s->nz), pp->theta_u,
                   pp->coarse_max_u, pp->max_levels)) { delete P; return 2; }
  } else {
    vec d(size_t(s->n_u) * s->n_u, 0.0);
    bsr_dense(Auu, d, 0, 0, s->n_u);
    P->lu_uu.factor(s->n_u, std::move(d));
  }
  // fixed-stress diagonal: the system's d_fs, or the row-sum lumping of the §5.1 remark,
  // D_sp = -diag(A_su A_uu^{-1} A_up e), D_pp = -diag(A_pu A_uu^{-1} A_up e), with A_uu^{-1} replaced by
  // one application of M_uu^{-1} (OR_FS_RSL) or taken exactly by dense LU (OR_FS_RSL_EXACT)
  P->dfs.assign(s->d_fs, s->d_fs + 2 * nc);
  if (pp->fs_mode == OR_FS_RSL || pp->fs_mode == OR_FS_RSL_EXACT) {
    BSR Auf = to_bsr(s, 1);
    vec aupe(3 * nn, 0.0), w(3 * nn, 0.0);
    for (int64_t I = 0; I < nn; ++I)
      for (int64_t q = Auf.rp[I]; q < Auf.rp[I + 1]; ++q)
        for (int d = 0; d < 3; ++d) aupe[3 * I + d] = aupe[3 * I + d] + Auf.v[q * 6 + d * 2 + 1];
    if (pp->fs_mode == OR_FS_RSL) {
      if (pp->mech_mode == OR_MECH_AMG) {
        mech_apply(P->amg_u, smooth_of(*pp), nn, aupe.data(), w.data());
      } else if (pp->mech_mode == OR_MECH_AMG_RBM) {
        vec wv;
        block_vcycle(P->amg_rbm, 0, aupe, wv, smooth_of(*pp));
        w = wv;
      } else {
        delete P;
        return 3;
      }
    } else {
      vec d(size_t(s->n_u) * s->n_u, 0.0);
      bsr_dense(Auu, d, 0, 0, s->n_u);
      DenseLU lu; lu.factor(s->n_u, std::move(d));
      lu.solve(aupe.data(), w.data());
    }
    for (int64_t c = 0; c < nc; ++c)
      for (int a = 0; a < 2; ++a) {
        double acc = 0.0;
        for (int64_t q = P->A_fu.rp[c]; q < P->A_fu.rp[c + 1]; ++q)
          for (int e = 0; e < 3; ++e) acc += P->A_fu.v[q * 6 + a * 3 + e] * w[3 * int64_t(P->A_fu.ci[q]) + e];
        P->dfs[2 * c + a] = -acc;
      }
  }
  // §5.1, fixed-stress Schur approximation: S_ff^(FS) = A_ff + blockdiag([[0, D_sp],[0, D_pp]])
  P->Sff = P->A_ff;
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nc; ++c) {
    int64_t q = P->Sff.find(c, c);
    P->Sff.v[q * 4 + 1] = P->Sff.v[q * 4 + 1] + P->dfs[2 * c];
    P->Sff.v[q * 4 + 3] = P->Sff.v[q * 4 + 3] + P->dfs[2 * c + 1];
  }
  // §5.3 quasi-IMPES: D_ss = diagm(A_ss), D_ps = diagm(A_ps); or true-IMPES: D_ss = diag(A_ss^T e),
  // D_ps = diag(A_ps^T e), column sums taken over the rows in ascending order;
  // S_pp = A_pp^(FS) - D_ps D_ss^{-1} A_sp^(FS)
  P->dss.resize(nc); P->dps.resize(nc);
  if (pp->cpr_reduction == OR_CPR_TRUE_IMPES) {
    for (int64_t c = 0; c < nc; ++c) { P->dss[c] = 0.0; P->dps[c] = 0.0; }
    for (int64_t r = 0; r < nc; ++r)
      for (int64_t q = P->A_ff.rp[r]; q < P->A_ff.rp[r + 1]; ++q) {
        int64_t c = P->A_ff.ci[q];
        P->dss[c] = P->dss[c] + P->A_ff.v[q * 4 + 0];
        P->dps[c] = P->dps[c] + P->A_ff.v[q * 4 + 2];
      }
  } else {
    for (int64_t c = 0; c < nc; ++c) {
      int64_t q = P->A_ff.find(c, c);
      P->dss[c] = P->A_ff.v[q * 4 + 0];
      P->dps[c] = P->A_ff.v[q * 4 + 2];
    }
  }
  P->spp.n = P->spp.m = nc; P->spp.nc = 1;
  P->spp.rp = P->Sff.rp; P->spp.ci = P->Sff.ci;
  P->spp.v.resize(P->Sff.ci.size());
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nc; ++c) {
    double ratio = P->dps[c] / P->dss[c];
    for (int64_t q = P->Sff.rp[c]; q < P->Sff.rp[c + 1]; ++q)
      P->spp.v[q] = P->Sff.v[q * 4 + 3] - ratio * P->Sff.v[q * 4 + 1];
  }
  if (pp->press_mode == OR_PRESS_AMG) {
    if (!build_amg(P->amg_p, P->spp, pp->theta_p, pp->coarse_max_p, pp->max_levels)) { delete P; return 2; }
  } else {
    vec d(size_t(nc) * nc, 0.0);
    for (int64_t i = 0; i < nc; ++i)
      for (int64_t q = P->spp.rp[i]; q < P->spp.rp[i + 1]; ++q) d[i * nc + P->spp.ci[q]] = P->spp.v[q];
    P->lu_pp.factor(nc, std::move(d));
  }
  // §5.3 option 2: block ILU(0) of the interleaved S_ff^(FS), natural cell order (IKJ).  Processor-local
  // ILU(0) (the paper's runs factor each process's own rows): the ILU(0) of S_ff with the blocks that couple
  // cells of different subdomains set to zero, a subdomain being a column of ty x tz cells in (y, z)
  P->ilu = P->Sff;
  if (pp->ilu_tile_y > 0 && pp->ilu_tile_z > 0) {
    const int64_t gx = s->nx, gy = s->ny;
    const int64_t nby = (gy + pp->ilu_tile_y - 1) / pp->ilu_tile_y;
    auto sub = [&](int64_t c) {
      const int64_t y = (c / gx) % gy, z = c / (gx * gy);
      return y / pp->ilu_tile_y + nby * (z / pp->ilu_tile_z);
    };
    for (int64_t i = 0; i < nc; ++i)
      for (int64_t q = P->ilu.rp[i]; q < P->ilu.rp[i + 1]; ++q)
        if (sub(P->ilu.ci[q]) != sub(i))
          for (int e = 0; e < 4; ++e) P->ilu.v[q * 4 + e] = 0.0;
  }
  P->dinv.assign(4 * nc, 0.0);
  for (int64_t i = 0; i < nc; ++i) {
    for (int64_t qk = P->ilu.rp[i]; qk < P->ilu.rp[i + 1]; ++qk) {
      int64_t k = P->ilu.ci[qk];
      if (k >= i) break;
      double L[4];
      mul22(&P->ilu.v[qk * 4], &P->dinv[4 * k], L);
      std::memcpy(&P->ilu.v[qk * 4], L, sizeof(L));
      for (int64_t qj = qk + 1; qj < P->ilu.rp[i + 1]; ++qj) {
        int64_t jj = P->ilu.ci[qj];
        int64_t qkj = P->ilu.find(k, jj);
        if (qkj < 0) continue;
        double t[4];
        mul22(L, &P->ilu.v[qkj * 4], t);
        for (int e = 0; e < 4; ++e) P->ilu.v[qj * 4 + e] -= t[e];
      }
    }
    inv22(&P->ilu.v[P->ilu.find(i, i) * 4], &P->dinv[4 * i]);
  }
  // §5.3 option 1: block Gauss-Seidel needs the inverse diagonal blocks of S_ff^(FS)
  P->gs_dinv.assign(4 * nc, 0.0);
  for (int64_t i = 0; i < nc; ++i) inv22(&P->Sff.v[P->Sff.find(i, i) * 4], &P->gs_dinv[4 * i]);
  if (pp->flow_mode == OR_FLOW_EXACT_FS || pp->local_mode == OR_LOCAL_EXACT) {
    vec d(size_t(s->n_f) * s->n_f, 0.0);
    bsr_dense(P->Sff, d, 0, 0, s->n_f);
    if (pp->flow_mode == OR_FLOW_EXACT_FS) P->lu_flow.factor(s->n_f, d);
    if (pp->local_mode == OR_LOCAL_EXACT) P->lu_local.factor(s->n_f, d);
  }
  if (pp->flow_mode == OR_FLOW_EXACT_SCHUR) {
    // S_ff = A_ff - A_fu A_uu^{-1} A_uf (Eq. (LU) of §5.1), dense
    int64_t nu = s->n_u, nf = s->n_f;
    vec duu(size_t(nu) * nu, 0.0), duf(size_t(nu) * nf, 0.0), dfu(size_t(nf) * nu, 0.0), dff(size_t(nf) * nf, 0.0);
    bsr_dense(Auu, duu, 0, 0, nu);
    bsr_dense(to_bsr(s, 1), duf, 0, 0, nf);
    bsr_dense(P->A_fu, dfu, 0, 0, nu);
    bsr_dense(P->A_ff, dff, 0, 0, nf);
    DenseLU lu; lu.factor(nu, duu);
    vec col(nu), xs(nu);
    for (int64_t j = 0; j < nf; ++j) {
      for (int64_t i = 0; i < nu; ++i) col[i] = duf[i * nf + j];
      lu.solve(col.data(), xs.data());
      for (int64_t i = 0; i < nf; ++i) {
        double t = 0.0;
        for (int64_t k = 0; k < nu; ++k) t += dfu[i * nu + k] * xs[k];
        dff[i * nf + j] -= t;
      }
    }
    P->lu_flow.factor(nf, std::move(dff));
  }
  if (pp->full_exact) {
    vec d; full_dense(s, d);
    P->lu_full.factor(s->n, std::move(d));
  }
  *out = P;
  return 0;
}

void or_prec_free(or_prec* p) { delete p; }

int or_ilu_apply(const or_prec* P, const double* w, double* dz) {
  int64_t nc = P->s->n_cells;
  vec y(2 * nc);
  for (int64_t i = 0; i < nc; ++i) {
    double a0 = w[2 * i], a1 = w[2 * i + 1];
    for (int64_t q = P->ilu.rp[i]; q < P->ilu.rp[i + 1]; ++q) {
      int64_t k = P->ilu.ci[q];
      if (k >= i) break;
      const double* L = &P->ilu.v[q * 4];
      a0 -= L[0] * y[2 * k] + L[1] * y[2 * k + 1];
      a1 -= L[2] * y[2 * k] + L[3] * y[2 * k + 1];
    }
    y[2 * i] = a0; y[2 * i + 1] = a1;
  }
  for (int64_t i = nc - 1; i >= 0; --i) {
    double a0 = y[2 * i], a1 = y[2 * i + 1];
    for (int64_t q = P->ilu.rp[i]; q < P->ilu.rp[i + 1]; ++q) {
      int64_t j = P->ilu.ci[q];
      if (j <= i) continue;
      const double* U = &P->ilu.v[q * 4];
      a0 -= U[0] * dz[2 * j] + U[1] * dz[2 * j + 1];
      a1 -= U[2] * dz[2 * j] + U[3] * dz[2 * j + 1];
    }
    const double* D = &P->dinv[4 * i];
    dz[2 * i] = D[0] * a0 + D[1] * a1;
    dz[2 * i + 1] = D[2] * a0 + D[3] * a1;
  }
  return 0;
}

// §5.3 option 1, block Gauss-Seidel on the interleaved S_ff^(FS): each sweep updates every cell in turn,
// z_i = inv(S_ii) (w_i - sum_{j != i} S_ij z_j) with the newest z_j.  The cells are taken in red-black order
// (colour (i + j + k) mod 2 of the cell's grid coordinates, colour 0 first): a face neighbour always has the
// other colour, so each colour's updates are independent of one another.
int or_gs_apply(const or_prec* P, const double* w, double* dz, int sweeps) {
  const or_system* s = P->s;
  int64_t nc = s->n_cells;
  const int64_t nx = s->nx, ny = s->ny;
  for (int64_t e = 0; e < 2 * nc; ++e) dz[e] = 0.0;
  for (int it = 0; it < sweeps; ++it)
    for (int colour = 0; colour < 2; ++colour)
      for (int64_t i = 0; i < nc; ++i) {
        const int64_t ci = i % nx, cj = (i / nx) % ny, ck = i / (nx * ny);
        if (((ci + cj + ck) & 1) != colour) continue;
        double a0 = w[2 * i], a1 = w[2 * i + 1];
        for (int64_t q = P->Sff.rp[i]; q < P->Sff.rp[i + 1]; ++q) {
          int64_t j = P->Sff.ci[q];
          if (j == i) continue;
          const double* S = &P->Sff.v[q * 4];
          a0 -= S[0] * dz[2 * j] + S[1] * dz[2 * j + 1];
          a1 -= S[2] * dz[2 * j] + S[3] * dz[2 * j + 1];
        }
        const double* D = &P->gs_dinv[4 * i];
        dz[2 * i] = D[0] * a0 + D[1] * a1;
        dz[2 * i + 1] = D[2] * a0 + D[3] * a1;
      }
  return 0;
}

// Algorithm 1: z = M^{-1} v
void or_prec_apply(or_prec* P, const double* v, double* z) {
  const or_system* s = P->s;
  int64_t nn = s->n_nodes, nc = s->n_cells, nu = s->n_u, nf = s->n_f;
  if (P->pp.full_exact) { P->lu_full.solve(v, z); return; }
  // step 1: z_u = M_uu^{-1} v_u
  vec zu(nu);
  if (P->pp.mech_mode == OR_MECH_AMG) {
    mech_apply(P->amg_u, smooth_of(P->pp), nn, v, zu.data());
  } else if (P->pp.mech_mode == OR_MECH_AMG_RBM) {
    vec vu(v, v + 3 * nn), xu;
    block_vcycle(P->amg_rbm, 0, vu, xu, smooth_of(P->pp));
    zu.assign(xu.begin(), xu.end());
  } else {
    P->lu_uu.solve(v, zu.data());
  }
  // step 2: y_f = v_f - A_fu z_u
  vec yf(nf);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nc; ++c)
    for (int a = 0; a < 2; ++a) {
      double acc = 0.0;
      for (int64_t q = P->A_fu.rp[c]; q < P->A_fu.rp[c + 1]; ++q)
        for (int e = 0; e < 3; ++e) acc += P->A_fu.v[q * 6 + a * 3 + e] * zu[3 * int64_t(P->A_fu.ci[q]) + e];
      yf[2 * c + a] = v[nu + 2 * c + a] - acc;
    }
  vec zf(nf);
  if (P->pp.flow_mode != OR_FLOW_CPR) {
    P->lu_flow.solve(yf.data(), zf.data());
  } else {
    // step 3: z_s = D_ss^{-1} y_s
    vec zs(nc), wp(nc), zp(nc);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nc; ++c) zs[c] = yf[2 * c] / P->dss[c];
    // step 4: w_p = y_p - A_ps z_s (complete A_ps)
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nc; ++c) {
      double acc = 0.0;
      for (int64_t q = P->A_ff.rp[c]; q < P->A_ff.rp[c + 1]; ++q) acc += P->A_ff.v[q * 4 + 2] * zs[P->A_ff.ci[q]];
      wp[c] = yf[2 * c + 1] - acc;
    }
    // step 5: z_p = M_pp^{-1} w_p
    if (P->pp.press_mode == OR_PRESS_AMG) {
      vec x;
      vcycle(P->amg_p, 0, 0, wp, x, smooth_of(P->pp));
      zp = x;
    } else {
      P->lu_pp.solve(wp.data(), zp.data());
    }
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nc; ++c) { zf[2 * c] = zs[c]; zf[2 * c + 1] = zp[c]; }
    // step 6: w_f = y_f - S_ff^(FS) z_f
    vec wf(nf);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nc; ++c)
      for (int a = 0; a < 2; ++a) {
        double acc = 0.0;
        for (int64_t q = P->Sff.rp[c]; q < P->Sff.rp[c + 1]; ++q)
          for (int e = 0; e < 2; ++e) acc += P->Sff.v[q * 4 + a * 2 + e] * zf[2 * int64_t(P->Sff.ci[q]) + e];
        wf[2 * c + a] = yf[2 * c + a] - acc;
      }
    // step 7: dz_f = M_L^{-1} w_f
    vec dz(nf);
    if (P->pp.local_mode == OR_LOCAL_ILU0) or_ilu_apply(P, wf.data(), dz.data());
    else if (P->pp.local_mode == OR_LOCAL_GS) or_gs_apply(P, wf.data(), dz.data(), P->pp.local_sweeps);
    else P->lu_local.solve(wf.data(), dz.data());
    // step 8: z_f += dz_f
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < nf; ++e) zf[e] += dz[e];
  }
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < nu; ++e) z[e] = zu[e];
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < nf; ++e) z[nu + e] = zf[e];
}

static const AMG* pick(const or_prec* p, int which) { return which == 0 ? &p->amg_u : &p->amg_p; }

int or_amg_nlevels(const or_prec* p, int which) { return int(pick(p, which)->L.size()); }
int64_t or_amg_level_n(const or_prec* p, int which, int level) { return pick(p, which)->L[level].A.n; }
int64_t or_amg_level_nnz(const or_prec* p, int which, int level) { return pick(p, which)->L[level].A.nnz(); }
int or_amg_level_matrix(const or_prec* p, int which, int level, int64_t* rp, int32_t* ci, double* v) {
  const CSR& A = pick(p, which)->L[level].A;
  std::memcpy(rp, A.rp.data(), A.rp.size() * sizeof(int64_t));
  std::memcpy(ci, A.ci.data(), A.ci.size() * sizeof(int32_t));
  std::memcpy(v, A.v.data(), A.v.size() * sizeof(double));
  return 0;
}
int64_t or_amg_aggregates(const or_prec* p, int which, int level, int32_t* agg) {
  const Level& L = pick(p, which)->L[level];
  if (!L.agg.empty()) std::memcpy(agg, L.agg.data(), L.agg.size() * sizeof(int32_t));
  return L.nagg;
}
int64_t or_amg_roots(const or_prec* p, int which, int level, uint8_t* root) {
  const Level& L = pick(p, which)->L[level];
  if (!L.root.empty()) std::memcpy(root, L.root.data(), L.root.size());
  return int64_t(L.root.size());
}
// aggregation of a caller-given level operator (CSR, nc values per entry, sorted columns): the
// strength graph, distance-2 MIS rounds under the priority key of `level`, phase 1 and phase 2
int64_t or_aggregate(int64_t n, int nc, const int64_t* rp, const int32_t* ci, const double* v, double theta,
                     int level, int32_t* agg, uint8_t* root) {
  Level lev;
  lev.A.n = lev.A.m = n; lev.A.nc = nc;
  lev.A.rp.assign(rp, rp + n + 1);
  lev.A.ci.assign(ci, ci + rp[n]);
  lev.A.v.assign(v, v + rp[n] * nc);
  aggregate(lev, theta, level);
  std::memcpy(agg, lev.agg.data(), size_t(n) * sizeof(int32_t));
  std::memcpy(root, lev.root.data(), size_t(n));
  return lev.nagg;
}
int or_rbm_nlevels(const or_prec* p) { return int(p->amg_rbm.L.size()); }
int or_rbm_level_shape(const or_prec* p, int level, int64_t* shape) {
  if (level < 0 || level >= int(p->amg_rbm.L.size())) return 1;
  const BLevel& L = p->amg_rbm.L[level];
  shape[0] = L.A.nbr; shape[1] = L.b; shape[2] = int64_t(L.A.ci.size()); shape[3] = L.nagg;
  shape[4] = int64_t(L.P.ci.size()); shape[5] = L.coarsest ? 1 : 0;
  return 0;
}
int or_rbm_level_matrix(const or_prec* p, int level, int64_t* rp, int32_t* ci, double* v) {
  if (level < 0 || level >= int(p->amg_rbm.L.size())) return 1;
  const BSR& A = p->amg_rbm.L[level].A;
  std::copy(A.rp.begin(), A.rp.end(), rp);
  std::copy(A.ci.begin(), A.ci.end(), ci);
  std::copy(A.v.begin(), A.v.end(), v);
  return 0;
}
int or_rbm_level_data(const or_prec* p, int level, int32_t* agg, double* B, double* Pt, double* lam) {
  if (level < 0 || level >= int(p->amg_rbm.L.size())) return 1;
  const BLevel& L = p->amg_rbm.L[level];
  if (agg) for (int64_t i = 0; i < L.A.nbr; ++i) agg[i] = L.coarsest ? -1 : L.agg[i];
  if (B) std::copy(L.B.begin(), L.B.end(), B);
  if (Pt) { if (L.coarsest) std::fill(Pt, Pt + L.A.nbr * L.b * kModes, 0.0); else std::copy(L.Pt.begin(), L.Pt.end(), Pt); }
  if (lam) *lam = L.lam;
  return 0;
}
int or_rbm_prolongator(const or_prec* p, int level, int64_t* rp, int32_t* ci, double* v) {
  if (level < 0 || level >= int(p->amg_rbm.L.size()) || p->amg_rbm.L[level].coarsest) return 1;
  const BSR& P = p->amg_rbm.L[level].P;
  std::copy(P.rp.begin(), P.rp.end(), rp);
  std::copy(P.ci.begin(), P.ci.end(), ci);
  std::copy(P.v.begin(), P.v.end(), v);
  return 0;
}
int or_rbm_vcycle(const or_prec* p, const double* b, double* x) {
  if (p->amg_rbm.L.empty()) return 1;
  vec bb(b, b + p->amg_rbm.L[0].A.nbr * 3), xx;
  block_vcycle(p->amg_rbm, 0, bb, xx, smooth_of(p->pp));
  std::copy(xx.begin(), xx.end(), x);
  return 0;
}
void or_rigid_body_modes(int nx, int ny, int nz, double* B) {
  vec v = rigid_body_modes(nx, ny, nz);
  std::copy(v.begin(), v.end(), B);
}

int64_t or_amg_p_nnz(const or_prec* p, int which, int level) { return pick(p, which)->L[level].P.nnz(); }
int or_amg_prolongator(const or_prec* p, int which, int level, int64_t* rp, int32_t* ci, double* v) {
  const CSR& A = pick(p, which)->L[level].P;
  std::memcpy(rp, A.rp.data(), A.rp.size() * sizeof(int64_t));
  std::memcpy(ci, A.ci.data(), A.ci.size() * sizeof(int32_t));
  std::memcpy(v, A.v.data(), A.v.size() * sizeof(double));
  return 0;
}
int or_amg_vcycle(const or_prec* p, int which, int comp, const double* b, double* x) {
  const AMG* H = pick(p, which);
  vec bb(b, b + H->L[0].A.n), xx;
  vcycle(*H, 0, comp, bb, xx, smooth_of(p->pp));
  std::memcpy(x, xx.data(), xx.size() * sizeof(double));
  return 0;
}
// one smoother application on a scalar CSR matrix (test access to the level-0 smoothers of the
// V-cycle): kind 1 = Chebyshev of the given degree over [lambda_hat/ratio, lambda_hat] of D^{-1}A,
// kind 0 = that many l1-Jacobi sweeps; x holds the start iterate unless zero != 0
int or_smoother_apply(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* b, double* x,
                      int kind, int count, double ratio, int zero) {
  Level lev;
  lev.A.n = lev.A.m = n;
  lev.A.nc = 1;
  lev.A.rp.assign(rp, rp + n + 1);
  lev.A.ci.assign(ci, ci + rp[n]);
  lev.A.v.assign(v, v + rp[n]);
  lev.dl1 = l1_diag(lev.A);
  lev.lam = gershgorin(lev.A);
  lev.dg.assign(n, 0.0);
  for (int64_t i = 0; i < n; ++i) {
    int64_t q = lev.A.find(i, i);
    if (q < 0) return 1;
    lev.dg[i] = lev.A.v[q];
  }
  vec bb(b, b + n), xx(n, 0.0);
  if (!zero) xx.assign(x, x + n);
  if (kind == 1) chebyshev(lev, 1, 0, bb, xx, count, ratio, zero != 0);
  else l1_jacobi(lev, 1, 0, bb, xx, count);
  std::memcpy(x, xx.data(), n * sizeof(double));
  return 0;
}

int64_t or_spp_nnz(const or_prec* p) { return p->spp.nnz(); }
int or_spp(const or_prec* p, int64_t* rp, int32_t* ci, double* v) {
  std::memcpy(rp, p->spp.rp.data(), p->spp.rp.size() * sizeof(int64_t));
  std::memcpy(ci, p->spp.ci.data(), p->spp.ci.size() * sizeof(int32_t));
  std::memcpy(v, p->spp.v.data(), p->spp.v.size() * sizeof(double));
  return 0;
}
int or_fs_diag(const or_prec* p, double* dfs) {
  std::memcpy(dfs, p->dfs.data(), p->dfs.size() * sizeof(double));
  return 0;
}

int or_ilu_dinv(const or_prec* p, double* dinv) {
  std::memcpy(dinv, p->dinv.data(), p->dinv.size() * sizeof(double));
  return 0;
}

int or_fgmres(const or_system* s, or_prec* p, const double* b, double* x, double tol, int restart, int max_iters,
              or_stats* st) {
  Op A = [s](const double* in, double* out) { or_spmv(s, in, out); };
  Op M = [p](const double* in, double* out) { or_prec_apply(p, in, out); };
  fgmres(s->n, A, M, b, x, tol, restart, max_iters, st);
  return st->converged ? 0 : 4;
}

// Sequential fixed-stress strategy of the §5.4 remark: the preconditioner inside a Richardson iteration,
// x_{k+1} = x_k + M^{-1} (b - A x_k), x_0 = 0.  Step 1 of Algorithm 1 corrects the displacements, steps 2-8
// then correct the flow unknowns, so each iteration is one mechanics-then-flow pass.
int or_richardson(const or_system* s, or_prec* p, const double* b, double* x, double tol, int max_iters,
                  or_stats* st) {
  std::memset(st, 0, sizeof(*st));
  const int64_t n = s->n;
  const double bn = std::sqrt(dot(b, b, n));
  vec r(n), z(n), Ax(n);
  for (int64_t e = 0; e < n; ++e) x[e] = 0.0;
  if (bn == 0.0) { st->converged = 1; return 0; }
  for (;;) {
    or_spmv(s, x, Ax.data());
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < n; ++e) r[e] = b[e] - Ax[e];
    const double rr = std::sqrt(dot(r.data(), r.data(), n)) / bn;
    st->true_relres = rr;
    st->est_relres = rr;
    if (std::isnan(rr)) return 0;
    if (rr <= tol) { st->converged = 1; return 0; }
    if (st->iters >= max_iters) return 0;
    or_prec_apply(p, r.data(), z.data());
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < n; ++e) x[e] = x[e] + z[e];
    st->iters++;
  }
}

int or_fgmres_diag(int64_t n, const double* diag, const double* b, double* x, double tol, int restart,
                   int max_iters, or_stats* st) {
  Op A = [n, diag](const double* in, double* out) { for (int64_t i = 0; i < n; ++i) out[i] = diag[i] * in[i]; };
  Op M = [n](const double* in, double* out) { for (int64_t i = 0; i < n; ++i) out[i] = in[i]; };
  fgmres(n, A, M, b, x, tol, restart, max_iters, st);
  return st->converged ? 0 : 4;
}

int or_dense_solve(const or_system* s, const double* b, double* x) {
  if (s->n > 6000) return 1;
  vec d; full_dense(s, d);
  DenseLU lu; lu.factor(s->n, std::move(d));
  if (!lu.ok) return 3;
  lu.solve(b, x);
  return 0;
}

int or_lu_solve(int64_t n, double* a, const double* b, double* x) {
  DenseLU lu; lu.factor(n, vec(a, a + size_t(n) * n));
  if (!lu.ok) return 3;
  lu.solve(b, x);
  return 0;
}

// Terzaghi column: homogeneous medium, identical phases, Corey exponent 1,
// no gravity, incompressible fluids, drained top, rollers, fixed base.
int or_terzaghi(const or_terzaghi_params* tp, double* tout, double* pout, double* p0out, double* cvout,
                double* newton_ratio) {
  or_gen_params gp;
  or_default_params(&gp, 0);
  gp.nx = 1; gp.ny = 1; gp.nz = tp->nz; gp.h = tp->h;
  gp.field_kind = OR_FIELDS_HOMOGENEOUS;
  gp.flags = OR_ACCUM | OR_FLUX | OR_FLUX_SAT | OR_COUPLING;
  gp.biot = tp->biot;
  gp.c_w = gp.c_nw = gp.c_r = 0.0;
  gp.mu_w = gp.mu_nw = tp->mu;
  gp.rho_w0 = gp.rho_nw0 = tp->rho0;
  gp.s_wr = gp.s_nwr = 0.0;
  gp.corey = 1.0;
  gp.p_ref = 0.0; gp.dp_amp = 0.0;
  gp.E0 = tp->E; gp.nu0 = tp->nu; gp.kappa0 = tp->kappa; gp.phi0 = tp->phi0; gp.sw0 = 0.5;
  Grid g{1, 1, tp->nz, tp->h};
  Fields F = make_fields(gp);
  ExtraBC bc;
  bc.active = true;
  bc.dir_u.assign(3 * g.nn(), 0);
  for (int k = 0; k <= g.nz; ++k)
    for (int j = 0; j <= 1; ++j)
      for (int i = 0; i <= 1; ++i) {
        int64_t I = g.node(i, j, k);
        bc.dir_u[3 * I + 0] = 1; bc.dir_u[3 * I + 1] = 1;
        if (k == 0) bc.dir_u[3 * I + 2] = 1;
      }
  bc.sigma_top = tp->sigma0;
  bc.top_drained = true;
  bc.p_top = 0.0; bc.s_top = 0.5;
  int64_t nu = 3 * g.nn(), nc = g.ncell(), n = nu + 2 * nc;
  State prev;
  prev.u.assign(nu, 0.0); prev.s.assign(nc, 0.5); prev.p.assign(nc, 0.0);
  double worst = 0.0, first_rn = -1.0;
  auto step = [&](double dt, State& x) {
    or_gen_params q = gp;
    q.dt = dt;
    x = prev;
    for (int it = 0; it < 4; ++it) {
      vec r;
      residual(q, g, F, prev, x, bc, r);
      Jac J;
      assemble(q, g, F, x, bc, J);
      finalize(q, g, J, false);
      for (int64_t i = 0; i < nu; ++i) if (bc.dir_u[i]) r[i] = 0.0;
      double rn = 0.0;
      for (double v : r) rn += v * v;
      rn = std::sqrt(rn);
      or_system tmp;
      std::memset(&tmp, 0, sizeof(tmp));
      tmp.n_nodes = g.nn(); tmp.n_cells = nc; tmp.n_u = nu; tmp.n_f = 2 * nc; tmp.n = n;
      tmp.uu_rp = J.uu.rp.data(); tmp.uu_ci = J.uu.ci.data(); tmp.uu_v = J.uu.v.data();
      tmp.uf_rp = J.uf.rp.data(); tmp.uf_ci = J.uf.ci.data(); tmp.uf_v = J.uf.v.data();
      tmp.fu_rp = J.fu.rp.data(); tmp.fu_ci = J.fu.ci.data(); tmp.fu_v = J.fu.v.data();
      tmp.ff_rp = J.ff.rp.data(); tmp.ff_ci = J.ff.ci.data(); tmp.ff_v = J.ff.v.data();
      vec d; full_dense(&tmp, d);
      DenseLU lu; lu.factor(n, std::move(d));
      vec mr(n), dx(n);
      for (int64_t i = 0; i < n; ++i) mr[i] = -r[i];
      lu.solve(mr.data(), dx.data());
      for (int64_t i = 0; i < nu; ++i) x.u[i] += dx[i];
      for (int64_t c = 0; c < nc; ++c) { x.s[c] += dx[nu + 2 * c]; x.p[c] += dx[nu + 2 * c + 1]; }
      vec r2;
      residual(q, g, F, prev, x, bc, r2);
      for (int64_t i = 0; i < nu; ++i) if (bc.dir_u[i]) r2[i] = 0.0;
      double rn2 = 0.0;
      for (double v : r2) rn2 += v * v;
      rn2 = std::sqrt(rn2);
      // one-step Newton contraction, on steps whose starting residual is well above round-off
      if (it == 0 && rn > 0.0) {
        if (first_rn < 0.0) first_rn = rn;
        if (rn >= 1e-3 * first_rn) worst = std::max(worst, rn2 / rn);
      }
      if (rn2 <= 1e-13 * rn) break;
    }
  };
  // undrained loading: no drainage during the instantaneous step
  State x;
  {
    or_gen_params saved = gp;
    gp.flags = OR_ACCUM | OR_COUPLING;
    step(1.0, x);
    gp = saved;
    first_rn = -1.0;
  }
  double p0 = 0.0;
  for (int64_t c = 0; c < nc; ++c) p0 += x.p[c];
  *p0out = p0 / double(nc);
  prev = x;
  Mat m = material(gp, tp->E, tp->nu, tp->phi0, 0.5, 0.0, 0.0);
  double Kv = m.Kdr + 4.0 * m.G / 3.0;
  double S = m.dphidp;
  *cvout = (tp->kappa / tp->mu) / (S + tp->biot * tp->biot / Kv);
  for (int n_ = 0; n_ < tp->nsteps; ++n_) {
    step(tp->dt, x);
    prev = x;
    tout[n_] = (n_ + 1) * tp->dt;
    for (int64_t c = 0; c < nc; ++c) pout[int64_t(n_) * nc + c] = x.p[c];
  }
  *newton_ratio = worst;
  return 0;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Newton's method for one time step (§4 and its remarks on inexact Newton).  The previous time level is the
// base state (u = 0, s = S_w, p of the fields) and is also the first iterate.  Each step evaluates the
// residual at base + x (Dirichlet rows set to zero), assembles the Jacobian there (or_generate_at: rows
// divided by that Jacobian's alpha_u, alpha_f, pressure unknowns in MPa), and solves J y = -R r by FGMRES
// under the two-stage preconditioner to the relative tolerance eta_k, keeping the mechanics hierarchy of the
// first step (§5.4); dx = C y.  Convergence is measured in the base state's row scaling R_0.
// ---------------------------------------------------------------------------
extern "C" {

void or_newton_params_default(or_newton_params* np) {
  std::memset(np, 0, sizeof(*np));
  np->rtol = 1e-5;  // the Newton tolerance of the paper's runs (Table 1)
  np->max_newton = 12;
  np->forcing = OR_FORCING_EW;
  np->eta_fixed = 1e-6;
  np->ew_gamma = 0.9;
  np->ew_omega = 2.0;
  np->ew_eta0 = 0.1;
  np->ew_eta_max = 0.1;
  np->max_backtracks = 4;
  np->restart = 100;
  np->max_linear = 1000;
}

// Krylov tolerance of Newton step k (Eisenstat and Walker's choice 2 with the safeguard the paper states,
// capped at eta_max and floored so that the step does not solve beyond the nonlinear tolerance)
double or_ew_eta(const or_newton_params* np, int k, double rk, double rkm1, double eta_prev, double r0) {
  if (np->forcing == OR_FORCING_FIXED) return np->eta_fixed;
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

int or_newton(const or_gen_params* gp, const or_prec_params* pp, const or_newton_params* np, double* x_out,
              or_newton_stats* st) {
  std::memset(st, 0, sizeof(*st));
  or_system* s0 = nullptr;
  if (generate_at(gp, nullptr, &s0)) return 1;
  const int64_t n = s0->n, nu = s0->n_u;
  const double au0 = s0->alpha_u, af0 = s0->alpha_f;
  auto resid = [&](const vec& x, vec& r) {
    r.assign(n, 0.0);
    or_residual(gp, x.data(), r.data());
    for (int64_t i = 0; i < nu; ++i)
      if (s0->dirichlet[i]) r[i] = 0.0;
  };
  auto snorm = [&](const vec& r, double au, double af) {
    double a = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      const double v = r[i] / (i < nu ? au : af);
      a += v * v;
    }
    return std::sqrt(a);
  };
  vec x(n, 0.0), r, rt, y(n), rhs(n), xt(n);
  resid(x, r);
  double rk = snorm(r, au0, af0);
  const double r0 = rk;
  st->rnorm[0] = rk;
  double rkm1 = rk, eta_prev = np->ew_eta0;
  int rc = 0;
  for (int k = 0; k < np->max_newton && k < 32; ++k) {
    if (rk <= np->rtol * r0) { st->converged = 1; break; }
    or_system* sk = nullptr;
    if (generate_at(gp, x.data(), &sk)) { rc = 1; break; }
    or_prec* P = nullptr;
    if (or_prec_setup_reuse(sk, s0, pp, &P)) { or_system_free(sk); rc = 2; break; }
    const double eta = or_ew_eta(np, k, rk, rkm1, eta_prev, r0);
    for (int64_t i = 0; i < n; ++i) rhs[i] = -r[i] / (i < nu ? sk->alpha_u : sk->alpha_f);
    or_stats ls;
    std::fill(y.begin(), y.end(), 0.0);
    or_fgmres(sk, P, rhs.data(), y.data(), eta, np->restart, np->max_linear, &ls);
    or_prec_free(P);
    or_system_free(sk);
    st->eta[k] = eta;
    st->lin_iters[k] = ls.iters;
    st->linear_iters += ls.iters;
    // dx = C y (pressure unknowns in MPa); backtracking on the R_0-scaled residual norm
    double lam = 1.0, rt_norm = 0.0;
    for (int bt = 0;; ++bt) {
      for (int64_t i = 0; i < n; ++i) {
        const bool pcol = i >= nu && ((i - nu) & 1);
        xt[i] = x[i] + lam * (pcol ? 1e6 * y[i] : y[i]);
      }
      resid(xt, rt);
      rt_norm = snorm(rt, au0, af0);
      if (rt_norm <= (1.0 - 1e-4 * lam) * rk || bt >= np->max_backtracks) break;
      lam *= 0.5;
      ++st->backtracks;
    }
    x = xt;
    r = rt;
    rkm1 = rk;
    rk = rt_norm;
    eta_prev = eta;
    st->newton_iters = k + 1;
    st->rnorm[k + 1] = rk;
  }
  if (!rc && rk <= np->rtol * r0) st->converged = 1;
  std::copy(x.begin(), x.end(), x_out);
  or_system_free(s0);
  return rc ? rc : (st->converged ? 0 : 4);
}

}  // extern "C"
