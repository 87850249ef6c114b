// Micro-element MD engine: host planner, CUDA-graph step loop and the C ABI
// entry points declared in include/mdgp.h (paper App. A and Sec. 2.1).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "mdgp.h"
#include "md_kernels.cuh"
#include "md_resident.cuh"
#include "md_ctx.h"

using namespace mdgp;

namespace {

long lround_half_up(double x) { return (long)std::floor(x + 0.5); }

int set_err(mdgp_ctx* c, cudaError_t e) {
  if (e == cudaSuccess) return MDGP_OK;
  if (c) std::snprintf(c->err, sizeof(c->err), "%s", cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? MDGP_E_NOMEM : MDGP_E_CUDA;
}

#define CK(expr)                                    \
  do {                                              \
    cudaError_t e_ = (expr);                        \
    if (e_ != cudaSuccess) return set_err(ctx, e_); \
  } while (0)

// Grow-only device buffer.
int ensure(mdgp_ctx* ctx, DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes) return MDGP_OK;
  if (b.ptr) cudaFree(b.ptr);
  b.ptr = nullptr;
  b.bytes = 0;
  size_t want = bytes < 256 ? 256 : bytes;
  CK(cudaMalloc(&b.ptr, want));
  b.bytes = want;
  return MDGP_OK;
}

// Element geometry from the paper's App. A with the stated readings: FCC
// fluid lattice filling the slab, FCC (100) wall planes, cells of side at
// least the list radius r_c + skin.
int describe(const mdgp_md_params& p, const mdgp_element& el, ElemDev& E, std::string* why) {
  if (!(el.h > 2.0 * p.fluid_margin)) { *why = "h must exceed twice the fluid margin"; return MDGP_E_ARG; }
  if (!(el.wall_amp >= 0.0 && el.wall_amp < 1.0)) { *why = "wall_amp must lie in [0, 1)"; return MDGP_E_ARG; }
  if (el.wall_amp > 0.0 && !(el.h * (1.0 - el.wall_amp) > 2.0 * p.fluid_margin)) {
    *why = "the narrowest gap h (1 - wall_amp) must exceed twice the fluid margin";
    return MDGP_E_ARG;
  }
  // the box and the fluid lattice are built for the widest gap H; N_fluid
  // and the pressure's volume take the mean gap h
  const double H = el.h * (1.0 + el.wall_amp);
  if (!(el.density >= 0.0) || !(el.T > 0.0) || el.steps_eq < 0 || el.steps_sample < 0) {
    *why = "density >= 0, T > 0 and non-negative step counts required";
    return MDGP_E_ARG;
  }
  std::memset(&E, 0, sizeof(E));
  E.Lx = el.Lx; E.Lz = el.Lz; E.h = H;
  E.hvol = el.h;
  E.amp = el.wall_amp;
  E.T = el.T;
  // Eq. momentumEq: F = F_ext - (m / rho) dp/dx with rho = m n
  E.g = el.density > 0.0 ? el.g_ext - el.dpdx / el.density : el.g_ext;
  E.vsd = std::sqrt(el.T / p.mass);
  E.beta_sd = std::sqrt(2.0 * p.gamma_wall * el.T * p.dt);
  E.seed = el.seed;
  E.id = el.id;
  E.steps_eq = el.steps_eq;
  E.steps_sample = el.steps_sample;
  E.steps_total = el.steps_eq + el.steps_sample;
  int nb = p.n_blocks < kMaxBlocks ? p.n_blocks : kMaxBlocks;
  if (el.steps_sample < nb) nb = (int)el.steps_sample;
  E.nb = nb;
  const long nf = lround_half_up(el.density * el.Lx * el.h * el.Lz);
  E.nf = (int)nf;
  const double af = std::cbrt(4.0 / el.density);
  const double ly = H - 2.0 * p.fluid_margin;
  long cx = (long)std::ceil(el.Lx / af - 1e-9), cy = (long)std::ceil(ly / af - 1e-9),
       cz = (long)std::ceil(el.Lz / af - 1e-9);
  if (cx < 1) cx = 1;
  if (cy < 1) cy = 1;
  if (cz < 1) cz = 1;
  for (int turn = 0; 4L * cx * cy * cz < nf; ++turn) {
    if (turn % 3 == 0) ++cy; else if (turn % 3 == 1) ++cx; else ++cz;
  }
  E.fc[0] = (int)cx; E.fc[1] = (int)cy; E.fc[2] = (int)cz;
  E.fb[0] = el.Lx / cx; E.fb[1] = ly / cy; E.fb[2] = el.Lz / cz;
  E.fy0 = p.fluid_margin;
  const double a0 = std::cbrt(4.0 / p.wall_density);
  long wnx = lround_half_up(el.Lx / a0), wnz = lround_half_up(el.Lz / a0);
  if (wnx < 1) wnx = 1;
  if (wnz < 1) wnz = 1;
  E.wnx = (int)wnx; E.wnz = (int)wnz;
  E.wax = el.Lx / wnx; E.waz = el.Lz / wnz; E.wdy = 0.5 * a0;
  E.nw = 2 * p.wall_planes * 2 * (int)wnx * (int)wnz;
  const double th = 0.5 * a0 * (p.wall_planes - 1);
  const double ylo = -th - 1.0, yhi = H + th + 1.0;
  E.ylo = ylo;
  const double rl = p.rc + p.skin;
  E.nc[0] = (int)std::floor(el.Lx / rl);
  E.nc[2] = (int)std::floor(el.Lz / rl);
  E.nc[1] = (int)std::floor((yhi - ylo) / rl);
  if (!(E.nc[0] >= 3) || !(E.nc[2] >= 3)) { *why = "Lx and Lz must be >= 3 (r_c + skin)"; return MDGP_E_ARG; }
  if (E.nc[1] < 1) E.nc[1] = 1;
  E.cs[0] = el.Lx / E.nc[0]; E.cs[1] = (yhi - ylo) / E.nc[1]; E.cs[2] = el.Lz / E.nc[2];
  for (int d = 0; d < 3; ++d) {
    E.inv_cs[d] = 1.0 / E.cs[d];
    E.csf[d] = (float)E.cs[d];
    E.cs_lo[d] = (float)(E.cs[d] - (double)E.csf[d]);
    E.inv_csf[d] = (float)E.inv_cs[d];
  }
  E.g_kick = (float)(0.5 * p.dt / p.mass * E.g);
  E.Tf = (float)E.T;
  E.beta_sdf = (float)E.beta_sd;
  return MDGP_OK;
}

// Initial positions of an element whose walls follow the channel profile
// (E.amp > 0), in k_init_atoms's atom order, 3 doubles per atom:
//  - the local gap h(x) = hvol (1 - amp cos(2 pi x / Lx)) and the lower
//    wall's inner plane yb(x) = (H - h(x)) / 2, H the widest gap;
//  - fluid: the FCC lattice of the widest gap, its sites in lattice order
//    kept where they lie at least the fluid margin inside the local walls,
//    the lattice grown (y, x, z in turn) until enough are kept, the
//    vacancies spread evenly over the kept sites;
//  - walls: the planar element's (100) planes with each site moved to
//    yb(x) - k dy (lower wall) or yb(x) + h(x) + k dy (upper wall).
void profiled_positions(const mdgp_md_params& p, const ElemDev& E, double* out) {
  const double m = p.fluid_margin, H = E.h;
  auto profile = [&](double x, double& hx, double& yb) {
    hx = E.hvol * (1.0 - E.amp * std::cos(2.0 * M_PI * x / E.Lx));
    yb = 0.5 * (H - hx);
  };
  long cx = E.fc[0], cy = E.fc[1], cz = E.fc[2];
  const double ly = H - 2.0 * m;
  const long long nf = E.nf;
  std::vector<double> pos;
  for (int turn = 0;; ++turn) {
    const double bx = E.Lx / cx, by = ly / cy, bz = E.Lz / cz;
    const long long sites = 4LL * cx * cy * cz;
    pos.clear();
    for (long long s = 0; s < sites; ++s) {
      const int b = (int)(s & 3);
      const long long c = s >> 2;
      const long long iz = c % cz, iy = (c / cz) % cy, ix = c / (cz * cy);
      const double ox = (b == 1 || b == 2) ? 0.5 : 0.0;
      const double oy = (b == 1 || b == 3) ? 0.5 : 0.0;
      const double oz = (b == 2 || b == 3) ? 0.5 : 0.0;
      const double px = ((double)ix + ox + 0.25) * bx;
      const double py = m + ((double)iy + oy + 0.25) * by;
      const double pz = ((double)iz + oz + 0.25) * bz;
      double hx, yb;
      profile(px, hx, yb);
      if (py >= yb + m && py <= yb + hx - m) {
        pos.push_back(px); pos.push_back(py); pos.push_back(pz);
      }
    }
    if ((long long)pos.size() / 3 >= nf) break;
    if (turn % 3 == 0) ++cy; else if (turn % 3 == 1) ++cx; else ++cz;
  }
  const long long kept = (long long)pos.size() / 3;
  for (long long l = 0; l < nf; ++l) {
    const long long k = (long long)(((__int128)l * kept) / nf);
    for (int d = 0; d < 3; ++d) out[3 * l + d] = pos[(size_t)(3 * k + d)];
  }
  const long long per_plane = 2LL * E.wnx * E.wnz, per_wall = per_plane * p.wall_planes;
  for (long long w = 0; w < E.nw; ++w) {
    const int wall = (int)(w / per_wall);
    const long long r = w % per_wall;
    const int k = (int)(r / per_plane);
    const long long r2 = r % per_plane;
    const long long i = r2 / (2LL * E.wnz), j = (r2 >> 1) % E.wnz;
    const int tt = (int)(r2 & 1);
    double ox, oz;
    if ((k & 1) == 0) { ox = tt ? 0.5 : 0.0; oz = tt ? 0.5 : 0.0; }
    else { ox = tt ? 0.0 : 0.5; oz = tt ? 0.5 : 0.0; }
    const double px = ((double)i + ox) * E.wax, pz = ((double)j + oz) * E.waz;
    double hx, yb;
    profile(px, hx, yb);
    double* o = out + 3 * (nf + w);
    o[0] = px;
    o[1] = wall == 0 ? yb - (double)k * E.wdy : yb + hx + (double)k * E.wdy;
    o[2] = pz;
  }
}

PhysDev make_phys(const mdgp_md_params& p, int list_cap) {
  PhysDev P;
  std::memset(&P, 0, sizeof(P));
  P.dt = p.dt;
  P.mass = p.mass;
  P.inv_m = 1.0 / p.mass;
  P.hdt_m = p.dt / (2.0 * p.mass);
  P.k_tether = p.k_tether;
  const double c = p.gamma_wall * p.dt / (2.0 * p.mass);
  P.gjf_a = (1.0 - c) / (1.0 + c);
  P.gjf_b = 1.0 / (1.0 + c);
  P.rc2 = p.rc * p.rc;
  P.rl2 = (p.rc + p.skin) * (p.rc + p.skin);
  const double eps[3] = {1.0, p.eps_wf, p.eps_ww};
  const double sig[3] = {1.0, p.sig_wf, p.sig_ww};
  P.uniform = 1;
  for (int t = 0; t < 3; ++t) {
    P.eps[t] = eps[t];
    P.sig2[t] = sig[t] * sig[t];
    const double sr6 = std::pow(sig[t] / p.rc, 6.0);
    P.eshift[t] = 4.0 * eps[t] * (sr6 * sr6 - sr6);
    P.active[t] = 1;
    P.epsf[t] = (float)eps[t];
    P.sig2f[t] = (float)(sig[t] * sig[t]);
    if (eps[t] != 1.0 || sig[t] != 1.0) P.uniform = 0;
  }
  if (p.mode == 1) { P.active[2] = 0; P.uniform = 0; }
  P.mode = p.mode;
  P.wall_planes = p.wall_planes;
  P.tau_T = p.tau_T;
  P.list_cap = list_cap;
  P.wait_ns = 1000000ull * (unsigned long long)(p.wait_timeout_ms > 0 ? p.wait_timeout_ms : 2000);
  P.inject_skip = p.inject_barrier_skip != 0 ? 1 : 0;
  P.rc2f = (float)(p.rc * p.rc);
  P.rl2f = (float)P.rl2;
  P.half_skin2f = (float)(0.25 * p.skin * p.skin);
  P.dtf = (float)p.dt;
  P.hdt_mf = (float)P.hdt_m;
  P.massf = (float)p.mass;
  P.inv_mf = (float)P.inv_m;
  P.k_tetherf = (float)p.k_tether;
  P.gjf_af = (float)P.gjf_a;
  P.gjf_bf = (float)P.gjf_b;
  P.dt_tauf = p.tau_T > 0.0 ? (float)(p.dt / p.tau_T) : 0.0f;
  return P;
}

inline unsigned grid_for(long long n, int threads) {
  long long g = (n + threads - 1) / threads;
  return (unsigned)(g < 1 ? 1 : g);
}

// Steps between list rebuilds: no atom may move more than skin/2 in that
// time; the speed bound is 8 thermal standard deviations per component.
int rebuild_interval(const mdgp_md_params& p, double Tmax) {
  if (p.rebuild_every > 0) return p.rebuild_every;
  const double vmax = 8.0 * std::sqrt(Tmax / p.mass);
  int r = (int)std::floor(0.5 * p.skin / (vmax * p.dt));
  return r < 1 ? 1 : r;
}

// ---------------------------------------------------------------------------
// Start states from snapshots (paper Sec. 2.4, Algorithm 1).
// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11) on the host, the generator the device
// uses: ten rounds of the two-multiply S-box, key advanced by the Weyl
// increments between rounds.
void philox_host(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0], p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0, n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
    c[0] = n0; c[1] = (uint32_t)p1; c[2] = n2; c[3] = (uint32_t)p0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

void philox_draw(uint32_t a, uint32_t b, uint32_t elem, uint32_t stream, uint64_t seed, uint32_t out[4]) {
  out[0] = a; out[1] = b; out[2] = elem; out[3] = stream;
  philox_host(out, (uint32_t)seed, (uint32_t)(seed >> 32));
}

double u01(uint32_t r) { return ((double)r + 0.5) * (1.0 / 4294967296.0); }

// Uniform grid over the element's atoms (periodic in x and z) for the
// insertion of fluid atoms: the shifted LJ energy (truncated at r_c, pair
// parameters by species) and force a fluid atom at a site has with the
// atoms present.
struct SiteGrid {
  double Lx, Lz, ylo, cs;
  int nx, ny, nz;
  std::vector<std::vector<int>> cell;
  std::vector<double> pos;   // 3 per site
  std::vector<int> wall;     // species per site
  SiteGrid(double Lx_, double Lz_, double ylo_, double yhi, double side) : Lx(Lx_), Lz(Lz_), ylo(ylo_) {
    nx = std::max(1, (int)std::floor(Lx / side));
    nz = std::max(1, (int)std::floor(Lz / side));
    ny = std::max(1, (int)std::floor((yhi - ylo) / side));
    cs = side;
    cell.resize((size_t)nx * ny * nz);
  }
  int index(double x, double y, double z, int& ix, int& iy, int& iz) const {
    ix = std::min(nx - 1, std::max(0, (int)(x / Lx * nx)));
    iz = std::min(nz - 1, std::max(0, (int)(z / Lz * nz)));
    iy = std::min(ny - 1, std::max(0, (int)((y - ylo) / cs)));
    return (ix * ny + iy) * nz + iz;
  }
  void add(double x, double y, double z, int is_wall) {
    int ix, iy, iz;
    cell[(size_t)index(x, y, z, ix, iy, iz)].push_back((int)(pos.size() / 3));
    pos.push_back(x); pos.push_back(y); pos.push_back(z);
    wall.push_back(is_wall);
  }
  void move(int i, double x, double y, double z) {
    int ix, iy, iz;
    std::vector<int>& from = cell[(size_t)index(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], ix, iy, iz)];
    from.erase(std::find(from.begin(), from.end(), i));
    cell[(size_t)index(x, y, z, ix, iy, iz)].push_back(i);
    pos[3 * i] = x; pos[3 * i + 1] = y; pos[3 * i + 2] = z;
  }
  // the cells of the sites within distance r of (x, y, z), each once
  // (periodic in x and z; rows outside the grid in y are skipped)
  template <class Fn>
  void near_cells(double x, double y, double z, double r, Fn&& fn) const {
    int ix, iy, iz;
    index(x, y, z, ix, iy, iz);
    const int rx = (int)std::ceil(r / (Lx / nx)), rz = (int)std::ceil(r / (Lz / nz)), ry = (int)std::ceil(r / cs);
    const bool allx = 2 * rx + 1 >= nx, allz = 2 * rz + 1 >= nz;
    for (int a = allx ? 0 : ix - rx; a <= (allx ? nx - 1 : ix + rx); ++a)
      for (int jy = std::max(0, iy - ry); jy <= std::min(ny - 1, iy + ry); ++jy)
        for (int c = allz ? 0 : iz - rz; c <= (allz ? nz - 1 : iz + rz); ++c) {
          const int jx = (a % nx + nx) % nx, jz = (c % nz + nz) % nz;
          fn(cell[(size_t)(jx * ny + jy) * nz + jz]);
        }
  }
  // shifted LJ pair energy of a fluid atom at (x, y, z) with site s, and
  // the force on the fluid atom added to f (0 beyond rc)
  double pair(double x, double y, double z, int s, const mdgp_md_params& p, double f[3]) const {
    double ax = x - pos[3 * s], ay = y - pos[3 * s + 1], az = z - pos[3 * s + 2];
    ax -= Lx * std::floor(ax / Lx + 0.5);
    az -= Lz * std::floor(az / Lz + 0.5);
    const double r2 = ax * ax + ay * ay + az * az, rc2 = p.rc * p.rc;
    if (r2 >= rc2) return 0.0;
    const double eps = wall[s] ? p.eps_wf : 1.0, sig = wall[s] ? p.sig_wf : 1.0;
    const double s2 = sig * sig / r2, s6 = s2 * s2 * s2;
    const double c2 = sig * sig / rc2, c6 = c2 * c2 * c2;
    const double fr = 24.0 * eps * (2.0 * s6 * s6 - s6) / r2;
    f[0] += fr * ax; f[1] += fr * ay; f[2] += fr * az;
    return 4.0 * eps * (s6 * s6 - s6) - 4.0 * eps * (c6 * c6 - c6);
  }
  // shifted LJ energy of a fluid atom at (x, y, z) with every site within
  // rc but site self (minimum image in x and z), and the force on it; uw
  // (if given) receives the part from wall sites
  double energy(double x, double y, double z, const mdgp_md_params& p, double f[3], int self = -1,
                double* uw = nullptr) const {
    double u = 0.0, w = 0.0;
    f[0] = f[1] = f[2] = 0.0;
    near_cells(x, y, z, p.rc, [&](const std::vector<int>& c) {
      for (int s : c) {
        if (s == self) continue;
        const double e = pair(x, y, z, s, p, f);
        u += e;
        if (wall[s]) w += e;
      }
    });
    if (uw) *uw = w;
    return u;
  }
  // the sites but self within distance r of (x, y, z)
  void within(double x, double y, double z, double r, int self, std::vector<int>& out) const {
    out.clear();
    near_cells(x, y, z, r, [&](const std::vector<int>& c) {
      for (int s : c) {
        if (s == self) continue;
        double ax = x - pos[3 * s], ay = y - pos[3 * s + 1], az = z - pos[3 * s + 2];
        ax -= Lx * std::floor(ax / Lx + 0.5);
        az -= Lz * std::floor(az / Lz + 0.5);
        if (ax * ax + ay * ay + az * az < r * r) out.push_back(s);
      }
    });
  }
};

// The start state of element E from snapshot S, the rule mdgp_micro_plan_from
// documents: xv gets (nf + nw) rows of (x y z vx vy vz); returns 0 for a cold
// start, 1 when the fluid comes from the snapshot, 2 when the walls do too.
int adapt_snapshot(const mdgp_md_params& p, const mdgp_element& el, const ElemDev& E, const mdgp_start& S,
                   std::vector<double>& xv) {
  if (!S.xv || S.n_fluid < 0 || S.n_wall != E.nw || std::fabs(S.h - E.h) > 1e-9 || std::fabs(S.Lx - E.Lx) > 1e-9 ||
      std::fabs(S.Lz - E.Lz) > 1e-9 || E.amp != 0.0)
    return 0;
  const long long nf = E.nf, nw = E.nw, n_old = S.n_fluid;
  xv.assign((size_t)6 * (nf + nw), 0.0);
  // which snapshot fluid atoms stay: all, or all but the n_old - nf with the smallest keys
  std::vector<long long> keep;
  keep.reserve((size_t)n_old);
  if (n_old > nf) {
    std::vector<std::pair<uint32_t, long long>> key((size_t)n_old);
    for (long long i = 0; i < n_old; ++i) {
      uint32_t r[4];
      philox_draw((uint32_t)i, 0u, (uint32_t)el.id, 2u, el.seed, r);
      key[(size_t)i] = {r[0], i};
    }
    std::sort(key.begin(), key.end());
    std::vector<char> gone((size_t)n_old, 0);
    for (long long i = 0; i < n_old - nf; ++i) gone[(size_t)key[(size_t)i].second] = 1;
    for (long long i = 0; i < n_old; ++i)
      if (!gone[(size_t)i]) keep.push_back(i);
  } else {
    for (long long i = 0; i < n_old; ++i) keep.push_back(i);
  }
  double vm[3] = {0.0, 0.0, 0.0};
  for (size_t k = 0; k < keep.size(); ++k) {
    const float* r = S.xv + 6 * keep[k];
    double* o = xv.data() + 6 * k;
    o[0] = (double)r[0] - E.Lx * std::floor((double)r[0] / E.Lx);
    o[1] = (double)r[1];
    o[2] = (double)r[2] - E.Lz * std::floor((double)r[2] / E.Lz);
    for (int d = 0; d < 3; ++d) { o[3 + d] = (double)r[3 + d]; vm[d] += (double)r[3 + d]; }
  }
  if (!keep.empty())
    for (int d = 0; d < 3; ++d) vm[d] /= (double)keep.size();
  for (long long w = 0; w < nw; ++w) {
    const float* r = S.xv + 6 * (n_old + w);
    double* o = xv.data() + 6 * (nf + w);
    for (int d = 0; d < 6; ++d) o[d] = (double)r[d];
    o[0] -= E.Lx * std::floor(o[0] / E.Lx);
    o[2] -= E.Lz * std::floor(o[2] / E.Lz);
  }
  // missing fluid atoms, one at a time: the lowest-energy of kInsertTries
  // Philox-drawn sites of the slab (the first at or below 0 ends the draw),
  // then steepest descent of the new atom's shifted LJ energy with the atoms
  // present (the USHER scheme of De Fabritiis, Delgado-Buscalioni and
  // Coveney, J. Chem. Phys. 121, 12139 (2004): steps along the force of
  // length U/|F|, at most kInsertStep, halved when U rises) until U <= 0 or
  // kInsertIters steps, then kRelaxIters steepest-descent steps of the new
  // atom and the fluid atoms within kRelaxR of it together (each atom moves
  // along its force, the largest move kRelaxStep) so the neighbours make
  // room; a site above kInsertUMax declines the snapshot.  The potential
  // energy this leaves above that of the kept fluid plus `add` atoms of its
  // mean per-atom energy is taken out of the fluid's peculiar kinetic
  // energy, so the total energy is that of the snapshot's state with nf
  // atoms and the temperature settles where it was.
  const long long add = nf - (long long)keep.size();
  if (add > 0) {
    constexpr double kInsertUMax = 1.0e3, kInsertStep = 0.05, kRelaxR = 2.0, kRelaxStep = 0.01;
    constexpr uint32_t kInsertTries = 64, kInsertIters = 200, kRelaxIters = 60;
    const int n_keep = (int)keep.size();
    SiteGrid grid(E.Lx, E.Lz, E.ylo, E.h - E.ylo, p.rc);
    for (int k = 0; k < n_keep; ++k) grid.add(xv[6 * k], xv[6 * k + 1], xv[6 * k + 2], 0);
    for (long long w = 0; w < nw; ++w) grid.add(xv[6 * (nf + w)], xv[6 * (nf + w) + 1], xv[6 * (nf + w) + 2], 1);
    const double y0 = 0.6, y1 = E.h - 0.6;
    if (!(y1 > y0)) return 0;
    // grid index of fluid atom a (kept atoms first, then the walls, then the new atoms)
    auto gi = [&](long long a) { return (int)(a < n_keep ? a : a + nw); };
    // potential energy of the fluid (fluid-fluid pairs once, fluid-wall pairs)
    auto fluid_energy = [&](long long n_fl, double* mean) {
      double tot = 0.0, sum = 0.0, f[3], w;
      for (long long a = 0; a < n_fl; ++a) {
        const int i = gi(a);
        const double u = grid.energy(grid.pos[3 * i], grid.pos[3 * i + 1], grid.pos[3 * i + 2], p, f, i, &w);
        tot += 0.5 * (u - w) + w;
        sum += u;
      }
      if (mean) *mean = n_fl > 0 ? sum / (double)n_fl : 0.0;
      return tot;
    };
    double ubar = 0.0;
    const double pe0 = fluid_energy(n_keep, &ubar);
    std::vector<int> set;
    std::vector<std::vector<int>> nbr;
    std::vector<double> fs, old;
    for (long long k = 0; k < add; ++k) {
      double best = INFINITY, c[3] = {0.0, 0.0, 0.0}, f[3];
      for (uint32_t tr = 0; tr < kInsertTries && best > 0.0; ++tr) {
        uint32_t r[4];
        philox_draw((uint32_t)k, tr, (uint32_t)el.id, 3u, el.seed, r);
        const double x = u01(r[0]) * E.Lx, y = y0 + u01(r[1]) * (y1 - y0), z = u01(r[2]) * E.Lz;
        const double u = grid.energy(x, y, z, p, f);
        if (u < best) { best = u; c[0] = x; c[1] = y; c[2] = z; }
      }
      double u = grid.energy(c[0], c[1], c[2], p, f), ds = kInsertStep;
      for (uint32_t it = 0; it < kInsertIters && u > 0.0 && ds > 1e-6; ++it) {
        const double fn = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
        if (!(fn > 0.0)) break;
        const double step = std::min(ds, u / fn);
        double t[3] = {c[0] + step * f[0] / fn, c[1] + step * f[1] / fn, c[2] + step * f[2] / fn};
        t[0] -= E.Lx * std::floor(t[0] / E.Lx);
        t[2] -= E.Lz * std::floor(t[2] / E.Lz);
        t[1] = std::min(y1, std::max(y0, t[1]));
        double ft[3];
        const double ut = grid.energy(t[0], t[1], t[2], p, ft);
        if (ut < u) {
          u = ut;
          for (int d = 0; d < 3; ++d) { c[d] = t[d]; f[d] = ft[d]; }
        } else {
          ds = 0.5 * step;
        }
      }
      if (!(u <= kInsertUMax)) return 0;
      const int g_new = n_keep + (int)nw + (int)k;
      grid.add(c[0], c[1], c[2], 0);
      // the new atom and its fluid neighbours relax together
      grid.within(c[0], c[1], c[2], kRelaxR, g_new, set);
      set.erase(std::remove_if(set.begin(), set.end(), [&](int i) { return grid.wall[i] != 0; }), set.end());
      set.insert(set.begin(), g_new);
      old.resize(3 * set.size());
      for (size_t m = 0; m < set.size(); ++m)
        for (int d = 0; d < 3; ++d) old[3 * m + d] = grid.pos[3 * set[m] + d];
      // the sites each set member can reach within rc while both move at
      // most kRelaxIters * kRelaxStep
      const double reach = p.rc + 2.0 * kRelaxIters * kRelaxStep;
      nbr.resize(set.size());
      for (size_t m = 0; m < set.size(); ++m) {
        const int i = set[m];
        grid.within(grid.pos[3 * i], grid.pos[3 * i + 1], grid.pos[3 * i + 2], reach, i, nbr[m]);
      }
      fs.resize(3 * set.size());
      for (uint32_t it = 0; it < kRelaxIters; ++it) {
        double fmax = 0.0;
        for (size_t m = 0; m < set.size(); ++m) {
          const int i = set[m];
          double* fm = &fs[3 * m];
          fm[0] = fm[1] = fm[2] = 0.0;
          for (int sidx : nbr[m]) grid.pair(grid.pos[3 * i], grid.pos[3 * i + 1], grid.pos[3 * i + 2], sidx, p, fm);
          fmax = std::max(fmax, std::sqrt(fm[0] * fm[0] + fm[1] * fm[1] + fm[2] * fm[2]));
        }
        if (!(fmax > 0.0)) break;
        const double alpha = kRelaxStep / fmax;
        for (size_t m = 0; m < set.size(); ++m) {
          const int i = set[m];
          double x = grid.pos[3 * i] + alpha * fs[3 * m], z = grid.pos[3 * i + 2] + alpha * fs[3 * m + 2];
          x -= E.Lx * std::floor(x / E.Lx);
          z -= E.Lz * std::floor(z / E.Lz);
          grid.pos[3 * i] = x;
          grid.pos[3 * i + 1] += alpha * fs[3 * m + 1];
          grid.pos[3 * i + 2] = z;
        }
      }
      // the moved atoms to their new cells
      for (size_t m = 0; m < set.size(); ++m) {
        const int i = set[m];
        const double x = grid.pos[3 * i], y = grid.pos[3 * i + 1], z = grid.pos[3 * i + 2];
        grid.pos[3 * i] = old[3 * m]; grid.pos[3 * i + 1] = old[3 * m + 1]; grid.pos[3 * i + 2] = old[3 * m + 2];
        grid.move(i, x, y, z);
      }
      const long long a = (long long)n_keep + k;
      double* o = xv.data() + 6 * a;
      uint32_t g[4];
      philox_draw((uint32_t)a, 0u, (uint32_t)el.id, 4u, el.seed, g);
      const double two_pi = 6.283185307179586476925286766559;
      const double rad1 = std::sqrt(-2.0 * std::log(u01(g[0]))), rad2 = std::sqrt(-2.0 * std::log(u01(g[2])));
      const double n3[3] = {rad1 * std::cos(two_pi * u01(g[1])), rad1 * std::sin(two_pi * u01(g[1])),
                            rad2 * std::cos(two_pi * u01(g[3]))};
      for (int d = 0; d < 3; ++d) o[3 + d] = E.vsd * n3[d] + vm[d];
    }
    // relaxed positions back, then the energy bookkeeping on the peculiar
    // kinetic energy (unit mass), scaled down at most to a quarter of itself
    for (long long a = 0; a < nf; ++a)
      for (int d = 0; d < 3; ++d) xv[6 * a + d] = grid.pos[3 * gi(a) + d];
    const double excess = fluid_energy(nf, nullptr) - pe0 - (double)add * ubar;
    double kin = 0.0;
    for (long long a = 0; a < nf; ++a)
      for (int d = 0; d < 3; ++d) kin += 0.5 * (xv[6 * a + 3 + d] - vm[d]) * (xv[6 * a + 3 + d] - vm[d]);
#ifdef DEBUG_ADAPT
    fprintf(stderr, "ubar %.3f excess %.2f (%.2f per atom) kin %.1f\n", ubar, excess, excess / add, kin);
#endif
    if (kin > 0.0) {
      const double s = std::sqrt(std::max(0.25, (kin - excess) / kin));
      for (long long a = 0; a < nf; ++a)
        for (int d = 0; d < 3; ++d) xv[6 * a + 3 + d] = vm[d] + s * (xv[6 * a + 3 + d] - vm[d]);
    }
  }
  return 1;
}

}  // namespace

// ---------------------------------------------------------------------------
// Kernel enqueue helpers (precision dispatch).
// ---------------------------------------------------------------------------
static void enqueue_integrate(mdgp_ctx* ctx, int k, int mode, cudaGraphConditionalHandle h = 0,
                              int use_cond = 0) {
  const unsigned g = grid_for(ctx->B.n_atoms, 256);
  const bool frozen = ctx->params.mode == 1;
  if (ctx->precision == MDGP_PREC_FP32) {
    if (frozen) k_integrate_df<true><<<g, 256, 0, ctx->stream>>>(ctx->B, ctx->P, k, mode, h, use_cond);
    else k_integrate_df<false><<<g, 256, 0, ctx->stream>>>(ctx->B, ctx->P, k, mode, h, use_cond);
  } else {
    if (frozen) k_integrate<double, Pos64, true><<<g, 256, 0, ctx->stream>>>(ctx->B, ctx->P, k, mode, h, use_cond);
    else k_integrate<double, Pos64, false><<<g, 256, 0, ctx->stream>>>(ctx->B, ctx->P, k, mode, h, use_cond);
  }
  ctx->launches++;
}

// Integration of one step: one fused launch, or for frozen-wall elements with
// the Berendsen thermostat two launches (the thermostat needs the element's
// sum of m v_z^2 between the half kick and the measurement).
static void enqueue_step_integrate(mdgp_ctx* ctx, int k, bool stage1, cudaGraphConditionalHandle h = 0,
                                   int use_cond = 0) {
  if (ctx->params.mode == 1) {
    enqueue_integrate(ctx, k, kFinish | kTzSum);
    enqueue_integrate(ctx, k, kTzApply | (stage1 ? kStage1 : 0), h, use_cond);
  } else {
    enqueue_integrate(ctx, k, kFinish | (stage1 ? kStage1 : 0), h, use_cond);
  }
}

// Neighbour-list rebuild: bin, per-element scan, permute into cell order,
// settle each cell's order while copying back, build the lists (5 kernels on
// `s`).
static void enqueue_rebuild(mdgp_ctx* ctx, cudaStream_t s) {
  const unsigned g = grid_for(ctx->B.n_atoms, 256);
  const unsigned gk = grid_for(ctx->B.n_cells, 1);
  if (ctx->precision == MDGP_PREC_FP32) {
    k_bin<true><<<g, 256, 0, s>>>(ctx->B);
    k_scan<<<(unsigned)ctx->n_el, 1024, 0, s>>>(ctx->B);
    k_permute<float4><<<g, 256, 0, s>>>(ctx->B);
    k_settle<float4><<<g, 256, 0, s>>>(ctx->B);
  } else {
    k_bin<false><<<g, 256, 0, s>>>(ctx->B);
    k_scan<<<(unsigned)ctx->n_el, 1024, 0, s>>>(ctx->B);
    k_permute<Pos64><<<g, 256, 0, s>>>(ctx->B);
    k_settle<Pos64><<<g, 256, 0, s>>>(ctx->B);
  }
  k_build_ballot_blk<<<gk, kBlkWarps * 32, kBlkSmem, s>>>(ctx->B, ctx->P);
}

// kernels in one rebuild: bin, scan, permute, settle, build
static int rebuild_kernels(const mdgp_ctx*) { return 5; }

static void enqueue_rebuild(mdgp_ctx* ctx) {
  enqueue_rebuild(ctx, ctx->stream);
  ctx->launches += rebuild_kernels(ctx);
}

// Pair forces of step *step_base + k (with per-atom energies if `energy`).
static void enqueue_force(mdgp_ctx* ctx, bool energy, int k) {
  const unsigned g = grid_for(ctx->B.n_atoms, 128);
  const bool uni = ctx->P.uniform != 0;
  cudaStream_t s = ctx->stream;
  if (ctx->precision == MDGP_PREC_FP32) {
    if (uni) {
      if (energy) k_force<float4, float, true, true><<<g, 128, 0, s>>>(ctx->B, ctx->P, k);
      else k_force<float4, float, true, false><<<g, 128, 0, s>>>(ctx->B, ctx->P, k);
    } else {
      if (energy) k_force<float4, float, false, true><<<g, 128, 0, s>>>(ctx->B, ctx->P, k);
      else k_force<float4, float, false, false><<<g, 128, 0, s>>>(ctx->B, ctx->P, k);
    }
  } else {
    if (uni) {
      if (energy) k_force<Pos64, double, true, true><<<g, 128, 0, s>>>(ctx->B, ctx->P, k);
      else k_force<Pos64, double, true, false><<<g, 128, 0, s>>>(ctx->B, ctx->P, k);
    } else {
      if (energy) k_force<Pos64, double, false, true><<<g, 128, 0, s>>>(ctx->B, ctx->P, k);
      else k_force<Pos64, double, false, false><<<g, 128, 0, s>>>(ctx->B, ctx->P, k);
    }
  }
  ctx->launches++;
}

// FP32 pair forces: one fused launch per step (forces + integration, the
// forces kept in registers); with the frozen-wall thermostat the fused launch
// finishes the step and sums m v_z^2 (storing the forces), and a second
// launch applies the thermostat and starts the next step.
static void enqueue_step_fused(mdgp_ctx* ctx, int k, bool stage1, cudaGraphConditionalHandle h = 0,
                               int use_cond = 0) {
  constexpr int kT = 128;
  const unsigned g = grid_for(ctx->B.n_atoms, kT);
  const bool uni = ctx->P.uniform != 0;
  cudaStream_t s = ctx->stream;
  if (ctx->params.mode == 1) {
    const int m = kFinish | kTzSum;
    if (uni) k_step_df<true, true, true><<<g, kT, 0, s>>>(ctx->B, ctx->P, k, m, 0, 0);
    else k_step_df<false, true, true><<<g, kT, 0, s>>>(ctx->B, ctx->P, k, m, 0, 0);
    ctx->launches++;
    enqueue_integrate(ctx, k, kTzApply | (stage1 ? kStage1 : 0), h, use_cond);
  } else {
    const int m = kFinish | (stage1 ? kStage1 : 0);
    if (uni) k_step_df<true, false, false><<<g, kT, 0, s>>>(ctx->B, ctx->P, k, m, h, use_cond);
    else k_step_df<false, false, false><<<g, kT, 0, s>>>(ctx->B, ctx->P, k, m, h, use_cond);
    ctx->launches++;
  }
}

static void enqueue_energy(mdgp_ctx* ctx, int which) {
  const unsigned g = grid_for(ctx->B.n_atoms, 256);
  if (ctx->precision == MDGP_PREC_FP32) k_energy<float><<<g, 256, 0, ctx->stream>>>(ctx->B, ctx->P, which);
  else k_energy<double><<<g, 256, 0, ctx->stream>>>(ctx->B, ctx->P, which);
  ctx->launches++;
}

static void enqueue_export(mdgp_ctx* ctx, int what) {
  const unsigned g = grid_for(ctx->B.n_atoms, 256);
  if (ctx->precision == MDGP_PREC_FP32) k_export<float><<<g, 256, 0, ctx->stream>>>(ctx->B, what);
  else k_export<double><<<g, 256, 0, ctx->stream>>>(ctx->B, what);
}

// Per element: means, block standard errors, temperature and energy drift.
__global__ void k_finalize(BatchDev B, mdgp_result* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B.n_el) return;
  const ElemDev& E = B.el[e];
  const double* acc = B.acc + (size_t)e * kAccStride;
  mdgp_result r;
  const int nb = E.nb;
  const long long S = E.steps_sample;
  const double vol = E.Lx * E.hvol * E.Lz;
  double qs = 0.0, ps = 0.0, qm[kMaxBlocks], pm[kMaxBlocks];
  for (int b = 0; b < nb; ++b) {
    const long long lo = (b * S + nb - 1) / nb, hi = ((b + 1) * S + nb - 1) / nb;
    const double cnt = (double)(hi - lo);
    qs += acc[kAccQ + b];
    ps += acc[kAccP + b];
    qm[b] = cnt > 0 ? acc[kAccQ + b] / cnt / E.Lx : 0.0;
    pm[b] = cnt > 0 ? acc[kAccP + b] / cnt / vol : 0.0;
  }
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  r.q = S > 0 ? qs / (double)S / E.Lx : nan;
  r.p = S > 0 ? ps / (double)S / vol : nan;
  if (nb >= 2) {
    double mq = 0.0, mp = 0.0;
    for (int b = 0; b < nb; ++b) { mq += qm[b]; mp += pm[b]; }
    mq /= nb; mp /= nb;
    double vq = 0.0, vp = 0.0;
    for (int b = 0; b < nb; ++b) { vq += (qm[b] - mq) * (qm[b] - mq); vp += (pm[b] - mp) * (pm[b] - mp); }
    r.q_se = sqrt(vq / (nb - 1) / nb);
    r.p_se = sqrt(vp / (nb - 1) / nb);
  } else {
    r.q_se = nan;
    r.p_se = nan;
  }
  r.T_meas = (S > 0 && E.nf > 0) ? acc[kAccT] / (3.0 * (double)E.nf * (double)S) : nan;
  const long long n = (long long)E.nf + E.nw;
  r.e_drift = n > 0 ? (acc[kAccE1] - acc[kAccE0]) / (double)n : 0.0;
  r.n_fluid = E.nf;
  r.n_wall = E.nw;
  r.status = B.status[e];
  r.start = E.warm;
  out[e] = r;
}

// ---------------------------------------------------------------------------
// Planning.
// ---------------------------------------------------------------------------
static void drop_graphs(mdgp_ctx* ctx) {
  if (ctx->graph_full) { cudaGraphExecDestroy(ctx->graph_full); ctx->graph_full = nullptr; }
  if (ctx->graph_rem) { cudaGraphExecDestroy(ctx->graph_rem); ctx->graph_rem = nullptr; }
  if (ctx->graph_while) { cudaGraphExecDestroy(ctx->graph_while); ctx->graph_while = nullptr; }
  ctx->graph_K = ctx->graph_rem_K = 0;
}

// Record `nsteps` steps into a graph.  Each step is: integrate, an IF node
// whose body rebuilds the neighbour lists (raised by the integrate kernel
// when some atom moved more than half the skin since the last build), and
// the force kernel.  The last node advances the step counter.
static int capture_steps(mdgp_ctx* ctx, long long nsteps, cudaGraphExec_t* out) {
  cudaGraph_t g;
  CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  for (long long k = 0; k < nsteps; ++k) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t cg;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edges = nullptr;
    size_t ndeps = 0;
    CK(cudaStreamGetCaptureInfo(ctx->stream, &cs, nullptr, &cg, &deps, &edges, &ndeps));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, cg, 0, cudaGraphCondAssignDefault));
    const bool fused = ctx->precision == MDGP_PREC_FP32;
    if (fused) enqueue_step_fused(ctx, (int)k, true, h, 1);
    else enqueue_step_integrate(ctx, (int)k, true, h, 1);
    CK(cudaStreamGetCaptureInfo(ctx->stream, &cs, nullptr, &cg, &deps, &edges, &ndeps));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, cg, deps, edges, ndeps, &cp));
    CK(cudaStreamUpdateCaptureDependencies(ctx->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(ctx->side_stream, body, nullptr, nullptr, 0,
                                     cudaStreamCaptureModeThreadLocal));
    enqueue_rebuild(ctx, ctx->side_stream);
    cudaGraph_t body_out;
    CK(cudaStreamEndCapture(ctx->side_stream, &body_out));
    if (!fused) enqueue_force(ctx, false, (int)k + 1);
  }
  k_advance<<<1, 32, 0, ctx->stream>>>((long long*)ctx->d_step.ptr, nsteps);
  cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
  if (e != cudaSuccess) return set_err(ctx, e);
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  return set_err(ctx, e);
}

// The persistent step kernel for a batch's pair types, wall mode and
// threads per atom (1, 2, 4 or 8).
using PersistFn = void (*)(mdgp::BatchDev, mdgp::PhysDev, long long, int, cudaGraphConditionalHandle,
                           cudaGraphConditionalHandle, int);
template <bool U, bool F>
static PersistFn persist_kernel_tpa(int tpa) {
  switch (tpa) {
    case 2: return k_steps_persist<U, F, 2>;
    case 4: return k_steps_persist<U, F, 4>;
    case 8: return k_steps_persist<U, F, 8>;
    default: return k_steps_persist<U, F, 1>;
  }
}
static PersistFn persist_kernel(bool uni, bool frozen, int tpa) {
  if (uni && !frozen) return persist_kernel_tpa<true, false>(tpa);
  if (!uni && !frozen) return persist_kernel_tpa<false, false>(tpa);
  if (uni) return persist_kernel_tpa<true, true>(tpa);
  return persist_kernel_tpa<false, true>(tpa);
}

// The resident-atom step kernel (tethered walls, 2, 4 or 8 threads per atom).
template <bool U>
static PersistFn resident_kernel_tpa(int tpa) {
  switch (tpa) {
    case 2: return k_steps_resident<U, 2>;
    case 4: return k_steps_resident<U, 4>;
    default: return k_steps_resident<U, 8>;
  }
}
static PersistFn resident_kernel(bool uni, int tpa) {
  return uni ? resident_kernel_tpa<true>(tpa) : resident_kernel_tpa<false>(tpa);
}

// The step-loop kernel the plan chose.
static PersistFn step_loop_kernel(const mdgp_ctx* ctx) {
  const bool uni = ctx->P.uniform != 0, frozen = ctx->params.mode == 1;
  return ctx->persist_resident ? resident_kernel(uni, ctx->persist_tpa)
                               : persist_kernel(uni, frozen, ctx->persist_tpa);
}

// Persistent step loop (FP32 pair forces): a graph with one WHILE node
// whose body is [cooperative k_steps_persist launch] -> IF (rebuild) {the 5
// rebuild kernels}.  The step kernel runs steps until the lists need a
// rebuild or all S steps have been started, and sets both conditions.
static int capture_while(mdgp_ctx* ctx, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle hw;
  cudaError_t e = cudaGraphConditionalHandleCreate(&hw, g, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams wp = {};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = hw;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wnode;
  if (e == cudaSuccess) e = cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &wp);
  if (e != cudaSuccess) { cudaGraphDestroy(g); return set_err(ctx, e); }
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  cudaGraphConditionalHandle hr;
  e = cudaGraphConditionalHandleCreate(&hr, body, 0, cudaGraphCondAssignDefault);
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(ctx->side_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) { cudaGraphDestroy(g); return set_err(ctx, e); }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctx->persist_grid);
  cfg.blockDim = dim3(ctx->persist_threads);
  cfg.dynamicSmemBytes = ctx->persist_smem;
  cfg.stream = ctx->side_stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const long long S = ctx->steps;
  const int A = ctx->persist_atoms;
  e = cudaLaunchKernelEx(&cfg, step_loop_kernel(ctx), ctx->B, ctx->P, S, A, hr, hw, 1);
  cudaStreamCaptureStatus cs;
  cudaGraph_t cg;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edges = nullptr;
  size_t ndeps = 0;
  if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(ctx->side_stream, &cs, nullptr, &cg, &deps, &edges, &ndeps);
  cudaGraphNodeParams ip = {};
  ip.type = cudaGraphNodeTypeConditional;
  ip.conditional.handle = hr;
  ip.conditional.type = cudaGraphCondTypeIf;
  ip.conditional.size = 1;
  cudaGraphNode_t inode;
  if (e == cudaSuccess) e = cudaGraphAddNode(&inode, cg, deps, edges, ndeps, &ip);
  if (e == cudaSuccess)
    e = cudaStreamUpdateCaptureDependencies(ctx->side_stream, &inode, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(ctx->side_stream2, ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    enqueue_rebuild(ctx, ctx->side_stream2);
    cudaGraph_t tmp;
    e = cudaStreamEndCapture(ctx->side_stream2, &tmp);
  }
  cudaGraph_t tmp2;
  const cudaError_t e2 = cudaStreamEndCapture(ctx->side_stream, &tmp2);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  return set_err(ctx, e);
}

static int plan_impl(mdgp_ctx* ctx, const mdgp_element* el, int64_t n, int list_cap_override,
                     const mdgp_start* starts = nullptr) {
  ctx->planned = false;
  drop_graphs(ctx);
  if (ctx->params.mode != 0 && ctx->params.mode != 1) {
    std::snprintf(ctx->err, sizeof(ctx->err), "mode must be 0 (tethered walls) or 1 (frozen walls)");
    return MDGP_E_ARG;
  }
  if (ctx->params.mode == 1 && !(ctx->params.tau_T > 0)) {
    std::snprintf(ctx->err, sizeof(ctx->err), "mode 1 needs tau_T > 0");
    return MDGP_E_ARG;
  }
  std::vector<ElemDev> Es((size_t)n);
  std::vector<long long> aoff((size_t)n + 1), coff((size_t)n + 1);
  long long atoms = 0, cells = 0, columns = 0;
  const long long S = el[0].steps_eq + el[0].steps_sample;
  double Tmax = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    std::string why;
    int st = describe(ctx->params, el[i], Es[i], &why);
    if (st != MDGP_OK) {
      std::snprintf(ctx->err, sizeof(ctx->err), "element %lld: %s", (long long)i, why.c_str());
      return st;
    }
    if (Es[i].steps_total != S) {
      std::snprintf(ctx->err, sizeof(ctx->err), "elements of one plan must share steps_eq + steps_sample");
      return MDGP_E_ARG;
    }
    Tmax = std::max(Tmax, el[i].T);
    Es[i].atom0 = atoms;
    Es[i].cell0 = cells;
    aoff[i] = atoms;
    coff[i] = cells;
    columns += (long long)Es[i].nc[0] * Es[i].nc[1];
    atoms += (long long)Es[i].nf + Es[i].nw;
    cells += (long long)Es[i].nc[0] * Es[i].nc[1] * Es[i].nc[2];
    if ((long long)Es[i].nf + Es[i].nw >= (1LL << 26)) {
      std::snprintf(ctx->err, sizeof(ctx->err), "element %lld has more than 2^26 atoms", (long long)i);
      return MDGP_E_ARG;
    }
  }
  aoff[n] = atoms;
  coff[n] = cells;
  // start states from snapshots, prepared on the host (copied to the device below)
  // (elements in parallel on host threads; each writes its own rows)
  std::vector<double> warm;
  bool any_warm = false;
  std::vector<int64_t> from;
  for (int64_t i = 0; starts && i < n; ++i)
    if (starts[i].xv) from.push_back(i);
  if (!from.empty()) {
    warm.assign((size_t)6 * atoms, 0.0);
    const int nt = (int)std::min<int64_t>((int64_t)from.size(),
                                          std::max(1u, std::min(16u, std::thread::hardware_concurrency())));
    auto work = [&](int t) {
      std::vector<double> xv;
      for (size_t q = (size_t)t; q < from.size(); q += (size_t)nt) {
        const int64_t i = from[q];
        Es[i].warm = adapt_snapshot(ctx->params, el[i], Es[i], starts[i], xv);
        if (Es[i].warm) std::copy(xv.begin(), xv.end(), warm.begin() + 6 * Es[i].atom0);
      }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(work, t);
    work(0);
    for (std::thread& th : pool) th.join();
    for (int64_t i : from) any_warm |= Es[i].warm != 0;
    if (!any_warm) std::vector<double>().swap(warm);
  }
  if (atoms >= (1LL << 31) - 1) {
    std::snprintf(ctx->err, sizeof(ctx->err), "batch too large (2^31 atoms max)");
    return MDGP_E_ARG;
  }
  // initial positions of elements with profiled walls, built on the host
  std::vector<double> pinit;
  for (int64_t i = 0; i < n; ++i) {
    if (Es[i].amp == 0.0) continue;
    if (pinit.empty()) pinit.assign((size_t)3 * atoms, 0.0);
    profiled_positions(ctx->params, Es[i], pinit.data() + 3 * Es[i].atom0);
  }
  int list_cap = ctx->params.list_capacity > 0 ? ctx->params.list_capacity : 128;
  if (list_cap_override > list_cap) list_cap = list_cap_override;
  list_cap = (list_cap + 3) / 4 * 4;  // whole groups of four
  const size_t fsz = ctx->precision == MDGP_PREC_FP32 ? 4 : 8;
  const size_t psz = ctx->precision == MDGP_PREC_FP32 ? sizeof(float4) : sizeof(Pos64);
  const size_t N = (size_t)atoms, C = (size_t)cells;
  int st;
  if ((st = ensure(ctx, ctx->d_el, sizeof(ElemDev) * n))) return st;
  if ((st = ensure(ctx, ctx->d_aoff, sizeof(long long) * (n + 1)))) return st;
  if ((st = ensure(ctx, ctx->d_coff, sizeof(long long) * (n + 1)))) return st;
  if ((st = ensure(ctx, ctx->d_state, sizeof(double) * 18 * N))) return st;
  if ((st = ensure(ctx, ctx->d_ints, sizeof(int) * 8 * N))) return st;
  if ((st = ensure(ctx, ctx->d_cells, sizeof(int) * 4 * C))) return st;
  const size_t npos = ctx->precision == MDGP_PREC_FP32 ? 2 : 1;
  if ((st = ensure(ctx, ctx->d_pos, npos * psz * N))) return st;
  if ((st = ensure(ctx, ctx->d_pbuild, sizeof(float4) * N))) return st;
  if ((st = ensure(ctx, ctx->d_force, fsz * 5 * N))) return st;
  if ((st = ensure(ctx, ctx->d_list, sizeof(unsigned) * (size_t)list_cap * N))) return st;
  if ((st = ensure(ctx, ctx->d_out, sizeof(double) * 6 * N))) return st;
  if ((st = ensure(ctx, ctx->d_acc, sizeof(double) * kAccStride * n))) return st;
  if ((st = ensure(ctx, ctx->d_grp, sizeof(double) * 2 * kGrpStride * n))) return st;
  if ((st = ensure(ctx, ctx->d_status, sizeof(int) * n))) return st;
  if ((st = ensure(ctx, ctx->d_results, sizeof(mdgp_result) * n))) return st;
  if ((st = ensure(ctx, ctx->d_step, sizeof(long long)))) return st;
  if ((st = ensure(ctx, ctx->d_flags, sizeof(int) * kFlags))) return st;
  if ((st = ensure(ctx, ctx->d_tz, sizeof(double) * 2 * n))) return st;
  if (any_warm && (st = ensure(ctx, ctx->d_warm, sizeof(double) * 6 * N))) return st;
  if (!pinit.empty() && (st = ensure(ctx, ctx->d_pinit, sizeof(double) * 3 * N))) return st;
  if (!pinit.empty())
    CK(cudaMemcpyAsync(ctx->d_pinit.ptr, pinit.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_el.ptr, Es.data(), sizeof(ElemDev) * n, cudaMemcpyHostToDevice, ctx->stream));
  ctx->el_host = Es;
  ctx->el_desc.assign(el, el + n);
  ctx->ran = false;
  CK(cudaMemcpyAsync(ctx->d_aoff.ptr, aoff.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_coff.ptr, coff.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice, ctx->stream));
  if (any_warm)
    CK(cudaMemcpyAsync(ctx->d_warm.ptr, warm.data(), sizeof(double) * 6 * N, cudaMemcpyHostToDevice, ctx->stream));
  ctx->any_warm = any_warm;

  BatchDev& B = ctx->B;
  std::memset(&B, 0, sizeof(B));
  B.el = (const ElemDev*)ctx->d_el.ptr;
  B.atom_off = (const long long*)ctx->d_aoff.ptr;
  B.cell_off = (const long long*)ctx->d_coff.ptr;
  B.n_el = (int)n;
  B.list_cap = list_cap;
  B.n_atoms = atoms;
  B.n_cells = cells;
  double* sd = (double*)ctx->d_state.ptr;
  for (int k = 0; k < 9; ++k) { B.st[k] = sd + k * N; B.st2[k] = sd + (9 + k) * N; }
  int* ip = (int*)ctx->d_ints.ptr;
  B.orig = ip; B.cell = ip + N; B.orig2 = ip + 2 * N; B.cell2 = ip + 3 * N;
  B.atom_el = ip + 4 * N; B.newcell = ip + 5 * N; B.slot = ip + 6 * N; B.nlist = ip + 7 * N;
  int* cp = (int*)ctx->d_cells.ptr;
  B.cell_el = cp; B.ccount = cp + C; B.cstart = cp + 2 * C; B.csize = cp + 3 * C;
  B.posb[0] = ctx->d_pos.ptr;
  B.posb[1] = (char*)ctx->d_pos.ptr + (npos - 1) * psz * N;
  B.pbuild = (float4*)ctx->d_pbuild.ptr;
  char* fb = (char*)ctx->d_force.ptr;
  B.fx = fb; B.fy = fb + fsz * N; B.fz = fb + 2 * fsz * N;
  B.wxx = fb + 3 * fsz * N; B.epot = fb + 4 * fsz * N;
  B.list = (unsigned*)ctx->d_list.ptr;
  B.out = (double*)ctx->d_out.ptr;
  B.acc = (double*)ctx->d_acc.ptr;
  B.grp = (double*)ctx->d_grp.ptr;
  B.status = (int*)ctx->d_status.ptr;
  B.step_base = (long long*)ctx->d_step.ptr;
  B.flags = (int*)ctx->d_flags.ptr;
  B.tz = (double*)ctx->d_tz.ptr;
  B.warm = any_warm ? (const double*)ctx->d_warm.ptr : nullptr;
  B.pinit = pinit.empty() ? nullptr : (const double*)ctx->d_pinit.ptr;
  ctx->P = make_phys(ctx->params, list_cap);
  ctx->n_el = n;
  ctx->steps = S;
  ctx->n_atoms = atoms;
  ctx->rebuild_every = rebuild_interval(ctx->params, Tmax > 0 ? Tmax : 1.0);
  const long long big = atoms > cells ? atoms : cells;
  const unsigned gm = grid_for(big, 256);
  k_fill_maps<<<gm < 4096 ? gm : 4096, 256, 0, ctx->stream>>>(B);
  CK(cudaGetLastError());

  // Step loop: FP32 pair forces run the persistent WHILE graph (when
  // params.persistent is set and the device takes the cooperative launch),
  // otherwise chunks of K steps with one conditional rebuild per step.
  const long long K = ctx->chunk;
  bool use_while = false;
  ctx->direct = S > 0 && ctx->precision == MDGP_PREC_FP32 && ctx->params.persistent == 2;
  if (S > 0 && ctx->precision == MDGP_PREC_FP32 && ctx->params.persistent) {
    // Persistent grid: R co-resident blocks per SM, each taking A = N / (R x
    // SMs) atoms rounded up, so that every SM holds about N / SMs atoms (the
    // step ends with the most loaded SM); the block is A x TPA threads
    // rounded up to whole warps.  The R with the fewest warps per SM (the
    // least idle lanes) among those that fit wins.  TPA, the threads per
    // atom, is the largest power of two up to 8 with N x TPA threads within
    // the SMs' capacity for this kernel (one thread per atom for batches that
    // fill the GPU; several share an atom's pair loop in smaller ones, which
    // shortens the step's critical path) unless the parameters fix it; where
    // the resident-atom kernel applies, the automatic choice steps down from
    // there to the most threads per atom at which that kernel fits.
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    const bool uni = ctx->P.uniform != 0, frozen = ctx->params.mode == 1;
    auto occupancy = [&](int tpa, int threads, int* per_sm) {
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, persist_kernel(uni, frozen, tpa), threads, 0);
    };
    int tpa = ctx->params.threads_per_atom;
    const bool auto_tpa = tpa <= 0;
    if (auto_tpa) {
      int per_sm = 0;
      if (occupancy(1, 256, &per_sm) != cudaSuccess) return set_err(ctx, cudaGetLastError());
      const long long cap = (long long)sms * per_sm * 256;
      tpa = 1;
      while (tpa < 8 && atoms * (2 * tpa) <= cap) tpa *= 2;
    }
    ctx->persist_tpa = tpa;
    ctx->persist_grid = 0;
    ctx->persist_resident = false;
    ctx->persist_smem = 0;
    // One block per chunk of A atoms, R blocks per SM, t threads per atom;
    // the resident-atom kernel (tethered walls, several threads per atom) is
    // tried first, with its lists' shared memory in the occupancy, then the
    // general one.
    const int list_cap = ctx->B.list_cap;
    size_t res_max_smem = 0;   // dynamic shared memory a block of the resident kernel may take
    auto search = [&](bool resident, int t) -> cudaError_t {
      long long best_warps = 1LL << 40;
      for (int R = 1; R <= 32; ++R) {
        const long long slots = (long long)sms * R;
        const long long A = (atoms + slots - 1) / slots;
        const int T = (int)((A * t + 31) / 32 * 32);
        // at least 128 threads: smaller blocks put more separate atom ranges on
        // an SM and lose L1 reuse of the neighbour positions (measured slower)
        if (T > 256 || T < 128) continue;   // larger batches: 256-thread blocks striding over chunks
        int per_sm = 0;
        const size_t smem = resident ? resident_smem_bytes((int)A, list_cap) : 0;
        if (smem > res_max_smem && resident) continue;   // the lists do not fit
        const cudaError_t oe =
            resident ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, resident_kernel(uni, t), T, smem)
                     : occupancy(t, T, &per_sm);
        if (oe != cudaSuccess) return oe;
        const long long warps = (long long)R * (T / 32);
        if (per_sm >= R && warps < best_warps) {
          best_warps = warps;
          ctx->persist_atoms = (int)A;
          ctx->persist_threads = T;
          ctx->persist_grid = (unsigned)((atoms + A - 1) / A);
          ctx->persist_tpa = t;
          ctx->persist_resident = resident;
          ctx->persist_smem = smem;
        }
      }
      return cudaSuccess;
    };
    // 256-thread blocks of 256 / t atoms, one chunk per block, for batches too
    // small for 128-thread blocks on every SM: the resident kernel when all
    // its blocks fit at once
    auto resident_small = [&](int t) -> cudaError_t {
      const int A = 256 / t;
      const long long chunks = (atoms + A - 1) / A;
      const size_t smem = resident_smem_bytes(A, list_cap);
      if (smem > res_max_smem) return cudaSuccess;
      int per_sm = 0;
      const cudaError_t oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, resident_kernel(uni, t), 256, smem);
      if (oe != cudaSuccess) return oe;
      if (chunks <= (long long)per_sm * sms) {
        ctx->persist_atoms = A;
        ctx->persist_threads = 256;
        ctx->persist_grid = (unsigned)chunks;
        ctx->persist_tpa = t;
        ctx->persist_resident = true;
        ctx->persist_smem = smem;
      }
      return cudaSuccess;
    };
    if (ctx->params.resident && !frozen && tpa > 1) {
      // with the automatic choice, the most threads per atom (from tpa down to
      // two) at which the resident kernel fits: in small batches it beats more
      // threads per atom with the general kernel
      for (int t = tpa; t >= 2 && ctx->persist_grid == 0; t = auto_tpa ? t / 2 : 1) {
        // the lists may need more than the default 48 KB of dynamic shared memory
        int optin = 0;
        cudaFuncAttributes fa = {};
        CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
        CK(cudaFuncGetAttributes(&fa, resident_kernel(uni, t)));
        res_max_smem = (size_t)(optin - (int)fa.sharedSizeBytes);
        CK(cudaFuncSetAttribute(resident_kernel(uni, t), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)res_max_smem));
        cudaError_t se = search(true, t);
        if (se == cudaSuccess && ctx->persist_grid == 0) se = resident_small(t);
        if (se != cudaSuccess) return set_err(ctx, se);
      }
    }
    if (ctx->persist_grid == 0) {
      ctx->persist_tpa = tpa;
      const cudaError_t se = search(false, tpa);
      if (se != cudaSuccess) return set_err(ctx, se);
    }
    if (ctx->persist_grid == 0) {
      int per_sm = 0;
      if (occupancy(tpa, 256, &per_sm) != cudaSuccess) return set_err(ctx, cudaGetLastError());
      const int A = 256 / tpa;
      const long long chunks = (atoms + A - 1) / A, cap = (long long)per_sm * sms;
      ctx->persist_atoms = A;
      ctx->persist_threads = 256;
      ctx->persist_grid = (unsigned)(chunks < cap ? chunks : cap);
    }
    const long long saved = ctx->launches;
    if (ctx->direct) use_while = true;   // no graphs: run_direct launches the persistent kernel itself
    else if (ctx->persist_grid > 0 && capture_while(ctx, &ctx->graph_while) == MDGP_OK) use_while = true;
    else cudaGetLastError();   // fall back to the per-step graphs
    ctx->launches = saved;
  }
  if (S > 0 && !use_while) {
    const long long saved = ctx->launches;
    if (S >= K) {
      if ((st = capture_steps(ctx, K, &ctx->graph_full))) return st;
      ctx->graph_K = K;
    }
    const long long rem = S % K;
    if (rem) {
      if ((st = capture_steps(ctx, rem, &ctx->graph_rem))) return st;
      ctx->graph_rem_K = rem;
    }
    ctx->launches = saved;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->planned = true;
  return MDGP_OK;
}

// kernels in one chunk graph, rebuild bodies not counted
// Kernel launches of a captured chunk of nsteps steps (rebuilds not counted):
// FP32 one fused launch per step (two with the frozen-wall thermostat), FP64
// integration (one or two) plus forces; one counter advance per chunk.
static long long graph_launches(long long nsteps, int mode, int precision) {
  const long long per = precision == MDGP_PREC_FP32 ? (mode == 1 ? 2 : 1) : (mode == 1 ? 3 : 2);
  return per * nsteps + 1;
}

// Reset the accumulators and build the elements (lattice, anchors,
// Maxwell-Boltzmann velocities).
static int start_batch(mdgp_ctx* ctx) {
  const int n = (int)ctx->n_el;
  CK(cudaMemsetAsync(ctx->d_acc.ptr, 0, sizeof(double) * kAccStride * n, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_grp.ptr, 0, sizeof(double) * 2 * kGrpStride * n, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_status.ptr, 0, sizeof(int) * n, ctx->stream));
  CK(cudaMemsetAsync(ctx->B.ccount, 0, sizeof(int) * ctx->B.n_cells, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_step.ptr, 0, sizeof(long long), ctx->stream));
  CK(cudaMemsetAsync(ctx->B.flags, 0, sizeof(int) * kFlags, ctx->stream));
  CK(cudaMemsetAsync(ctx->B.tz, 0, sizeof(double) * 2 * n, ctx->stream));
  const unsigned ga = grid_for(ctx->B.n_atoms, 256);
  const unsigned ge = (unsigned)ctx->n_el;
  if (ctx->precision == MDGP_PREC_FP32) {
    k_init_atoms<true><<<ga, 256, 0, ctx->stream>>>(ctx->B, ctx->P);
    k_group_sums<true><<<ge, 256, 0, ctx->stream>>>(ctx->B);
    k_init_fix<true><<<ga, 256, 0, ctx->stream>>>(ctx->B, ctx->P);
    if (ctx->any_warm) k_apply_warm<true><<<ga, 256, 0, ctx->stream>>>(ctx->B);
  } else {
    k_init_atoms<false><<<ga, 256, 0, ctx->stream>>>(ctx->B, ctx->P);
    k_group_sums<false><<<ge, 256, 0, ctx->stream>>>(ctx->B);
    k_init_fix<false><<<ga, 256, 0, ctx->stream>>>(ctx->B, ctx->P);
    if (ctx->any_warm) k_apply_warm<false><<<ga, 256, 0, ctx->stream>>>(ctx->B);
  }
  ctx->launches += ctx->any_warm ? 4 : 3;
  return MDGP_OK;
}

// Persistent step loop launched from the host (persistent = 2): one
// cooperative launch per list-rebuild interval, no graph.  After each
// launch the host reads the step counter back; short of the last step, the
// kernel stopped for a rebuild (or gave up a barrier wait, which flags
// record), and the host enqueues the rebuild and launches again.  Slower
// than the WHILE graph (a host round trip per interval) but every launch is
// an ordinary kernel launch, which a profiler can capture.
static int run_direct(mdgp_ctx* ctx) {
  const long long S = ctx->steps;
  const int A = ctx->persist_atoms;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctx->persist_grid);
  cfg.blockDim = dim3(ctx->persist_threads);
  cfg.dynamicSmemBytes = ctx->persist_smem;
  cfg.stream = ctx->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaGraphConditionalHandle h0 = 0;
  for (cudaEvent_t& ev : ctx->dir_ev)
    if (!ev) CK(cudaEventCreate(&ev));
  ctx->dir_kernel_ms = ctx->dir_rebuild_ms = 0.0;
  ctx->dir_steps = ctx->dir_launches = ctx->dir_rebuilds = 0;
  long long prev = 0;
  bool rebuilt = false;
  for (long long guard = 0; guard <= S; ++guard) {
    CK(cudaEventRecord(ctx->dir_ev[1], ctx->stream));
    cudaError_t e;
    e = cudaLaunchKernelEx(&cfg, step_loop_kernel(ctx), ctx->B, ctx->P, S, A, h0, h0, 0);
    if (e != cudaSuccess) return set_err(ctx, e);
    CK(cudaEventRecord(ctx->dir_ev[2], ctx->stream));
    ++ctx->launches;
    long long step = 0;
    int failed = 0;
    CK(cudaMemcpyAsync(&step, ctx->d_step.ptr, sizeof(long long), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(&failed, ctx->B.flags + kFlagExit, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    float ms = 0.f;
    if (rebuilt && cudaEventElapsedTime(&ms, ctx->dir_ev[0], ctx->dir_ev[1]) == cudaSuccess) {
      ctx->dir_rebuild_ms += ms;
      ++ctx->dir_rebuilds;
    }
    if (cudaEventElapsedTime(&ms, ctx->dir_ev[1], ctx->dir_ev[2]) == cudaSuccess) ctx->dir_kernel_ms += ms;
    ctx->dir_steps += step - prev;
    ++ctx->dir_launches;
    prev = step;
    if (step >= S || failed) break;
    CK(cudaEventRecord(ctx->dir_ev[0], ctx->stream));
    enqueue_rebuild(ctx);
    rebuilt = true;
  }
  return MDGP_OK;
}

// A continued run (resume) keeps the atom state of the last launch and
// clears only the measurements, the counters and the step.
static int resume_batch(mdgp_ctx* ctx) {
  const int n = (int)ctx->n_el;
  CK(cudaMemsetAsync(ctx->d_acc.ptr, 0, sizeof(double) * kAccStride * n, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_status.ptr, 0, sizeof(int) * n, ctx->stream));
  CK(cudaMemsetAsync(ctx->B.ccount, 0, sizeof(int) * ctx->B.n_cells, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_step.ptr, 0, sizeof(long long), ctx->stream));
  CK(cudaMemsetAsync(ctx->B.flags, 0, sizeof(int) * kFlags, ctx->stream));
  CK(cudaMemsetAsync(ctx->B.tz, 0, sizeof(double) * 2 * n, ctx->stream));
  return MDGP_OK;
}

static int launch_impl(mdgp_ctx* ctx, bool resume = false) {
  if (!ctx->planned) return MDGP_E_STATE;
  ctx->launches = 0;
  int st;
  if ((st = resume ? resume_batch(ctx) : start_batch(ctx))) return st;
  enqueue_rebuild(ctx);
  enqueue_force(ctx, true, 0);
  enqueue_energy(ctx, kAccE0);
  const long long S = ctx->steps;
  if (S > 0) {
    if (ctx->direct) {
      if ((st = run_direct(ctx))) return st;
    } else if (ctx->graph_while) {
      CK(cudaGraphLaunch(ctx->graph_while, ctx->stream));   // persistent launches counted on the device
    }
    if (ctx->graph_K > 0) {
      const long long full = S / ctx->graph_K;
      for (long long r = 0; r < full; ++r) {
        CK(cudaGraphLaunch(ctx->graph_full, ctx->stream));
        ctx->launches += graph_launches(ctx->graph_K, ctx->params.mode, ctx->precision);
      }
    }
    if (ctx->graph_rem_K) {
      CK(cudaGraphLaunch(ctx->graph_rem, ctx->stream));
      ctx->launches += graph_launches(ctx->graph_rem_K, ctx->params.mode, ctx->precision);
    }
    // finish the last step (s = S), then the energy at the final positions
    if (ctx->precision == MDGP_PREC_FP32) enqueue_step_fused(ctx, 0, false);
    else enqueue_step_integrate(ctx, 0, false);
    enqueue_force(ctx, true, 0);
  }
  enqueue_energy(ctx, kAccE1);
  k_finalize<<<grid_for(ctx->n_el, 128), 128, 0, ctx->stream>>>(ctx->B, (mdgp_result*)ctx->d_results.ptr);
  ctx->launches++;
  CK(cudaGetLastError());
  ctx->ran = true;
  return MDGP_OK;
}

static int results_impl(mdgp_ctx* ctx, mdgp_result* out, int64_t n) {
  if (!ctx->planned) return MDGP_E_STATE;
  if (n != ctx->n_el || !out) return MDGP_E_ARG;
  int flags[16];   // the counters; the barrier words are not needed here
  CK(cudaMemcpyAsync(out, ctx->d_results.ptr, sizeof(mdgp_result) * n, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(flags, ctx->B.flags, sizeof(flags), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  // every rebuild is rebuild_kernels() launches; the launch sequence counted one eagerly
  ctx->rebuilds = flags[2];
  ctx->launches_with_rebuilds = ctx->launches + (long long)rebuild_kernels(ctx) * (flags[2] - 1) + flags[3];
  return MDGP_OK;
}

static int export_impl(mdgp_ctx* ctx, int what, std::vector<double>& buf) {
  const size_t N = (size_t)ctx->n_atoms;
  enqueue_export(ctx, what);
  CK(cudaGetLastError());
  buf.resize(6 * N);
  CK(cudaMemcpyAsync(buf.data(), ctx->B.out, sizeof(double) * 6 * N, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return MDGP_OK;
}

// ---------------------------------------------------------------------------
// C ABI.
// ---------------------------------------------------------------------------
extern "C" {

int mdgp_md_params_default(mdgp_md_params* out) {
  if (!out) return MDGP_E_ARG;
  std::memset(out, 0, sizeof(*out));
  out->dt = 0.005;
  out->rc = 2.5;
  out->k_tether = 150.0;
  out->gamma_wall = 1.0;
  out->wall_density = 1.0;
  out->eps_wf = 1.0; out->sig_wf = 1.0;
  out->eps_ww = 1.0; out->sig_ww = 1.0;
  out->fluid_margin = 0.7;
  out->tau_T = 0.5;
  out->mass = 1.0;
  out->n_blocks = 10;
  out->mode = 0;
  out->wall_planes = 3;
  out->list_capacity = 128;
  out->skin = 0.4;
  out->rebuild_every = 0;
  out->build_variant = 3;
  out->persistent = 1;
  out->wait_timeout_ms = 2000;
  out->inject_barrier_skip = 0;
  out->threads_per_atom = 0;
  out->resident = 1;
  return MDGP_OK;
}

int mdgp_create(mdgp_ctx** out, int device, int precision) {
  if (!out || (precision != MDGP_PREC_FP64 && precision != MDGP_PREC_FP32)) return MDGP_E_ARG;
  *out = nullptr;
  mdgp_ctx* ctx = new (std::nothrow) mdgp_ctx();
  if (!ctx) return MDGP_E_NOMEM;
  ctx->device = device;
  ctx->precision = precision;
  mdgp_md_params_default(&ctx->params);
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->side_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->side_stream2, cudaStreamNonBlocking);
  int prio_low = 0, prio_high = 0;
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
  if (e == cudaSuccess)
    e = cudaStreamCreateWithPriority(&ctx->fact_stream[0], cudaStreamNonBlocking, prio_high);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&ctx->fact_stream[1], cudaStreamNonBlocking, prio_low);
  for (int k = 0; k < 4 && e == cudaSuccess; ++k)
    e = cudaEventCreateWithFlags(&ctx->fact_event[k], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    mdgp_destroy(ctx);
    return MDGP_E_CUDA;
  }
  ctx->stream = ctx->own_stream;
  *out = ctx;
  return MDGP_OK;
}

int mdgp_destroy(mdgp_ctx* ctx) {
  if (!ctx) return MDGP_E_ARG;
  cudaSetDevice(ctx->device);
  drop_graphs(ctx);
  for (DevBuf* b : ctx->all_bufs()) if (b->ptr) cudaFree(b->ptr);
  ctx->release_extra();
  if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
  if (ctx->side_stream) cudaStreamDestroy(ctx->side_stream);
  if (ctx->side_stream2) cudaStreamDestroy(ctx->side_stream2);
  for (cudaStream_t fs : ctx->fact_stream) if (fs) cudaStreamDestroy(fs);
  for (cudaEvent_t fe : ctx->fact_event) if (fe) cudaEventDestroy(fe);
  for (cudaEvent_t de : ctx->dir_ev) if (de) cudaEventDestroy(de);
  delete ctx;
  return MDGP_OK;
}

static bool params_valid(const mdgp_md_params* p) {
  return p->dt > 0 && p->rc > 0 && p->n_blocks >= 1 && p->wall_planes >= 1 && p->mass > 0 &&
         p->wall_density > 0 && p->gamma_wall >= 0 && p->list_capacity >= 0 && p->skin >= 0 &&
         p->rebuild_every >= 0 && (p->build_variant == 0 || p->build_variant == 3) && p->persistent >= 0 &&
         p->persistent <= 2 && (p->threads_per_atom == 0 || p->threads_per_atom == 1 || p->threads_per_atom == 2 ||
                                p->threads_per_atom == 4 || p->threads_per_atom == 8) &&
         (p->resident == 0 || p->resident == 1);
}

int mdgp_set_md_params(mdgp_ctx* ctx, const mdgp_md_params* p) {
  if (!ctx || !p) return MDGP_E_ARG;
  if (!params_valid(p)) return MDGP_E_ARG;
  ctx->params = *p;
  ctx->planned = false;
  return MDGP_OK;
}

int mdgp_set_stream(mdgp_ctx* ctx, void* stream) {
  if (!ctx) return MDGP_E_ARG;
  ctx->stream = stream ? (cudaStream_t)stream : ctx->own_stream;
  ctx->planned = false;
  return MDGP_OK;
}

int mdgp_micro_plan(mdgp_ctx* ctx, const mdgp_element* el, int64_t n, int64_t* n_atoms) {
  if (!ctx || !el || n < 1) return MDGP_E_ARG;
  cudaSetDevice(ctx->device);
  int st = plan_impl(ctx, el, n, 0);
  if (st == MDGP_OK && n_atoms) *n_atoms = ctx->n_atoms;
  return st;
}

int mdgp_micro_plan_from(mdgp_ctx* ctx, const mdgp_element* el, int64_t n, const mdgp_start* starts,
                         int64_t* n_atoms) {
  if (!ctx || !el || n < 1) return MDGP_E_ARG;
  cudaSetDevice(ctx->device);
  int st = plan_impl(ctx, el, n, 0, starts);
  if (st == MDGP_OK && n_atoms) *n_atoms = ctx->n_atoms;
  return st;
}

int mdgp_start_state(const mdgp_md_params* params, const mdgp_element* el, const mdgp_start* start, double* xv,
                     int64_t cap, int64_t* n_rows, int32_t* kind) {
  if (!el || !start || !n_rows || !kind) return MDGP_E_ARG;
  mdgp_md_params p;
  if (params) p = *params;
  else mdgp_md_params_default(&p);
  if (!params_valid(&p)) return MDGP_E_ARG;
  ElemDev E;
  std::string why;
  const int st = describe(p, *el, E, &why);
  if (st) return st;
  *n_rows = (int64_t)E.nf + E.nw;
  if (!xv) return MDGP_OK;
  if (cap < *n_rows) return MDGP_E_ARG;
  std::vector<double> out;
  *kind = start->xv ? adapt_snapshot(p, *el, E, *start, out) : 0;
  if (*kind) std::copy(out.begin(), out.end(), xv);
  return MDGP_OK;
}

int mdgp_micro_launch(mdgp_ctx* ctx) {
  if (!ctx) return MDGP_E_ARG;
  cudaSetDevice(ctx->device);
  return launch_impl(ctx);
}

int mdgp_micro_results(mdgp_ctx* ctx, mdgp_result* out, int64_t n) {
  if (!ctx) return MDGP_E_ARG;
  cudaSetDevice(ctx->device);
  return results_impl(ctx, out, n);
}

int64_t mdgp_micro_launch_count(const mdgp_ctx* ctx) { return ctx ? ctx->launches_with_rebuilds : -1; }

int mdgp_micro_path(const mdgp_ctx* ctx) {
  if (!ctx) return MDGP_E_ARG;
  if (!ctx->planned) return MDGP_E_STATE;
  return ctx->direct ? 2 : (ctx->graph_while ? 1 : 0);
}

int mdgp_micro_continue(mdgp_ctx* ctx, const double* g_ext, const double* dpdx) {
  if (!ctx) return MDGP_E_ARG;
  if (!ctx->planned || !ctx->ran) return MDGP_E_STATE;
  cudaSetDevice(ctx->device);
  const unsigned S = (unsigned)ctx->steps;
  for (size_t e = 0; e < ctx->el_host.size(); ++e) {
    ElemDev& E = ctx->el_host[e];
    mdgp_element& d = ctx->el_desc[e];
    if (g_ext) d.g_ext = g_ext[e];
    if (dpdx) d.dpdx = dpdx[e];
    // Eq. momentumEq with the element's density as described
    E.g = d.density > 0.0 ? d.g_ext - d.dpdx / d.density : d.g_ext;
    E.g_kick = (float)(0.5 * ctx->params.dt / ctx->params.mass * E.g);
    E.step0 += S;
  }
  CK(cudaMemcpyAsync(ctx->d_el.ptr, ctx->el_host.data(), sizeof(ElemDev) * ctx->el_host.size(),
                     cudaMemcpyHostToDevice, ctx->stream));
  return launch_impl(ctx, true);
}

int mdgp_micro_launch_shape(const mdgp_ctx* ctx, int32_t* out) {
  if (!ctx || !out) return MDGP_E_ARG;
  if (!ctx->planned || !(ctx->direct || ctx->graph_while)) return MDGP_E_STATE;
  out[0] = (int32_t)ctx->persist_grid;
  out[1] = ctx->persist_threads;
  out[2] = ctx->persist_atoms;
  out[3] = ctx->persist_tpa;
  out[4] = ctx->persist_resident ? 1 : 0;
  return MDGP_OK;
}

int64_t mdgp_micro_rebuild_count(const mdgp_ctx* ctx) { return ctx ? ctx->rebuilds : -1; }

int mdgp_micro_batch(mdgp_ctx* ctx, const mdgp_element* el, int64_t n, mdgp_result* out) {
  if (!ctx || !el || !out || n < 1) return MDGP_E_ARG;
  cudaSetDevice(ctx->device);
  // group elements by total step count; each group is one plan
  std::map<long long, std::vector<int64_t>> groups;
  for (int64_t i = 0; i < n; ++i) groups[el[i].steps_eq + el[i].steps_sample].push_back(i);
  for (auto& kv : groups) {
    std::vector<mdgp_element> sub;
    for (int64_t i : kv.second) sub.push_back(el[i]);
    std::vector<mdgp_result> res(sub.size());
    int cap = 0;
    for (int attempt = 0; attempt < 3; ++attempt) {
      int st = plan_impl(ctx, sub.data(), (int64_t)sub.size(), cap);
      if (!st) st = launch_impl(ctx);
      if (!st) st = results_impl(ctx, res.data(), (int64_t)sub.size());
      if (st) return st;
      bool overflow = false;
      for (auto& r : res) overflow |= r.status == MDGP_E_OVERFLOW;
      if (!overflow) break;
      cap = 2 * ctx->B.list_cap;  // longer neighbour lists and run again
    }
    for (size_t j = 0; j < sub.size(); ++j) out[kv.second[j]] = res[j];
  }
  return MDGP_OK;
}

int mdgp_micro_state(mdgp_ctx* ctx, double* x, double* v, int64_t n_atoms) {
  if (!ctx) return MDGP_E_ARG;
  if (!ctx->planned) return MDGP_E_STATE;
  if (n_atoms != ctx->n_atoms) return MDGP_E_ARG;
  cudaSetDevice(ctx->device);
  std::vector<double> buf;
  int st = export_impl(ctx, 0, buf);
  if (st) return st;
  for (int64_t i = 0; i < n_atoms; ++i)
    for (int d = 0; d < 3; ++d) {
      if (x) x[3 * i + d] = buf[(size_t)d * n_atoms + i];
      if (v) v[3 * i + d] = buf[(size_t)(3 + d) * n_atoms + i];
    }
  return MDGP_OK;
}

int mdgp_md_forces(mdgp_ctx* ctx, const mdgp_element* el, const double* x, int64_t n_atoms, double* f,
                   double* wxx, double* epot) {
  if (!ctx || !el || !x) return MDGP_E_ARG;
  cudaSetDevice(ctx->device);
  mdgp_element e1 = *el;
  e1.steps_eq = 0;
  e1.steps_sample = 0;
  int st = plan_impl(ctx, &e1, 1, 0);
  if (st) return st;
  if (n_atoms != ctx->n_atoms) return MDGP_E_ARG;
  if ((st = start_batch(ctx))) return st;
  // replace the lattice positions by the caller's (absolute, original order;
  // the freshly built element is still in original order)
  // (double-float state with FP32 pair forces: each value as the float pair
  // hi = fl(x), lo = fl(x - hi) in the same 8 bytes)
  std::vector<double> soa((size_t)3 * n_atoms);
  for (int64_t i = 0; i < n_atoms; ++i)
    for (int d = 0; d < 3; ++d) {
      const double v = x[3 * i + d];
      if (ctx->precision == MDGP_PREC_FP32) {
        const float pair[2] = {(float)v, (float)(v - (double)(float)v)};
        std::memcpy(&soa[(size_t)d * n_atoms + i], pair, sizeof(pair));
      } else {
        soa[(size_t)d * n_atoms + i] = v;
      }
    }
  for (int d = 0; d < 3; ++d)
    CK(cudaMemcpyAsync(ctx->B.st[d], soa.data() + (size_t)d * n_atoms, sizeof(double) * n_atoms,
                       cudaMemcpyHostToDevice, ctx->stream));
  enqueue_rebuild(ctx);
  enqueue_force(ctx, true, 0);
  std::vector<double> buf;
  if ((st = export_impl(ctx, 1, buf))) return st;
  int status = 0;
  CK(cudaMemcpy(&status, ctx->d_status.ptr, sizeof(int), cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < n_atoms; ++i) {
    if (f) for (int d = 0; d < 3; ++d) f[3 * i + d] = buf[(size_t)d * n_atoms + i];
    if (wxx) wxx[i] = buf[(size_t)3 * n_atoms + i];
    if (epot) epot[i] = buf[(size_t)4 * n_atoms + i];
  }
  return status ? status : MDGP_OK;
}

int mdgp_micro_direct_timing(const mdgp_ctx* ctx, double* out) {
  if (!ctx || !out) return MDGP_E_ARG;
  if (!ctx->planned || !ctx->direct) return MDGP_E_STATE;
  out[0] = ctx->dir_kernel_ms;
  out[1] = (double)ctx->dir_steps;
  out[2] = (double)ctx->dir_launches;
  out[3] = ctx->dir_rebuild_ms;
  out[4] = (double)ctx->dir_rebuilds;
  return MDGP_OK;
}

int mdgp_micro_profile(mdgp_ctx* ctx, int64_t steps, double* ms) {
  if (!ctx || !ms || steps < 1) return MDGP_E_ARG;
  if (!ctx->planned) return MDGP_E_STATE;
  if (steps > ctx->steps) steps = ctx->steps;
  cudaSetDevice(ctx->device);
  int st;
  if ((st = start_batch(ctx))) return st;
  enqueue_rebuild(ctx);
  const bool fused = ctx->precision == MDGP_PREC_FP32;
  if (!fused) enqueue_force(ctx, false, 0);
  std::vector<cudaEvent_t> ev((size_t)(3 * steps + 1));
  for (auto& e : ev) CK(cudaEventCreate(&e));
  CK(cudaEventRecord(ev[0], ctx->stream));
  for (int64_t k = 0; k < steps; ++k) {
    // the step counter stays 0: launch k works on step k.  FP32: the fused
    // step (forces + integration), then the rebuild; FP64: integration,
    // rebuild, forces of the next step.
    if (fused) enqueue_step_fused(ctx, (int)k, true);
    else enqueue_step_integrate(ctx, (int)k, true);
    CK(cudaEventRecord(ev[3 * k + 1], ctx->stream));
    if (k % ctx->rebuild_every == 0) enqueue_rebuild(ctx);
    CK(cudaEventRecord(ev[3 * k + 2], ctx->stream));
    if (!fused) enqueue_force(ctx, false, (int)k + 1);
    CK(cudaEventRecord(ev[3 * k + 3], ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  double t_int = 0.0, t_reb = 0.0, t_force = 0.0;
  long long nreb = 0;
  for (int64_t k = 0; k < steps; ++k) {
    float a = 0.f, b = 0.f, c = 0.f;
    cudaEventElapsedTime(&a, ev[3 * k], ev[3 * k + 1]);
    cudaEventElapsedTime(&b, ev[3 * k + 1], ev[3 * k + 2]);
    cudaEventElapsedTime(&c, ev[3 * k + 2], ev[3 * k + 3]);
    t_int += a;
    t_force += c;
    if (k % ctx->rebuild_every == 0) { t_reb += b; ++nreb; }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (fused) {
    ms[0] = 0.0;
    ms[1] = t_int / steps;
  } else {
    ms[0] = t_int / steps;
    ms[1] = t_force / steps;
  }
  ms[2] = nreb ? t_reb / nreb : 0.0;
  ms[3] = (double)ctx->n_atoms;
  ms[4] = (double)ctx->B.n_cells;
  ms[5] = (double)ctx->rebuild_every;
  return MDGP_OK;
}

int mdgp_autotune(mdgp_ctx* ctx, const mdgp_element* el, int64_t n, int64_t probe_steps, mdgp_md_params* best,
                  double* best_rate) {
  if (!ctx || !el || n < 1 || probe_steps < 1) return MDGP_E_ARG;
  cudaSetDevice(ctx->device);
  const mdgp_md_params base = ctx->params;
  std::vector<mdgp_element> probe(el, el + n);
  for (auto& e : probe) { e.steps_eq = probe_steps; e.steps_sample = 0; }
  const double skins[] = {0.3, 0.4, 0.5, 0.6};
  double top = -1.0;
  mdgp_md_params chosen = base;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  for (double skin : skins) {
    mdgp_md_params trial = base;
    trial.skin = skin;
    ctx->params = trial;
    int st = plan_impl(ctx, probe.data(), n, 0);
    if (st == MDGP_E_ARG) continue;       // geometry too small for this skin
    if (st) { ctx->params = base; return st; }
    if ((st = launch_impl(ctx))) { ctx->params = base; return st; }   // warm-up
    CK(cudaEventRecord(e0, ctx->stream));
    if ((st = launch_impl(ctx))) { ctx->params = base; return st; }
    CK(cudaEventRecord(e1, ctx->stream));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    const double rate = (double)ctx->n_atoms * (double)probe_steps / (ms * 1e-3);
    if (rate > top) { top = rate; chosen = trial; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->params = top > 0 ? chosen : base;
  ctx->planned = false;
  if (best) *best = ctx->params;
  if (best_rate) *best_rate = top;
  return top > 0 ? MDGP_OK : MDGP_E_ARG;
}

const char* mdgp_last_error(const mdgp_ctx* ctx) { return ctx ? ctx->err : "null context"; }

}  // extern "C"
