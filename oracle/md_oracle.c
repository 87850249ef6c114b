/*
 * md_oracle.c -- plain, slow, double-precision reference for one LJ micro-element.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link or call this
 * file; only tests/, the smoke check and the CPU-baseline leg of bench.py use it.
 * It shares no code, header or table with the CUDA library.
 *
 * What it computes (paper: Stephenson, Kermode & Lockerby, arXiv:1603.04628):
 *   - App. A: a fluid slab of Lennard-Jones atoms (Eq. LJ, truncated at r_c),
 *     periodic in the streamwise (x) and spanwise (z) directions, integrated by
 *     velocity Verlet;
 *   - Sec. 2.1, Eq. momentumEq: every fluid atom feels the body force F that
 *     stands for the local pressure gradient;
 *   - Sec. 2.1, Eq. continuityEq: the element returns the time-averaged mass
 *     flow rate q = (m / L_x) * sum_fluid v_x, and Sec. 2.2 / 2.3 footnote the
 *     cross-section averaged pressure (here P_xx from the virial);
 *   - Sec. 2.3: the standard error of the mean output from the raw
 *     time-instantaneous samples (block averaging);
 *   - Sec. 3 (the full MD the hybrid is judged against): with wall_amp > 0
 *     the walls follow the converging-diverging profile h(x) of the channel
 *     (the benchmark's form of the paper's channel shape), so that one
 *     element of length L is a whole periodic channel.
 * Readings where the paper is silent (tethered FCC walls, G-JF Langevin
 * thermostat on wall atoms, lattice layout, block count) are listed in the
 * design notes and restated at each function below.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11), written
 * here from its published definition; Box-Muller turns pairs of uniforms into
 * normals.
 *
 * Everything is double precision; the build uses -ffp-contract=off so that no
 * fused multiply-adds are introduced.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXB 64

/* ------------------------------------------------------------------------ */
/* Parameters of one element plus the shared physics constants.             */
/* ------------------------------------------------------------------------ */
typedef struct {
  /* element (reduced LJ units: eps = sigma = m = 1) */
  double h;          /* distance between the innermost wall planes */
  double Lx, Lz;     /* periodic box lengths */
  double density;    /* fluid number density */
  double T;          /* target temperature */
  double g;          /* total body force on each fluid atom, along x (Eq. momentumEq) */
  /* physics */
  double dt, rc;
  double k_tether;   /* wall spring constant; walls frozen when mode == 1 */
  double gamma_wall; /* Langevin friction on wall atoms (G-JF) */
  double wall_density;
  double eps_wf, sig_wf;  /* wall-fluid LJ pair */
  double eps_ww, sig_ww;  /* wall-wall LJ pair (tethered walls only) */
  double fluid_margin;    /* lattice gap between wall plane and first fluid layer */
  double tau_T;           /* Berendsen time constant (mode 1) */
  double mass;
  int64_t steps_eq, steps_sample;
  uint64_t seed;
  int32_t elem_id;
  int32_t n_blocks;
  int32_t mode;       /* 0: tethered walls + Langevin walls; 1: frozen walls + Berendsen on fluid v_z;
                         2: bulk test box (no walls, periodic in y with L_y = h) */
  int32_t wall_planes;
  double wall_amp;    /* walls following h(x) = h (1 - wall_amp cos(2 pi x / Lx)) about the
                         mid-plane of the widest gap H = h (1 + wall_amp); 0: planar walls */
} or_params;

typedef struct {
  double q_block[OR_MAXB];   /* sum over samples in block b of q_inst */
  double p_block[OR_MAXB];   /* sum over samples in block b of P_xx,inst */
  int64_t n_block[OR_MAXB];
  double T_sum;              /* sum over samples of fluid kinetic temperature */
  int64_t n_samples;
  double e_first, e_last;    /* total energy before the first and after the last step */
  int32_t status;
} or_accum;

typedef struct {
  double q, q_se, p, p_se, T_meas, e_drift;
  int64_t n_fluid, n_wall;
  int32_t status;
} or_result;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11): ten rounds of two 32x32->64 multiplies, key bumped  */
/* by the Weyl constants between rounds.                                     */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    if (round < 9) { k0 += W0; k1 += W1; }
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in the open interval (0, 1) from 32 random bits. */
static double or_u01(uint32_t r) { return ((double)r + 0.5) * (1.0 / 4294967296.0); }

/* Four standard normals from one Philox block: Box-Muller on (u0,u1), (u2,u3). */
void or_normals4(uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint64_t seed, double out[4]) {
  uint32_t ctr[4] = {a, b, c, d};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t r[4];
  or_philox4x32_10(ctr, key, r);
  const double two_pi = 6.283185307179586476925286766559;
  for (int k = 0; k < 2; ++k) {
    double u1 = or_u01(r[2 * k]), u2 = or_u01(r[2 * k + 1]);
    double rad = sqrt(-2.0 * log(u1));
    out[2 * k] = rad * cos(two_pi * u2);
    out[2 * k + 1] = rad * sin(two_pi * u2);
  }
}

/* Philox counter streams: word 3 of the counter names the use. */
#define OR_STREAM_INIT 0u
#define OR_STREAM_LANGEVIN 1u

/* ------------------------------------------------------------------------ */
/* Element geometry (reading: the paper gives only "fluid atoms in a         */
/* lattice" and FCC walls; layout restated in the design notes).             */
/* ------------------------------------------------------------------------ */
static long or_lround(double x) { return (long)floor(x + 0.5); }

static void or_wall_cells(const or_params* P, long* nx, long* nz, double* a0) {
  *a0 = cbrt(4.0 / P->wall_density);
  long cx = or_lround(P->Lx / *a0), cz = or_lround(P->Lz / *a0);
  *nx = cx < 1 ? 1 : cx;
  *nz = cz < 1 ? 1 : cz;
}

int64_t or_n_fluid(const or_params* P) {
  return (int64_t)or_lround(P->density * P->Lx * P->h * P->Lz);
}

int64_t or_n_wall(const or_params* P) {
  if (P->mode == 2) return 0;
  long nx, nz; double a0;
  or_wall_cells(P, &nx, &nz, &a0);
  return (int64_t)2 * P->wall_planes * 2 * nx * nz;
}

/* The widest gap between the walls: h for planar walls, h (1 + wall_amp)
 * for walls that follow the profile (the box is built for it). */
static double or_gap_max(const or_params* P) { return P->h * (1.0 + P->wall_amp); }

/* Fluid FCC lattice cell counts: spacing near (4/n)^(1/3), enough sites. */
static void or_fluid_cells(const or_params* P, int64_t nf, long* cx, long* cy, long* cz, double* y0, double* ly) {
  double af = cbrt(4.0 / P->density);
  if (P->mode == 2) { *y0 = 0.0; *ly = P->h; }
  else { *y0 = P->fluid_margin; *ly = or_gap_max(P) - 2.0 * P->fluid_margin; }
  *cx = (long)ceil(P->Lx / af - 1e-9);
  *cy = (long)ceil(*ly / af - 1e-9);
  *cz = (long)ceil(P->Lz / af - 1e-9);
  if (*cx < 1) *cx = 1;
  if (*cy < 1) *cy = 1;
  if (*cz < 1) *cz = 1;
  int turn = 0;
  while ((int64_t)4 * (*cx) * (*cy) * (*cz) < nf) {
    if (turn % 3 == 0) ++(*cy); else if (turn % 3 == 1) ++(*cx); else ++(*cz);
    ++turn;
  }
}

/* Build positions, anchors and species (0 fluid, 1 wall) and Maxwell-Boltzmann
 * velocities.  Atom order: fluid atoms first, then the bottom wall planes
 * (k = 0, 1, 2 going outwards), then the top wall planes. */
/* Walls that follow the profile (wall_amp > 0): the local gap at x and the
 * height of the lower wall's inner plane, yb(x) = (H - h(x)) / 2, so that
 * both walls are symmetric about the mid-plane of the widest gap H. */
static void or_profile(const or_params* P, double x, double* hx, double* yb) {
  *hx = P->h * (1.0 - P->wall_amp * cos(2.0 * M_PI * x / P->Lx));
  *yb = 0.5 * (or_gap_max(P) - *hx);
}

static const double or_basis[4][3] = {{0, 0, 0}, {0.5, 0.5, 0}, {0.5, 0, 0.5}, {0, 0.5, 0.5}};

/* Fluid of a profiled element: the FCC lattice of the widest gap, its sites
 * taken in lattice order and kept where they lie at least the fluid margin
 * inside the local walls; the lattice grows (y, x, z in turn) until enough
 * sites are kept, and the vacancies are spread evenly over the kept sites. */
static int or_init_fluid_profiled(const or_params* P, int64_t nf, double* x) {
  long cx, cy, cz; double y0, ly;
  or_fluid_cells(P, nf, &cx, &cy, &cz, &y0, &ly);
  double m = P->fluid_margin;
  for (int turn = 0;; ++turn) {
    double bx = P->Lx / cx, by = ly / cy, bz = P->Lz / cz;
    int64_t sites = (int64_t)4 * cx * cy * cz, kept = 0;
    double* pos = (double*)malloc(sizeof(double) * 3 * (size_t)sites);
    if (!pos) return -1;
    for (int64_t s = 0; s < sites; ++s) {
      int64_t b = s % 4, c = s / 4;
      int64_t iz = c % cz, iy = (c / cz) % cy, ix = c / (cz * cy);
      double px = (ix + or_basis[b][0] + 0.25) * bx;
      double py = y0 + (iy + or_basis[b][1] + 0.25) * by;
      double pz = (iz + or_basis[b][2] + 0.25) * bz;
      double hx, yb;
      or_profile(P, px, &hx, &yb);
      if (py >= yb + m && py <= yb + hx - m) {
        pos[3 * kept] = px; pos[3 * kept + 1] = py; pos[3 * kept + 2] = pz;
        ++kept;
      }
    }
    if (kept >= nf) {
      for (int64_t i = 0; i < nf; ++i) {
        int64_t k = (int64_t)(((__int128)i * kept) / nf);
        for (int d = 0; d < 3; ++d) x[3 * i + d] = pos[3 * k + d];
      }
      free(pos);
      return 0;
    }
    free(pos);
    if (turn % 3 == 0) ++cy; else if (turn % 3 == 1) ++cx; else ++cz;
  }
}

int or_init(const or_params* P, double* x, double* v, double* anchor, int32_t* sp) {
  int64_t nf = or_n_fluid(P), nw = or_n_wall(P), n = nf + nw;
  long cx, cy, cz; double y0, ly;
  or_fluid_cells(P, nf, &cx, &cy, &cz, &y0, &ly);
  double bx = P->Lx / cx, by = ly / cy, bz = P->Lz / cz;
  const double (*basis)[3] = or_basis;
  int64_t sites = (int64_t)4 * cx * cy * cz;
  if (P->wall_amp > 0.0 && P->mode != 2) {
    if (or_init_fluid_profiled(P, nf, x)) return -1;
    for (int64_t i = 0; i < nf; ++i) sp[i] = 0;
  }
  for (int64_t i = 0; i < nf && !(P->wall_amp > 0.0 && P->mode != 2); ++i) {
    /* spread the vacancies evenly over the lattice */
    int64_t s = (int64_t)(((__int128)i * sites) / nf);
    int64_t b = s % 4, c = s / 4;
    int64_t iz = c % cz, iy = (c / cz) % cy, ix = c / (cz * cy);
    x[3 * i + 0] = (ix + basis[b][0] + 0.25) * bx;
    x[3 * i + 1] = y0 + (iy + basis[b][1] + 0.25) * by;
    x[3 * i + 2] = (iz + basis[b][2] + 0.25) * bz;
    sp[i] = 0;
  }
  if (nw > 0) {
    long nx, nz; double a0;
    or_wall_cells(P, &nx, &nz, &a0);
    double ax = P->Lx / nx, az = P->Lz / nz, dy = 0.5 * a0;
    int64_t a = nf;
    for (int wall = 0; wall < 2; ++wall) {
      for (int k = 0; k < P->wall_planes; ++k) {
        double y = wall == 0 ? -k * dy : P->h + k * dy;
        for (long i = 0; i < nx; ++i)
          for (long j = 0; j < nz; ++j)
            for (int t = 0; t < 2; ++t) {
              double ox, oz;
              if (k % 2 == 0) { ox = t ? 0.5 : 0.0; oz = t ? 0.5 : 0.0; }
              else { ox = t ? 0.0 : 0.5; oz = t ? 0.5 : 0.0; }
              x[3 * a + 0] = (i + ox) * ax;
              x[3 * a + 1] = y;
              if (P->wall_amp > 0.0) {
                /* the planes follow the local inner wall: yb(x) - k dy and yb(x) + h(x) + k dy */
                double hx, yb;
                or_profile(P, x[3 * a + 0], &hx, &yb);
                x[3 * a + 1] = wall == 0 ? yb - k * dy : yb + hx + k * dy;
              }
              x[3 * a + 2] = (j + oz) * az;
              sp[a] = 1;
              ++a;
            }
      }
    }
  }
  for (int64_t i = 0; i < n; ++i)
    for (int d = 0; d < 3; ++d) anchor[3 * i + d] = x[3 * i + d];
  /* velocities: N(0, T/m) per component from the init stream */
  double sd = sqrt(P->T / P->mass);
  for (int64_t i = 0; i < n; ++i) {
    double z[4];
    or_normals4((uint32_t)i, 0u, (uint32_t)P->elem_id, OR_STREAM_INIT, P->seed, z);
    for (int d = 0; d < 3; ++d) v[3 * i + d] = sd * z[d];
  }
  /* per group: remove the mean velocity, then rescale to exactly T with
   * 3(N_g - 1) degrees of freedom; frozen walls (mode 1) get zero velocity */
  for (int grp = 0; grp < 2; ++grp) {
    int64_t lo = grp == 0 ? 0 : nf, hi = grp == 0 ? nf : n, cnt = hi - lo;
    if (cnt <= 0) continue;
    if (grp == 1 && P->mode == 1) {
      for (int64_t i = lo; i < hi; ++i) v[3 * i] = v[3 * i + 1] = v[3 * i + 2] = 0.0;
      continue;
    }
    double mean[3] = {0, 0, 0};
    for (int64_t i = lo; i < hi; ++i)
      for (int d = 0; d < 3; ++d) mean[d] += v[3 * i + d];
    for (int d = 0; d < 3; ++d) mean[d] /= (double)cnt;
    double ke2 = 0.0;
    for (int64_t i = lo; i < hi; ++i)
      for (int d = 0; d < 3; ++d) {
        v[3 * i + d] -= mean[d];
        ke2 += P->mass * v[3 * i + d] * v[3 * i + d];
      }
    if (cnt > 1 && ke2 > 0.0) {
      double Tg = ke2 / (3.0 * (double)(cnt - 1));
      double s = sqrt(P->T / Tg);
      for (int64_t i = lo; i < hi; ++i)
        for (int d = 0; d < 3; ++d) v[3 * i + d] *= s;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Pair interaction, Eq. LJ: U = 4 eps [(s/r)^12 - (s/r)^6].                 */
/* Reading of "shifted": energy shifted so U(r_c) = 0, force left unchanged. */
/* Returns the scalar F(r)/r so that F_vec = (F/r) * r_vec.                  */
/* ------------------------------------------------------------------------ */
double or_lj_energy(double r, double eps, double sig) {
  double sr6 = pow(sig / r, 6.0);
  return 4.0 * eps * (sr6 * sr6 - sr6);
}

double or_lj_force(double r, double eps, double sig) {
  /* F(r) = -dU/dr = (24 eps / r) [2 (s/r)^12 - (s/r)^6] */
  double sr6 = pow(sig / r, 6.0);
  return 24.0 * eps * (2.0 * sr6 * sr6 - sr6) / r;
}

static void or_pair_params(const or_params* P, int si, int sj, double* eps, double* sig) {
  if (si == 0 && sj == 0) { *eps = 1.0; *sig = 1.0; }
  else if (si == 1 && sj == 1) { *eps = P->eps_ww; *sig = P->sig_ww; }
  else { *eps = P->eps_wf; *sig = P->sig_wf; }
}

/* Do atoms of these species interact?  Frozen walls (mode 1) do not
 * interact with each other. */
static int or_pair_active(const or_params* P, int si, int sj) {
  if (si == 1 && sj == 1 && P->mode == 1) return 0;
  return 1;
}

static double or_min_image(double d, double L) { return d - L * floor(d / L + 0.5); }

/* Accumulate one pair (i < j): force, per-atom x-virial share and energy. */
static void or_add_pair(const or_params* P, int64_t i, int64_t j, const double* d, double r2,
                        const int32_t* sp, double* f, double* wxx, double* epot) {
  double eps, sig;
  or_pair_params(P, sp[i], sp[j], &eps, &sig);
  double r = sqrt(r2);
  double fr = or_lj_force(r, eps, sig) / r;
  for (int k = 0; k < 3; ++k) {
    f[3 * i + k] += fr * d[k];
    f[3 * j + k] -= fr * d[k];
  }
  /* pair virial x_ij * F_x,ij, split half to each atom */
  double w = 0.5 * d[0] * fr * d[0];
  wxx[i] += w;
  wxx[j] += w;
  double u = or_lj_energy(r, eps, sig) - or_lj_energy(P->rc, eps, sig);
  epot[i] += 0.5 * u;
  epot[j] += 0.5 * u;
}

/* All-pairs O(N^2) LJ forces with minimum image in x and z (and y in the bulk
 * test box).  Outputs are overwritten. */
void or_lj_brute(const or_params* P, int64_t n, const double* x, const int32_t* sp,
                 double* f, double* wxx, double* epot) {
  memset(f, 0, sizeof(double) * 3 * n);
  memset(wxx, 0, sizeof(double) * n);
  memset(epot, 0, sizeof(double) * n);
  double rc2 = P->rc * P->rc;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j) {
      if (!or_pair_active(P, sp[i], sp[j])) continue;
      double d[3] = {x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1], x[3 * i + 2] - x[3 * j + 2]};
      d[0] = or_min_image(d[0], P->Lx);
      d[2] = or_min_image(d[2], P->Lz);
      if (P->mode == 2) d[1] = or_min_image(d[1], P->h);
      double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      if (r2 < rc2) or_add_pair(P, i, j, d, r2, sp, f, wxx, epot);
    }
}

/* Linked-cell LJ forces: cells of side >= r_c; x and z periodic; in y the
 * cell range covers the walls and atoms beyond it fall into the edge cells
 * (periodic in the bulk test box).  Same outputs as or_lj_brute. */
void or_lj_cells(const or_params* P, int64_t n, const double* x, const int32_t* sp,
                 double* f, double* wxx, double* epot) {
  memset(f, 0, sizeof(double) * 3 * n);
  memset(wxx, 0, sizeof(double) * n);
  memset(epot, 0, sizeof(double) * n);
  double rc2 = P->rc * P->rc;
  double ylo, yhi;
  int ybulk = P->mode == 2;
  if (ybulk) { ylo = 0.0; yhi = P->h; }
  else {
    long nx, nz; double a0;
    or_wall_cells(P, &nx, &nz, &a0);
    double th = 0.5 * a0 * (P->wall_planes - 1);
    ylo = -th - 1.0; yhi = or_gap_max(P) + th + 1.0;
  }
  long ncx = (long)floor(P->Lx / P->rc), ncz = (long)floor(P->Lz / P->rc);
  long ncy = (long)floor((yhi - ylo) / P->rc);
  if (ncy < 1) ncy = 1;
  if (ncx < 3 || ncz < 3 || (ybulk && ncy < 3)) {  /* stencil needs >= 3 cells per periodic axis */
    or_lj_brute(P, n, x, sp, f, wxx, epot);
    return;
  }
  double csx = P->Lx / ncx, csy = (yhi - ylo) / ncy, csz = P->Lz / ncz;
  long ncell = ncx * ncy * ncz;
  long* head = (long*)malloc(sizeof(long) * ncell);
  long* next = (long*)malloc(sizeof(long) * n);
  for (long c = 0; c < ncell; ++c) head[c] = -1;
  for (int64_t i = 0; i < n; ++i) {
    double px = x[3 * i] - P->Lx * floor(x[3 * i] / P->Lx);
    double pz = x[3 * i + 2] - P->Lz * floor(x[3 * i + 2] / P->Lz);
    double py = x[3 * i + 1];
    if (ybulk) py -= P->h * floor(py / P->h);
    long ix = (long)floor(px / csx), iy = (long)floor((py - ylo) / csy), iz = (long)floor(pz / csz);
    if (ix >= ncx) ix = ncx - 1;
    if (iz >= ncz) iz = ncz - 1;
    if (iy < 0) iy = 0;
    if (iy >= ncy) iy = ncy - 1;
    long c = (ix * ncy + iy) * ncz + iz;
    next[i] = head[c];
    head[c] = i;
  }
  for (long ix = 0; ix < ncx; ++ix)
    for (long iy = 0; iy < ncy; ++iy)
      for (long iz = 0; iz < ncz; ++iz) {
        long c = (ix * ncy + iy) * ncz + iz;
        for (int dx = -1; dx <= 1; ++dx)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz) {
              long jx = (ix + dx + ncx) % ncx, jz = (iz + dz + ncz) % ncz, jy = iy + dy;
              if (ybulk) jy = (jy + ncy) % ncy;
              else if (jy < 0 || jy >= ncy) continue;
              long c2 = (jx * ncy + jy) * ncz + jz;
              for (long i = head[c]; i >= 0; i = next[i])
                for (long j = head[c2]; j >= 0; j = next[j]) {
                  if (j <= i) continue;  /* each unordered pair once */
                  if (!or_pair_active(P, sp[i], sp[j])) continue;
                  double d[3] = {x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1], x[3 * i + 2] - x[3 * j + 2]};
                  d[0] = or_min_image(d[0], P->Lx);
                  d[2] = or_min_image(d[2], P->Lz);
                  if (ybulk) d[1] = or_min_image(d[1], P->h);
                  double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                  if (r2 < rc2) or_add_pair(P, i, j, d, r2, sp, f, wxx, epot);
                }
            }
      }
  free(head);
  free(next);
}

/* Total force: LJ (cells or brute), plus the tether -k (r - r0) on tethered
 * wall atoms (minimum image in x and z), plus the body force g on fluid atoms
 * (Eq. momentumEq).  epot gets the tether energy k|r - r0|^2 / 2. */
void or_forces(const or_params* P, int64_t n, const double* x, const double* anchor, const int32_t* sp,
               int use_cells, double* f, double* wxx, double* epot) {
  if (use_cells) or_lj_cells(P, n, x, sp, f, wxx, epot);
  else or_lj_brute(P, n, x, sp, f, wxx, epot);
  for (int64_t i = 0; i < n; ++i) {
    if (sp[i] == 0) {
      f[3 * i] += P->g;
    } else if (P->mode == 0) {
      double d[3] = {x[3 * i] - anchor[3 * i], x[3 * i + 1] - anchor[3 * i + 1], x[3 * i + 2] - anchor[3 * i + 2]};
      d[0] = or_min_image(d[0], P->Lx);
      d[2] = or_min_image(d[2], P->Lz);
      for (int k = 0; k < 3; ++k) f[3 * i + k] -= P->k_tether * d[k];
      epot[i] += 0.5 * P->k_tether * (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    }
  }
}

static double or_total_energy(const or_params* P, int64_t n, const double* v, const double* epot, const int32_t* sp) {
  double e = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    if (sp[i] == 1 && P->mode == 1) continue;
    e += epot[i] + 0.5 * P->mass * (v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2]);
  }
  return e;
}

/* ------------------------------------------------------------------------ */
/* Time integration.                                                         */
/* Fluid: velocity Verlet (App. A).  Tethered wall atoms: the G-JF Langevin   */
/* scheme of Gronbech-Jensen & Farago (Mol. Phys. 2013), which is velocity   */
/* Verlet when gamma = 0:                                                    */
/*   x' = x + b dt v + b dt^2/(2m) f + b dt/(2m) beta                        */
/*   v' = a v + dt/(2m) (a f + f') + (b/m) beta                              */
/*   a = (1 - g dt/2m)/(1 + g dt/2m), b = 1/(1 + g dt/2m),                    */
/*   beta ~ N(0, 2 gamma T dt) per component, drawn from the Langevin stream  */
/*   with counter (atom, step, element, 1).                                  */
/* Frozen walls (mode 1) do not move; the fluid's v_z is rescaled by the      */
/* Berendsen factor sqrt(1 + dt/tau (T0/T_z - 1)), T_z = m <v_z^2> (fluid).  */
/* ------------------------------------------------------------------------ */
int or_simulate(const or_params* P, int64_t n, double* x, double* v, const double* anchor, const int32_t* sp,
                int64_t s0, int64_t s1, int use_cells, or_accum* acc) {
  int64_t nf = 0;
  for (int64_t i = 0; i < n; ++i) nf += sp[i] == 0;
  double* f = (double*)malloc(sizeof(double) * 3 * n);
  double* wxx = (double*)malloc(sizeof(double) * n);
  double* epot = (double*)malloc(sizeof(double) * n);
  double* u = (double*)malloc(sizeof(double) * 3 * n);
  int nb = P->n_blocks;
  if (nb > OR_MAXB) nb = OR_MAXB;
  if (P->steps_sample < nb) nb = (int)P->steps_sample;
  double m = P->mass, dt = P->dt;
  double c = P->gamma_wall * dt / (2.0 * m);
  double aw = (1.0 - c) / (1.0 + c), bw = 1.0 / (1.0 + c);
  double beta_sd = sqrt(2.0 * P->gamma_wall * P->T * dt);
  double vol = P->Lx * P->h * P->Lz;
  or_forces(P, n, x, anchor, sp, use_cells, f, wxx, epot);
  if (s0 == 0) acc->e_first = or_total_energy(P, n, v, epot, sp);
  for (int64_t s = s0; s < s1; ++s) {
    /* first stage: half kick and drift */
    for (int64_t i = 0; i < n; ++i) {
      if (sp[i] == 1) {
        if (P->mode == 1) { u[3 * i] = u[3 * i + 1] = u[3 * i + 2] = 0.0; continue; }
        double beta[3] = {0.0, 0.0, 0.0};
        if (P->gamma_wall > 0.0) {
          double z[4];
          or_normals4((uint32_t)i, (uint32_t)s, (uint32_t)P->elem_id, OR_STREAM_LANGEVIN, P->seed, z);
          for (int k = 0; k < 3; ++k) beta[k] = beta_sd * z[k];
        }
        for (int k = 0; k < 3; ++k) {
          x[3 * i + k] += bw * dt * (v[3 * i + k] + dt / (2.0 * m) * f[3 * i + k] + beta[k] / (2.0 * m));
          u[3 * i + k] = aw * v[3 * i + k] + dt / (2.0 * m) * aw * f[3 * i + k] + bw / m * beta[k];
        }
      } else {
        for (int k = 0; k < 3; ++k) {
          u[3 * i + k] = v[3 * i + k] + dt / (2.0 * m) * f[3 * i + k];
          x[3 * i + k] += dt * u[3 * i + k];
        }
      }
      /* keep x and z inside the periodic box */
      x[3 * i] -= P->Lx * floor(x[3 * i] / P->Lx);
      x[3 * i + 2] -= P->Lz * floor(x[3 * i + 2] / P->Lz);
      if (P->mode == 2) x[3 * i + 1] -= P->h * floor(x[3 * i + 1] / P->h);
    }
    or_forces(P, n, x, anchor, sp, use_cells, f, wxx, epot);
    /* second stage: half kick with the new force */
    for (int64_t i = 0; i < n; ++i)
      for (int k = 0; k < 3; ++k) v[3 * i + k] = u[3 * i + k] + dt / (2.0 * m) * f[3 * i + k];
    if (P->mode == 1 && nf > 0 && P->tau_T > 0.0) {
      double tz = 0.0;
      for (int64_t i = 0; i < n; ++i)
        if (sp[i] == 0) tz += m * v[3 * i + 2] * v[3 * i + 2];
      tz /= (double)nf;
      if (tz > 0.0) {
        double lam = sqrt(1.0 + dt / P->tau_T * (P->T / tz - 1.0));
        for (int64_t i = 0; i < n; ++i)
          if (sp[i] == 0) v[3 * i + 2] *= lam;
      }
    }
    /* sampling: q_inst = (m / L_x) sum_fluid v_x;
     * P_xx,inst = (sum_fluid m v_x^2 + W_xx) / V with W_xx the fluid atoms'
     * virial shares (fluid-fluid pairs in full, fluid-wall pairs half). */
    for (int64_t i = 0; i < n; ++i) {
      double vv = v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2];
      if (!isfinite(vv) || !isfinite(x[3 * i + 1]) || fabs(x[3 * i + 1]) > 1e6) acc->status = -4;
    }
    if (s >= P->steps_eq && nb > 0) {
      int64_t k = s - P->steps_eq;
      int b = (int)((k * nb) / P->steps_sample);
      double sq = 0.0, sp2 = 0.0, ke2 = 0.0;
      for (int64_t i = 0; i < n; ++i) {
        if (sp[i] != 0) continue;
        sq += m * v[3 * i];
        sp2 += m * v[3 * i] * v[3 * i] + wxx[i];
        ke2 += m * (v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2]);
      }
      acc->q_block[b] += sq / P->Lx;
      acc->p_block[b] += sp2 / vol;
      acc->n_block[b] += 1;
      acc->T_sum += nf > 0 ? ke2 / (3.0 * (double)nf) : 0.0;
      acc->n_samples += 1;
    }
  }
  acc->e_last = or_total_energy(P, n, v, epot, sp);
  free(f); free(wxx); free(epot); free(u);
  return acc->status;
}

/* Mean over all samples and standard error from the block means
 * (std with ddof = 1 over n_b blocks, divided by sqrt(n_b)). */
void or_finalize(const or_params* P, const or_accum* acc, int64_t nf, int64_t nw, or_result* out) {
  int nb = P->n_blocks;
  if (nb > OR_MAXB) nb = OR_MAXB;
  if (P->steps_sample < nb) nb = (int)P->steps_sample;
  double qs = 0.0, ps = 0.0;
  int64_t ns = 0;
  double qm[OR_MAXB], pm[OR_MAXB];
  for (int b = 0; b < nb; ++b) {
    qs += acc->q_block[b];
    ps += acc->p_block[b];
    ns += acc->n_block[b];
    qm[b] = acc->n_block[b] ? acc->q_block[b] / acc->n_block[b] : 0.0;
    pm[b] = acc->n_block[b] ? acc->p_block[b] / acc->n_block[b] : 0.0;
  }
  out->q = ns ? qs / ns : NAN;
  out->p = ns ? ps / ns : NAN;
  if (nb >= 2) {
    double mq = 0.0, mp = 0.0;
    for (int b = 0; b < nb; ++b) { mq += qm[b]; mp += pm[b]; }
    mq /= nb; mp /= nb;
    double vq = 0.0, vp = 0.0;
    for (int b = 0; b < nb; ++b) { vq += (qm[b] - mq) * (qm[b] - mq); vp += (pm[b] - mp) * (pm[b] - mp); }
    out->q_se = sqrt(vq / (nb - 1) / nb);
    out->p_se = sqrt(vp / (nb - 1) / nb);
  } else {
    out->q_se = NAN;
    out->p_se = NAN;
  }
  out->T_meas = acc->n_samples ? acc->T_sum / acc->n_samples : NAN;
  int64_t n = nf + nw;
  out->e_drift = n ? (acc->e_last - acc->e_first) / (double)n : 0.0;
  out->n_fluid = nf;
  out->n_wall = nw;
  out->status = acc->status;
}

/* One whole element: build, run steps_eq + steps_sample steps, reduce. */
int or_element(const or_params* P, int use_cells, or_result* out) {
  int64_t nf = or_n_fluid(P), nw = or_n_wall(P), n = nf + nw;
  double* x = (double*)malloc(sizeof(double) * 3 * n);
  double* v = (double*)malloc(sizeof(double) * 3 * n);
  double* a = (double*)malloc(sizeof(double) * 3 * n);
  int32_t* sp = (int32_t*)malloc(sizeof(int32_t) * n);
  or_accum acc;
  memset(&acc, 0, sizeof(acc));
  or_init(P, x, v, a, sp);
  or_simulate(P, n, x, v, a, sp, 0, P->steps_eq + P->steps_sample, use_cells, &acc);
  or_finalize(P, &acc, nf, nw, out);
  free(x); free(v); free(a); free(sp);
  return out->status;
}
