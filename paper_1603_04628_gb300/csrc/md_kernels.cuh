// Device kernels of the micro-element MD engine (paper App. A, Sec. 2.1).
// Included once, by md_engine.cu.
#pragma once
#include "md_internal.cuh"

namespace mdgp {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// Philox4x32-10 counter-based generator (Salmon et al., SC'11): ten rounds of
// the two-multiply S-box with the key advanced by the golden-ratio and
// sqrt(3)-1 Weyl increments.  Counter = (atom, step, element, stream).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Three standard normals (Box-Muller on the block's first and second pairs).
__device__ __forceinline__ void normals3(uint32_t atom, uint32_t step, uint32_t elem, uint32_t stream,
                                         unsigned long long seed, double& n0, double& n1, double& n2) {
  const uint4 r = philox10(make_uint4(atom, step, elem, stream), (uint32_t)seed, (uint32_t)(seed >> 32));
  const double inv32 = 2.3283064365386962890625e-10;  // 2^-32
  double u1 = ((double)r.x + 0.5) * inv32, u2 = ((double)r.y + 0.5) * inv32;
  double u3 = ((double)r.z + 0.5) * inv32, u4 = ((double)r.w + 0.5) * inv32;
  double rad1 = sqrt(-2.0 * log(u1)), rad2 = sqrt(-2.0 * log(u3));
  double s1, c1, s2, c2;
  sincospi(2.0 * u2, &s1, &c1);
  sincospi(2.0 * u4, &s2, &c2);
  n0 = rad1 * c1;
  n1 = rad1 * s1;
  n2 = rad2 * c2;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Warp-cooperative segmented reduction: lanes with equal key >= 0 add their
// NV values; one atomicAdd per (key, value) at dst(key)[i].  All 32 lanes
// must call it.
template <int NV, typename DstFn>
__device__ __forceinline__ void seg_add(int key, const double (&val)[NV], DstFn dst) {
  const int lane = threadIdx.x & 31;
  unsigned pending = __ballot_sync(kFull, key >= 0);
  while (pending) {
    const int leader = __ffs(pending) - 1;
    const int k = __shfl_sync(kFull, key, leader);
    const bool mine = key == k;
    pending &= ~__ballot_sync(kFull, mine);
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double s = warp_sum(mine ? val[i] : 0.0);
      if (lane == leader) atomicAdd(dst(k, i), s);
    }
  }
}

__device__ __forceinline__ double wrap_periodic(double x, double L) {
  // into [0, L); atoms move far less than L per step
  if (x >= L) x -= L;
  if (x < 0.0) x += L;
  if (x >= L || x < 0.0) x -= L * floor(x / L);
  return x;
}

__device__ __forceinline__ double min_image(double d, double L) { return d - L * rint(d / L); }

// ---------------------------------------------------------------------------
// Maps: atom -> element and cell -> element by binary search on the offsets.
// ---------------------------------------------------------------------------
__global__ void k_fill_maps(BatchDev B) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long a = t; a < B.n_atoms; a += stride) {
    int lo = 0, hi = B.n_el - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (B.atom_off[mid] <= a) lo = mid; else hi = mid - 1;
    }
    B.atom_el[a] = lo;
  }
  for (long long c = t; c < B.n_cells; c += stride) {
    int lo = 0, hi = B.n_el - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (B.cell_off[mid] <= c) lo = mid; else hi = mid - 1;
    }
    B.cell_el[c] = lo;
  }
}

// ---------------------------------------------------------------------------
// Element build: FCC fluid lattice with evenly spread vacancies, FCC (100)
// wall planes with anchors, Maxwell-Boltzmann velocities from the init stream
// (paper: "fluid atoms in a lattice, with zero mean velocity").  Group sums
// for the mean-velocity removal go to B.grp.
// ---------------------------------------------------------------------------
__global__ void k_init_atoms(BatchDev B, PhysDev P) {
  const long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int key = -1;
  double val[4] = {0.0, 0.0, 0.0, 0.0};
  if (a < B.n_atoms) {
    const int e = B.atom_el[a];
    const ElemDev& E = B.el[e];
    const long long l = a - E.atom0;
    double px, py, pz;
    int group;
    if (l < E.nf) {
      group = 0;
      const long long sites = 4LL * E.fc[0] * E.fc[1] * E.fc[2];
      const long long s = (l * sites) / E.nf;
      const int b = (int)(s & 3);
      const long long c = s >> 2;
      const long long iz = c % E.fc[2], iy = (c / E.fc[2]) % E.fc[1], ix = c / ((long long)E.fc[2] * E.fc[1]);
      const double bx = (b == 1 || b == 2) ? 0.5 : 0.0;
      const double by = (b == 1 || b == 3) ? 0.5 : 0.0;
      const double bz = (b == 2 || b == 3) ? 0.5 : 0.0;
      px = ((double)ix + bx + 0.25) * E.fb[0];
      py = E.fy0 + ((double)iy + by + 0.25) * E.fb[1];
      pz = ((double)iz + bz + 0.25) * E.fb[2];
    } else {
      group = 1;
      const long long w = l - E.nf;
      const long long per_plane = 2LL * E.wnx * E.wnz;
      const long long per_wall = per_plane * P.wall_planes;
      const int wall = (int)(w / per_wall);
      const long long r = w % per_wall;
      const int k = (int)(r / per_plane);
      const long long r2 = r % per_plane;
      const long long i = r2 / (2LL * E.wnz), j = (r2 >> 1) % E.wnz;
      const int t = (int)(r2 & 1);
      double ox, oz;
      if ((k & 1) == 0) { ox = t ? 0.5 : 0.0; oz = t ? 0.5 : 0.0; }
      else { ox = t ? 0.0 : 0.5; oz = t ? 0.5 : 0.0; }
      px = ((double)i + ox) * E.wax;
      py = wall == 0 ? -(double)k * E.wdy : E.h + (double)k * E.wdy;
      pz = ((double)j + oz) * E.waz;
    }
    B.x[a] = px; B.y[a] = py; B.z[a] = pz;
    B.ax[a] = px; B.ay[a] = py; B.az[a] = pz;
    double n0, n1, n2;
    normals3((uint32_t)l, 0u, (uint32_t)E.id, 0u, E.seed, n0, n1, n2);
    const double vx = E.vsd * n0, vy = E.vsd * n1, vz = E.vsd * n2;
    B.vx[a] = vx; B.vy[a] = vy; B.vz[a] = vz;
    key = 2 * e + group;
    val[0] = vx; val[1] = vy; val[2] = vz; val[3] = vx * vx + vy * vy + vz * vz;
  }
  seg_add<4>(key, val, [&](int k, int i) { return B.grp + (size_t)k * kGrpStride + i; });
}

// Remove each group's mean velocity, then rescale it to exactly T with
// 3 (N_g - 1) degrees of freedom.
__global__ void k_init_fix(BatchDev B, PhysDev P) {
  const long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (a >= B.n_atoms) return;
  const int e = B.atom_el[a];
  const ElemDev& E = B.el[e];
  const long long l = a - E.atom0;
  const int group = l < E.nf ? 0 : 1;
  const double cnt = group == 0 ? (double)E.nf : (double)E.nw;
  const double* g = B.grp + (size_t)(2 * e + group) * kGrpStride;
  const double mx = g[0] / cnt, my = g[1] / cnt, mz = g[2] / cnt;
  double vx = B.vx[a] - mx, vy = B.vy[a] - my, vz = B.vz[a] - mz;
  const double ke2 = P.mass * (g[3] - cnt * (mx * mx + my * my + mz * mz));
  if (cnt > 1.0 && ke2 > 0.0) {
    const double s = sqrt(E.T / (ke2 / (3.0 * (cnt - 1.0))));
    vx *= s; vy *= s; vz *= s;
  }
  B.vx[a] = vx; B.vy[a] = vy; B.vz[a] = vz;
}

// ---------------------------------------------------------------------------
// Fused integration kernel.  With s the step being started:
//   kFinish  completes step s-1: v = u + dt/(2m) F(x) and samples it;
//   kStage1  first stage of step s: fluid velocity-Verlet half kick + drift,
//            tethered wall atoms G-JF (Gronbech-Jensen & Farago 2013);
//   kBin     bins the new positions into cell slots of count buffer (s & 1)
//            and clears the other count buffer.
// F(x) = LJ (from the force kernel) + body force g on fluid atoms (Eq.
// momentumEq) + tether -k (r - r0) on wall atoms.
// ---------------------------------------------------------------------------
template <typename FT, typename Slot>
__global__ void __launch_bounds__(256) k_integrate(BatchDev B, PhysDev P, int k, int mode) {
  const long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long s = *B.step_base + k;
  int mkey = -1;
  int mblk = 0;
  double mval[3] = {0.0, 0.0, 0.0};
  if (a < B.n_atoms) {
    const int e = B.atom_el[a];
    const ElemDev& E = B.el[e];
    const long long l = a - E.atom0;
    const bool fluid = l < E.nf;
    double x = B.x[a], y = B.y[a], z = B.z[a];
    double vx = B.vx[a], vy = B.vy[a], vz = B.vz[a];
    if (mode & (kFinish | kStage1)) {
      double fx = (double)static_cast<const FT*>(B.fx)[a];
      double fy = (double)static_cast<const FT*>(B.fy)[a];
      double fz = (double)static_cast<const FT*>(B.fz)[a];
      if (fluid) {
        fx += E.g;
      } else {
        const double dx = min_image(x - B.ax[a], E.Lx), dy = y - B.ay[a], dz = min_image(z - B.az[a], E.Lz);
        fx -= P.k_tether * dx; fy -= P.k_tether * dy; fz -= P.k_tether * dz;
      }
      if (mode & kFinish) {
        vx += P.hdt_m * fx; vy += P.hdt_m * fy; vz += P.hdt_m * fz;
        const long long ks = s - 1 - E.steps_eq;
        const double v2 = vx * vx + vy * vy + vz * vz;
        if (!(v2 < 1e30) || !(fabs(y) < 1e6)) atomicMin(&B.status[e], -4);
        if (fluid && ks >= 0 && ks < E.steps_sample && E.nb > 0) {
          mkey = e;
          mblk = (int)((ks * E.nb) / E.steps_sample);
          mval[0] = P.mass * vx;
          mval[1] = P.mass * vx * vx + (double)static_cast<const FT*>(B.wxx)[a];
          mval[2] = P.mass * v2;
        }
      }
      if (mode & kStage1) {
        if (fluid) {
          vx += P.hdt_m * fx; vy += P.hdt_m * fy; vz += P.hdt_m * fz;
          x += P.dt * vx; y += P.dt * vy; z += P.dt * vz;
        } else {
          double b0 = 0.0, b1 = 0.0, b2 = 0.0;
          if (E.beta_sd > 0.0) {
            normals3((uint32_t)l, (uint32_t)s, (uint32_t)E.id, 1u, E.seed, b0, b1, b2);
            b0 *= E.beta_sd; b1 *= E.beta_sd; b2 *= E.beta_sd;
          }
          const double bdt = P.gjf_b * P.dt, h2m = P.dt / (2.0 * P.mass), i2m = 1.0 / (2.0 * P.mass);
          x += bdt * (vx + h2m * fx + b0 * i2m);
          y += bdt * (vy + h2m * fy + b1 * i2m);
          z += bdt * (vz + h2m * fz + b2 * i2m);
          const double bm = P.gjf_b * P.inv_m;
          vx = P.gjf_a * vx + h2m * P.gjf_a * fx + bm * b0;
          vy = P.gjf_a * vy + h2m * P.gjf_a * fy + bm * b1;
          vz = P.gjf_a * vz + h2m * P.gjf_a * fz + bm * b2;
        }
        x = wrap_periodic(x, E.Lx);
        z = wrap_periodic(z, E.Lz);
        B.x[a] = x; B.y[a] = y; B.z[a] = z;
      }
      B.vx[a] = vx; B.vy[a] = vy; B.vz[a] = vz;
    }
    if (mode & kBin) {
      // cell of the (wrapped) position; y outside the grid clamps to the edge cells
      const double xw = wrap_periodic(x, E.Lx), zw = wrap_periodic(z, E.Lz);
      int ix = (int)(xw * E.inv_cs[0]), iz = (int)(zw * E.inv_cs[2]);
      const double yr = (y - E.ylo) * E.inv_cs[1];
      int iy = yr < 0.0 ? 0 : (yr >= (double)E.nc[1] ? E.nc[1] - 1 : (int)yr);
      ix = ix >= E.nc[0] ? E.nc[0] - 1 : ix;
      iz = iz >= E.nc[2] ? E.nc[2] - 1 : iz;
      const long long c = E.cell0 + ((long long)ix * E.nc[1] + iy) * E.nc[2] + iz;
      const int slot = atomicAdd(&B.counts[(s & 1) * B.n_cells + c], 1);
      if (slot < B.cap) {
        Slot q;
        q.x = xw - ((double)ix + 0.5) * E.cs[0];
        q.y = y - (E.ylo + ((double)iy + 0.5) * E.cs[1]);
        q.z = zw - ((double)iz + 0.5) * E.cs[2];
        q.tag = (int)((a << 1) | (fluid ? 0 : 1));
        static_cast<Slot*>(B.slots)[c * B.cap + slot] = q;
      } else {
        atomicMin(&B.status[e], -8);
      }
    }
  }
  if (mode & kFinish) {
    seg_add<3>(mkey, mval, [&](int e, int i) {
      return B.acc + (size_t)e * kAccStride + (i == 0 ? kAccQ + mblk : (i == 1 ? kAccP + mblk : kAccT));
    });
  }
  if (mode & kBin) {
    int* other = B.counts + ((s + 1) & 1) * B.n_cells;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = a; c < B.n_cells; c += stride) other[c] = 0;
  }
}

// ---------------------------------------------------------------------------
// LJ pair forces by a warp-cooperative cell sweep: one warp per target cell,
// one lane per atom of the cell; the lanes walk the 27 neighbour cells'
// slots together (every lane reads the same slot: a broadcast).  Eq. LJ with
// cut-off r_c; energy shifted by U(r_c) per pair type.  Positions are
// relative to cell centres, so the FP32 path forms x_i - x_j from small
// numbers: t = (p_i - lo) - p_j, d = t - hi, where hi + lo is the cell shift.
// Writes the LJ force, the x-virial share (fluid atoms only, half per pair)
// and, with ENERGY, half the shifted pair energy per atom.
// ---------------------------------------------------------------------------
template <typename Slot, typename T, bool ENERGY>
__global__ void __launch_bounds__(128) k_force_cells(BatchDev B, PhysDev P, int k) {
  const long long s = *B.step_base + k;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= B.n_cells) return;
  const int e = B.cell_el[warp];
  const ElemDev& E = B.el[e];
  const long long lc = warp - E.cell0;
  const int ncx = E.nc[0], ncy = E.nc[1], ncz = E.nc[2];
  const int cz = (int)(lc % ncz), cy = (int)((lc / ncz) % ncy), cx = (int)(lc / ((long long)ncz * ncy));
  const int* counts = B.counts + (s & 1) * B.n_cells;
  const Slot* slots = static_cast<const Slot*>(B.slots);
  const int cap = B.cap;
  const int nown = min(counts[warp], cap);
  T rc2, eps[3], sig2[3];
  if constexpr (sizeof(T) == 4) {
    rc2 = P.rc2f;
    for (int t = 0; t < 3; ++t) { eps[t] = P.epsf[t]; sig2[t] = P.sig2f[t]; }
  } else {
    rc2 = P.rc2;
    for (int t = 0; t < 3; ++t) { eps[t] = P.eps[t]; sig2[t] = P.sig2[t]; }
  }
  for (int base = 0; base < nown; base += 32) {
    const int i = base + lane;
    const bool act = i < nown;
    Slot me;
    if (act) me = slots[warp * cap + i];
    else { me.x = me.y = me.z = (T)0; me.tag = -1; }
    const int spi = me.tag & 1;
    T fx = 0, fy = 0, fz = 0, w = 0, u = 0;
    for (int dx = -1; dx <= 1; ++dx) {
      int jx = cx + dx;
      jx = jx < 0 ? jx + ncx : (jx >= ncx ? jx - ncx : jx);
      for (int dy = -1; dy <= 1; ++dy) {
        const int jy = cy + dy;
        if (jy < 0 || jy >= ncy) continue;
        for (int dz = -1; dz <= 1; ++dz) {
          int jz = cz + dz;
          jz = jz < 0 ? jz + ncz : (jz >= ncz ? jz - ncz : jz);
          const long long c2 = E.cell0 + ((long long)jx * ncy + jy) * ncz + jz;
          // x_i - x_j = p_i - p_j - delta * cs, cs split into hi + lo
          T hx, hy, hz, qx, qy, qz;
          if constexpr (sizeof(T) == 4) {
            const float hix = (float)E.cs[0], hiy = (float)E.cs[1], hiz = (float)E.cs[2];
            const float lox = (float)(E.cs[0] - (double)hix), loy = (float)(E.cs[1] - (double)hiy),
                        loz = (float)(E.cs[2] - (double)hiz);
            hx = dx * hix; hy = dy * hiy; hz = dz * hiz;
            qx = me.x - dx * lox; qy = me.y - dy * loy; qz = me.z - dz * loz;
          } else {
            hx = dx * E.cs[0]; hy = dy * E.cs[1]; hz = dz * E.cs[2];
            qx = me.x; qy = me.y; qz = me.z;
          }
          const int n2 = min(counts[c2], cap);
          const Slot* sl = slots + c2 * cap;
          for (int j = 0; j < n2; ++j) {
            const Slot o = sl[j];
            const T ddx = (qx - o.x) - hx, ddy = (qy - o.y) - hy, ddz = (qz - o.z) - hz;
            const T r2 = ddx * ddx + ddy * ddy + ddz * ddz;
            const int t = spi + (o.tag & 1);
            if (act && r2 < rc2 && o.tag != me.tag && P.active[t]) {
              T inv2;
              if constexpr (sizeof(T) == 4) inv2 = __frcp_rn(r2); else inv2 = 1.0 / r2;
              const T s2 = sig2[t] * inv2;
              const T s6 = s2 * s2 * s2;
              const T fs = (T)24 * eps[t] * inv2 * s6 * ((T)2 * s6 - (T)1);
              fx += fs * ddx; fy += fs * ddy; fz += fs * ddz;
              if (spi == 0) w += (T)0.5 * fs * ddx * ddx;
              if (ENERGY) u += (T)0.5 * ((T)4 * eps[t] * (s6 * s6 - s6) - (T)P.eshift[t]);
            }
          }
        }
      }
    }
    if (act) {
      const long long atom = me.tag >> 1;
      static_cast<T*>(B.fx)[atom] = fx;
      static_cast<T*>(B.fy)[atom] = fy;
      static_cast<T*>(B.fz)[atom] = fz;
      static_cast<T*>(B.wxx)[atom] = w;
      if (ENERGY) static_cast<T*>(B.epot)[atom] = u;
    }
  }
}

// Total energy per element (kinetic + shifted LJ + tether) into acc[which].
template <typename FT>
__global__ void k_energy(BatchDev B, PhysDev P, int which) {
  const long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int key = -1;
  double val[1] = {0.0};
  if (a < B.n_atoms) {
    const int e = B.atom_el[a];
    const ElemDev& E = B.el[e];
    const bool fluid = (a - E.atom0) < E.nf;
    const double vx = B.vx[a], vy = B.vy[a], vz = B.vz[a];
    double en = 0.5 * P.mass * (vx * vx + vy * vy + vz * vz) + (double)static_cast<const FT*>(B.epot)[a];
    if (!fluid) {
      const double dx = min_image(B.x[a] - B.ax[a], E.Lx), dy = B.y[a] - B.ay[a],
                   dz = min_image(B.z[a] - B.az[a], E.Lz);
      en += 0.5 * P.k_tether * (dx * dx + dy * dy + dz * dz);
    }
    key = e;
    val[0] = en;
  }
  seg_add<1>(key, val, [&](int e, int) { return B.acc + (size_t)e * kAccStride + which; });
}

__global__ void k_advance(long long* step, long long by) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *step += by;
}

}  // namespace mdgp
