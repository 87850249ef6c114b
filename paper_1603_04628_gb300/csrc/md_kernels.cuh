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

// Three standard normals by Box-Muller on the block's two pairs of uniforms,
// in double (FP64 path) or in single precision from the top 24 bits (FP32
// path: the noise enters the FP64 update as a small term).
template <typename T>
__device__ __forceinline__ void normals3(uint32_t atom, uint32_t step, uint32_t elem, uint32_t stream,
                                         unsigned long long seed, double& n0, double& n1, double& n2) {
  const uint4 r = philox10(make_uint4(atom, step, elem, stream), (uint32_t)seed, (uint32_t)(seed >> 32));
  if constexpr (sizeof(T) == 8) {
    const double inv32 = 2.3283064365386962890625e-10;  // 2^-32
    const double u1 = ((double)r.x + 0.5) * inv32, u2 = ((double)r.y + 0.5) * inv32;
    const double u3 = ((double)r.z + 0.5) * inv32, u4 = ((double)r.w + 0.5) * inv32;
    const double rad1 = sqrt(-2.0 * log(u1)), rad2 = sqrt(-2.0 * log(u3));
    double s1, c1, s2, c2;
    sincospi(2.0 * u2, &s1, &c1);
    sincospi(2.0 * u4, &s2, &c2);
    n0 = rad1 * c1; n1 = rad1 * s1; n2 = rad2 * c2;
  } else {
    const float inv24 = 5.9604644775390625e-8f;  // 2^-24
    const float u1 = ((float)(r.x >> 8) + 0.5f) * inv24, u2 = ((float)(r.y >> 8) + 0.5f) * inv24;
    const float u3 = ((float)(r.z >> 8) + 0.5f) * inv24, u4 = ((float)(r.w >> 8) + 0.5f) * inv24;
    const float rad1 = sqrtf(-2.0f * logf(u1)), rad2 = sqrtf(-2.0f * logf(u3));
    float s1, c1, s2, c2;
    sincospif(2.0f * u2, &s1, &c1);
    sincospif(2.0f * u4, &s2, &c2);
    n0 = (double)(rad1 * c1); n1 = (double)(rad1 * s1); n2 = (double)(rad2 * c2);
  }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Warp-cooperative segmented reduction: lanes with equal key >= 0 add their
// NV values; one atomicAdd per (key, value) at dst(key, i).  All 32 lanes of
// the warp must call it.
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
  if (x >= L) x -= L;
  if (x < 0.0) x += L;
  if (x >= L || x < 0.0) x -= L * floor(x / L);
  return x;
}

__device__ __forceinline__ double min_image(double d, double L) { return d - L * rint(d / L); }

__device__ __forceinline__ void cell_coords(const ElemDev& E, long long c, int& ix, int& iy, int& iz) {
  const long long l = c - E.cell0;
  iz = (int)(l % E.nc[2]);
  iy = (int)((l / E.nc[2]) % E.nc[1]);
  ix = (int)(l / ((long long)E.nc[2] * E.nc[1]));
}

__device__ __forceinline__ void cell_center(const ElemDev& E, long long c, double& cx, double& cy, double& cz) {
  int ix, iy, iz;
  cell_coords(E, c, ix, iy, iz);
  cx = ((double)ix + 0.5) * E.cs[0];
  cy = E.ylo + ((double)iy + 0.5) * E.cs[1];
  cz = ((double)iz + 0.5) * E.cs[2];
}

// Absolute position of atom i (x and z wrapped into the periodic box).
__device__ __forceinline__ void abs_position(const BatchDev& B, const ElemDev& E, long long i, double& x,
                                             double& y, double& z) {
  x = B.st[0][i]; y = B.st[1][i]; z = B.st[2][i];
  const int c = B.cell[i];
  if (c >= 0) {
    double cx, cy, cz;
    cell_center(E, c, cx, cy, cz);
    x += cx; y += cy; z += cz;
  }
  x = wrap_periodic(x, E.Lx);
  z = wrap_periodic(z, E.Lz);
}

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
// (paper: "fluid atoms in a lattice, with zero mean velocity").  Positions are
// written absolute (reference cell -1) until the first rebuild.
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
    B.st[0][a] = px; B.st[1][a] = py; B.st[2][a] = pz;
    B.st[6][a] = px; B.st[7][a] = py; B.st[8][a] = pz;
    B.orig[a] = (int)l;
    B.cell[a] = -1;
    double n0, n1, n2;
    normals3<double>((uint32_t)l, 0u, (uint32_t)E.id, 0u, E.seed, n0, n1, n2);
    const double vx = E.vsd * n0, vy = E.vsd * n1, vz = E.vsd * n2;
    B.st[3][a] = vx; B.st[4][a] = vy; B.st[5][a] = vz;
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
  const int group = B.orig[a] < E.nf ? 0 : 1;
  const double cnt = group == 0 ? (double)E.nf : (double)E.nw;
  const double* g = B.grp + (size_t)(2 * e + group) * kGrpStride;
  const double mx = g[0] / cnt, my = g[1] / cnt, mz = g[2] / cnt;
  double vx = B.st[3][a] - mx, vy = B.st[4][a] - my, vz = B.st[5][a] - mz;
  const double ke2 = P.mass * (g[3] - cnt * (mx * mx + my * my + mz * mz));
  if (cnt > 1.0 && ke2 > 0.0) {
    const double s = sqrt(E.T / (ke2 / (3.0 * (cnt - 1.0))));
    vx *= s; vy *= s; vz *= s;
  }
  B.st[3][a] = vx; B.st[4][a] = vy; B.st[5][a] = vz;
}

// ---------------------------------------------------------------------------
// Neighbour-list rebuild, step 1: bin every atom into its cell (counting
// sort histogram by atomics; x and z periodic, y clamped to the edge cells).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_bin(BatchDev B) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i == 0) atomicAdd(&B.flags[2], 1);
  if (i >= B.n_atoms) return;
  const ElemDev& E = B.el[B.atom_el[i]];
  double x, y, z;
  abs_position(B, E, i, x, y, z);
  int ix = (int)(x * E.inv_cs[0]), iz = (int)(z * E.inv_cs[2]);
  const double yr = (y - E.ylo) * E.inv_cs[1];
  const int iy = yr < 0.0 ? 0 : (yr >= (double)E.nc[1] ? E.nc[1] - 1 : (int)yr);
  ix = ix < 0 ? 0 : (ix >= E.nc[0] ? E.nc[0] - 1 : ix);
  iz = iz < 0 ? 0 : (iz >= E.nc[2] ? E.nc[2] - 1 : iz);
  const long long c = E.cell0 + ((long long)ix * E.nc[1] + iy) * E.nc[2] + iz;
  B.newcell[i] = (int)c;
  B.slot[i] = atomicAdd(&B.ccount[c], 1);
}

// Step 2: per element (one block), exclusive scan of the cell counts; cell c
// then owns sorted atoms [start, start + size).  Counts are cleared for the
// next rebuild.
__global__ void __launch_bounds__(1024) k_scan(BatchDev B) {
  __shared__ int warp_tot[32];
  __shared__ int carry;
  const ElemDev& E = B.el[blockIdx.x];
  const long long ncell = (long long)E.nc[0] * E.nc[1] * E.nc[2];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (long long base = 0; base < ncell; base += blockDim.x) {
    const long long c = base + threadIdx.x;
    const int v = c < ncell ? B.ccount[E.cell0 + c] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, t, o);
        if (lane >= o) t += y;
      }
      warp_tot[lane] = t;  // inclusive prefix of warp totals
    }
    __syncthreads();
    const int before = carry + (wid > 0 ? warp_tot[wid - 1] : 0) + x - v;
    if (c < ncell) {
      B.cstart[E.cell0 + c] = (int)(E.atom0 + before);
      B.csize[E.cell0 + c] = v;
      B.ccount[E.cell0 + c] = 0;
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = before + v;
    __syncthreads();
  }
}

// Step 3: move every atom to its cell-ordered slot; positions become offsets
// from the new reference cell's centre, anchors likewise (minimum image).
template <typename PT>
__global__ void __launch_bounds__(256) k_permute(BatchDev B) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= B.n_atoms) return;
  const ElemDev& E = B.el[B.atom_el[i]];
  const int c = B.newcell[i];
  const long long dst = (long long)B.cstart[c] + B.slot[i];
  double x, y, z;
  abs_position(B, E, i, x, y, z);
  double cx, cy, cz;
  cell_center(E, c, cx, cy, cz);
  const double ox = x - cx, oy = y - cy, oz = z - cz;
  const int l = B.orig[i];
  const bool wall = l >= E.nf;
  double ax = 0.0, ay = 0.0, az = 0.0;
  if (wall) {
    ax = B.st[6][i]; ay = B.st[7][i]; az = B.st[8][i];
    const int c0 = B.cell[i];
    if (c0 >= 0) {
      double px, py, pz;
      cell_center(E, c0, px, py, pz);
      ax += px; ay += py; az += pz;
    }
    ax = min_image(ax - cx, E.Lx);
    ay = ay - cy;
    az = min_image(az - cz, E.Lz);
  }
  B.st2[0][dst] = ox; B.st2[1][dst] = oy; B.st2[2][dst] = oz;
  B.st2[3][dst] = B.st[3][i]; B.st2[4][dst] = B.st[4][i]; B.st2[5][dst] = B.st[5][i];
  B.st2[6][dst] = ax; B.st2[7][dst] = ay; B.st2[8][dst] = az;
  B.orig2[dst] = l;
  B.cell2[dst] = c;
  const float spf = wall ? 1.0f : 0.0f;
  if constexpr (sizeof(PT) == 16) {
    static_cast<float4*>(B.pos)[dst] = make_float4((float)ox, (float)oy, (float)oz, spf);
  } else {
    static_cast<Pos64*>(B.pos)[dst] = Pos64{ox, oy, oz, (double)spf};
  }
  B.pbuild[dst] = make_float4((float)ox, (float)oy, (float)oz, 0.0f);
}

__global__ void __launch_bounds__(256) k_copy_back(BatchDev B) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= B.n_atoms) return;
#pragma unroll
  for (int k = 0; k < 9; ++k) B.st[k][i] = B.st2[k][i];
  B.orig[i] = B.orig2[i];
  B.cell[i] = B.cell2[i];
}

// Step 4: Verlet lists by a warp-cooperative sweep: one warp per cell, one
// lane per atom of the cell; the lanes walk each neighbour cell's atoms
// together (same address on every lane: a broadcast) and keep those within
// r_c + skin.  The shift between the two reference cells is warp-uniform.
// Lists are stored in groups of four entries, [k / 4][atom][4]: a lane
// collects four entries in registers and writes them with one 16-byte store;
// the last group is padded with an entry that is always beyond r_c (the atom
// itself one cell over in x), so readers never test the count inside a group.
__device__ __forceinline__ unsigned pad_entry(long long i, const ElemDev& E) {
  return (unsigned)(i - E.atom0) | (2u << 26) | (1u << 28) | (1u << 30);
}

template <typename PT>
__global__ void __launch_bounds__(128) k_build(BatchDev B, PhysDev P) {
  using T = decltype(PT::x);
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= B.n_cells) return;
  const int cap4 = B.list_cap >> 2;   // groups per atom
  const int e = B.cell_el[warp];
  const ElemDev& E = B.el[e];
  int cx, cy, cz;
  cell_coords(E, warp, cx, cy, cz);
  const int ncx = E.nc[0], ncy = E.nc[1], ncz = E.nc[2];
  const int s0 = B.cstart[warp], n0 = B.csize[warp];
  const PT* pos = static_cast<const PT*>(B.pos);
  const T rl2 = sizeof(T) == 4 ? (T)P.rl2f : (T)P.rl2;
  const long long N = B.n_atoms;
  uint4* L4 = reinterpret_cast<uint4*>(B.list);
  for (int base = 0; base < n0; base += 32) {
    const int i = s0 + base + lane;
    const bool act = base + lane < n0;
    PT me;
    if (act) me = pos[i];
    else { me.x = me.y = me.z = (T)1e9; me.w = (T)0; }
    int cnt = 0;
    unsigned b0 = 0, b1 = 0, b2 = 0;
    auto push = [&](unsigned ent) {
      const int slot = cnt & 3;
      if (slot == 0) b0 = ent;
      else if (slot == 1) b1 = ent;
      else if (slot == 2) b2 = ent;
      else if ((cnt >> 2) < cap4) L4[(long long)(cnt >> 2) * N + i] = make_uint4(b0, b1, b2, ent);
      ++cnt;
    };
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
          const T qx = me.x - (T)dx * (T)E.cs[0], qy = me.y - (T)dy * (T)E.cs[1], qz = me.z - (T)dz * (T)E.cs[2];
          const int j0 = B.cstart[c2], j1 = j0 + B.csize[c2];
          const unsigned code = ((unsigned)(dx + 1) << 26) | ((unsigned)(dy + 1) << 28) | ((unsigned)(dz + 1) << 30);
          const unsigned jb = (unsigned)(j0 - E.atom0) | code;
          int j = j0;
          for (; j + 3 < j1; j += 4) {
            const PT o0 = pos[j], o1 = pos[j + 1], o2 = pos[j + 2], o3 = pos[j + 3];
            T d0, d1, d2, d3;
            { const T ax = qx - o0.x, ay = qy - o0.y, az = qz - o0.z; d0 = ax * ax + ay * ay + az * az; }
            { const T ax = qx - o1.x, ay = qy - o1.y, az = qz - o1.z; d1 = ax * ax + ay * ay + az * az; }
            { const T ax = qx - o2.x, ay = qy - o2.y, az = qz - o2.z; d2 = ax * ax + ay * ay + az * az; }
            { const T ax = qx - o3.x, ay = qy - o3.y, az = qz - o3.z; d3 = ax * ax + ay * ay + az * az; }
            const unsigned ej = jb + (unsigned)(j - j0);
            if (act && d0 < rl2 && j != i) push(ej);
            if (act && d1 < rl2 && j + 1 != i) push(ej + 1);
            if (act && d2 < rl2 && j + 2 != i) push(ej + 2);
            if (act && d3 < rl2 && j + 3 != i) push(ej + 3);
          }
          for (; j < j1; ++j) {
            const PT o0 = pos[j];
            const T ax = qx - o0.x, ay = qy - o0.y, az = qz - o0.z;
            if (act && ax * ax + ay * ay + az * az < rl2 && j != i) push(jb + (unsigned)(j - j0));
          }
        }
      }
    }
    if (act) {
      // pad and write the last, partial group
      if ((cnt & 3) != 0 && (cnt >> 2) < cap4) {
        const unsigned pe = pad_entry(i, E);
        const int slot = cnt & 3;
        L4[(long long)(cnt >> 2) * N + i] =
            make_uint4(b0, slot > 1 ? b1 : pe, slot > 2 ? b2 : pe, pe);
      }
      if (cnt > B.list_cap) atomicMin(&B.status[e], kStOverflow);
      B.nlist[i] = cnt < B.list_cap ? cnt : B.list_cap;
    }
  }
}

// ---------------------------------------------------------------------------
// LJ pair forces over the Verlet lists: one thread per atom (cell order, so
// a warp's neighbours are shared in L1).  Eq. LJ truncated at r_c, energy
// shifted by U(r_c) per pair type.  The displacement is formed from
// cell-centre offsets: d = (p_i - p_j) - delta * cs, delta in {-1, 0, 1}^3
// from the entry's shift bits, so FP32 only ever rounds numbers below ~3.
// Writes the LJ force, the x-virial share of fluid atoms (half per pair) and,
// with ENERGY, half the shifted pair energy per atom.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float shift_unit(unsigned bits2) {
  // bits2 in {0, 1, 2} -> {-1, 0, 1}, exactly, without an int-to-float convert
  return __int_as_float(0x4B400000 | (int)bits2) - 12582913.0f;
}

template <typename PT, typename T, bool UNIFORM, bool ENERGY>
struct PairAcc {
  T fx = 0, fy = 0, fz = 0, w = 0, u = 0;
  __device__ __forceinline__ void add(const PT& me, const PT& o, unsigned ent, T csx, T csy, T csz, int spi,
                                      T rc2, const T (&eps)[3], const T (&sig2)[3], const PhysDev& P) {
    const float sx = shift_unit((ent >> 26) & 3u), sy = shift_unit((ent >> 28) & 3u), sz = shift_unit(ent >> 30);
    T ddx, ddy, ddz;
    if constexpr (sizeof(T) == 4) {
      ddx = fmaf(-sx, csx, me.x - o.x);
      ddy = fmaf(-sy, csy, me.y - o.y);
      ddz = fmaf(-sz, csz, me.z - o.z);
    } else {
      ddx = (me.x - o.x) - (double)sx * csx;
      ddy = (me.y - o.y) - (double)sy * csy;
      ddz = (me.z - o.z) - (double)sz * csz;
    }
    const T r2 = ddx * ddx + ddy * ddy + ddz * ddz;
    T inv2;
    if constexpr (sizeof(T) == 4) inv2 = __frcp_rn(r2); else inv2 = 1.0 / r2;
    T e_, s2;
    int t = 0;
    if constexpr (UNIFORM) {
      e_ = (T)1; s2 = inv2;
    } else {
      t = spi + (o.w != (T)0 ? 1 : 0);
      e_ = eps[t];
      s2 = sig2[t] * inv2;
    }
    const T s6 = s2 * s2 * s2;
    T fs = (T)24 * e_ * inv2 * s6 * ((T)2 * s6 - (T)1);
    bool in = r2 < rc2;
    if constexpr (!UNIFORM) in = in && P.active[t];
    fs = in ? fs : (T)0;
    fx += fs * ddx; fy += fs * ddy; fz += fs * ddz;
    w += fs * ddx * ddx;
    if (ENERGY) u += in ? ((T)4 * e_ * (s6 * s6 - s6) - (T)P.eshift[t]) : (T)0;
  }
};

template <typename PT, typename T, bool UNIFORM, bool ENERGY>
__global__ void __launch_bounds__(128) k_force(BatchDev B, PhysDev P) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= B.n_atoms) return;
  const ElemDev& E = B.el[B.atom_el[i]];
  const PT* pos = static_cast<const PT*>(B.pos);
  const PT me = pos[i];
  const T csx = (T)E.cs[0], csy = (T)E.cs[1], csz = (T)E.cs[2];
  const PT* posj = pos + E.atom0;
  const int n = B.nlist[i];
  const long long N = B.n_atoms;
  T rc2, eps[3], sig2[3];
  if constexpr (sizeof(T) == 4) {
    rc2 = P.rc2f;
    for (int t = 0; t < 3; ++t) { eps[t] = P.epsf[t]; sig2[t] = P.sig2f[t]; }
  } else {
    rc2 = P.rc2;
    for (int t = 0; t < 3; ++t) { eps[t] = P.eps[t]; sig2[t] = P.sig2[t]; }
  }
  const int spi = me.w != (T)0 ? 1 : 0;
  PairAcc<PT, T, UNIFORM, ENERGY> acc;
  const uint4* L4 = reinterpret_cast<const uint4*>(B.list) + i;
  const int ng = (n + 3) >> 2;
  for (int k = 0; k < ng; ++k) {
    const uint4 e = __ldg(L4 + (long long)k * N);
    const PT o0 = posj[e.x & kJMask], o1 = posj[e.y & kJMask], o2 = posj[e.z & kJMask], o3 = posj[e.w & kJMask];
    acc.add(me, o0, e.x, csx, csy, csz, spi, rc2, eps, sig2, P);
    acc.add(me, o1, e.y, csx, csy, csz, spi, rc2, eps, sig2, P);
    acc.add(me, o2, e.z, csx, csy, csz, spi, rc2, eps, sig2, P);
    acc.add(me, o3, e.w, csx, csy, csz, spi, rc2, eps, sig2, P);
  }
  static_cast<T*>(B.fx)[i] = acc.fx;
  static_cast<T*>(B.fy)[i] = acc.fy;
  static_cast<T*>(B.fz)[i] = acc.fz;
  static_cast<T*>(B.wxx)[i] = spi == 0 ? (T)0.5 * acc.w : (T)0;
  if (ENERGY) static_cast<T*>(B.epot)[i] = (T)0.5 * acc.u;
}

// ---------------------------------------------------------------------------
// Fused integration kernel, one thread per atom.  With s the step started:
//   kFinish  completes step s-1: v = u + dt/(2m) F(x), samples it;
//   kStage1  first stage of step s: fluid velocity-Verlet half kick + drift,
//            tethered wall atoms G-JF (Gronbech-Jensen & Farago 2013);
// then publishes the pair-force input position and checks the list skin.
// F(x) = LJ (force kernel) + body force g on fluid atoms (Eq. momentumEq) +
// tether -k (r - r0) on wall atoms.
// ---------------------------------------------------------------------------
template <typename FT, typename PT>
__global__ void __launch_bounds__(256) k_integrate(BatchDev B, PhysDev P, int k, int mode,
                                                   cudaGraphConditionalHandle hcond, int use_cond) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long s = *B.step_base + k;
  int mkey = -1;
  int mblk = 0;
  double mval[3] = {0.0, 0.0, 0.0};
  if (i < B.n_atoms) {
    const int e = B.atom_el[i];
    const ElemDev& E = B.el[e];
    const int l = B.orig[i];
    const bool fluid = l < E.nf;
    double x = B.st[0][i], y = B.st[1][i], z = B.st[2][i];
    double vx = B.st[3][i], vy = B.st[4][i], vz = B.st[5][i];
    double fx = (double)static_cast<const FT*>(B.fx)[i];
    double fy = (double)static_cast<const FT*>(B.fy)[i];
    double fz = (double)static_cast<const FT*>(B.fz)[i];
    if (fluid) {
      fx += E.g;
    } else {
      fx -= P.k_tether * (x - B.st[6][i]);
      fy -= P.k_tether * (y - B.st[7][i]);
      fz -= P.k_tether * (z - B.st[8][i]);
    }
    if ((mode & kFinish) && s >= 1 && s - 1 < E.steps_total) {
      vx += P.hdt_m * fx; vy += P.hdt_m * fy; vz += P.hdt_m * fz;
      const long long ks = s - 1 - E.steps_eq;
      const double v2 = vx * vx + vy * vy + vz * vz;
      if (!(v2 < 1e30) || !(fabs(y) < 1e6)) atomicMin(&B.status[e], kStUnstable);
      if (fluid && ks >= 0 && ks < E.steps_sample && E.nb > 0) {
        mkey = e;
        mblk = (int)((ks * E.nb) / E.steps_sample);
        mval[0] = P.mass * vx;
        mval[1] = P.mass * vx * vx + (double)static_cast<const FT*>(B.wxx)[i];
        mval[2] = P.mass * v2;
      }
    }
    if ((mode & kStage1) && s < E.steps_total) {
      if (fluid) {
        vx += P.hdt_m * fx; vy += P.hdt_m * fy; vz += P.hdt_m * fz;
        x += P.dt * vx; y += P.dt * vy; z += P.dt * vz;
      } else {
        double b0 = 0.0, b1 = 0.0, b2 = 0.0;
        if (E.beta_sd > 0.0) {
          normals3<FT>((uint32_t)l, (uint32_t)s, (uint32_t)E.id, 1u, E.seed, b0, b1, b2);
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
      B.st[0][i] = x; B.st[1][i] = y; B.st[2][i] = z;
      const float xf = (float)x, yf = (float)y, zf = (float)z;
      if constexpr (sizeof(PT) == 16) {
        static_cast<float4*>(B.pos)[i] = make_float4(xf, yf, zf, fluid ? 0.0f : 1.0f);
      } else {
        static_cast<Pos64*>(B.pos)[i] = Pos64{x, y, z, fluid ? 0.0 : 1.0};
      }
      // an atom that moved more than half the skin since the lists were
      // built asks for a rebuild before the next force evaluation
      const float4 pb = B.pbuild[i];
      const float ex = xf - pb.x, ey = yf - pb.y, ez = zf - pb.z;
      if (ex * ex + ey * ey + ez * ez > P.half_skin2f) {
        if (use_cond) atomicOr(&B.flags[0], 1);
        else atomicMin(&B.status[e], kStSkin);
      }
    }
    B.st[3][i] = vx; B.st[4][i] = vy; B.st[5][i] = vz;
  }
  if (mode & kFinish) {
    seg_add<3>(mkey, mval, [&](int e, int q) {
      return B.acc + (size_t)e * kAccStride + (q == 0 ? kAccQ + mblk : (q == 1 ? kAccP + mblk : kAccT));
    });
  }
  if (use_cond) {
    // the last block to finish turns the flag into the graph condition (one
    // caller of cudaGraphSetConditional) and clears the flag words
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const int prev = atomicAdd(&B.flags[1], 1);
      if (prev == (int)gridDim.x - 1) {
        const int need = atomicExch(&B.flags[0], 0);
        atomicExch(&B.flags[1], 0);
        if (need) cudaGraphSetConditional(hcond, 1u);
      }
    }
  }
}

// Total energy per element (kinetic + shifted LJ + tether) into acc[which].
template <typename FT>
__global__ void k_energy(BatchDev B, PhysDev P, int which) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int key = -1;
  double val[1] = {0.0};
  if (i < B.n_atoms) {
    const int e = B.atom_el[i];
    const ElemDev& E = B.el[e];
    const double vx = B.st[3][i], vy = B.st[4][i], vz = B.st[5][i];
    double en = 0.5 * P.mass * (vx * vx + vy * vy + vz * vz) + (double)static_cast<const FT*>(B.epot)[i];
    if (B.orig[i] >= E.nf) {
      const double dx = B.st[0][i] - B.st[6][i], dy = B.st[1][i] - B.st[7][i], dz = B.st[2][i] - B.st[8][i];
      en += 0.5 * P.k_tether * (dx * dx + dy * dy + dz * dz);
    }
    key = e;
    val[0] = en;
  }
  seg_add<1>(key, val, [&](int e, int) { return B.acc + (size_t)e * kAccStride + which; });
}

// Copy state (what = 0: wrapped positions and velocities; what = 1: forces,
// virial shares and energies) into B.out in the original atom order.
template <typename FT>
__global__ void k_export(BatchDev B, int what) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= B.n_atoms) return;
  const ElemDev& E = B.el[B.atom_el[i]];
  const long long dst = E.atom0 + B.orig[i];
  const long long N = B.n_atoms;
  if (what == 0) {
    double x, y, z;
    abs_position(B, E, i, x, y, z);
    B.out[dst] = x; B.out[N + dst] = y; B.out[2 * N + dst] = z;
    B.out[3 * N + dst] = B.st[3][i]; B.out[4 * N + dst] = B.st[4][i]; B.out[5 * N + dst] = B.st[5][i];
  } else {
    B.out[dst] = (double)static_cast<const FT*>(B.fx)[i];
    B.out[N + dst] = (double)static_cast<const FT*>(B.fy)[i];
    B.out[2 * N + dst] = (double)static_cast<const FT*>(B.fz)[i];
    B.out[3 * N + dst] = (double)static_cast<const FT*>(B.wxx)[i];
    B.out[4 * N + dst] = (double)static_cast<const FT*>(B.epot)[i];
    B.out[5 * N + dst] = 0.0;
  }
}

__global__ void k_advance(long long* step, long long by) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *step += by;
}

}  // namespace mdgp
