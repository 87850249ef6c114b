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
__device__ __forceinline__ void normals3f(uint32_t atom, uint32_t step, uint32_t elem, uint32_t stream,
                                          unsigned long long seed, float& n0, float& n1, float& n2) {
  const uint4 r = philox10(make_uint4(atom, step, elem, stream), (uint32_t)seed, (uint32_t)(seed >> 32));
  const float inv24 = 5.9604644775390625e-8f;  // 2^-24
  const float u1 = ((float)(r.x >> 8) + 0.5f) * inv24, u2 = ((float)(r.y >> 8) + 0.5f) * inv24;
  const float u3 = ((float)(r.z >> 8) + 0.5f) * inv24, u4 = ((float)(r.w >> 8) + 0.5f) * inv24;
  const float rad1 = sqrtf(-2.0f * logf(u1)), rad2 = sqrtf(-2.0f * logf(u3));
  float s1, c1, s2, c2;
  sincospif(2.0f * u2, &s1, &c1);
  sincospif(2.0f * u4, &s2, &c2);
  n0 = rad1 * c1; n1 = rad1 * s1; n2 = rad2 * c2;
}

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
    float a, b, c;
    normals3f(atom, step, elem, stream, seed, a, b, c);
    n0 = (double)a; n1 = (double)b; n2 = (double)c;
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

// Block-level segmented reduction for blocks of up to 256 threads: every
// thread puts (key, NV values) into shared memory.  When the whole block
// shares one key (the usual case: atoms of one element are contiguous) a
// shared-memory tree over 256 slots (the slots past the block zeroed) adds
// the values and one atomicAdd per value writes the sum; otherwise up to 8
// threads each scan 32 entries and add each run of equal keys.  Keys < 0 are
// skipped.  All threads of the block must call it.
template <int NV, typename DstFn>
__device__ __forceinline__ void block_seg_add(int key, const double (&val)[NV], DstFn dst) {
  __shared__ int skey[256];
  __shared__ double sval[NV][256];
  const int t = threadIdx.x;
  skey[t] = key;
#pragma unroll
  for (int i = 0; i < NV; ++i) sval[i][t] = val[i];
  for (int t2 = t + (int)blockDim.x; t2 < 256; t2 += (int)blockDim.x)
#pragma unroll
    for (int i = 0; i < NV; ++i) sval[i][t2] = 0.0;
  __syncthreads();
  const int k0 = skey[0];
  if (__syncthreads_and(key == k0)) {
    if (k0 < 0) return;
    for (int h = 128; h > 0; h >>= 1) {
      for (int t2 = t; t2 < h; t2 += (int)blockDim.x)
#pragma unroll
        for (int i = 0; i < NV; ++i) sval[i][t2] += sval[i][t2 + h];
      __syncthreads();
    }
    if (t < NV) atomicAdd(dst(k0, t), sval[t][0]);
    return;
  }
  if (t * 32 < (int)blockDim.x) {
    int cur = -1;
    double acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.0;
    for (int r = t * 32; r < t * 32 + 32 && r < (int)blockDim.x; ++r) {
      const int k = skey[r];
      if (k != cur) {
        if (cur >= 0)
#pragma unroll
          for (int i = 0; i < NV; ++i) atomicAdd(dst(cur, i), acc[i]);
        cur = k;
#pragma unroll
        for (int i = 0; i < NV; ++i) acc[i] = 0.0;
      }
      if (k >= 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) acc[i] += sval[i][r];
    }
    if (cur >= 0)
#pragma unroll
      for (int i = 0; i < NV; ++i) atomicAdd(dst(cur, i), acc[i]);
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

// ---------------------------------------------------------------------------
// Double-float state (pair forces in FP32).  A value is hi + lo with
// hi = fl(hi + lo).  Sums use Knuth's TwoSum of the high parts, products the
// exact FMA product (Dekker), so every update runs on the FP32 pipes (FP64
// issues at 1/64 of the FP32 rate on this part) and keeps about 44
// significant bits.  Stored as float2 in the 8-byte state slots.
// ---------------------------------------------------------------------------
struct dfl {
  float hi, lo;
};

__device__ __forceinline__ dfl df_norm(float s, float e) {   // Fast2Sum, |s| >= |e|
  const float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ dfl df_add(dfl a, float b) {
  const float s = __fadd_rn(a.hi, b), bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b, bb)), a.lo);
  return df_norm(s, e);
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  const float s = __fadd_rn(a.hi, b.hi), bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb)), __fadd_rn(a.lo, b.lo));
  return df_norm(s, e);
}
__device__ __forceinline__ dfl df_mul(float c, dfl a) {
  const float p = __fmul_rn(c, a.hi);
  const float e = __fmaf_rn(c, a.lo, __fmaf_rn(c, a.hi, -p));
  return df_norm(p, e);
}
// a - b rounded to float (the two are close: tether stretch, displacement)
__device__ __forceinline__ float df_diff(dfl a, dfl b) { return __fsub_rn(a.hi, b.hi) + __fsub_rn(a.lo, b.lo); }
__device__ __forceinline__ dfl df_from(double d) {
  const float h = (float)d;
  return {h, (float)(d - (double)h)};
}
__device__ __forceinline__ double df_to(dfl a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ dfl df_ld(const double* p, long long i) {
  const float2 v = reinterpret_cast<const float2*>(p)[i];
  return {v.x, v.y};
}
__device__ __forceinline__ void df_st(double* p, long long i, dfl a) {
  reinterpret_cast<float2*>(p)[i] = make_float2(a.hi, a.lo);
}

// Loads of data a step reads once (the lists, the atom state): kept out of
// the L1, so that the L1 holds the neighbour positions the pair loop gathers
// over and over.  The lists are read-only while the step kernels run
// (non-coherent path, no L1 allocation); the state is also written by the
// same kernel, so it is read at the L2 (ld.global.cg).
__device__ __forceinline__ uint4 ld_list4(const uint4* p) {
  uint4 r;
  asm("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
      : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
  return r;
}
__device__ __forceinline__ dfl df_ld_cg(const double* p, long long i) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p) + i);
  return {v.x, v.y};
}

// One state value as a double, in either representation.
template <bool DF>
__device__ __forceinline__ double st_get(const double* p, long long i) {
  if constexpr (DF) return df_to(df_ld(p, i)); else return p[i];
}
template <bool DF>
__device__ __forceinline__ void st_put(double* p, long long i, double v) {
  if constexpr (DF) df_st(p, i, df_from(v)); else p[i] = v;
}

// The standard-error block of sampling step ks (0 <= ks < steps_sample):
// floor(ks nb / steps_sample), in 32-bit unsigned arithmetic whenever
// steps_sample nb fits (the 64-bit division is a long software sequence and
// this runs for every atom every step).
__device__ __forceinline__ int sample_block(long long ks, const ElemDev& E) {
  if (E.steps_sample * (long long)E.nb < (1LL << 32))
    return (int)((unsigned)ks * (unsigned)E.nb / (unsigned)E.steps_sample);
  return (int)((ks * E.nb) / E.steps_sample);
}

// Absolute position of atom i (x and z wrapped into the periodic box).
template <bool DF>
__device__ __forceinline__ void abs_position(const BatchDev& B, const ElemDev& E, long long i, double& x,
                                             double& y, double& z) {
  x = st_get<DF>(B.st[0], i); y = st_get<DF>(B.st[1], i); z = st_get<DF>(B.st[2], i);
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
template <bool DF>
__global__ void k_init_atoms(BatchDev B, PhysDev P) {
  const long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (a < B.n_atoms) {
    const int e = B.atom_el[a];
    const ElemDev& E = B.el[e];
    const long long l = a - E.atom0;
    double px, py, pz;
    int group;
    if (E.amp != 0.0) {
      // walls that follow the channel profile: positions built by the host
      group = l < E.nf ? 0 : 1;
      px = B.pinit[3 * a]; py = B.pinit[3 * a + 1]; pz = B.pinit[3 * a + 2];
    } else if (l < E.nf) {
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
    st_put<DF>(B.st[0], a, px); st_put<DF>(B.st[1], a, py); st_put<DF>(B.st[2], a, pz);
    st_put<DF>(B.st[6], a, px); st_put<DF>(B.st[7], a, py); st_put<DF>(B.st[8], a, pz);
    B.orig[a] = (int)l;
    B.cell[a] = -1;
    double n0, n1, n2;
    normals3<double>((uint32_t)l, 0u, (uint32_t)E.id, 0u, E.seed, n0, n1, n2);
    const double vx = E.vsd * n0, vy = E.vsd * n1, vz = E.vsd * n2;
    st_put<DF>(B.st[3], a, vx); st_put<DF>(B.st[4], a, vy); st_put<DF>(B.st[5], a, vz);
  }
}

// Per element and group (fluid, walls): sum of v and of |v|^2 in a fixed
// order -- one block per element, each thread striding over the element's
// atoms, then a fixed tree over the threads -- so that the mean removal and
// rescale of k_init_fix give the same velocities on every run.
template <bool DF>
__global__ void __launch_bounds__(256) k_group_sums(BatchDev B) {
  __shared__ double red[8][256];
  const ElemDev& E = B.el[blockIdx.x];
  const long long n = (long long)E.nf + E.nw;
  const int t = threadIdx.x;
  double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (long long l = t; l < n; l += blockDim.x) {
    const long long a = E.atom0 + l;   // still in original order
    const double vx = st_get<DF>(B.st[3], a), vy = st_get<DF>(B.st[4], a), vz = st_get<DF>(B.st[5], a);
    const int g = l < E.nf ? 0 : 4;
    acc[g] += vx; acc[g + 1] += vy; acc[g + 2] += vz; acc[g + 3] += vx * vx + vy * vy + vz * vz;
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) red[k][t] = acc[k];
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (t < h)
#pragma unroll
      for (int k = 0; k < 8; ++k) red[k][t] += red[k][t + h];
    __syncthreads();
  }
  if (t < 8) B.grp[(size_t)(2 * blockIdx.x + t / 4) * kGrpStride + (t & 3)] = red[t][0];
}

// Remove each group's mean velocity, then rescale it to exactly T with
// 3 (N_g - 1) degrees of freedom.
template <bool DF>
__global__ void k_init_fix(BatchDev B, PhysDev P) {
  const long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (a >= B.n_atoms) return;
  const int e = B.atom_el[a];
  const ElemDev& E = B.el[e];
  const int group = B.orig[a] < E.nf ? 0 : 1;
  const double cnt = group == 0 ? (double)E.nf : (double)E.nw;
  const double* g = B.grp + (size_t)(2 * e + group) * kGrpStride;
  const double mx = g[0] / cnt, my = g[1] / cnt, mz = g[2] / cnt;
  double vx = st_get<DF>(B.st[3], a) - mx, vy = st_get<DF>(B.st[4], a) - my, vz = st_get<DF>(B.st[5], a) - mz;
  const double ke2 = P.mass * (g[3] - cnt * (mx * mx + my * my + mz * mz));
  if (group == 1 && P.mode == 1) {       // frozen walls do not move
    vx = vy = vz = 0.0;
  } else if (cnt > 1.0 && ke2 > 0.0) {
    const double s = sqrt(E.T / (ke2 / (3.0 * (cnt - 1.0))));
    vx *= s; vy *= s; vz *= s;
  }
  st_put<DF>(B.st[3], a, vx); st_put<DF>(B.st[4], a, vy); st_put<DF>(B.st[5], a, vz);
}

// Start states from snapshots (elements with warm != 0): overwrite the
// lattice positions and velocities of the fluid and the walls by the
// prepared state; the tether anchors stay the lattice sites.  Runs after
// k_init_fix, while the atoms are still in original order.
template <bool DF>
__global__ void k_apply_warm(BatchDev B) {
  const long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (a >= B.n_atoms) return;
  const ElemDev& E = B.el[B.atom_el[a]];
  if (E.warm == 0) return;
  const double* w = B.warm + 6 * a;
  st_put<DF>(B.st[0], a, w[0]); st_put<DF>(B.st[1], a, w[1]); st_put<DF>(B.st[2], a, w[2]);
  st_put<DF>(B.st[3], a, w[3]); st_put<DF>(B.st[4], a, w[4]); st_put<DF>(B.st[5], a, w[5]);
}

// ---------------------------------------------------------------------------
// Neighbour-list rebuild, step 1: bin every atom into its cell, the counting
// sort's histogram (x and z periodic, y clamped to the edge cells).  The atoms
// of a block are in cell order from the last rebuild, so their new cells span
// a short range: the block counts them in shared memory (slot = rank among
// the block's atoms of that cell), then adds each cell's count to the global
// histogram with one atomic, whose old value is the block's base in the cell.
// A block whose cells span more than kBinCells (the first rebuild, from the
// lattice order) counts in the global histogram directly.  Slots differ from
// run to run either way; k_settle orders each cell's atoms afterwards.
// ---------------------------------------------------------------------------
// With the double-float state an atom already in a reference cell is binned
// from its offset: the new cell is the reference cell plus
// floor(offset / cs + 1/2) per axis (x, z wrapped, y clamped), in FP32.
constexpr int kBinCells = 1024;

template <bool DF>
__global__ void __launch_bounds__(256) k_bin(BatchDev B) {
  __shared__ int s_cnt[kBinCells];
  __shared__ int s_lo, s_hi;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i == 0) atomicAdd(&B.flags[2], 1);
  if (threadIdx.x == 0) { s_lo = 0x7fffffff; s_hi = -1; }
  int c = -1;
  if (i < B.n_atoms) {
    const ElemDev& E = B.el[B.atom_el[i]];
    int ix, iy, iz;
    const int c0 = B.cell[i];
    if (DF && c0 >= 0) {
      int rx, ry, rz;
      cell_coords(E, c0, rx, ry, rz);
      const float ox = df_ld(B.st[0], i).hi, oy = df_ld(B.st[1], i).hi, oz = df_ld(B.st[2], i).hi;
      ix = rx + (int)floorf(fmaf(ox, E.inv_csf[0], 0.5f));
      iy = ry + (int)floorf(fmaf(oy, E.inv_csf[1], 0.5f));
      iz = rz + (int)floorf(fmaf(oz, E.inv_csf[2], 0.5f));
      ix = ix < 0 ? ix + E.nc[0] : (ix >= E.nc[0] ? ix - E.nc[0] : ix);
      iz = iz < 0 ? iz + E.nc[2] : (iz >= E.nc[2] ? iz - E.nc[2] : iz);
      ix = ix < 0 ? 0 : (ix >= E.nc[0] ? E.nc[0] - 1 : ix);
      iz = iz < 0 ? 0 : (iz >= E.nc[2] ? E.nc[2] - 1 : iz);
      iy = iy < 0 ? 0 : (iy >= E.nc[1] ? E.nc[1] - 1 : iy);
    } else {
      double x, y, z;
      abs_position<DF>(B, E, i, x, y, z);
      ix = (int)(x * E.inv_cs[0]); iz = (int)(z * E.inv_cs[2]);
      const double yr = (y - E.ylo) * E.inv_cs[1];
      iy = yr < 0.0 ? 0 : (yr >= (double)E.nc[1] ? E.nc[1] - 1 : (int)yr);
      ix = ix < 0 ? 0 : (ix >= E.nc[0] ? E.nc[0] - 1 : ix);
      iz = iz < 0 ? 0 : (iz >= E.nc[2] ? E.nc[2] - 1 : iz);
    }
    c = (int)(E.cell0 + ((long long)ix * E.nc[1] + iy) * E.nc[2] + iz);
    B.newcell[i] = c;
  }
  __syncthreads();
  if (c >= 0) { atomicMin(&s_lo, c); atomicMax(&s_hi, c); }
  __syncthreads();
  if (s_hi < 0) return;                // no atom in this block
  const int lo = s_lo, range = s_hi - s_lo + 1;
  if (range > kBinCells) {            // whole block: the same lo and hi
    if (c >= 0) B.slot[i] = atomicAdd(&B.ccount[c], 1);
    return;
  }
  for (int r = threadIdx.x; r < range; r += blockDim.x) s_cnt[r] = 0;
  __syncthreads();
  const int rank = c >= 0 ? atomicAdd(&s_cnt[c - lo], 1) : 0;
  __syncthreads();
  for (int r = threadIdx.x; r < range; r += blockDim.x) {
    const int n = s_cnt[r];
    s_cnt[r] = n > 0 ? atomicAdd(&B.ccount[lo + r], n) : 0;   // the block's base in cell lo + r
  }
  __syncthreads();
  if (c >= 0) B.slot[i] = s_cnt[c - lo] + rank;
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

// Step 3: move every atom to a slot of its cell; positions become offsets
// from the new reference cell's centre, anchors likewise (minimum image).
// With the double-float state an atom that had a reference cell is rebased
// by the cell step between the two centres (-delta * cs per axis, delta
// wrapped to the nearest image in x and z), in FP32 arithmetic.
template <typename PT>
__global__ void __launch_bounds__(256) k_permute(BatchDev B) {
  constexpr bool DF = sizeof(PT) == 16;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= B.n_atoms) return;
  const ElemDev& E = B.el[B.atom_el[i]];
  const int c = B.newcell[i];
  const long long dst = (long long)B.cstart[c] + B.slot[i];
  const int l = B.orig[i];
  const bool wall = l >= E.nf;
  const int c0 = B.cell[i];
  if constexpr (DF) {
    if (c0 >= 0) {
      int rx, ry, rz, jx, jy, jz;
      cell_coords(E, c0, rx, ry, rz);
      cell_coords(E, c, jx, jy, jz);
      int dx = jx - rx, dz = jz - rz;
      const int dy = jy - ry;
      if (2 * dx > E.nc[0]) dx -= E.nc[0]; else if (2 * dx < -E.nc[0]) dx += E.nc[0];
      if (2 * dz > E.nc[2]) dz -= E.nc[2]; else if (2 * dz < -E.nc[2]) dz += E.nc[2];
      const dfl sx = df_mul(-(float)dx, dfl{E.csf[0], E.cs_lo[0]});
      const dfl sy = df_mul(-(float)dy, dfl{E.csf[1], E.cs_lo[1]});
      const dfl sz = df_mul(-(float)dz, dfl{E.csf[2], E.cs_lo[2]});
      const dfl ox = df_add(df_ld(B.st[0], i), sx), oy = df_add(df_ld(B.st[1], i), sy),
                oz = df_add(df_ld(B.st[2], i), sz);
      df_st(B.st2[0], dst, ox); df_st(B.st2[1], dst, oy); df_st(B.st2[2], dst, oz);
      if (wall) {
        df_st(B.st2[6], dst, df_add(df_ld(B.st[6], i), sx));
        df_st(B.st2[7], dst, df_add(df_ld(B.st[7], i), sy));
        df_st(B.st2[8], dst, df_add(df_ld(B.st[8], i), sz));
      } else {
        df_st(B.st2[6], dst, dfl{0.f, 0.f}); df_st(B.st2[7], dst, dfl{0.f, 0.f}); df_st(B.st2[8], dst, dfl{0.f, 0.f});
      }
    }
  }
  if (!DF || c0 < 0) {
    double x, y, z;
    abs_position<DF>(B, E, i, x, y, z);
    double cx, cy, cz;
    cell_center(E, c, cx, cy, cz);
    const double ox = x - cx, oy = y - cy, oz = z - cz;
    double ax = 0.0, ay = 0.0, az = 0.0;
    if (wall) {
      ax = st_get<DF>(B.st[6], i); ay = st_get<DF>(B.st[7], i); az = st_get<DF>(B.st[8], i);
      if (c0 >= 0) {
        double px, py, pz;
        cell_center(E, c0, px, py, pz);
        ax += px; ay += py; az += pz;
      }
      ax = min_image(ax - cx, E.Lx);
      ay = ay - cy;
      az = min_image(az - cz, E.Lz);
    }
    st_put<DF>(B.st2[0], dst, ox); st_put<DF>(B.st2[1], dst, oy); st_put<DF>(B.st2[2], dst, oz);
    st_put<DF>(B.st2[6], dst, ax); st_put<DF>(B.st2[7], dst, ay); st_put<DF>(B.st2[8], dst, az);
  }
  // velocities move as raw 8-byte words in either representation
  B.st2[3][dst] = B.st[3][i]; B.st2[4][dst] = B.st[4][i]; B.st2[5][dst] = B.st[5][i];
  B.orig2[dst] = l;
  B.cell2[dst] = c;
}

// Step 4: settle each cell's atoms in the order of their original index (the
// binning atomics leave them in arbitrary order) while copying the permuted
// state back, so that the sorted order, the lists and every later summation
// order are the same on every run.  The pair-force input positions (both
// buffers: the next force evaluation reads one of them) and the rebuild-time
// copy for the skin check are written at the settled slot.
template <typename PT>
__global__ void __launch_bounds__(256) k_settle(BatchDev B) {
  constexpr bool DF = sizeof(PT) == 16;
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= B.n_atoms) return;
  const int c = B.cell2[p];
  const int start = B.cstart[c], n = B.csize[c];
  const int me = B.orig2[p];
  int rank = 0;
  for (int q = start; q < start + n; ++q) rank += B.orig2[q] < me ? 1 : 0;
  const long long f = (long long)start + rank;
#pragma unroll
  for (int k = 0; k < 9; ++k) B.st[k][f] = B.st2[k][p];
  B.orig[f] = me;
  B.cell[f] = c;
  const ElemDev& E = B.el[B.atom_el[p]];
  const bool wall = me >= E.nf;
  float fx, fy, fz;
  if constexpr (DF) {
    fx = df_ld(B.st2[0], p).hi; fy = df_ld(B.st2[1], p).hi; fz = df_ld(B.st2[2], p).hi;
    const float4 q = make_float4(fx, fy, fz, wall ? 1.0f : 0.0f);
    static_cast<float4*>(B.posb[0])[f] = q;
    static_cast<float4*>(B.posb[1])[f] = q;
  } else {
    const double ox = B.st2[0][p], oy = B.st2[1][p], oz = B.st2[2][p];
    static_cast<Pos64*>(B.posb[0])[f] = Pos64{ox, oy, oz, wall ? 1.0 : 0.0};
    fx = (float)ox; fy = (float)oy; fz = (float)oz;
  }
  B.pbuild[f] = make_float4(fx, fy, fz, 0.0f);
}

// Step 5: Verlet lists.  Lists are stored in groups of four entries,
// [k / 4][atom][4] (a warp's 16-byte loads coalesce); the last group is
// padded with an entry that is always beyond r_c (the atom itself one cell
// over in x), so readers never test the count inside a group.
// A list entry: the neighbour's index within its element (bits 0-25) and
// its cell's place among the 27 neighbour cells, k = 9 (dx + 1) + 3 (dy + 1)
// + (dz + 1) (bits 26-30).  The pad entry points at the atom itself shifted
// by one cell in x (k = 22): its distance, the cell side, exceeds r_c.
constexpr unsigned kCodePad = 22u;
__device__ __forceinline__ unsigned pad_entry(long long i, const ElemDev& E) {
  return (unsigned)(i - E.atom0) | (kCodePad << 26);
}

// Ballot list build.  The candidates of a cell are gathered from its 27
// neighbour cells: the atoms within r_c + skin of the bounding box of the
// cell's own atoms (any other atom is out of range of every atom of the
// cell), each shifted into the home cell's frame with its list entry in w.
// The gather walks the 27 cells as one flat index range (lane k of a warp
// holds cell k's start, size and shift; a lane finds its cell by a binary
// search over the size prefix), so consecutive chunks load independently.
// The cell's atoms are then taken octant by octant (sign of the offset from
// the cell centre): the buffer is filtered once more against the octant's
// box into an index list, about half as long, and for each atom of the
// octant the 32 lanes test 32 listed candidates at once; accepted entries
// go to the atom's list at its running count plus their rank in the ballot
// mask.  Entries keep the candidate order, the neighbour cells in
// (dx, dy, dz) order.  A neighbourhood larger than the buffer is swept in
// several passes; the running counts then persist in nlist between passes.
// Works from pbuild (float4), so one kernel serves both pair-force
// precisions.  The same atom never tests itself: its own candidate is at
// distance exactly 0 (the zero shift adds 0), which the range test
// 0 < d^2 < (r_c + skin)^2 excludes.
// What one warp knows of its cell for the ballot build: the bounding box of
// the cell's atoms and the 27-entry neighbour table with its size prefix.
struct BallotCell {
  float lx, ly, lz, hx, hy, hz;   // bounding box of the cell's own atoms
  int nst, nsz;                   // lane k < 27: start and size of neighbour cell k
  unsigned ncode;                 // lane k: code of neighbour cell k (k << 26)
  float nsx, nsy, nsz_f;          // lane k: shift of neighbour cell k in length units
  int pre, excl, total;           // inclusive / exclusive size prefix, total candidates
};

__device__ __forceinline__ void ballot_cell(const BatchDev& B, const ElemDev& E, long long cell, int s0, int n0,
                                            int lane, BallotCell& C) {
  int cx, cy, cz;
  cell_coords(E, cell, cx, cy, cz);
  const int ncx = E.nc[0], ncy = E.nc[1], ncz = E.nc[2];
  const float4* pb = B.pbuild;
  float lx = 3.0e38f, ly = 3.0e38f, lz = 3.0e38f, hx = -3.0e38f, hy = -3.0e38f, hz = -3.0e38f;
  for (int a = lane; a < n0; a += 32) {
    const float4 p = pb[s0 + a];
    lx = fminf(lx, p.x); ly = fminf(ly, p.y); lz = fminf(lz, p.z);
    hx = fmaxf(hx, p.x); hy = fmaxf(hy, p.y); hz = fmaxf(hz, p.z);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lx = fminf(lx, __shfl_xor_sync(kFull, lx, o)); ly = fminf(ly, __shfl_xor_sync(kFull, ly, o));
    lz = fminf(lz, __shfl_xor_sync(kFull, lz, o)); hx = fmaxf(hx, __shfl_xor_sync(kFull, hx, o));
    hy = fmaxf(hy, __shfl_xor_sync(kFull, hy, o)); hz = fmaxf(hz, __shfl_xor_sync(kFull, hz, o));
  }
  C.lx = lx; C.ly = ly; C.lz = lz; C.hx = hx; C.hy = hy; C.hz = hz;
  // neighbour table: lane k < 27 holds cell k = 9 (dx+1) + 3 (dy+1) + (dz+1)
  C.nst = 0; C.nsz = 0; C.ncode = 0;
  C.nsx = 0.f; C.nsy = 0.f; C.nsz_f = 0.f;
  if (lane < 27) {
    const int dx = lane / 9 - 1, dy = (lane / 3) % 3 - 1, dz = lane % 3 - 1;
    const int jy = cy + dy;
    if (jy >= 0 && jy < ncy) {
      int jx = cx + dx, jz = cz + dz;
      jx = jx < 0 ? jx + ncx : (jx >= ncx ? jx - ncx : jx);
      jz = jz < 0 ? jz + ncz : (jz >= ncz ? jz - ncz : jz);
      const long long c2 = E.cell0 + ((long long)jx * ncy + jy) * ncz + jz;
      C.nst = B.cstart[c2];
      C.nsz = B.csize[c2];
    }
    C.ncode = (unsigned)lane << 26;
    C.nsx = (float)dx * E.csf[0]; C.nsy = (float)dy * E.csf[1]; C.nsz_f = (float)dz * E.csf[2];
  }
  int pre = C.nsz;   // inclusive prefix of the sizes over the lanes
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(kFull, pre, o);
    if (lane >= o) pre += t;
  }
  C.pre = pre;
  C.excl = pre - C.nsz;
  C.total = __shfl_sync(kFull, pre, 31);
}

// Candidate f of the flat neighbour range (f < C.total), shifted into the
// home cell's frame with its list entry in w, and whether it lies within
// sqrt(rl2) of the cell's box.  Lanes with f >= C.total return far4, not kept.
__device__ __forceinline__ bool ballot_candidate(const float4* pb, const ElemDev& E, const BallotCell& C, int f,
                                                 float rl2, float4 far4, float4& out) {
  int k = 0;
#pragma unroll
  for (int st = 16; st > 0; st >>= 1) {
    const int pv = __shfl_sync(kFull, C.pre, k + st - 1);
    if (pv <= f) k += st;
  }
  const int jn = __shfl_sync(kFull, C.nst, k), je = __shfl_sync(kFull, C.excl, k);
  const unsigned code = __shfl_sync(kFull, C.ncode, k);
  const float ox = __shfl_sync(kFull, C.nsx, k), oy = __shfl_sync(kFull, C.nsy, k),
              oz = __shfl_sync(kFull, C.nsz_f, k);
  const bool valid = f < C.total;
  const int j = jn + (f - je);
  float4 p = valid ? pb[j] : far4;
  p.x += ox; p.y += oy; p.z += oz;
  const float ex = fmaxf(fmaxf(C.lx - p.x, p.x - C.hx), 0.0f);
  const float ey = fmaxf(fmaxf(C.ly - p.y, p.y - C.hy), 0.0f);
  const float ez = fmaxf(fmaxf(C.lz - p.z, p.z - C.hz), 0.0f);
  out = make_float4(p.x, p.y, p.z, __uint_as_float((unsigned)(j - E.atom0) | code));
  return valid && ex * ex + ey * ey + ez * ez < rl2;
}

// One warp's share of the list sweep over a gathered buffer cbuf[0, mpad)
// (cbuf[pad_idx] = far4): the octants o0, o0 + ostep, ... of the cell's
// atoms, each with its own filtered index list in oidx.  `first` / `last`
// mark the first and the last pass over the neighbourhood.
__device__ __forceinline__ void ballot_sweep(const BatchDev& B, const ElemDev& E, int e, const BallotCell& C,
                                             long long s0, int n0, const float4* cbuf, unsigned short* oidx,
                                             int mpad, int pad_idx, int o0, int ostep, bool first, bool last,
                                             float rl2, int lane) {
  const unsigned rl2u = __float_as_uint(rl2) - 1u;
  const unsigned lt = (1u << lane) - 1u;
  const long long N4 = B.n_atoms * 4;
  const int cap = B.list_cap;
  unsigned* L = B.list;
  const float4* pb = B.pbuild;
  for (int base = 0; base < n0; base += 32) {
    const int na = n0 - base < 32 ? n0 - base : 32;
    const float4 mine = lane < na ? pb[s0 + base + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int oct = lane < na ? ((mine.x > 0.f ? 1 : 0) | (mine.y > 0.f ? 2 : 0) | (mine.z > 0.f ? 4 : 0)) : 8;
    for (int o = o0; o < 8; o += ostep) {
      unsigned mo = __ballot_sync(kFull, oct == o);
      if (mo == 0) continue;
      // the octant's box: the cell's box split at the centre
      const float bxl = (o & 1) ? fmaxf(C.lx, 0.f) : C.lx, bxh = (o & 1) ? C.hx : fminf(C.hx, 0.f);
      const float byl = (o & 2) ? fmaxf(C.ly, 0.f) : C.ly, byh = (o & 2) ? C.hy : fminf(C.hy, 0.f);
      const float bzl = (o & 4) ? fmaxf(C.lz, 0.f) : C.lz, bzh = (o & 4) ? C.hz : fminf(C.hz, 0.f);
      int q = 0;
      for (int c = 0; c < mpad; c += 32) {
        const float4 p = cbuf[c + lane];
        const float ex = fmaxf(fmaxf(bxl - p.x, p.x - bxh), 0.0f);
        const float ey = fmaxf(fmaxf(byl - p.y, p.y - byh), 0.0f);
        const float ez = fmaxf(fmaxf(bzl - p.z, p.z - bzh), 0.0f);
        const bool keep = ex * ex + ey * ey + ez * ez < rl2;
        const unsigned mk = __ballot_sync(kFull, keep);
        if (keep) oidx[q + __popc(mk & lt)] = (unsigned short)(c + lane);
        q += __popc(mk);
      }
      const int qpad = (q + 31) & ~31;
      if (q + lane < qpad) oidx[q + lane] = (unsigned short)pad_idx;
      __syncwarp();
      while (mo) {
        const int a = __ffs(mo) - 1;
        mo &= mo - 1;
        const long long i = s0 + base + a;
        const float mx = __shfl_sync(kFull, mine.x, a), my = __shfl_sync(kFull, mine.y, a),
                    mz = __shfl_sync(kFull, mine.z, a);
        int cnt = first ? 0 : B.nlist[i];
        unsigned* Li = L + i * 4;
#pragma unroll 2
        for (int c = 0; c < qpad; c += 32) {
          const float4 cq = cbuf[oidx[c + lane]];
          const float ax = mx - cq.x, ay = my - cq.y, az = mz - cq.z;
          const float d2 = ax * ax + ay * ay + az * az;
          const bool take = __float_as_uint(d2) - 1u < rl2u;   // 0 < d2 < rl2
          const unsigned mk = __ballot_sync(kFull, take);
          const int kk = cnt + __popc(mk & lt);
          if (take && kk < cap) Li[(long long)(kk >> 2) * N4 + (kk & 3)] = __float_as_uint(cq.w);
          cnt += __popc(mk);
        }
        if (last) {
          // pad the last partial group with an entry beyond r_c
          const int kk = cnt + lane;
          if (cnt < cap && lane < ((4 - (cnt & 3)) & 3))
            Li[(long long)(kk >> 2) * N4 + (kk & 3)] = pad_entry(i, E);
          if (lane == 0) {
            if (cnt > cap) atomicMin(&B.status[e], kStOverflow);
            B.nlist[i] = cnt < cap ? cnt : cap;
          }
        } else if (lane == 0) {
          B.nlist[i] = cnt;
        }
      }
      __syncwarp();
    }
  }
}

// One block of kBlkWarps warps per cell.  The warps gather together, two
// chunks of 32 candidates each per round (warp w takes chunks w and
// kBlkWarps + w of the round's 2 kBlkWarps); a prefix over the warps'
// ballot counts places the kept candidates in flat index order.  Warp w then
// sweeps the octants w, w + kBlkWarps, ... with its own index list.  Each
// atom is swept by one warp over the candidates in a fixed order, so its
// list does not depend on scheduling.  Four warps per cell (against one)
// keep a cell on its SM for about a quarter of the time, so more warps are
// resident and the launch's tail is shorter.
constexpr int kBlkWarps = 4;
constexpr int kBlkCap = 1024;     // buffered candidates per block
constexpr int kBlkSmem = (kBlkCap + 32) * 16 + kBlkWarps * (kBlkCap + 32) * 2;

__global__ void __launch_bounds__(kBlkWarps * 32, 6) k_build_ballot_blk(BatchDev B, PhysDev P) {
  extern __shared__ __align__(16) unsigned char bsm[];
  __shared__ int s_cnt[2][2 * kBlkWarps];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long cell = blockIdx.x;
  if (cell >= B.n_cells) return;
  const int s0 = B.cstart[cell], n0 = B.csize[cell];
  if (n0 == 0) return;
  float4* cbuf = reinterpret_cast<float4*>(bsm);
  unsigned short* oidx = reinterpret_cast<unsigned short*>(cbuf + kBlkCap + 32) + wid * (kBlkCap + 32);
  const int e = B.cell_el[cell];
  const ElemDev& E = B.el[e];
  BallotCell C;
  ballot_cell(B, E, cell, s0, n0, lane, C);
  const float rl2 = P.rl2f;
  const float4 far4 = make_float4(1.0e18f, 1.0e18f, 1.0e18f, 0.0f);
  const unsigned lt = (1u << lane) - 1u;
  if (threadIdx.x == 0) cbuf[kBlkCap] = far4;   // the padding target of the index lists
  int f0 = 0, round = 0;
  bool first = true, last = false;
  while (!last) {
    // gather up to kBlkCap candidates; f0, m and round are the same in every warp
    int m = 0;
    for (; f0 < C.total && m + 64 * kBlkWarps <= kBlkCap; f0 += 64 * kBlkWarps, ++round) {
      float4 pa, pc;
      const bool ka = ballot_candidate(B.pbuild, E, C, f0 + 32 * wid + lane, rl2, far4, pa);
      const bool kc = ballot_candidate(B.pbuild, E, C, f0 + 32 * (kBlkWarps + wid) + lane, rl2, far4, pc);
      const unsigned ma = __ballot_sync(kFull, ka), mc = __ballot_sync(kFull, kc);
      int* cnt = s_cnt[round & 1];   // two slots: a slot is rewritten only two barriers later
      if (lane == 0) {
        cnt[wid] = __popc(ma);
        cnt[kBlkWarps + wid] = __popc(mc);
      }
      __syncthreads();
      int offa = m, offc = m, tot = 0;
#pragma unroll
      for (int v = 0; v < kBlkWarps; ++v) {
        const int a = cnt[v], c = cnt[kBlkWarps + v];
        offa += v < wid ? a : 0;
        offc += a + (v < wid ? c : 0);
        tot += a + c;
      }
      if (ka) cbuf[offa + __popc(ma & lt)] = pa;
      if (kc) cbuf[offc + __popc(mc & lt)] = pc;
      m += tot;
    }
    last = f0 >= C.total;
    const int mpad = (m + 31) & ~31;
    if (wid == 0 && m + lane < mpad) cbuf[m + lane] = far4;
    __syncthreads();
    ballot_sweep(B, E, e, C, s0, n0, cbuf, oidx, mpad, kBlkCap, wid, kBlkWarps, first, last, rl2, lane);
    __syncthreads();   // the next pass refills cbuf
    first = false;
  }
}

// ---------------------------------------------------------------------------
// LJ pair forces over the Verlet lists: one thread per atom (cell order, so
// a warp's neighbours are shared in L1).  Eq. LJ truncated at r_c, energy
// shifted by U(r_c) per pair type.  The displacement is formed from
// cell-centre offsets: d = (p_i - p_j) - delta * cs, delta in {-1, 0, 1}^3
// from the entry's cell code, so FP32 only ever rounds numbers below ~3.
// Writes the LJ force, the x-virial share of fluid atoms (half per pair) and,
// with ENERGY, half the shifted pair energy per atom.
// ---------------------------------------------------------------------------
// Approximate reciprocal (PTX rcp.approx.ftz.f32: one MUFU op, <= 1 ulp).
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// The unit cell shifts (dx, dy, dz) of the 27 neighbour-cell codes, one
// array per axis in shared memory (27 words: any mix of codes in a warp
// reads without bank conflicts).  Every thread of the block calls it; the
// caller synchronises before the first use.
struct ShiftTab {
  float d[3][32];
};
__device__ __forceinline__ void shift_tab_init(ShiftTab& t) {
  for (int k = threadIdx.x; k < 96; k += blockDim.x) {
    const int a = k >> 5, c = k & 31;
    const int v = c < 27 ? (a == 0 ? c / 9 : (a == 1 ? (c / 3) % 3 : c % 3)) - 1 : 0;
    t.d[a][c] = (float)v;
  }
}

template <typename PT, typename T, bool UNIFORM, bool ENERGY>
struct PairAcc {
  T fx = 0, fy = 0, fz = 0, w = 0, u = 0;
  __device__ __forceinline__ void add(const PT& me, const PT& o, unsigned ent, T csx, T csy, T csz, int spi,
                                      T rc2, const T (&eps)[3], const T (&sig2)[3], const PhysDev& P,
                                      const ShiftTab& tab) {
    const unsigned code = ent >> 26;
    const float sx = tab.d[0][code], sy = tab.d[1][code], sz = tab.d[2][code];
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
    if constexpr (sizeof(T) == 4) inv2 = rcp_approx(r2); else inv2 = 1.0 / r2;
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
    // F/r = 24 eps inv2 s6 (2 s6 - 1) = eps inv2 s6 (48 s6 - 24)
    T fs = e_ * inv2 * s6 * ((T)48 * s6 - (T)24);
    bool in = r2 < rc2;
    if constexpr (!UNIFORM) in = in && P.active[t];
    fs = in ? fs : (T)0;
    const T tx = fs * ddx;
    fx += tx; fy += fs * ddy; fz += fs * ddz;
    w += tx * ddx;
    if (ENERGY) u += in ? ((T)4 * e_ * (s6 * s6 - s6) - (T)P.eshift[t]) : (T)0;
  }
};

// Pair forces on atom i over its list, positions from pos (this step's
// buffer); spi = the atom's species.
template <typename PT, typename T, bool UNIFORM, bool ENERGY>
__device__ __forceinline__ PairAcc<PT, T, UNIFORM, ENERGY> pair_force(const BatchDev& B, const PhysDev& P,
                                                                      long long i, const PT* pos, int& spi,
                                                                      const ShiftTab& tab) {
  const ElemDev& E = B.el[__ldcg(B.atom_el + i)];
  const PT me = pos[i];
  const T csx = (T)E.cs[0], csy = (T)E.cs[1], csz = (T)E.cs[2];
  const PT* posj = pos + E.atom0;
  const int n = __ldcg(B.nlist + i);
  const long long N = B.n_atoms;
  T rc2, eps[3], sig2[3];
  if constexpr (sizeof(T) == 4) {
    rc2 = P.rc2f;
    for (int t = 0; t < 3; ++t) { eps[t] = P.epsf[t]; sig2[t] = P.sig2f[t]; }
  } else {
    rc2 = P.rc2;
    for (int t = 0; t < 3; ++t) { eps[t] = P.eps[t]; sig2[t] = P.sig2[t]; }
  }
  spi = me.w != (T)0 ? 1 : 0;
  PairAcc<PT, T, UNIFORM, ENERGY> acc;
  const uint4* L4 = reinterpret_cast<const uint4*>(B.list) + i;
  const int ng = (n + 3) >> 2;
  int k = 0;
  // two groups of four entries per iteration: eight gathers in flight
  // (loading the next iteration's list groups ahead costs registers the
  // persistent kernel does not have: measured slower)
  for (; k + 1 < ng; k += 2) {
    const uint4 e = ld_list4(L4 + (long long)k * N);
    const uint4 f = ld_list4(L4 + (long long)(k + 1) * N);
    const PT o0 = posj[e.x & kJMask], o1 = posj[e.y & kJMask], o2 = posj[e.z & kJMask], o3 = posj[e.w & kJMask];
    const PT o4 = posj[f.x & kJMask], o5 = posj[f.y & kJMask], o6 = posj[f.z & kJMask], o7 = posj[f.w & kJMask];
    acc.add(me, o0, e.x, csx, csy, csz, spi, rc2, eps, sig2, P, tab);
    acc.add(me, o1, e.y, csx, csy, csz, spi, rc2, eps, sig2, P, tab);
    acc.add(me, o2, e.z, csx, csy, csz, spi, rc2, eps, sig2, P, tab);
    acc.add(me, o3, e.w, csx, csy, csz, spi, rc2, eps, sig2, P, tab);
    acc.add(me, o4, f.x, csx, csy, csz, spi, rc2, eps, sig2, P, tab);
    acc.add(me, o5, f.y, csx, csy, csz, spi, rc2, eps, sig2, P, tab);
    acc.add(me, o6, f.z, csx, csy, csz, spi, rc2, eps, sig2, P, tab);
    acc.add(me, o7, f.w, csx, csy, csz, spi, rc2, eps, sig2, P, tab);
  }
  if (k < ng) {
    const uint4 e = ld_list4(L4 + (long long)k * N);
    const PT o0 = posj[e.x & kJMask], o1 = posj[e.y & kJMask], o2 = posj[e.z & kJMask], o3 = posj[e.w & kJMask];
    acc.add(me, o0, e.x, csx, csy, csz, spi, rc2, eps, sig2, P, tab);
    acc.add(me, o1, e.y, csx, csy, csz, spi, rc2, eps, sig2, P, tab);
    acc.add(me, o2, e.z, csx, csy, csz, spi, rc2, eps, sig2, P, tab);
    acc.add(me, o3, e.w, csx, csy, csz, spi, rc2, eps, sig2, P, tab);
  }
  return acc;
}

// ---------------------------------------------------------------------------
// FP32 pair forces with packed two-lane arithmetic.  The SMs of this GPU
// family execute add, mul and fma on two FP32 values held in one 64-bit
// register pair (PTX .f32x2) as one instruction.  The loop below takes its
// list entries two at a time and evaluates both pair terms with each packed
// instruction; per pair the arithmetic is PairAcc's (Eq. LJ): d = (p_i - p_j)
// - delta * cs, r^2, 1/r^2 by rcp.approx, F/r = eps (1/r^2) s^6 (48 s^6 - 24)
// with s^2 = sig^2 / r^2, and 1/r^2 set to zero beyond r_c or for an inactive
// pair type, so that such an entry adds nothing.
// With TPA > 1, TPA consecutive lanes share an atom: lane `sub` of the group
// takes the list groups sub, sub + TPA, ... and the sums are combined by
// shuffles, so every lane of the group returns the atom's totals.
// ---------------------------------------------------------------------------
typedef unsigned long long f2x;   // two FP32 values: bits 0-31 and 32-63

__device__ __forceinline__ f2x f2_pk(float lo, float hi) {
  f2x r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_upk(f2x v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2x f2_add(f2x a, f2x b) {
  f2x r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2x f2_mul(f2x a, f2x b) {
  f2x r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2x f2_fma(f2x a, f2x b, f2x c) {
  f2x r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// Per-atom constants of the packed pair loop: the negated cell side in both
// lanes, and for the neighbour species 0 / 1 the pair type's eps, sig^2,
// energy shift and whether it interacts.
struct PairConst {
  f2x ncsx, ncsy, ncsz, cmh;   // -cs per axis; (-1/2, -1/2)
  float rc2;
  float eps0, eps1, sig0, sig1, esh0, esh1;
  bool act0, act1;
};

struct PairSum {
  float fx, fy, fz, w, u;
};

template <bool UNIFORM, bool ENERGY>
struct PairAcc2 {
  f2x fx = 0ull, fy = 0ull, fz = 0ull, w = 0ull;   // all-zero bits: (0, 0)
  float u = 0.f;
  __device__ __forceinline__ void add(const float4& me, const float4& oa, const float4& ob, unsigned ea,
                                      unsigned eb, const PairConst& c, const ShiftTab& tab) {
    const unsigned ka = ea >> 26, kb = eb >> 26;
    const f2x dx = f2_fma(f2_pk(tab.d[0][ka], tab.d[0][kb]), c.ncsx, f2_pk(me.x - oa.x, me.x - ob.x));
    const f2x dy = f2_fma(f2_pk(tab.d[1][ka], tab.d[1][kb]), c.ncsy, f2_pk(me.y - oa.y, me.y - ob.y));
    const f2x dz = f2_fma(f2_pk(tab.d[2][ka], tab.d[2][kb]), c.ncsz, f2_pk(me.z - oa.z, me.z - ob.z));
    const f2x r2 = f2_fma(dz, dz, f2_fma(dy, dy, f2_mul(dx, dx)));
    float r2a, r2b;
    f2_upk(r2, r2a, r2b);
    bool ina = r2a < c.rc2, inb = r2b < c.rc2;
    float sga = 1.f, sgb = 1.f, epa = 1.f, epb = 1.f, sha = 0.f, shb = 0.f;
    if constexpr (!UNIFORM) {
      const bool wa = oa.w != 0.f, wb = ob.w != 0.f;
      ina = ina && (wa ? c.act1 : c.act0);
      inb = inb && (wb ? c.act1 : c.act0);
      sga = wa ? c.sig1 : c.sig0; sgb = wb ? c.sig1 : c.sig0;
      epa = wa ? c.eps1 : c.eps0; epb = wb ? c.eps1 : c.eps0;
      if (ENERGY) { sha = wa ? c.esh1 : c.esh0; shb = wb ? c.esh1 : c.esh0; }
    } else if (ENERGY) {
      sha = c.esh0; shb = c.esh0;
    }
    const float ia = ina ? rcp_approx(r2a) : 0.f, ib = inb ? rcp_approx(r2b) : 0.f;
    const f2x inv2 = f2_pk(ia, ib);
    const f2x s2 = UNIFORM ? inv2 : f2_mul(f2_pk(sga, sgb), inv2);
    const f2x s6 = f2_mul(f2_mul(s2, s2), s2);
    // F/r over 48: eps (1/r^2) s^6 (s^6 - 1/2); the sums are scaled by 48 at the end
    f2x fs = f2_mul(f2_mul(inv2, s6), f2_add(s6, c.cmh));
    if constexpr (!UNIFORM) fs = f2_mul(fs, f2_pk(epa, epb));
    const f2x tx = f2_mul(fs, dx);
    fx = f2_add(fx, tx);
    fy = f2_fma(fs, dy, fy);
    fz = f2_fma(fs, dz, fz);
    w = f2_fma(tx, dx, w);
    if constexpr (ENERGY) {
      float s6a, s6b;
      f2_upk(s6, s6a, s6b);
      u += ina ? 4.f * epa * (s6a * s6a - s6a) - sha : 0.f;
      u += inb ? 4.f * epb * (s6b * s6b - s6b) - shb : 0.f;
    }
  }
};

template <int TPA>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = 1; o < TPA; o <<= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

template <bool UNIFORM, bool ENERGY, int TPA>
__device__ __forceinline__ PairSum pair_force_f32(const BatchDev& B, const PhysDev& P, long long i, int sub,
                                                  const float4* pos, int& spi, const ShiftTab& tab) {
  PairAcc2<UNIFORM, ENERGY> acc;
  int n = 0;
  if (i < B.n_atoms) {
    const ElemDev& E = B.el[__ldcg(B.atom_el + i)];
    const float4 me = pos[i];
    const float4* posj = pos + E.atom0;
    n = __ldcg(B.nlist + i);
    spi = me.w != 0.f ? 1 : 0;
    PairConst c;
    const float csx = E.csf[0], csy = E.csf[1], csz = E.csf[2];
    c.ncsx = f2_pk(-csx, -csx); c.ncsy = f2_pk(-csy, -csy); c.ncsz = f2_pk(-csz, -csz);
    c.cmh = f2_pk(-0.5f, -0.5f);
    c.rc2 = P.rc2f;
    c.eps0 = P.epsf[spi]; c.eps1 = P.epsf[spi + 1];
    c.sig0 = P.sig2f[spi]; c.sig1 = P.sig2f[spi + 1];
    c.esh0 = (float)P.eshift[spi]; c.esh1 = (float)P.eshift[spi + 1];
    c.act0 = P.active[spi] != 0; c.act1 = P.active[spi + 1] != 0;
    const uint4* L4 = reinterpret_cast<const uint4*>(B.list) + i;
    const long long N = B.n_atoms;
    const int ng = (n + 3) >> 2;
    int k = sub;
    // two groups of four entries per iteration: eight gathers in flight
    for (; k + TPA < ng; k += 2 * TPA) {
      const uint4 e = ld_list4(L4 + (long long)k * N);
      const uint4 f = ld_list4(L4 + (long long)(k + TPA) * N);
      const float4 o0 = posj[e.x & kJMask], o1 = posj[e.y & kJMask], o2 = posj[e.z & kJMask],
                   o3 = posj[e.w & kJMask];
      const float4 o4 = posj[f.x & kJMask], o5 = posj[f.y & kJMask], o6 = posj[f.z & kJMask],
                   o7 = posj[f.w & kJMask];
      acc.add(me, o0, o1, e.x, e.y, c, tab);
      acc.add(me, o2, o3, e.z, e.w, c, tab);
      acc.add(me, o4, o5, f.x, f.y, c, tab);
      acc.add(me, o6, o7, f.z, f.w, c, tab);
    }
    if (k < ng) {
      const uint4 e = ld_list4(L4 + (long long)k * N);
      const float4 o0 = posj[e.x & kJMask], o1 = posj[e.y & kJMask], o2 = posj[e.z & kJMask],
                   o3 = posj[e.w & kJMask];
      acc.add(me, o0, o1, e.x, e.y, c, tab);
      acc.add(me, o2, o3, e.z, e.w, c, tab);
    }
  }
  float ax, bx, ay, by, az, bz, aw, bw;
  f2_upk(acc.fx, ax, bx); f2_upk(acc.fy, ay, by); f2_upk(acc.fz, az, bz); f2_upk(acc.w, aw, bw);
  PairSum r{48.f * (ax + bx), 48.f * (ay + by), 48.f * (az + bz), 48.f * (aw + bw), acc.u};
  if constexpr (TPA > 1) {
    r.fx = group_sum<TPA>(r.fx); r.fy = group_sum<TPA>(r.fy); r.fz = group_sum<TPA>(r.fz);
    r.w = group_sum<TPA>(r.w);
    if (ENERGY) r.u = group_sum<TPA>(r.u);
  }
  return r;
}

// Pair forces of step *step_base + k into fx, fy, fz (+ virial share, energy).
template <typename PT, typename T, bool UNIFORM, bool ENERGY>
__global__ void __launch_bounds__(128) k_force(BatchDev B, PhysDev P, int k) {
  __shared__ ShiftTab tab;
  shift_tab_init(tab);
  __syncthreads();
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= B.n_atoms) return;
  const long long s = *B.step_base + k;
  int spi = 0;
  T afx, afy, afz, aw, au;
  if constexpr (sizeof(T) == 4) {
    const PairSum acc =
        pair_force_f32<UNIFORM, ENERGY, 1>(B, P, i, 0, static_cast<const float4*>(B.posb[s & 1]), spi, tab);
    afx = acc.fx; afy = acc.fy; afz = acc.fz; aw = acc.w; au = acc.u;
  } else {
    const PairAcc<PT, T, UNIFORM, ENERGY> acc =
        pair_force<PT, T, UNIFORM, ENERGY>(B, P, i, static_cast<const PT*>(B.posb[s & 1]), spi, tab);
    afx = acc.fx; afy = acc.fy; afz = acc.fz; aw = acc.w; au = acc.u;
  }
  static_cast<T*>(B.fx)[i] = afx;
  static_cast<T*>(B.fy)[i] = afy;
  static_cast<T*>(B.fz)[i] = afz;
  static_cast<T*>(B.wxx)[i] = spi == 0 ? (T)0.5 * aw : (T)0;
  if (ENERGY) static_cast<T*>(B.epot)[i] = (T)0.5 * au;
}

// ---------------------------------------------------------------------------
// Fused integration kernel, one thread per atom.  With s the step started:
//   kFinish  completes step s-1: v = u + dt/(2m) F(x), samples it;
//   kStage1  first stage of step s: fluid velocity-Verlet half kick + drift,
//            tethered wall atoms G-JF (Gronbech-Jensen & Farago 2013);
// then publishes the pair-force input position and checks the list skin.
// F(x) = LJ (force kernel) + body force g on fluid atoms (Eq. momentumEq) +
// tether -k (r - r0) on wall atoms.  Between launches a fluid atom stores the
// half-step velocity u; when both phases run, the two half kicks with the
// same force are one update u <- u + dt F/m, and the full-step velocity is
// formed only where it is sampled.  Frozen-wall elements (FROZEN) with the
// Berendsen thermostat split a step over two launches (kTzSum, kTzApply).
template <typename FT, typename PT, bool FROZEN>
__global__ void __launch_bounds__(256) k_integrate(BatchDev B, PhysDev P, int k, int mode,
                                                   cudaGraphConditionalHandle hcond, int use_cond) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long s = *B.step_base + k;
  int mkey = -1, tzkey = -1;
  double mval[3] = {0.0, 0.0, 0.0}, tzval[1] = {0.0};
  if (i < B.n_atoms) {
    const int e = B.atom_el[i];
    const ElemDev& E = B.el[e];
    const int l = B.orig[i];
    const bool fluid = l < E.nf;
    const bool frozen = FROZEN && !fluid;
    const bool stepped = s >= 1 && s - 1 < E.steps_total;   // a step s-1 to finish
    const bool starting = s < E.steps_total;                // a step s to start
    const bool fin = (mode & kFinish) && stepped;
    const bool st1 = (mode & kStage1) && starting;
    const long long ks = s - 1 - E.steps_eq;
    const bool sample = stepped && ks >= 0 && ks < E.steps_sample && E.nb > 0 &&
                        ((mode & kTzApply) || ((mode & kFinish) && !(mode & kTzSum)));
    double x = B.st[0][i], y = B.st[1][i], z = B.st[2][i];
    double vx = B.st[3][i], vy = B.st[4][i], vz = B.st[5][i];
    double fx = (double)static_cast<const FT*>(B.fx)[i];
    double fy = (double)static_cast<const FT*>(B.fy)[i];
    double fz = (double)static_cast<const FT*>(B.fz)[i];
    bool moved = false;
    if (fluid) {
      fx += E.g;
      if (sample) {
        // full-step velocity of step s-1 (this thread holds u unless a
        // previous launch already finished the step)
        const bool have_full = !(mode & kFinish);
        const double wx = have_full ? vx : vx + P.hdt_m * fx;
        const double wy = have_full ? vy : vy + P.hdt_m * fy;
        double wz = have_full ? vz : vz + P.hdt_m * fz;
        if (FROZEN && (mode & kTzApply) && E.nf > 0) {
          const double tzm = B.tz[2 * e + ((s - 1) & 1)] / (double)E.nf;
          if (tzm > 0.0) wz *= sqrt(1.0 + P.dt / P.tau_T * (E.T / tzm - 1.0));
        }
        mval[0] = P.mass * wx;
        mval[1] = P.mass * wx * wx + (double)static_cast<const FT*>(B.wxx)[i];
        mval[2] = P.mass * (wx * wx + wy * wy + wz * wz);
      }
      if (FROZEN && (mode & (kTzSum | kTzApply))) {
        // thermostat path: finish and start are separate launches
        if (fin) { vx += P.hdt_m * fx; vy += P.hdt_m * fy; vz += P.hdt_m * fz; }
        if ((mode & kTzSum) && stepped) tzval[0] = P.mass * vz * vz;
        if ((mode & kTzApply) && stepped && E.nf > 0) {
          const double tzm = B.tz[2 * e + ((s - 1) & 1)] / (double)E.nf;
          if (tzm > 0.0) vz *= sqrt(1.0 + P.dt / P.tau_T * (E.T / tzm - 1.0));
        }
        if (st1) {
          vx += P.hdt_m * fx; vy += P.hdt_m * fy; vz += P.hdt_m * fz;
          x += P.dt * vx; y += P.dt * vy; z += P.dt * vz;
          moved = true;
        }
      } else if (fin && st1) {
        const double dtm = 2.0 * P.hdt_m;
        vx += dtm * fx; vy += dtm * fy; vz += dtm * fz;
        x += P.dt * vx; y += P.dt * vy; z += P.dt * vz;
        moved = true;
      } else if (fin) {
        vx += P.hdt_m * fx; vy += P.hdt_m * fy; vz += P.hdt_m * fz;
      } else if (st1) {
        vx += P.hdt_m * fx; vy += P.hdt_m * fy; vz += P.hdt_m * fz;
        x += P.dt * vx; y += P.dt * vy; z += P.dt * vz;
        moved = true;
      }
    } else if (!frozen) {
      fx -= P.k_tether * (x - B.st[6][i]);
      fy -= P.k_tether * (y - B.st[7][i]);
      fz -= P.k_tether * (z - B.st[8][i]);
      if (fin) { vx += P.hdt_m * fx; vy += P.hdt_m * fy; vz += P.hdt_m * fz; }
      if (st1) {
        double b0 = 0.0, b1 = 0.0, b2 = 0.0;
        if (E.beta_sd > 0.0) {
          normals3<FT>((uint32_t)l, (uint32_t)s + E.step0, (uint32_t)E.id, 1u, E.seed, b0, b1, b2);
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
        moved = true;
      }
    } else {
      vx = vy = vz = 0.0;
    }
    if (sample || (FROZEN && (mode & kTzSum) && stepped)) {
      // every atom of the element joins its element's reduction (walls add 0)
      mkey = e * kMaxBlocks + (sample ? sample_block(ks, E) : 0);
      tzkey = e;
    }
    if (moved) {
      B.st[0][i] = x; B.st[1][i] = y; B.st[2][i] = z;
      const float xf = (float)x, yf = (float)y, zf = (float)z;
      if (!(fabsf(yf) < 1e6f) || !(fabsf(xf) < 1e6f) || !(fabsf(zf) < 1e6f)) atomicMin(&B.status[e], kStUnstable);
      if constexpr (sizeof(PT) == 16) {
        static_cast<float4*>(B.posb[0])[i] = make_float4(xf, yf, zf, fluid ? 0.0f : 1.0f);
      } else {
        static_cast<Pos64*>(B.posb[0])[i] = Pos64{x, y, z, fluid ? 0.0 : 1.0};
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
  if (FROZEN && (mode & kTzSum)) {
    const int slot = (int)((s - 1) & 1);
    const int key = (mode & kTzSum) ? tzkey : -1;
    block_seg_add<1>(key, tzval, [&](int e, int) { return B.tz + 2 * e + slot; });
  }
  if (FROZEN && (mode & kTzApply)) {
    // clear the other parity slot for the next step's sum
    const long long tcount = (long long)gridDim.x * blockDim.x;
    for (long long t = i; t < B.n_el; t += tcount) B.tz[2 * t + (s & 1)] = 0.0;
  }
  if ((mode & kTzApply) || ((mode & kFinish) && !(mode & kTzSum))) {
    block_seg_add<3>(mkey, mval, [&](int kk, int q) {
      const int e = kk / kMaxBlocks, b = kk % kMaxBlocks;
      return B.acc + (size_t)e * kAccStride + (q == 0 ? kAccQ + b : (q == 1 ? kAccP + b : kAccT));
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

// Block-level segmented reduction of FP32 values for 256-thread blocks: when
// the whole block shares one key, each warp adds its lanes in FP32 and the
// eight warp sums are added in FP64 by NV threads (one atomicAdd each);
// otherwise each warp adds its runs of equal keys in FP64 (seg_add), which
// needs no shared arrays (they would take L1 capacity from the gathers).
// All threads of the block must call it.
template <int NV, typename DstFn>
__device__ __forceinline__ void block_seg_add_f(int key, const float (&val)[NV], DstFn dst) {
  __shared__ int k0s;
  __shared__ float wsum[NV][8];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  if (t == 0) k0s = key;
  __syncthreads();
  const int k0 = k0s;
  if (__syncthreads_and(key == k0)) {
    if (k0 < 0) return;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const float v = warp_sum(val[q]);
      if (lane == 0) wsum[q][w] = v;
    }
    __syncthreads();
    if (t < NV) {
      double acc = 0.0;
      for (int r = 0; r < (int)(blockDim.x >> 5); ++r) acc += (double)wsum[t][r];
      atomicAdd(dst(k0, t), acc);
    }
    return;
  }
  double dv[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) dv[q] = (double)val[q];
  seg_add<NV>(key, dv, dst);
}

// The integration step with the double-float state (FP32 pair forces): the
// same phases and formulas as k_integrate, every update in FP32 operations.
// Per-atom measurement terms are formed in FP32 and summed per warp in FP32,
// then across warps, blocks and steps in FP64.  Positions are double
// buffered: the pair forces of step s read posb[s & 1], and the launch that
// runs stage 1 of step s writes every atom's new position to
// posb[(s + 1) & 1] (moved or not), so a fused kernel can read one buffer
// while it writes the other.
struct StepOut {
  int mkey = -1, tzkey = -1;
  float mval[3] = {0.f, 0.f, 0.f};
  float tz[1] = {0.f};
};

template <bool FROZEN>
__device__ __forceinline__ void integrate_df_atom(const BatchDev& B, const PhysDev& P, long long i, long long s,
                                                  int mode, int* skin_flag, float fx, float fy, float fz, float wxx,
                                                  StepOut& o) {
  const int e = __ldcg(B.atom_el + i);
  const ElemDev& E = B.el[e];
  const int l = __ldcg(B.orig + i);
  const bool fluid = l < E.nf;
  const bool frozen = FROZEN && !fluid;
  const bool stepped = s >= 1 && s - 1 < E.steps_total;
  const bool starting = s < E.steps_total;
  const bool fin = (mode & kFinish) && stepped;
  const bool st1 = (mode & kStage1) && starting;
  const long long ks = s - 1 - E.steps_eq;
  const bool sample = stepped && ks >= 0 && ks < E.steps_sample && E.nb > 0 &&
                      ((mode & kTzApply) || ((mode & kFinish) && !(mode & kTzSum)));
  dfl x = df_ld_cg(B.st[0], i), y = df_ld_cg(B.st[1], i), z = df_ld_cg(B.st[2], i);
  dfl vx = df_ld_cg(B.st[3], i), vy = df_ld_cg(B.st[4], i), vz = df_ld_cg(B.st[5], i);
  const float h = P.hdt_mf, dt = P.dtf;
  bool moved = false;
  if (fluid) {
    // the body force enters as its own kick, dt/(2m) g, so that it is not
    // rounded against the much larger pair force
    const float gk = E.g_kick;
    float lam = 1.0f;
    if (FROZEN && (mode & kTzApply) && E.nf > 0) {
      // summed by atomics in L2 by this step's first phase: read past L1
      const float tzm = (float)__ldcg(&B.tz[2 * e + ((s - 1) & 1)]) / (float)E.nf;
      if (tzm > 0.0f) lam = sqrtf(1.0f + P.dt_tauf * (E.Tf / tzm - 1.0f));
    }
    if (sample) {
      const bool have_full = !(mode & kFinish);
      const float wx = have_full ? vx.hi + vx.lo : vx.hi + (vx.lo + (__fmul_rn(h, fx) + gk));
      const float wy = have_full ? vy.hi + vy.lo : vy.hi + __fmaf_rn(h, fy, vy.lo);
      float wz = have_full ? vz.hi + vz.lo : vz.hi + __fmaf_rn(h, fz, vz.lo);
      wz *= lam;
      o.mval[0] = P.massf * wx;
      o.mval[1] = P.massf * wx * wx + wxx;
      o.mval[2] = P.massf * (wx * wx + wy * wy + wz * wz);
    }
    const float hfx = __fmul_rn(h, fx), hfy = __fmul_rn(h, fy), hfz = __fmul_rn(h, fz);
    if (FROZEN && (mode & (kTzSum | kTzApply))) {
      if (fin) { vx = df_add(df_add(vx, hfx), gk); vy = df_add(vy, hfy); vz = df_add(vz, hfz); }
      if ((mode & kTzSum) && stepped) o.tz[0] = P.massf * vz.hi * vz.hi;
      if ((mode & kTzApply) && stepped) vz = df_mul(lam, vz);
      if (st1) {
        vx = df_add(df_add(vx, hfx), gk); vy = df_add(vy, hfy); vz = df_add(vz, hfz);
        moved = true;
      }
    } else {
      // both half kicks of a fused launch use the same force
      const int kicks = (fin ? 1 : 0) + (st1 ? 1 : 0);
      if (kicks > 0) {
        const float kf = (float)kicks;
        vx = df_add(df_add(vx, __fmul_rn(kf, hfx)), __fmul_rn(kf, gk));
        vy = df_add(vy, __fmul_rn(kf, hfy));
        vz = df_add(vz, __fmul_rn(kf, hfz));
      }
      moved = st1;
    }
    if (moved) {
      x = df_add(x, df_mul(dt, vx)); y = df_add(y, df_mul(dt, vy)); z = df_add(z, df_mul(dt, vz));
    }
  } else if (!frozen) {
    fx = __fmaf_rn(-P.k_tetherf, df_diff(x, df_ld_cg(B.st[6], i)), fx);
    fy = __fmaf_rn(-P.k_tetherf, df_diff(y, df_ld_cg(B.st[7], i)), fy);
    fz = __fmaf_rn(-P.k_tetherf, df_diff(z, df_ld_cg(B.st[8], i)), fz);
    if (fin) { vx = df_add(vx, __fmul_rn(h, fx)); vy = df_add(vy, __fmul_rn(h, fy)); vz = df_add(vz, __fmul_rn(h, fz)); }
    if (st1) {
      float b0 = 0.f, b1 = 0.f, b2 = 0.f;
      if (E.beta_sdf > 0.f) {
        normals3f((uint32_t)l, (uint32_t)s + E.step0, (uint32_t)E.id, 1u, E.seed, b0, b1, b2);
        b0 *= E.beta_sdf; b1 *= E.beta_sdf; b2 *= E.beta_sdf;
      }
      // G-JF: x += b dt (v + dt/(2m) f + beta/(2m)); v = a v + a dt/(2m) f + (b/m) beta
      const float bdt = P.gjf_bf * dt, i2m = 0.5f * P.inv_mf, bm = P.gjf_bf * P.inv_mf, a = P.gjf_af;
      const float px = __fmaf_rn(h, fx, b0 * i2m), py = __fmaf_rn(h, fy, b1 * i2m), pz = __fmaf_rn(h, fz, b2 * i2m);
      x = df_add(x, df_mul(bdt, df_add(vx, px)));
      y = df_add(y, df_mul(bdt, df_add(vy, py)));
      z = df_add(z, df_mul(bdt, df_add(vz, pz)));
      vx = df_add(df_mul(a, vx), __fmaf_rn(h * a, fx, bm * b0));
      vy = df_add(df_mul(a, vy), __fmaf_rn(h * a, fy, bm * b1));
      vz = df_add(df_mul(a, vz), __fmaf_rn(h * a, fz, bm * b2));
      moved = true;
    }
  } else {
    vx = vy = vz = dfl{0.f, 0.f};
  }
  if (sample || (FROZEN && (mode & kTzSum) && stepped)) {
    o.mkey = e * kMaxBlocks + (sample ? sample_block(ks, E) : 0);
    o.tzkey = e;
  }
  if (moved) {
    df_st(B.st[0], i, x); df_st(B.st[1], i, y); df_st(B.st[2], i, z);
    const float xf = x.hi, yf = y.hi, zf = z.hi;
    if (!(fabsf(yf) < 1e6f) || !(fabsf(xf) < 1e6f) || !(fabsf(zf) < 1e6f)) atomicMin(&B.status[e], kStUnstable);
    const float4 pb = __ldcg(B.pbuild + i);
    const float ex = xf - pb.x, ey = yf - pb.y, ez = zf - pb.z;
    if (ex * ex + ey * ey + ez * ez > P.half_skin2f) {
      if (skin_flag) atomicOr(skin_flag, 1);
      else atomicMin(&B.status[e], kStSkin);
    }
  }
  if (mode & kStage1) static_cast<float4*>(B.posb[(s + 1) & 1])[i] = make_float4(x.hi, y.hi, z.hi, fluid ? 0.0f : 1.0f);
  df_st(B.st[3], i, vx); df_st(B.st[4], i, vy); df_st(B.st[5], i, vz);
}

// Block reductions of the step's measurement terms and, with use_cond, the
// rebuild condition: the last block to finish turns the skin flag into the
// graph condition (one caller of cudaGraphSetConditional) and clears the
// flag words.  All threads of the block call it.
template <bool FROZEN>
__device__ __forceinline__ void integrate_df_epilogue(const BatchDev& B, long long s, int mode, const StepOut& o,
                                                      cudaGraphConditionalHandle hcond, int use_cond) {
  if (FROZEN && (mode & kTzSum)) {
    const int slot = (int)((s - 1) & 1);
    block_seg_add_f<1>(o.tzkey, o.tz, [&](int e, int) { return B.tz + 2 * e + slot; });
  }
  if (FROZEN && (mode & kTzApply)) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long tcount = (long long)gridDim.x * blockDim.x;
    for (long long t = i; t < B.n_el; t += tcount) B.tz[2 * t + (s & 1)] = 0.0;
  }
  if ((mode & kTzApply) || ((mode & kFinish) && !(mode & kTzSum))) {
    block_seg_add_f<3>(o.mkey, o.mval, [&](int kk, int q) {
      const int e = kk / kMaxBlocks, b = kk % kMaxBlocks;
      return B.acc + (size_t)e * kAccStride + (q == 0 ? kAccQ + b : (q == 1 ? kAccP + b : kAccT));
    });
  }
  if (use_cond) {
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

template <bool FROZEN>
__global__ void __launch_bounds__(256) k_integrate_df(BatchDev B, PhysDev P, int k, int mode,
                                                      cudaGraphConditionalHandle hcond, int use_cond) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long s = *B.step_base + k;
  StepOut o;
  if (i < B.n_atoms)
    integrate_df_atom<FROZEN>(B, P, i, s, mode, use_cond ? &B.flags[0] : nullptr, static_cast<const float*>(B.fx)[i],
                              static_cast<const float*>(B.fy)[i], static_cast<const float*>(B.fz)[i],
                              static_cast<const float*>(B.wxx)[i], o);
  integrate_df_epilogue<FROZEN>(B, s, mode, o, hcond, use_cond);
}

// One whole MD step per launch with the double-float state: the pair forces
// of step s (positions posb[s & 1]) and, in the same thread, the integration
// phases in `mode` with them (finish step s-1, stage 1 of step s writing
// posb[(s + 1) & 1]).  The forces stay in registers unless STORE (the
// frozen-wall thermostat path, whose second launch needs them).
template <bool UNIFORM, bool FROZEN, bool STORE>
__global__ void __launch_bounds__(128) k_step_df(BatchDev B, PhysDev P, int k, int mode,
                                                 cudaGraphConditionalHandle hcond, int use_cond) {
  __shared__ ShiftTab tab;
  shift_tab_init(tab);
  __syncthreads();
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long s = *B.step_base + k;
  StepOut o;
  if (i < B.n_atoms) {
    const float4* pos = static_cast<const float4*>(B.posb[s & 1]);
    int spi = 0;
    const PairSum f = pair_force_f32<UNIFORM, false, 1>(B, P, i, 0, pos, spi, tab);
    const float wxx = spi == 0 ? 0.5f * f.w : 0.0f;
    if (STORE) {
      static_cast<float*>(B.fx)[i] = f.fx;
      static_cast<float*>(B.fy)[i] = f.fy;
      static_cast<float*>(B.fz)[i] = f.fz;
      static_cast<float*>(B.wxx)[i] = wxx;
    }
    integrate_df_atom<FROZEN>(B, P, i, s, mode, use_cond ? &B.flags[0] : nullptr, f.fx, f.fy, f.fz, wxx, o);
  }
  integrate_df_epilogue<FROZEN>(B, s, mode, o, hcond, use_cond);
}

// Grid-wide barrier for a cooperative launch (every block resident).  The
// arrival count never resets within a run: before barrier k of a launch it
// holds (g0 + k) x gridDim, g0 the count's whole multiples of the grid when
// the launch began (each block's leader reads it before its first arrival,
// and no barrier completes before every block has arrived, so every leader
// reads the same g0).  A leader makes its block's writes visible (fence),
// adds its arrival without waiting for the result, and waits until the
// count reaches its target: the last arrival is itself the release, with no
// second round trip.  The wait is bounded by wait_ns nanoseconds of the
// global timer: false if it gave up.  skip (test only) leaves this block's
// arrival out, so no block is released and every wait runs out.
__device__ __forceinline__ unsigned long long ld_acquire_gpu_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// The first target of a launch (leader thread only, before its first arrival).
__device__ __forceinline__ unsigned long long grid_barrier_base(int* flags) {
  const unsigned long long* cnt = reinterpret_cast<const unsigned long long*>(flags + kFlagBarCount);
  return ld_acquire_gpu_u64(cnt) / gridDim.x * gridDim.x;
}

__device__ __forceinline__ bool grid_barrier(int* flags, unsigned long long& target, unsigned long long wait_ns,
                                             bool skip = false) {
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(flags + kFlagBarCount);
    target += gridDim.x;
    __threadfence();
    if (!skip) atomicAdd(cnt, 1ull);
    const unsigned long long t0 = global_ns();
    while (ld_acquire_gpu_u64(cnt) < target) {
      if (global_ns() - t0 > wait_ns) { ok = 0; break; }
      __nanosleep(32);
    }
  }
  return __syncthreads_and(ok) != 0;
}

// Persistent MD steps with the double-float state (FP32 pair forces): one
// cooperative launch runs whole steps (the k_step_df work, blocks striding
// over 128-atom chunks) separated by grid barriers, until an atom has moved
// half the skin (the lists must be rebuilt before the next force evaluation)
// or step S has been started.  Step s writes its skin flag to word s mod 3
// of flags[kFlagSkin..]; every block reads it after the step's last barrier,
// before the next barrier, so the word of step s + 1 (last read two barriers
// ago) is cleared during step s.  On
// exit block 0 stores the step counter and sets the graph conditions: the
// rebuild (IF) and whether steps remain (WHILE).  With the frozen-wall
// thermostat a step is two phases with a barrier between them.  A barrier
// that gives up marks every element MDGP_E_TIMEOUT and ends the run.  Block c
// takes atoms [c A, (c + 1) A) with A <= blockDim.x chosen by the host so
// that every SM holds the same number of atoms (the step ends with the
// most loaded SM).  TPA consecutive threads share an atom's pair forces
// (batches too small to fill the GPU with one thread per atom): the group's
// first thread integrates the atom.
template <bool UNIFORM, bool FROZEN, int TPA>
__global__ void __maxnreg__(56) k_steps_persist(BatchDev B, PhysDev P, long long S, int A,
                                                      cudaGraphConditionalHandle h_rebuild,
                                                      cudaGraphConditionalHandle h_more, int use_cond) {
  __shared__ ShiftTab tab;
  shift_tab_init(tab);
  __syncthreads();
  const long long nchunks = (B.n_atoms + A - 1) / A;
  const int slot = (int)threadIdx.x / TPA, sub = (int)threadIdx.x % TPA;
  const bool lane_used = slot < A;
  long long s = *B.step_base;
  bool rebuild = false, failed = false, first_wait = true;
  unsigned long long bar_target = threadIdx.x == 0 ? grid_barrier_base(B.flags) : 0ull;
  while (s < S && !failed) {
    if (blockIdx.x == 0 && threadIdx.x == 0) B.flags[kFlagSkin + (int)((s + 1) % 3)] = 0;
    int* skin = &B.flags[kFlagSkin + (int)(s % 3)];
    const float4* pos = static_cast<const float4*>(B.posb[s & 1]);
    const int m1 = FROZEN ? (kFinish | kTzSum) : (kFinish | kStage1);
    for (long long c = blockIdx.x; c < nchunks; c += gridDim.x) {
      const long long i = lane_used ? c * A + slot : B.n_atoms;
      StepOut o;
      int spi = 0;
      const PairSum f = pair_force_f32<UNIFORM, false, TPA>(B, P, i, sub, pos, spi, tab);
      if (i < B.n_atoms && sub == 0) {
        const float wxx = spi == 0 ? 0.5f * f.w : 0.0f;
        if (FROZEN) {
          static_cast<float*>(B.fx)[i] = f.fx;
          static_cast<float*>(B.fy)[i] = f.fy;
          static_cast<float*>(B.fz)[i] = f.fz;
          static_cast<float*>(B.wxx)[i] = wxx;
        }
        integrate_df_atom<FROZEN>(B, P, i, s, m1, skin, f.fx, f.fy, f.fz, wxx, o);
      }
      integrate_df_epilogue<FROZEN>(B, s, m1, o, 0, 0);
    }
    if (!grid_barrier(B.flags, bar_target, P.wait_ns, P.inject_skip && first_wait && blockIdx.x == 0)) {
      failed = true;
      break;
    }
    first_wait = false;
    if (FROZEN) {
      const int m2 = kTzApply | kStage1;
      for (long long c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const long long i = lane_used ? c * A + slot : B.n_atoms;
        StepOut o;
        if (i < B.n_atoms && sub == 0)
          integrate_df_atom<FROZEN>(B, P, i, s, m2, skin, static_cast<const float*>(B.fx)[i],
                                    static_cast<const float*>(B.fy)[i], static_cast<const float*>(B.fz)[i],
                                    static_cast<const float*>(B.wxx)[i], o);
        integrate_df_epilogue<FROZEN>(B, s, m2, o, 0, 0);
      }
      if (!grid_barrier(B.flags, bar_target, P.wait_ns)) { failed = true; break; }
    }
    rebuild = *(volatile int*)skin != 0;
    ++s;
    if (rebuild) break;
  }
  if (failed) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < B.n_el;
         e += (long long)gridDim.x * blockDim.x)
      atomicMin(&B.status[e], kStTimeout);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *B.step_base = s;
    atomicAdd(&B.flags[3], 1);
    if (failed) B.flags[kFlagExit] = 1;
    if (use_cond) {
      cudaGraphSetConditional(h_rebuild, (rebuild && !failed) ? 1u : 0u);
      cudaGraphSetConditional(h_more, (s < S && !failed) ? 1u : 0u);
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
    constexpr bool DF = sizeof(FT) == 4;
    const double vx = st_get<DF>(B.st[3], i), vy = st_get<DF>(B.st[4], i), vz = st_get<DF>(B.st[5], i);
    double en = 0.5 * P.mass * (vx * vx + vy * vy + vz * vz) + (double)static_cast<const FT*>(B.epot)[i];
    if (B.orig[i] >= E.nf && P.mode == 1) {
      en = 0.0;                     // frozen walls carry no dynamical energy
    } else if (B.orig[i] >= E.nf) {
      const double dx = st_get<DF>(B.st[0], i) - st_get<DF>(B.st[6], i),
                   dy = st_get<DF>(B.st[1], i) - st_get<DF>(B.st[7], i),
                   dz = st_get<DF>(B.st[2], i) - st_get<DF>(B.st[8], i);
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
    constexpr bool DF = sizeof(FT) == 4;
    double x, y, z;
    abs_position<DF>(B, E, i, x, y, z);
    B.out[dst] = x; B.out[N + dst] = y; B.out[2 * N + dst] = z;
    B.out[3 * N + dst] = st_get<DF>(B.st[3], i);
    B.out[4 * N + dst] = st_get<DF>(B.st[4], i);
    B.out[5 * N + dst] = st_get<DF>(B.st[5], i);
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
