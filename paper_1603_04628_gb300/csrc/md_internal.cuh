// Internal device-side types of the micro-element MD engine.
//
// Layout in HBM (one flattened batch, elements back to back; element e owns
// atoms [atom0, atom0 + nf + nw) and cells [cell0, cell0 + ncx*ncy*ncz)):
//   atoms  kept in cell order (re-sorted at every neighbour-list rebuild);
//          SoA, FP64 with FP64 pair forces and double-float (two FP32 words,
//          hi + lo, ~44-bit significand) with FP32 pair forces, in the same
//          8 bytes per value: position as an offset from the centre of the atom's
//          reference cell (the cell it was binned into at the last rebuild),
//          velocity, and for wall atoms the tether anchor in the same frame;
//          int32 original index (element-local, fluid first) and reference
//          cell; the pair-force input position (float4 or double4: offset
//          from the cell centre, w = species) and its value at the last
//          rebuild (skin check); forces, fluid x-virial share and energy in
//          the pair-force precision.
//   lists  per atom up to list_cap neighbour entries in groups of four,
//          [k / 4][atom][4] (a warp's 16-byte loads coalesce); an entry holds
//          in bits 0-25 the neighbour's element-local sorted index and in bits
//          26-31 the cell shift (dx+1, dy+1, dz+1), 2 bits each; the last
//          group is padded with an entry that is always beyond r_c.
//   cells  count (binning atomics), start and size after the per-element scan;
//          within a cell the atoms are ordered by original index (the order
//          does not depend on the binning atomics, so runs are reproducible).
//   accum  per element FP64 block sums of q and P_xx, temperature sum and the
//          start/end energies (the time-averaged measurements of Sec. 2.1).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mdgp {

constexpr int kMaxBlocks = 64;
constexpr int kAccQ = 0;                      // q block sums [kMaxBlocks]
constexpr int kAccP = kMaxBlocks;             // P_xx block sums [kMaxBlocks]
constexpr int kAccT = 2 * kMaxBlocks;         // sum of fluid m|v|^2 over samples
constexpr int kAccE0 = 2 * kMaxBlocks + 1;    // total energy before the first step
constexpr int kAccE1 = 2 * kMaxBlocks + 2;    // total energy after the last step
constexpr int kAccStride = 2 * kMaxBlocks + 4;
constexpr int kGrpStride = 8;                 // init sums per group: sum v, sum v^2
constexpr unsigned kJMask = 0x03FFFFFFu;      // neighbour index bits of a list entry
constexpr int kFlagSkin = 4;                  // flag words (see BatchDev::flags)
constexpr int kFlagBarCount = 10;             // grid-barrier arrivals, 64-bit, words 10-11
constexpr int kFlags = 16;

// status codes written per element (match mdgp_status)
constexpr int kStUnstable = -4;
constexpr int kStTimeout = -6;
constexpr int kStOverflow = -8;
constexpr int kStSkin = -9;

constexpr int kFlagExit = 7;         // flags[7]: 1 when the persistent step kernel gave up a barrier wait

// FP64 pair-force input position (offset from the cell centre, w = species).
struct __align__(32) Pos64 {
  double x, y, z, w;
};

struct ElemDev {
  double Lx, Lz, h, ylo;
  double cs[3], inv_cs[3];
  double g;            // body force on each fluid atom along x (Eq. momentumEq)
  double T;
  double vsd;          // sqrt(T / m)
  double beta_sd;      // sqrt(2 gamma T dt): G-JF noise amplitude
  double fb[3];        // fluid lattice spacings
  double fy0;          // fluid lattice y origin
  double wax, waz, wdy;
  long long atom0, cell0;
  long long steps_eq, steps_sample, steps_total;
  unsigned long long seed;
  int fc[3];           // fluid lattice cells
  int nf, nw;
  int wnx, wnz;
  int nc[3];           // cell grid
  int id;
  int warm;            // 0 cold start (lattice); 1 fluid and walls from a snapshot
  int nb;              // blocks actually used
  float csf[3];        // cell sizes as float
  float cs_lo[3];      // cs - csf: the cell sizes as double-float numbers
  float inv_csf[3];
  float g_kick;        // dt/(2m) g as float (double-float state)
  float Tf, beta_sdf;
  double amp;          // profiled walls: h(x) = hvol (1 - amp cos(2 pi x / Lx)); 0 = planar
  double hvol;         // mean gap: the fluid volume is Lx hvol Lz (h is the widest gap)
  unsigned step0;      // steps run before this launch (continued runs): Philox step offset
};

struct PhysDev {
  double dt, hdt_m, inv_m, mass;
  double k_tether;
  double gjf_a, gjf_b;
  double rc2, rl2;                     // cut-off and list radius squared
  double eps[3], sig2[3], eshift[3];   // pair type t = species_i + species_j
  int active[3];
  int uniform;                         // all three pair types (1, 1) and active
  int mode;
  int wall_planes;
  double tau_T;                        // Berendsen time constant (mode 1)
  int list_cap;
  unsigned long long wait_ns;          // limit of a bounded device-side wait (grid barrier)
  int inject_skip;                     // test only: block 0 skips its first grid-barrier arrival
  float rc2f, rl2f, half_skin2f;
  float epsf[3], sig2f[3];
  // float copies for the double-float state updates (pair-force precision FP32)
  float dtf, hdt_mf, massf, inv_mf, k_tetherf, gjf_af, gjf_bf, dt_tauf;
};

struct BatchDev {
  const ElemDev* el;
  const long long* atom_off;   // [n_el + 1]
  const long long* cell_off;   // [n_el + 1]
  int n_el;
  int list_cap;
  long long n_atoms, n_cells;
  // current atom state (cell order) and the permutation target
  double* st[9];               // ox oy oz vx vy vz ax ay az
  double* st2[9];
  int *orig, *cell, *orig2, *cell2;
  int* atom_el;                // fixed: elements keep their atom ranges
  int* cell_el;
  void* posb[2];               // pair-force input positions, float4 or Pos64 [n_atoms]:
                               // the forces of step s read posb[s & 1] (FP32: two
                               // buffers; FP64: both point to one)
  float4* pbuild;              // pos at the last rebuild
  const double* pinit;         // [3 n_atoms] initial positions of profiled elements (else null)
  void *fx, *fy, *fz, *wxx, *epot;
  int *ccount, *cstart, *csize;   // [n_cells]
  int *newcell, *slot;            // [n_atoms]
  unsigned* list;                 // [list_cap * n_atoms]
  int* nlist;                     // [n_atoms]
  double* acc;                    // [n_el * kAccStride]
  double* grp;                    // [n_el * 2 * kGrpStride]
  int* status;                    // [n_el]
  long long* step_base;           // device step counter (advanced per graph chunk or by the
                                  // persistent step kernel)
  double* out;                    // export scratch [6 * n_atoms] (original order)
  int* flags;                     // [kFlags]: [0] rebuild needed, [1] blocks done, [2] rebuilds
                                  // run, [3] persistent step launches, [4..6] skin flags by
                                  // step mod 3, [7] barrier wait given up, [10..11] the grid
                                  // barrier's 64-bit arrival count
  double* tz;                     // [2 * n_el] per-element sum of m v_z^2 (two step-parity slots)
  const double* warm;             // [6 * n_atoms] start state (x y z vx vy vz, absolute, original
                                  // order) of the atoms of elements with warm != 0
};

// integration kernel phases: kFinish = second half kick (+ measurement unless
// kTzSum), kStage1 = first half kick + drift.  Frozen-wall elements with the
// Berendsen thermostat on v_z split a step over two launches: kFinish | kTzSum
// (half kick, per-element sum of m v_z^2), then kTzApply | kStage1 (scale v_z,
// measure, next half kick and drift).
enum : int { kFinish = 1, kStage1 = 2, kTzSum = 4, kTzApply = 8 };

}  // namespace mdgp
