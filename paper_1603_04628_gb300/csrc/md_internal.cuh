// Internal device-side types of the micro-element MD engine.
//
// Layout in HBM (one flattened batch, elements back to back):
//   atoms   SoA FP64 x, y, z, v_x, v_y, v_z, anchor x/y/z (wall tether sites);
//           forces in the pair-force precision (float or double) SoA;
//           per-atom x-virial share and shifted LJ energy; atom -> element map.
//           Within an element: fluid atoms first, then bottom and top walls.
//   cells   per element a grid of ncx x ncy x ncz cells of side >= r_c
//           (x, z periodic; y spans both walls); a fixed-capacity slot array
//           per cell holding cell-centre-relative positions + a tag
//           (atom << 1 | species); two count buffers used on alternate steps.
//   accum   per element FP64 block sums of q and P_xx, temperature sum and
//           energies (the time-averaged measurements of the paper's Sec. 2.1).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mdgp {

constexpr int kMaxBlocks = 64;
// per-element accumulator layout (doubles)
constexpr int kAccQ = 0;                      // q block sums [kMaxBlocks]
constexpr int kAccP = kMaxBlocks;             // P_xx block sums [kMaxBlocks]
constexpr int kAccT = 2 * kMaxBlocks;         // sum of fluid kinetic temperature
constexpr int kAccE0 = 2 * kMaxBlocks + 1;    // total energy before the first step
constexpr int kAccE1 = 2 * kMaxBlocks + 2;    // total energy after the last step
constexpr int kAccStride = 2 * kMaxBlocks + 4;
// per-element init sums: per group (fluid, wall) sum v_x, v_y, v_z, sum v^2
constexpr int kGrpStride = 8;

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
  int nb;              // blocks actually used
  float csf[3];        // cell sizes as float
  float pad;
};

struct PhysDev {
  double dt, hdt_m, inv_m, mass;
  double k_tether;
  double gjf_a, gjf_b;
  double rc2;
  double eps[3], sig2[3], eshift[3];   // pair type t = species_i + species_j
  int active[3];
  int mode;
  int wall_planes;
  int cap;
  float rc2f;
  float epsf[3], sig2f[3];
};

// Cell slot entries: position relative to the cell centre and a tag.
struct SlotF { float x, y, z; int tag; };
struct __align__(16) SlotD { double x, y, z; int tag; int pad; };

struct BatchDev {
  const ElemDev* el;
  const long long* atom_off;   // [n_el + 1]
  const long long* cell_off;   // [n_el + 1]
  int n_el;
  int cap;
  long long n_atoms, n_cells;
  double *x, *y, *z, *vx, *vy, *vz, *ax, *ay, *az;
  void *fx, *fy, *fz;          // float or double
  void *wxx, *epot;            // float or double
  int* atom_el;
  int* cell_el;
  int* counts;                 // [2 * n_cells]
  void* slots;                 // [n_cells * cap]
  double* acc;                 // [n_el * kAccStride]
  double* grp;                 // [n_el * 2 * kGrpStride]
  int* status;                 // [n_el]
  const long long* step_base;  // device step counter (advanced per graph chunk)
};

enum : int { kFinish = 1, kStage1 = 2, kBin = 4 };

}  // namespace mdgp
