// Micro-element MD engine: host planner, CUDA-graph step loop and the C ABI
// entry points declared in include/mdgp.h (paper App. A and Sec. 2.1).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "mdgp.h"
#include "md_kernels.cuh"
#include "md_ctx.h"

using namespace mdgp;

namespace {

long lround_half_up(double x) { return (long)std::floor(x + 0.5); }

int set_err(mdgp_ctx* c, cudaError_t e) {
  if (e == cudaSuccess) return MDGP_OK;
  if (c) std::snprintf(c->err, sizeof(c->err), "%s", cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? MDGP_E_NOMEM : MDGP_E_CUDA;
}

#define CK(expr)                                   \
  do {                                             \
    cudaError_t e_ = (expr);                       \
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

// Element geometry (shared definition with the paper's App. A readings:
// FCC fluid lattice in the slab, FCC (100) wall planes, cells >= r_c).
int describe(const mdgp_md_params& p, const mdgp_element& el, ElemDev& E, std::string* why) {
  if (!(el.Lx >= 3.0 * p.rc) || !(el.Lz >= 3.0 * p.rc)) { *why = "Lx and Lz must be >= 3 r_c"; return MDGP_E_ARG; }
  if (!(el.h > 2.0 * p.fluid_margin)) { *why = "h must exceed twice the fluid margin"; return MDGP_E_ARG; }
  if (!(el.density >= 0.0) || !(el.T > 0.0) || el.steps_eq < 0 || el.steps_sample < 0) {
    *why = "density >= 0, T > 0 and non-negative step counts required";
    return MDGP_E_ARG;
  }
  std::memset(&E, 0, sizeof(E));
  E.Lx = el.Lx; E.Lz = el.Lz; E.h = el.h;
  E.T = el.T;
  E.g = el.g_ext - (p.mass / (p.mass * el.density > 0 ? p.mass * el.density : 1.0)) * el.dpdx;
  if (el.density <= 0.0) E.g = el.g_ext;
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
  // fluid
  const long nf = lround_half_up(el.density * el.Lx * el.h * el.Lz);
  E.nf = (int)nf;
  const double af = std::cbrt(4.0 / el.density);
  const double ly = el.h - 2.0 * p.fluid_margin;
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
  // walls
  const double a0 = std::cbrt(4.0 / p.wall_density);
  long wnx = lround_half_up(el.Lx / a0), wnz = lround_half_up(el.Lz / a0);
  if (wnx < 1) wnx = 1;
  if (wnz < 1) wnz = 1;
  E.wnx = (int)wnx; E.wnz = (int)wnz;
  E.wax = el.Lx / wnx; E.waz = el.Lz / wnz; E.wdy = 0.5 * a0;
  E.nw = 2 * p.wall_planes * 2 * (int)wnx * (int)wnz;
  // cells
  const double th = 0.5 * a0 * (p.wall_planes - 1);
  const double ylo = -th - 1.0, yhi = el.h + th + 1.0;
  E.ylo = ylo;
  E.nc[0] = (int)std::floor(el.Lx / p.rc);
  E.nc[2] = (int)std::floor(el.Lz / p.rc);
  E.nc[1] = (int)std::floor((yhi - ylo) / p.rc);
  if (E.nc[1] < 1) E.nc[1] = 1;
  E.cs[0] = el.Lx / E.nc[0]; E.cs[1] = (yhi - ylo) / E.nc[1]; E.cs[2] = el.Lz / E.nc[2];
  for (int d = 0; d < 3; ++d) { E.inv_cs[d] = 1.0 / E.cs[d]; E.csf[d] = (float)E.cs[d]; }
  return MDGP_OK;
}

// Slots needed per cell: the densest layer (fluid density peaks about 1.6x
// next to a wall) plus every wall plane falling into one cell, with margin.
int auto_capacity(const mdgp_md_params& p, const std::vector<ElemDev>& Es, const std::vector<mdgp_element>& els) {
  double worst = 0.0;
  for (size_t i = 0; i < Es.size(); ++i) {
    const ElemDev& E = Es[i];
    const double vol = E.cs[0] * E.cs[1] * E.cs[2];
    const double fluid = 1.8 * els[i].density * vol;
    const double per_plane = 2.0 * E.cs[0] * E.cs[2] / (E.wax * E.waz);
    const double planes = std::fmin((double)p.wall_planes, std::ceil(E.cs[1] / E.wdy) + 1.0);
    worst = std::fmax(worst, fluid + per_plane * planes);
  }
  int cap = (int)std::ceil(1.5 * worst + 8.0);
  cap = (cap + 31) / 32 * 32;
  return cap < 32 ? 32 : cap;
}

PhysDev make_phys(const mdgp_md_params& p, int cap) {
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
  const double eps[3] = {1.0, p.eps_wf, p.eps_ww};
  const double sig[3] = {1.0, p.sig_wf, p.sig_ww};
  for (int t = 0; t < 3; ++t) {
    P.eps[t] = eps[t];
    P.sig2[t] = sig[t] * sig[t];
    const double sr6 = std::pow(sig[t] / p.rc, 6.0);
    P.eshift[t] = 4.0 * eps[t] * (sr6 * sr6 - sr6);
    P.active[t] = 1;
    P.epsf[t] = (float)eps[t];
    P.sig2f[t] = (float)(sig[t] * sig[t]);
  }
  if (p.mode == 1) P.active[2] = 0;
  P.mode = p.mode;
  P.wall_planes = p.wall_planes;
  P.cap = cap;
  P.rc2f = (float)(p.rc * p.rc);
  return P;
}

inline unsigned grid_for(long long n, int threads) {
  long long g = (n + threads - 1) / threads;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

// ---------------------------------------------------------------------------
// Kernel enqueue helpers (precision dispatch).
// ---------------------------------------------------------------------------
static void enqueue_integrate(mdgp_ctx* ctx, int k, int mode) {
  const unsigned g = grid_for(ctx->B.n_atoms, 256);
  if (ctx->precision == MDGP_PREC_FP32)
    k_integrate<float, SlotF><<<g, 256, 0, ctx->stream>>>(ctx->B, ctx->P, k, mode);
  else
    k_integrate<double, SlotD><<<g, 256, 0, ctx->stream>>>(ctx->B, ctx->P, k, mode);
  ctx->launches++;
}

static void enqueue_force(mdgp_ctx* ctx, int k, bool energy) {
  const unsigned g = grid_for(ctx->B.n_cells * 32, 128);
  if (ctx->precision == MDGP_PREC_FP32) {
    if (energy) k_force_cells<SlotF, float, true><<<g, 128, 0, ctx->stream>>>(ctx->B, ctx->P, k);
    else k_force_cells<SlotF, float, false><<<g, 128, 0, ctx->stream>>>(ctx->B, ctx->P, k);
  } else {
    if (energy) k_force_cells<SlotD, double, true><<<g, 128, 0, ctx->stream>>>(ctx->B, ctx->P, k);
    else k_force_cells<SlotD, double, false><<<g, 128, 0, ctx->stream>>>(ctx->B, ctx->P, k);
  }
  ctx->launches++;
}

static void enqueue_energy(mdgp_ctx* ctx, int which) {
  const unsigned g = grid_for(ctx->B.n_atoms, 256);
  if (ctx->precision == MDGP_PREC_FP32) k_energy<float><<<g, 256, 0, ctx->stream>>>(ctx->B, ctx->P, which);
  else k_energy<double><<<g, 256, 0, ctx->stream>>>(ctx->B, ctx->P, which);
  ctx->launches++;
}

// Per element: means, block standard errors, temperature and energy drift.
__global__ void k_finalize(BatchDev B, PhysDev P, mdgp_result* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B.n_el) return;
  const ElemDev& E = B.el[e];
  const double* acc = B.acc + (size_t)e * kAccStride;
  mdgp_result r;
  const int nb = E.nb;
  const long long S = E.steps_sample;
  const double vol = E.Lx * E.h * E.Lz;
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
  r.reserved = 0;
  out[e] = r;
}

// ---------------------------------------------------------------------------
// Planning.
// ---------------------------------------------------------------------------
static int plan_impl(mdgp_ctx* ctx, const mdgp_element* el, int64_t n, int cap_override) {
  ctx->planned = false;
  if (ctx->graph_full) { cudaGraphExecDestroy(ctx->graph_full); ctx->graph_full = nullptr; }
  if (ctx->graph_rem) { cudaGraphExecDestroy(ctx->graph_rem); ctx->graph_rem = nullptr; }
  if (ctx->params.mode != 0) {
    std::snprintf(ctx->err, sizeof(ctx->err), "only mode 0 (tethered walls) runs on the GPU");
    return MDGP_E_ARG;
  }
  std::vector<ElemDev> Es((size_t)n);
  std::vector<mdgp_element> els(el, el + n);
  std::vector<long long> aoff((size_t)n + 1), coff((size_t)n + 1);
  long long atoms = 0, cells = 0;
  const long long S = el[0].steps_eq + el[0].steps_sample;
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
    Es[i].atom0 = atoms;
    Es[i].cell0 = cells;
    aoff[i] = atoms;
    coff[i] = cells;
    atoms += (long long)Es[i].nf + Es[i].nw;
    cells += (long long)Es[i].nc[0] * Es[i].nc[1] * Es[i].nc[2];
  }
  aoff[n] = atoms;
  coff[n] = cells;
  if (atoms >= (1LL << 30)) {
    std::snprintf(ctx->err, sizeof(ctx->err), "batch too large (2^30 atoms max)");
    return MDGP_E_ARG;
  }
  int cap = ctx->params.cell_capacity > 0 ? ctx->params.cell_capacity : auto_capacity(ctx->params, Es, els);
  if (cap_override > cap) cap = cap_override;
  const size_t fsz = ctx->precision == MDGP_PREC_FP32 ? 4 : 8;
  const size_t ssz = ctx->precision == MDGP_PREC_FP32 ? sizeof(SlotF) : sizeof(SlotD);
  int st;
  if ((st = ensure(ctx, ctx->d_el, sizeof(ElemDev) * n))) return st;
  if ((st = ensure(ctx, ctx->d_aoff, sizeof(long long) * (n + 1)))) return st;
  if ((st = ensure(ctx, ctx->d_coff, sizeof(long long) * (n + 1)))) return st;
  if ((st = ensure(ctx, ctx->d_atomf64, sizeof(double) * 9 * atoms))) return st;
  if ((st = ensure(ctx, ctx->d_force, fsz * 5 * atoms))) return st;
  if ((st = ensure(ctx, ctx->d_atom_el, sizeof(int) * atoms))) return st;
  if ((st = ensure(ctx, ctx->d_cell_el, sizeof(int) * cells))) return st;
  if ((st = ensure(ctx, ctx->d_counts, sizeof(int) * 2 * cells))) return st;
  if ((st = ensure(ctx, ctx->d_slots, ssz * (size_t)cap * cells))) return st;
  if ((st = ensure(ctx, ctx->d_acc, sizeof(double) * kAccStride * n))) return st;
  if ((st = ensure(ctx, ctx->d_grp, sizeof(double) * 2 * kGrpStride * n))) return st;
  if ((st = ensure(ctx, ctx->d_status, sizeof(int) * n))) return st;
  if ((st = ensure(ctx, ctx->d_results, sizeof(mdgp_result) * n))) return st;
  if ((st = ensure(ctx, ctx->d_step, sizeof(long long)))) return st;
  CK(cudaMemcpyAsync(ctx->d_el.ptr, Es.data(), sizeof(ElemDev) * n, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_aoff.ptr, aoff.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_coff.ptr, coff.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice, ctx->stream));

  BatchDev& B = ctx->B;
  std::memset(&B, 0, sizeof(B));
  B.el = (const ElemDev*)ctx->d_el.ptr;
  B.atom_off = (const long long*)ctx->d_aoff.ptr;
  B.cell_off = (const long long*)ctx->d_coff.ptr;
  B.n_el = (int)n;
  B.cap = cap;
  B.n_atoms = atoms;
  B.n_cells = cells;
  double* f64 = (double*)ctx->d_atomf64.ptr;
  B.x = f64; B.y = f64 + atoms; B.z = f64 + 2 * atoms;
  B.vx = f64 + 3 * atoms; B.vy = f64 + 4 * atoms; B.vz = f64 + 5 * atoms;
  B.ax = f64 + 6 * atoms; B.ay = f64 + 7 * atoms; B.az = f64 + 8 * atoms;
  char* fb = (char*)ctx->d_force.ptr;
  B.fx = fb; B.fy = fb + fsz * atoms; B.fz = fb + 2 * fsz * atoms;
  B.wxx = fb + 3 * fsz * atoms; B.epot = fb + 4 * fsz * atoms;
  B.atom_el = (int*)ctx->d_atom_el.ptr;
  B.cell_el = (int*)ctx->d_cell_el.ptr;
  B.counts = (int*)ctx->d_counts.ptr;
  B.slots = ctx->d_slots.ptr;
  B.acc = (double*)ctx->d_acc.ptr;
  B.grp = (double*)ctx->d_grp.ptr;
  B.status = (int*)ctx->d_status.ptr;
  B.step_base = (const long long*)ctx->d_step.ptr;
  ctx->P = make_phys(ctx->params, cap);
  ctx->n_el = n;
  ctx->steps = S;
  ctx->n_atoms = atoms;
  k_fill_maps<<<grid_for(atoms > cells ? atoms : cells, 256) < 2048 ? grid_for(atoms > cells ? atoms : cells, 256) : 2048,
                256, 0, ctx->stream>>>(B);
  CK(cudaGetLastError());

  // Capture the step loop: chunks of K steps, each kernel reading the step
  // counter that a final node advances by K.
  const long long K = ctx->chunk;
  // The first step of a chunk must also finish the previous step; only the
  // very first step of the run has nothing to finish.  Chunk graphs therefore
  // always finish at k = 0, and the launch does step 0 eagerly.
  ctx->graph_K = 0;
  ctx->graph_rem_K = 0;
  if (S > 1) {
    const long long body = S - 1;
    const long long Kc = body < K ? body : K;
    auto capture_fin = [&](long long nsteps, cudaGraphExec_t* out) -> int {
      cudaGraph_t g;
      CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
      for (long long k = 0; k < nsteps; ++k) {
        enqueue_integrate(ctx, (int)k, kFinish | kStage1 | kBin);
        enqueue_force(ctx, (int)k, false);
      }
      k_advance<<<1, 32, 0, ctx->stream>>>((long long*)ctx->d_step.ptr, nsteps);
      cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
      if (e != cudaSuccess) return set_err(ctx, e);
      e = cudaGraphInstantiate(out, g, 0);
      cudaGraphDestroy(g);
      return set_err(ctx, e);
    };
    const long long saved = ctx->launches;
    if ((st = capture_fin(Kc, &ctx->graph_full))) return st;
    ctx->graph_K = Kc;
    const long long rem = body % Kc;
    if (rem) {
      if ((st = capture_fin(rem, &ctx->graph_rem))) return st;
      ctx->graph_rem_K = rem;
    }
    ctx->launches = saved;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->planned = true;
  return MDGP_OK;
}

static int launch_impl(mdgp_ctx* ctx) {
  if (!ctx->planned) return MDGP_E_STATE;
  ctx->launches = 0;
  const int n = (int)ctx->n_el;
  const long long S = ctx->steps;
  CK(cudaMemsetAsync(ctx->d_acc.ptr, 0, sizeof(double) * kAccStride * n, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_grp.ptr, 0, sizeof(double) * 2 * kGrpStride * n, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_status.ptr, 0, sizeof(int) * n, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_counts.ptr, 0, sizeof(int) * 2 * ctx->B.n_cells, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_step.ptr, 0, sizeof(long long), ctx->stream));
  k_init_atoms<<<grid_for(ctx->B.n_atoms, 256), 256, 0, ctx->stream>>>(ctx->B, ctx->P);
  k_init_fix<<<grid_for(ctx->B.n_atoms, 256), 256, 0, ctx->stream>>>(ctx->B, ctx->P);
  ctx->launches += 2;
  // forces and energy at the initial positions (step "-1" count buffer)
  enqueue_integrate(ctx, -1, kBin);
  enqueue_force(ctx, -1, true);
  enqueue_energy(ctx, kAccE0);
  if (S > 0) {
    // step 0 has nothing to finish
    enqueue_integrate(ctx, 0, kStage1 | kBin);
    enqueue_force(ctx, 0, false);
    k_advance<<<1, 32, 0, ctx->stream>>>((long long*)ctx->d_step.ptr, 1);
    ctx->launches++;
    if (ctx->graph_K > 0) {
      const long long body = S - 1;
      const long long full = body / ctx->graph_K;
      for (long long r = 0; r < full; ++r) {
        CK(cudaGraphLaunch(ctx->graph_full, ctx->stream));
        ctx->launches += 2 * ctx->graph_K + 1;
      }
      if (ctx->graph_rem_K) {
        CK(cudaGraphLaunch(ctx->graph_rem, ctx->stream));
        ctx->launches += 2 * ctx->graph_rem_K + 1;
      }
    }
    // finish the last step (s = S), then its energy at the final positions
    enqueue_integrate(ctx, 0, kFinish);
    enqueue_force(ctx, -1, true);
  }
  enqueue_energy(ctx, kAccE1);
  k_finalize<<<grid_for(n, 128), 128, 0, ctx->stream>>>(ctx->B, ctx->P, (mdgp_result*)ctx->d_results.ptr);
  ctx->launches++;
  CK(cudaGetLastError());
  return MDGP_OK;
}

static int results_impl(mdgp_ctx* ctx, mdgp_result* out, int64_t n) {
  if (!ctx->planned) return MDGP_E_STATE;
  if (n != ctx->n_el || !out) return MDGP_E_ARG;
  CK(cudaMemcpyAsync(out, ctx->d_results.ptr, sizeof(mdgp_result) * n, cudaMemcpyDeviceToHost, ctx->stream));
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
  out->cell_capacity = 0;
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
  if (e != cudaSuccess) {
    std::snprintf(ctx->err, sizeof(ctx->err), "%s", cudaGetErrorString(e));
    delete ctx;
    return MDGP_E_CUDA;
  }
  ctx->stream = ctx->own_stream;
  *out = ctx;
  return MDGP_OK;
}

int mdgp_destroy(mdgp_ctx* ctx) {
  if (!ctx) return MDGP_E_ARG;
  cudaSetDevice(ctx->device);
  if (ctx->graph_full) cudaGraphExecDestroy(ctx->graph_full);
  if (ctx->graph_rem) cudaGraphExecDestroy(ctx->graph_rem);
  for (DevBuf* b : ctx->all_bufs()) if (b->ptr) cudaFree(b->ptr);
  ctx->release_extra();
  if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
  delete ctx;
  return MDGP_OK;
}

int mdgp_set_md_params(mdgp_ctx* ctx, const mdgp_md_params* p) {
  if (!ctx || !p) return MDGP_E_ARG;
  if (!(p->dt > 0) || !(p->rc > 0) || p->n_blocks < 1 || p->wall_planes < 1 || !(p->mass > 0) ||
      !(p->wall_density > 0) || p->gamma_wall < 0 || p->cell_capacity < 0)
    return MDGP_E_ARG;
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

int64_t mdgp_micro_launch_count(const mdgp_ctx* ctx) { return ctx ? ctx->launches : -1; }

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
      if (st) return st;
      if ((st = launch_impl(ctx))) return st;
      if ((st = results_impl(ctx, res.data(), (int64_t)sub.size()))) return st;
      bool overflow = false;
      for (auto& r : res) overflow |= r.status == MDGP_E_OVERFLOW;
      if (!overflow) break;
      cap = 2 * ctx->B.cap;  // more slots per cell and run again
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
  std::vector<double> buf((size_t)6 * n_atoms);
  CK(cudaMemcpyAsync(buf.data(), ctx->B.x, sizeof(double) * 3 * n_atoms, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(buf.data() + 3 * n_atoms, ctx->B.vx, sizeof(double) * 3 * n_atoms, cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
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
  std::vector<double> soa((size_t)3 * n_atoms);
  for (int64_t i = 0; i < n_atoms; ++i)
    for (int d = 0; d < 3; ++d) soa[(size_t)d * n_atoms + i] = x[3 * i + d];
  CK(cudaMemcpyAsync(ctx->B.x, soa.data(), sizeof(double) * 3 * n_atoms, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_counts.ptr, 0, sizeof(int) * 2 * ctx->B.n_cells, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_status.ptr, 0, sizeof(int), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_step.ptr, 0, sizeof(long long), ctx->stream));
  enqueue_integrate(ctx, -1, kBin);
  enqueue_force(ctx, -1, true);
  CK(cudaGetLastError());
  const size_t fsz = ctx->precision == MDGP_PREC_FP32 ? 4 : 8;
  std::vector<char> raw(fsz * 5 * n_atoms);
  int status = 0;
  CK(cudaMemcpyAsync(raw.data(), ctx->B.fx, fsz * 5 * n_atoms, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(&status, ctx->d_status.ptr, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  auto get = [&](int arr, int64_t i) -> double {
    if (fsz == 4) return (double)((const float*)raw.data())[(size_t)arr * n_atoms + i];
    return ((const double*)raw.data())[(size_t)arr * n_atoms + i];
  };
  for (int64_t i = 0; i < n_atoms; ++i) {
    if (f) for (int d = 0; d < 3; ++d) f[3 * i + d] = get(d, i);
    if (wxx) wxx[i] = get(3, i);
    if (epot) epot[i] = get(4, i);
  }
  return status ? status : MDGP_OK;
}

int mdgp_micro_profile(mdgp_ctx* ctx, int64_t steps, double* ms) {
  if (!ctx || !ms || steps < 1) return MDGP_E_ARG;
  if (!ctx->planned) return MDGP_E_STATE;
  if (steps > ctx->steps) steps = ctx->steps;
  cudaSetDevice(ctx->device);
  const int n = (int)ctx->n_el;
  CK(cudaMemsetAsync(ctx->d_acc.ptr, 0, sizeof(double) * kAccStride * n, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_grp.ptr, 0, sizeof(double) * 2 * kGrpStride * n, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_status.ptr, 0, sizeof(int) * n, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_counts.ptr, 0, sizeof(int) * 2 * ctx->B.n_cells, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_step.ptr, 0, sizeof(long long), ctx->stream));
  k_init_atoms<<<grid_for(ctx->B.n_atoms, 256), 256, 0, ctx->stream>>>(ctx->B, ctx->P);
  k_init_fix<<<grid_for(ctx->B.n_atoms, 256), 256, 0, ctx->stream>>>(ctx->B, ctx->P);
  enqueue_integrate(ctx, -1, kBin);
  enqueue_force(ctx, -1, false);
  std::vector<cudaEvent_t> ev((size_t)(3 * steps + 1));
  for (auto& e : ev) CK(cudaEventCreate(&e));
  CK(cudaEventRecord(ev[0], ctx->stream));
  for (int64_t k = 0; k < steps; ++k) {
    // step_base stays 0: kernel k uses step k
    enqueue_integrate(ctx, (int)k, (k == 0 ? 0 : kFinish) | kStage1 | kBin);
    CK(cudaEventRecord(ev[3 * k + 1], ctx->stream));
    enqueue_force(ctx, (int)k, false);
    CK(cudaEventRecord(ev[3 * k + 2], ctx->stream));
    CK(cudaEventRecord(ev[3 * k + 3], ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  double t_int = 0.0, t_force = 0.0;
  for (int64_t k = 0; k < steps; ++k) {
    float a = 0.f, b = 0.f;
    cudaEventElapsedTime(&a, ev[3 * k], ev[3 * k + 1]);
    cudaEventElapsedTime(&b, ev[3 * k + 1], ev[3 * k + 2]);
    t_int += a;
    t_force += b;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  ms[0] = t_int / steps;
  ms[1] = t_force / steps;
  ms[2] = (double)ctx->n_atoms;
  ms[3] = (double)ctx->B.n_cells;
  return MDGP_OK;
}

const char* mdgp_last_error(const mdgp_ctx* ctx) { return ctx ? ctx->err : "null context"; }

}  // extern "C"
