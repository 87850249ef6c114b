// Persistent MD step loop for small batches, with the atom state on chip.
//
// In the regime of the hybrid scheme's MD calls (a few elements of one to
// two thousand atoms) the step kernel has far more threads than atoms and
// every step is a chain of dependent global round trips: the atom's element,
// its list count and list groups, the neighbour positions, its state, the
// skin reference, then the grid barrier.  Between two list rebuilds none of
// that changes except the positions, so this kernel loads it once per launch:
// each atom's double-float position and velocity stay in registers, its
// tether anchor, skin reference and element constants in a shared-memory
// record, and the block's lists are staged into shared memory by bulk
// asynchronous copies (one per list group, completed on an mbarrier whose
// wait is bounded).  A step then reads global memory only to gather the
// neighbour positions of the previous step (Eq. LJ), integrates
// in registers (velocity Verlet for the fluid, G-JF Langevin for the
// tethered walls, the body force as its own kick), publishes the new
// position and meets the other blocks at the grid barrier.  The state is
// written back when the launch ends (a rebuild is due, the last step was
// started, or a barrier wait ran out).
//
// The arithmetic and its order are those of k_steps_persist with the same
// threads per atom (pair entries evaluated two at a time in the same group
// order, the same group sums, the same double-float updates), so the two
// produce the same trajectory bit for bit.  The measurements are not part of
// the state: their per-atom terms are FP32 expressions the compiler may fuse
// differently in the two kernels, and their sums are FP64 atomics in
// arbitrary order, so they agree to FP32 rounding of the terms.
//
// Requirements, checked by the host before it picks this kernel: tethered
// walls (mode 0; the frozen-wall thermostat's two phases per step stay with
// k_steps_persist), FP32 pair forces with the double-float state, and one
// block per chunk of A atoms (the grid covers every atom once, no striding),
// with the dynamic shared memory of resident_smem_bytes (the lists, A x
// list_cap x 4 bytes, and A slot records).
#pragma once
#include "md_kernels.cuh"

namespace mdgp {

// List groups a lane loads and gathers per round of the resident pair loop.
constexpr int kResDepth = 2;

// The pair loop of pair_force_f32 over a list held in shared memory
// (group k of the block's atom `slot` at sl[k * A + slot]) with the atom's
// own position me: up to kResDepth list groups per round are loaded and
// their neighbour positions gathered before any is used, so one round trip
// to the L2 serves them all (a lane of an eight-thread group has two or
// three groups at the usual list lengths: one or two rounds; a depth of
// three spills at the two-blocks-per-SM register budget).  Groups are added
// in the order sub, sub + TPA, sub + 2 TPA, ..., as in pair_force_f32.
template <bool UNIFORM, int TPA>
__device__ __forceinline__ PairSum pair_force_resident(const float4& me, const float4* posj, const uint4* sl,
                                                       int A, int slot, int sub, int n, bool live,
                                                       const PairConst& c, const ShiftTab& tab) {
  constexpr int D = kResDepth;
  PairAcc2<UNIFORM, false> acc;
  if (live) {
    const int ng = (n + 3) >> 2;
    for (int k0 = sub; k0 < ng; k0 += D * TPA) {
      uint4 e[D];
      float4 o[D][4];
#pragma unroll
      for (int u = 0; u < D; ++u) {
        const int k = k0 + u * TPA;
        if (k < ng) {
          e[u] = sl[k * A + slot];
          o[u][0] = posj[e[u].x & kJMask]; o[u][1] = posj[e[u].y & kJMask];
          o[u][2] = posj[e[u].z & kJMask]; o[u][3] = posj[e[u].w & kJMask];
        }
      }
#pragma unroll
      for (int u = 0; u < D; ++u) {
        if (k0 + u * TPA < ng) {
          acc.add(me, o[u][0], o[u][1], e[u].x, e[u].y, c, tab);
          acc.add(me, o[u][2], o[u][3], e[u].z, e[u].w, c, tab);
        }
      }
    }
  }
  float ax, bx, ay, by, az, bz, aw, bw;
  f2_upk(acc.fx, ax, bx); f2_upk(acc.fy, ay, by); f2_upk(acc.fz, az, bz); f2_upk(acc.w, aw, bw);
  PairSum r{48.f * (ax + bx), 48.f * (ay + by), 48.f * (az + bz), 48.f * (aw + bw), 0.f};
  if constexpr (TPA > 1) {
    r.fx = group_sum<TPA>(r.fx); r.fy = group_sum<TPA>(r.fy); r.fz = group_sum<TPA>(r.fz);
    r.w = group_sum<TPA>(r.w);
  }
  return r;
}

// Bulk asynchronous copy (the TMA's one-dimensional form) of `bytes` from
// global to this block's shared memory, completed on the mbarrier `bar`.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ unsigned res_smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void res_bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               :: "r"(res_smem_addr(dst)), "l"(src), "r"(bytes), "r"(res_smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool res_mbar_try_wait(uint64_t* bar, unsigned phase) {
  unsigned ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
               : "=r"(ok) : "r"(res_smem_addr(bar)), "r"(phase) : "memory");
  return ok != 0;
}
// Wait for phase 0 of bar, bounded by wait_ns of the global timer.
__device__ __forceinline__ bool res_mbar_wait(uint64_t* bar, unsigned long long wait_ns) {
  const unsigned long long t0 = global_ns();
  while (!res_mbar_try_wait(bar, 0))
    if (global_ns() - t0 > wait_ns) return false;
  return true;
}

// What one atom keeps for a whole launch: its double-float state and list
// length in registers, the rest in a shared-memory slot record (read by
// broadcast to the atom's threads; kept out of the registers, which the
// gathers of the pair loop need).
struct ResidentState {
  dfl x, y, z, vx, vy, vz;        // offset from the reference cell's centre; velocity
  int n;                          // list entries
  bool fluid;
};
struct ResidentSlot {
  dfl ax, ay, az;                 // tether anchor (walls)
  float pbx, pby, pbz;            // pair-force position at the last rebuild (skin check)
  float g_kick, beta_sdf;
  long long steps_eq, steps_sample, steps_total, atom0;
  unsigned long long seed;
  int e, l, nb, id;
  unsigned step0;
};

// Dynamic shared memory of k_steps_resident for A atoms per block: the lists
// (A x list_cap entries), then the slot records.
inline size_t resident_lists_bytes(int A, int list_cap) { return (size_t)A * (size_t)list_cap * 4u; }
inline size_t resident_smem_bytes(int A, int list_cap) {
  return resident_lists_bytes(A, list_cap) + (size_t)A * sizeof(ResidentSlot);
}

// One step of integrate_df_atom for a tethered-wall element in the fused
// phases (finish step s - 1, stage 1 of step s) on the registers of `a`:
// the same operations in the same order.  Writes the measurement terms into
// o when `owner` (the group's first thread), and reports instability and a
// due rebuild by the same flags.
__device__ __forceinline__ void integrate_resident(const BatchDev& B, const PhysDev& P, ResidentState& a,
                                                   const ResidentSlot& k,
                                                   long long s, float fx, float fy, float fz, float wxx,
                                                   int* skin_flag, bool owner, StepOut& o) {
  const bool stepped = s >= 1 && s - 1 < k.steps_total;
  const bool starting = s < k.steps_total;
  const bool fin = stepped, st1 = starting;
  const long long ks = s - 1 - k.steps_eq;
  const bool sample = stepped && ks >= 0 && ks < k.steps_sample && k.nb > 0;
  const float h = P.hdt_mf, dt = P.dtf;
  bool moved = false;
  if (a.fluid) {
    const float gk = k.g_kick;
    if (sample && owner) {
      const float wx = a.vx.hi + (a.vx.lo + (__fmul_rn(h, fx) + gk));
      const float wy = a.vy.hi + __fmaf_rn(h, fy, a.vy.lo);
      const float wz = a.vz.hi + __fmaf_rn(h, fz, a.vz.lo);
      o.mval[0] = P.massf * wx;
      o.mval[1] = P.massf * wx * wx + wxx;
      o.mval[2] = P.massf * (wx * wx + wy * wy + wz * wz);
    }
    const float hfx = __fmul_rn(h, fx), hfy = __fmul_rn(h, fy), hfz = __fmul_rn(h, fz);
    const int kicks = (fin ? 1 : 0) + (st1 ? 1 : 0);
    if (kicks > 0) {
      const float kf = (float)kicks;
      a.vx = df_add(df_add(a.vx, __fmul_rn(kf, hfx)), __fmul_rn(kf, gk));
      a.vy = df_add(a.vy, __fmul_rn(kf, hfy));
      a.vz = df_add(a.vz, __fmul_rn(kf, hfz));
    }
    moved = st1;
    if (moved) {
      a.x = df_add(a.x, df_mul(dt, a.vx)); a.y = df_add(a.y, df_mul(dt, a.vy)); a.z = df_add(a.z, df_mul(dt, a.vz));
    }
  } else {
    fx = __fmaf_rn(-P.k_tetherf, df_diff(a.x, k.ax), fx);
    fy = __fmaf_rn(-P.k_tetherf, df_diff(a.y, k.ay), fy);
    fz = __fmaf_rn(-P.k_tetherf, df_diff(a.z, k.az), fz);
    if (fin) {
      a.vx = df_add(a.vx, __fmul_rn(h, fx)); a.vy = df_add(a.vy, __fmul_rn(h, fy)); a.vz = df_add(a.vz, __fmul_rn(h, fz));
    }
    if (st1) {
      float b0 = 0.f, b1 = 0.f, b2 = 0.f;
      if (k.beta_sdf > 0.f) {
        normals3f((uint32_t)k.l, (uint32_t)s + k.step0, (uint32_t)k.id, 1u, k.seed, b0, b1, b2);
        b0 *= k.beta_sdf; b1 *= k.beta_sdf; b2 *= k.beta_sdf;
      }
      // G-JF: x += b dt (v + dt/(2m) f + beta/(2m)); v = a v + a dt/(2m) f + (b/m) beta
      const float bdt = P.gjf_bf * dt, i2m = 0.5f * P.inv_mf, bm = P.gjf_bf * P.inv_mf, ga = P.gjf_af;
      const float px = __fmaf_rn(h, fx, b0 * i2m), py = __fmaf_rn(h, fy, b1 * i2m), pz = __fmaf_rn(h, fz, b2 * i2m);
      a.x = df_add(a.x, df_mul(bdt, df_add(a.vx, px)));
      a.y = df_add(a.y, df_mul(bdt, df_add(a.vy, py)));
      a.z = df_add(a.z, df_mul(bdt, df_add(a.vz, pz)));
      a.vx = df_add(df_mul(ga, a.vx), __fmaf_rn(h * ga, fx, bm * b0));
      a.vy = df_add(df_mul(ga, a.vy), __fmaf_rn(h * ga, fy, bm * b1));
      a.vz = df_add(df_mul(ga, a.vz), __fmaf_rn(h * ga, fz, bm * b2));
      moved = true;
    }
  }
  if (!owner) return;
  if (sample) {
    const unsigned long long span = (unsigned long long)k.steps_sample * (unsigned long long)k.nb;
    const int b = span < (1ull << 32) ? (int)((unsigned)ks * (unsigned)k.nb / (unsigned)k.steps_sample)
                                      : (int)((ks * k.nb) / k.steps_sample);
    o.mkey = k.e * kMaxBlocks + b;
    o.tzkey = k.e;
  }
  if (moved) {
    const float xf = a.x.hi, yf = a.y.hi, zf = a.z.hi;
    if (!(fabsf(yf) < 1e6f) || !(fabsf(xf) < 1e6f) || !(fabsf(zf) < 1e6f)) atomicMin(&B.status[k.e], kStUnstable);
    const float ex = xf - k.pbx, ey = yf - k.pby, ez = zf - k.pbz;
    if (ex * ex + ey * ey + ez * ez > P.half_skin2f) atomicOr(skin_flag, 1);
  }
}

// The persistent step loop with resident atoms (see the top of this file).
// Block b owns atoms [b A, (b + 1) A); TPA consecutive threads share an atom:
// every thread of the group keeps the atom's state and integrates it (the
// group sums are the same in every lane), the group's first thread alone
// writes.  Step control, skin words, graph conditions and the bounded grid
// barrier are those of k_steps_persist.
template <bool UNIFORM, int TPA>
__global__ void __launch_bounds__(256, 2) k_steps_resident(BatchDev B, PhysDev P, long long S, int A,
                                                          cudaGraphConditionalHandle h_rebuild,
                                                          cudaGraphConditionalHandle h_more, int use_cond) {
  extern __shared__ __align__(16) uint4 s_list[];
  __shared__ ShiftTab tab;
  __shared__ uint64_t s_bar;
  shift_tab_init(tab);
  const int slot = (int)threadIdx.x / TPA, sub = (int)threadIdx.x % TPA;
  const long long N = B.n_atoms;
  const long long i = slot < A ? (long long)blockIdx.x * A + slot : N;
  const bool live = i < N;
  const bool owner = live && sub == 0;
  // the block's lists, group g of atom slot a at s_list[g A + a]: group g of
  // the block's atoms is one contiguous run of 16-byte entries in the
  // [group][atom] layout, so one bulk copy per group stages it
  const long long a0 = (long long)blockIdx.x * A;
  const int nslot = (int)(N - a0 < A ? N - a0 : A);   // >= 1: the grid covers the atoms once
  if (threadIdx.x == 0) {
    const int G = B.list_cap >> 2;
    const uint4* L4 = reinterpret_cast<const uint4*>(B.list);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(res_smem_addr(&s_bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(res_smem_addr(&s_bar)), "r"((unsigned)(G * nslot * 16)) : "memory");
    for (int g = 0; g < G; ++g)
      res_bulk_g2s(s_list + (size_t)g * A, L4 + (long long)g * N + a0, (unsigned)(nslot * 16), &s_bar);
  }
  // the atoms' slot records follow the lists (16-byte aligned: list_cap is a
  // multiple of four entries)
  ResidentSlot* slots = reinterpret_cast<ResidentSlot*>(s_list + (size_t)(B.list_cap >> 2) * A);
  ResidentState a = {};
  PairConst c = {};
  if (live) {
    const int e = __ldcg(B.atom_el + i);
    const ElemDev& E = B.el[e];
    const int l = __ldcg(B.orig + i);
    a.fluid = l < E.nf;
    a.n = __ldcg(B.nlist + i);
    a.x = df_ld_cg(B.st[0], i); a.y = df_ld_cg(B.st[1], i); a.z = df_ld_cg(B.st[2], i);
    a.vx = df_ld_cg(B.st[3], i); a.vy = df_ld_cg(B.st[4], i); a.vz = df_ld_cg(B.st[5], i);
    if (sub == 0) {
      ResidentSlot& k = slots[slot];
      k.e = e; k.l = l;
      k.atom0 = E.atom0;
      k.steps_eq = E.steps_eq; k.steps_sample = E.steps_sample; k.steps_total = E.steps_total;
      k.nb = E.nb; k.id = E.id; k.seed = E.seed; k.step0 = E.step0;
      k.g_kick = E.g_kick; k.beta_sdf = E.beta_sdf;
      k.ax = a.fluid ? dfl{0.f, 0.f} : df_ld_cg(B.st[6], i);
      k.ay = a.fluid ? dfl{0.f, 0.f} : df_ld_cg(B.st[7], i);
      k.az = a.fluid ? dfl{0.f, 0.f} : df_ld_cg(B.st[8], i);
      const float4 pb = __ldcg(B.pbuild + i);
      k.pbx = pb.x; k.pby = pb.y; k.pbz = pb.z;
    }
    const int spi = a.fluid ? 0 : 1;
    const float csx = E.csf[0], csy = E.csf[1], csz = E.csf[2];
    c.ncsx = f2_pk(-csx, -csx); c.ncsy = f2_pk(-csy, -csy); c.ncsz = f2_pk(-csz, -csz);
    c.cmh = f2_pk(-0.5f, -0.5f);
    c.rc2 = P.rc2f;
    c.eps0 = P.epsf[spi]; c.eps1 = P.epsf[spi + 1];
    c.sig0 = P.sig2f[spi]; c.sig1 = P.sig2f[spi + 1];
    c.esh0 = (float)P.eshift[spi]; c.esh1 = (float)P.eshift[spi + 1];
    c.act0 = P.active[spi] != 0; c.act1 = P.active[spi + 1] != 0;
  }
  __syncthreads();   // the mbarrier is initialised before anyone waits on it
  // a copy that has not landed within the wait limit ends this block's run
  // (after a second bounded wait for the copies in flight): the other blocks'
  // barrier waits then run out and the launch ends with MDGP_E_TIMEOUT
  const bool staged = __syncthreads_and(res_mbar_wait(&s_bar, P.wait_ns) ? 1 : 0) != 0;
  if (!staged) res_mbar_wait(&s_bar, P.wait_ns);
  long long s = *B.step_base;
  bool rebuild = false, failed = !staged, first_wait = true;
  unsigned long long bar_target = threadIdx.x == 0 ? grid_barrier_base(B.flags) : 0ull;
  while (s < S && !failed) {
    if (blockIdx.x == 0 && threadIdx.x == 0) B.flags[kFlagSkin + (int)((s + 1) % 3)] = 0;
    int* skin = &B.flags[kFlagSkin + (int)(s % 3)];
    const float4* pos = static_cast<const float4*>(B.posb[s & 1]);
    // the atom's own pair-force position is its state's high part, as stage 1
    // of the previous step (or the rebuild) wrote it to pos
    const float4 me = make_float4(a.x.hi, a.y.hi, a.z.hi, a.fluid ? 0.0f : 1.0f);
    const ResidentSlot& k = slots[slot < A ? slot : 0];
    const float4* posj = pos + (live ? k.atom0 : 0);
    const PairSum f = pair_force_resident<UNIFORM, TPA>(me, posj, s_list, A, slot, sub, a.n, live, c, tab);
    StepOut o;
    if (live) {
      const float wxx = a.fluid ? 0.5f * f.w : 0.0f;
      integrate_resident(B, P, a, k, s, f.fx, f.fy, f.fz, wxx, skin, owner, o);
      if (owner)
        static_cast<float4*>(B.posb[(s + 1) & 1])[i] = make_float4(a.x.hi, a.y.hi, a.z.hi, a.fluid ? 0.0f : 1.0f);
    }
    integrate_df_epilogue<false>(B, s, kFinish | kStage1, o, 0, 0);
    if (!grid_barrier(B.flags, bar_target, P.wait_ns, P.inject_skip && first_wait && blockIdx.x == 0)) {
      failed = true;
      break;
    }
    first_wait = false;
    rebuild = *(volatile int*)skin != 0;
    ++s;
    if (rebuild) break;
  }
  if (owner) {
    df_st(B.st[0], i, a.x); df_st(B.st[1], i, a.y); df_st(B.st[2], i, a.z);
    df_st(B.st[3], i, a.vx); df_st(B.st[4], i, a.vy); df_st(B.st[5], i, a.vz);
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

}  // namespace mdgp
