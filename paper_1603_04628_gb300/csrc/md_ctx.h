// Library context: device buffers, stream, captured step graphs.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "mdgp.h"
#include "md_internal.cuh"

struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

struct mdgp_ctx {
  int device = 0;
  int precision = MDGP_PREC_FP64;
  mdgp_md_params params;
  cudaStream_t stream = nullptr;      // stream all work is enqueued on
  cudaStream_t own_stream = nullptr;  // created with the context
  cudaStream_t side_stream = nullptr; // captures the conditional rebuild bodies
  cudaStream_t side_stream2 = nullptr;  // nested capture (rebuild inside the step loop's WHILE body)
  // GP factorisation with lookahead: [0] the diagonal/panel chain (high
  // priority), [1] the bulk trailing updates; events order the two
  cudaStream_t fact_stream[2] = {nullptr, nullptr};
  cudaEvent_t fact_event[4] = {nullptr, nullptr, nullptr, nullptr};
  char err[256] = {0};
  // MD batch
  bool planned = false;
  long long n_el = 0, steps = 0, n_atoms = 0;
  long long chunk = 256;  // steps per captured graph (rounded to the rebuild interval)
  long long rebuild_every = 1;
  long long graph_K = 0, graph_rem_K = 0;
  cudaGraphExec_t graph_full = nullptr, graph_rem = nullptr;
  cudaGraphExec_t graph_while = nullptr;  // persistent step loop (FP32 pair forces)
  unsigned persist_grid = 0;              // co-resident blocks of the persistent step kernel
  int persist_threads = 128;              // its block size
  int persist_atoms = 128;                // atoms per block (persist_atoms x persist_tpa <= persist_threads)
  int persist_tpa = 1;                    // threads per atom in its pair loop
  bool persist_resident = false;          // k_steps_resident (state in registers, lists in shared memory)
  size_t persist_smem = 0;                // its dynamic shared memory per block
  bool direct = false;        // persistent = 2: the host launches the persistent kernel itself
  // persistent = 2: CUDA-event times of the last batch's persistent launches
  // and of the rebuilds between them, and the steps they covered
  cudaEvent_t dir_ev[3] = {nullptr, nullptr, nullptr};
  double dir_kernel_ms = 0.0, dir_rebuild_ms = 0.0;
  long long dir_steps = 0, dir_launches = 0, dir_rebuilds = 0;
  bool any_warm = false;      // some element of the plan starts from a snapshot
  bool ran = false;           // a launch has run: the device state can be continued
  std::vector<mdgp::ElemDev> el_host;   // the plan's element records (host copy)
  std::vector<mdgp_element> el_desc;    // and the descriptors they came from
  long long launches = 0;              // kernels enqueued by the last launch (graph bodies: 2 per step)
  long long launches_with_rebuilds = 0;  // ... plus the rebuild kernels that ran
  long long rebuilds = 0;
  mdgp::BatchDev B;
  mdgp::PhysDev P;
  DevBuf d_el, d_aoff, d_coff, d_state, d_ints, d_cells, d_pos, d_pbuild, d_force, d_list, d_out, d_acc,
      d_grp, d_status, d_results, d_step, d_flags, d_tz, d_warm, d_pinit;
  std::vector<DevBuf*> all_bufs() {
    return {&d_el, &d_aoff, &d_coff, &d_state, &d_ints, &d_cells, &d_pos, &d_pbuild, &d_force, &d_list,
            &d_out, &d_acc, &d_grp, &d_status, &d_results, &d_step, &d_flags, &d_tz, &d_warm, &d_pinit};
  }
  void release_extra() {}
};
