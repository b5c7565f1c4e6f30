// Host-side launchers of the kernels in bq_kernels.cu.
#pragma once

#include <cuda_runtime.h>

#include "bq_internal.h"

#define BQ_MAX_DYN_SMEM (200 * 1024)
// bytes of each of the three buffers of the fixed RK4 scratch (bq_step_fixed_scratch)
#define BQ_FIXED_SCRATCH_BYTES (4u << 20)

namespace bq {

struct InitEntry {
  long long off;  // complex element offset in the state
  double re, im;
};

cudaError_t launch_stage(const StageArgs& a, int dtype, int nm, int n_work, int smem_bytes, cudaStream_t s);
// Single-mode fast path (one CTA per system, whole system in shared memory); the caller
// checks bq_m1_eligible().
cudaError_t launch_stage_m1(const StageArgs& a, const M1Sys* m1, int variant, int dtype, int n_work, int smem_bytes,
                            cudaStream_t s);
// Batched persistent solve; capacity_class 0 = systems of up to 1792 points; at most
// cap_per_sm resident CTAs per SM (0: the occupancy limit).
cudaError_t launch_solve_m1(const SolveArgs& a, int dtype, int capacity_class, int smem_bytes, int cap_per_sm,
                            cudaStream_t s, int* grid_out);
// Adjoint RK4 stage (transposed-source pre-pass when max_s > 0, then the stage kernel).
cudaError_t launch_adjoint(const AdjArgs& a, int dtype, int nm, int n_work, int smem_bytes, int n_sys, int max_s,
                           cudaStream_t s);
cudaError_t launch_adj_seed(const SysDesc* sys, const EvalGroup* groups, const EvalEntry* entries, const void* y,
                            void* lam, int n_groups, int dtype, cudaStream_t s);
// Pipelined single-mode stage (persistent CTAs, bulk-copy pipeline, drive envelopes evaluated
// in the kernel), RK4 stage `stage` (1..4).
cudaError_t launch_stage_pipe(const PipeArgs& a, int variant, int dtype, int stage, int grid, int smem_bytes,
                              cudaStream_t s);
// n_steps RK4 steps of the pipelined path in one launch (stage inputs alternating between ua
// and ub; the step counter advances by n_steps), and its resident CTAs per SM.
cudaError_t launch_steps_pipe(const PipeArgs& a, void* ua, void* ub, int n_steps, int variant, int dtype, int grid,
                              int smem_bytes, cudaStream_t s);
cudaError_t steps_pipe_blocks_per_sm(int dtype, int variant, int smem_bytes, int* out);
cudaError_t pipe_blocks_per_sm(int dtype, int variant, int stage, int smem_bytes, int* out);
// Batched persistent solve, merged-stencil form (256 threads, M <= 45, shifts in {-1,0,1}).
cudaError_t launch_solve_mg(const SolveArgs& a, int dtype, int smem_bytes, int cap_per_sm, cudaStream_t s,
                            int* grid_out);
// Occupancy (CTAs per SM) of the persistent solve kernels at the given shared memory.
cudaError_t solve_blocks_per_sm(int dtype, int merged, int smem_bytes, int* out);
cudaError_t launch_eval(const SysDesc* sys, const EvalGroup* groups, const EvalEntry* entries, const void* y,
                        const void* comp, double2* out, int n_groups, int dtype, int small, cudaStream_t s);
// Cooperative segment kernels of the gradient (forward with or without recording, adjoint):
// the largest grid whose CTAs are all resident (0 if the device has no cooperative launch),
// and the launch itself (grid CTAs of BQ_BLOCK threads, at most that largest grid).
cudaError_t coop_max_grid(int dtype, int nm, bool bwd, int smem_bytes, int* out);
cudaError_t launch_coop(int dtype, int nm, bool bwd, CoopArgs P, int smem_bytes, int grid, cudaStream_t s);
// Per-problem sums of the per-system Tr(rho0 A) contributions of the pipelined stage 4.
cudaError_t launch_obs_sum(const double2* obs, const EvalGroup* groups, int n_groups, double2* out, cudaStream_t s);
// Device address of the fixed RK4 scratch on the current device (looked up once per device).
cudaError_t fixed_scratch(void** ptr);
cudaError_t launch_scatter(const InitEntry* ent, int n, void* y, int dtype, cudaStream_t s);

}  // namespace bq
