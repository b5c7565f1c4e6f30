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
cudaError_t launch_eval(const SysDesc* sys, const EvalGroup* groups, const EvalEntry* entries, const void* y,
                        double2* out, int n_groups, int dtype, cudaStream_t s);
// Device address of the fixed RK4 scratch on the current device (looked up once per device).
cudaError_t fixed_scratch(void** ptr);
cudaError_t launch_scatter(const InitEntry* ent, int n, void* y, int dtype, cudaStream_t s);

}  // namespace bq
