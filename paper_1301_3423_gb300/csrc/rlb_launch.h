// Host-side launchers, one set per (order, storage) instantiation (rlb_inst.cu is compiled once
// per pair so that the translation units build in parallel).
#pragma once
#include <cuda_runtime.h>

namespace rlb {
struct StepParams;
struct PipeParams;
struct BatchMember;

struct Launchers {
  cudaError_t (*step)(const void* src, void* dst, const StepParams& p, int* status, bool general, int variant,
                      cudaStream_t s);
  cudaError_t (*fields)(const void* src, const StepParams& p, double* fields, double* partial, int* status, bool pull,
                        cudaStream_t s);
  cudaError_t (*init)(const double* n, const double* T, const double* u, void* dst, const StepParams& p, int* status,
                      cudaStream_t s);
  cudaError_t (*convert)(void* pop, double* dbl, int i0, int i1, bool to_f64, const StepParams& p, cudaStream_t s);
  int step_variants;  // number of step-kernel variants the autotuner may choose from
  // one time step of the persistent batched kernels: a launch over the row tiles [0, row_tiles) and
  // one over the shell tiles [row_tiles, row_tiles + shell_tiles) of the tile -> member table, with
  // counters[2 launch_index] and counters[2 launch_index + 1]; walls != 0 selects the kernels with
  // the bounce-back test (some member has walls)
  cudaError_t (*batch_step)(const BatchMember* members, const int* tile_member, int row_tiles, int shell_tiles,
                            int launch_index, int* counters, int variant, int walls, int grid, cudaStream_t s);
  // resident blocks per SM of the batched step for a variant
  int (*batch_blocks_per_sm)(int variant);
  // one time step of the pipelined kernel with tile width tx (32 or 64)
  cudaError_t (*pipe_step)(const void* src, void* dst, const StepParams& p, const PipeParams& pp, int* status, int tx,
                           int grid, int threads, int smem, cudaStream_t s);
};

#define RLB_DECLARE_LAUNCHERS(ORDER, STORAGE) extern const Launchers launchers_o##ORDER##_s##STORAGE;
RLB_DECLARE_LAUNCHERS(3, 0)
RLB_DECLARE_LAUNCHERS(3, 1)
RLB_DECLARE_LAUNCHERS(3, 2)
RLB_DECLARE_LAUNCHERS(2, 0)
RLB_DECLARE_LAUNCHERS(2, 1)
RLB_DECLARE_LAUNCHERS(2, 2)
#undef RLB_DECLARE_LAUNCHERS

cudaError_t launch_reduce_partials(const double* partial, int nblocks, double* totals, cudaStream_t s);
}  // namespace rlb
