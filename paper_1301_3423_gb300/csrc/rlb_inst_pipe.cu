// Pipelined step kernel (k_step_pipe) of one (order, storage, tile width, tile kind); RLB_INST_TX
// selects the width and RLB_INST_ROWS = 1 the row tiles.  One unit per width and kind so that the
// translation units build in parallel.
#include "rlb_inst_select.h"
#include "rlb_pipe.cuh"

#ifndef RLB_INST_TX
#error "RLB_INST_TX must be defined"
#endif
#ifndef RLB_INST_ROWS
#define RLB_INST_ROWS 0
#endif
#if RLB_INST_ROWS
#define RLB_PIPE_FN(fn, tx) RLB_RFN(fn, tx)
#else
#define RLB_PIPE_FN(fn, tx) RLB_PFN(fn, tx)
#endif

namespace rlb {
using namespace inst;

namespace {
template <bool W>
cudaError_t launch_pipe(const void* src, void* dst, const StepParams& p, const PipeParams& pp, int* status, int grid,
                        int threads, int smem, cudaStream_t s) {
  auto kern = k_step_pipe<L, S, RLB_INST_TX, W, (bool)RLB_INST_ROWS>;
  // the opt-in shared-memory limit, set once per kernel (idempotent, so a race between threads is harmless)
  static bool attr_set = false;
  if (!attr_set) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  kern<<<grid, threads, smem, s>>>((const T*)src, (T*)dst, p, pp, status);
  return cudaGetLastError();
}
template <bool W>
cudaError_t launch_pipe_batch(const BatchMember* m, const int* tm, int launch, const PipeParams& pp, int* timeout,
                              int grid, int threads, int smem, cudaStream_t s) {
  auto kern = k_step_pipe_batch<L, S, RLB_INST_TX, W, (bool)RLB_INST_ROWS>;
  static bool attr_set = false;
  if (!attr_set) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  kern<<<grid, threads, smem, s>>>(m, tm, launch, pp, timeout);
  return cudaGetLastError();
}
}  // namespace

// One time step of every active batch member on the pipelined kernel (walls: some member has
// bounce-back walls).
cudaError_t RLB_PIPE_FN(pipe_batch, RLB_INST_TX)(const BatchMember* m, const int* tm, int launch, const PipeParams& pp,
                                             int* timeout, int walls, int grid, int threads, int smem,
                                             cudaStream_t s) {
  if (walls) return launch_pipe_batch<true>(m, tm, launch, pp, timeout, grid, threads, smem, s);
  return launch_pipe_batch<false>(m, tm, launch, pp, timeout, grid, threads, smem, s);
}

// One time step of the whole lattice in one launch, compiled with the bounce-back patch only for
// lattices that have walls.
cudaError_t RLB_PIPE_FN(pipe, RLB_INST_TX)(const void* src, void* dst, const StepParams& p, const PipeParams& pp,
                                       int* status, int grid, int threads, int smem, cudaStream_t s) {
  if (p.has_wall) return launch_pipe<true>(src, dst, p, pp, status, grid, threads, smem, s);
  return launch_pipe<false>(src, dst, p, pp, status, grid, threads, smem, s);
}
}  // namespace rlb
