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
// The opt-in shared-memory limit of kernel `kern`, set once per kernel (idempotent, so a race
// between threads is harmless).
template <class K>
cudaError_t allow_smem(K kern, bool* done) {
  if (*done) return cudaSuccess;
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if (e == cudaSuccess) *done = true;
  return e;
}

template <bool W, bool ONE>
cudaError_t launch_pipe(const void* src, void* dst, const StepParams& p, const PipeParams& pp, int* status, int grid,
                        int threads, int smem, cudaStream_t s) {
  auto kern = k_step_pipe<L, S, RLB_INST_TX, W, (bool)RLB_INST_ROWS, ONE>;
  static bool attr_set = false;
  cudaError_t e = allow_smem(kern, &attr_set);
  if (e != cudaSuccess) return e;
  kern<<<grid, threads, smem, s>>>((const T*)src, (T*)dst, p, pp, status);
  return cudaGetLastError();
}
template <bool W, bool ONE>
cudaError_t launch_pipe_batch(const BatchMember* m, const int* tm, int launch, const PipeParams& pp, int* timeout,
                              int grid, int threads, int smem, cudaStream_t s) {
  auto kern = k_step_pipe_batch<L, S, RLB_INST_TX, W, (bool)RLB_INST_ROWS, ONE>;
  static bool attr_set = false;
  cudaError_t e = allow_smem(kern, &attr_set);
  if (e != cudaSuccess) return e;
  kern<<<grid, threads, smem, s>>>(m, tm, launch, pp, timeout);
  return cudaGetLastError();
}

// One warp per float cell exists for float storage with 128-cell tiles and 96-cell row tiles.
constexpr bool kOneWarp = std::is_same<S, StoreF32>::value && (RLB_INST_TX == 128 || RLB_INST_TX == 96);
}  // namespace

// One time step of every active batch member on the pipelined kernel (walls: some member has
// bounce-back walls; split = 0: one warp per float cell).
cudaError_t RLB_PIPE_FN(pipe_batch, RLB_INST_TX)(const BatchMember* m, const int* tm, int launch, const PipeParams& pp,
                                                 int* timeout, int split, int walls, int grid, int threads, int smem,
                                                 cudaStream_t s) {
  if constexpr (kOneWarp) {
    if (!split) {
      if (walls) return launch_pipe_batch<true, true>(m, tm, launch, pp, timeout, grid, threads, smem, s);
      return launch_pipe_batch<false, true>(m, tm, launch, pp, timeout, grid, threads, smem, s);
    }
  } else if (!split && std::is_same<S, StoreF32>::value) {
    return cudaErrorInvalidValue;
  }
  if (walls) return launch_pipe_batch<true, false>(m, tm, launch, pp, timeout, grid, threads, smem, s);
  return launch_pipe_batch<false, false>(m, tm, launch, pp, timeout, grid, threads, smem, s);
}

// One time step of the whole lattice in one launch, compiled with the bounce-back patch only for
// lattices that have walls.
cudaError_t RLB_PIPE_FN(pipe, RLB_INST_TX)(const void* src, void* dst, const StepParams& p, const PipeParams& pp,
                                           int* status, int split, int grid, int threads, int smem, cudaStream_t s) {
  if constexpr (kOneWarp) {
    if (!split) {
      if (p.has_wall) return launch_pipe<true, true>(src, dst, p, pp, status, grid, threads, smem, s);
      return launch_pipe<false, true>(src, dst, p, pp, status, grid, threads, smem, s);
    }
  } else if (!split && std::is_same<S, StoreF32>::value) {
    return cudaErrorInvalidValue;
  }
  if (p.has_wall) return launch_pipe<true, false>(src, dst, p, pp, status, grid, threads, smem, s);
  return launch_pipe<false, false>(src, dst, p, pp, status, grid, threads, smem, s);
}
}  // namespace rlb
