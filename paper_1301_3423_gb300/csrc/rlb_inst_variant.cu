// Step kernels of one (order, storage, variant): the interior and shell kernels of a solo step and
// the persistent batched kernel.  RLB_INST_VARIANT selects the variant (see StepVariant).
#include "rlb_inst_select.h"

#ifndef RLB_INST_VARIANT
#error "RLB_INST_VARIANT must be defined"
#endif

namespace rlb {
using namespace inst;
constexpr int V = RLB_INST_VARIANT;

namespace {
template <bool W>
void launch_step(const void* src, void* dst, const StepParams& p, int* status, bool general, cudaStream_t s) {
  if (p.int_warps > 0) {
    const int blocks = (p.int_warps + kStepThreads / 32 - 1) / (kStepThreads / 32);
    k_step_interior<L, S, V, W><<<blocks, kStepThreads, 0, s>>>((const T*)src, (T*)dst, p, status);
  }
  if (p.shell_cells > 0) {
    if (general) {
      const int blocks = (p.shell_cells + kStepThreads - 1) / kStepThreads;
      k_step_shell<L, S, true, V, W><<<blocks, kStepThreads, 0, s>>>((const T*)src, (T*)dst, p, status);
    } else {
      k_step_shell_rows<L, S, V, W><<<p.shell_warps, 32, 0, s>>>((const T*)src, (T*)dst, p, status);
    }
  }
}
}  // namespace

// One time step = the interior kernel plus the shell kernel (disjoint cells, same source), compiled
// with the bounce-back test only for lattices that have walls.
cudaError_t RLB_VFN(step, RLB_INST_VARIANT)(const void* src, void* dst, const StepParams& p, int* status,
                                            bool general, cudaStream_t s) {
  if (p.has_wall) launch_step<true>(src, dst, p, status, general, s);
  else launch_step<false>(src, dst, p, status, general, s);
  return cudaGetLastError();
}

namespace {
template <bool W>
void launch_batch(const BatchMember* m, const int* tm, int row_tiles, int shell_tiles, int li, int* counters, int grid,
                  cudaStream_t s) {
  if (row_tiles > 0)
    k_step_batch<L, S, V, W, true><<<grid, kStepThreads, 0, s>>>(m, tm, 0, row_tiles, li, counters + 2 * li);
  if (shell_tiles > 0)
    k_step_batch<L, S, V, W, false>
        <<<grid, kStepThreads, 0, s>>>(m, tm, row_tiles, row_tiles + shell_tiles, li, counters + 2 * li + 1);
}
}  // namespace

cudaError_t RLB_VFN(batch, RLB_INST_VARIANT)(const BatchMember* m, const int* tm, int row_tiles, int shell_tiles,
                                             int li, int* counters, int walls, int grid, cudaStream_t s) {
  if (walls) launch_batch<true>(m, tm, row_tiles, shell_tiles, li, counters, grid, s);
  else launch_batch<false>(m, tm, row_tiles, shell_tiles, li, counters, grid, s);
  return cudaGetLastError();
}

int RLB_VFN(occupancy, RLB_INST_VARIANT)() {
  int nb = 0;  // both instantiations have the same launch bounds
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_batch<L, S, V, false, true>, kStepThreads, 0) !=
      cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return nb > 0 ? nb : 1;
}
}  // namespace rlb
