// Kernels of one (order, storage) pair that do not depend on the step variant (fields, initial
// state, format conversion, the reduction's second pass) and the dispatch to the per-variant units.
#include "rlb_inst_select.h"

namespace rlb {
namespace {
using namespace inst;

cudaError_t step(const void* src, void* dst, const StepParams& p, int* status, bool general, int variant,
                 cudaStream_t s) {
  if (kFloat) {
    switch (variant < kVariants ? variant : 0) {
      case 1: return RLB_VFN(step, 1)(src, dst, p, status, general, s);
      case 2: return RLB_VFN(step, 2)(src, dst, p, status, general, s);
      case 3: return RLB_VFN(step, 3)(src, dst, p, status, general, s);
      default: break;
    }
  }
  return RLB_VFN(step, 0)(src, dst, p, status, general, s);
}

cudaError_t batch_step(const BatchMember* m, const int* tm, int row_tiles, int shell_tiles, int li, int* counters,
                       int variant, int walls, int grid, cudaStream_t s) {
  if (kFloat) {
    switch (variant < kVariants ? variant : 0) {
      case 1: return RLB_VFN(batch, 1)(m, tm, row_tiles, shell_tiles, li, counters, walls, grid, s);
      case 2: return RLB_VFN(batch, 2)(m, tm, row_tiles, shell_tiles, li, counters, walls, grid, s);
      case 3: return RLB_VFN(batch, 3)(m, tm, row_tiles, shell_tiles, li, counters, walls, grid, s);
      default: break;
    }
  }
  return RLB_VFN(batch, 0)(m, tm, row_tiles, shell_tiles, li, counters, walls, grid, s);
}

int batch_blocks_per_sm(int variant) {
  if (kFloat) {
    switch (variant < kVariants ? variant : 0) {
      case 1: return RLB_VFN(occupancy, 1)();
      case 2: return RLB_VFN(occupancy, 2)();
      case 3: return RLB_VFN(occupancy, 3)();
      default: break;
    }
  }
  return RLB_VFN(occupancy, 0)();
}

cudaError_t fields(const void* src, const StepParams& p, const FieldOut& f, double* partial, int* status, bool pull,
                   int block0, int block1, cudaStream_t s) {
  const int blocks = block1 - block0;
  if (blocks <= 0) return cudaSuccess;
  // the modulo wrap only for lattices with a periodic axis shorter than the stencil reach
  if (pull && p.general)
    k_fields<L, S, true, true><<<blocks, kMomThreads, 0, s>>>((const T*)src, p, f, partial, status, block0);
  else if (pull)
    k_fields<L, S, true, false><<<blocks, kMomThreads, 0, s>>>((const T*)src, p, f, partial, status, block0);
  else
    k_fields<L, S, false, false><<<blocks, kMomThreads, 0, s>>>((const T*)src, p, f, partial, status, block0);
  return cudaGetLastError();
}

cudaError_t init(const double* n, const double* Tf, const double* u, void* dst, const StepParams& p, int* status,
                 int c0, int c1, cudaStream_t s) {
  if (c1 <= c0) return cudaSuccess;
  const int blocks = (c1 - c0 + 127) / 128;
  k_init<L, S><<<blocks, 128, 0, s>>>(n, Tf, u, (T*)dst, p, status, c0, c1);
  return cudaGetLastError();
}

cudaError_t convert_pops(void* pop, double* dbl, int i0, int i1, bool to_f64, const StepParams& p, cudaStream_t s) {
  const int blocks = (p.cells + 127) / 128;
  if (to_f64)
    k_convert<L, S, true><<<blocks, 128, 0, s>>>((T*)pop, dbl, 0, i0, i1, p);
  else
    k_convert<L, S, false><<<blocks, 128, 0, s>>>((T*)pop, dbl, 0, i0, i1, p);
  return cudaGetLastError();
}

cudaError_t pipe_step(const void* src, void* dst, const StepParams& p, const PipeParams& pp, int* status, int tx,
                      int rows, int split, int grid, int threads, int smem, cudaStream_t s) {
  if (rows) {
    if (tx == 96) return RLB_RFN(pipe, 96)(src, dst, p, pp, status, split, grid, threads, smem, s);
    if (tx != 128) return cudaErrorInvalidValue;
    return RLB_RFN(pipe, 128)(src, dst, p, pp, status, split, grid, threads, smem, s);
  }
  if (tx == 128) return RLB_PFN(pipe, 128)(src, dst, p, pp, status, split, grid, threads, smem, s);
  return RLB_PFN(pipe, 64)(src, dst, p, pp, status, split, grid, threads, smem, s);
}

cudaError_t pipe_batch_step(const BatchMember* m, const int* tm, int launch, const PipeParams& pp, int* timeout, int tx,
                            int rows, int split, int walls, int grid, int threads, int smem, cudaStream_t s) {
  if (rows) {
    if (tx == 96) return RLB_RFN(pipe_batch, 96)(m, tm, launch, pp, timeout, split, walls, grid, threads, smem, s);
    if (tx != 128) return cudaErrorInvalidValue;
    return RLB_RFN(pipe_batch, 128)(m, tm, launch, pp, timeout, split, walls, grid, threads, smem, s);
  }
  if (tx == 128) return RLB_PFN(pipe_batch, 128)(m, tm, launch, pp, timeout, split, walls, grid, threads, smem, s);
  return RLB_PFN(pipe_batch, 64)(m, tm, launch, pp, timeout, split, walls, grid, threads, smem, s);
}

}  // namespace

#define RLB_CAT_(a, b, c, d) a##b##c##d
#define RLB_NAME(o, s) RLB_CAT_(launchers_o, o, _s, s)
extern const Launchers RLB_NAME(RLB_INST_ORDER, RLB_INST_STORAGE) = {
    step, fields, init, convert_pops, inst::kVariants, batch_step, batch_blocks_per_sm, pipe_step, pipe_batch_step};

#if RLB_INST_ORDER == 3 && RLB_INST_STORAGE == 0
// Second pass of the conserved-density sums: one block adds the per-block partials in a fixed
// order (thread t takes blocks t, t + 256, ...; then a shuffle and shared-memory tree), so the
// totals are bitwise reproducible.
__global__ void __launch_bounds__(kReduceThreads) k_reduce_partials(const double* __restrict__ partial, int nblocks,
                                                                     double* __restrict__ totals) {
  __shared__ double ws[kReduceThreads / 32][5];
  double d[5] = {0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblocks; b += kReduceThreads)
#pragma unroll
    for (int k = 0; k < 5; ++k) d[k] += partial[(long long)b * 5 + k];
#pragma unroll
  for (int k = 0; k < 5; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d[k] += __shfl_down_sync(0xffffffffu, d[k], o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 5; ++k) ws[warp][k] = d[k];
  __syncthreads();
  if (threadIdx.x < 5) {
    double s = 0.0;
    for (int w = 0; w < kReduceThreads / 32; ++w) s += ws[w][threadIdx.x];
    totals[threadIdx.x] = s;
  }
}

cudaError_t launch_reduce_partials(const double* partial, int nblocks, double* totals, cudaStream_t s) {
  k_reduce_partials<<<1, kReduceThreads, 0, s>>>(partial, nblocks, totals);
  return cudaGetLastError();
}
#endif
}  // namespace rlb
