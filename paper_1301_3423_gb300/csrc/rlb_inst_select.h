// Selects the lattice L and storage S of an instantiation unit from RLB_INST_ORDER (2 or 3) and
// RLB_INST_STORAGE (0 = double, 1 = float, 2 = half deviation), and names its per-variant entry
// points: RLB_VFN(step, V) is step_o<order>_s<storage>_v<V>.
#pragma once
#include "rlb_kernels.cuh"
#include "rlb_launch.h"

#ifndef RLB_INST_ORDER
#error "RLB_INST_ORDER must be defined"
#endif
#ifndef RLB_INST_STORAGE
#error "RLB_INST_STORAGE must be defined"
#endif

#define RLB_CAT7_(a, b, c, d, e, f, g) a##b##c##d##e##f##g
#define RLB_CAT7(a, b, c, d, e, f, g) RLB_CAT7_(a, b, c, d, e, f, g)
#define RLB_VFN(fn, v) RLB_CAT7(fn, _o, RLB_INST_ORDER, _s, RLB_INST_STORAGE, _v, v)

namespace rlb {
namespace inst {
#if RLB_INST_ORDER == 3
using L = Quad3;
#else
using L = Quad2;
#endif
#if RLB_INST_STORAGE == 0
using S = StoreF64;
#elif RLB_INST_STORAGE == 1
using S = StoreF32;
#else
using S = StoreF16Dev;
#endif
using T = typename S::T;
constexpr bool kFloat = std::is_same<typename S::A, float>::value;
constexpr int kVariants = kFloat ? kNumVariants : 1;
}  // namespace inst

// Per-variant entry points (defined in rlb_inst_variant.cu, one unit per variant).
#define RLB_DECLARE_VARIANT(v)                                                                               \
  cudaError_t RLB_VFN(step, v)(const void* src, void* dst, const StepParams& p, int* status, bool general,   \
                               cudaStream_t s);                                                              \
  cudaError_t RLB_VFN(batch, v)(const BatchMember* m, const int* tm, int row_tiles, int shell_tiles, int li, \
                                int* counters, int walls, int grid, cudaStream_t s);                                                             \
  int RLB_VFN(occupancy, v)();
// Pipelined step kernel per tile width (rlb_inst_pipe.cu, one unit per width).
#define RLB_PFN(fn, tx) RLB_CAT7(fn, _o, RLB_INST_ORDER, _s, RLB_INST_STORAGE, _x, tx)
#define RLB_DECLARE_PIPE(tx)                                                                                   \
  cudaError_t RLB_PFN(pipe, tx)(const void* src, void* dst, const StepParams& p, const PipeParams& pp, int* status, \
                                int split, int grid, int threads, int smem, cudaStream_t s);                      \
  cudaError_t RLB_PFN(pipe_batch, tx)(const BatchMember* m, const int* tm, int launch, const PipeParams& pp,        \
                                      int* timeout, int split, int walls, int grid, int threads, int smem,          \
                                      cudaStream_t s);
RLB_DECLARE_PIPE(64)
RLB_DECLARE_PIPE(128)
#undef RLB_DECLARE_PIPE
// ... and with row tiles (RLB_INST_ROWS = 1), tile widths 128 and 96.
#define RLB_RFN(fn, tx) RLB_CAT7(fn, _o, RLB_INST_ORDER, _s, RLB_INST_STORAGE, _r, tx)
#define RLB_DECLARE_ROWS(tx)                                                                                   \
  cudaError_t RLB_RFN(pipe, tx)(const void* src, void* dst, const StepParams& p, const PipeParams& pp, int* status, \
                                int split, int grid, int threads, int smem, cudaStream_t s);                      \
  cudaError_t RLB_RFN(pipe_batch, tx)(const BatchMember* m, const int* tm, int launch, const PipeParams& pp,        \
                                      int* timeout, int split, int walls, int grid, int threads, int smem,          \
                                      cudaStream_t s);
RLB_DECLARE_ROWS(128)
RLB_DECLARE_ROWS(96)
#undef RLB_DECLARE_ROWS

RLB_DECLARE_VARIANT(0)
RLB_DECLARE_VARIANT(1)
RLB_DECLARE_VARIANT(2)
RLB_DECLARE_VARIANT(3)
#undef RLB_DECLARE_VARIANT
}  // namespace rlb
