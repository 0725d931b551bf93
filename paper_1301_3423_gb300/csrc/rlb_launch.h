// Host-side launchers, one set per (order, storage) instantiation (rlb_inst.cu is compiled once
// per pair so that the translation units build in parallel).
#pragma once
#include <cuda_runtime.h>

#include "rlb_common.h"

namespace rlb {
struct StepParams;
struct PipeParams;
struct BatchMember;

struct Launchers {
  cudaError_t (*step)(const void* src, void* dst, const StepParams& p, int* status, bool general, int variant,
                      cudaStream_t s);
  // fields and partial sums of the lattice's kMomThreads-cell blocks [block0, block1)
  cudaError_t (*fields)(const void* src, const StepParams& p, const FieldOut& out, double* partial, int* status,
                        bool pull, int block0, int block1, cudaStream_t s);
  // initial populations of cells [c0, c1)
  cudaError_t (*init)(const double* n, const double* T, const double* u, void* dst, const StepParams& p, int* status,
                      int c0, int c1, cudaStream_t s);
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
  // one time step of the pipelined kernel with tile width tx (64 or 128), row tiles if rows != 0
  // (tx 128 or 96), float cells split between two warps if split != 0 (float storage)
  cudaError_t (*pipe_step)(const void* src, void* dst, const StepParams& p, const PipeParams& pp, int* status, int tx,
                           int rows, int split, int grid, int threads, int smem, cudaStream_t s);
  // one time step of the batched pipelined kernel (launch index `launch`) over the members' tiles;
  // walls != 0 selects the kernel with the bounce-back patch
  cudaError_t (*pipe_batch_step)(const BatchMember* members, const int* tile_member, int launch, const PipeParams& pp,
                                 int* timeout, int tx, int rows, int split, int walls, int grid, int threads, int smem,
                                 cudaStream_t s);
};

// Block layout of pipelined variant v (>= kNumRegVariants) for q populations of `elem` bytes:
// stages (the largest multiple of the consumer-group count that fits the shared memory of one
// block, at least one per group and two in all), groups, threads and shared-memory bytes.  False if the variant
// does not exist for this storage.
struct PipeLayout {
  int tx, nstage, groups, producers, threads, smem, ctas_per_sm, rows, split;
};

// A lattice row of nx cells suits tiles of tx cells when its rows start on 16-byte boundaries and
// the tiles' lanes are at least `eighths` / 8 used.  Two warps per float cell want 7/8 (a 96-cell
// row in 128-cell tiles leaves 1/4 idle and ran slower than the register kernel); one warp per
// float cell 3/4 (200-cell rows in 128-cell tiles ran faster than the register kernel).
inline bool pipe_fits(int nx, int tx, int elem, int eighths = 7) {
  if (nx % (16 / elem) != 0) return false;
  const long long used = (long long)((nx + tx - 1) / tx) * tx;
  return 8LL * nx >= eighths * used;
}

// The fill rule of a layout: 3/4 for one warp per float cell, 7/8 otherwise.
inline int fill_eighths(const PipeLayout& lay, int elem) { return (elem == 4 && !lay.split) ? 6 : 7; }

// Row tiles of tx cells can take a lattice whose x axis is periodic and at least the stencil reach
// vmax_x long (one wrap per pull), with nx <= tx cells per row starting on 16-byte boundaries.
inline bool rows_possible(int nx, int tx, int elem, int bc_x, int vmax_x) {
  return bc_x == kPeriodic && nx <= tx && nx >= vmax_x && nx % (16 / elem) == 0;
}

// ... and suit it when the tile's G = tx / nx rows use at least 3/4 of its lanes (the batch's
// rule: in the batched mix of 32- to 128-cell rows every such member stepped faster in row tiles
// than on the register kernels).
inline bool rows_fit(int nx, int tx, int elem, int bc_x, int vmax_x) {
  return rows_possible(nx, tx, elem, bc_x, vmax_x) && 4 * (tx / nx) * nx >= 3 * tx;
}

// A single lattice's rule for layouts with two warps per float cell and half storage: several
// rows per tile (G >= 2) at 3/4 of the lanes, or one row that fills the tile (measured on GB300
// alone: 32-, 48- and 64-cell rows as fast as or faster than the register kernels, 128-cell rows
// as fast as row segments with float storage and 1.26x faster with half storage, while one 96-cell
// row per tile ran 1.4x slower than the register kernels).  One warp per float cell takes rows_fit
// (a 96-cell row per tile ran 1.07x faster than the register kernels).
inline bool rows_fit_solo(int nx, int tx, int elem, int bc_x, int vmax_x) {
  if (!rows_fit(nx, tx, elem, bc_x, vmax_x)) return false;
  return tx / nx >= 2 || nx == tx;
}

// Tiles of one lattice: row tiles (groups of tx / nx rows) or tx-cell row segments.
inline long long pipe_tile_count(int nx, int ny, int nz, int tx, int rows) {
  if (rows) {
    const long long g = tx / nx;
    return ((long long)ny * nz + g - 1) / g;
  }
  return (long long)((nx + tx - 1) / tx) * ny * nz;
}

inline bool pipe_layout(int v, int q, int elem, int smem_per_sm, int smem_optin, PipeLayout* out) {
  if (v < kNumRegVariants || v >= kNumVariantsTotal) return false;
  const PipeConfig& cf = kPipeConfigs[v - kNumRegVariants];
  const int A = 16 / elem;
  const long long stage = (long long)q * (cf.tx + A) * elem;
  long long budget = smem_per_sm / cf.ctas_per_sm - 1024;
  if (budget > smem_optin) budget = smem_optin;
  const bool split = elem == 4 && cf.split;  // float storage: two consumer warps per cell
  const int wpt = cf.tx / 32 * (split ? 2 : 1);
  const int groups = cf.cons_warps / wpt;
  if (groups < 1 || cf.cons_warps % wpt != 0 || cf.producers < 1 || cf.producers > q) return false;
  if (cf.producers > kPipeMaxProducerWarps || cf.cons_warps > kPipeMaxConsumerWarps ||
      cf.cons_warps + cf.producers > kPipeMaxWarps)
    return false;
  const long long xchg = split ? (long long)cf.cons_warps / 2 * kPipeXchgBytesPerPair : 0;
  long long fit = (budget - kPipeHeaderBytes - xchg) / stage;
  if (fit > kPipeMaxStages) fit = kPipeMaxStages;
  const int nstage = (int)(fit / groups * groups);
  if (nstage < groups || nstage < 2) return false;
  if (out) *out = PipeLayout{cf.tx, nstage, groups, cf.producers, (cf.cons_warps + cf.producers) * 32,
                             (int)(kPipeHeaderBytes + nstage * stage + xchg), cf.ctas_per_sm, cf.rows, split};
  return true;
}

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
