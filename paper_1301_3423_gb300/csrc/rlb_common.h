// Definitions shared by the host-side C ABI and the kernels.
#pragma once

namespace rlb {

constexpr int kStepThreads = 128;    // threads per block of the step kernel (one cell each)
constexpr int kMomThreads = 128;     // threads per block of the fields kernel
constexpr int kReduceThreads = 256;  // threads of the single-block second reduction pass
constexpr int kDefaultStepVariant = 0;  // step-kernel variant before autotuning (float storage)

// Step-kernel variants.  0..3: one cell per thread with all populations in registers (float
// storages; double storage has variant 0 only, which reads its populations twice).  4 and up: the
// pipelined kernel (k_step_pipe) in the shapes of kPipeConfigs, for every storage, on lattices whose
// rows start on 16-byte boundaries.
constexpr int kNumRegVariants = 4;
struct PipeConfig {
  int tx;           // tile width in cells (64 or 128; 96 for row tiles)
  int cons_warps;   // consumer warps per block: TX / 32 per tile, twice that with float storage
                    // (two warps per cell); a multiple of the warps per tile
  int ctas_per_sm;  // resident blocks per SM (the shared memory is split between them)
  int producers;    // producer warps per block (each copies every producers-th population of every tile)
  int rows;         // 0: a tile is a TX-cell segment of one row; 1: a tile is TX / nx whole rows of
                    // an x-periodic lattice with nx <= TX ("row tiles", one copy per population)
  int split;        // float storage: 1 = two warps per cell (each half the populations), 0 = one;
                    // other storages always take one warp per cell (the flag makes no difference)
};
// A block's stage count is a multiple of its consumer-group count, so that every stage is read by
// one consumer group, in the order of the stage's uses like every producer: a parity wait then
// always refers to the phase it means.  With as many stages as groups each group refills its one
// stage while the other groups compute.
constexpr PipeConfig kPipeConfigs[] = {
    {128, 8, 1, 8, 0, 1}, {128, 8, 1, 4, 0, 1},  {64, 8, 1, 8, 0, 1},  {64, 4, 1, 4, 0, 1},
    {128, 8, 1, 6, 0, 1}, {64, 8, 1, 4, 0, 1},   {128, 4, 1, 4, 0, 1}, {64, 2, 1, 4, 0, 1},
    {128, 8, 1, 4, 1, 1}, {128, 8, 1, 8, 1, 1},  {128, 4, 1, 4, 1, 1}, {128, 12, 1, 4, 0, 0},
    {128, 12, 1, 4, 1, 0}, {128, 12, 1, 2, 0, 0}, {128, 12, 1, 2, 1, 0}, {96, 12, 1, 4, 1, 0}};
constexpr int kNumPipeConfigs = sizeof(kPipeConfigs) / sizeof(kPipeConfigs[0]);
constexpr int kNumVariantsTotal = kNumRegVariants + kNumPipeConfigs;
constexpr int kPipeMaxStages = 16;
constexpr int kPipeMaxConsumerWarps = 12;
constexpr int kPipeMaxProducerWarps = 12;
constexpr int kPipeMaxWarps = 16;  // consumers + producers: the launch bound of k_step_pipe (128 registers)
constexpr int kPipeHeaderBytes = 1024;  // mbarriers (2 x 16 x 8 B) and the per-population velocity table
constexpr int kPipeXchgBytesPerPair = 2 * 2 * 13 * 32 * 4;  // partial moments a consumer warp pair exchanges
// Bytes of slack before and after every population buffer: the pipelined kernel's copies of a row
// segment next to a lattice end may start up to one granule before the row and end up to one tile
// plus a granule plus the stencil reach after it ((128 + 2 + 6) doubles = 1088 bytes at most).
constexpr int kPopGuardBytes = 2048;

// ---------------------------------------------------------------------------------------------
// launch parameters
// ---------------------------------------------------------------------------------------------
struct StepParams {
  int nx, ny, nz, nxy, cells;
  int bc[3];                // 0 periodic, 1 copy-out
  long long off[128];       // interior pull offset of population i: i*cells - (vx + vy*nx + vz*nxy)
  double tau_fixed;         // > 0.5: constant tau'
  double tau_coef;          // tau' = 1/2 + tau_coef / T
  int tau_local;            // T = local Landau temperature (1) or T_ref (0)
  double T_ref;
  // the same in float for the float step paths (no double instruction on their hot path)
  int tau_is_fixed;
  float tau_fixed_f, tau_coef_f, T_ref_f;
  float gamma_thr2;         // reduced-precision paths: Landau in double above this gamma^2
  int landau_fp64;
  float half_nref;          // F16DEV: n_ref / 2
  int general;              // a periodic axis is shorter than the stencil reach (modulo wrap)
  int debug;                // kDebug* bits (testing only; 0 in normal use)
  int has_wall;             // some axis has bounce-back walls (bc == kBounceBack)
  // Interior box: cells whose whole stencil stays inside the lattice, x in [ix0, ix0 + ixn) etc.
  int ix0, ixn, iy0, iyn, iz0, izn;
  int int_segs;             // 32-aligned warp segments per row of the row kernel (all nx cells)
  int int_warps;            // interior segments in total
  int shell_cells;          // cells outside the interior box
  int row_segs;             // 32-aligned warp segments per row (all nx cells)
  int shell_rows;           // rows whose y or z lies outside the interior box
  int shell_warps;          // shell_rows * row_segs
};

// per-axis boundary codes, as in rlb_bc
enum : int { kPeriodic = 0, kCopyOut = 1, kBounceBack = 2 };

// status words: cell updates without a Landau frame, cells with invalid initial fields, bounded
// device-side waits that ran out, cells with non-finite moments (found by the fields kernel), pull
// addresses outside the population buffer and its guard bytes (found and skipped by the pipelined
// kernel)
enum : int {
  kStatusNonconv = 0,
  kStatusBadInit = 1,
  kStatusTimeout = 2,
  kStatusNan = 3,
  kStatusBounds = 4,
  kStatusWords = 8
};

// StepParams::debug bits (testing only)
enum : int { kDebugStallProducers = 1 };  // the pipelined step's producers do nothing: every wait runs out

// Launch shape of a pipelined step (k_step_pipe, k_step_pipe_batch): tiles are TX-cell segments of
// the lattice rows, tile t = row * ceil(nx / TX) + seg, or with row tiles groups of TX / nx
// consecutive rows, tile t = rows t G .. t G + G - 1; block b takes tiles b, b + grid, ...
struct PipeParams {
  int producers;  // producer warps per block
  int ntiles;     // tiles of the launch: ceil(nx / TX) * ny * nz per lattice (ceil(ny nz / G) with row tiles)
  int nstage;     // shared-memory stages per block (<= 16)
  int groups;     // consumer groups per block (TX / 32 warps each, twice that for float storage)
};

// Output arrays of the fields kernel: n, eps, U0, U1, U2, U3, one value per cell each (device
// memory, or host memory the device can address).
struct FieldOut {
  double* f[6];
};

// One lattice of a batched step (see k_step_batch).
struct BatchMember {
  StepParams p;
  void* buf[2];       // population buffers
  int* status;        // the member's status words
  int parity0;        // buffer holding the state before launch 0 of this run
  int steps_left;     // launches with index >= steps_left leave this member alone
  int row_tile_begin;    // first of its row tiles (4 row-kernel warps each) in the row queue
  int shell_tile_begin;  // first of its shell tiles (kStepThreads shell cells each) in the shell queue
  int pipe_tile_begin;   // first of its tiles in the pipelined kernel's tile list (k_step_pipe_batch)
};

}  // namespace rlb
