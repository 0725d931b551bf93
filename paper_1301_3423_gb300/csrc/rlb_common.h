// Definitions shared by the host-side C ABI and the kernels.
#pragma once

namespace rlb {

constexpr int kStepThreads = 128;    // threads per block of the step kernel (one cell each)
constexpr int kMomThreads = 128;     // threads per block of the fields kernel
constexpr int kReduceThreads = 256;  // threads of the single-block second reduction pass
constexpr int kDefaultStepVariant = 0;  // step-kernel variant before autotuning (float storage)

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

enum : int { kStatusNonconv = 0, kStatusBadInit = 1, kStatusWords = 4 };

// One lattice of a batched step (see k_step_batch).
struct BatchMember {
  StepParams p;
  void* buf[2];       // population buffers
  int* status;        // the member's status words
  int parity0;        // buffer holding the state before launch 0 of this run
  int steps_left;     // launches with index >= steps_left leave this member alone
  int row_tile_begin;    // first of its row tiles (4 row-kernel warps each) in the row queue
  int shell_tile_begin;  // first of its shell tiles (kStepThreads shell cells each) in the shell queue
};

}  // namespace rlb
