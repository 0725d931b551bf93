// C ABI of librlb (declared in include/rlb.h): context management, validation, kernel launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "rlb.h"
#include "rlb_common.h"
#include "rlb_ctx.h"
#include "rlb_launch.h"
#include "rlb_quadrature.h"

using namespace rlb;

namespace {

constexpr double kHbarcGeVfm = 0.1973269804;  // CODATA hbar*c: (GeV * fm/c) -> pure number

template <class L>
struct QuadHost {
  int vel[L::Q * 3], level[L::Q];
  double p0[L::Q], w[L::Q];
  QuadHost() {
    for (int i = 0; i < L::Q; ++i) {
      vel[3 * i] = L::VX[i];
      vel[3 * i + 1] = L::VY[i];
      vel[3 * i + 2] = L::VZ[i];
      level[i] = L::LEV[i];
      p0[i] = L::P0[L::LEV[i]];
      w[i] = L::W[i];
    }
  }
};
const QuadHost<Quad3> kQuad3;
const QuadHost<Quad2> kQuad2;

size_t storage_bytes(int storage) { return storage == RLB_F64 ? 8 : (storage == RLB_F32 ? 4 : 2); }

}  // namespace



// Errors of calls that have no context (rlb_create with invalid parameters) are kept per thread.
static thread_local std::string g_create_err;

namespace rlb {
// Sets the text rlb_last_error(NULL) returns on this thread (used by context-free entry points).
__attribute__((visibility("hidden"))) void set_thread_error(const std::string& msg) { g_create_err = msg; }
}  // namespace rlb

static rlb_status fail(rlb_ctx* c, rlb_status st, const std::string& msg) {
  if (c) c->err = msg;
  else g_create_err = msg;
  return st;
}

static rlb_status cuda_fail(rlb_ctx* c, cudaError_t e, const char* where) {
  return fail(c, RLB_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define RLB_CUDA(ctx, call)                                        \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);     \
  } while (0)

extern "C" void rlb_default_params(rlb_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->order = 3;
  p->nx = p->ny = p->nz = 1;
  p->eta_over_s = 0.1;
  p->tau_prime = 0.0;
  p->tau_local_T = 1;
  p->T_ref = 1.0;
  p->dx_fm = 0.008;
  p->T_unit_GeV = 0.4;
  p->storage = RLB_F64;
  p->landau_fp64 = 0;
  p->gamma_thr = 2.0;
  p->n_ref = 1.0;
  p->step_variant = -1;
}

extern "C" rlb_status rlb_quadrature(int order, int* q, const int** vel, const int** level, const double** p0,
                                     const double** w) {
  if (order != 2 && order != 3) return RLB_EINVAL;
  const bool o3 = order == 3;
  if (q) *q = o3 ? Quad3::Q : Quad2::Q;
  if (vel) *vel = o3 ? kQuad3.vel : kQuad2.vel;
  if (level) *level = o3 ? kQuad3.level : kQuad2.level;
  if (p0) *p0 = o3 ? kQuad3.p0 : kQuad2.p0;
  if (w) *w = o3 ? kQuad3.w : kQuad2.w;
  return RLB_OK;
}

static std::string validate(const rlb_params* p) {
  if (!p) return "params is NULL";
  if (p->order != 2 && p->order != 3) return "order must be 2 or 3";
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return "lattice dimensions must be >= 1";
  const long long cells = (long long)p->nx * p->ny * p->nz;
  if (cells > 0x7fffffffll) return "more than 2^31 - 1 cells";
  for (int a = 0; a < 3; ++a)
    if (p->bc[a] != RLB_BC_PERIODIC && p->bc[a] != RLB_BC_COPYOUT && p->bc[a] != RLB_BC_BOUNCEBACK)
      return "bc must be periodic, copy-out or bounce-back";
  if (p->storage != RLB_F64 && p->storage != RLB_F32 && p->storage != RLB_F16DEV) return "unknown storage";
  if (!(p->tau_prime > 0.5)) {
    if (!(p->eta_over_s > 0) || !std::isfinite(p->eta_over_s)) return "eta_over_s must be > 0 (or tau_prime > 1/2)";
    if (!(p->dx_fm > 0) || !(p->T_unit_GeV > 0)) return "dx_fm and T_unit_GeV must be > 0";
    if (!p->tau_local_T && !(p->T_ref > 0)) return "T_ref must be > 0";
  } else if (!std::isfinite(p->tau_prime)) {
    return "tau_prime must be finite";
  }
  if (!(p->gamma_thr >= 1.0)) return "gamma_thr must be >= 1";
  if (p->storage == RLB_F16DEV && !(p->n_ref > 0)) return "n_ref must be > 0";
  if (p->step_variant < -1 || p->step_variant >= RLB_MAX_VARIANTS) return "step_variant must be -1 or 0..23";
  if (p->q > 0) {
    int q;
    const int *vel, *lev;
    const double *p0, *w;
    rlb_quadrature(p->order, &q, &vel, &lev, &p0, &w);
    if (p->q != q) return "quadrature size differs from the built-in one";
    if (!p->vel || !p->level || !p->p0 || !p->w) return "quadrature arrays missing";
    for (int i = 0; i < q; ++i) {
      if (p->vel[3 * i] != vel[3 * i] || p->vel[3 * i + 1] != vel[3 * i + 1] || p->vel[3 * i + 2] != vel[3 * i + 2] ||
          p->level[i] != lev[i] || p->p0[i] != p0[i] || p->w[i] != w[i])
        return "quadrature differs from the built-in one at population " + std::to_string(i);
    }
  }
  return "";
}

extern "C" size_t rlb_bytes_required(const rlb_params* p) {
  if (!validate(p).empty()) return 0;
  const size_t cells = (size_t)p->nx * p->ny * p->nz;
  const size_t q = p->order == 3 ? Quad3::Q : Quad2::Q;
  const size_t blocks = (cells + kMomThreads - 1) / kMomThreads;
  return 2 * (q * cells * storage_bytes(p->storage) + 2 * kPopGuardBytes) + 6 * cells * sizeof(double) +
         5 * blocks * sizeof(double) + 5 * sizeof(double) + kStatusWords * sizeof(int);
}

template <class L>
static void fill_offsets(StepParams& sp) {
  for (int i = 0; i < L::Q; ++i)
    sp.off[i] = (long long)i * sp.cells - ((long long)L::VX[i] + (long long)L::VY[i] * sp.nx +
                                           (long long)L::VZ[i] * sp.nxy);
}

template <class L>
static bool needs_general_wrap(const rlb_params& p) {
  static_assert(RLB_BC_PERIODIC == kPeriodic && RLB_BC_COPYOUT == kCopyOut && RLB_BC_BOUNCEBACK == kBounceBack,
                "boundary codes of the ABI and the kernels agree");
  return (p.bc[0] == RLB_BC_PERIODIC && p.nx < L::VMAX_X) || (p.bc[1] == RLB_BC_PERIODIC && p.ny < L::VMAX_Y) ||
         (p.bc[2] == RLB_BC_PERIODIC && p.nz < L::VMAX_Z);
}

static int vmax_x(const rlb_ctx* c) { return c->prm.order == 3 ? Quad3::VMAX_X : Quad2::VMAX_X; }

// Shape of pipelined variant v (>= kNumRegVariants) on this context's lattice: the block layout
// (pipe_layout) and the tiles.  False if the variant does not exist or the lattice cannot use it
// (rows must start on 16-byte boundaries; row tiles also need a periodic x of vmax_x .. tx cells).
static bool pipe_shape(const rlb_ctx* c, int v, PipeParams* pp, int* grid, int* threads, int* smem, int* tx = nullptr,
                       int* rows = nullptr, int* split = nullptr) {
  PipeLayout lay;
  if (c->sms <= 0 || !pipe_layout(v, c->q, (int)c->elem, c->smem_per_sm, c->smem_optin, &lay)) return false;
  if (c->sp.nx % (16 / (int)c->elem) != 0) return false;
  if (lay.rows && !rows_possible(c->sp.nx, lay.tx, (int)c->elem, c->sp.bc[0], vmax_x(c))) return false;
  const long long ntiles = pipe_tile_count(c->sp.nx, c->sp.ny, c->sp.nz, lay.tx, lay.rows);
  if (ntiles > 0x7fffffffll) return false;
  if (pp) *pp = PipeParams{lay.producers, (int)ntiles, lay.nstage, lay.groups};
  if (grid) *grid = (int)std::min<long long>((long long)c->sms * lay.ctas_per_sm, ntiles);
  if (threads) *threads = lay.threads;
  if (smem) *smem = lay.smem;
  if (tx) *tx = lay.tx;
  if (rows) *rows = lay.rows;
  if (split) *split = lay.split;
  return true;
}

static bool variant_available(const rlb_ctx* c, int v) {
  if (v < 0) return false;
  if (v < kNumRegVariants) return v < c->launch->step_variants;
  return pipe_shape(c, v, nullptr, nullptr, nullptr, nullptr);
}

// The variant rlb_step uses unless asked otherwise: the first one that suits the context in an
// order measured on GB300 (32^3 to 256^3 lattices, third order): for float storage one warp per
// cell in 96-cell row tiles where the rows fill them exactly, then in 128-cell row tiles, then in
// row segments (0.83 of the copy bandwidth at 256^3), then the two-warp shapes; for half storage row tiles first (whose 128-cell rows step 1.26x faster in row tiles),
// then row segments in three consumer groups; then the register kernels; the register kernel for double storage (whose step is bound by the
// double-precision pipe, which the register kernel's 4 warps per scheduler keep busier).
static int default_variant(const rlb_ctx* c) {
  static const int pref_f32[] = {19, 16, 15, 18, 17, 5, 12, 4, 13, 8, 6, 9, 7, 3};
  static const int pref_f16[] = {12, 16, 15, 13, 4, 8, 6, 5, 9, 7, 2};
  const int* pref = c->prm.storage == RLB_F32 ? pref_f32 : pref_f16;
  const int n = c->prm.storage == RLB_F32 ? (int)(sizeof(pref_f32) / sizeof(int)) : (int)(sizeof(pref_f16) / sizeof(int));
  if (c->prm.storage != RLB_F64)
    for (int k = 0; k < n; ++k) {
      // pipelined shapes only where the lattice's rows fill their tiles (rows_fit / rows_fit_solo
      // for row tiles, pipe_fits for row segments); a forced variant may still run on any lattice
      // it can take
      if (pref[k] >= kNumRegVariants) {
        PipeLayout lay;
        if (!pipe_layout(pref[k], c->q, (int)c->elem, c->smem_per_sm, c->smem_optin, &lay)) continue;
        const int elem = (int)c->elem;
        const bool one = elem == 4 && !lay.split;  // one warp per float cell
        bool fits = lay.rows ? (one ? rows_fit(c->sp.nx, lay.tx, elem, c->sp.bc[0], vmax_x(c))
                                    : rows_fit_solo(c->sp.nx, lay.tx, elem, c->sp.bc[0], vmax_x(c)))
                             : pipe_fits(c->sp.nx, lay.tx, elem, fill_eighths(lay, elem));
        // 96-cell row tiles only where the rows fill them exactly (96-, 48- and 32-cell rows)
        if (lay.tx == 96) fits = fits && (96 / c->sp.nx) * c->sp.nx == 96;
        if (!fits) continue;
      }
      if (variant_available(c, pref[k])) return pref[k];
    }
  return kDefaultStepVariant;
}

static rlb_status check_launch(rlb_ctx* c, cudaError_t e, const char* what);

// One time step of the whole lattice with step-kernel variant v: the register kernels (two
// launches: interior rows, then the shell) or the pipelined kernel (one launch).
static rlb_status launch_step(rlb_ctx* c, int v) {
  if (v >= kNumRegVariants) {
    PipeParams pp;
    int grid = 0, threads = 0, smem = 0, tx = 0, rows = 0, split = 0;
    if (!pipe_shape(c, v, &pp, &grid, &threads, &smem, &tx, &rows, &split))
      return fail(c, RLB_EINVAL, "step variant not available");
    return check_launch(c,
                        c->launch->pipe_step(c->buf[c->cur], c->buf[1 - c->cur], c->sp, pp, c->status, tx, rows,
                                             split, grid, threads, smem, c->stream),
                        "pipelined step kernel");
  }
  rlb_status st = check_launch(
      c, c->launch->step(c->buf[c->cur], c->buf[1 - c->cur], c->sp, c->status, c->general_wrap, v, c->stream),
      "step kernels");
  if (st == RLB_OK && c->sp.int_warps > 0 && c->sp.shell_cells > 0) ++c->launches;  // interior + shell
  return st;
}

extern "C" rlb_status rlb_create(const rlb_params* p, rlb_ctx** out) {
  if (!out) return fail(nullptr, RLB_EINVAL, "rlb_create: out is NULL");
  *out = nullptr;
  const std::string why = validate(p);
  if (!why.empty()) return fail(nullptr, RLB_EINVAL, "rlb_create: " + why);
  rlb_ctx* c = new (std::nothrow) rlb_ctx();
  if (!c) return fail(nullptr, RLB_ENOMEM, "rlb_create: out of host memory");
  c->prm = *p;
  c->prm.vel = nullptr;
  c->prm.level = nullptr;
  c->prm.p0 = nullptr;
  c->prm.w = nullptr;
  c->q = p->order == 3 ? Quad3::Q : Quad2::Q;
  c->cells = p->nx * p->ny * p->nz;
  c->elem = storage_bytes(p->storage);
  c->stream = (cudaStream_t)p->stream;

  StepParams& sp = c->sp;
  std::memset(&sp, 0, sizeof(sp));
  sp.nx = p->nx;
  sp.ny = p->ny;
  sp.nz = p->nz;
  sp.nxy = p->nx * p->ny;
  sp.cells = c->cells;
  for (int a = 0; a < 3; ++a) sp.bc[a] = p->bc[a];
  sp.has_wall = (p->bc[0] == RLB_BC_BOUNCEBACK || p->bc[1] == RLB_BC_BOUNCEBACK || p->bc[2] == RLB_BC_BOUNCEBACK);
  const double R = p->order == 3 ? Quad3::R : Quad2::R;
  sp.tau_fixed = p->tau_prime > 0.5 ? p->tau_prime : 0.0;
  const double kappa = p->T_unit_GeV * p->dx_fm / kHbarcGeVfm;
  sp.tau_coef = (p->tau_prime > 0.5) ? 0.0 : 6.0 * p->eta_over_s / (R * kappa);
  sp.tau_local = p->tau_local_T ? 1 : 0;
  sp.T_ref = p->T_ref;
  sp.tau_is_fixed = sp.tau_fixed > 0.5 ? 1 : 0;
  sp.tau_fixed_f = (float)sp.tau_fixed;
  sp.tau_coef_f = (float)sp.tau_coef;
  sp.T_ref_f = (float)sp.T_ref;
  sp.gamma_thr2 = (float)(p->gamma_thr * p->gamma_thr);
  sp.landau_fp64 = p->landau_fp64 ? 1 : 0;
  sp.half_nref = (float)(0.5 * p->n_ref);
  sp.debug = p->debug_flags;
  static const Launchers* const table[2][3] = {{&launchers_o2_s0, &launchers_o2_s1, &launchers_o2_s2},
                                               {&launchers_o3_s0, &launchers_o3_s1, &launchers_o3_s2}};
  c->launch = table[p->order == 3 ? 1 : 0][p->storage];
  int vmax[3];
  if (p->order == 3) {
    fill_offsets<Quad3>(sp);
    c->general_wrap = needs_general_wrap<Quad3>(*p);
    vmax[0] = Quad3::VMAX_X, vmax[1] = Quad3::VMAX_Y, vmax[2] = Quad3::VMAX_Z;
  } else {
    fill_offsets<Quad2>(sp);
    c->general_wrap = needs_general_wrap<Quad2>(*p);
    vmax[0] = Quad2::VMAX_X, vmax[1] = Quad2::VMAX_Y, vmax[2] = Quad2::VMAX_Z;
  }
  sp.general = c->general_wrap ? 1 : 0;
  // interior box: the stencil of every cell in it stays inside the lattice
  const int dims[3] = {p->nx, p->ny, p->nz};
  int i0[3], in[3];
  for (int a = 0; a < 3; ++a) {
    in[a] = dims[a] - 2 * vmax[a];
    if (in[a] <= 0) in[a] = 0;
    i0[a] = in[a] > 0 ? vmax[a] : 0;
  }
  if (in[0] == 0 || in[1] == 0 || in[2] == 0) in[0] = in[1] = in[2] = 0, i0[0] = i0[1] = i0[2] = 0;
  sp.ix0 = i0[0], sp.ixn = in[0], sp.iy0 = i0[1], sp.iyn = in[1], sp.iz0 = i0[2], sp.izn = in[2];
  // the row kernel takes every row with interior y and z, in 32-aligned x segments; the shell the rest
  sp.int_segs = in[0] > 0 ? (p->nx + 31) / 32 : 0;
  sp.int_warps = sp.int_segs * in[1] * in[2];
  sp.shell_cells = c->cells - (in[0] > 0 ? p->nx * in[1] * in[2] : 0);
  sp.row_segs = (p->nx + 31) / 32;
  sp.shell_rows = sp.shell_cells / p->nx;  // the shell is made of whole rows
  sp.shell_warps = sp.shell_rows * sp.row_segs;

  const size_t pop_bytes = (size_t)c->q * c->cells * c->elem;
  c->fblocks = (c->cells + kMomThreads - 1) / kMomThreads;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) {
    const int want = p->step_variant;
    c->variant = (want >= 0 && variant_available(c, want)) ? want : default_variant(c);
  }
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    e = cudaMalloc(&c->raw[b], pop_bytes + 2 * kPopGuardBytes);
    if (e == cudaSuccess) {
      c->buf[b] = static_cast<char*>(c->raw[b]) + kPopGuardBytes;
      e = cudaMemsetAsync(c->raw[b], 0, pop_bytes + 2 * kPopGuardBytes, c->stream);
    }
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->fields, 6 * (size_t)c->cells * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->partial, 5 * (size_t)c->fblocks * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->totals, 5 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->status, kStatusWords * sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, kStatusWords * sizeof(int), c->stream);
  if (e != cudaSuccess) {
    const rlb_status st = (e == cudaErrorMemoryAllocation) ? RLB_ENOMEM : RLB_ECUDA;
    cudaGetLastError();
    rlb_destroy(c);
    return fail(nullptr, st, std::string("rlb_create: ") + cudaGetErrorString(e));
  }
  *out = c;
  return RLB_OK;
}

extern "C" rlb_status rlb_destroy(rlb_ctx* c) {
  if (!c) return RLB_OK;
  if (c->stream || c->buf[0]) cudaStreamSynchronize(c->stream);
  if (c->copy_stream) {
    cudaStreamSynchronize(c->copy_stream);
    cudaStreamDestroy(c->copy_stream);
  }
  if (c->ev_ready) cudaEventDestroy(c->ev_ready);
  for (cudaEvent_t& e : c->ev_chunk)
    if (e) cudaEventDestroy(e);
  for (int b = 0; b < 2; ++b)
    if (c->raw[b]) cudaFree(c->raw[b]);
  if (c->fields) cudaFree(c->fields);
  if (c->partial) cudaFree(c->partial);
  if (c->totals) cudaFree(c->totals);
  if (c->status) cudaFree(c->status);
  delete c;
  return RLB_OK;
}

extern "C" const char* rlb_last_error(const rlb_ctx* c) { return c ? c->err.c_str() : g_create_err.c_str(); }
extern "C" long rlb_steps_done(const rlb_ctx* c) { return c ? c->steps : -1; }
extern "C" int rlb_step_variant(const rlb_ctx* c) { return c ? c->variant : -1; }
extern "C" long rlb_kernel_launches(const rlb_ctx* c) { return c ? c->launches : -1; }

static rlb_status check_launch(rlb_ctx* c, cudaError_t e, const char* what) {
  ++c->launches;
  if (e != cudaSuccess) return cuda_fail(c, e, what);
  return RLB_OK;
}

static rlb_status read_status(rlb_ctx* c) {
  int st[kStatusWords];
  RLB_CUDA(c, cudaMemcpyAsync(st, c->status, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
  RLB_CUDA(c, cudaStreamSynchronize(c->stream));
  if (st[kStatusBadInit] > 0) {
    RLB_CUDA(c, cudaMemsetAsync(c->status, 0, kStatusWords * sizeof(int), c->stream));
    return fail(c, RLB_EINVAL, std::to_string(st[kStatusBadInit]) + " cells with invalid initial fields");
  }
  if (st[kStatusNan] > 0) {
    RLB_CUDA(c, cudaMemsetAsync(c->status, 0, kStatusWords * sizeof(int), c->stream));
    return fail(c, RLB_ENAN, std::to_string(st[kStatusNan]) + " cells with non-finite populations");
  }
  if (st[kStatusBounds] > 0) {
    RLB_CUDA(c, cudaMemsetAsync(c->status, 0, kStatusWords * sizeof(int), c->stream));
    return fail(c, RLB_ECUDA, std::to_string(st[kStatusBounds]) + " pull addresses outside the population buffer");
  }
  if (st[kStatusTimeout] > 0) {
    RLB_CUDA(c, cudaMemsetAsync(c->status, 0, kStatusWords * sizeof(int), c->stream));
    return fail(c, RLB_ETIMEOUT, std::to_string(st[kStatusTimeout]) + " bounded device-side waits ran out");
  }
  if (st[kStatusNonconv] > 0) {
    RLB_CUDA(c, cudaMemsetAsync(c->status, 0, kStatusWords * sizeof(int), c->stream));
    return fail(c, RLB_ENONCONV, std::to_string(st[kStatusNonconv]) + " cell updates without a Landau frame");
  }
  return RLB_OK;
}

extern "C" rlb_status rlb_sync(rlb_ctx* c) {
  if (!c) return RLB_EINVAL;
  return read_status(c);
}

// Chunks of host transfers: ranges of whole kMomThreads-cell blocks, kChunks of them (fewer for
// small lattices), so that chunk j's copy overlaps chunk j - 1's kernel.
constexpr int kChunks = 8;

static int chunk_blocks(const rlb_ctx* c) {
  const int blocks = (c->cells + kMomThreads - 1) / kMomThreads;
  return (blocks + kChunks - 1) / kChunks;
}

static rlb_status ensure_copy_stream(rlb_ctx* c) {
  if (c->copy_stream) return RLB_OK;
  RLB_CUDA(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
  RLB_CUDA(c, cudaEventCreateWithFlags(&c->ev_ready, cudaEventDisableTiming));
  for (cudaEvent_t& e : c->ev_chunk) RLB_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  return RLB_OK;
}

// The device address of host array p[0 .. count) when the whole array is page-locked host memory
// the device can address (cudaHostAlloc, cudaHostRegister): its first and last elements are both
// mapped, at device addresses as far apart as the host addresses.  nullptr otherwise (pageable
// memory, or an array only partly registered), and then the data go through copies.
static double* mapped_host(const double* p, size_t count) {
  if (!p || count == 0) return nullptr;
  cudaPointerAttributes a{}, b{};
  const double* last = p + (count - 1);
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess || cudaPointerGetAttributes(&b, last) != cudaSuccess) {
    cudaGetLastError();  // an address CUDA does not know: not an error of this context
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer || !b.devicePointer)
    return nullptr;
  if ((const char*)b.devicePointer - (const char*)a.devicePointer != (const char*)last - (const char*)p)
    return nullptr;
  return static_cast<double*>(a.devicePointer);
}

extern "C" rlb_status rlb_init(rlb_ctx* c, const double* n, const double* T, const double* u, int on_device) {
  if (!c) return RLB_EINVAL;
  if (!n || !T || !u) return fail(c, RLB_EINVAL, "rlb_init: null field pointer");
  rlb_status st = RLB_OK;
  const size_t ncell = (size_t)c->cells;
  const double* hn = on_device ? nullptr : mapped_host(n, ncell);
  const double* hT = on_device ? nullptr : mapped_host(T, ncell);
  const double* hu = on_device ? nullptr : mapped_host(u, 3 * ncell);
  if (hn && hT && hu) {
    // page-locked host fields: the init kernel reads them where they are (over the CPU-GPU link),
    // one launch, no staging copies; the host arrays are free again once the call returns
    st = check_launch(c, c->launch->init(hn, hT, hu, c->buf[c->cur], c->sp, c->status, 0, c->cells, c->stream),
                      "init kernel");
    if (st != RLB_OK) return st;
    RLB_CUDA(c, cudaStreamSynchronize(c->stream));
  } else if (on_device) {
    st = check_launch(c, c->launch->init(n, T, u, c->buf[c->cur], c->sp, c->status, 0, c->cells, c->stream),
                      "init kernel");
    if (st != RLB_OK) return st;
  } else {
    // host fields: chunk j is copied into the staging buffer on the copy stream while the init
    // kernel of chunk j - 1 runs on the context's stream
    st = ensure_copy_stream(c);
    if (st != RLB_OK) return st;
    RLB_CUDA(c, cudaEventRecord(c->ev_ready, c->stream));  // earlier work on the staging buffer is done
    RLB_CUDA(c, cudaStreamWaitEvent(c->copy_stream, c->ev_ready, 0));
    const size_t cells = (size_t)c->cells;
    const int per = chunk_blocks(c) * kMomThreads;
    for (int j = 0; j < kChunks; ++j) {
      const int a = std::min(c->cells, j * per), b = std::min(c->cells, (j + 1) * per);
      if (a >= b) break;
      const size_t nb = (size_t)(b - a) * sizeof(double);
      const double* src[5] = {n + a, T + a, u + a, u + cells + a, u + 2 * cells + a};
      for (int k = 0; k < 5; ++k)
        RLB_CUDA(c, cudaMemcpyAsync(c->fields + k * cells + a, src[k], nb, cudaMemcpyHostToDevice, c->copy_stream));
      RLB_CUDA(c, cudaEventRecord(c->ev_chunk[j], c->copy_stream));
      RLB_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_chunk[j], 0));
      st = check_launch(c,
                        c->launch->init(c->fields, c->fields + cells, c->fields + 2 * cells, c->buf[c->cur], c->sp,
                                        c->status, a, b, c->stream),
                        "init kernel");
      if (st != RLB_OK) return st;
    }
    RLB_CUDA(c, cudaStreamSynchronize(c->stream));  // host buffers may be reused (every copy preceded a kernel)
  }
  c->steps = 0;
  c->have_prev = false;
  return RLB_OK;
}

extern "C" rlb_status rlb_step(rlb_ctx* c, long nsteps) {
  if (!c) return RLB_EINVAL;
  if (nsteps < 0) return fail(c, RLB_EINVAL, "nsteps < 0");
  for (long s = 0; s < nsteps; ++s) {
    rlb_status st = launch_step(c, c->variant);
    if (st != RLB_OK) return st;
    c->cur = 1 - c->cur;
    c->have_prev = true;
    ++c->steps;
  }
  return RLB_OK;
}

extern "C" rlb_status rlb_autotune(rlb_ctx* c, int reps, int* variant, double ms[RLB_MAX_VARIANTS]) {
  if (!c) return RLB_EINVAL;
  if (reps < 1) return fail(c, RLB_EINVAL, "rlb_autotune: reps < 1");
  if (c->have_prev) return fail(c, RLB_ESTATE, "rlb_autotune: only before the first step after init");
  cudaEvent_t e0, e1;
  RLB_CUDA(c, cudaEventCreate(&e0));
  RLB_CUDA(c, cudaEventCreate(&e1));
  double best = 1e300;
  int choice = c->variant;
  double t[RLB_MAX_VARIANTS] = {0};
  for (int v = 0; v < kNumVariantsTotal && v < RLB_MAX_VARIANTS; ++v) {
    if (!variant_available(c, v)) continue;
    // warm-up launch, then the timed repetitions; every launch recomputes the same next state
    for (int r = 0; r <= reps; ++r) {
      if (r == 1) RLB_CUDA(c, cudaEventRecord(e0, c->stream));
      rlb_status st = launch_step(c, v);
      if (st != RLB_OK) return st;
    }
    RLB_CUDA(c, cudaEventRecord(e1, c->stream));
    RLB_CUDA(c, cudaEventSynchronize(e1));
    float msv = 0.f;
    RLB_CUDA(c, cudaEventElapsedTime(&msv, e0, e1));
    t[v] = msv / reps;
    if (t[v] < best) {
      best = t[v];
      choice = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->variant = choice;
  if (variant) *variant = choice;
  if (ms)
    for (int v = 0; v < RLB_MAX_VARIANTS; ++v) ms[v] = t[v];
  return read_status(c);
}

extern "C" rlb_status rlb_moments(rlb_ctx* c, double* n, double* eps, double* U, double totals[5], int on_device) {
  if (!c) return RLB_EINVAL;
  const bool pull = c->have_prev;
  const void* src = pull ? c->buf[1 - c->cur] : c->buf[c->cur];
  const size_t cells = (size_t)c->cells;
  rlb_status st = RLB_OK;
  const FieldOut staged{{c->fields, c->fields + cells, c->fields + 2 * cells, c->fields + 3 * cells,
                        c->fields + 4 * cells, c->fields + 5 * cells}};
  double* hn = (on_device || !n) ? nullptr : mapped_host(n, cells);
  double* he = (on_device || !eps) ? nullptr : mapped_host(eps, cells);
  double* hU = (on_device || !U) ? nullptr : mapped_host(U, 4 * cells);
  if (hn && he && hU) {
    // page-locked host outputs: the fields kernel writes them where they are, one launch
    const FieldOut host{{hn, he, hU, hU + cells, hU + 2 * cells, hU + 3 * cells}};
    st = check_launch(c, c->launch->fields(src, c->sp, host, c->partial, c->status, pull, 0, c->fblocks, c->stream),
                      "fields kernel");
    if (st != RLB_OK) return st;
  } else if (on_device || (!n && !eps && !U)) {
    st = check_launch(c, c->launch->fields(src, c->sp, staged, c->partial, c->status, pull, 0, c->fblocks, c->stream),
                      "fields kernel");
    if (st != RLB_OK) return st;
    const size_t cb = cells * sizeof(double);
    if (n) RLB_CUDA(c, cudaMemcpyAsync(n, c->fields, cb, cudaMemcpyDeviceToDevice, c->stream));
    if (eps) RLB_CUDA(c, cudaMemcpyAsync(eps, c->fields + cells, cb, cudaMemcpyDeviceToDevice, c->stream));
    if (U) RLB_CUDA(c, cudaMemcpyAsync(U, c->fields + 2 * cells, 4 * cb, cudaMemcpyDeviceToDevice, c->stream));
  } else {
    // host outputs: the fields of chunk j are copied out on the copy stream while the fields kernel
    // of chunk j + 1 runs on the context's stream
    st = ensure_copy_stream(c);
    if (st != RLB_OK) return st;
    const int per_blocks = chunk_blocks(c);
    for (int j = 0; j < kChunks; ++j) {
      const int b0 = std::min(c->fblocks, j * per_blocks), b1 = std::min(c->fblocks, (j + 1) * per_blocks);
      if (b0 >= b1) break;
      st = check_launch(c, c->launch->fields(src, c->sp, staged, c->partial, c->status, pull, b0, b1, c->stream),
                        "fields kernel");
      if (st != RLB_OK) return st;
      RLB_CUDA(c, cudaEventRecord(c->ev_chunk[j], c->stream));
      RLB_CUDA(c, cudaStreamWaitEvent(c->copy_stream, c->ev_chunk[j], 0));
      const size_t a = (size_t)b0 * kMomThreads, b = std::min(cells, (size_t)b1 * kMomThreads);
      const size_t nb = (b - a) * sizeof(double);
      double* dst[6] = {n ? n + a : nullptr, eps ? eps + a : nullptr, U ? U + a : nullptr, U ? U + cells + a : nullptr,
                        U ? U + 2 * cells + a : nullptr, U ? U + 3 * cells + a : nullptr};
      for (int k = 0; k < 6; ++k)
        if (dst[k]) RLB_CUDA(c, cudaMemcpyAsync(dst[k], c->fields + k * cells + a, nb, cudaMemcpyDeviceToHost,
                                                c->copy_stream));
    }
  }
  st = check_launch(c, launch_reduce_partials(c->partial, c->fblocks, c->totals, c->stream), "reduce kernel");
  if (st != RLB_OK) return st;
  if (totals) RLB_CUDA(c, cudaMemcpyAsync(totals, c->totals, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (c->copy_stream) RLB_CUDA(c, cudaStreamSynchronize(c->copy_stream));
  return read_status(c);
}

// Populations cross the boundary as double[q][cells].  Host transfers are staged one population
// plane at a time through the field buffer (6 * cells doubles), device transfers convert in place.
static rlb_status convert(rlb_ctx* c, double* dbl, int on_device, bool to_f64) {
  void* pop = c->buf[c->cur];
  const size_t cb = (size_t)c->cells * sizeof(double);
  auto launch = [&](double* d, int i0, int i1) {
    return check_launch(c, c->launch->convert(pop, d, i0, i1, to_f64, c->sp, c->stream), "convert kernel");
  };
  if (on_device) return launch(dbl, 0, c->q);
  for (int i = 0; i < c->q; ++i) {
    double* h = dbl + (size_t)i * c->cells;
    if (!to_f64) RLB_CUDA(c, cudaMemcpyAsync(c->fields, h, cb, cudaMemcpyHostToDevice, c->stream));
    rlb_status st = launch(c->fields, i, i + 1);
    if (st != RLB_OK) return st;
    if (to_f64) RLB_CUDA(c, cudaMemcpyAsync(h, c->fields, cb, cudaMemcpyDeviceToHost, c->stream));
    RLB_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  return RLB_OK;
}

extern "C" rlb_status rlb_get_populations(rlb_ctx* c, double* f, int on_device) {
  if (!c) return RLB_EINVAL;
  if (!f) return fail(c, RLB_EINVAL, "rlb_get_populations: null pointer");
  rlb_status st = convert(c, f, on_device, true);
  if (st != RLB_OK) return st;
  return read_status(c);
}

extern "C" rlb_status rlb_set_populations(rlb_ctx* c, const double* f, int on_device) {
  if (!c) return RLB_EINVAL;
  if (!f) return fail(c, RLB_EINVAL, "rlb_set_populations: null pointer");
  rlb_status st = convert(c, const_cast<double*>(f), on_device, false);
  if (st != RLB_OK) return st;
  c->steps = 0;
  c->have_prev = false;
  return RLB_OK;
}
