// Batched stepping of independent contexts (C ABI, include/rlb.h): a persistent kernel over a shared
// tile queue advances every member by one time step per launch; runs of several steps can be
// captured once as a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "rlb.h"
#include "rlb_common.h"
#include "rlb_ctx.h"
#include "rlb_launch.h"
#include "rlb_quadrature.h"

using namespace rlb;

namespace {

struct Member {
  rlb_ctx* ctx;
  long steps_left;
};

struct GraphCache {
  cudaGraphExec_t exec = nullptr;
  long nsteps = 0, version = -1;
  int variant = -1, nmembers = 0, tiles = 0, row_tiles = -1, walls = -1, pipe_tiles = -1, pipe_walls = -1,
      rtile_tiles = -1, r96_tiles = -1;
};

}  // namespace

struct rlb_batch {
  int order = 3, storage = RLB_F32;
  cudaStream_t stream = nullptr;
  std::vector<Member> members;   // slot -> member (ctx == nullptr: free slot)
  BatchMember* d_members = nullptr;
  int d_capacity = 0;
  int* d_tile_member = nullptr;  // member index of every tile of the uploaded table
  int tm_capacity = 0;
  int* d_counters = nullptr;     // two tile counters (row queue, shell queue) per step of a run
  long counters_capacity = 0;
  const Launchers* launch = nullptr;
  int variant = 0;               // step variant: 0..3 register kernels for every member; 4 and up the
                                 // pipelined kernel for the members whose rows suit it (row tiles for
                                 // rows_fit members if the variant has row tiles, row segments for
                                 // pipe_fits members) and the register fallback (reg_fallback) for the others
  int walls = 0;                 // some register-kernel member of the uploaded table has bounce-back walls
  int row_tiles = 0, shell_tiles = 0;  // of the uploaded table: row tiles first, then shell tiles
  int* d_pipe_tm = nullptr;      // member index of every pipelined tile of the uploaded table
  int pipe_tm_capacity = 0;
  int pipe_tiles = 0, pipe_walls = 0;
  int* d_rtile_tm = nullptr;     // member index of every row tile (pipelined kernel with row tiles)
  int rtile_tm_capacity = 0;
  int rtile_tiles = 0;
  PipeLayout lay96{};            // 96-cell row tiles beside a 128-cell row-tile variant (tx 0: none)
  int v96 = -1;                  // their variant
  int* d_r96_tm = nullptr;       // member index of every 96-cell row tile
  int r96_tm_capacity = 0;
  int r96_tiles = 0;
  int* pipe_timeout = nullptr;   // status word that counts the pipelined kernel's expired waits
  PipeLayout lay{};              // block layout of the current pipelined variant
  int sms = 0, smem_per_sm = 0, smem_optin = 0;
  long version = 0;              // bumps when the member set changes
  long launches = 0;
  GraphCache graph;
  std::string err;
};

static rlb_status bfail(rlb_batch* b, rlb_status st, const std::string& msg) {
  if (b) b->err = msg;
  return st;
}

#define BATCH_CUDA(b, call)                                                                          \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) return bfail((b), RLB_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

extern "C" rlb_status rlb_batch_create(int order, int storage, void* stream, rlb_batch** out) {
  if (!out) return RLB_EINVAL;
  *out = nullptr;
  if ((order != 2 && order != 3) || storage < RLB_F64 || storage > RLB_F16DEV) return RLB_EINVAL;
  rlb_batch* b = new (std::nothrow) rlb_batch();
  if (!b) return RLB_ENOMEM;
  b->order = order;
  b->storage = storage;
  b->stream = static_cast<cudaStream_t>(stream);
  static const Launchers* const table[2][3] = {{&launchers_o2_s0, &launchers_o2_s1, &launchers_o2_s2},
                                               {&launchers_o3_s0, &launchers_o3_s1, &launchers_o3_s2}};
  b->launch = table[order == 3 ? 1 : 0][storage];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return RLB_ECUDA;
  }
  if (cudaDeviceGetAttribute(&b->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return RLB_ECUDA;
  }
  b->variant = storage == RLB_F64 ? 0 : kDefaultStepVariant;
  *out = b;
  return RLB_OK;
}

static int elem_of(int storage) { return storage == RLB_F64 ? 8 : (storage == RLB_F32 ? 4 : 2); }

// The register-kernel variant for members the pipelined kernel cannot take (rows not on 16-byte
// boundaries): the one a context of that storage runs when no pipelined variant exists for it.
static int reg_fallback(const rlb_batch* b) { return b->storage == RLB_F32 ? 3 : (b->storage == RLB_F16DEV ? 2 : 0); }

static bool variant_exists(const rlb_batch* b, int v, PipeLayout* lay = nullptr) {
  if (v < 0) return false;
  if (v < kNumRegVariants) return v < b->launch->step_variants;
  const int q = b->order == 3 ? 128 : 66;
  return pipe_layout(v, q, elem_of(b->storage), b->smem_per_sm, b->smem_optin, lay);
}

// Lanes of a row tile of tx cells that hold cells (0 if the rows do not fit).
static int row_tile_fill(int nx, int tx) { return nx <= tx ? (tx / nx) * nx : 0; }

// How a member runs under step variant v: 3 the 96-cell row tiles beside a 128-cell row-tile
// variant, 2 the variant's row tiles, 1 row segments (pipelined kernel), 0 the register kernels
// (variant v itself, or reg_fallback for a pipelined v).  A member takes the row tiles whose lanes
// it fills the larger share of (96-cell rows: all of a 96-cell tile against 3/4 of a 128-cell one).
// Rows that fill segment tiles go to row tiles too, except with two warps per float cell (measured
// on GB300 at 128^3: one warp per float cell 1.13x faster in row tiles, half storage 1.26x; two
// warps per float cell 1.04x faster in segments).  96-cell tiles exist as row tiles only.
static int member_mode(const rlb_batch* b, const StepParams& p, int v, const PipeLayout& lay, const PipeLayout& lay96) {
  if (v < kNumRegVariants) return 0;
  const int vmax = b->order == 3 ? Quad3::VMAX_X : Quad2::VMAX_X;
  const int elem = elem_of(b->storage);
  const bool seg = lay.tx != 96 && pipe_fits(p.nx, lay.tx, elem, fill_eighths(lay, elem));
  const bool rows = lay.rows && rows_fit(p.nx, lay.tx, elem, p.bc[0], vmax);
  if (lay96.tx == 96 && rows_fit(p.nx, 96, elem, p.bc[0], vmax) &&
      (!rows || row_tile_fill(p.nx, 96) * lay.tx > row_tile_fill(p.nx, lay.tx) * 96))
    return 3;
  if (rows && (!seg || !lay.split)) return 2;
  return seg ? 1 : 0;
}

// The 96-cell row-tile variant with the warps of 128-cell row-tile variant v (-1 if none).
static int rows96_sibling(int v) {
  if (v < kNumRegVariants || v >= kNumVariantsTotal) return -1;
  const PipeConfig& c = kPipeConfigs[v - kNumRegVariants];
  if (!c.rows || c.tx != 128) return -1;
  for (int k = 0; k < kNumPipeConfigs; ++k) {
    const PipeConfig& d = kPipeConfigs[k];
    if (d.rows && d.tx == 96 && d.cons_warps == c.cons_warps && d.producers == c.producers &&
        d.ctas_per_sm == c.ctas_per_sm && d.split == c.split)
      return kNumRegVariants + k;
  }
  return -1;
}

// The row-segment variant with the block layout of row-tile variant v (the shape the batch runs its
// row-segment members in); v itself if it has no row tiles, -1 if none exists.
static int segment_sibling(int v) {
  if (v < kNumRegVariants || v >= kNumVariantsTotal) return v;
  const PipeConfig& c = kPipeConfigs[v - kNumRegVariants];
  if (!c.rows) return v;
  for (int k = 0; k < kNumPipeConfigs; ++k) {
    const PipeConfig& d = kPipeConfigs[k];
    if (!d.rows && d.tx == c.tx && d.cons_warps == c.cons_warps && d.ctas_per_sm == c.ctas_per_sm &&
        d.producers == c.producers && d.split == c.split)
      return kNumRegVariants + k;
  }
  return -1;
}

// The 96-cell companion of variant v for this batch's storage: its variant (-1 if none) and
// layout in *lay96 (tx 0 if none).
static int companion96(const rlb_batch* b, int v, PipeLayout* lay96) {
  *lay96 = PipeLayout{};
  const int v96 = rows96_sibling(v);
  if (v96 < 0 || !variant_exists(b, v96, lay96)) {
    *lay96 = PipeLayout{};
    return -1;
  }
  return v96;
}

// Grow a device tile table to hold n entries and upload `tm` into it.
static rlb_status upload_tiles(rlb_batch* b, int** d, int* capacity, const std::vector<int>& tm, const char* what) {
  if ((int)tm.size() > *capacity) {
    if (*d) cudaFree(*d);
    *d = nullptr;
    const int cap = std::max<int>((int)tm.size(), 2 * *capacity);
    cudaError_t e = cudaMalloc((void**)d, (size_t)cap * sizeof(int));
    if (e != cudaSuccess) {
      *capacity = 0;
      return bfail(b, RLB_ENOMEM, std::string(what) + ": " + cudaGetErrorString(e));
    }
    *capacity = cap;
    ++b->version;  // a captured graph holds the old table pointer
  }
  if (!tm.empty())
    BATCH_CUDA(b, cudaMemcpyAsync(*d, tm.data(), tm.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
  return RLB_OK;
}

extern "C" rlb_status rlb_batch_add(rlb_batch* b, rlb_ctx* ctx, long steps, int* slot) {
  if (!b) return RLB_EINVAL;
  if (!ctx || steps < 0) return bfail(b, RLB_EINVAL, "rlb_batch_add: null context or negative steps");
  if (ctx->prm.order != b->order || ctx->prm.storage != b->storage)
    return bfail(b, RLB_EINVAL, "rlb_batch_add: the context's order or storage differs from the batch's");
  for (const Member& m : b->members)
    if (m.ctx == ctx) return bfail(b, RLB_EINVAL, "rlb_batch_add: context already in the batch");
  int s = -1;
  for (size_t i = 0; i < b->members.size(); ++i)
    if (!b->members[i].ctx) {
      s = (int)i;
      break;
    }
  if (s < 0) {
    s = (int)b->members.size();
    b->members.push_back(Member{nullptr, 0});
  }
  b->members[s] = Member{ctx, steps};
  ++b->version;
  if (slot) *slot = s;
  return RLB_OK;
}

extern "C" rlb_status rlb_batch_remove(rlb_batch* b, int slot) {
  if (!b) return RLB_EINVAL;
  if (slot < 0 || slot >= (int)b->members.size() || !b->members[slot].ctx)
    return bfail(b, RLB_EINVAL, "rlb_batch_remove: no member in this slot");
  b->members[slot] = Member{nullptr, 0};
  ++b->version;
  return RLB_OK;
}

extern "C" long rlb_batch_steps_left(const rlb_batch* b, int slot) {
  if (!b || slot < 0 || slot >= (int)b->members.size() || !b->members[slot].ctx) return -1;
  return b->members[slot].steps_left;
}

// Member table of a run with step variant `variant`: the active members in slot order with their
// tile ranges (pipelined tiles for the members the pipelined kernel takes, register-kernel row and
// shell tiles for the others).
static rlb_status upload_table(rlb_batch* b, long nsteps, int variant, int* nmembers, int* total_tiles) {
  std::vector<BatchMember> t;
  std::vector<int> row_tm, shell_tm, pipe_tm, rtile_tm;
  b->walls = 0;
  b->pipe_walls = 0;
  b->pipe_timeout = nullptr;
  const bool pipe = variant >= kNumRegVariants && variant_exists(b, variant, &b->lay);
  if (!pipe) b->lay = PipeLayout{};
  b->v96 = pipe ? companion96(b, variant, &b->lay96) : -1;
  if (!pipe) b->lay96 = PipeLayout{};
  std::vector<int> r96_tm;
  for (const Member& m : b->members) {
    if (!m.ctx || m.steps_left <= 0) continue;
    BatchMember d{};
    d.p = m.ctx->sp;
    d.buf[0] = m.ctx->buf[0];
    d.buf[1] = m.ctx->buf[1];
    d.status = m.ctx->status;
    d.parity0 = m.ctx->cur;
    d.steps_left = (int)std::min<long>(m.steps_left, nsteps);
    const int mode = member_mode(b, d.p, pipe ? variant : 0, b->lay, b->lay96);
    if (mode > 0) {
      // pipelined: ceil(nx / TX) segment tiles per row, or groups of TX / nx rows
      std::vector<int>& tm = mode == 3 ? r96_tm : (mode == 2 ? rtile_tm : pipe_tm);
      d.pipe_tile_begin = (int)tm.size();
      const long long nt = pipe_tile_count(d.p.nx, d.p.ny, d.p.nz, mode == 3 ? 96 : b->lay.tx, mode >= 2);
      if ((long long)tm.size() + nt > 0x7fffffffll) return bfail(b, RLB_EINVAL, "too many tiles in one batch");
      tm.resize(tm.size() + nt, (int)t.size());
      if (d.p.has_wall) b->pipe_walls = 1;
      if (!b->pipe_timeout) b->pipe_timeout = d.status + kStatusTimeout;
      t.push_back(d);
      continue;
    }
    if (d.p.has_wall) b->walls = 1;
    // row tiles: 4 row-kernel warps; shell tiles: 4 shell-row warps (kStepThreads shell cells for
    // members that need the modulo wrap)
    d.row_tile_begin = (int)row_tm.size();
    row_tm.resize(row_tm.size() + (d.p.int_warps + kStepThreads / 32 - 1) / (kStepThreads / 32), (int)t.size());
    d.shell_tile_begin = (int)shell_tm.size();  // shifted by the row tiles below
    const int shell_tiles = d.p.general ? (d.p.shell_cells + kStepThreads - 1) / kStepThreads
                                        : (d.p.shell_warps + kStepThreads / 32 - 1) / (kStepThreads / 32);
    shell_tm.resize(shell_tm.size() + shell_tiles, (int)t.size());
    t.push_back(d);
  }
  b->row_tiles = (int)row_tm.size();
  b->shell_tiles = (int)shell_tm.size();
  b->pipe_tiles = (int)pipe_tm.size();
  b->rtile_tiles = (int)rtile_tm.size();
  b->r96_tiles = (int)r96_tm.size();
  for (BatchMember& d : t) d.shell_tile_begin += b->row_tiles;
  std::vector<int> tm(row_tm);
  tm.insert(tm.end(), shell_tm.begin(), shell_tm.end());
  const int tiles = (int)tm.size();
  *nmembers = (int)t.size();
  *total_tiles = tiles + b->pipe_tiles + b->rtile_tiles + b->r96_tiles;
  if (t.empty()) return RLB_OK;
  rlb_status st = upload_tiles(b, &b->d_pipe_tm, &b->pipe_tm_capacity, pipe_tm, "pipelined tile table");
  if (st != RLB_OK) return st;
  st = upload_tiles(b, &b->d_rtile_tm, &b->rtile_tm_capacity, rtile_tm, "row-tile table");
  if (st != RLB_OK) return st;
  st = upload_tiles(b, &b->d_r96_tm, &b->r96_tm_capacity, r96_tm, "96-cell row-tile table");
  if (st != RLB_OK) return st;
  if ((int)t.size() > b->d_capacity) {
    if (b->d_members) cudaFree(b->d_members);
    b->d_members = nullptr;
    const int cap = std::max<int>((int)t.size(), 2 * b->d_capacity);
    cudaError_t e = cudaMalloc((void**)&b->d_members, (size_t)cap * sizeof(BatchMember));
    if (e != cudaSuccess) {
      b->d_capacity = 0;
      return bfail(b, RLB_ENOMEM, std::string("member table: ") + cudaGetErrorString(e));
    }
    b->d_capacity = cap;
    ++b->version;  // a captured graph holds the old table pointer
  }
  if (tiles > 0 && tiles > b->tm_capacity) {
    if (b->d_tile_member) cudaFree(b->d_tile_member);
    b->d_tile_member = nullptr;
    const int cap = std::max<int>(tiles, 2 * b->tm_capacity);
    cudaError_t e = cudaMalloc((void**)&b->d_tile_member, (size_t)cap * sizeof(int));
    if (e != cudaSuccess) {
      b->tm_capacity = 0;
      return bfail(b, RLB_ENOMEM, std::string("tile table: ") + cudaGetErrorString(e));
    }
    b->tm_capacity = cap;
    ++b->version;  // a captured graph holds the old table pointer
  }
  BATCH_CUDA(b, cudaMemcpyAsync(b->d_members, t.data(), t.size() * sizeof(BatchMember), cudaMemcpyHostToDevice,
                                b->stream));
  if (tiles > 0)
    BATCH_CUDA(b, cudaMemcpyAsync(b->d_tile_member, tm.data(), tm.size() * sizeof(int), cudaMemcpyHostToDevice,
                                  b->stream));
  BATCH_CUDA(b, cudaStreamSynchronize(b->stream));  // the host vector goes away
  return RLB_OK;
}

static rlb_status ensure_counters(rlb_batch* b, long nsteps) {
  if (nsteps <= b->counters_capacity) return RLB_OK;
  if (b->d_counters) cudaFree(b->d_counters);
  b->d_counters = nullptr;
  cudaError_t e = cudaMalloc((void**)&b->d_counters, (size_t)nsteps * sizeof(int));
  if (e != cudaSuccess) {
    b->counters_capacity = 0;
    return bfail(b, RLB_ENOMEM, std::string("tile counters: ") + cudaGetErrorString(e));
  }
  b->counters_capacity = nsteps;
  ++b->version;
  return RLB_OK;
}

static int grid_of(rlb_batch* b, int variant) { return b->sms * b->launch->batch_blocks_per_sm(variant); }

// One time step (launch index k) of the uploaded table: the pipelined kernel over its tiles, then
// the register kernels (row tiles, shell tiles) over the other members' tiles.
static rlb_status enqueue_step(rlb_batch* b, int k, int variant, int* counters) {
  cudaError_t e = cudaSuccess;
  // row segments, 128-cell row tiles, 96-cell row tiles
  for (int kind = 0; kind < 3; ++kind) {
    const int ntiles = kind == 0 ? b->pipe_tiles : (kind == 1 ? b->rtile_tiles : b->r96_tiles);
    if (ntiles == 0) continue;
    const PipeLayout& lay = kind == 2 ? b->lay96 : b->lay;
    const int* tm = kind == 0 ? b->d_pipe_tm : (kind == 1 ? b->d_rtile_tm : b->d_r96_tm);
    const PipeParams pp{lay.producers, ntiles, lay.nstage, lay.groups};
    const int grid = std::min(b->sms * lay.ctas_per_sm, ntiles);
    e = b->launch->pipe_batch_step(b->d_members, tm, k, pp, b->pipe_timeout, lay.tx, kind > 0, lay.split,
                                   b->pipe_walls, grid, lay.threads, lay.smem, b->stream);
    ++b->launches;
    if (e != cudaSuccess) return bfail(b, RLB_ECUDA, std::string("batched pipelined step: ") + cudaGetErrorString(e));
  }
  if (b->row_tiles + b->shell_tiles > 0) {
    const int rv = variant < kNumRegVariants ? variant : reg_fallback(b);
    e = b->launch->batch_step(b->d_members, b->d_tile_member, b->row_tiles, b->shell_tiles, k, counters, rv, b->walls,
                              grid_of(b, rv), b->stream);
    b->launches += (b->row_tiles > 0) + (b->shell_tiles > 0);
    if (e != cudaSuccess) return bfail(b, RLB_ECUDA, std::string("batched step: ") + cudaGetErrorString(e));
  }
  return RLB_OK;
}

// Enqueue nsteps launches (launch index 0..nsteps-1) directly on the stream.
static rlb_status enqueue_run(rlb_batch* b, long nsteps, int nmem, int tiles, int variant) {
  (void)nmem;
  (void)tiles;
  BATCH_CUDA(b, cudaMemsetAsync(b->d_counters, 0, (size_t)(2 * nsteps) * sizeof(int), b->stream));
  for (long k = 0; k < nsteps; ++k) {
    const rlb_status st = enqueue_step(b, (int)k, variant, b->d_counters);
    if (st != RLB_OK) return st;
  }
  return RLB_OK;
}

extern "C" rlb_status rlb_batch_run(rlb_batch* b, long nsteps, int use_graph, int* active) {
  if (!b) return RLB_EINVAL;
  if (nsteps < 0 || nsteps > (1L << 30)) return bfail(b, RLB_EINVAL, "rlb_batch_run: nsteps out of range");
  for (const Member& m : b->members)
    if (m.ctx && m.ctx->stream != b->stream)
      return bfail(b, RLB_EINVAL, "rlb_batch_run: a member uses another stream than the batch");
  int nmem = 0, tiles = 0;
  if (nsteps > 0) {
    rlb_status st = ensure_counters(b, 2 * nsteps);
    if (st != RLB_OK) return st;
    st = upload_table(b, nsteps, b->variant, &nmem, &tiles);
    if (st != RLB_OK) return st;
  }
  if (nmem > 0) {
    if (use_graph) {
      // the table lives at a fixed device address and is refreshed before every replay, so the
      // captured launches stay valid while nsteps, the variant, the member set and the active
      // members' row and shell tile counts stay the same
      GraphCache& gc = b->graph;
      if (!gc.exec || gc.nsteps != nsteps || gc.version != b->version || gc.variant != b->variant ||
          gc.nmembers != nmem || gc.tiles != tiles || gc.row_tiles != b->row_tiles || gc.walls != b->walls ||
          gc.pipe_tiles != b->pipe_tiles || gc.pipe_walls != b->pipe_walls || gc.rtile_tiles != b->rtile_tiles ||
          gc.r96_tiles != b->r96_tiles) {
        if (b->graph.exec) cudaGraphExecDestroy(b->graph.exec);
        b->graph.exec = nullptr;
        cudaStream_t cs;
        BATCH_CUDA(b, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        BATCH_CUDA(b, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        cudaStream_t saved = b->stream;
        b->stream = cs;
        const long l0 = b->launches;
        rlb_status st = enqueue_run(b, nsteps, nmem, tiles, b->variant);
        b->stream = saved;
        b->launches = l0;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(cs, &g);
        cudaStreamDestroy(cs);
        if (st != RLB_OK) {
          if (g) cudaGraphDestroy(g);
          return st;
        }
        if (e != cudaSuccess) return bfail(b, RLB_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&b->graph.exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return bfail(b, RLB_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        gc.nsteps = nsteps;
        gc.version = b->version;
        gc.variant = b->variant;
        gc.nmembers = nmem;
        gc.tiles = tiles;
        gc.row_tiles = b->row_tiles;
        gc.walls = b->walls;
        gc.pipe_tiles = b->pipe_tiles;
        gc.pipe_walls = b->pipe_walls;
        gc.rtile_tiles = b->rtile_tiles;
        gc.r96_tiles = b->r96_tiles;
      }
      BATCH_CUDA(b, cudaGraphLaunch(b->graph.exec, b->stream));
      b->launches += nsteps * ((b->row_tiles > 0) + (b->shell_tiles > 0) + (b->pipe_tiles > 0) + (b->rtile_tiles > 0) +
                               (b->r96_tiles > 0));
    } else {
      rlb_status st = enqueue_run(b, nsteps, nmem, tiles, b->variant);
      if (st != RLB_OK) return st;
    }
  }
  // every member advanced min(steps_left, nsteps) steps
  int act = 0;
  for (Member& m : b->members) {
    if (!m.ctx) continue;
    const long k = std::min(m.steps_left, nsteps);
    if (k > 0) {
      m.ctx->cur = (int)((m.ctx->cur + k) & 1);
      m.ctx->have_prev = true;
      m.ctx->steps += k;  // the launches are counted once, by the batch
      m.steps_left -= k;
    }
    if (m.steps_left > 0) ++act;
  }
  if (active) *active = act;
  return RLB_OK;
}

extern "C" rlb_status rlb_batch_autotune(rlb_batch* b, int reps, int* variant, double ms[RLB_MAX_VARIANTS]) {
  if (!b) return RLB_EINVAL;
  if (reps < 1) return bfail(b, RLB_EINVAL, "rlb_batch_autotune: reps < 1");
  for (const Member& m : b->members)
    if (m.ctx && m.ctx->have_prev)
      return bfail(b, RLB_ESTATE, "rlb_batch_autotune: only while no member has taken a step");
  rlb_status st = ensure_counters(b, 2 * (reps + 1));
  if (st != RLB_OK) return st;
  double t[RLB_MAX_VARIANTS] = {0};
  cudaEvent_t e0, e1;
  BATCH_CUDA(b, cudaEventCreate(&e0));
  BATCH_CUDA(b, cudaEventCreate(&e1));
  double best = 1e300;
  int choice = b->variant;
  for (int v = 0; v < kNumVariantsTotal && v < RLB_MAX_VARIANTS; ++v) {
    if (!variant_exists(b, v)) continue;
    int nmem = 0, tiles = 0;
    st = upload_table(b, 1, v, &nmem, &tiles);  // steps_left = 1: every launch redoes launch 0
    if (st != RLB_OK) return st;
    if (nmem == 0) break;
    BATCH_CUDA(b, cudaMemsetAsync(b->d_counters, 0, (size_t)(2 * (reps + 1)) * sizeof(int), b->stream));
    for (int r = 0; r <= reps; ++r) {
      if (r == 1) BATCH_CUDA(b, cudaEventRecord(e0, b->stream));
      // every repetition is launch 0 of the same run: the same next state into the spare buffers
      st = enqueue_step(b, 0, v, b->d_counters + 2 * r);
      if (st != RLB_OK) return st;
    }
    BATCH_CUDA(b, cudaEventRecord(e1, b->stream));
    BATCH_CUDA(b, cudaEventSynchronize(e1));
    float msv = 0.f;
    BATCH_CUDA(b, cudaEventElapsedTime(&msv, e0, e1));
    t[v] = msv / reps;
    if (t[v] < best) {
      best = t[v];
      choice = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->variant = choice;
  if (variant) *variant = b->variant;
  if (ms)
    for (int v = 0; v < RLB_MAX_VARIANTS; ++v) ms[v] = t[v];
  return RLB_OK;
}

extern "C" rlb_status rlb_batch_set_variant(rlb_batch* b, int variant) {
  if (!b) return RLB_EINVAL;
  if (!variant_exists(b, variant)) return bfail(b, RLB_EINVAL, "rlb_batch_set_variant: no such variant");
  b->variant = variant;
  return RLB_OK;
}

extern "C" int rlb_batch_member_variant(const rlb_batch* b, int slot) {
  if (!b || slot < 0 || slot >= (int)b->members.size() || !b->members[slot].ctx) return -1;
  if (b->variant < kNumRegVariants) return b->variant;
  PipeLayout lay;
  if (!variant_exists(b, b->variant, &lay)) return reg_fallback(b);
  PipeLayout lay96;
  const int v96 = companion96(b, b->variant, &lay96);
  const int mode = member_mode(b, b->members[slot].ctx->sp, b->variant, lay, lay96);
  if (mode == 3) return v96;
  if (mode == 2) return b->variant;
  if (mode == 1) return segment_sibling(b->variant);
  return reg_fallback(b);
}

extern "C" long rlb_batch_kernel_launches(const rlb_batch* b) { return b ? b->launches : -1; }

extern "C" const char* rlb_batch_last_error(const rlb_batch* b) { return b ? b->err.c_str() : "null batch"; }

extern "C" rlb_status rlb_batch_destroy(rlb_batch* b) {
  if (!b) return RLB_OK;
  cudaStreamSynchronize(b->stream);
  if (b->graph.exec) cudaGraphExecDestroy(b->graph.exec);
  if (b->d_members) cudaFree(b->d_members);
  if (b->d_tile_member) cudaFree(b->d_tile_member);
  if (b->d_pipe_tm) cudaFree(b->d_pipe_tm);
  if (b->d_rtile_tm) cudaFree(b->d_rtile_tm);
  if (b->d_r96_tm) cudaFree(b->d_r96_tm);
  if (b->d_counters) cudaFree(b->d_counters);
  delete b;
  return RLB_OK;
}
