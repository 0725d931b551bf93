// Pipelined step kernel: the pull of Eq. (rlb:disc) staged through shared memory by the bulk-copy
// (TMA) engine, with warp-specialised producer and consumer warps (sm_90+ PTX: mbarrier,
// cp.async.bulk).
//
// A tile is one 64- or 128-cell segment of a lattice row (fixed y, z; x0 a multiple of the tile
// width TX).  For every population i the cells x0 .. x0 + TX - 1 pull from the row
// (y - vy_i, z - vz_i) at x - vx_i, i.e. from one contiguous run of the source plane.  The
// producer warp copies that run, widened to 16-byte boundaries, into the tile's stage with one
// bulk copy per population (cp.async.bulk, completion counted on the stage's mbarrier).  y and z
// are resolved per row by the producer (periodic wrap or copy-out clamp); a periodic x is resolved
// by splitting the run at the lattice ends into copies of whole 16-byte units.  Everything the
// copies cannot express (a copy-out or bounce-back x, the reversed population beyond a y or z
// wall) is patched in shared memory by the consumer warp before it reads the stage.
//
// Consumer warps own one 32-cell part of a tile each (with float storage optionally two warps per
// part, each taking half the populations) and read population i of lane x at the compile-time
// offset i * BX + r_i + x of the stage (r_i = -vx_i mod the copy granule), twice: once for the
// moments and once for the collision, whose result goes straight to global memory with one
// coalesced store per population.  The populations never sit in registers as a whole, so a
// consumer needs at most 128 registers instead of Q + ~40, and the loads that feed a tile are
// issued by one producer lane per population instead of 32 lanes each computing an address.
//
// Row tiles (ROWS): on an x-periodic lattice with rows of nx <= TX cells a tile is G = TX / nx
// consecutive rows (lane q of the tile is cell x = q mod nx of row q / nx).  Population i of those
// rows pulls from G source rows, consecutive in memory except where y or z wraps, so the producer
// copies each run of them whole with one bulk copy, and the consumer lane reads its pulled value at
// (x - vx_i) mod nx of its row's stage: the periodic x costs neither split copies nor slack, and
// every lane holds one stage offset per x velocity, computed once per tile.
//
// Stages form a ring of NSTAGE slots per block: tile k of a block goes to stage k % NSTAGE and to
// consumer group k % groups; every producer warp copies its share of the populations of every
// tile.  NSTAGE is a multiple of the group count, so each stage is read by one group, and every
// producer and that group take the stage's uses in order: when either waits for use u of a stage,
// use u - 1 is complete and use u + 1 cannot be, and the parity of u names the right phase.
// full[s] completes when every producer has arrived for the stage's tile and its copies have
// landed; empty[s] when every consumer warp of that tile has finished reading it.  Every wait is
// bounded (kPipeWaitNs); a wait that runs out counts in status[kStatusTimeout], and the producer
// then waits (bounded) for the copies it has in flight before it returns.
#pragma once

#include <stdint.h>

#include "rlb_kernels.cuh"

namespace rlb {

constexpr int kPipeMaxThreads = kPipeMaxWarps * 32;
constexpr unsigned long long kPipeWaitNs = 2000000000ull;  // 2 s

// Geometry of one staged row for storage S and tile width TX.
template <class S, int TX>
struct PipeShape {
  using T = typename S::T;
  static constexpr int A = 16 / (int)sizeof(T);  // elements per 16-byte copy granule
  static constexpr int BX = TX + A;              // the tile plus the slack of rounding down to a granule
  static constexpr int ROW_BYTES = BX * (int)sizeof(T);
  static_assert(ROW_BYTES % 16 == 0, "bulk copies move whole 16-byte units");
};

// -------------------------------------------------------------------------------------------------
// PTX helpers (shared-memory mbarrier and bulk copy)
// -------------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the phase of parity `parity` to complete; false after kPipeWaitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > kPipeWaitNs) return false;
  }
}

// Bulk copy global -> shared of `bytes` (a multiple of 16; both addresses 16-byte aligned), counted
// on `bar` as transaction bytes.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Orders this thread's generic-proxy shared-memory writes before later bulk copies into them.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Named barrier over `threads` threads (a multiple of 32).
__device__ __forceinline__ void named_barrier(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// The direction pair at which the populations split into two halves of (nearly) equal size.
template <class L>
struct DpSplit {
  static constexpr int find() {
    int acc = 0;
    for (int k = 0; k < L::NDP; ++k) {
      acc += 2 * L::DP_NPAIR[k];
      if (2 * acc >= L::Q) return k + 1;
    }
    return L::NDP;
  }
  static constexpr int value = find();
};

// Floats a consumer warp pair exchanges per tile: two buffers (alternate tiles) x two halves x 13
// partial moments x 32 lanes.
constexpr int kPipeXchgFloatsPerPair = kPipeXchgBytesPerPair / 4;

// Publish this warp's 13 partial moments (T^zz follows from the trace later), wait for the partner
// warp at named barrier `id`, and add the partner's.  Both warps add the same two numbers, so they
// hold identical moments.  The buffers alternate between tiles: a warp writes a buffer again only
// after the partner has passed the next barrier, i.e. after it has read that buffer.
__device__ __forceinline__ void exchange_moments(Mom<float>& m, float* mine, const float* other, int id) {
  mine[0 * 32] = m.N0;
  mine[1 * 32] = m.Nx;
  mine[2 * 32] = m.Ny;
  mine[3 * 32] = m.Nz;
  mine[4 * 32] = m.T00;
  mine[5 * 32] = m.T0x;
  mine[6 * 32] = m.T0y;
  mine[7 * 32] = m.T0z;
  mine[8 * 32] = m.Txx;
  mine[9 * 32] = m.Tyy;
  mine[10 * 32] = m.Txy;
  mine[11 * 32] = m.Txz;
  mine[12 * 32] = m.Tyz;
  named_barrier(id, 64);
  m.N0 += other[0 * 32];
  m.Nx += other[1 * 32];
  m.Ny += other[2 * 32];
  m.Nz += other[3 * 32];
  m.T00 += other[4 * 32];
  m.T0x += other[5 * 32];
  m.T0y += other[6 * 32];
  m.T0z += other[7 * 32];
  m.Txx += other[8 * 32];
  m.Tyy += other[9 * 32];
  m.Txy += other[10 * 32];
  m.Txz += other[11 * 32];
  m.Tyz += other[12 * 32];
}

// -------------------------------------------------------------------------------------------------
// the kernel
// -------------------------------------------------------------------------------------------------
// Source row of a pull along y or z: periodic wrap (any length) or copy-out clamp.  Beyond a
// bounce-back wall any in-range row will do: the consumer replaces those populations.
__device__ __forceinline__ int pipe_src_row(int s, int n, int bc) {
  if ((unsigned)s < (unsigned)n) return s;
  if (bc == kPeriodic) {
    s %= n;
    return s < 0 ? s + n : s;
  }
  return min(max(s, 0), n - 1);
}

// The pipeline of one launch over tiles t = blockIdx.x + k gridDim.x, k = 0, 1, ... < pp.ntiles.
// `tiles` maps a tile to its lattice: tiles.member(t) names the lattice and tiles.at(t, member)
// gives a TileRef (the lattice's parameters, buffers and status words, the tile's index within that
// lattice, and whether the lattice steps in this launch); a tile of a lattice that does not step
// still passes through its stage (no copies, no stores) so that every producer and consumer keeps
// the stage order.
template <class L, class S, int TX, bool WALLS, bool ROWS, bool ONEWARP, class Tiles>
__device__ __forceinline__ void pipe_body(const PipeParams& pp, const Tiles& tiles) {
  using T = typename S::T;
  using A = typename S::A;
  using Sh = PipeShape<S, TX>;
  constexpr bool PACKED = std::is_same<A, float>::value;
  // float storage: two warps per cell (see the consumer section) unless ONEWARP; half storage,
  // whose stages are half the size, runs more consumer groups instead
  constexpr bool SPLIT = std::is_same<S, StoreF32>::value && !ONEWARP;
  constexpr int HALVES = SPLIT ? 2 : 1;
  constexpr int KS = SPLIT ? DpSplit<L>::value : L::NDP;
  constexpr int BX = Sh::BX, AL = Sh::A, WPT = TX / 32 * HALVES;
  constexpr int kStageElems = L::Q * BX;
  constexpr bool DEV = std::is_same<S, StoreF16Dev>::value;
  static_assert(TX % 32 == 0 && TX >= 32, "tile width");

  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + kPipeMaxStages;
  char4* sv = reinterpret_cast<char4*>(smem + 2 * 8 * kPipeMaxStages);
  T* const stage0 = reinterpret_cast<T*>(smem + kPipeHeaderBytes);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cons_warps = pp.groups * WPT;  // warps [0, cons_warps) consume, the next pp.producers produce
  if (threadIdx.x == 0) {
    for (int s = 0; s < pp.nstage; ++s) {
      mbar_init(&full[s], pp.producers);
      mbar_init(&empty[s], WPT);
    }
    static_for<L::Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      constexpr signed char vx = L::VX[i], vy = L::VY[i], vz = L::VZ[i];
      sv[i] = make_char4(vx, vy, vz, 0);
    });
    mbar_fence_init();
  }
  __syncthreads();
  const long long G = gridDim.x;

  if (warp >= cons_warps) {
    // ---- producer warps, a team over every tile: producer w copies populations i = w, w + P, ...
    // (lane l takes i = l P + w, then i + 32 P), one bulk copy each (a few at a periodic x end),
    // and arrives once per tile on the stage's full barrier with its share of the bytes
    const int pw = warp - cons_warps;
    const int P = pp.producers;
    const int mine = (L::Q - pw + P - 1) / P;  // populations of this producer
    if (tiles.debug() & kDebugStallProducers) return;  // testing: nothing arrives, every wait runs out
    int k = 0;
    bool ok = true;
    for (;; ++k) {
      const long long t = blockIdx.x + (long long)k * G;
      if (t >= pp.ntiles) break;
      const int s = k % pp.nstage;
      if (k >= pp.nstage && !mbar_wait(&empty[s], (uint32_t)((k / pp.nstage) - 1) & 1u)) {
        ok = false;
        break;
      }
      const auto tr = tiles.at(t, tiles.member(t));
      const StepParams& p = tr.p;
      // row tiles: rows r0 .. r0 + gt - 1 of the lattice, gt * nx elements per population
      const int rpt = ROWS ? TX / p.nx : 1;  // rows per tile
      const int nrows = p.ny * p.nz;
      const int r0 = ROWS ? tr.lt * rpt : 0;
      const int gt = ROWS ? min(rpt, nrows - r0) : 1;
      const uint32_t pop_bytes = ROWS ? (uint32_t)(gt * p.nx * (int)sizeof(T)) : (uint32_t)Sh::ROW_BYTES;
      if (lane == 0) mbar_arrive_expect_tx(&full[s], tr.active ? (uint32_t)mine * pop_bytes : 0u);
      __syncwarp();
      if (!tr.active) continue;
      const T* __restrict__ src = tr.src;
      const int segs = ROWS ? 1 : (p.nx + TX - 1) / TX;
      const int seg = ROWS ? 0 : tr.lt % segs, row = ROWS ? r0 : tr.lt / segs;
      const int y = row % p.ny, z = row / p.ny;
      const int x0 = seg * TX;
      const bool xperiodic = p.bc[0] == kPeriodic;
      T* const st = stage0 + (size_t)s * kStageElems;
      // every copy must lie in the buffer and its guard bytes; one that does not is counted and
      // read from the buffer's start instead (the byte count of the stage stays the same)
      const long long lo = -(long long)(kPopGuardBytes / sizeof(T));
      const long long hi = (long long)L::Q * p.cells + kPopGuardBytes / sizeof(T);
      auto copy = [&](T* d, long long from, int n) {
        if (from < lo || from + n > hi) {
          atomicAdd(&tr.status[kStatusBounds], 1);
          from = 0;
        }
        bulk_g2s(d, src + from, (uint32_t)(n * sizeof(T)), &full[s]);
      };
      if constexpr (ROWS) {
        // each run of consecutive source rows of population i with one copy of whole rows
        for (int i = lane * P + pw; i < L::Q; i += 32 * P) {
          const char4 v = sv[i];
          const long long base = (long long)i * p.cells;
          T* d = st + i * BX;
          int r = 0, yr = y, zr = z;
          long long run0 = 0, next = -1;
          int runlen = 0;
          for (; r < gt; ++r) {
            const long long sr = (long long)pipe_src_row(zr - v.z, p.nz, p.bc[2]) * p.ny +
                                 pipe_src_row(yr - v.y, p.ny, p.bc[1]);
            if (sr != next) {
              if (runlen > 0) copy(d + (r - runlen) * p.nx, base + run0 * p.nx, runlen * p.nx);
              run0 = sr;
              runlen = 0;
            }
            ++runlen;
            next = sr + 1;
            if (++yr == p.ny) {
              yr = 0;
              ++zr;
            }
          }
          copy(d + (r - runlen) * p.nx, base + run0 * p.nx, runlen * p.nx);
        }
        continue;
      }
      for (int i = lane * P + pw; i < L::Q; i += 32 * P) {
        const char4 v = sv[i];
        const int ys = pipe_src_row(y - v.y, p.ny, p.bc[1]);
        const int zs = pipe_src_row(z - v.z, p.nz, p.bc[2]);
        const long long row0 = (long long)i * p.cells + ((long long)zs * p.ny + ys) * p.nx;
        const int xs = (x0 - v.x) & ~(AL - 1);  // round down to a granule (two's complement: floor)
        T* d = st + i * BX;
        if (xperiodic && (xs < 0 || xs + BX > p.nx)) {
          // split [xs, xs + BX) at multiples of nx; each piece is whole granules of one period
          int a = xs;
          const int e = xs + BX;
          while (a < e) {
            const int per = (a >= 0) ? a / p.nx : -((-a + p.nx - 1) / p.nx);
            const int pe = min(e, (per + 1) * p.nx);
            copy(d + (a - xs), row0 + (a - per * p.nx), pe - a);
            a = pe;
          }
        } else {
          // x beyond the ends reads neighbouring memory (guard bytes around every buffer); the
          // consumer patches those cells
          copy(d, row0 + xs, BX);
        }
      }
    }
    if (!ok) {
      if (lane == 0) atomicAdd(tiles.timeout_word(), 1);
      // let the copies already issued land before the block's shared memory goes away (each stage's
      // latest use among the last nstage tiles)
      for (int j = max(0, k - pp.nstage); j < k; ++j) mbar_wait(&full[j % pp.nstage], (uint32_t)(j / pp.nstage) & 1u);
    }
    return;
  }
  // ---- consumer warps.  Float storage splits every cell between two warps of a pair (HALVES =
  // 2): one takes the direction pairs [0, KS), the other [KS, NDP), each sums its partial moments,
  // the pair adds them through shared memory (a named barrier per pair and tile), both solve the
  // same Landau matching and each collides its own half.  Lane x of part `part` of the tile is
  // cell x0 + 32 part + x.
  const int group = warp / WPT, wt = warp % WPT;
  const int part = wt / HALVES, half = wt % HALVES;
  float* const xb = SPLIT ? reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(stage0) +
                                                     (size_t)pp.nstage * kStageElems * sizeof(T)) +
                                (warp >> 1) * kPipeXchgFloatsPerPair + lane
                          : nullptr;
  int iter = 0;
  // the lattice of this group's next tile, read one tile ahead (a batch looks it up in memory)
  int next_member = 0;
  if (blockIdx.x + (long long)group * G < pp.ntiles) next_member = tiles.member(blockIdx.x + (long long)group * G);
  for (int k = group;; k += pp.groups, ++iter) {
    const long long t = blockIdx.x + (long long)k * G;
    if (t >= pp.ntiles) break;
    const int s = k % pp.nstage;
    const auto tr = tiles.at(t, next_member);
    {
      const long long tn = t + (long long)pp.groups * G;
      if (tn < pp.ntiles) next_member = tiles.member(tn);
    }
    // a batch works out the tile's cells and stage offsets (from the member's parameters in
    // memory) before the wait for the stage, so that their loads overlap it; a single lattice, whose
    // parameters are kernel arguments, waits first (measured 2% faster)
    if constexpr (!Tiles::kEarlyGeometry) {
      if (!mbar_wait(&full[s], (uint32_t)(k / pp.nstage) & 1u)) {
        if (lane == 0) atomicAdd(tiles.timeout_word(), 1);
        return;
      }
    }
    const StepParams& p = tr.p;
    const T* __restrict__ src = tr.src;
    T* __restrict__ dst = tr.dst;
    int* __restrict__ status = tr.status;
    Cell cl;
    bool valid;
    T* lb;
    // row tiles: the stage offset of lane x's pull for each x velocity vx = j - VMAX_X, wrapped
    // into its row (unused otherwise)
    int xo[ROWS ? 2 * L::VMAX_X + 1 : 1];
    if constexpr (ROWS) {
      const int rpt = TX / p.nx;  // rows per tile
      const int q = part * 32 + lane;
      int r = q / p.nx;
      const int rl = tr.lt * rpt + r;  // the lattice row
      valid = r < rpt && rl < p.ny * p.nz;
      // lanes past the tile's rows read the first cell of the tile (their results are not stored)
      const int x = valid ? q - r * p.nx : 0;
      if (!valid) r = 0;
      const int rv = valid ? rl : tr.lt * rpt;
      cl.x = x;
      cl.y = rv % p.ny;
      cl.z = rv / p.ny;
      cl.c = rv * p.nx + x;
      lb = stage0 + (size_t)s * kStageElems + r * p.nx;
#pragma unroll
      for (int j = 0; j <= 2 * L::VMAX_X; ++j) {
        int o = x - (j - L::VMAX_X);
        o += o < 0 ? p.nx : 0;
        o -= o >= p.nx ? p.nx : 0;
        xo[j] = o;
      }
    } else {
      const int segs = (p.nx + TX - 1) / TX;
      const int seg = tr.lt % segs, row = tr.lt / segs;
      cl.y = row % p.ny;
      cl.z = row / p.ny;
      const int x = seg * TX + part * 32 + lane;
      valid = x < p.nx;
      cl.x = valid ? x : p.nx - 1;
      cl.c = (cl.z * p.ny + cl.y) * p.nx + cl.x;
      lb = stage0 + (size_t)s * kStageElems + part * 32 + lane;
      xo[0] = 0;
    }
    // the stage element lane x reads for population i
    auto slot = [&](auto I) -> int {
      constexpr int i = decltype(I)::value;
      if constexpr (ROWS) return i * BX + xo[L::VX[i] + L::VMAX_X];
      else return i * BX + ((-L::VX[i]) % AL + AL) % AL;
    };
    if constexpr (Tiles::kEarlyGeometry) {
      if (!mbar_wait(&full[s], (uint32_t)(k / pp.nstage) & 1u)) {
        if (lane == 0) atomicAdd(tiles.timeout_word(), 1);
        return;
      }
    }
    // a lattice that does not step, or a warp none of whose lanes holds a cell of the tile (the
    // last part of a tile of 96-cell rows, a ragged row end): release the stage and leave the issue
    // slots to the other warps (both warps of a float pair skip together)
    if (!tr.active || !__any_sync(0xffffffffu, valid)) {
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
      continue;
    }

    // patch what the copies could not express (warp-uniform test), for the populations this warp
    // reads: a copy-out or bounce-back x (segment tiles only), the walls
    const bool xperiodic = p.bc[0] == kPeriodic;
    bool patch = false;
    if constexpr (!ROWS) {
      const int x0 = (tr.lt % ((p.nx + TX - 1) / TX)) * TX;
      patch = !xperiodic && (x0 < L::VMAX_X || x0 + TX - 1 + L::VMAX_X >= p.nx);
    }
    if constexpr (WALLS) {
      const bool near = (p.bc[1] == kBounceBack && (cl.y < L::VMAX_Y || cl.y >= p.ny - L::VMAX_Y)) ||
                        (p.bc[2] == kBounceBack && (cl.z < L::VMAX_Z || cl.z >= p.nz - L::VMAX_Z));
      patch = patch || (ROWS ? __any_sync(0xffffffffu, near) : near);
    }
    if (patch) {
      static_for<L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int vx = L::VX[i];
        constexpr int ih = i < L::DP_FIRST[KS % L::NDP] || KS == L::NDP ? 0 : 1;  // half of population i
        if (SPLIT && ih != half) return;
        bool need = false;
        if constexpr (WALLS) need = p.has_wall && beyond_wall<L, i>(cl, p);
        if constexpr (vx != 0 && !ROWS) need = need || (!xperiodic && (unsigned)(cl.x - vx) >= (unsigned)p.nx);
        if (need) {
          const long long idx = pull_index<L, i, true, WALLS>(cl, p);
          if ((unsigned long long)idx < (unsigned long long)((long long)L::Q * p.cells)) {
            lb[slot(I)] = src[idx];
          } else {
            atomicAdd(&status[kStatusBounds], 1);
          }
        }
      });
      fence_proxy_async_smem();
      __syncwarp();
    }

    auto get = [&](auto I) -> A {
      const T v = lb[slot(I)];
      if constexpr (DEV) return __half2float(v);
      else return (A)v;
    };
    T* const out = dst + cl.c;
    auto store = [&](auto I, A v) {
      constexpr int i = decltype(I)::value;
      if (valid) {
        if constexpr (DEV) S::template store_dev<L, i>(out + (long long)i * p.cells, v, p);
        else S::template store<L, i>(out + (long long)i * p.cells, v, p);
      }
    };
    if constexpr (!SPLIT) {
      relax_cell<L, S, PACKED, true>(get, store, p, status, valid);
    } else {
      auto get2 = [&](auto I) -> float2 {
        constexpr int i = decltype(I)::value;
        return make_float2(get(ic<i>{}), get(ic<i + 1>{}));
      };
      const float c_dev = DEV ? p.half_nref : 0.f;
      Mom<float> m = half == 0 ? moments_f2_part<L, DEV, 0, KS>(get2) : moments_f2_part<L, DEV, KS, L::NDP>(get2);
      // exchange the 13 partial sums with the partner warp (buffer iter & 1) and add them
      float* mine = xb + ((iter & 1) * 2 + half) * 13 * 32;
      const float* other = xb + ((iter & 1) * 2 + (half ^ 1)) * 13 * 32;
      exchange_moments(m, mine, other, 1 + (warp >> 1));
      finish_moments_f2<L, DEV>(m, c_dev);
      reload_barrier();
      const Landau<float> lw = landau_step<float>(m, p);
      if (!lw.ok) {
        // no Landau frame: counted once per cell, each half streamed without collision
        if (valid) {
          if (half == 0) atomicAdd(&status[kStatusNonconv], 1);
          auto stream_half = [&](auto B, auto E) {
            static_for<decltype(E)::value - decltype(B)::value>([&](auto K) {
              constexpr int kk = decltype(B)::value + decltype(K)::value;
              static_for<2 * L::DP_NPAIR[kk]>([&](auto J) {
                constexpr int i = L::DP_FIRST[kk] + decltype(J)::value;
                store(ic<i>{}, get(ic<i>{}));
              });
            });
          };
          if (half == 0) stream_half(ic<0>{}, ic<KS>{});
          else stream_half(ic<KS>{}, ic<L::NDP>{});
        }
      } else {
        const float Tl = lw.eps / (3.f * lw.n);
        const float inv_tau = 1.f / tau_prime<float>(Tl, p);
        auto put2 = [&](auto I, float2 v) {
          constexpr int i = decltype(I)::value;
          store(ic<i>{}, v.x);
          store(ic<i + 1>{}, v.y);
        };
        if (half == 0) collide_f2<L, DEV, 0, KS>(lw, Tl, inv_tau, get2, put2, c_dev);
        else collide_f2<L, DEV, KS, L::NDP>(lw, Tl, inv_tau, get2, put2, c_dev);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
}


// A tile and the lattice it belongs to.
template <class T>
struct TileRef {
  const StepParams& p;
  const T* src;
  T* dst;
  int* status;
  int lt;       // the tile's index within its lattice: row * segs + seg
  bool active;  // the lattice steps in this launch
};

// One lattice: tile t is the lattice's tile t.
template <class T>
struct SoloTiles {
  static constexpr bool kEarlyGeometry = false;
  const StepParams& p;
  const T* src;
  T* dst;
  int* status;
  __device__ __forceinline__ int member(long long) const { return 0; }
  __device__ __forceinline__ TileRef<T> at(long long t, int) const {
    return TileRef<T>{p, src, dst, status, (int)t, true};
  }
  __device__ __forceinline__ int* timeout_word() const { return status + kStatusTimeout; }
  __device__ __forceinline__ int debug() const { return p.debug; }
};

// Many lattices (batch members): tile t belongs to member tile_member[t], whose tiles start at its
// pipe_tile_begin; the member reads buf[(parity0 + launch) & 1] and writes the other buffer, and
// steps only while launch < steps_left.
template <class T>
struct BatchTiles {
  static constexpr bool kEarlyGeometry = true;
  const BatchMember* members;
  const int* tile_member;
  int launch;
  int* timeout;
  __device__ __forceinline__ int member(long long t) const { return __ldg(&tile_member[t]); }
  __device__ __forceinline__ TileRef<T> at(long long t, int mi) const {
    const BatchMember& m = members[mi];
    const int par = (m.parity0 + launch) & 1;
    return TileRef<T>{m.p, static_cast<const T*>(m.buf[par]), static_cast<T*>(m.buf[par ^ 1]), m.status,
                      (int)(t - m.pipe_tile_begin), launch < m.steps_left};
  }
  __device__ __forceinline__ int* timeout_word() const { return timeout; }
  __device__ __forceinline__ int debug() const { return 0; }
};

// One time step of one lattice.
template <class L, class S, int TX, bool WALLS, bool ROWS, bool ONEWARP>
__global__ void __launch_bounds__(kPipeMaxThreads, 1)
    k_step_pipe(const typename S::T* __restrict__ src, typename S::T* __restrict__ dst,
                const __grid_constant__ StepParams p, const __grid_constant__ PipeParams pp,
                int* __restrict__ status) {
  using T = typename S::T;
  pipe_body<L, S, TX, WALLS, ROWS, ONEWARP>(pp, SoloTiles<T>{p, src, dst, status});
}

// One time step of every batch member with steps left (launch index `launch`), persistent over the
// members' tiles.  A member's result is bitwise that of k_step_pipe on it alone.  Waits that run
// out are counted in *timeout (the first member's status words).
template <class L, class S, int TX, bool WALLS, bool ROWS, bool ONEWARP>
__global__ void __launch_bounds__(kPipeMaxThreads, 1)
    k_step_pipe_batch(const BatchMember* __restrict__ members, const int* __restrict__ tile_member, int launch,
                      const __grid_constant__ PipeParams pp, int* __restrict__ timeout) {
  using T = typename S::T;
  pipe_body<L, S, TX, WALLS, ROWS, ONEWARP>(pp, BatchTiles<T>{members, tile_member, launch, timeout});
}

}  // namespace rlb
