// rlb_totals_noalloc: the conserved-density sums of a caller-owned population buffer, computed
// without allocating any memory.
//
// rlb_moments sums N^0 and T^{0 nu} through per-block partials that live in memory the context
// allocated with cudaMalloc.  Some callers cannot call the device allocator at all: plug-ins whose
// host application owns every device allocation, processes that have reserved the whole device for
// their own pools, or code under a hard memory budget.  This entry point keeps its scratch in a
// fixed array in the library's own device data segment, which exists on every device that loads
// the library, from load until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "rlb.h"
#include "rlb_kernels.cuh"

namespace {

using namespace rlb;

constexpr int kNoallocMaxBlocks = RLB_NOALLOC_MAX_CELLS / kMomThreads;

// Scratch shared by every call: one slot of 5 partial sums per block, and the 5 totals.
// Every slot a call reads is written by the same call first, so nothing needs clearing.
static __device__ __align__(256) double g_noalloc_scratch[kNoallocMaxBlocks * 5 + 5];

// Per-block sums of N^0, T^00, T^0x, T^0y, T^0z of the stored populations of each cell; the same
// per-cell arithmetic, block size, warp shuffles and shared-memory tree as the fields kernel,
// written to partial[].
template <class L, class S>
__global__ void __launch_bounds__(kMomThreads) k_densities_noalloc(const typename S::T* __restrict__ src,
                                                                   const __grid_constant__ StepParams p,
                                                                   double* __restrict__ partial) {
  const int gid = blockIdx.x * kMomThreads + threadIdx.x;
  const bool valid = gid < p.cells;
  const int c = valid ? gid : p.cells - 1;
  // per-cell moments in the arithmetic rlb_moments uses for this storage (double for double
  // populations; the fields kernel's float sums for float and half-deviation ones), summed across
  // cells in double
  Mom<double> m;
  if constexpr (std::is_same<typename S::A, double>::value) {
    m = moments<L, double>([&](auto I) -> double { return src[(long long)decltype(I)::value * p.cells + c]; });
  } else {
    constexpr bool DEV = std::is_same<S, StoreF16Dev>::value;
    auto getf = [&](auto I) -> float {
      constexpr int i = decltype(I)::value;
      if constexpr (DEV) return S::template load_dev<L, i>(src + (long long)i * p.cells + c, p);
      else return (float)src[(long long)i * p.cells + c];
    };
    m = moments_pd<L, DEV>(getf, (double)p.half_nref);
  }
  double d[5] = {valid ? m.N0 : 0.0, valid ? m.T00 : 0.0, valid ? m.T0x : 0.0, valid ? m.T0y : 0.0,
                 valid ? m.T0z : 0.0};
#pragma unroll
  for (int k = 0; k < 5; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d[k] += __shfl_down_sync(0xffffffffu, d[k], o);
  __shared__ double ws[kMomThreads / 32][5];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 5; ++k) ws[warp][k] = d[k];
  __syncthreads();
  if (threadIdx.x < 5) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kMomThreads / 32; ++w) s += ws[w][threadIdx.x];
    partial[(long long)blockIdx.x * 5 + threadIdx.x] = s;
  }
}

// Second pass: one block adds the partials in a fixed order and writes the 5 totals.
__global__ void __launch_bounds__(kReduceThreads) k_totals_noalloc(const double* __restrict__ partial, int nblocks,
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

// Device address of the scratch array, looked up once per device with that device current.
// In host code g_noalloc_scratch names a host-side stand-in, never the device array itself.  The
// per-device cache is guarded by a mutex: calls from several host threads see either no entry
// (and one of them looks it up) or the finished one.
constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(ptr);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

template <class L, class S>
cudaError_t launch(const void* f, const StepParams& p, double* scratch, int blocks, cudaStream_t s) {
  k_densities_noalloc<L, S><<<blocks, kMomThreads, 0, s>>>(static_cast<const typename S::T*>(f), p, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_totals_noalloc<<<1, kReduceThreads, 0, s>>>(scratch, blocks, scratch + (size_t)kNoallocMaxBlocks * 5);
  return cudaGetLastError();
}

}  // namespace

namespace rlb {
void set_thread_error(const std::string& msg);  // rlb_api.cu: the text rlb_last_error(NULL) returns
}

extern "C" rlb_status rlb_totals_noalloc(int order, int storage, int nx, int ny, int nz, double n_ref, const void* f,
                                         double totals[5], void* stream) {
  if ((order != 2 && order != 3) || (storage != RLB_F64 && storage != RLB_F32 && storage != RLB_F16DEV)) {
    rlb::set_thread_error("rlb_totals_noalloc: order must be 2 or 3 and storage one of RLB_F64/F32/F16DEV");
    return RLB_EINVAL;
  }
  if (!f || !totals || nx < 1 || ny < 1 || nz < 1) {
    rlb::set_thread_error("rlb_totals_noalloc: null pointer or empty lattice");
    return RLB_EINVAL;
  }
  const long long cells = (long long)nx * ny * nz;
  if (cells > RLB_NOALLOC_MAX_CELLS) {
    rlb::set_thread_error("rlb_totals_noalloc: " + std::to_string(cells) + " cells exceed the fixed scratch limit of " +
                          std::to_string((long long)RLB_NOALLOC_MAX_CELLS) + " cells");
    return RLB_EINVAL;
  }
  if (storage == RLB_F16DEV && !(n_ref > 0)) {
    rlb::set_thread_error("rlb_totals_noalloc: n_ref must be > 0");
    return RLB_EINVAL;
  }
  double* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) {
    rlb::set_thread_error(std::string("rlb_totals_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    return RLB_ECUDA;
  }
  StepParams p{};
  p.nx = nx;
  p.ny = ny;
  p.nz = nz;
  p.nxy = nx * ny;
  p.cells = (int)cells;
  p.half_nref = (float)(0.5 * n_ref);
  const int blocks = (int)((cells + kMomThreads - 1) / kMomThreads);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (order == 3)
    e = storage == RLB_F64 ? launch<Quad3, StoreF64>(f, p, scratch, blocks, s)
        : storage == RLB_F32 ? launch<Quad3, StoreF32>(f, p, scratch, blocks, s)
                             : launch<Quad3, StoreF16Dev>(f, p, scratch, blocks, s);
  else
    e = storage == RLB_F64 ? launch<Quad2, StoreF64>(f, p, scratch, blocks, s)
        : storage == RLB_F32 ? launch<Quad2, StoreF32>(f, p, scratch, blocks, s)
                             : launch<Quad2, StoreF16Dev>(f, p, scratch, blocks, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(totals, scratch + (size_t)kNoallocMaxBlocks * 5, 5 * sizeof(double), cudaMemcpyDeviceToHost,
                        s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    rlb::set_thread_error(std::string("rlb_totals_noalloc: ") + cudaGetErrorString(e));
    return RLB_ECUDA;
  }
  return RLB_OK;
}
