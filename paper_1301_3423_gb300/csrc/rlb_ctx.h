// The simulation context behind the opaque rlb_ctx handle (host side; shared by the C-ABI units).
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "rlb.h"
#include "rlb_common.h"
#include "rlb_launch.h"

struct rlb_ctx {
  rlb_params prm;
  int q = 0;
  int cells = 0;
  size_t elem = 0;
  void* raw[2] = {nullptr, nullptr};  // allocations: kPopGuardBytes, the buffer, kPopGuardBytes
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;              // buf[cur] holds the current (post-collision) state
  bool have_prev = false;   // buf[1 - cur] holds the state the last step pulled from
  long steps = 0;
  long launches = 0;
  cudaStream_t stream = nullptr;
  rlb::StepParams sp;
  bool general_wrap = false;
  double* fields = nullptr;   // 6 * cells; also staging for host inputs
  double* partial = nullptr;  // 5 * blocks
  double* totals = nullptr;   // 5
  int* status = nullptr;      // kStatusWords
  int fblocks = 0;
  const rlb::Launchers* launch = nullptr;
  int variant = 0;            // step-kernel variant (kNumRegVariants register kernels, then pipelined shapes)
  int sms = 0, smem_per_sm = 0, smem_optin = 0;  // device: SMs, shared memory per SM, per block (opt-in)
  // host transfers of rlb_init / rlb_moments run in chunks on a copy stream that overlaps the
  // kernels on `stream` (created on first use)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_ready = nullptr;
  cudaEvent_t ev_chunk[8] = {nullptr};
  std::string err;
};
