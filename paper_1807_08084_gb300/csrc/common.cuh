// common.cuh -- host-side helpers shared by the libzinv.so translation units:
// device checks, launch sizing, pointer checks, and the packed-pixel struct.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <mutex>

#include "zinv.h"

namespace zinv {

constexpr int kMaxDevices = 64;

struct DeviceInfo {
  bool ok = false;      // sm_103 and queried
  int sm_count = 0;
  int max_threads_per_sm = 0;
};

// Device properties, queried once per device.  Returns ZINV_OK or ZINV_ERR_DEVICE.
int device_info(DeviceInfo* out, int* dev_out = nullptr);

// True when the GPU can dereference p (device, managed, or mapped host memory).
bool device_accessible(const void* p);

// Blocks for a grid-stride kernel: enough to cover `items` work items at
// `threads` per block, capped at (resident blocks per SM) x (SM count) so the
// grid is a whole number of waves over the 152 SMs.
int64_t grid_blocks(const void* kernel, int threads, size_t smem, int64_t items,
                    const DeviceInfo& di);

inline bool aligned(const void* p, uintptr_t a) {
  return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0;
}

// Largest plane stride whose nine planes of 4-byte elements stay addressable
// with int64 offsets.
constexpr int64_t kMaxLd = (int64_t)1 << 58;

inline int launch_status() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ZINV_OK : ZINV_ERR_LAUNCH;
}

}  // namespace zinv
