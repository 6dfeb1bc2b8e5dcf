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

// Blocks covering `items` work items at `threads` per block and `per_thread`
// items per thread (every kernel here keeps a grid-stride loop, so any grid
// size stays correct).  The hardware block scheduler then walks memory in
// order and backfills each SM as its blocks finish.  On GB300 a covering grid
// streamed ~8% faster than a persistent one-wave grid-stride launch of the
// same kernel (7.0 vs 6.45 TB/s); kernels heavy in registers and arithmetic
// gain from a few items per thread (fewer block launches per SM), as long as
// the grid keeps at least `min_blocks` blocks (several per SM, so the last
// wave is short): below that, items per thread drop toward one.
inline int64_t cover_blocks(int64_t items, int threads, int per_thread = 1,
                            int64_t min_blocks = 0) {
  const int64_t span = (int64_t)threads * per_thread;
  int64_t b = (items + span - 1) / span;
  if (b < min_blocks) {
    const int64_t one = (items + threads - 1) / threads;  // one item per thread
    b = one < min_blocks ? one : min_blocks;
  }
  if (b < 1) b = 1;
  return b > 2147483647 ? 2147483647 : b;
}

// Blocks per SM a multi-item launch keeps at least (see cover_blocks).
constexpr int kMinBlocksPerSm = 8;

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
