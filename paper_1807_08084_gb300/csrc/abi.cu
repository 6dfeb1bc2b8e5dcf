// abi.cu -- version, status strings, per-device properties, pointer checks and
// launch sizing shared by the entry points.
#include <atomic>

#include "common.cuh"

namespace zinv {

namespace {
struct DeviceSlot {
  std::once_flag once;
  int rc = ZINV_ERR_DEVICE;
  DeviceInfo info;
};
DeviceSlot g_devices[kMaxDevices];
}  // namespace

int device_info(DeviceInfo* out, int* dev_out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return ZINV_ERR_DEVICE;
  }
  DeviceSlot& slot = g_devices[dev];
  std::call_once(slot.once, [&]() {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    // The kernels are compiled for sm_103a only.
    if (prop.major != 10 || prop.minor != 3) return;
    slot.info.ok = true;
    slot.info.sm_count = prop.multiProcessorCount;
    slot.info.max_threads_per_sm = prop.maxThreadsPerMultiProcessor;
    slot.rc = ZINV_OK;
  });
  if (slot.rc != ZINV_OK) return slot.rc;
  *out = slot.info;
  if (dev_out) *dev_out = dev;
  return ZINV_OK;
}

bool device_accessible(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  switch (a.type) {
    case cudaMemoryTypeDevice:
    case cudaMemoryTypeManaged:
      return true;
    case cudaMemoryTypeHost:
      return a.devicePointer != nullptr;
    default:
      return false;
  }
}

}  // namespace zinv

extern "C" int zinv_abi_version(void) { return ZINV_ABI_VERSION; }

extern "C" const char* zinv_status_string(int code) {
  switch (code) {
    case ZINV_OK: return "ok";
    case ZINV_ERR_ARG: return "invalid argument";
    case ZINV_ERR_LAUNCH: return "CUDA call or kernel launch failed";
    case ZINV_ERR_DEVICE: return "no sm_103 CUDA device is current";
    default: return "unknown status";
  }
}
