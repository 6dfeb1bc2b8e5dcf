// zinv_host.cu -- zinv_det over host buffers (§4.3 of the paper: an image that
// does not fit is fed through the GPU in pieces, processed and pulled back).
//
// Two ways, chosen per call:
//   - direct: when every host buffer is GPU-accessible (page-locked, or
//     registered), the kernel reads and writes host memory itself over the
//     coherent CPU-GPU link; one launch, no copies, no workspace.  On GB300 this
//     was ~15% faster than staging (both are bound by the host side: ~330 GB/s
//     read + write);
//   - staged (otherwise, or with ZINV_HOST_STAGED): three ring slots in the
//     caller's workspace; per chunk one stream copies the nine planes in, one
//     runs the kernel in place, one copies the nine planes and det out, so the
//     two copy directions and the SMs work on three chunks at once.
#include <mutex>

#include "common.cuh"

namespace zinv {
int inv_det_entry(int alg, const float* z, int64_t n, int64_t ld, float* zinv, float* det,
                  float tau, uint8_t* status, int64_t* counts, cudaStream_t s);
int alg_from_flags(uint32_t flags);

namespace {
constexpr int kSlots = 3;
constexpr size_t kAlign = 256;

inline size_t round_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// bytes of one slot: nine planes (input, overwritten by the inverse) and det
inline size_t slot_bytes(int64_t chunk) {
  return round_up((size_t)chunk * 9 * sizeof(float)) + round_up((size_t)chunk * sizeof(float));
}

struct Pipe {
  std::once_flag once;
  bool ok = false;
  cudaStream_t st[3];  // 0: host->device, 1: compute, 2: device->host
  cudaEvent_t start, done[3];
  cudaEvent_t in_ready[kSlots], computed[kSlots], drained[kSlots];
};
Pipe g_pipes[kMaxDevices];

bool make_pipe(Pipe& p) {
  for (auto& s : p.st)
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return false;
  auto mk = [](cudaEvent_t* e) {
    return cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
  };
  if (!mk(&p.start)) return false;
  for (auto& e : p.done)
    if (!mk(&e)) return false;
  for (int i = 0; i < kSlots; ++i)
    if (!mk(&p.in_ready[i]) || !mk(&p.computed[i]) || !mk(&p.drained[i])) return false;
  return true;
}
}  // namespace
}  // namespace zinv

extern "C" size_t zinv_det_host_workspace_bytes(int64_t chunk) {
  if (chunk < 1) return 0;
  return zinv::kSlots * zinv::slot_bytes(chunk);
}

extern "C" int zinv_det_host(const float* z_host, int64_t n, int64_t ld, float* zinv_host,
                             float* det_host, uint32_t flags, float tau, void* d_ws,
                             size_t ws_bytes, void* stream) {
  using namespace zinv;
  const bool staged = flags & ZINV_HOST_STAGED;
  const int alg = alg_from_flags(flags & ~ZINV_HOST_STAGED);
  if (alg < 0 || n < 0 || ld < n || ld > kMaxLd) return ZINV_ERR_ARG;
  if (!(tau >= 0.0f) || isinf(tau)) return ZINV_ERR_ARG;
  if (n > 0 && (!z_host || !zinv_host || !det_host)) return ZINV_ERR_ARG;
  if (d_ws && !aligned(d_ws, kAlign)) return ZINV_ERR_ARG;
  DeviceInfo di;
  int dev = -1;
  int rc = device_info(&di, &dev);
  if (rc != ZINV_OK) return rc;
  if (n == 0) return ZINV_OK;
  cudaStream_t user = static_cast<cudaStream_t>(stream);
  if (!staged && device_accessible(z_host) && device_accessible(zinv_host) &&
      device_accessible(det_host))
    return inv_det_entry(alg, z_host, n, ld, zinv_host, det_host, tau, nullptr, nullptr, user);
  if (!d_ws || !aligned(d_ws, kAlign) || !device_accessible(d_ws)) return ZINV_ERR_ARG;
  // largest chunk whose three slots fit, a multiple of 4 pixels when possible
  int64_t chunk = (int64_t)(ws_bytes / kSlots / 40);
  while (chunk > 0 && zinv_det_host_workspace_bytes(chunk) > ws_bytes) --chunk;
  if (chunk < 1) return ZINV_ERR_ARG;
  if (chunk > 4) chunk &= ~(int64_t)3;
  if (chunk > n) {
    const int64_t r = (n + 3) & ~(int64_t)3;
    if (r < chunk) chunk = r;  // only shrinks, so it still fits
  }

  Pipe& p = g_pipes[dev];
  std::call_once(p.once, [&]() { p.ok = make_pipe(p); });
  if (!p.ok) return ZINV_ERR_LAUNCH;
  const size_t sb = slot_bytes(chunk);
  char* ws = static_cast<char*>(d_ws);

  // Once the first copy is queued, every way out -- success or error -- records
  // the three streams' ends and makes the caller's stream wait for them, so
  // a caller that sees an error and synchronizes its stream before freeing the
  // host buffers never races with a transfer still in flight.
  bool enqueued = false;
  auto join = [&]() {
    bool ok = true;
    for (int i = 0; i < 3; ++i) {
      ok = ok && cudaEventRecord(p.done[i], p.st[i]) == cudaSuccess;
      ok = ok && cudaStreamWaitEvent(user, p.done[i], 0) == cudaSuccess;
    }
    return ok;
  };
  auto fail = [&](int code) {
    cudaGetLastError();
    if (enqueued && !join()) {
      // the join itself failed: wait on the host so nothing is left in flight
      for (auto& st : p.st) cudaStreamSynchronize(st);
      cudaGetLastError();
    }
    return code;
  };
#define ZCHK(x)                                   \
  do {                                            \
    if ((x) != cudaSuccess) return fail(ZINV_ERR_LAUNCH); \
  } while (0)

  ZCHK(cudaEventRecord(p.start, user));
  for (auto& s : p.st) ZCHK(cudaStreamWaitEvent(s, p.start, 0));
  const int64_t nchunks = (n + chunk - 1) / chunk;
  for (int64_t c = 0; c < nchunks; ++c) {
    const int slot = (int)(c % kSlots);
    const int64_t p0 = c * chunk;
    const int64_t m = (n - p0) < chunk ? (n - p0) : chunk;
    float* dz = reinterpret_cast<float*>(ws + slot * sb);
    float* dd = reinterpret_cast<float*>(ws + slot * sb + round_up((size_t)chunk * 9 * 4));
    // copy in (after the slot's previous chunk has drained)
    if (c >= kSlots) ZCHK(cudaStreamWaitEvent(p.st[0], p.drained[slot], 0));
    enqueued = true;
    for (int k = 0; k < 9; ++k)
      ZCHK(cudaMemcpyAsync(dz + k * chunk, z_host + k * ld + p0, (size_t)m * 4,
                           cudaMemcpyHostToDevice, p.st[0]));
    ZCHK(cudaEventRecord(p.in_ready[slot], p.st[0]));
    // compute in place
    ZCHK(cudaStreamWaitEvent(p.st[1], p.in_ready[slot], 0));
    rc = inv_det_entry(alg, dz, m, chunk, dz, dd, tau, nullptr, nullptr, p.st[1]);
    if (rc != ZINV_OK) return fail(rc);
    ZCHK(cudaEventRecord(p.computed[slot], p.st[1]));
    // copy out
    ZCHK(cudaStreamWaitEvent(p.st[2], p.computed[slot], 0));
    for (int k = 0; k < 9; ++k)
      ZCHK(cudaMemcpyAsync(zinv_host + k * ld + p0, dz + k * chunk, (size_t)m * 4,
                           cudaMemcpyDeviceToHost, p.st[2]));
    ZCHK(cudaMemcpyAsync(det_host + p0, dd, (size_t)m * 4, cudaMemcpyDeviceToHost, p.st[2]));
    ZCHK(cudaEventRecord(p.drained[slot], p.st[2]));
  }
  if (!join()) return fail(ZINV_ERR_LAUNCH);
#undef ZCHK
  return ZINV_OK;
}
