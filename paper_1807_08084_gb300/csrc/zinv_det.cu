// zinv_det.cu -- kernels and C entry points zinv_det (Alg. 2 of the paper,
// with compensated and FP64-recompute variants) and chol_zinv_det (Alg. 1).
//
// The path is HBM-bound: 36 bytes in and 40 bytes out per pixel against ~64
// FP32 operations.  Layout is planar SoA, so a warp's access to one plane is
// one contiguous run.  The main kernel gives each thread four consecutive
// pixels: nine 128-bit streaming loads (one per plane), the arithmetic on four
// independent pixels, ten 128-bit streaming stores.  The grid covers the
// image (see kGroupsPerThread for the per-variant split), which streamed
// faster than a persistent grid.  Pixels that do not fill a float4 (n % 4) and
// unaligned layouts take the one-pixel-per-thread kernel, still coalesced.
#include "common.cuh"
#include "pixel.cuh"

namespace zinv {

constexpr int kThreads = 256;

// Launch shape per variant, from a sweep on GB300 over a 16384 x 16384 image.
// The light variants stream best with one group of four pixels per thread.
// The compensated ones hold more registers and arithmetic per group and run
// best with several groups per thread: 32 for compensated (3.21 -> 3.02 ms),
// 16 for compensated + FP64, whose register cap for three blocks per SM (at
// the cost of some spills) took it from 4.22 to 3.43 ms.
template <int ALG>
constexpr int kGroupsPerThread = ALG == kComp ? 32 : ALG == kCompF64 ? 16 : 1;

template <int ALG, bool STAT>
__device__ __forceinline__ void one_pixel(const float* __restrict__ z, int64_t ld, int64_t p,
                                          float* __restrict__ zinv, float* __restrict__ det,
                                          float tau, uint8_t* __restrict__ status, uint32_t& c0,
                                          uint32_t& c1) {
  float x[9], w[9], dt;
#pragma unroll
  for (int k = 0; k < 9; ++k) x[k] = __ldcs(z + k * ld + p);
  const uint32_t st = pixel_inv_det<ALG>(x, w, dt, tau);
#pragma unroll
  for (int k = 0; k < 9; ++k) __stcs(zinv + k * ld + p, w[k]);
  __stcs(det + p, dt);
  if (STAT) {
    if (status) status[p] = (uint8_t)st;
    c0 += st & ZINV_PIX_NOT_PD;
    c1 += (st & ZINV_PIX_RECOMPUTED) >> 1;
  }
}

template <int ALG, bool STAT>
__device__ __forceinline__ void inv_det_vec4(const float* __restrict__ z, int64_t n, int64_t ld,
                                             float* __restrict__ zinv, float* __restrict__ det,
                                             float tau, uint8_t* __restrict__ status,
                                             unsigned long long* __restrict__ counts) {
  const int64_t groups = n >> 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  uint32_t c0 = 0, c1 = 0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += stride) {
    float4 v[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) v[k] = __ldcs(reinterpret_cast<const float4*>(z + k * ld) + g);
    float4 o[9], dv;
    uint32_t sv = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float x[9], w[9], dt;
#pragma unroll
      for (int k = 0; k < 9; ++k) x[k] = lane(v[k], j);
      const uint32_t st = pixel_inv_det<ALG>(x, w, dt, tau);
#pragma unroll
      for (int k = 0; k < 9; ++k) set_lane(o[k], j, w[k]);
      set_lane(dv, j, dt);
      if (STAT) {
        sv |= st << (8 * j);
        c0 += st & ZINV_PIX_NOT_PD;
        c1 += (st & ZINV_PIX_RECOMPUTED) >> 1;
      }
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) __stcs(reinterpret_cast<float4*>(zinv + k * ld) + g, o[k]);
    __stcs(reinterpret_cast<float4*>(det) + g, dv);
    if (STAT && status) reinterpret_cast<uint32_t*>(status)[g] = sv;
  }
  // ragged tail: n % 4 pixels after the last full group
  const int64_t p = (groups << 2) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.x == 0 && p < n) one_pixel<ALG, STAT>(z, ld, p, zinv, det, tau, status, c0, c1);
  if (STAT && counts) add_counts(counts, c0, c1);
}

template <int ALG, bool STAT>
__global__ void __launch_bounds__(kThreads)
    k_inv_det_vec4(const float* __restrict__ z, int64_t n, int64_t ld, float* __restrict__ zinv,
                   float* __restrict__ det, float tau, uint8_t* __restrict__ status,
                   unsigned long long* __restrict__ counts) {
  inv_det_vec4<ALG, STAT>(z, n, ld, zinv, det, tau, status, counts);
}

// Compensated + FP64 recompute, held to three blocks per SM.
template <bool STAT>
__global__ void __launch_bounds__(kThreads, 3)
    k_inv_det_vec4_c64(const float* __restrict__ z, int64_t n, int64_t ld,
                       float* __restrict__ zinv, float* __restrict__ det, float tau,
                       uint8_t* __restrict__ status, unsigned long long* __restrict__ counts) {
  inv_det_vec4<kCompF64, STAT>(z, n, ld, zinv, det, tau, status, counts);
}

template <int ALG, bool STAT>
__global__ void __launch_bounds__(kThreads)
    k_inv_det_scalar(const float* __restrict__ z, int64_t n, int64_t ld, float* __restrict__ zinv,
                     float* __restrict__ det, float tau, uint8_t* __restrict__ status,
                     unsigned long long* __restrict__ counts) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  uint32_t c0 = 0, c1 = 0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride)
    one_pixel<ALG, STAT>(z, ld, p, zinv, det, tau, status, c0, c1);
  if (STAT && counts) add_counts(counts, c0, c1);
}

template <int ALG, bool STAT>
static int launch_inv_det(const float* z, int64_t n, int64_t ld, float* zinv, float* det,
                          float tau, uint8_t* status, unsigned long long* counts,
                          cudaStream_t s, int64_t min_blocks) {
  const bool vec = (ld % 4 == 0) && aligned(z, 16) && aligned(zinv, 16) && aligned(det, 16) &&
                   (status == nullptr || aligned(status, 4));
  if (vec) {
    const int64_t items = (n >> 2) > 0 ? (n >> 2) : 1;
    const unsigned blocks =
        (unsigned)cover_blocks(items, kThreads, kGroupsPerThread<ALG>, min_blocks);
    if constexpr (ALG == kCompF64)
      k_inv_det_vec4_c64<STAT><<<blocks, kThreads, 0, s>>>(z, n, ld, zinv, det, tau, status,
                                                           counts);
    else
      k_inv_det_vec4<ALG, STAT><<<blocks, kThreads, 0, s>>>(z, n, ld, zinv, det, tau, status,
                                                            counts);
  } else {
    auto k = k_inv_det_scalar<ALG, STAT>;
    k<<<(unsigned)cover_blocks(n, kThreads), kThreads, 0, s>>>(z, n, ld, zinv, det, tau, status,
                                                               counts);
  }
  return launch_status();
}

template <int ALG>
static int dispatch_stat(const float* z, int64_t n, int64_t ld, float* zinv, float* det,
                         float tau, uint8_t* status, unsigned long long* counts, cudaStream_t s,
                         int64_t min_blocks) {
  if (status || counts)
    return launch_inv_det<ALG, true>(z, n, ld, zinv, det, tau, status, counts, s, min_blocks);
  return launch_inv_det<ALG, false>(z, n, ld, zinv, det, tau, status, counts, s, min_blocks);
}

// Shared argument checks of zinv_det / chol_zinv_det: sizes and pointer
// alignment first (pure host logic), accessibility after the device check.
static int check_scalar_args(const float* z, int64_t n, int64_t ld, const float* zinv,
                             const float* det, float tau, const int64_t* counts) {
  if (n < 0 || ld < n || ld > kMaxLd) return ZINV_ERR_ARG;
  if (!(tau >= 0.0f) || isinf(tau)) return ZINV_ERR_ARG;
  if (n > 0 && (!z || !zinv || !det)) return ZINV_ERR_ARG;
  if (!aligned(z, 4) || !aligned(zinv, 4) || !aligned(det, 4) || !aligned(counts, 8))
    return ZINV_ERR_ARG;
  return ZINV_OK;
}

static int check_pointers(const float* z, int64_t n, const float* zinv, const float* det,
                          const uint8_t* status, const int64_t* counts) {
  if (n > 0 && (!device_accessible(z) || !device_accessible(zinv) || !device_accessible(det)))
    return ZINV_ERR_ARG;
  if (status && !device_accessible(status)) return ZINV_ERR_ARG;
  if (counts && !device_accessible(counts)) return ZINV_ERR_ARG;
  return ZINV_OK;
}

int inv_det_entry(int alg, const float* z, int64_t n, int64_t ld, float* zinv, float* det,
                  float tau, uint8_t* status, int64_t* counts, cudaStream_t s) {
  int rc = check_scalar_args(z, n, ld, zinv, det, tau, counts);
  if (rc != ZINV_OK) return rc;
  DeviceInfo di;
  rc = device_info(&di);
  if (rc != ZINV_OK) return rc;
  rc = check_pointers(z, n, zinv, det, status, counts);
  if (rc != ZINV_OK) return rc;
  auto* cnt = reinterpret_cast<unsigned long long*>(counts);
  if (cnt && cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), s) != cudaSuccess)
    return ZINV_ERR_LAUNCH;
  if (n == 0) return ZINV_OK;
  const int64_t mb = (int64_t)kMinBlocksPerSm * di.sm_count;
  switch (alg) {
    case kPlain: return dispatch_stat<kPlain>(z, n, ld, zinv, det, tau, status, cnt, s, mb);
    case kComp: return dispatch_stat<kComp>(z, n, ld, zinv, det, tau, status, cnt, s, mb);
    case kPlainF64:
      return dispatch_stat<kPlainF64>(z, n, ld, zinv, det, tau, status, cnt, s, mb);
    case kCompF64:
      return dispatch_stat<kCompF64>(z, n, ld, zinv, det, tau, status, cnt, s, mb);
    case kChol: return dispatch_stat<kChol>(z, n, ld, zinv, det, tau, status, cnt, s, mb);
  }
  return ZINV_ERR_ARG;
}

int alg_from_flags(uint32_t flags) {
  if (flags & ~(ZINV_COMPENSATED | ZINV_FP64_RECOMPUTE)) return -1;
  const bool comp = flags & ZINV_COMPENSATED, f64 = flags & ZINV_FP64_RECOMPUTE;
  return comp ? (f64 ? kCompF64 : kComp) : (f64 ? kPlainF64 : kPlain);
}

}  // namespace zinv

extern "C" int zinv_det(const float* z, int64_t n, int64_t ld, float* zinv, float* det,
                        uint32_t flags, float tau, uint8_t* status, int64_t* counts,
                        void* stream) {
  const int alg = zinv::alg_from_flags(flags);
  if (alg < 0) return ZINV_ERR_ARG;
  return zinv::inv_det_entry(alg, z, n, ld, zinv, det, tau, status, counts,
                             static_cast<cudaStream_t>(stream));
}

extern "C" int chol_zinv_det(const float* z, int64_t n, int64_t ld, float* zinv, float* det,
                             uint32_t flags, float tau, uint8_t* status, int64_t* counts,
                             void* stream) {
  if (flags != ZINV_PLAIN) return ZINV_ERR_ARG;
  return zinv::inv_det_entry(zinv::kChol, z, n, ld, zinv, det, tau, status, counts,
                             static_cast<cudaStream_t>(stream));
}
