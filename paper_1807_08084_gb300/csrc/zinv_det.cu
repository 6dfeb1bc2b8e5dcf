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
//
// FP64 recompute variants: the four-pixel kernel takes every pixel through
// the FP32 route and stores it; each warp queues its flagged pixels in shared
// memory and recomputes them 32 at a time, one per lane, overwriting the FP32
// results.  FP64 runs at 1/64 of the FP32 rate on GB300, so a warp that took
// the FP64 branch for whichever of its lanes were flagged (about half of them
// on an ill-conditioned scene) spent most of its time on idle lanes.
#include "common.cuh"
#include "pixel.cuh"

namespace zinv {

constexpr int kThreads = 256;

// z and zinv carry no __restrict__: zinv == z (in place) is allowed, and the
// FP64 queue reads back the inputs it parked in zinv.  Every access to them is
// an explicit streaming load or store (__ldcs, __ldcg, __stcs), so the code
// does not rely on the two being distinct.  det, status and counts never alias
// an input.

// Launch shape per variant, from sweeps on GB300 over the 16384 x 16384 image
// (nothing flagged) and the 4096 x 4096 cond-controlled one (54% flagged).
// The light variants stream best with one group of four pixels per thread.
// The compensated one holds more registers and arithmetic per group and runs
// best with 32 groups per thread (3.21 -> 3.02 ms).  The FP64 variants take
// 16 (plain) and 32 (compensated) groups, so a warp's queue fills whole rounds
// of 32 and a partial round runs once per thread's share: on the ill-
// conditioned image 7.66 ms with one group, 6.04 with 16, for 2% more on the
// image where nothing is flagged.
template <int ALG>
constexpr int kGroupsPerThread =
    ALG == kComp ? 32 : ALG == kCompF64 ? 32 : ALG == kPlainF64 ? 16 : 1;

// Per-warp queue of flagged pixels: at most 31 left from the last flush plus
// 128 from one step (four pixels per lane).
constexpr int kQueue = 160;

template <int ALG, bool STAT>
__device__ __forceinline__ void one_pixel(const float* z, int64_t ld, int64_t p,
                                          float* zinv, float* __restrict__ det,
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
__device__ __forceinline__ void inv_det_vec4(const float* z, int64_t n, int64_t ld,
                                             float* zinv, float* __restrict__ det,
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

// Recomputes queued pixel p in FP64.  Its owning lane parked the input in the
// pixel's zinv slots (so zinv == z, in place, works too), ordered before this
// by a __syncwarp; the FP64 results overwrite it.
template <bool STAT>
__device__ __forceinline__ void recompute_queued(int64_t ld, int64_t p, float* zinv,
                                                 float* __restrict__ det,
                                                 uint8_t* __restrict__ status, uint32_t& c0) {
  float x[9], w[9], dt;
#pragma unroll
  for (int k = 0; k < 9; ++k) x[k] = __ldcg(zinv + k * ld + p);
  const uint32_t st = recompute_f64(x, w, dt);
#pragma unroll
  for (int k = 0; k < 9; ++k) __stcs(zinv + k * ld + p, w[k]);
  __stcs(det + p, dt);
  if (STAT) {
    if (status) status[p] = (uint8_t)st;
    c0 += st & ZINV_PIX_NOT_PD;
  }
}

// Recomputes the warp's queued pixels in whole rounds of 32, from the end of
// the queue; returns how many are left (< 32).  (Out of line it ran 3-4%
// slower on images with nothing flagged: the call's register saves.)
template <bool STAT>
__device__ __forceinline__ int flush_rounds(const int64_t* q, int qn, int ln, int64_t ld,
                                         float* zinv, float* det, uint8_t* status,
                                         uint32_t& c0) {
  __syncwarp();  // queue entries and the FP32 stores are visible to the warp
  do {
    qn -= 32;
    recompute_queued<STAT>(ld, q[qn + ln], zinv, det, status, c0);
  } while (qn >= 32);
  __syncwarp();  // the queue slots are read before the next step refills them
  return qn;
}

// Four-pixel kernel of the FP64 variants.  The loop is warp-uniform (lanes
// past the last group idle through a step), so ballots and __syncwarp see the
// whole warp.  For a flagged pixel the owning lane stores its input in place
// of the inverse and status RECOMPUTED; the lane that recomputes it stores the
// FP64 results, the status byte (with NOT_PD from the FP64 det) and counts
// NOT_PD.
template <int ALG, bool STAT>
__device__ __forceinline__ void inv_det_vec4_queued(const float* z, int64_t n,
                                                    int64_t ld, float* zinv,
                                                    float* __restrict__ det, float tau,
                                                    uint8_t* __restrict__ status,
                                                    unsigned long long* __restrict__ counts) {
  constexpr int BASE = kBaseAlg<ALG>;
  __shared__ int64_t queue[kThreads / 32][kQueue];
  int64_t* q = queue[threadIdx.x >> 5];
  const int ln = threadIdx.x & 31;
  const unsigned below = (1u << ln) - 1u;
  int qn = 0;  // warp-uniform
  const int64_t groups = n >> 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  uint32_t c0 = 0, c1 = 0;
  for (int64_t g0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); g0 < groups;
       g0 += stride) {
    const int64_t g = g0 + ln;
    uint32_t flags = 0;  // bit j: pixel 4g + j waits for the FP64 recompute
    if (g < groups) {
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
        uint32_t st = pixel_inv_det<BASE>(x, w, dt, tau);
        if (needs_recompute(dt, x, tau)) {
          flags |= 1u << j;
          st = ZINV_PIX_RECOMPUTED;
#pragma unroll
          for (int k = 0; k < 9; ++k) w[k] = x[k];
        }
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
    if (__any_sync(0xffffffffu, flags != 0u)) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const unsigned m = __ballot_sync(0xffffffffu, (flags >> j) & 1u);
        if ((flags >> j) & 1u) q[qn + __popc(m & below)] = 4 * g + j;
        qn += __popc(m);
      }
      if (qn >= 32) qn = flush_rounds<STAT>(q, qn, ln, ld, zinv, det, status, c0);
    }
  }
  if (qn > 0) {
    __syncwarp();
    if (ln < qn) recompute_queued<STAT>(ld, q[ln], zinv, det, status, c0);
  }
  // ragged tail: n % 4 pixels after the last full group, recomputed inline
  const int64_t p = (groups << 2) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.x == 0 && p < n) one_pixel<ALG, STAT>(z, ld, p, zinv, det, tau, status, c0, c1);
  if (STAT && counts) add_counts(counts, c0, c1);
}

template <int ALG, bool STAT>
__global__ void __launch_bounds__(kThreads)
    k_inv_det_vec4(const float* z, int64_t n, int64_t ld, float* zinv,
                   float* __restrict__ det, float tau, uint8_t* __restrict__ status,
                   unsigned long long* __restrict__ counts) {
  inv_det_vec4<ALG, STAT>(z, n, ld, zinv, det, tau, status, counts);
}

// FP64 recompute variants, held to three blocks per SM (their FP64 code would
// otherwise cost the FP32 streaming pass a block).
template <int ALG, bool STAT>
__global__ void __launch_bounds__(kThreads, 3)
    k_inv_det_vec4_f64(const float* z, int64_t n, int64_t ld,
                       float* zinv, float* __restrict__ det, float tau,
                       uint8_t* __restrict__ status, unsigned long long* __restrict__ counts) {
  inv_det_vec4_queued<ALG, STAT>(z, n, ld, zinv, det, tau, status, counts);
}

template <int ALG, bool STAT>
__global__ void __launch_bounds__(kThreads)
    k_inv_det_scalar(const float* z, int64_t n, int64_t ld, float* zinv,
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
    if constexpr (kHasF64<ALG>)
      k_inv_det_vec4_f64<ALG, STAT><<<blocks, kThreads, 0, s>>>(z, n, ld, zinv, det, tau,
                                                                status, counts);
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
