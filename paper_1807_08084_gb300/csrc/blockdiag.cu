// blockdiag.cu -- multifrequency PolSAR pixels (§5 of the paper): each pixel's
// matrix is block diagonal with nb Hermitian 3x3 blocks (one per band), so its
// inverse is the block-diagonal matrix of the blocks' inverses and its
// determinant the product of theirs; Algorithm 2 runs on each block.
//
// Same streaming scheme as zinv_det: four pixels per thread with 128-bit
// accesses per plane, the blocks of a pixel group processed one after another
// by the same thread so the det product stays in registers.
#include "common.cuh"
#include "pixel.cuh"

namespace zinv {
namespace {

constexpr int kBT = 256;
constexpr int kMaxBlocks = 8;

struct BdArgs {
  const float* z;
  float* zinv;
  float* det;
  uint8_t* status;
  unsigned long long* counts;
  int64_t n, ld;
  int nb;
  float tau;
};

template <int ALG, bool STAT>
__device__ __forceinline__ void bd_pixel(const BdArgs& a, int64_t p, uint32_t& c0, uint32_t& c1) {
  float dprod = 1.0f;
  uint32_t st = 0;
  for (int b = 0; b < a.nb; ++b) {
    const float* zb = a.z + (int64_t)b * 9 * a.ld;
    float* wb = a.zinv + (int64_t)b * 9 * a.ld;
    float x[9], w[9], dt;
#pragma unroll
    for (int k = 0; k < 9; ++k) x[k] = __ldcs(zb + k * a.ld + p);
    st |= pixel_inv_det<ALG>(x, w, dt, a.tau);
#pragma unroll
    for (int k = 0; k < 9; ++k) __stcs(wb + k * a.ld + p, w[k]);
    dprod *= dt;
  }
  __stcs(a.det + p, dprod);
  if (STAT) {
    if (a.status) a.status[p] = (uint8_t)st;
    c0 += st & ZINV_PIX_NOT_PD;
    c1 += (st & ZINV_PIX_RECOMPUTED) >> 1;
  }
}

template <int ALG, bool STAT>
__global__ void __launch_bounds__(kBT) k_blockdiag_vec4(BdArgs a) {
  const int64_t groups = a.n >> 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  uint32_t c0 = 0, c1 = 0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += stride) {
    float4 dprod = make_float4(1.f, 1.f, 1.f, 1.f);
    uint32_t sv = 0;
    for (int b = 0; b < a.nb; ++b) {
      const float* zb = a.z + (int64_t)b * 9 * a.ld;
      float* wb = a.zinv + (int64_t)b * 9 * a.ld;
      float4 v[9], o[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) v[k] = __ldcs(reinterpret_cast<const float4*>(zb + k * a.ld) + g);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float x[9], w[9], dt;
#pragma unroll
        for (int k = 0; k < 9; ++k) x[k] = lane(v[k], j);
        const uint32_t st = pixel_inv_det<ALG>(x, w, dt, a.tau);
#pragma unroll
        for (int k = 0; k < 9; ++k) set_lane(o[k], j, w[k]);
        set_lane(dprod, j, lane(dprod, j) * dt);
        if (STAT) sv |= st << (8 * j);
      }
#pragma unroll
      for (int k = 0; k < 9; ++k) __stcs(reinterpret_cast<float4*>(wb + k * a.ld) + g, o[k]);
    }
    __stcs(reinterpret_cast<float4*>(a.det) + g, dprod);
    if (STAT) {
      if (a.status) reinterpret_cast<uint32_t*>(a.status)[g] = sv;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t st = (sv >> (8 * j)) & 0xffu;
        c0 += st & ZINV_PIX_NOT_PD;
        c1 += (st & ZINV_PIX_RECOMPUTED) >> 1;
      }
    }
  }
  const int64_t p = (groups << 2) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.x == 0 && p < a.n) bd_pixel<ALG, STAT>(a, p, c0, c1);
  if (STAT && a.counts) add_counts(a.counts, c0, c1);
}

template <int ALG, bool STAT>
__global__ void __launch_bounds__(kBT) k_blockdiag_scalar(BdArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  uint32_t c0 = 0, c1 = 0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.n; p += stride)
    bd_pixel<ALG, STAT>(a, p, c0, c1);
  if (STAT && a.counts) add_counts(a.counts, c0, c1);
}

template <int ALG, bool STAT>
int launch_bd(const BdArgs& a, cudaStream_t s) {
  const bool vec = (a.ld % 4 == 0) && aligned(a.z, 16) && aligned(a.zinv, 16) &&
                   aligned(a.det, 16) && (a.status == nullptr || aligned(a.status, 4));
  if (vec) {
    auto k = k_blockdiag_vec4<ALG, STAT>;
    const int64_t items = (a.n >> 2) > 0 ? (a.n >> 2) : 1;
    k<<<(unsigned)cover_blocks(items, kBT), kBT, 0, s>>>(a);
  } else {
    auto k = k_blockdiag_scalar<ALG, STAT>;
    k<<<(unsigned)cover_blocks(a.n, kBT), kBT, 0, s>>>(a);
  }
  return launch_status();
}

template <int ALG>
int dispatch_bd(const BdArgs& a, cudaStream_t s) {
  if (a.status || a.counts) return launch_bd<ALG, true>(a, s);
  return launch_bd<ALG, false>(a, s);
}

}  // namespace

int alg_from_flags(uint32_t flags);

}  // namespace zinv

extern "C" int zinv_det_blockdiag(const float* z, int nblocks, int64_t n, int64_t ld, float* zinv,
                                  float* det, uint32_t flags, float tau, uint8_t* status,
                                  int64_t* counts, void* stream) {
  using namespace zinv;
  const int alg = alg_from_flags(flags);
  if (alg < 0 || nblocks < 1 || nblocks > kMaxBlocks) return ZINV_ERR_ARG;
  if (n < 0 || ld < n || ld > kMaxLd / (9 * nblocks)) return ZINV_ERR_ARG;
  if (!(tau >= 0.0f) || isinf(tau)) return ZINV_ERR_ARG;
  if (n > 0 && (!z || !zinv || !det)) return ZINV_ERR_ARG;
  if (!aligned(z, 4) || !aligned(zinv, 4) || !aligned(det, 4) || !aligned(counts, 8))
    return ZINV_ERR_ARG;
  DeviceInfo di;
  int rc = device_info(&di);
  if (rc != ZINV_OK) return rc;
  if (n > 0 && (!device_accessible(z) || !device_accessible(zinv) || !device_accessible(det)))
    return ZINV_ERR_ARG;
  if ((status && !device_accessible(status)) || (counts && !device_accessible(counts)))
    return ZINV_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto* cnt = reinterpret_cast<unsigned long long*>(counts);
  if (cnt && cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), s) != cudaSuccess)
    return ZINV_ERR_LAUNCH;
  if (n == 0) return ZINV_OK;
  BdArgs a{z, zinv, det, status, cnt, n, ld, nblocks, tau};
  switch (alg) {
    case kPlain: return dispatch_bd<kPlain>(a, s);
    case kComp: return dispatch_bd<kComp>(a, s);
    case kPlainF64: return dispatch_bd<kPlainF64>(a, s);
    case kCompF64: return dispatch_bd<kCompF64>(a, s);
  }
  return ZINV_ERR_ARG;
}
