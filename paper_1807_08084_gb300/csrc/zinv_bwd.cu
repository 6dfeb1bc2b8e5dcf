// zinv_bwd.cu -- backward of the per-pixel (Z^-1, det, log det) w.r.t. the nine
// packed reals of Z, from the forward's saved W = Z^-1 and det:
//     M = -W G W + (g_det det + g_logdet) W,
//     g_z = [M00, 2Re M01, 2Im M01, 2Re M02, 2Im M02, M11, 2Re M12, 2Im M12, M22],
// with G the Hermitian matrix of the upstream packed gradient (off-diagonal
// entries halved, because each packed real stands for two entries of W).
// HBM-bound (up to 84 bytes in, 36 out per pixel); same SoA streaming scheme
// as the forward: four pixels per thread with 128-bit accesses.
#include "common.cuh"
#include "pixel.cuh"

namespace zinv {

namespace {
constexpr int kBwdThreads = 256;

struct cf {
  float r, i;
};
__device__ __forceinline__ cf cmul(cf a, cf b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__device__ __forceinline__ cf cj(cf a) { return {a.r, -a.i}; }
__device__ __forceinline__ cf cadd3(cf a, cf b, cf c) { return {a.r + b.r + c.r, a.i + b.i + c.i}; }

template <bool HG, bool HD, bool HL>
__device__ __forceinline__ void pixel_bwd(const float w[9], float det, const float g[9], float gd,
                                          float gl, float out[9]) {
  float s = 0.0f;
  if (HD) s = gd * det;
  if (HL) s += gl;
  float m[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) m[k] = s * w[k];
  if (HG) {
    const cf wa = {w[0], 0.f}, wb = {w[1], w[2]}, wc = {w[3], w[4]};
    const cf wd = {w[5], 0.f}, we = {w[6], w[7]}, wf = {w[8], 0.f};
    const cf ga = {g[0], 0.f}, gb = {0.5f * g[1], 0.5f * g[2]}, gc = {0.5f * g[3], 0.5f * g[4]};
    const cf gdd = {g[5], 0.f}, ge = {0.5f * g[6], 0.5f * g[7]}, gf = {g[8], 0.f};
    // P = W G
    const cf p00 = cadd3(cmul(wa, ga), cmul(wb, cj(gb)), cmul(wc, cj(gc)));
    const cf p01 = cadd3(cmul(wa, gb), cmul(wb, gdd), cmul(wc, cj(ge)));
    const cf p02 = cadd3(cmul(wa, gc), cmul(wb, ge), cmul(wc, gf));
    const cf p10 = cadd3(cmul(cj(wb), ga), cmul(wd, cj(gb)), cmul(we, cj(gc)));
    const cf p11 = cadd3(cmul(cj(wb), gb), cmul(wd, gdd), cmul(we, cj(ge)));
    const cf p12 = cadd3(cmul(cj(wb), gc), cmul(wd, ge), cmul(we, gf));
    const cf p20 = cadd3(cmul(cj(wc), ga), cmul(cj(we), cj(gb)), cmul(wf, cj(gc)));
    const cf p21 = cadd3(cmul(cj(wc), gb), cmul(cj(we), gdd), cmul(wf, cj(ge)));
    const cf p22 = cadd3(cmul(cj(wc), gc), cmul(cj(we), ge), cmul(wf, gf));
    // upper triangle of P W (Hermitian)
    const cf q00 = cadd3(cmul(p00, wa), cmul(p01, cj(wb)), cmul(p02, cj(wc)));
    const cf q01 = cadd3(cmul(p00, wb), cmul(p01, wd), cmul(p02, cj(we)));
    const cf q02 = cadd3(cmul(p00, wc), cmul(p01, we), cmul(p02, wf));
    const cf q11 = cadd3(cmul(p10, wb), cmul(p11, wd), cmul(p12, cj(we)));
    const cf q12 = cadd3(cmul(p10, wc), cmul(p11, we), cmul(p12, wf));
    const cf q22 = cadd3(cmul(p20, wc), cmul(p21, we), cmul(p22, wf));
    m[0] -= q00.r;
    m[1] -= q01.r;
    m[2] -= q01.i;
    m[3] -= q02.r;
    m[4] -= q02.i;
    m[5] -= q11.r;
    m[6] -= q12.r;
    m[7] -= q12.i;
    m[8] -= q22.r;
  }
  out[0] = m[0];
  out[1] = 2.0f * m[1];
  out[2] = 2.0f * m[2];
  out[3] = 2.0f * m[3];
  out[4] = 2.0f * m[4];
  out[5] = m[5];
  out[6] = 2.0f * m[6];
  out[7] = 2.0f * m[7];
  out[8] = m[8];
}

struct BwdArgs {
  const float* w;
  const float* det;
  const float* g;
  const float* gd;
  const float* gl;
  float* out;
  int64_t n, ld;
};

template <bool HG, bool HD, bool HL>
__device__ __forceinline__ void bwd_one(const BwdArgs& a, int64_t p) {
  float w[9], g[9], o[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) w[k] = __ldcs(a.w + k * a.ld + p);
  const float dt = HD ? __ldcs(a.det + p) : 0.f;
  if (HG) {
#pragma unroll
    for (int k = 0; k < 9; ++k) g[k] = __ldcs(a.g + k * a.ld + p);
  }
  const float gd = HD ? __ldcs(a.gd + p) : 0.f;
  const float gl = HL ? __ldcs(a.gl + p) : 0.f;
  pixel_bwd<HG, HD, HL>(w, dt, g, gd, gl, o);
#pragma unroll
  for (int k = 0; k < 9; ++k) __stcs(a.out + k * a.ld + p, o[k]);
}

template <bool HG, bool HD, bool HL>
__global__ void __launch_bounds__(kBwdThreads) k_bwd_vec4(BwdArgs a) {
  const int64_t groups = a.n >> 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < groups; q += stride) {
    float4 w[9], g[9], dt, gd, gl;
#pragma unroll
    for (int k = 0; k < 9; ++k) w[k] = __ldcs(reinterpret_cast<const float4*>(a.w + k * a.ld) + q);
    if (HD) dt = __ldcs(reinterpret_cast<const float4*>(a.det) + q);
    if (HG) {
#pragma unroll
      for (int k = 0; k < 9; ++k)
        g[k] = __ldcs(reinterpret_cast<const float4*>(a.g + k * a.ld) + q);
    }
    if (HD) gd = __ldcs(reinterpret_cast<const float4*>(a.gd) + q);
    if (HL) gl = __ldcs(reinterpret_cast<const float4*>(a.gl) + q);
    float4 o[9];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float wj[9], gj[9], oj[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        wj[k] = lane(w[k], j);
        gj[k] = HG ? lane(g[k], j) : 0.f;
      }
      pixel_bwd<HG, HD, HL>(wj, HD ? lane(dt, j) : 0.f, gj, HD ? lane(gd, j) : 0.f,
                            HL ? lane(gl, j) : 0.f, oj);
#pragma unroll
      for (int k = 0; k < 9; ++k) set_lane(o[k], j, oj[k]);
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) __stcs(reinterpret_cast<float4*>(a.out + k * a.ld) + q, o[k]);
  }
  const int64_t p = (groups << 2) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.x == 0 && p < a.n) bwd_one<HG, HD, HL>(a, p);
}

template <bool HG, bool HD, bool HL>
__global__ void __launch_bounds__(kBwdThreads) k_bwd_scalar(BwdArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.n; p += stride)
    bwd_one<HG, HD, HL>(a, p);
}

template <bool HG, bool HD, bool HL>
int launch_bwd(const BwdArgs& a, cudaStream_t s, int64_t min_blocks) {
  const bool vec = (a.ld % 4 == 0) && aligned(a.w, 16) && aligned(a.det, 16) &&
                   aligned(a.g, 16) && aligned(a.gd, 16) && aligned(a.gl, 16) &&
                   aligned(a.out, 16);
  if (vec) {
    auto k = k_bwd_vec4<HG, HD, HL>;
    const int64_t items = (a.n >> 2) > 0 ? (a.n >> 2) : 1;
    // With g_W given the kernel holds 128 registers (two blocks per SM); 32
    // groups per thread streamed 3.5% faster there than one (GB300 sweep).
    k<<<(unsigned)cover_blocks(items, kBwdThreads, HG ? 32 : 1, min_blocks), kBwdThreads, 0,
        s>>>(a);
  } else {
    auto k = k_bwd_scalar<HG, HD, HL>;
    k<<<(unsigned)cover_blocks(a.n, kBwdThreads), kBwdThreads, 0, s>>>(a);
  }
  return launch_status();
}
}  // namespace

}  // namespace zinv

extern "C" int zinv_det_bwd(const float* zinv, const float* det, int64_t n, int64_t ld,
                            const float* g_zinv, const float* g_det, const float* g_logdet,
                            float* g_z, void* stream) {
  using namespace zinv;
  if (n < 0 || ld < n || ld > kMaxLd) return ZINV_ERR_ARG;
  if (n > 0 && (!zinv || !g_z || (g_det && !det))) return ZINV_ERR_ARG;
  const void* ptrs[6] = {zinv, det, g_zinv, g_det, g_logdet, g_z};
  for (const void* p : ptrs)
    if (!aligned(p, 4)) return ZINV_ERR_ARG;
  DeviceInfo di;
  int rc = device_info(&di);
  if (rc != ZINV_OK) return rc;
  if (n == 0) return ZINV_OK;
  for (const void* p : ptrs)
    if (p && !device_accessible(p)) return ZINV_ERR_ARG;
  BwdArgs a{zinv, det, g_zinv, g_det, g_logdet, g_z, n, ld};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int key = (g_zinv ? 4 : 0) | (g_det ? 2 : 0) | (g_logdet ? 1 : 0);
  const int64_t mb = (int64_t)kMinBlocksPerSm * di.sm_count;
  switch (key) {
    case 0: return launch_bwd<false, false, false>(a, s, mb);
    case 1: return launch_bwd<false, false, true>(a, s, mb);
    case 2: return launch_bwd<false, true, false>(a, s, mb);
    case 3: return launch_bwd<false, true, true>(a, s, mb);
    case 4: return launch_bwd<true, false, false>(a, s, mb);
    case 5: return launch_bwd<true, false, true>(a, s, mb);
    case 6: return launch_bwd<true, true, false>(a, s, mb);
    default: return launch_bwd<true, true, true>(a, s, mb);
  }
}
