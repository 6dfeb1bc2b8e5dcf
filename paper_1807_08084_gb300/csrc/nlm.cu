// nlm.cu -- nonlocal-means filter of a packed covariance image with the Wishart
// equal-looks distance (the paper's motivating workload, §1: for every pixel,
// a 23 x 23 search window of determinants of 3x3 Hermitian matrices).
//
// For pixels i, j:  d(i, j) = ln det((Z_i + Z_j)/2) - (ln det Z_i + ln det Z_j)/2,
// w_ij = exp(-L d(i, j) / h) over the in-image neighbours within the search
// radius, and Z'_i = sum_j w_ij Z_j / sum_j w_ij.
//
// The per-pixel log-dets are formed once per staged pixel (compensated route);
// the per-pair determinant -- 529 per pixel for a 23 x 23 window -- is the hot
// arithmetic.  It is computed either by Algorithm 2's cofactor expansion
// (Eq. adjoint_elements, Eq. detr: no division, no square root) or by
// Algorithm 1's Cholesky route (three square roots, two reciprocals), so the
// two can be compared where arithmetic, not memory, sets the time.
//
// Tiles of 32 x 8 outputs, one thread per output; the tile plus a halo of the
// search radius (Z and its log-det) sits in shared memory, rows warp-contiguous.
#include "common.cuh"
#include "pixel.cuh"

namespace zinv {
namespace {

constexpr int kNT = 256;
constexpr int kNW = 32;  // tile width
constexpr int kNH = 8;   // tile height

struct NlmArgs {
  const float* z;
  int64_t H, W, ld;
  int radius;
  float c;  // -L / (h ln 2): w = 2^(c d)
  float* out;
};

// det by Algorithm 1's factorization: (l00 l11 l22)^2 with l00 = sqrt(a), the
// first column scaled by 1/l00, l11 = sqrt(d - |l10|^2), l21 scaled by 1/l11,
// l22 = sqrt(f - |l20|^2 - |l21|^2) (correctly rounded sqrt and reciprocal).
__device__ __forceinline__ float det_cholesky(const float x[9]) {
  const float a = x[0], br = x[1], bi = x[2], cr = x[3], ci = x[4];
  const float d = x[5], er = x[6], ei = x[7], f = x[8];
  const float l00 = __fsqrt_rn(a);
  const float v0 = __frcp_rn(l00);
  const float l10r = br * v0, l10i = -bi * v0;
  const float l20r = cr * v0, l20i = -ci * v0;
  const float l11 = __fsqrt_rn(d - (l10r * l10r + l10i * l10i));
  const float v1 = __frcp_rn(l11);
  const float l21r = (er - (l20r * l10r + l20i * l10i)) * v1;
  const float l21i = (-ei - (l20i * l10r - l20r * l10i)) * v1;
  const float l22 = __fsqrt_rn(f - (l20r * l20r + l20i * l20i) - (l21r * l21r + l21i * l21i));
  const float p = l00 * l11 * l22;
  return p * p;
}

template <int METHOD, int RAD>
__global__ void __launch_bounds__(kNT) k_nlm(NlmArgs a) {
  constexpr int SW = kNW + 2 * RAD, SH = kNH + 2 * RAD;
  extern __shared__ __align__(16) float smem[];
  float* Zs = smem;                   // [9][SH][SW]
  float* Ls = smem + 9 * SH * SW;     // [SH][SW] log-dets
  const int64_t n = a.H * a.W;
  const int64_t tiles_x = (a.W + kNW - 1) / kNW;
  const int64_t tiles = tiles_x * ((a.H + kNH - 1) / kNH);
  const int tx = threadIdx.x % kNW, ty = threadIdx.x / kNW;
  const float three_ln2 = 2.0794415416798357f;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int64_t y0 = (t / tiles_x) * kNH, x0 = (t % tiles_x) * kNW;
    __syncthreads();
    for (int i = threadIdx.x; i < SH * SW; i += kNT) {
      const int sy = i / SW, sx = i - (i / SW) * SW;
      const int64_t gy = y0 - RAD + sy, gx = x0 - RAD + sx;
      if (gy < 0 || gy >= a.H || gx < 0 || gx >= a.W) continue;  // never read
      const int64_t p = gy * a.W + gx;
      float v[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        v[c] = __ldg(a.z + c * a.ld + p);
        Zs[(c * SH + sy) * SW + sx] = v[c];
      }
      const dd<float> dt = det_comp<float>(v);
      Ls[sy * SW + sx] = logf(dt.hi) + dt.lo / dt.hi;
    }
    __syncthreads();
    const int64_t gy = y0 + ty, gx = x0 + tx;
    if (gy >= a.H || gx >= a.W) continue;
    const int cy = ty + RAD, cx = tx + RAD;
    float zi[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) zi[c] = Zs[(c * SH + cy) * SW + cx];
    const float li = Ls[cy * SW + cx];
    // in-image part of the search window
    const int dy0 = (int)(gy - RAD < 0 ? -gy : -RAD);
    const int dy1 = (int)(gy + RAD >= a.H ? a.H - 1 - gy : RAD);
    const int dx0 = (int)(gx - RAD < 0 ? -gx : -RAD);
    const int dx1 = (int)(gx + RAD >= a.W ? a.W - 1 - gx : RAD);
    float out[9], wsum;
    if constexpr (METHOD == 0) {
      // Algorithm 2: neighbours two at a time (dx, dx + 1); the sums, the pair
      // determinants and the weighted accumulation run on packed float2 pairs
      // (f32x2, each half rounded as the scalar operation), the logs and exp2s
      // stay scalar; even and odd neighbours accumulate in the two halves.
      float2 zi2[9], acc[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        zi2[c] = make_float2(zi[c], zi[c]);
        acc[c] = make_float2(0.0f, 0.0f);
      }
      float2 ws = make_float2(0.0f, 0.0f);
      for (int dy = dy0; dy <= dy1; ++dy) {
        const int row = cy + dy;
        const float* lrow = Ls + row * SW + cx;
        int dx = dx0;
        for (; dx < dx1; dx += 2) {
          const int col = cx + dx;
          float2 zj[9], zs[9];
#pragma unroll
          for (int c = 0; c < 9; ++c) {
            const float* q = Zs + (c * SH + row) * SW + col;
            zj[c] = make_float2(q[0], q[1]);
            zs[c] = add_rn(zi2[c], zj[c]);
          }
          const float2 det = det_adjugate<float2>(zs);
          // ln det((Zi+Zj)/2) = ln det(Zi+Zj) - 3 ln 2
          const float d0 = (logf(det.x) - three_ln2) - 0.5f * (li + lrow[dx]);
          const float d1 = (logf(det.y) - three_ln2) - 0.5f * (li + lrow[dx + 1]);
          const float2 w =
              make_float2(exp2f(a.c * fmaxf(d0, 0.0f)), exp2f(a.c * fmaxf(d1, 0.0f)));
#pragma unroll
          for (int c = 0; c < 9; ++c) acc[c] = fma_rn(w, zj[c], acc[c]);
          ws = add_rn(ws, w);
        }
        if (dx == dx1) {  // an odd count leaves one neighbour: the first halves
          const int col = cx + dx;
          float zj[9], zs[9];
#pragma unroll
          for (int c = 0; c < 9; ++c) {
            zj[c] = Zs[(c * SH + row) * SW + col];
            zs[c] = add_rn(zi[c], zj[c]);
          }
          const float det = det_adjugate<float>(zs);
          const float d0 = (logf(det) - three_ln2) - 0.5f * (li + lrow[dx]);
          const float w = exp2f(a.c * fmaxf(d0, 0.0f));
#pragma unroll
          for (int c = 0; c < 9; ++c) acc[c].x = fmaf(w, zj[c], acc[c].x);
          ws.x += w;
        }
      }
#pragma unroll
      for (int c = 0; c < 9; ++c) out[c] = acc[c].x + acc[c].y;
      wsum = ws.x + ws.y;
    } else {
      // Algorithm 1: one neighbour at a time (pairing its scalar square roots
      // and reciprocals only cost it registers)
#pragma unroll
      for (int c = 0; c < 9; ++c) out[c] = 0.0f;
      wsum = 0.0f;
      for (int dy = dy0; dy <= dy1; ++dy) {
        const int row = cy + dy;
        for (int dx = dx0; dx <= dx1; ++dx) {
          const int col = cx + dx;
          float zj[9], zs[9];
#pragma unroll
          for (int c = 0; c < 9; ++c) {
            zj[c] = Zs[(c * SH + row) * SW + col];
            zs[c] = zi[c] + zj[c];
          }
          const float det = det_cholesky(zs);
          // ln det((Zi+Zj)/2) = ln det(Zi+Zj) - 3 ln 2
          const float dist = (logf(det) - three_ln2) - 0.5f * (li + Ls[row * SW + col]);
          const float w = exp2f(a.c * fmaxf(dist, 0.0f));
#pragma unroll
          for (int c = 0; c < 9; ++c) out[c] = fmaf(w, zj[c], out[c]);
          wsum += w;
        }
      }
    }
    const float inv = 1.0f / wsum;
    const int64_t p = gy * a.W + gx;
#pragma unroll
    for (int c = 0; c < 9; ++c) a.out[c * n + p] = out[c] * inv;
  }
}

template <int METHOD, int RAD>
int launch_nlm(const NlmArgs& a, cudaStream_t s) {
  constexpr int SW = kNW + 2 * RAD, SH = kNH + 2 * RAD;
  const size_t smem = (size_t)10 * SH * SW * sizeof(float);
  auto k = k_nlm<METHOD, RAD>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return ZINV_ERR_LAUNCH;
  }
  const int64_t tiles = ((a.W + kNW - 1) / kNW) * ((a.H + kNH - 1) / kNH);
  const int64_t blocks = cover_blocks(tiles * kNT, kNT);
  k<<<(unsigned)blocks, kNT, smem, s>>>(a);
  return launch_status();
}

template <int METHOD>
int dispatch_nlm(const NlmArgs& a, cudaStream_t s) {
  switch (a.radius) {
    case 1: return launch_nlm<METHOD, 1>(a, s);
    case 2: return launch_nlm<METHOD, 2>(a, s);
    case 3: return launch_nlm<METHOD, 3>(a, s);
    case 5: return launch_nlm<METHOD, 5>(a, s);
    case 7: return launch_nlm<METHOD, 7>(a, s);
    case 11: return launch_nlm<METHOD, 11>(a, s);
    case 15: return launch_nlm<METHOD, 15>(a, s);
  }
  return ZINV_ERR_ARG;
}

}  // namespace
}  // namespace zinv

extern "C" int nlm_wishart(const float* z, int64_t H, int64_t W, int64_t ld, int radius,
                           float looks, float h, int method, float* z_out, void* stream) {
  using namespace zinv;
  if (H < 1 || W < 1 || H > kMaxLd / W || ld < H * W || ld > kMaxLd) return ZINV_ERR_ARG;
  if (radius != 1 && radius != 2 && radius != 3 && radius != 5 && radius != 7 &&
      radius != 11 && radius != 15)
    return ZINV_ERR_ARG;
  if (!(looks > 0.0f) || !(h > 0.0f) || isinf(looks) || isinf(h)) return ZINV_ERR_ARG;
  if (method != 0 && method != 1) return ZINV_ERR_ARG;
  if (!z || !z_out || !aligned(z, 4) || !aligned(z_out, 4)) return ZINV_ERR_ARG;
  DeviceInfo di;
  int rc = device_info(&di);
  if (rc != ZINV_OK) return rc;
  if (!device_accessible(z) || !device_accessible(z_out)) return ZINV_ERR_ARG;
  NlmArgs a{z, H, W, ld, radius, -looks / (h * 0.69314718055994531f), z_out};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return method == 0 ? dispatch_nlm<0>(a, s) : dispatch_nlm<1>(a, s);
}
