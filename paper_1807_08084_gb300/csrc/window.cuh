// window.cuh -- weighted window sums over tiles of single-look data, shared by
// the Wishart statistic (wishart.cu) and the weighted multilook (multilook.cu).
//
// A CTA of 64 threads covers a tile of 32 x 16 outputs; each thread owns a
// 4 x 2 block of them, so every input row it loads from shared memory feeds
// two output rows.  The tile's single-look block (tile plus an R-pixel halo,
// clamp-to-edge) is copied with cp.async into Sb; its nine channel products
// (the packed entries of s s^H) go to P [9][SH][SWP]; window_all sums a
// (2R+1)^2 window of them for all nine channels, the input rows as the outer
// loop, with each output's taps added in row-major order.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "async.cuh"

namespace zinv {
namespace win {

constexpr int kWT = 64;       // threads per CTA (two warps)
constexpr int kTW = 32;       // tile width (outputs)
constexpr int kTH = 16;       // tile height (outputs)
constexpr int kTX = kTW / 4;  // threads across a tile row (4 outputs each)
static_assert(kTX * (kTH / 2) == kWT, "each thread owns a 4 x 2 block of outputs");

template <int R>
struct WTile {
  static constexpr int L = 2 * R + 1;
  static constexpr int K = L * L;
  static constexpr int SH = kTH + 2 * R;
  static constexpr int SW = kTW + 2 * R;
  static constexpr int SWP = (SW + 3) / 4 * 4;
  static constexpr int NV = (4 + 2 * R + 3) / 4;            // float4 loads per row segment
  static constexpr int KO = (SH * SW + kWT - 1) / kWT;     // staged pixels per thread
  static constexpr int PLANE = SH * SWP;                   // one channel's products
  static constexpr int P_FLOATS = 9 * PLANE;               // one date's products
  static constexpr int Z_FLOATS = 9 * kTH * kTW;           // one date's Z
  static_assert(P_FLOATS >= Z_FLOATS, "a date's Z fits in place of its products");
  static constexpr int WROW = 8;                           // tap rows padded for 128-bit loads
  static constexpr int S_F2 = 3 * SH * SW;                 // one date's single-look block (float2)
  static_assert(P_FLOATS % 4 == 0 && S_F2 % 2 == 0, "16-byte aligned regions");
};

__device__ __forceinline__ int64_t clampi(int64_t v, int64_t hi) {
  return v < 0 ? 0 : (v > hi ? hi : v);
}

__device__ __forceinline__ void products(float2 s0, float2 s1, float2 s2, float p[9]) {
  p[0] = s0.x * s0.x + s0.y * s0.y;
  p[1] = s0.x * s1.x + s0.y * s1.y;
  p[2] = s0.y * s1.x - s0.x * s1.y;
  p[3] = s0.x * s2.x + s0.y * s2.y;
  p[4] = s0.y * s2.x - s0.x * s2.y;
  p[5] = s1.x * s1.x + s1.y * s1.y;
  p[6] = s1.x * s2.x + s1.y * s2.y;
  p[7] = s1.y * s2.x - s1.x * s2.y;
  p[8] = s2.x * s2.x + s2.y * s2.y;
}

template <int R>
__device__ __forceinline__ void load_row(const float* src, float (&row)[4 * WTile<R>::NV]) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int q = 0; q < WTile<R>::NV; ++q) {
    const float4 v = s4[q];
    row[4 * q] = v.x;
    row[4 * q + 1] = v.y;
    row[4 * q + 2] = v.z;
    row[4 * q + 3] = v.w;
  }
}

// One input row of all nine channels for the thread's 4 x 2 outputs: the row
// y0 + iy feeds output row 0 with tap row iy (ROW0) and output row 1 with tap
// row iy - 1 (ROW1).  Taps come from the shared table wsh [L][WROW].
template <int R, bool ROW0, bool ROW1>
__device__ __forceinline__ void row_step(const float* P, const float* wsh, int iy, int y0,
                                         int x0, float (&z)[9][2][4]) {
  using T = WTile<R>;
  constexpr int L = T::L;
  float w0[2 * 4], w1[2 * 4];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (ROW0) {
      const float4 q = *reinterpret_cast<const float4*>(wsh + iy * T::WROW + 4 * h);
      w0[4 * h] = q.x, w0[4 * h + 1] = q.y, w0[4 * h + 2] = q.z, w0[4 * h + 3] = q.w;
    }
    if (ROW1) {
      const float4 q = *reinterpret_cast<const float4*>(wsh + (iy - 1) * T::WROW + 4 * h);
      w1[4 * h] = q.x, w1[4 * h + 1] = q.y, w1[4 * h + 2] = q.z, w1[4 * h + 3] = q.w;
    }
  }
  const float* src = P + (y0 + iy) * T::SWP + x0;
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    float row[4 * T::NV];
    load_row<R>(src + c * T::PLANE, row);
#pragma unroll
    for (int dx = 0; dx < L; ++dx)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (ROW0) z[c][0][i] = fmaf(w0[dx], row[i + dx], z[c][0][i]);
        if (ROW1) z[c][1][i] = fmaf(w1[dx], row[i + dx], z[c][1][i]);
      }
  }
}

// Window sums of all nine channels for the thread's 4 x 2 outputs from one
// date's staged products P: the L + 1 input rows in order, the first and last
// feeding one output row each.  Per output the taps are added in row-major
// order, as in window_4x2.
template <int R>
__device__ __forceinline__ void window_all(const float* P, const float* wsh, int y0, int x0,
                                           float (&z)[9][2][4]) {
  constexpr int L = WTile<R>::L;
#pragma unroll
  for (int c = 0; c < 9; ++c)
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int i = 0; i < 4; ++i) z[c][r][i] = 0.0f;
  row_step<R, true, false>(P, wsh, 0, y0, x0, z);
#pragma unroll 1
  for (int iy = 1; iy < L; ++iy) row_step<R, true, true>(P, wsh, iy, y0, x0, z);
  row_step<R, false, true>(P, wsh, L, y0, x0, z);
}

// Copies the taps into the shared table [L][WROW] (pad entries unused).
template <int R>
__device__ __forceinline__ void stage_taps(const float* weights, float* wsh) {
  using T = WTile<R>;
  for (int k = threadIdx.x; k < T::K; k += kWT) wsh[(k / T::L) * T::WROW + k % T::L] = weights[k];
}

// Issues, as one cp.async group, the copies of an image's single-look block of
// a tile plus halo (clamp-to-edge) into Sb [3][SH][SW]; s holds the three
// component planes of an H x W image, plane_ld apart.
template <int R>
__device__ __forceinline__ void issue_block(const float2* s, int64_t plane_ld, int64_t H,
                                            int64_t W, int64_t tile, float2* Sb) {
  using T = WTile<R>;
  const int64_t tiles_x = (W + kTW - 1) / kTW;
  const int64_t ty0 = (tile / tiles_x) * kTH, tx0 = (tile % tiles_x) * kTW;
  for (int i = threadIdx.x; i < T::SH * T::SW; i += kWT) {
    const int r = i / T::SW, x = i - r * T::SW;
    const int64_t q = clampi(ty0 - R + r, H - 1) * W + clampi(tx0 - R + x, W - 1);
#pragma unroll
    for (int p = 0; p < 3; ++p) cp_async8(Sb + p * T::SH * T::SW + i, s + p * plane_ld + q);
  }
  cp_async_commit();
}

// The nine channel products of the staged block Sb -> P[c][SH][SWP].
template <int R>
__device__ __forceinline__ void block_products(const float2* Sb, float* P) {
  using T = WTile<R>;
  for (int i = threadIdx.x; i < T::SH * T::SW; i += kWT) {
    const int r = i / T::SW, x = i - r * T::SW;
    float p[9];
    products(Sb[i], Sb[T::SH * T::SW + i], Sb[2 * T::SH * T::SW + i], p);
#pragma unroll
    for (int c = 0; c < 9; ++c) P[c * T::PLANE + r * T::SWP + x] = p[c];
  }
}

// Stores the thread's 4 x 2 block of one channel into a [kTH][kTW] plane.
__device__ __forceinline__ void store_block(float* Zc, int y0, int x0, const float (&z)[2][4]) {
#pragma unroll
  for (int r = 0; r < 2; ++r)
    *reinterpret_cast<float4*>(Zc + (y0 + r) * kTW + x0) =
        make_float4(z[r][0], z[r][1], z[r][2], z[r][3]);
}

}  // namespace win
}  // namespace zinv
