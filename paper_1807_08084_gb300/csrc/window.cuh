// window.cuh -- weighted window sums over tiles of single-look data, shared by
// the Wishart statistic (wishart.cu) and the weighted multilook (multilook.cu).
//
// A CTA of 64 threads covers a tile of 32 x 16 outputs; each thread owns a
// 4 x 2 block of them, so every input row it loads from shared memory feeds
// two output rows.  The tile's single-look block (tile plus an R-pixel halo,
// clamp-to-edge) is copied with cp.async into Sb; its nine channel products
// (the packed entries of s s^H) go to P in the channel-paired layout below;
// window_all_paired sums a (2R+1)^2 window of them for all nine channels, the
// input rows as the outer loop, with each output's taps added in row-major
// order, two channels per packed f32x2 FMA.  window_split is the same sums
// with two threads per 4 x 2 block (128 per tile), each on half the channels.
// (The Wishart backward keeps the scalar layout P [9][SH][SWP] and sums one
// channel at a time.)
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

// Issues, as one cp.async group, the copies of an image's single-look block of
// a tile plus halo (clamp-to-edge) into Sb [3][SH][SW]; s holds the three
// component planes of an H x W image, plane_ld apart.
template <int R, int NT = kWT>
__device__ __forceinline__ void issue_block(const float2* s, int64_t plane_ld, int64_t H,
                                            int64_t W, int64_t tile, float2* Sb) {
  using T = WTile<R>;
  const int64_t tiles_x = (W + kTW - 1) / kTW;
  const int64_t ty0 = (tile / tiles_x) * kTH, tx0 = (tile % tiles_x) * kTW;
  for (int i = threadIdx.x; i < T::SH * T::SW; i += NT) {
    const int r = i / T::SW, x = i - r * T::SW;
    const int64_t q = clampi(ty0 - R + r, H - 1) * W + clampi(tx0 - R + x, W - 1);
#pragma unroll
    for (int p = 0; p < 3; ++p) cp_async8(Sb + p * T::SH * T::SW + i, s + p * plane_ld + q);
  }
  cp_async_commit();
}

// Channel-paired products.  The window sums of window_all_paired run on
// packed f32x2 FMAs with a pair of channels per instruction: channels (0, 1),
// (2, 3), (4, 5) and (6, 7) are stored as float2 planes [SH][SWP] over the
// memory of the scalar planes 2j and 2j + 1, channel 8 as scalar plane 8.
// Within a row the 16-byte unit u (float2 columns 2u and 2u + 1) sits at unit
// u ^ ((u >> 3) & 1): the eight threads of a quarter-warp read units 2t + q
// (t = 0..7) of one row, which that spreads over the eight 16-byte bank groups
// for every q (with units in plain order, t and t + 4 would collide).
__device__ __forceinline__ int pcol(int x) { return x ^ ((x >> 3) & 2); }

// The nine channel products of the staged block Sb in the channel-paired layout.
template <int R, int NT = kWT>
__device__ __forceinline__ void block_products_paired(const float2* Sb, float* P) {
  using T = WTile<R>;
  float2* P2 = reinterpret_cast<float2*>(P);
  for (int i = threadIdx.x; i < T::SH * T::SW; i += NT) {
    const int r = i / T::SW, x = i - r * T::SW;
    float p[9];
    products(Sb[i], Sb[T::SH * T::SW + i], Sb[2 * T::SH * T::SW + i], p);
    const int o = r * T::SWP + pcol(x);
#pragma unroll
    for (int j = 0; j < 4; ++j) P2[j * T::PLANE + o] = make_float2(p[2 * j], p[2 * j + 1]);
    P[8 * T::PLANE + r * T::SWP + x] = p[8];
  }
}

// Copies the taps, each duplicated into both halves of a float2, into the
// shared table [L][WROW] of float2 (the packed FMAs' weight operand).
template <int R, int NT = kWT>
__device__ __forceinline__ void stage_taps_paired(const float* weights, float2* wsh2) {
  using T = WTile<R>;
  for (int k = threadIdx.x; k < T::K; k += NT) {
    const float w = weights[k];
    wsh2[(k / T::L) * T::WROW + k % T::L] = make_float2(w, w);
  }
}

// One input row of all nine channels for the thread's 4 x 2 outputs: the row
// y0 + iy feeds output row 0 with tap row iy (ROW0) and output row 1 with tap
// row iy - 1 (ROW1).  Channel pairs take one packed FMA per tap and output
// (each half rounded as a scalar fmaf, so the sums are the bits of the scalar
// loop), channel 8 a scalar one.  On GB300 a packed FMA completes no more
// FMAs per cycle than scalar ones, but it halves the instructions issued: the
// weighted 7 x 7 multilook ran 2.38 -> 2.00 ms with it.
template <int R, bool ROW0, bool ROW1>
__device__ __forceinline__ void row_step_paired(const float* P, const float2* wsh2, int iy,
                                                int y0, int x0, float2 (&zp)[4][2][4],
                                                float (&z8)[2][4]) {
  using T = WTile<R>;
  constexpr int L = T::L;
  constexpr int NU = 2 + R;  // 16-byte units of a row segment: 4 + 2R columns
  float2 w0[L + 1], w1[L + 1];
#pragma unroll
  for (int h = 0; h < (L + 1) / 2; ++h) {
    if (ROW0) {
      const float4 q = *reinterpret_cast<const float4*>(wsh2 + iy * T::WROW + 2 * h);
      w0[2 * h] = make_float2(q.x, q.y), w0[2 * h + 1] = make_float2(q.z, q.w);
    }
    if (ROW1) {
      const float4 q = *reinterpret_cast<const float4*>(wsh2 + (iy - 1) * T::WROW + 2 * h);
      w1[2 * h] = make_float2(q.x, q.y), w1[2 * h + 1] = make_float2(q.z, q.w);
    }
  }
  const float2* src = reinterpret_cast<const float2*>(P) + (y0 + iy) * T::SWP;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float2 row[2 * NU];
#pragma unroll
    for (int q = 0; q < NU; ++q) {
      const float4 v = *reinterpret_cast<const float4*>(src + j * T::PLANE + pcol(x0 + 2 * q));
      row[2 * q] = make_float2(v.x, v.y);
      row[2 * q + 1] = make_float2(v.z, v.w);
    }
#pragma unroll
    for (int dx = 0; dx < L; ++dx)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (ROW0) zp[j][0][i] = __ffma2_rn(w0[dx], row[i + dx], zp[j][0][i]);
        if (ROW1) zp[j][1][i] = __ffma2_rn(w1[dx], row[i + dx], zp[j][1][i]);
      }
  }
  float row[4 * T::NV];
  load_row<R>(P + 8 * T::PLANE + (y0 + iy) * T::SWP + x0, row);
#pragma unroll
  for (int dx = 0; dx < L; ++dx)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (ROW0) z8[0][i] = fmaf(w0[dx].x, row[i + dx], z8[0][i]);
      if (ROW1) z8[1][i] = fmaf(w1[dx].x, row[i + dx], z8[1][i]);
    }
}

// Window sums of all nine channels for the thread's 4 x 2 outputs from one
// date's staged products P (channel-paired layout): the L + 1 input rows in
// order, the first and last feeding one output row each.  Per output the taps
// are added in row-major order.  ROW_UNROLL: middle rows per loop iteration
// (the Wishart forward takes 2, 2.6% faster at 7 x 7; the weighted multilook
// 1, which the unroll did not help).
template <int R, int ROW_UNROLL = 1>
__device__ __forceinline__ void window_all_paired(const float* P, const float2* wsh2, int y0,
                                                  int x0, float (&z)[9][2][4]) {
  constexpr int L = WTile<R>::L;
  float2 zp[4][2][4];
  float z8[2][4];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
      for (int j = 0; j < 4; ++j) zp[j][r][i] = make_float2(0.0f, 0.0f);
      z8[r][i] = 0.0f;
    }
  row_step_paired<R, true, false>(P, wsh2, 0, y0, x0, zp, z8);
#pragma unroll ROW_UNROLL
  for (int iy = 1; iy < L; ++iy) row_step_paired<R, true, true>(P, wsh2, iy, y0, x0, zp, z8);
  row_step_paired<R, false, true>(P, wsh2, L, y0, x0, zp, z8);
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        z[2 * j][r][i] = zp[j][r][i].x;
        z[2 * j + 1][r][i] = zp[j][r][i].y;
      }
      z[8][r][i] = z8[r][i];
    }
}

// ---------------------------------------------------------------------------
// Channel-split engine: two threads per 4 x 2 block of outputs, 128 per tile.
// Lanes l and l ^ 8 of a warp share a block; half h = (l >> 3) & 1 sums
// channel pairs 2h and 2h + 1 for both output rows and channel 8 for output
// row h alone, so both halves issue the same FMAs (per tap: 16 packed ones,
// two channel pairs for eight outputs, and 4 scalar ones, channel 8 for four
// outputs), and each quarter-warp reads one plane, as in the paired engine.  Every accumulator adds its taps in the same order as the
// paired engine: the sums are the same bits.  After the sums the halves swap
// the pairs of the other's row with one shuffle each, so half h holds all nine
// channels of row h.  Twice the threads on the same shared memory doubles the
// warps per SM.
constexpr int kWS = 2 * kWT;  // threads per CTA of the split engine

struct Split {
  int h;       // channel pairs 2h, 2h + 1; channel 8 and the inverses of output row h
  int y0, x0;  // the block: output rows y0, y0 + 1, columns x0 .. x0 + 3
};

__device__ __forceinline__ Split split_of(int t) {
  const int lane = t & 31;
  const int b = 16 * (t >> 5) + (lane & 7) + 8 * (lane >> 4);  // block 0..63
  return {(lane >> 3) & 1, 2 * (b / kTX), 4 * (b % kTX)};
}

// One input row for a half block: row y0 + iy feeds output row 0 with tap row
// iy (ROW0) and output row 1 with tap row iy - 1 (ROW1), as row_step_paired.
template <int R, bool ROW0, bool ROW1>
__device__ __forceinline__ void row_step_split(const float* P, const float2* wsh2, int iy,
                                               const Split& sp, float2 (&zp)[2][2][4],
                                               float (&z8)[4]) {
  using T = WTile<R>;
  constexpr int L = T::L;
  constexpr int NU = 2 + R;
  float2 w0[L + 1], w1[L + 1];
#pragma unroll
  for (int h = 0; h < (L + 1) / 2; ++h) {
    if (ROW0) {
      const float4 q = *reinterpret_cast<const float4*>(wsh2 + iy * T::WROW + 2 * h);
      w0[2 * h] = make_float2(q.x, q.y), w0[2 * h + 1] = make_float2(q.z, q.w);
    }
    if (ROW1) {
      const float4 q = *reinterpret_cast<const float4*>(wsh2 + (iy - 1) * T::WROW + 2 * h);
      w1[2 * h] = make_float2(q.x, q.y), w1[2 * h + 1] = make_float2(q.z, q.w);
    }
  }
  const float2* src =
      reinterpret_cast<const float2*>(P) + 2 * sp.h * T::PLANE + (sp.y0 + iy) * T::SWP;
#pragma unroll
  for (int jj = 0; jj < 2; ++jj) {
    float2 row[2 * NU];
#pragma unroll
    for (int q = 0; q < NU; ++q) {
      const float4 v =
          *reinterpret_cast<const float4*>(src + jj * T::PLANE + pcol(sp.x0 + 2 * q));
      row[2 * q] = make_float2(v.x, v.y);
      row[2 * q + 1] = make_float2(v.z, v.w);
    }
#pragma unroll
    for (int dx = 0; dx < L; ++dx)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (ROW0) zp[jj][0][i] = __ffma2_rn(w0[dx], row[i + dx], zp[jj][0][i]);
        if (ROW1) zp[jj][1][i] = __ffma2_rn(w1[dx], row[i + dx], zp[jj][1][i]);
      }
  }
  // channel 8 of output row h: tap row iy - h; the first input row feeds only
  // row 0, the last only row 1
  if ((ROW0 && ROW1) || (ROW0 ? sp.h == 0 : sp.h == 1)) {
    float row[4 * T::NV];
    load_row<R>(P + 8 * T::PLANE + (sp.y0 + iy) * T::SWP + sp.x0, row);
#pragma unroll
    for (int dx = 0; dx < L; ++dx) {
      const float w = (ROW0 && ROW1) ? (sp.h ? w1[dx].x : w0[dx].x) : (ROW0 ? w0[dx].x : w1[dx].x);
#pragma unroll
      for (int i = 0; i < 4; ++i) z8[i] = fmaf(w, row[i + dx], z8[i]);
    }
  }
}

// Window sums of all nine channels for output row y0 + h of the half block's
// 4 x 2 outputs (z[c][i]: channel c, column x0 + i).  Every lane of the warp
// must call it (the exchange is a full-warp shuffle).
template <int R, int ROW_UNROLL = 1>
__device__ __forceinline__ void window_split(const float* P, const float2* wsh2, const Split& sp,
                                             float (&z)[9][4]) {
  constexpr int L = WTile<R>::L;
  float2 zp[2][2][4];
  float z8[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) zp[jj][0][i] = zp[jj][1][i] = make_float2(0.0f, 0.0f);
    z8[i] = 0.0f;
  }
  row_step_split<R, true, false>(P, wsh2, 0, sp, zp, z8);
#pragma unroll ROW_UNROLL
  for (int iy = 1; iy < L; ++iy) row_step_split<R, true, true>(P, wsh2, iy, sp, zp, z8);
  row_step_split<R, false, true>(P, wsh2, L, sp, zp, z8);
  // half h keeps its pairs of row h and gives its pairs of the other row; it
  // receives the partner's pairs of row h
#pragma unroll
  for (int jj = 0; jj < 2; ++jj)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 keep = sp.h ? zp[jj][1][i] : zp[jj][0][i];
      const float2 give = sp.h ? zp[jj][0][i] : zp[jj][1][i];
      const float2 got = make_float2(__shfl_xor_sync(0xffffffffu, give.x, 8),
                                     __shfl_xor_sync(0xffffffffu, give.y, 8));
      const float2 lo = sp.h ? got : keep;  // pair jj: channels 2 jj, 2 jj + 1
      const float2 hi = sp.h ? keep : got;  // pair 2 + jj: channels 4 + 2 jj, 5 + 2 jj
      z[2 * jj][i] = lo.x;
      z[2 * jj + 1][i] = lo.y;
      z[4 + 2 * jj][i] = hi.x;
      z[5 + 2 * jj][i] = hi.y;
    }
#pragma unroll
  for (int i = 0; i < 4; ++i) z[8][i] = z8[i];
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
