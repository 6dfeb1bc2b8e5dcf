// multilook.cu -- fused multilook + inverse + determinant.
//
// Per output pixel p the window covariance Z(p) = (1/N) sum_{k in win} s s^H
// (Eq. ZN, boxcar, N = win^2) or sum_k w_k s s^H (weighted window) is formed in
// shared memory and registers from the single-look vectors s, then inverted by
// Algorithm 2 (same per-pixel code and flags as zinv_det).  Z never reaches HBM:
// 24 B are read and 40 B written per pixel.
//
// Boxcar: each CTA walks one strip segment (kTW columns x kSeg rows) down
// the image in steps of kCH output rows.  Per step:
//   - cp.async copies of the step's raw input rows (three planes, the r-column
//     halo, clamp-to-edge rows; 16-byte copies inside the image, clamped 8-byte
//     copies on border strips) were issued two steps earlier into a
//     three-deep ring of raw buffers, so two steps of loads are always in
//     flight behind the arithmetic;
//   - phase H: the nine channel products |s0|^2, Re/Im s0 conj s1, Re/Im s0
//     conj s2, |s1|^2, Re/Im s1 conj s2, |s2|^2 of the 4 + 2r inputs of four
//     adjacent outputs and their horizontal window sums, into a ring of
//     kCH + 2r rows (128-bit stores);
//   - phase V: vertical window sums over the ring (four rows per thread), scale
//     by 1/N, invert, store (warp-contiguous along x).
// Each input row is loaded once per strip (plus 2r rows at a segment start and
// 2r halo columns): ~1.1x the ideal read traffic.  Phase H reads the raw rows
// and writes the ring in whole 16-byte units, and both store their units
// swizzled (unit u at u ^ ((u >> 3) & 1)), so neither access has bank
// conflicts (8-byte reads of two rows per half-warp replayed 2-way, and so did
// the unswizzled 16-byte ring stores: 0.861 -> 0.821 ms at 7 x 7).
//
// Weighted windows (general taps, not separable) of 3 x 3, 5 x 5 and 7 x 7 run
// on the window engines of window.cuh (32 x 16 output tiles, 4 x 2 blocks of
// outputs, two channels per packed FMA, cp.async staging of the next tile
// behind the window sums; at 7 x 7 two threads share a block, splitting its
// channels); each thread then inverts its outputs from registers and stores
// four adjacent outputs of a plane with one 128-bit store.
// Other odd windows up to 15 x 15 use a simpler tiled kernel.
#include "async.cuh"
#include "common.cuh"
#include "pixel.cuh"
#include "window.cuh"

namespace zinv {

namespace {

constexpr int kMlThreads = 256;
constexpr int kTW = 64;  // output tile width
constexpr int kTH = 16;  // output tile height

struct MlArgs {
  const float2* s;
  int64_t H, W, plane_ld;
  float* zinv;
  float* det;
  float tau;
  uint8_t* status;
  unsigned long long* counts;
  const float* weights;  // device, win*win, or null (boxcar)
  int win;
};

__device__ __forceinline__ int64_t clamp64(int64_t v, int64_t hi) {
  return v < 0 ? 0 : (v > hi ? hi : v);
}

// The nine channels of s s^H in packed order: a, Re b, Im b, Re c, Im c, d,
// Re e, Im e, f with b = s0 conj s1, c = s0 conj s2, e = s1 conj s2.
__device__ __forceinline__ void channels(float2 s0, float2 s1, float2 s2, float p[9]) {
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

__device__ __forceinline__ float vadd(float a, float b) { return a + b; }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }

// Sums of L = 2R+1 consecutive values for four adjacent outputs:
// out[j] = v[j] + ... + v[j+L-1], j = 0..3, sharing the common middle.
// float2 sums two channels at once with Blackwell's packed FP32 adds.
template <int R, typename V>
__device__ __forceinline__ void window4v(const V* v, V out[4]) {
  constexpr int L = 2 * R + 1;
  if constexpr (L == 3) {
    const V a = vadd(v[1], v[2]), b = vadd(v[3], v[4]);
    out[0] = vadd(v[0], a);
    out[1] = vadd(a, v[3]);
    out[2] = vadd(v[2], b);
    out[3] = vadd(b, v[5]);
  } else {
    V core = v[3];
#pragma unroll
    for (int k = 4; k < L; ++k) core = vadd(core, v[k]);
    const V a = vadd(v[1], v[2]), b = vadd(v[L], v[L + 1]);
    out[0] = vadd(core, vadd(v[0], a));
    out[1] = vadd(core, vadd(a, v[L]));
    out[2] = vadd(core, vadd(v[2], b));
    out[3] = vadd(core, vadd(b, v[L + 2]));
  }
}

template <int R>
__device__ __forceinline__ void window4(const float* v, float out[4]) {
  constexpr int L = 2 * R + 1;
  if constexpr (L == 3) {
    const float a = v[1] + v[2], b = v[3] + v[4];
    out[0] = v[0] + a;
    out[1] = a + v[3];
    out[2] = v[2] + b;
    out[3] = b + v[5];
  } else {
    float core = v[3];
#pragma unroll
    for (int k = 4; k < L; ++k) core += v[k];
    const float a = v[1] + v[2], b = v[L] + v[L + 1];
    out[0] = core + (v[0] + a);
    out[1] = core + (a + v[L]);
    out[2] = core + (v[2] + b);
    out[3] = core + (b + v[L + 2]);
  }
}

template <int ALG, bool STAT>
__device__ __forceinline__ void finish_pixel(const MlArgs& a, int64_t gy, int64_t gx, float z[9],
                                             uint32_t& c0, uint32_t& c1) {
  const int64_t n = a.H * a.W;
  const int64_t p = gy * a.W + gx;
  float w[9], dt;
  const uint32_t st = pixel_inv_det<ALG>(z, w, dt, a.tau);
#pragma unroll
  for (int k = 0; k < 9; ++k) __stcs(a.zinv + k * n + p, w[k]);
  __stcs(a.det + p, dt);
  if (STAT) {
    if (a.status) a.status[p] = (uint8_t)st;
    c0 += st & ZINV_PIX_NOT_PD;
    c1 += (st & ZINV_PIX_RECOMPUTED) >> 1;
  }
}

// Phase 1, shared by the boxcar and the weighted kernels.  Each thread first
// issues the loads of all its staged pixels (one memory round trip per tile),
// then forms their products and writes them to shared memory.
template <int R, int SH, int SWP, int SW>
__device__ __forceinline__ void stage_products(const MlArgs& a, int64_t ty0, int64_t tx0,
                                               float* P) {
  constexpr int KMAX = (SH * SW + kMlThreads - 1) / kMlThreads;
  float2 v[KMAX][3];
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    const int i = threadIdx.x + k * kMlThreads;
    if (i < SH * SW) {
      const int iy = i / SW, ix = i - (i / SW) * SW;
      const int64_t gy = clamp64(ty0 - R + iy, a.H - 1);
      const int64_t gx = clamp64(tx0 - R + ix, a.W - 1);
      const int64_t q = gy * a.W + gx;
      v[k][0] = __ldg(a.s + q);
      v[k][1] = __ldg(a.s + a.plane_ld + q);
      v[k][2] = __ldg(a.s + 2 * a.plane_ld + q);
    }
  }
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    const int i = threadIdx.x + k * kMlThreads;
    if (i < SH * SW) {
      const int iy = i / SW, ix = i - (i / SW) * SW;
      float p[9];
      channels(v[k][0], v[k][1], v[k][2], p);
#pragma unroll
      for (int c = 0; c < 9; ++c) P[(c * SH + iy) * SWP + ix] = p[c];
    }
  }
}

// ---------------------------------------------------------------------------
// Boxcar strip walker
// ---------------------------------------------------------------------------
constexpr int kSThreads = 128;
constexpr int kCH = 8;       // output rows per step
constexpr int kSeg = 256;    // rows per strip segment
constexpr int kStages = 3;   // raw-row buffers in flight
constexpr int kRawW = kTW + 8;  // raw columns x0-4 .. x0+67 (covers r <= 4), 16-byte aligned
// Row stride of the raw buffers, in float2: one 16-byte unit more than the
// copied columns, so consecutive rows start one bank group apart (37 units,
// odd).  Phase H gives a half-warp 8 column groups of two rows, and the 16
// lanes' 8-byte reads of input k then fall into 8 distinct bank groups (2-way
// instead of 4-way conflicts).
constexpr int kRawS = kRawW + 2;
static_assert(kCH % 2 == 0, "phase H pairs rows");

// 16-byte units (two float2 columns) of a raw row and of a ring row are
// stored swizzled, unit u at u ^ ((u >> 3) & 1): the eight lanes of a
// quarter-warp then touch eight distinct bank groups in phase H's 128-bit
// reads of the raw rows and 128-bit stores to the ring.
__device__ __forceinline__ int swu(int u) { return u ^ ((u >> 3) & 1); }
__device__ __forceinline__ int swcol(int c) { return 2 * swu(c >> 1) + (c & 1); }

template <int R>
struct Strip {
  static_assert(R <= 4, "raw rows cover a halo of at most 4");
  static constexpr int RING = kCH + 2 * R;                      // rows of horizontal sums
  static constexpr size_t stage_f2 = 3 * kCH * kRawS;           // float2 per raw buffer
  // horizontal sums: float2 [4][RING][kTW] (channel pairs) then float [RING][kTW]
  static constexpr size_t ring_f = 9 * RING * kTW;
  static constexpr size_t smem = kStages * stage_f2 * sizeof(float2) + ring_f * sizeof(float);
};

// Issues the asynchronous copies of `rows` input rows (relative rows rr0 ..,
// absolute y_begin - R + rr, clamped) of the three planes, columns x0-4 ..
// x0+67, into raw buffer `buf`: 16-byte copies inside the image, 8-byte copies
// with clamped columns on strips that touch the left or right border.
template <int R, int ROWS, bool VEC16>
__device__ __forceinline__ void issue_rows_t(const MlArgs& a, float2* buf, int64_t y_begin,
                                             int64_t x0, int rr0) {
  constexpr int nch = VEC16 ? kRawW / 2 : kRawW;  // copies per plane-row
  constexpr int n = 3 * ROWS * nch;
#pragma unroll 2
  for (int e = threadIdx.x; e < n; e += kSThreads) {
    const int pr = e / nch, ch = e - (e / nch) * nch;
    const int p = pr / ROWS, r = pr - p * ROWS;
    const int64_t gy = clamp64(y_begin - R + rr0 + r, a.H - 1);
    const float2* row = a.s + p * a.plane_ld + gy * a.W;
    float2* dst = buf + (p * kCH + r) * kRawS;
    if (VEC16)
      cp_async16(dst + 2 * swu(ch), row + (x0 - 4) + 2 * ch);
    else
      cp_async8(dst + swcol(ch), row + clamp64(x0 - 4 + ch, a.W - 1));
  }
}

template <int R>
__device__ __forceinline__ void issue_rows(const MlArgs& a, float2* buf, int64_t y_begin,
                                           int64_t x0, int rr0, int rows, bool vec16) {
  if (rows == kCH) {
    if (vec16) issue_rows_t<R, kCH, true>(a, buf, y_begin, x0, rr0);
    else issue_rows_t<R, kCH, false>(a, buf, y_begin, x0, rr0);
  } else {
    if (vec16) issue_rows_t<R, 2 * R, true>(a, buf, y_begin, x0, rr0);
    else issue_rows_t<R, 2 * R, false>(a, buf, y_begin, x0, rr0);
  }
}

template <int R, int ALG, bool STAT>
__global__ void __launch_bounds__(kSThreads, 3) k_multilook_strip(MlArgs a) {
  using T = Strip<R>;
  extern __shared__ __align__(16) float smem[];
  float2* raw = reinterpret_cast<float2*>(smem);
  float2* ring2 = reinterpret_cast<float2*>(smem + 2 * kStages * T::stage_f2);
  float* ring1 = smem + 2 * kStages * T::stage_f2 + 8 * T::RING * kTW;
  const int64_t strips_x = (a.W + kTW - 1) / kTW;
  const int64_t segs = (a.H + kSeg - 1) / kSeg;
  const int64_t units = strips_x * segs;
  const float invN = 1.0f / (float)((2 * R + 1) * (2 * R + 1));
  const bool aligned16 = ((a.W & 1) == 0) && ((a.plane_ld & 1) == 0) &&
                         ((reinterpret_cast<uintptr_t>(a.s) & 15) == 0);
  uint32_t c0 = 0, c1 = 0;
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int64_t x0 = (u % strips_x) * kTW;
    const int64_t y_begin = (u / strips_x) * kSeg;
    const int64_t y_end = (y_begin + kSeg < a.H) ? y_begin + kSeg : a.H;
    const int out_rows = (int)(y_end - y_begin);
    const bool vec16 = aligned16 && x0 >= 4 && x0 + kTW + 4 <= a.W;
    // job 0: input rows 0 .. 2R-1 (relative to y_begin - R), no output;
    // job j >= 1: input rows 2R + (j-1) kCH .. + kCH, output rows (j-1) kCH .. + kCH.
    const int jobs = 1 + (out_rows + kCH - 1) / kCH;
    __syncthreads();  // the previous unit is done with the raw buffers and the ring
    for (int j = 0; j < kStages - 1; ++j) {
      if (j < jobs)
        issue_rows<R>(a, raw + j * T::stage_f2, y_begin, x0, j == 0 ? 0 : 2 * R + (j - 1) * kCH,
                      j == 0 ? 2 * R : kCH, vec16);
      cp_async_commit();
    }
    for (int j = 0; j < jobs; ++j) {
      const int jn = j + kStages - 1;  // the job whose copies start now
      if (jn < jobs)
        issue_rows<R>(a, raw + (jn % kStages) * T::stage_f2, y_begin, x0, 2 * R + (jn - 1) * kCH,
                      kCH, vec16);
      cp_async_commit();
      cp_async_wait<kStages - 1>();  // this thread's copies of job j have landed
      __syncthreads();               // everyone's have
      const int rr0 = j == 0 ? 0 : 2 * R + (j - 1) * kCH;
      const int rows = j == 0 ? 2 * R : kCH;
      const float2* rb = raw + (j % kStages) * T::stage_f2;
      // phase H: products of 4 + 2R pixels and horizontal sums of four adjacent
      // outputs per work item, rows of this job -> ring
      for (int i = threadIdx.x; i < rows * (kTW / 4); i += kSThreads) {
        // items in groups of 16: rows 2 (g / 2) and 2 (g / 2) + 1, column
        // groups 8 (g % 2) .. + 7 (rows is even: kCH or 2R)
        const int g = i >> 4, sub = i & 15;
        const int r = 2 * (g >> 1) + (sub >> 3), xr = 4 * (8 * (g & 1) + (sub & 7));
        // raw columns xr + 4 - R .. of the run's inputs, read as whole 16-byte
        // units from unit u0 on; input k is value k + O of the units read
        constexpr int O = (4 - R) & 1;
        constexpr int NU = (O + 4 + 2 * R + 1) / 2;
        const int u0 = (xr + 4 - R) >> 1;
        float2 sv[3][2 * NU];
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
          for (int q = 0; q < NU; ++q) {
            const float4 v =
                *reinterpret_cast<const float4*>(rb + (p * kCH + r) * kRawS + 2 * swu(u0 + q));
            sv[p][2 * q] = make_float2(v.x, v.y);
            sv[p][2 * q + 1] = make_float2(v.z, v.w);
          }
        float2 pv2[4][4 + 2 * R];
        float pv8[4 + 2 * R];
#pragma unroll
        for (int k = 0; k < 4 + 2 * R; ++k) {
          const float2 s0 = sv[0][k + O];
          const float2 s1 = sv[1][k + O];
          const float2 s2 = sv[2][k + O];
          float pp[9];
          channels(s0, s1, s2, pp);
          pv2[0][k] = make_float2(pp[0], pp[5]);
          pv2[1][k] = make_float2(pp[1], pp[2]);
          pv2[2][k] = make_float2(pp[3], pp[4]);
          pv2[3][k] = make_float2(pp[6], pp[7]);
          pv8[k] = pp[8];
        }
        const int slot = (rr0 + r) % T::RING;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float2 o[4];
          window4v<R>(pv2[q], o);
          float2* rowp = ring2 + (q * T::RING + slot) * kTW;
          *reinterpret_cast<float4*>(rowp + 2 * swu(xr >> 1)) =
              make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
          *reinterpret_cast<float4*>(rowp + 2 * swu((xr >> 1) + 1)) =
              make_float4(o[2].x, o[2].y, o[3].x, o[3].y);
        }
        float o8[4];
        window4v<R>(pv8, o8);
        *reinterpret_cast<float4*>(ring1 + slot * kTW + xr) = make_float4(o8[0], o8[1], o8[2], o8[3]);
      }
      __syncthreads();
      if (j == 0) continue;
      // phase V: output rows (j-1) kCH .. of this job
      const int oy0 = (j - 1) * kCH;
      const int orows = (out_rows - oy0) < kCH ? (out_rows - oy0) : kCH;
      for (int i = threadIdx.x; i < kTW * ((orows + 3) / 4); i += kSThreads) {
        const int x = i % kTW, yq = (i / kTW) * 4;
        int off[4 + 2 * R];  // ring row offsets of the rows this item reads
        {
          int slot = (oy0 + yq) % T::RING;
#pragma unroll
          for (int k = 0; k < 4 + 2 * R; ++k) {
            off[k] = slot * kTW;
            slot = (slot + 1 == T::RING) ? 0 : slot + 1;
          }
        }
        const int xp = swcol(x);  // the float2 column's place in a swizzled ring row
        float z[4][9];
        const float2 inv2 = make_float2(invN, invN);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float2 w[4 + 2 * R];
#pragma unroll
          for (int k = 0; k < 4 + 2 * R; ++k) w[k] = ring2[q * T::RING * kTW + off[k] + xp];
          float2 o[4];
          window4v<R>(w, o);
          constexpr int lo[4] = {0, 1, 3, 6}, hi[4] = {5, 2, 4, 7};
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const float2 zz = __fmul2_rn(o[m], inv2);
            z[m][lo[q]] = zz.x;
            z[m][hi[q]] = zz.y;
          }
        }
        {
          float w[4 + 2 * R];
#pragma unroll
          for (int k = 0; k < 4 + 2 * R; ++k) w[k] = ring1[off[k] + x];
          float o[4];
          window4v<R>(w, o);
#pragma unroll
          for (int m = 0; m < 4; ++m) z[m][8] = o[m] * invN;
        }
        const int64_t gx = x0 + x;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int oy = oy0 + yq + q;
          if (oy < out_rows && gx < a.W) finish_pixel<ALG, STAT>(a, y_begin + oy, gx, z[q], c0, c1);
        }
      }
    }
  }
  cp_async_wait<0>();
  if (STAT && a.counts) add_counts(a.counts, c0, c1);
}

// Weighted (or any odd window up to kMaxWin) covariance: Z(p) = sum_k w_k P(p+k),
// one output per work item over all taps.  Weights in shared memory.
constexpr int kMaxWin = 15;
constexpr int kWR = (kMaxWin - 1) / 2;
constexpr int kWSH = kTH + 2 * kWR, kWSW = kTW + 2 * kWR, kWSWP = (kWSW + 3) / 4 * 4;
constexpr size_t kWSmem = (9 * kWSH * kWSWP + kMaxWin * kMaxWin) * sizeof(float);

template <int ALG, bool STAT>
__global__ void __launch_bounds__(kMlThreads) k_multilook_weighted(MlArgs a) {
  extern __shared__ __align__(16) float smem[];
  float* P = smem;
  float* wsh = smem + 9 * kWSH * kWSWP;
  const int r = (a.win - 1) / 2;
  for (int i = threadIdx.x; i < a.win * a.win; i += blockDim.x) wsh[i] = a.weights[i];
  const int64_t tiles_x = (a.W + kTW - 1) / kTW;
  const int64_t tiles = tiles_x * ((a.H + kTH - 1) / kTH);
  uint32_t c0 = 0, c1 = 0;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int64_t ty0 = (t / tiles_x) * kTH, tx0 = (t % tiles_x) * kTW;
    // stage with the maximal halo; taps only reach r <= kWR of it
    stage_products<kWR, kWSH, kWSWP, kWSW>(a, ty0, tx0, P);
    __syncthreads();
    for (int i = threadIdx.x; i < kTW * kTH; i += blockDim.x) {
      const int x = i % kTW, y = i / kTW;
      float z[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) z[c] = 0.0f;
      for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx) {
          const float wk = wsh[(dy + r) * a.win + (dx + r)];
          const int iy = y + kWR + dy, ix = x + kWR + dx;
#pragma unroll
          for (int c = 0; c < 9; ++c) z[c] = fmaf(wk, P[(c * kWSH + iy) * kWSWP + ix], z[c]);
        }
      const int64_t gy = ty0 + y, gx = tx0 + x;
      if (gy < a.H && gx < a.W) finish_pixel<ALG, STAT>(a, gy, gx, z, c0, c1);
    }
    __syncthreads();
  }
  if (STAT && a.counts) add_counts(a.counts, c0, c1);
}

// Weighted windows of 2R + 1 (R = 1..3) on the window engines of window.cuh.
// 7 x 7 runs the channel-split engine (128 threads per 32 x 16 tile, two per
// 4 x 2 block: twice the warps per SM on the same shared memory, 4% faster;
// its input-row loop unrolled by two, 3% more);
// 3 x 3 and 5 x 5 the paired engine (64 threads), which the split made 9% and
// 1% slower, having too few taps to hide its exchange and its duplicated
// channel-8 loads.
__host__ __device__ constexpr bool uses_split(int r) { return r == 3; }
__host__ __device__ constexpr int window_threads(int r) {
  return uses_split(r) ? win::kWS : win::kWT;
}
// Four CTAs per SM; the split engine's FP64-recompute routes need more than
// its 128 registers and take three (a few bytes of spills, 24% faster than two).
__host__ __device__ constexpr int window_min_blocks(int r, int alg) {
  return uses_split(r) && (alg == kPlainF64 || alg == kCompF64) ? 3 : 4;
}

// Per tile: the staged single-look block's products, the window sums in
// registers (each output's taps in row-major order, as the simpler kernel adds
// them), then each thread inverts its outputs with Algorithm 2 -- both rows of
// its 4 x 2 block (paired engine) or row h of it (split engine) -- and writes
// four adjacent outputs of a plane with one 128-bit store (parking Z in shared
// memory for a warp per row of 32 outputs took 6% longer).
template <int R, int ALG, bool STAT>
__global__ void __launch_bounds__(window_threads(R), window_min_blocks(R, ALG))
    k_multilook_window(MlArgs a) {
  using T = win::WTile<R>;
  constexpr bool SPLIT = uses_split(R);
  constexpr int NT = window_threads(R);
  constexpr int ROWS = SPLIT ? 1 : 2;  // output rows a thread inverts
  extern __shared__ __align__(16) float smem[];
  float* P = smem;  // the tile's channel-paired products
  float2* Sb = reinterpret_cast<float2*>(smem + T::P_FLOATS);  // next single-look block
  float2* wsh2 = reinterpret_cast<float2*>(Sb + T::S_F2);      // duplicated taps [L][WROW]
  const int64_t tiles_x = (a.W + win::kTW - 1) / win::kTW;
  const int64_t tiles = tiles_x * ((a.H + win::kTH - 1) / win::kTH);
  win::Split sp;
  if (SPLIT) {
    sp = win::split_of(threadIdx.x);
  } else {
    sp = {0, 2 * ((int)threadIdx.x / win::kTX), 4 * ((int)threadIdx.x % win::kTX)};
  }
  uint32_t c0 = 0, c1 = 0;
  const bool vec = (a.W & 3) == 0 && (reinterpret_cast<uintptr_t>(a.zinv) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(a.det) & 15) == 0;
  const int64_t n = a.H * a.W;
  win::stage_taps_paired<R, NT>(a.weights, wsh2);
  if ((int64_t)blockIdx.x < tiles)
    win::issue_block<R, NT>(a.s, a.plane_ld, a.H, a.W, blockIdx.x, Sb);
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t ty0 = (tile / tiles_x) * win::kTH, tx0 = (tile % tiles_x) * win::kTW;
    cp_async_wait<0>();
    __syncthreads();  // the block is in Sb; the last tile's window sums are done with P
    win::block_products_paired<R, NT>(Sb, P);
    __syncthreads();  // Sb is free; P holds the products
    const int64_t next = tile + gridDim.x;
    if (next < tiles) win::issue_block<R, NT>(a.s, a.plane_ld, a.H, a.W, next, Sb);
    float z[9][ROWS][4];
    if constexpr (SPLIT) {
      float zr[9][4];
      win::window_split<R, 2>(P, wsh2, sp, zr);
#pragma unroll
      for (int c = 0; c < 9; ++c)
#pragma unroll
        for (int i = 0; i < 4; ++i) z[c][0][i] = zr[c][i];
    } else {
      win::window_all_paired<R>(P, wsh2, sp.y0, sp.x0, z);
    }
    const int64_t gx = tx0 + sp.x0;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      const int64_t gy = ty0 + sp.y0 + (SPLIT ? sp.h : r);
      float4 wv[9], dv;
      uint32_t stv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float zz[9], w[9], dt;
#pragma unroll
        for (int c = 0; c < 9; ++c) zz[c] = z[c][r][i];
        stv[i] = pixel_inv_det<ALG>(zz, w, dt, a.tau);
#pragma unroll
        for (int c = 0; c < 9; ++c) set_lane(wv[c], i, w[c]);
        set_lane(dv, i, dt);
      }
      if (gy >= a.H) continue;
      const int64_t p = gy * a.W + gx;
      if (vec && gx + 4 <= a.W) {
#pragma unroll
        for (int c = 0; c < 9; ++c) __stcs(reinterpret_cast<float4*>(a.zinv + c * n + p), wv[c]);
        __stcs(reinterpret_cast<float4*>(a.det + p), dv);
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (gx + i >= a.W) continue;
#pragma unroll
          for (int c = 0; c < 9; ++c) __stcs(a.zinv + c * n + p + i, lane(wv[c], i));
          __stcs(a.det + p + i, lane(dv, i));
        }
      }
      if (STAT) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (gx + i >= a.W) continue;
          if (a.status) a.status[p + i] = (uint8_t)stv[i];
          c0 += stv[i] & ZINV_PIX_NOT_PD;
          c1 += (stv[i] & ZINV_PIX_RECOMPUTED) >> 1;
        }
      }
    }
  }
  cp_async_wait<0>();
  if (STAT && a.counts) add_counts(a.counts, c0, c1);
}

template <int R>
constexpr size_t window_smem() {
  using T = win::WTile<R>;
  return T::P_FLOATS * sizeof(float) + (T::L * T::WROW + T::S_F2) * sizeof(float2);
}

template <typename K>
int launch_window(K kernel, size_t smem, int threads, const MlArgs& a, cudaStream_t s) {
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return ZINV_ERR_LAUNCH;
  }
  const int64_t tiles = ((a.W + win::kTW - 1) / win::kTW) * ((a.H + win::kTH - 1) / win::kTH);
  const int64_t blocks = cover_blocks(tiles * threads, threads);
  kernel<<<(unsigned)blocks, threads, smem, s>>>(a);
  return launch_status();
}

template <typename K>
int launch_ml(K kernel, size_t smem, const MlArgs& a, cudaStream_t s) {
  static_assert(sizeof(K) > 0, "");
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return ZINV_ERR_LAUNCH;
  }
  const int64_t tiles = ((a.W + kTW - 1) / kTW) * ((a.H + kTH - 1) / kTH);
  const int64_t blocks = cover_blocks(tiles * kMlThreads, kMlThreads);
  kernel<<<(unsigned)blocks, kMlThreads, smem, s>>>(a);
  return launch_status();
}

template <typename K>
int launch_strip(K kernel, size_t smem, const MlArgs& a, cudaStream_t s) {
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return ZINV_ERR_LAUNCH;
  }
  const int64_t units = ((a.W + kTW - 1) / kTW) * ((a.H + kSeg - 1) / kSeg);
  const int64_t blocks = cover_blocks(units * kSThreads, kSThreads);
  kernel<<<(unsigned)blocks, kSThreads, smem, s>>>(a);
  return launch_status();
}

template <int ALG, bool STAT>
int dispatch_ml(const MlArgs& a, cudaStream_t s) {
  if (a.weights) {
    switch (a.win) {
      case 3: return launch_window(k_multilook_window<1, ALG, STAT>, window_smem<1>(),
                                   window_threads(1), a, s);
      case 5: return launch_window(k_multilook_window<2, ALG, STAT>, window_smem<2>(),
                                   window_threads(2), a, s);
      case 7: return launch_window(k_multilook_window<3, ALG, STAT>, window_smem<3>(),
                                   window_threads(3), a, s);
    }
    return launch_ml(k_multilook_weighted<ALG, STAT>, kWSmem, a, s);
  }
  switch (a.win) {
    case 3: return launch_strip(k_multilook_strip<1, ALG, STAT>, Strip<1>::smem, a, s);
    case 5: return launch_strip(k_multilook_strip<2, ALG, STAT>, Strip<2>::smem, a, s);
    case 7: return launch_strip(k_multilook_strip<3, ALG, STAT>, Strip<3>::smem, a, s);
  }
  return ZINV_ERR_ARG;
}

template <int ALG>
int dispatch_ml_stat(const MlArgs& a, cudaStream_t s) {
  if (a.status || a.counts) return dispatch_ml<ALG, true>(a, s);
  return dispatch_ml<ALG, false>(a, s);
}

}  // namespace

int alg_from_flags(uint32_t flags);

}  // namespace zinv

extern "C" int multilook_zinv_det(const float* s, int64_t H, int64_t W, int64_t plane_ld,
                                  int win, const float* weights, float* zinv, float* det,
                                  uint32_t flags, float tau, uint8_t* status, int64_t* counts,
                                  void* stream) {
  using namespace zinv;
  const int alg = alg_from_flags(flags);
  if (alg < 0 || H < 0 || W < 0 || (W > 0 && H > kMaxLd / W)) return ZINV_ERR_ARG;
  if (!(tau >= 0.0f) || isinf(tau)) return ZINV_ERR_ARG;
  if (plane_ld < H * W || plane_ld > kMaxLd) return ZINV_ERR_ARG;
  if (weights ? (win < 1 || win > kMaxWin || win % 2 == 0) : (win != 3 && win != 5 && win != 7))
    return ZINV_ERR_ARG;
  const int64_t n = H * W;
  if (n > 0 && (!s || !zinv || !det)) return ZINV_ERR_ARG;
  if (!aligned(s, 8) || !aligned(zinv, 4) || !aligned(det, 4) || !aligned(counts, 8) ||
      !aligned(weights, 4))
    return ZINV_ERR_ARG;
  DeviceInfo di;
  int rc = device_info(&di);
  if (rc != ZINV_OK) return rc;
  if (n > 0 && (!device_accessible(s) || !device_accessible(zinv) || !device_accessible(det)))
    return ZINV_ERR_ARG;
  if ((weights && !device_accessible(weights)) || (status && !device_accessible(status)) ||
      (counts && !device_accessible(counts)))
    return ZINV_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  auto* cnt = reinterpret_cast<unsigned long long*>(counts);
  if (cnt && cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), st) != cudaSuccess)
    return ZINV_ERR_LAUNCH;
  if (n == 0) return ZINV_OK;
  MlArgs a{reinterpret_cast<const float2*>(s), H, W, plane_ld, zinv, det, tau, status, cnt,
           weights, win};
  switch (alg) {
    case kPlain: return dispatch_ml_stat<kPlain>(a, st);
    case kComp: return dispatch_ml_stat<kComp>(a, st);
    case kPlainF64: return dispatch_ml_stat<kPlainF64>(a, st);
    case kCompF64: return dispatch_ml_stat<kCompF64>(a, st);
  }
  return ZINV_ERR_ARG;
}
