// wishart.cu -- differentiable Wishart change statistic between two dates with a
// learnable window (the likelihood-ratio change test the paper cites, §1).
//
// Per pixel p and date t, Z_t(p) = sum_k w_k S_t(p+k) S_t(p+k)^H over a win x win
// window (clamp-to-edge), and
//     q(p) = ln det Z1 + ln det Z2 - 2 ln det((Z1 + Z2)/2)  (<= 0, = 0 iff Z1 = Z2),
//     L    = sum_p q(p).
// Backward (recomputes Z from the single-look vectors, nothing is stored):
//     dq = tr(M1 dZ1) + tr(M2 dZ2),  M_t = Z_t^-1 - 2 (Z1 + Z2)^-1,
//     dL/dw_k = sum_p sum_t S_t(p+k)^H M_t(p) S_t(p+k)
//             = sum_p sum_t sum_c G_t[c](p) P_t[c](p+k),
// with P the nine channel products of S S^H and G the packed form of M (off-
// diagonal entries doubled).  Determinants and inverses use the compensated
// route of Algorithm 2 (Dot2), so the log-dets keep FP32 accuracy: on scenes
// with strongly correlated channels det / (a d f) falls to a few 10^-3, where
// the plain expansion loses most of its digits.
//
// Tiles of 32 x 16 outputs in blocks of 4 x 2 outputs, so each input row a
// thread loads from shared memory feeds both output rows of its block
// (2 x 4 x win FMAs per loaded row).  One date's channel products for the tile
// and its halo sit in shared memory at a time.
//   Forward: each date's single-look block is copied with cp.async while the
//   other date's window sums run; the window is summed with the input rows as
//   the outer loop, two channels per packed f32x2 FMA, by 128 threads per tile,
//   two per block each summing half the channels (window_split of window.cuh;
//   Z in registers); date 1's Z stays in registers while date 2's is summed,
//   and each thread then takes the log-dets of the four outputs of its row
//   from registers, two adjacent outputs per pass with the compensated
//   arithmetic on packed float2 pairs (f32x2: one instruction for both, each
//   half rounded as the scalar operation).  ~52 KB of shared memory per CTA,
//   four CTAs per SM.
//   Backward (64 threads per tile, one per block): blocks are loaded directly; the window is summed one channel at a
//   time (the registers go to the 49 tap accumulators); Z, then the packed
//   M_t, are parked in shared memory for the correlations; the inverses run
//   as packed pairs where registers allow (3 x 3 and 5 x 5 windows).
//   (Packed FMAs over pairs of adjacent output columns instead of channel
//   pairs ran 11% slower: they need odd-offset input pairs, which cost
//   register moves.)
// Each tile writes its partial sums (FP64) to the workspace; a one-block-per-
// output kernel adds them in tile order.  No float atomics: the results are the
// same bits on every run.
#include "async.cuh"
#include "common.cuh"
#include "pixel.cuh"
#include "window.cuh"

namespace zinv {

namespace {

using namespace win;

constexpr int kRedThreads = 256;

struct WsArgs {
  const float2* s[2];
  int64_t H, W, plane_ld;
  const float* weights;
  float* q_map;
  double* partial;  // [tiles][K]
  float* z_save = nullptr;   // forward: both dates' Z, [18][H*W], or null
  bool z_vec = false;        // z_save takes 16-byte stores (16-byte aligned, W % 4 == 0)
  const float* m = nullptr;  // saved-Z backward: the packed M_1, M_2, [18][H*W]
  bool m_vec = false;        // m takes 16-byte copies (16-byte aligned, W % 4 == 0)
};

// Loads into registers the three components of the staged pixels this thread
// owns (pixel i = tid + k*kWT of the tile plus halo, row-major, clamp-to-edge).
template <int R>
__device__ __forceinline__ void prefetch(const WsArgs& a, int t, int64_t tile,
                                         float2 (&v)[WTile<R>::KO][3]) {
  using T = WTile<R>;
  const int64_t tiles_x = (a.W + kTW - 1) / kTW;
  const int64_t ty0 = (tile / tiles_x) * kTH, tx0 = (tile % tiles_x) * kTW;
  int r = threadIdx.x / T::SW, x = threadIdx.x - r * T::SW;
  constexpr int dr = kWT / T::SW, dx = kWT - dr * T::SW;
#pragma unroll
  for (int k = 0; k < T::KO; ++k) {
    if (r < T::SH) {
      const int64_t q = clampi(ty0 - R + r, a.H - 1) * a.W + clampi(tx0 - R + x, a.W - 1);
      v[k][0] = __ldg(a.s[t] + q);
      v[k][1] = __ldg(a.s[t] + a.plane_ld + q);
      v[k][2] = __ldg(a.s[t] + 2 * a.plane_ld + q);
    }
    x += dx;
    r += dr;
    if (x >= T::SW) {
      x -= T::SW;
      ++r;
    }
  }
}

// The nine channel products of the prefetched pixels -> P[c][SH][SWP].
template <int R>
__device__ __forceinline__ void store_products(const float2 (&v)[WTile<R>::KO][3], float* P) {
  using T = WTile<R>;
  int r = threadIdx.x / T::SW, x = threadIdx.x - r * T::SW;
  constexpr int dr = kWT / T::SW, dx = kWT - dr * T::SW;
#pragma unroll
  for (int k = 0; k < T::KO; ++k) {
    if (r < T::SH) {
      float p[9];
      products(v[k][0], v[k][1], v[k][2], p);
#pragma unroll
      for (int c = 0; c < 9; ++c) P[c * T::PLANE + r * T::SWP + x] = p[c];
    }
    x += dx;
    r += dr;
    if (x >= T::SW) {
      x -= T::SW;
      ++r;
    }
  }
}

template <int R>
__device__ __forceinline__ void load_weights(const float* weights, float (&w)[WTile<R>::K]) {
#pragma unroll
  for (int k = 0; k < WTile<R>::K; ++k) w[k] = __ldg(weights + k);
}

// One channel's window sums for the thread's 4 x 2 outputs (tile rows y0 and
// y0 + 1, columns x0..x0+3) from that channel's staged products Pc [SH][SWP].
// Each of the L + 1 input rows is loaded once and feeds both output rows; per
// output the taps are added in row-major order.
template <int R>
__device__ __forceinline__ void window_4x2(const float* Pc, const float (&w)[WTile<R>::K], int y0,
                                           int x0, float (&z)[2][4]) {
  using T = WTile<R>;
  constexpr int L = T::L;
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int i = 0; i < 4; ++i) z[r][i] = 0.0f;
#pragma unroll
  for (int iy = 0; iy <= L; ++iy) {
    float row[4 * T::NV];
    load_row<R>(Pc + (y0 + iy) * T::SWP + x0, row);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int dy = iy - r;
      if (dy < 0 || dy >= L) continue;
#pragma unroll
      for (int dx = 0; dx < L; ++dx)
#pragma unroll
        for (int i = 0; i < 4; ++i) z[r][i] = fmaf(w[dy * L + dx], row[i + dx], z[r][i]);
    }
  }
}

// Stages date t's products of a tile (plus halo) into P with direct loads.
template <int R>
__device__ __forceinline__ void stage(const WsArgs& a, int t, int64_t tile, float* P) {
  float2 v[WTile<R>::KO][3];
  prefetch<R>(a, t, tile, v);
  store_products<R>(v, P);
}

// Fixed-order block reduction of one double per thread; returns the sum in thread 0.
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  __syncthreads();
  return s;
}

// Both dates' Z of one output row (tile row yr, columns x0 .. x0 + 3) ->
// z_save: date 1's nine packed planes, then date 2's, plane stride H*W.
// Outputs outside the image are not stored.
__device__ __forceinline__ void save_z_row(const WsArgs& a, int64_t ty0, int64_t tx0, int yr,
                                           int x0, const float (&z1)[9][4],
                                           const float (&z2)[9][4]) {
  const int64_t n = a.H * a.W, gx = tx0 + x0, gy = ty0 + yr;
  if (gy >= a.H) return;
  const bool vec = a.z_vec && gx + 4 <= a.W;
  float* base = a.z_save + gy * a.W + gx;
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    if (vec) {
      __stcs(reinterpret_cast<float4*>(base + c * n),
             make_float4(z1[c][0], z1[c][1], z1[c][2], z1[c][3]));
      __stcs(reinterpret_cast<float4*>(base + (9 + c) * n),
             make_float4(z2[c][0], z2[c][1], z2[c][2], z2[c][3]));
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (gx + i < a.W) {
          __stcs(base + c * n + i, z1[c][i]);
          __stcs(base + (9 + c) * n + i, z2[c][i]);
        }
    }
  }
}

// The forward runs the channel-split window engine (128 threads per tile, two
// per 4 x 2 block of outputs, each summing half the channels), four CTAs per
// SM: 16 warps with 4 tiles in flight, against 8 warps on the paired engine
// (3 x 3 / 5 x 5 13% / 9% faster, 7 x 7 unchanged, same bits).  The saving
// 7 x 7 forward, with its Z stores, runs three CTAs with more registers (2%).
__host__ __device__ constexpr int fwd_min_blocks(int r, bool save) {
  return save && r == 3 ? 3 : 4;
}

template <int R, bool SAVE>
__global__ void __launch_bounds__(kWS, fwd_min_blocks(R, SAVE)) k_wishart_fwd(WsArgs a) {
  using T = WTile<R>;
  extern __shared__ __align__(16) float smem[];
  float* P = smem;  // one date's products, channel-paired layout
  float2* Sb = reinterpret_cast<float2*>(smem + T::P_FLOATS);  // next single-look block
  float2* wsh2 = reinterpret_cast<float2*>(Sb + T::S_F2);      // duplicated taps [L][WROW]
  double* red = reinterpret_cast<double*>(wsh2 + T::L * T::WROW);
  const int64_t tiles_x = (a.W + kTW - 1) / kTW;
  const int64_t tiles = tiles_x * ((a.H + kTH - 1) / kTH);
  const Split sp = split_of(threadIdx.x);
  const float six_ln2 = 4.15888308335967185650f;
  stage_taps_paired<R, kWS>(a.weights, wsh2);
  if ((int64_t)blockIdx.x < tiles)
    issue_block<R, kWS>(a.s[0], a.plane_ld, a.H, a.W, blockIdx.x, Sb);
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t ty0 = (tile / tiles_x) * kTH, tx0 = (tile % tiles_x) * kTW;
    float z0[9][4];  // date 1's Z of the thread's output row
    double qsum = 0.0;
#pragma unroll 1
    for (int t = 0; t < 2; ++t) {
      cp_async_wait<0>();
      __syncthreads();  // date t's block is in Sb; P is free (and the taps are in place)
      block_products_paired<R, kWS>(Sb, P);
      __syncthreads();  // Sb is free; P holds date t's products
      // the next block (date 2 of this tile, then date 1 of the next) loads
      // while this date's window sums run
      const int64_t next = t == 0 ? tile : tile + gridDim.x;
      if (next < tiles) issue_block<R, kWS>(a.s[1 - t], a.plane_ld, a.H, a.W, next, Sb);
      float z[9][4];
      window_split<R, 2>(P, wsh2, sp, z);
      if (t == 0) {
#pragma unroll
        for (int c = 0; c < 9; ++c)
#pragma unroll
          for (int i = 0; i < 4; ++i) z0[c][i] = z[c][i];
        continue;
      }
      if constexpr (SAVE) save_z_row(a, ty0, tx0, sp.y0 + sp.h, sp.x0, z0, z);
      // Both dates' Z of row h are in registers: the thread takes the
      // compensated log-dets of Z1, Z2 and Z1 + Z2 of its four outputs, two
      // adjacent outputs per pass on packed float2 pairs, and stores and adds
      // its q in column order.
      const int64_t gy = ty0 + sp.y0 + sp.h;
#pragma unroll
      for (int i = 0; i < 4; i += 2) {
        float2 z1[9], z2[9], z12[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) {
          z1[c] = make_float2(z0[c][i], z0[c][i + 1]);
          z2[c] = make_float2(z[c][i], z[c][i + 1]);
          z12[c] = add_rn(z1[c], z2[c]);
        }
        const float2 l1 = log_dd(det_comp<float2>(z1));
        const float2 l2 = log_dd(det_comp<float2>(z2));
        const float2 l12 = log_dd(det_comp<float2>(z12));
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int64_t gx = tx0 + sp.x0 + i + e;
          if (gy >= a.H || gx >= a.W) continue;
          const float q = e == 0 ? (l1.x + l2.x) - 2.0f * l12.x + six_ln2
                                 : (l1.y + l2.y) - 2.0f * l12.y + six_ln2;
          if (a.q_map) a.q_map[gy * a.W + gx] = q;
          qsum += (double)q;
        }
      }
    }
    const double s = block_sum(qsum, red);
    if (threadIdx.x == 0) a.partial[tile] = s;
  }
  cp_async_wait<0>();
}

// M_t of one output o in packed gradient form over the Z slots of G, from
// the inverses W_1, W_2, W_12: M_t = W_t - 2 W_12, off-diagonal packed reals
// doubled; zero outside the image.
__device__ __forceinline__ void store_m(const WsArgs& a, float* G, int64_t ty0, int64_t tx0,
                                        int o, const float w1[9], const float w2[9],
                                        const float w12[9]) {
  const int64_t gy = ty0 + o / kTW, gx = tx0 + o % kTW;
  const bool inside = gy < a.H && gx < a.W;
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    const float two = (c == 0 || c == 5 || c == 8) ? 1.0f : 2.0f;
    G[c * kTH * kTW + o] = inside ? two * fmaf(-2.0f, w12[c], w1[c]) : 0.0f;
    G[(9 + c) * kTH * kTW + o] = inside ? two * fmaf(-2.0f, w12[c], w2[c]) : 0.0f;
  }
}

// The three compensated inverses of every output of the tile, over the Z
// slots of G, two outputs per pass (o and o + kWT, so a warp reads one row's
// 32 entries of a plane) as packed pairs.  The 3 x 3 and 5 x 5 kernels inline
// the three inverses.  The 7 x 7 kernel (LOOPED) runs one inverse routine three
// times, W12 = (Z1 + Z2)^-1 first, then W1 and W2, each turned into its M_t and
// stored at once: with three inlined copies its larger body stalled on
// instruction fetch, and the loop took 7% off its time (the 3 x 3 kernel lost
// 5% that way).  Both forms round identically.
template <bool LOOPED>
__device__ __forceinline__ void bwd_inverses(const WsArgs& a, float* G, int64_t ty0,
                                             int64_t tx0) {
  constexpr int TILE = kTH * kTW;
  static_assert(TILE % (2 * kWT) == 0, "outputs o and o + kWT are in the tile");
  if constexpr (!LOOPED) {
#pragma unroll 1
    for (int o = threadIdx.x; o < kTH * kTW; o += 2 * kWT) {
      float2 z1[9], z2[9], z12[9], w1[9], w2[9], w12[9], d;
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        z1[c] = make_float2(G[c * kTH * kTW + o], G[c * kTH * kTW + o + kWT]);
        z2[c] = make_float2(G[(9 + c) * kTH * kTW + o], G[(9 + c) * kTH * kTW + o + kWT]);
        z12[c] = add_rn(z1[c], z2[c]);
      }
      adjugate_inv_det_comp<float2>(z1, w1, d);
      adjugate_inv_det_comp<float2>(z2, w2, d);
      adjugate_inv_det_comp<float2>(z12, w12, d);
      float v1[9], v2[9], v12[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) v1[c] = w1[c].x, v2[c] = w2[c].x, v12[c] = w12[c].x;
      store_m(a, G, ty0, tx0, o, v1, v2, v12);
#pragma unroll
      for (int c = 0; c < 9; ++c) v1[c] = w1[c].y, v2[c] = w2[c].y, v12[c] = w12[c].y;
      store_m(a, G, ty0, tx0, o + kWT, v1, v2, v12);
    }
  } else {
#pragma unroll 1
    for (int o = threadIdx.x; o < TILE; o += 2 * kWT) {
      float2 z[9], w[9], w12[9], d;
#pragma unroll 1
      for (int m = 0; m < 3; ++m) {
        // m = 0: Z1 + Z2; m = 1: Z1 (+ 0); m = 2: Z2 (0 +)
#pragma unroll
        for (int c = 0; c < 9; ++c) {
          const float2 zero = make_float2(0.0f, 0.0f);
          const float2 z1 = m != 2 ? make_float2(G[c * TILE + o], G[c * TILE + o + kWT]) : zero;
          const float2 z2 =
              m != 1 ? make_float2(G[(9 + c) * TILE + o], G[(9 + c) * TILE + o + kWT]) : zero;
          z[c] = add_rn(z1, z2);
        }
        adjugate_inv_det_comp<float2>(z, w, d);
        if (m == 0) {
#pragma unroll
          for (int c = 0; c < 9; ++c) w12[c] = w[c];
          continue;
        }
        // M_t = W_t - 2 W12 over date t's Z slot, as store_m does
        float* Gt = G + (m - 1) * 9 * TILE;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int oh = o + h * kWT;
          const int64_t gy = ty0 + oh / kTW, gx = tx0 + oh % kTW;
          const bool inside = gy < a.H && gx < a.W;
#pragma unroll
          for (int c = 0; c < 9; ++c) {
            const float two = (c == 0 || c == 5 || c == 8) ? 1.0f : 2.0f;
            const float wt = h ? w[c].y : w[c].x, wd = h ? w12[c].y : w12[c].x;
            Gt[c * TILE + oh] = inside ? two * fmaf(-2.0f, wd, wt) : 0.0f;
          }
        }
      }
    }
  }
}

// One thread's weight-gradient tap accumulators: tap (dy, dx) with dx < L - 1
// in the float2 pair (dx even, dx + 1), the last column dx = L - 1 scalar.
template <int R>
struct TapAcc {
  static constexpr int L = 2 * R + 1;
  float2 p[L][R];
  float s[L];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int dy = 0; dy < L; ++dy) {
#pragma unroll
      for (int j = 0; j < R; ++j) p[dy][j] = make_float2(0.0f, 0.0f);
      s[dy] = 0.0f;
    }
  }
  // tap k = dy L + dx (k a compile-time constant after unrolling)
  __device__ __forceinline__ float get(int k) const {
    const int dy = k / L, dx = k - (k / L) * L;
    return dx == L - 1 ? s[dy] : ((dx & 1) ? p[dy][dx >> 1].y : p[dy][dx >> 1].x);
  }
};

// The correlation terms of one staged input row (row y0 + iy of the thread's
// columns x0 .. x0 + 3 + 2R): tap (dy, dx) += g[r][i] row[i + dx] for output
// rows r with dy = iy - r, each tap's terms in order i = 0..3.  For even i the
// pair (row[i + dx], row[i + dx + 1]) of an even dx is an aligned pair of the
// loaded row, so one packed f32x2 FMA adds to both taps of a pair (each half
// rounded as the scalar fmaf: the bits of the scalar loop); odd i and the last
// column take scalar FMAs.
template <int R>
__device__ __forceinline__ void corr_row(const float (&g)[2][4],
                                         const float (&row)[4 * WTile<R>::NV], int iy,
                                         TapAcc<R>& acc) {
  constexpr int L = 2 * R + 1;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int dy = iy - r;
    if (dy < 0 || dy >= L) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if ((i & 1) == 0) {
        const float2 gg = make_float2(g[r][i], g[r][i]);
#pragma unroll
        for (int j = 0; j < R; ++j)
          acc.p[dy][j] =
              __ffma2_rn(gg, make_float2(row[i + 2 * j], row[i + 2 * j + 1]), acc.p[dy][j]);
      } else {
#pragma unroll
        for (int j = 0; j < R; ++j) {
          acc.p[dy][j].x = fmaf(g[r][i], row[i + 2 * j], acc.p[dy][j].x);
          acc.p[dy][j].y = fmaf(g[r][i], row[i + 2 * j + 1], acc.p[dy][j].y);
        }
      }
      acc.s[dy] = fmaf(g[r][i], row[i + L - 1], acc.s[dy]);
    }
  }
}

template <int R>
__global__ void __launch_bounds__(kWT, 3) k_wishart_bwd(WsArgs a) {
  using T = WTile<R>;
  constexpr int L = T::L;
  constexpr int K = T::K;
  extern __shared__ __align__(16) float smem[];
  float* P = smem;
  float* G = smem + T::P_FLOATS;  // [2][9][kTH][kTW]: Z_t, then the packed M_t
  static_assert(T::K * (kWT + 1) <= T::P_FLOATS, "the tap partials fit in P");
  const int64_t tiles_x = (a.W + kTW - 1) / kTW;
  const int64_t tiles = tiles_x * ((a.H + kTH - 1) / kTH);
  const int y0 = 2 * (threadIdx.x / kTX), x0 = 4 * (threadIdx.x % kTX);
  // P holds one date at a time.  Per tile, three stages: date 1 (its Z), date 2
  // (its Z, the inverses, then its correlation while still staged), date 1
  // again (its correlation).  Staging loads directly (no register prefetch:
  // the registers go to the 49 tap accumulators; the other CTAs on the SM
  // cover the load latency).
  // 3 x 3 and 5 x 5: each stage's single-look data is loaded into registers
  // during the previous phase (1.36 -> 1.30 and 1.80 -> 1.68 ms on the 4096^2
  // pair); the 7 x 7 kernel, whose 49 taps and 49 accumulators fill the
  // registers, spilled that way (2.70 -> 3.21 ms) and loads each stage directly.
  constexpr bool PREFETCH = R < 3;
  float2 v[PREFETCH ? T::KO : 1][3];
  if constexpr (PREFETCH) {
    if ((int64_t)blockIdx.x < tiles) prefetch<R>(a, 0, blockIdx.x, v);
  }
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t ty0 = (tile / tiles_x) * kTH, tx0 = (tile % tiles_x) * kTW;
    TapAcc<R> acc;
    acc.zero();
#pragma unroll 1
    for (int phase = 0; phase < 3; ++phase) {
      const int t = phase == 1 ? 1 : 0;  // the date staged now
      __syncthreads();
      if constexpr (PREFETCH) {
        store_products<R>(v, P);
        if (phase == 0) {
          prefetch<R>(a, 1, tile, v);
        } else if (phase == 1) {
          prefetch<R>(a, 0, tile, v);
        } else if (tile + gridDim.x < tiles) {
          prefetch<R>(a, 0, tile + gridDim.x, v);
        }
      } else {
        stage<R>(a, t, tile, P);
      }
      __syncthreads();
      if (phase < 2) {
        float w[K];
        load_weights<R>(a.weights, w);
#pragma unroll 1
        for (int c = 0; c < 9; ++c) {
          float z[2][4];
          window_4x2<R>(P + c * T::PLANE, w, y0, x0, z);
          store_block(G + (t * 9 + c) * kTH * kTW, y0, x0, z);
        }
      }
      if (phase == 1) {
        // per output: three compensated inverses, M_t = W_t - 2 W_12 in packed
        // gradient form over the Z slots
        __syncthreads();
        bwd_inverses<(R == 3)>(a, G, ty0, tx0);
        __syncthreads();
      }
      if (phase > 0) {
        // dL/dw_k over the thread's 4 x 2 pixels: sum_c G_t[c](p) P_t[c](p + k)
#pragma unroll 1
        for (int c = 0; c < 9; ++c) {
          const float* Gc = G + (t * 9 + c) * kTH * kTW;
          float g[2][4];
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            const float4 gv = *reinterpret_cast<const float4*>(Gc + (y0 + r) * kTW + x0);
            g[r][0] = gv.x;
            g[r][1] = gv.y;
            g[r][2] = gv.z;
            g[r][3] = gv.w;
          }
          const float* Pc = P + c * T::PLANE;
#pragma unroll
          for (int iy = 0; iy <= L; ++iy) {
            float row[4 * T::NV];
            load_row<R>(Pc + (y0 + iy) * T::SWP + x0, row);
            corr_row<R>(g, row, iy, acc);
          }
        }
      }
    }
    // Fixed-order sum of the K taps over the block: the threads' accumulators
    // go to shared memory (P is free: [K][kWT + 1], conflict-free both ways),
    // then thread k adds tap k over the block's threads in thread order with
    // TwoSum (compensated FP32, as accurate as FP64 for 64 terms) and stores it
    // as a double.  An FP64 shuffle tree per tap kept GB300's FP64 pipe, at
    // 1/64 of the FP32 rate, 28% busy.
    __syncthreads();
    float* accs = P;
#pragma unroll
    for (int k = 0; k < K; ++k) accs[k * (kWT + 1) + threadIdx.x] = acc.get(k);
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += kWT) {
      float sum = 0.0f, err = 0.0f;
#pragma unroll 8
      for (int t = 0; t < kWT; ++t) {
        float e;
        two_sum(sum, accs[k * (kWT + 1) + t], sum, e);
        err += e;
      }
      a.partial[tile * K + k] = (double)sum + (double)err;
    }
  }
}

// ---------------------------------------------------------------------------
// Backward from saved Z (the forward's z_save): the window sums are not
// recomputed.  k_wishart_m turns each pixel's saved Z1, Z2 into the packed
// gradient forms of M_t = W_t - 2 W12 (the same compensated inverses and
// rounding as the recomputing backward); k_wishart_corr then correlates them
// with the staged channel products.  Results are the recomputing backward's
// bits, as both compute Z with the same tap order.
// ---------------------------------------------------------------------------

// Pixels p and p + half of `n` (half = ceil(n/2)) as the two halves of packed
// pairs; the last thread of an odd n computes its second pixel twice and
// stores it once.
__global__ void __launch_bounds__(256) k_wishart_m(const float* z, float* m, int64_t n) {
  const int64_t half = (n + 1) / 2;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < half;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = p + half < n ? p + half : p;
    float2 z1[9], z2[9], z12[9], w1[9], w2[9], w12[9], d;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      z1[c] = make_float2(__ldcs(z + c * n + p), __ldcs(z + c * n + q));
      z2[c] = make_float2(__ldcs(z + (9 + c) * n + p), __ldcs(z + (9 + c) * n + q));
      z12[c] = add_rn(z1[c], z2[c]);
    }
    adjugate_inv_det_comp<float2>(z12, w12, d);
    adjugate_inv_det_comp<float2>(z1, w1, d);
    adjugate_inv_det_comp<float2>(z2, w2, d);
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      const float two = (c == 0 || c == 5 || c == 8) ? 1.0f : 2.0f;
      m[c * n + p] = two * fmaf(-2.0f, w12[c].x, w1[c].x);
      m[(9 + c) * n + p] = two * fmaf(-2.0f, w12[c].x, w2[c].x);
      if (q != p) {
        m[c * n + q] = two * fmaf(-2.0f, w12[c].y, w1[c].y);
        m[(9 + c) * n + q] = two * fmaf(-2.0f, w12[c].y, w2[c].y);
      }
    }
  }
}

// dL/dw_k per tile from saved M: per date (date 2 first, the recomputing
// backward's order), the tile's products P and its M_t (zero outside the
// image) are staged in shared memory, then the same correlation.  With no
// window sums to hold, the registers take the next stage's single-look data,
// loaded while the current date's correlation runs (1.98 -> 1.84 ms for the
// 4096^2 backward).
template <int R>
__global__ void __launch_bounds__(kWT, 4) k_wishart_corr(WsArgs a) {
  using T = WTile<R>;
  constexpr int L = T::L;
  constexpr int K = T::K;
  constexpr int TILE = kTH * kTW;
  extern __shared__ __align__(16) float smem[];
  float* P = smem;
  float* G = smem + T::P_FLOATS;  // [9][kTH][kTW]: one date's packed M
  static_assert(T::K * (kWT + 1) <= T::P_FLOATS, "the tap partials fit in P");
  const int64_t n = a.H * a.W;
  const int64_t tiles_x = (a.W + kTW - 1) / kTW;
  const int64_t tiles = tiles_x * ((a.H + kTH - 1) / kTH);
  const int y0 = 2 * (threadIdx.x / kTX), x0 = 4 * (threadIdx.x % kTX);
  // the single-look data of the next stage is loaded into registers while
  // the current date's correlation runs
  float2 v[T::KO][3];
  if ((int64_t)blockIdx.x < tiles) prefetch<R>(a, 1, blockIdx.x, v);
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t ty0 = (tile / tiles_x) * kTH, tx0 = (tile % tiles_x) * kTW;
    TapAcc<R> acc;
    acc.zero();
#pragma unroll 1
    for (int t = 1; t >= 0; --t) {
      __syncthreads();
      // M_t of the tile (zero outside the image) copied asynchronously while
      // the products are formed
      if (a.m_vec) {
        // 16-byte groups: with W % 4 == 0 the four outputs of a group are all
        // inside the image or all outside
#pragma unroll 2
        for (int e = threadIdx.x; e < 9 * TILE / 4; e += kWT) {
          const int c = e / (TILE / 4), o = 4 * (e - c * (TILE / 4));
          const int64_t gy = ty0 + o / kTW, gx = tx0 + o % kTW;
          const bool in = gy < a.H && gx < a.W;
          cp_async16_zfill(G + c * TILE + o, in ? a.m + (9 * t + c) * n + gy * a.W + gx : a.m,
                           in);
        }
      } else {
#pragma unroll 8
        for (int e = threadIdx.x; e < 9 * TILE; e += kWT) {
          const int c = e / TILE, o = e - c * TILE;
          const int64_t gy = ty0 + o / kTW, gx = tx0 + o % kTW;
          const bool in = gy < a.H && gx < a.W;
          cp_async4_zfill(G + e, in ? a.m + (9 * t + c) * n + gy * a.W + gx : a.m, in);
        }
      }
      cp_async_commit();
      store_products<R>(v, P);
      if (t == 1) {
        prefetch<R>(a, 0, tile, v);
      } else if (tile + gridDim.x < tiles) {
        prefetch<R>(a, 1, tile + gridDim.x, v);
      }
      cp_async_wait<0>();
      __syncthreads();
#pragma unroll 1
      for (int c = 0; c < 9; ++c) {
        const float* Gc = G + c * TILE;
        float g[2][4];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const float4 gv = *reinterpret_cast<const float4*>(Gc + (y0 + r) * kTW + x0);
          g[r][0] = gv.x;
          g[r][1] = gv.y;
          g[r][2] = gv.z;
          g[r][3] = gv.w;
        }
        const float* Pc = P + c * T::PLANE;
#pragma unroll
        for (int iy = 0; iy <= L; ++iy) {
          float row[4 * T::NV];
          load_row<R>(Pc + (y0 + iy) * T::SWP + x0, row);
          corr_row<R>(g, row, iy, acc);
        }
      }
    }
    // fixed-order tap sums over the block, as the recomputing backward
    __syncthreads();
    float* accs = P;
#pragma unroll
    for (int k = 0; k < K; ++k) accs[k * (kWT + 1) + threadIdx.x] = acc.get(k);
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += kWT) {
      float sum = 0.0f, err = 0.0f;
#pragma unroll 8
      for (int t = 0; t < kWT; ++t) {
        float e;
        two_sum(sum, accs[k * (kWT + 1) + t], sum, e);
        err += e;
      }
      a.partial[tile * K + k] = (double)sum + (double)err;
    }
  }
}

// out[k] = scale * sum_tiles partial[tile][k], summed in a fixed order.
// double_out: out is double (the loss); otherwise float (the weight gradient)
// and scale is read from *g (the upstream gradient, a device double).
__global__ void __launch_bounds__(kRedThreads)
    k_reduce_tiles(const double* partial, int64_t tiles, int K, const double* g, void* out,
                   int double_out) {
  __shared__ double red[kRedThreads / 32];
  const int k = blockIdx.x;
  double v = 0.0;
  for (int64_t t = threadIdx.x; t < tiles; t += blockDim.x) v += partial[t * K + k];
  const double s = block_sum(v, red);
  if (threadIdx.x == 0) {
    const double scale = g ? *g : 1.0;
    if (double_out)
      static_cast<double*>(out)[k] = scale * s;
    else
      static_cast<float*>(out)[k] = (float)(scale * s);
  }
}

template <int R>
size_t fwd_smem() {
  using T = WTile<R>;
  return T::P_FLOATS * sizeof(float) + (T::L * T::WROW + T::S_F2) * sizeof(float2) +
         (kWS / 32) * sizeof(double);
}
template <int R>
size_t bwd_smem() {
  using T = WTile<R>;
  return (T::P_FLOATS + 2 * T::Z_FLOATS) * sizeof(float);
}

int64_t tile_count(int64_t H, int64_t W);

template <int R>
size_t corr_smem() {
  using T = WTile<R>;
  return (T::P_FLOATS + T::Z_FLOATS) * sizeof(float);
}

// Workspace of the saved-Z backward: the per-tile partials, then (256-byte
// aligned) the packed M_1, M_2 of every pixel.
size_t partials_bytes(int64_t H, int64_t W, int win) {
  const size_t b = (size_t)tile_count(H, W) * (size_t)(win * win) * sizeof(double);
  return (b + 255) / 256 * 256;
}

int64_t tile_count(int64_t H, int64_t W) {
  return ((W + kTW - 1) / kTW) * ((H + kTH - 1) / kTH);
}

template <typename Kern>
int launch_tiles(Kern kernel, size_t smem, const WsArgs& a, cudaStream_t s, int threads = kWT) {
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return ZINV_ERR_LAUNCH;
  }
  const int64_t tiles = tile_count(a.H, a.W);
  const int64_t blocks = cover_blocks(tiles * threads, threads);
  kernel<<<(unsigned)blocks, threads, smem, s>>>(a);
  return launch_status();
}

// Shared argument checks; fills a.  `weights` may be null only when
// !need_weights; the workspace must hold `need` bytes (0: the per-tile
// partials).  Returns ZINV_OK or an error.
int prepare(const float* s1, const float* s2, int64_t H, int64_t W, int64_t plane_ld, int win,
            const float* weights, void* ws, size_t ws_bytes, WsArgs& a, DeviceInfo& di,
            bool need_weights = true, size_t need = 0) {
  if (H < 1 || W < 1 || H > kMaxLd / W) return ZINV_ERR_ARG;
  if (win != 3 && win != 5 && win != 7) return ZINV_ERR_ARG;
  if (plane_ld < H * W || plane_ld > kMaxLd) return ZINV_ERR_ARG;
  if (!s1 || !s2 || (need_weights && !weights) || !ws) return ZINV_ERR_ARG;
  if (!aligned(s1, 8) || !aligned(s2, 8) || !aligned(weights, 4) || !aligned(ws, 8))
    return ZINV_ERR_ARG;
  if (need == 0) need = (size_t)tile_count(H, W) * (size_t)(win * win) * sizeof(double);
  if (ws_bytes < need) return ZINV_ERR_ARG;
  int rc = device_info(&di);
  if (rc != ZINV_OK) return rc;
  if (!device_accessible(s1) || !device_accessible(s2) ||
      (weights && !device_accessible(weights)) || !device_accessible(ws))
    return ZINV_ERR_ARG;
  a.s[0] = reinterpret_cast<const float2*>(s1);
  a.s[1] = reinterpret_cast<const float2*>(s2);
  a.H = H;
  a.W = W;
  a.plane_ld = plane_ld;
  a.weights = weights;
  a.q_map = nullptr;
  a.partial = static_cast<double*>(ws);
  return ZINV_OK;
}

}  // namespace
}  // namespace zinv

extern "C" size_t wishart_workspace_bytes(int64_t H, int64_t W, int win) {
  if (H < 1 || W < 1 || win < 1) return 0;
  return (size_t)zinv::tile_count(H, W) * (size_t)(win * win) * sizeof(double);
}

extern "C" int wishart_stat_fwd(const float* s1, const float* s2, int64_t H, int64_t W,
                                int64_t plane_ld, int win, const float* weights, float* q_map,
                                double* d_loss, void* ws, size_t ws_bytes, void* stream) {
  using namespace zinv;
  WsArgs a;
  DeviceInfo di;
  if (!d_loss || !aligned(d_loss, 8) || !aligned(q_map, 4)) return ZINV_ERR_ARG;
  int rc = prepare(s1, s2, H, W, plane_ld, win, weights, ws, ws_bytes, a, di);
  if (rc != ZINV_OK) return rc;
  if (!device_accessible(d_loss) || (q_map && !device_accessible(q_map))) return ZINV_ERR_ARG;
  a.q_map = q_map;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (win) {
    case 3: rc = launch_tiles(k_wishart_fwd<1, false>, fwd_smem<1>(), a, st, kWS); break;
    case 5: rc = launch_tiles(k_wishart_fwd<2, false>, fwd_smem<2>(), a, st, kWS); break;
    default: rc = launch_tiles(k_wishart_fwd<3, false>, fwd_smem<3>(), a, st, kWS); break;
  }
  if (rc != ZINV_OK) return rc;
  k_reduce_tiles<<<1, kRedThreads, 0, st>>>(a.partial, tile_count(H, W), 1, nullptr, d_loss, 1);
  return launch_status();
}

extern "C" int wishart_stat_bwd(const float* s1, const float* s2, int64_t H, int64_t W,
                                int64_t plane_ld, int win, const float* weights,
                                const double* d_grad_loss, float* grad_weights, void* ws,
                                size_t ws_bytes, void* stream) {
  using namespace zinv;
  WsArgs a;
  DeviceInfo di;
  if (!grad_weights || !aligned(grad_weights, 4) || !aligned(d_grad_loss, 8))
    return ZINV_ERR_ARG;
  int rc = prepare(s1, s2, H, W, plane_ld, win, weights, ws, ws_bytes, a, di);
  if (rc != ZINV_OK) return rc;
  if (!device_accessible(grad_weights) || (d_grad_loss && !device_accessible(d_grad_loss)))
    return ZINV_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (win) {
    case 3: rc = launch_tiles(k_wishart_bwd<1>, bwd_smem<1>(), a, st); break;
    case 5: rc = launch_tiles(k_wishart_bwd<2>, bwd_smem<2>(), a, st); break;
    default: rc = launch_tiles(k_wishart_bwd<3>, bwd_smem<3>(), a, st); break;
  }
  if (rc != ZINV_OK) return rc;
  k_reduce_tiles<<<win * win, kRedThreads, 0, st>>>(a.partial, tile_count(H, W), win * win,
                                                    d_grad_loss, grad_weights, 0);
  return launch_status();
}

namespace zinv {
namespace {
// Largest image of the saved-Z calls: 72 bytes per pixel stay within size_t.
constexpr int64_t kMaxSavedPixels = (int64_t)1 << 56;
}  // namespace
}  // namespace zinv

extern "C" size_t wishart_saved_bytes(int64_t H, int64_t W) {
  if (H < 1 || W < 1 || H > zinv::kMaxSavedPixels / W) return 0;
  return (size_t)18 * (size_t)(H * W) * sizeof(float);
}

extern "C" size_t wishart_bwd_saved_workspace_bytes(int64_t H, int64_t W, int win) {
  if (H < 1 || W < 1 || win < 1 || H > zinv::kMaxSavedPixels / W) return 0;
  return zinv::partials_bytes(H, W, win) + (size_t)18 * (size_t)(H * W) * sizeof(float);
}

extern "C" int wishart_stat_fwd_save(const float* s1, const float* s2, int64_t H, int64_t W,
                                     int64_t plane_ld, int win, const float* weights,
                                     float* q_map, double* d_loss, float* z_saved, void* ws,
                                     size_t ws_bytes, void* stream) {
  using namespace zinv;
  WsArgs a;
  DeviceInfo di;
  if (!d_loss || !z_saved || !aligned(d_loss, 8) || !aligned(q_map, 4) || !aligned(z_saved, 4))
    return ZINV_ERR_ARG;
  if (H < 1 || W < 1 || H > kMaxSavedPixels / W) return ZINV_ERR_ARG;
  int rc = prepare(s1, s2, H, W, plane_ld, win, weights, ws, ws_bytes, a, di);
  if (rc != ZINV_OK) return rc;
  if (!device_accessible(d_loss) || !device_accessible(z_saved) ||
      (q_map && !device_accessible(q_map)))
    return ZINV_ERR_ARG;
  a.q_map = q_map;
  a.z_save = z_saved;
  a.z_vec = aligned(z_saved, 16) && (W % 4) == 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (win) {
    case 3: rc = launch_tiles(k_wishart_fwd<1, true>, fwd_smem<1>(), a, st, kWS); break;
    case 5: rc = launch_tiles(k_wishart_fwd<2, true>, fwd_smem<2>(), a, st, kWS); break;
    default: rc = launch_tiles(k_wishart_fwd<3, true>, fwd_smem<3>(), a, st, kWS); break;
  }
  if (rc != ZINV_OK) return rc;
  k_reduce_tiles<<<1, kRedThreads, 0, st>>>(a.partial, tile_count(H, W), 1, nullptr, d_loss, 1);
  return launch_status();
}

extern "C" int wishart_stat_bwd_saved(const float* s1, const float* s2, int64_t H, int64_t W,
                                      int64_t plane_ld, int win, const float* z_saved,
                                      const double* d_grad_loss, float* grad_weights, void* ws,
                                      size_t ws_bytes, void* stream) {
  using namespace zinv;
  WsArgs a;
  DeviceInfo di;
  if (!z_saved || !grad_weights || !aligned(z_saved, 4) || !aligned(grad_weights, 4) ||
      !aligned(d_grad_loss, 8))
    return ZINV_ERR_ARG;
  if (H < 1 || W < 1 || H > kMaxSavedPixels / W || win < 1) return ZINV_ERR_ARG;
  const size_t need = wishart_bwd_saved_workspace_bytes(H, W, win);
  int rc = prepare(s1, s2, H, W, plane_ld, win, nullptr, ws, ws_bytes, a, di, false, need);
  if (rc != ZINV_OK) return rc;
  if (!device_accessible(z_saved) || !device_accessible(grad_weights) ||
      (d_grad_loss && !device_accessible(d_grad_loss)))
    return ZINV_ERR_ARG;
  float* m = reinterpret_cast<float*>(static_cast<char*>(ws) + partials_bytes(H, W, win));
  a.m = m;
  a.m_vec = aligned(m, 16) && (W % 4) == 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t n = H * W;
  k_wishart_m<<<(unsigned)cover_blocks((n + 1) / 2, 256), 256, 0, st>>>(z_saved, m, n);
  rc = launch_status();
  if (rc != ZINV_OK) return rc;
  switch (win) {
    case 3: rc = launch_tiles(k_wishart_corr<1>, corr_smem<1>(), a, st); break;
    case 5: rc = launch_tiles(k_wishart_corr<2>, corr_smem<2>(), a, st); break;
    default: rc = launch_tiles(k_wishart_corr<3>, corr_smem<3>(), a, st); break;
  }
  if (rc != ZINV_OK) return rc;
  k_reduce_tiles<<<win * win, kRedThreads, 0, st>>>(a.partial, tile_count(H, W), win * win,
                                                    d_grad_loss, grad_weights, 0);
  return launch_status();
}

// ---------------------------------------------------------------------------
// Allocation-free variant of wishart_stat_fwd.  Some callers cannot hand the
// library a workspace: a plugin inside a host application that owns every
// device allocation, or a processing loop that must not allocate once it runs.
// For them the per-tile partial sums live in this fixed device array instead
// of a caller buffer.  It is part of the module, so every device that loads the
// library holds these kNoAllocTiles doubles (1 MiB) until the process exits.
// ---------------------------------------------------------------------------
namespace zinv {
namespace {
constexpr int64_t kNoAllocTiles = 131072;  // one slot per 32 x 16 tile: 8192 x 8192 pixels
__device__ __align__(256) double g_noalloc_partials[kNoAllocTiles];

// Device address of g_noalloc_partials per device.  A successful lookup is
// kept; a failed one is not, so a later call on that device tries again.
struct NoAllocScratch {
  std::mutex mu;
  double* ptr = nullptr;
};
NoAllocScratch g_noalloc[kMaxDevices];

double* noalloc_scratch(int dev) {
  NoAllocScratch& sc = g_noalloc[dev];
  std::lock_guard<std::mutex> lock(sc.mu);
  if (!sc.ptr) {
    double* p = nullptr;
    if (cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_noalloc_partials) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    sc.ptr = p;
  }
  return sc.ptr;
}
}  // namespace
}  // namespace zinv

extern "C" int wishart_stat_fwd_noalloc(const float* s1, const float* s2, int64_t H, int64_t W,
                                        int64_t plane_ld, int win, const float* weights,
                                        float* q_map, double* d_loss, void* stream) {
  using namespace zinv;
  if (H < 1 || W < 1 || H > kMaxLd / W) return ZINV_ERR_ARG;
  if (win != 3 && win != 5 && win != 7) return ZINV_ERR_ARG;
  if (plane_ld < H * W || plane_ld > kMaxLd) return ZINV_ERR_ARG;
  if (!s1 || !s2 || !weights || !d_loss) return ZINV_ERR_ARG;
  if (!aligned(s1, 8) || !aligned(s2, 8) || !aligned(weights, 4) || !aligned(d_loss, 8) ||
      !aligned(q_map, 4))
    return ZINV_ERR_ARG;
  const int64_t tiles = tile_count(H, W);
  if (tiles > kNoAllocTiles) return ZINV_ERR_ARG;  // image larger than the fixed scratch
  DeviceInfo di;
  int dev = -1;
  int rc = device_info(&di, &dev);
  if (rc != ZINV_OK) return rc;
  // Host code cannot use g_noalloc_partials directly (here it names a host-side
  // stand-in); take the device address once per device, with that device current.
  double* scratch = noalloc_scratch(dev);
  if (!scratch) return ZINV_ERR_LAUNCH;
  if (!device_accessible(s1) || !device_accessible(s2) || !device_accessible(weights) ||
      !device_accessible(d_loss) || (q_map && !device_accessible(q_map)))
    return ZINV_ERR_ARG;
  WsArgs a;
  a.s[0] = reinterpret_cast<const float2*>(s1);
  a.s[1] = reinterpret_cast<const float2*>(s2);
  a.H = H;
  a.W = W;
  a.plane_ld = plane_ld;
  a.weights = weights;
  a.q_map = q_map;
  a.partial = scratch;  // every tile writes its own slot before the reduce reads it
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (win) {
    case 3: rc = launch_tiles(k_wishart_fwd<1, false>, fwd_smem<1>(), a, st, kWS); break;
    case 5: rc = launch_tiles(k_wishart_fwd<2, false>, fwd_smem<2>(), a, st, kWS); break;
    default: rc = launch_tiles(k_wishart_fwd<3, false>, fwd_smem<3>(), a, st, kWS); break;
  }
  if (rc != ZINV_OK) return rc;
  k_reduce_tiles<<<1, kRedThreads, 0, st>>>(a.partial, tiles, 1, nullptr, d_loss, 1);
  return launch_status();
}
