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
// route of Algorithm 2 (Dot2), so the log-dets keep FP32 accuracy.
//
// Tiles of 64 x 8 outputs, 128 threads, each thread four adjacent outputs of one
// row.  One date's channel products for the tile and its halo sit in shared
// memory at a time, staged from values each thread prefetched into registers
// while the previous stage was being used; a thread slides over a product row
// with 128-bit loads, 28 FMAs per loaded row, one channel at a time.  Each tile writes its partial sums (FP64) to the workspace; a
// one-block-per-output kernel adds them in tile order.  No float atomics: the
// results are the same bits on every run.
#include "common.cuh"
#include "pixel.cuh"

namespace zinv {

namespace {

constexpr int kWT = 128;  // threads per CTA
constexpr int kTW = 64;   // tile width (outputs)
constexpr int kTH = 8;    // tile height (outputs)
constexpr int kRedThreads = 256;

struct WsArgs {
  const float2* s[2];
  int64_t H, W, plane_ld;
  const float* weights;
  float* q_map;
  double* partial;  // [tiles][K]
};

template <int R>
struct WTile {
  static constexpr int SH = kTH + 2 * R;
  static constexpr int SW = kTW + 2 * R;
  static constexpr int SWP = (SW + 3) / 4 * 4;
  static constexpr int NV = (4 + 2 * R + 3) / 4;              // float4 loads per row segment
  static constexpr int KO = (SH * SW + kWT - 1) / kWT;       // staged pixels per thread
  static constexpr int P_FLOATS = 9 * SH * SWP;              // one date's products
  static constexpr int Z_FLOATS = 2 * 9 * kTH * kTW;         // Z (then G) of both dates
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
      for (int c = 0; c < 9; ++c) P[(c * T::SH + r) * T::SWP + x] = p[c];
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
__device__ __forceinline__ void load_row(const float* P, int c, int iy, int x0,
                                         float row[4 * WTile<R>::NV]) {
  using T = WTile<R>;
  const float4* src = reinterpret_cast<const float4*>(P + (c * T::SH + iy) * T::SWP + x0);
#pragma unroll
  for (int q = 0; q < T::NV; ++q) {
    const float4 v = src[q];
    row[4 * q] = v.x;
    row[4 * q + 1] = v.y;
    row[4 * q + 2] = v.z;
    row[4 * q + 3] = v.w;
  }
}

// Z_t of the thread's four outputs (tile row y, columns x0..x0+3), one channel
// at a time (a runtime loop: small code), into Zb[t][c][y][x0..x0+3].
template <int R>
__device__ __forceinline__ void window_cov(const float* P, const float* wsh, int t, int y,
                                           int x0, float* Zb) {
  constexpr int L = 2 * R + 1;
#pragma unroll 1
  for (int c = 0; c < 9; ++c) {
    float z[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int dy = 0; dy < L; ++dy) {
      float row[4 * WTile<R>::NV];
      load_row<R>(P, c, y + dy, x0, row);
#pragma unroll
      for (int dx = 0; dx < L; ++dx) {
        const float wk = wsh[dy * L + dx];
#pragma unroll
        for (int i = 0; i < 4; ++i) z[i] = fmaf(wk, row[i + dx], z[i]);
      }
    }
    *reinterpret_cast<float4*>(Zb + ((t * 9 + c) * kTH + y) * kTW + x0) =
        make_float4(z[0], z[1], z[2], z[3]);
  }
}

__device__ __forceinline__ float log_dd(const dd<float>& d) {
  // ln(hi + lo) = ln(hi) + ln(1 + lo/hi), |lo/hi| <= 2^-24
  return logf(d.hi) + d.lo / d.hi;
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

template <int R>
__global__ void __launch_bounds__(kWT, 3) k_wishart_fwd(WsArgs a) {
  using T = WTile<R>;
  constexpr int L = 2 * R + 1;
  extern __shared__ __align__(16) float smem[];
  float* P = smem;
  float* Zb = smem + T::P_FLOATS;
  float* wsh = Zb + T::Z_FLOATS;
  double* red = reinterpret_cast<double*>(wsh + 64);
  for (int i = threadIdx.x; i < L * L; i += blockDim.x) wsh[i] = a.weights[i];
  const int64_t tiles_x = (a.W + kTW - 1) / kTW;
  const int64_t tiles = tiles_x * ((a.H + kTH - 1) / kTH);
  const int y = threadIdx.x / (kTW / 4), x0 = (threadIdx.x % (kTW / 4)) * 4;
  const float six_ln2 = 4.15888308335967185650f;
  float2 v[T::KO][3];
  if ((int64_t)blockIdx.x < tiles) prefetch<R>(a, 0, blockIdx.x, v);
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t ty0 = (tile / tiles_x) * kTH, tx0 = (tile % tiles_x) * kTW;
#pragma unroll 1
    for (int t = 0; t < 2; ++t) {
      __syncthreads();  // everyone is done reading P
      store_products<R>(v, P);
      if (t == 0)
        prefetch<R>(a, 1, tile, v);
      else if (tile + gridDim.x < tiles)
        prefetch<R>(a, 0, tile + gridDim.x, v);
      __syncthreads();
      window_cov<R>(P, wsh, t, y, x0, Zb);
    }
    // per output: compensated log-dets of Z1, Z2 and Z1 + Z2 (own Zb entries only)
    double qsum = 0.0;
    const int64_t gy = ty0 + y;
#pragma unroll 1
    for (int i = 0; i < 4; ++i) {
      const int64_t gx = tx0 + x0 + i;
      if (gy >= a.H || gx >= a.W) continue;
      float z1[9], z2[9], z12[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        z1[c] = Zb[((0 * 9 + c) * kTH + y) * kTW + x0 + i];
        z2[c] = Zb[((1 * 9 + c) * kTH + y) * kTW + x0 + i];
        z12[c] = z1[c] + z2[c];
      }
      const float l1 = log_dd(det_comp<float>(z1));
      const float l2 = log_dd(det_comp<float>(z2));
      const float l12 = log_dd(det_comp<float>(z12));
      const float q = (l1 + l2) - 2.0f * l12 + six_ln2;
      if (a.q_map) a.q_map[gy * a.W + gx] = q;
      qsum += (double)q;
    }
    const double s = block_sum(qsum, red);
    if (threadIdx.x == 0) a.partial[tile] = s;
  }
}

template <int R>
__global__ void __launch_bounds__(kWT, 3) k_wishart_bwd(WsArgs a) {
  using T = WTile<R>;
  constexpr int L = 2 * R + 1;
  constexpr int K = L * L;
  extern __shared__ __align__(16) float smem[];
  float* P = smem;
  float* G = smem + T::P_FLOATS;  // [2][9][kTH][kTW]: Z_t, then the packed M_t
  float* wsh = G + T::Z_FLOATS;
  double* red = reinterpret_cast<double*>(wsh + 64);  // [4 warps][K]
  for (int i = threadIdx.x; i < K; i += blockDim.x) wsh[i] = a.weights[i];
  const int64_t tiles_x = (a.W + kTW - 1) / kTW;
  const int64_t tiles = tiles_x * ((a.H + kTH - 1) / kTH);
  const int y = threadIdx.x / (kTW / 4), x0 = (threadIdx.x % (kTW / 4)) * 4;
  float2 v[T::KO][3];
  // P holds one date at a time.  Per tile: stage date 0 (Z_0), stage date 1
  // (Z_1, then its correlation while still staged), stage date 0 again (its
  // correlation).  Each stage's loads were issued during the previous stage.
  if ((int64_t)blockIdx.x < tiles) prefetch<R>(a, 0, blockIdx.x, v);
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t ty0 = (tile / tiles_x) * kTH, tx0 = (tile % tiles_x) * kTW;
    // Z_0 and Z_1
#pragma unroll 1
    for (int t = 0; t < 2; ++t) {
      __syncthreads();
      store_products<R>(v, P);
      if (t == 0) prefetch<R>(a, 1, tile, v);
      else prefetch<R>(a, 0, tile, v);  // date 0 again, for its correlation
      __syncthreads();
      window_cov<R>(P, wsh, t, y, x0, G);
    }
    // per output: three compensated inverses, M_t = W_t - 2 W_12 in packed
    // gradient form written over the thread's own Z slots
    {
      const int64_t gy = ty0 + y;
#pragma unroll 1
      for (int i = 0; i < 4; ++i) {
        const int64_t gx = tx0 + x0 + i;
        float z1[9], z2[9], z12[9], w1[9], w2[9], w12[9], d;
#pragma unroll
        for (int c = 0; c < 9; ++c) {
          z1[c] = G[((0 * 9 + c) * kTH + y) * kTW + x0 + i];
          z2[c] = G[((1 * 9 + c) * kTH + y) * kTW + x0 + i];
          z12[c] = z1[c] + z2[c];
        }
        const bool inside = gy < a.H && gx < a.W;
        adjugate_inv_det_comp<float>(z1, w1, d);
        adjugate_inv_det_comp<float>(z2, w2, d);
        adjugate_inv_det_comp<float>(z12, w12, d);
#pragma unroll
        for (int c = 0; c < 9; ++c) {
          // packed M_t = W_t - 2 W_12; off-diagonal packed reals count twice
          const float two = (c == 0 || c == 5 || c == 8) ? 1.0f : 2.0f;
          G[((0 * 9 + c) * kTH + y) * kTW + x0 + i] = inside ? two * fmaf(-2.0f, w12[c], w1[c]) : 0.0f;
          G[((1 * 9 + c) * kTH + y) * kTW + x0 + i] = inside ? two * fmaf(-2.0f, w12[c], w2[c]) : 0.0f;
        }
      }
    }
    // dL/dw_k over this thread's four pixels: sum_t sum_c G_t[c](p) P_t[c](p + k);
    // P still holds date 1: correlate it first, then stage date 0.
    float acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0f;
#pragma unroll 1
    for (int step = 0; step < 2; ++step) {
      const int t = 1 - step;
      if (step == 1) {
        __syncthreads();
        store_products<R>(v, P);
        if (tile + gridDim.x < tiles) prefetch<R>(a, 0, tile + gridDim.x, v);
        __syncthreads();
      }
#pragma unroll 1
      for (int c = 0; c < 9; ++c) {
        const float4 gv = *reinterpret_cast<const float4*>(G + ((t * 9 + c) * kTH + y) * kTW + x0);
        const float gi[4] = {gv.x, gv.y, gv.z, gv.w};
#pragma unroll
        for (int dy = 0; dy < L; ++dy) {
          float row[4 * WTile<R>::NV];
          load_row<R>(P, c, y + dy, x0, row);
#pragma unroll
          for (int dx = 0; dx < L; ++dx)
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[dy * L + dx] = fmaf(gi[i], row[i + dx], acc[dy * L + dx]);
        }
      }
    }
    // fixed-order reduction of the K taps over the block
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double vsum = (double)acc[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) vsum += __shfl_down_sync(0xffffffffu, vsum, o);
      if (lane == 0) red[warp * K + k] = vsum;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
      double ssum = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) ssum += red[w * K + k];
      a.partial[tile * K + k] = ssum;
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
  return (WTile<R>::P_FLOATS + WTile<R>::Z_FLOATS + 64) * sizeof(float) + 8 * sizeof(double);
}
template <int R>
size_t bwd_smem() {
  constexpr int K = (2 * R + 1) * (2 * R + 1);
  return (WTile<R>::P_FLOATS + WTile<R>::Z_FLOATS + 64) * sizeof(float) + 4 * K * sizeof(double);
}

int64_t tile_count(int64_t H, int64_t W) {
  return ((W + kTW - 1) / kTW) * ((H + kTH - 1) / kTH);
}

template <typename Kern>
int launch_tiles(Kern kernel, size_t smem, const WsArgs& a, cudaStream_t s) {
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return ZINV_ERR_LAUNCH;
  }
  const int64_t tiles = tile_count(a.H, a.W);
  const int64_t blocks = cover_blocks(tiles * kWT, kWT);
  kernel<<<(unsigned)blocks, kWT, smem, s>>>(a);
  return launch_status();
}

// Shared argument checks; fills a and tiles.  Returns ZINV_OK or an error.
int prepare(const float* s1, const float* s2, int64_t H, int64_t W, int64_t plane_ld, int win,
            const float* weights, void* ws, size_t ws_bytes, WsArgs& a, DeviceInfo& di) {
  if (H < 1 || W < 1 || H > kMaxLd / W) return ZINV_ERR_ARG;
  if (win != 3 && win != 5 && win != 7) return ZINV_ERR_ARG;
  if (plane_ld < H * W || plane_ld > kMaxLd) return ZINV_ERR_ARG;
  if (!s1 || !s2 || !weights || !ws) return ZINV_ERR_ARG;
  if (!aligned(s1, 8) || !aligned(s2, 8) || !aligned(weights, 4) || !aligned(ws, 8))
    return ZINV_ERR_ARG;
  const size_t need = (size_t)tile_count(H, W) * (size_t)(win * win) * sizeof(double);
  if (ws_bytes < need) return ZINV_ERR_ARG;
  int rc = device_info(&di);
  if (rc != ZINV_OK) return rc;
  if (!device_accessible(s1) || !device_accessible(s2) || !device_accessible(weights) ||
      !device_accessible(ws))
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
    case 3: rc = launch_tiles(k_wishart_fwd<1>, fwd_smem<1>(), a, st); break;
    case 5: rc = launch_tiles(k_wishart_fwd<2>, fwd_smem<2>(), a, st); break;
    default: rc = launch_tiles(k_wishart_fwd<3>, fwd_smem<3>(), a, st); break;
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
constexpr int64_t kNoAllocTiles = 131072;  // one slot per 64 x 8 tile: 8192 x 8192 pixels
__device__ __align__(256) double g_noalloc_partials[kNoAllocTiles];

struct NoAllocScratch {
  std::once_flag once;
  cudaError_t err = cudaErrorNotReady;
  double* ptr = nullptr;
};
NoAllocScratch g_noalloc[kMaxDevices];
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
  NoAllocScratch& sc = g_noalloc[dev];
  std::call_once(sc.once, [&]() {
    sc.err = cudaGetSymbolAddress(reinterpret_cast<void**>(&sc.ptr), g_noalloc_partials);
    if (sc.err != cudaSuccess) cudaGetLastError();
  });
  if (sc.err != cudaSuccess || !sc.ptr) return ZINV_ERR_LAUNCH;
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
  a.partial = sc.ptr;  // every tile writes its own slot before the reduce reads it
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (win) {
    case 3: rc = launch_tiles(k_wishart_fwd<1>, fwd_smem<1>(), a, st); break;
    case 5: rc = launch_tiles(k_wishart_fwd<2>, fwd_smem<2>(), a, st); break;
    default: rc = launch_tiles(k_wishart_fwd<3>, fwd_smem<3>(), a, st); break;
  }
  if (rc != ZINV_OK) return rc;
  k_reduce_tiles<<<1, kRedThreads, 0, st>>>(a.partial, tiles, 1, nullptr, d_loss, 1);
  return launch_status();
}
