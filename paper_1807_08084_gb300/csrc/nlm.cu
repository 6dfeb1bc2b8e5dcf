// nlm.cu -- nonlocal-means filter of a packed covariance image with stochastic
// distances between the pixels' complex Wishart laws of L looks (the paper's
// motivating workload, §1: for every pixel, a 23 x 23 search window of 3x3
// Hermitian determinants or inverses; §1 lists these divergences among the
// uses of det Z and Z^-1).
//
// For pixels i, j the weight is w_ij = exp(-d(i, j) / h) over the in-image
// neighbours within the search radius, and Z'_i = sum_j w_ij Z_j / sum_j w_ij,
// with d one of (closed forms for equal looks, m = 3):
//   Bhattacharyya  d_B = L [ln det((Z_i + Z_j)/2) - (ln det Z_i + ln det Z_j)/2]
//                  (= L [ln det((Z_i^-1 + Z_j^-1)/2) + (ln det Z_i + ln det Z_j)/2],
//                  as Z_i^-1 + Z_j^-1 = Z_i^-1 (Z_i + Z_j) Z_j^-1),
//   Hellinger      d_H = 1 - exp(-d_B),
//   Kullback-Leibler (mean of both directions)
//                  d_KL = L [(tr(Z_i^-1 Z_j) + tr(Z_j^-1 Z_i))/2 - 3],
//   Renyi of order b in (0, 1) (mean of both directions)
//                  d_R = L/(1-b) [(ln det((1-b) Z_i + b Z_j) + ln det(b Z_i + (1-b) Z_j))/2
//                                 - (ln det Z_i + ln det Z_j)/2].
//
// Bhattacharyya and Hellinger, in base 2 with D_ij = det(Z_i + Z_j) and
// h_i = log2(det Z_i) / 2:  d_B = L ln2 t_ij,  t_ij = max(log2 D_ij - (3 + h_i) - h_j, 0)
// (det((Z_i + Z_j)/2) = D_ij / 8; t >= 0 in exact arithmetic, the clamp absorbs
// rounding), so w = 2^(-(L/h) t) and, for Hellinger, w = 2^(-(log2 e / h)(1 - 2^(-L t))).
// h_i is formed once per staged pixel (compensated route); per pair the work is
// D_ij -- 529 determinants per pixel for a 23 x 23 window -- one log2 and one
// or two exp2.  D_ij is computed either by Algorithm 2's cofactor expansion
// (Eq. adjoint_elements, Eq. detr: no division, no square root) or by
// Algorithm 1's Cholesky route (three square roots, two reciprocals);
// everything else is shared, so the two can be compared where arithmetic, not
// memory, sets the time.
// Renyi: the same staging; per pair the two convex combinations (1-b) Z_A +
// b Z_j and b Z_A + (1-b) Z_j (packed FMAs from the pre-scaled own matrices),
// both determinants by Algorithm 2 or 1, and w = 2^(-(L/((1-b) h)) t) with
// t = max((log2 D1 + log2 D2)/2 - h_i - h_j, 0).
// Kullback-Leibler: Z^-1 of every staged pixel by Algorithm 2 with compensated
// (Dot2) cofactors and det, once per staged pixel; per pair two traces of
// packed Hermitian products (nine FMAs each: tr(A B) = a a' + d d' + f f' +
// 2 (Re b Re b' + Im b Im b' + ...)) and one exp2.
//
// Tiles of 32 x 16 outputs, 256 threads (Kullback-Leibler up to radius 11:
// 32 x 32 outputs, 512 threads, as its 18 planes leave room for one CTA per
// SM; 16 warps per SM instead of 8 took its 1024^2 launch from 1.155 to
// 0.916 ms); each thread owns two vertically
// adjacent outputs A and B, held as the two halves of packed f32x2 values:
// every neighbour loaded from shared memory serves both outputs' pairs (one
// packed sum Z_A + Z_j | Z_B + Z_j, one packed determinant by Algorithm 2, one
// packed weighted accumulation).  The rows of the two windows are walked
// together; a row outside one output's window gets weight 0 for that output.
// The tile plus a halo of the search radius (Z and h, or Z and Z^-1) sits in
// shared memory.
#include "common.cuh"
#include "pixel.cuh"

namespace zinv {
namespace {

constexpr int kNW = 32;  // tile width
constexpr int kNH = 16;  // tile height: 8 row pairs, 256 threads

// Distances (the values of nlm_stochastic's `distance`).
constexpr int kBhattacharyya = 0, kHellinger = 1, kKullbackLeibler = 2, kRenyi = 3;

struct NlmArgs {
  const float* z;
  int64_t H, W, ld;
  int radius;
  float p;      // Bhattacharyya: L / h; Kullback-Leibler: L log2(e) / h; Renyi: L / ((1-b) h)
  float looks;  // Hellinger: L
  float qh;     // Hellinger: log2(e) / h
  float b, b1;  // Renyi: the order b and 1 - b
  float* out;
};

// Shared-memory planes per staged pixel: Z and h, or Z and Z^-1.
template <int DIST>
constexpr int nlm_planes() {
  return DIST == kKullbackLeibler ? 18 : 10;
}

// Tile height and threads: Kullback-Leibler's 18 planes leave room for one CTA
// per SM, which then takes a 32 x 32 tile with 512 threads (radius <= 11).
template <int RAD, int DIST>
struct NlmTile {
  static constexpr int TH = (DIST == kKullbackLeibler && RAD <= 11) ? 32 : kNH;
  static constexpr int NT = kNW / 2 * TH;
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
  const float q = l00 * l11 * l22;
  return q * q;
}

// sum_k c_k cof_k(x) e_k over the packed entries (c_k = 2 off the diagonal):
// the first-order change of det(x) when x moves by e (d det = tr(adj dZ)),
// with the cofactors of Eq. adjoint_elements in plain arithmetic.
__device__ __forceinline__ float2 det_first_order(const float2 x[9], const float2 e[9]) {
  const float2 a = x[0], br = x[1], bi = x[2], cr = x[3], ci = x[4];
  const float2 d = x[5], er = x[6], ei = x[7], f = x[8];
  const float2 cof[9] = {
      fma_rn(-er, er, fma_rn(-ei, ei, mul_rn(d, f))),    // a_c
      fma_rn(-br, f, fma_rn(ci, ei, mul_rn(cr, er))),    // Re b_c
      fma_rn(-bi, f, fma_rn(-cr, ei, mul_rn(ci, er))),   // Im b_c
      fma_rn(-cr, d, fma_rn(-bi, ei, mul_rn(br, er))),   // Re c_c
      fma_rn(-ci, d, fma_rn(bi, er, mul_rn(br, ei))),    // Im c_c
      fma_rn(-cr, cr, fma_rn(-ci, ci, mul_rn(a, f))),    // d_c
      fma_rn(-a, er, fma_rn(ci, bi, mul_rn(cr, br))),    // Re e_c
      fma_rn(-a, ei, fma_rn(-cr, bi, mul_rn(ci, br))),   // Im e_c
      fma_rn(-br, br, fma_rn(-bi, bi, mul_rn(a, d)))};   // f_c
  float2 s = mul_rn(cof[0], e[0]);
#pragma unroll
  for (int k = 1; k < 9; ++k) {
    const float two = (k == 5 || k == 8) ? 1.0f : 2.0f;
    s = fma_rn(mul_rn(make_float2(two, two), cof[k]), e[k], s);
  }
  return s;
}

template <int METHOD, int RAD, int DIST>
__global__ void __launch_bounds__(NlmTile<RAD, DIST>::NT, 512 / NlmTile<RAD, DIST>::NT)
    k_nlm(NlmArgs a) {
  constexpr int TH = NlmTile<RAD, DIST>::TH, NT = NlmTile<RAD, DIST>::NT;
  constexpr int SW = kNW + 2 * RAD, SH = TH + 2 * RAD;
  constexpr bool KL = DIST == kKullbackLeibler;
  extern __shared__ __align__(16) float smem[];
  float* Zs = smem;                // [9][SH][SW]
  float* Hs = smem + 9 * SH * SW;  // [SH][SW] half log2-dets, or [9][SH][SW] Z^-1 (KL)
  const int64_t n = a.H * a.W;
  const int64_t tiles_x = (a.W + kNW - 1) / kNW;
  const int64_t tiles = tiles_x * ((a.H + TH - 1) / TH);
  const int tx = threadIdx.x % kNW, ty = 2 * (threadIdx.x / kNW);
  const float inv_ln2 = 1.44269504088896340736f;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int64_t y0 = (t / tiles_x) * TH, x0 = (t % tiles_x) * kNW;
    __syncthreads();
    for (int i = threadIdx.x; i < SH * SW; i += NT) {
      const int sy = i / SW, sx = i - (i / SW) * SW;
      const int64_t gy = y0 - RAD + sy, gx = x0 - RAD + sx;
      if (gy < 0 || gy >= a.H || gx < 0 || gx >= a.W) continue;  // never read
      const int64_t q = gy * a.W + gx;
      float v[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        v[c] = __ldg(a.z + c * a.ld + q);
        Zs[(c * SH + sy) * SW + sx] = v[c];
      }
      if constexpr (KL) {
        float w[9], dt;
        adjugate_inv_det_comp<float>(v, w, dt);
#pragma unroll
        for (int c = 0; c < 9; ++c) Hs[(c * SH + sy) * SW + sx] = w[c];
      } else {
        const dd<float> dt = det_comp<float>(v);
        Hs[sy * SW + sx] = 0.5f * (log2f(dt.hi) + (dt.lo / dt.hi) * inv_ln2);
      }
    }
    __syncthreads();
    const int64_t gyA = y0 + ty, gx = x0 + tx;
    if (gyA >= a.H || gx >= a.W) continue;
    const bool hasB = gyA + 1 < a.H;
    const int cy = ty + RAD, cx = tx + RAD;  // shared-memory position of output A
    // own values of A | B: Z, and for KL Z and Z^-1 with the off-diagonal
    // packed reals doubled (the trace's factor 2, exact)
    float2 zi[9], acc[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      const float za = Zs[(c * SH + cy) * SW + cx];
      zi[c] = make_float2(za, hasB ? Zs[(c * SH + cy + 1) * SW + cx] : za);
      acc[c] = make_float2(0.0f, 0.0f);
    }
    float2 ii2[KL ? 9 : 1], zi2[KL ? 9 : 1];
    constexpr bool RY = DIST == kRenyi;
    float2 zb1[RY ? 9 : 1], zb[RY ? 9 : 1];  // Renyi: (1-b) Z and b Z of A | B
    float kA = 0.0f, kB = 0.0f;
    if constexpr (RY) {
      const float2 b2 = make_float2(a.b, a.b), b12 = make_float2(a.b1, a.b1);
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        zb1[c] = mul_rn(b12, zi[c]);
        zb[c] = mul_rn(b2, zi[c]);
      }
      kA = Hs[cy * SW + cx];
      kB = hasB ? Hs[(cy + 1) * SW + cx] : kA;
    } else if constexpr (KL) {
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        const float two = (c == 0 || c == 5 || c == 8) ? 1.0f : 2.0f;
        const float ia = Hs[(c * SH + cy) * SW + cx];
        ii2[c] = make_float2(two * ia, two * (hasB ? Hs[(c * SH + cy + 1) * SW + cx] : ia));
        zi2[c] = make_float2(two * zi[c].x, two * zi[c].y);
      }
    } else {
      kA = 3.0f + Hs[cy * SW + cx];
      kB = hasB ? 3.0f + Hs[(cy + 1) * SW + cx] : kA;
    }
    // in-image rows of the two windows (B's starts one row later) and columns
    const int64_t a_lo = gyA - RAD < 0 ? 0 : gyA - RAD;
    const int64_t a_hi = gyA + RAD >= a.H ? a.H - 1 : gyA + RAD;
    const int64_t b_lo = gyA + 1 - RAD < 0 ? 0 : gyA + 1 - RAD;
    const int64_t b_hi = hasB ? (gyA + 1 + RAD >= a.H ? a.H - 1 : gyA + 1 + RAD) : a_hi;
    const int dx0 = (int)(gx - RAD < 0 ? -gx : -RAD);
    const int dx1 = (int)(gx + RAD >= a.W ? a.W - 1 - gx : RAD);
    const float np = -a.p, nl = -a.looks, nq = -a.qh;
    float2 ws = make_float2(0.0f, 0.0f);
    for (int64_t gy = a_lo; gy <= b_hi; ++gy) {
      const float2 m = make_float2(gy <= a_hi ? 1.0f : 0.0f, hasB && gy >= b_lo ? 1.0f : 0.0f);
      const int srow = (int)(gy - y0) + RAD;
      const float* zrow = Zs + srow * SW + cx;
      const float* hrow = Hs + srow * SW + cx;
      // two neighbours per iteration: their dependent chains (sum, det, log2,
      // exp2) interleave (1.059 -> 0.996 ms for the 1024^2 adjugate filter)
#pragma unroll 2
      for (int dx = dx0; dx <= dx1; ++dx) {
        float zj[9];
        float2 w;
        if constexpr (KL) {
          // t = (tr(Z_A^-1 Z_j) + tr(Z_j^-1 Z_A)) / 2 - 3, both traces in
          // channel order as packed FMAs
          float ij[9];
#pragma unroll
          for (int c = 0; c < 9; ++c) {
            zj[c] = zrow[c * SH * SW + dx];
            ij[c] = hrow[c * SH * SW + dx];
          }
          float2 t1 = mul_rn(ii2[0], make_float2(zj[0], zj[0]));
          float2 t2 = mul_rn(zi2[0], make_float2(ij[0], ij[0]));
#pragma unroll
          for (int c = 1; c < 9; ++c) {
            t1 = fma_rn(ii2[c], make_float2(zj[c], zj[c]), t1);
            t2 = fma_rn(zi2[c], make_float2(ij[c], ij[c]), t2);
          }
          const float2 tk = fma_rn(make_float2(0.5f, 0.5f), add_rn(t1, t2),
                                   make_float2(-3.0f, -3.0f));
          w = mul_rn(make_float2(exp2f(np * fmaxf(tk.x, 0.0f)), exp2f(np * fmaxf(tk.y, 0.0f))),
                     m);
        } else if constexpr (RY) {
          float2 m1[9], m2[9];
#pragma unroll
          for (int c = 0; c < 9; ++c) {
            zj[c] = zrow[c * SH * SW + dx];
            m1[c] = fma_rn(make_float2(a.b, a.b), make_float2(zj[c], zj[c]), zb1[c]);
            m2[c] = fma_rn(make_float2(a.b1, a.b1), make_float2(zj[c], zj[c]), zb[c]);
          }
          float2 D1, D2;
          if constexpr (METHOD == 0) {
            D1 = det_adjugate<float2>(m1);
            D2 = det_adjugate<float2>(m2);
          } else {
            float x1[9], x2[9], x3[9], x4[9];
#pragma unroll
            for (int c = 0; c < 9; ++c)
              x1[c] = m1[c].x, x2[c] = m1[c].y, x3[c] = m2[c].x, x4[c] = m2[c].y;
            D1 = make_float2(det_cholesky(x1), det_cholesky(x2));
            D2 = make_float2(det_cholesky(x3), det_cholesky(x4));
          }
          const float hj = hrow[dx];
          const float ta = fmaxf(0.5f * (__log2f(D1.x) + __log2f(D2.x)) - (kA + hj), 0.0f);
          const float tb = fmaxf(0.5f * (__log2f(D1.y) + __log2f(D2.y)) - (kB + hj), 0.0f);
          w = mul_rn(make_float2(exp2f(np * ta), exp2f(np * tb)), m);
        } else {
          float ta, tb;
          if constexpr (METHOD == 2) {
            // compensated: the pair sum exactly as hi + lo, det(hi) by Dot2,
            // plus the first-order term of lo, sum_k c_k cof_k(hi) lo_k
            // (c_k = 2 off the diagonal: the gradient of det in packed form)
            float2 hi[9], lo[9];
#pragma unroll
            for (int c = 0; c < 9; ++c) {
              zj[c] = zrow[c * SH * SW + dx];
              two_sum(zi[c], make_float2(zj[c], zj[c]), hi[c], lo[c]);
            }
            const dd<float2> D = det_comp<float2>(hi);
            const float2 dlo = add_rn(D.lo, det_first_order(hi, lo));
            const float hj = hrow[dx];
            // log2(hi + lo) = log2 hi + lo / (hi ln2) to first order; the lo / hi
            // term is ~u, so the fast division and log2 (2^-21.4 absolute)
            // cost nothing against the determinant's own error bound
            ta = fmaxf(__log2f(D.hi.x) + __fdividef(dlo.x, D.hi.x) * inv_ln2 - (kA + hj), 0.0f);
            tb = fmaxf(__log2f(D.hi.y) + __fdividef(dlo.y, D.hi.y) * inv_ln2 - (kB + hj), 0.0f);
          } else {
            float2 zs[9];
#pragma unroll
            for (int c = 0; c < 9; ++c) {
              zj[c] = zrow[c * SH * SW + dx];
              zs[c] = add_rn(zi[c], make_float2(zj[c], zj[c]));
            }
            float2 D;
            if constexpr (METHOD == 0) {
              D = det_adjugate<float2>(zs);
            } else {
              float xa[9], xb[9];
#pragma unroll
              for (int c = 0; c < 9; ++c) xa[c] = zs[c].x, xb[c] = zs[c].y;
              D = make_float2(det_cholesky(xa), det_cholesky(xb));
            }
            const float hj = hrow[dx];
            ta = fmaxf(__log2f(D.x) - (kA + hj), 0.0f);
            tb = fmaxf(__log2f(D.y) - (kB + hj), 0.0f);
          }
          if constexpr (DIST == kHellinger) {
            // d_H = 1 - 2^(-L t), w = 2^(-(log2 e / h) d_H)
            const float ha = 1.0f - exp2f(nl * ta), hb = 1.0f - exp2f(nl * tb);
            w = mul_rn(make_float2(exp2f(nq * ha), exp2f(nq * hb)), m);
          } else {
            w = mul_rn(make_float2(exp2f(np * ta), exp2f(np * tb)), m);
          }
        }
#pragma unroll
        for (int c = 0; c < 9; ++c) acc[c] = fma_rn(w, make_float2(zj[c], zj[c]), acc[c]);
        ws = add_rn(ws, w);
      }
    }
    const int64_t q = gyA * a.W + gx;
    const float ia = 1.0f / ws.x;
#pragma unroll
    for (int c = 0; c < 9; ++c) a.out[c * n + q] = acc[c].x * ia;
    if (hasB) {
      const float ib = 1.0f / ws.y;
#pragma unroll
      for (int c = 0; c < 9; ++c) a.out[c * n + q + a.W] = acc[c].y * ib;
    }
  }
}

template <int METHOD, int RAD, int DIST>
int launch_nlm(const NlmArgs& a, cudaStream_t s) {
  constexpr int TH = NlmTile<RAD, DIST>::TH, NT = NlmTile<RAD, DIST>::NT;
  constexpr int SW = kNW + 2 * RAD, SH = TH + 2 * RAD;
  const size_t smem = (size_t)nlm_planes<DIST>() * SH * SW * sizeof(float);
  auto k = k_nlm<METHOD, RAD, DIST>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return ZINV_ERR_LAUNCH;
  }
  const int64_t tiles = ((a.W + kNW - 1) / kNW) * ((a.H + TH - 1) / TH);
  const int64_t blocks = cover_blocks(tiles * NT, NT);
  k<<<(unsigned)blocks, NT, smem, s>>>(a);
  return launch_status();
}

template <int METHOD, int DIST>
int dispatch_nlm(const NlmArgs& a, cudaStream_t s) {
  switch (a.radius) {
    case 1: return launch_nlm<METHOD, 1, DIST>(a, s);
    case 2: return launch_nlm<METHOD, 2, DIST>(a, s);
    case 3: return launch_nlm<METHOD, 3, DIST>(a, s);
    case 5: return launch_nlm<METHOD, 5, DIST>(a, s);
    case 7: return launch_nlm<METHOD, 7, DIST>(a, s);
    case 11: return launch_nlm<METHOD, 11, DIST>(a, s);
    case 15: return launch_nlm<METHOD, 15, DIST>(a, s);
  }
  return ZINV_ERR_ARG;
}

}  // namespace
}  // namespace zinv

extern "C" int nlm_stochastic(const float* z, int64_t H, int64_t W, int64_t ld, int radius,
                              float looks, float h, int distance, float order, int method,
                              float* z_out, void* stream) {
  using namespace zinv;
  if (H < 1 || W < 1 || H > kMaxLd / W || ld < H * W || ld > kMaxLd) return ZINV_ERR_ARG;
  if (radius != 1 && radius != 2 && radius != 3 && radius != 5 && radius != 7 &&
      radius != 11 && radius != 15)
    return ZINV_ERR_ARG;
  if (!(looks > 0.0f) || !(h > 0.0f) || isinf(looks) || isinf(h)) return ZINV_ERR_ARG;
  if (distance != kBhattacharyya && distance != kHellinger && distance != kKullbackLeibler &&
      distance != kRenyi)
    return ZINV_ERR_ARG;
  if (distance == kRenyi && !(order > 0.0f && order < 1.0f)) return ZINV_ERR_ARG;
  if (method != 0 && method != 1 && method != 2) return ZINV_ERR_ARG;
  if (distance == kKullbackLeibler && method != 0) return ZINV_ERR_ARG;  // no pair det
  if (method == 2 && distance != kBhattacharyya && distance != kHellinger) return ZINV_ERR_ARG;
  if (!z || !z_out || !aligned(z, 4) || !aligned(z_out, 4)) return ZINV_ERR_ARG;
  DeviceInfo di;
  int rc = device_info(&di);
  if (rc != ZINV_OK) return rc;
  if (!device_accessible(z) || !device_accessible(z_out)) return ZINV_ERR_ARG;
  const double log2e = 1.44269504088896340736;
  NlmArgs a{z, H, W, ld, radius, 0.0f, looks, (float)(log2e / h), 0.0f, 0.0f, z_out};
  a.p = distance == kKullbackLeibler ? (float)(looks * log2e / h) : looks / h;
  if (distance == kRenyi) {
    a.b = order;
    a.b1 = (float)(1.0 - (double)order);
    a.p = (float)((double)looks / ((1.0 - (double)order) * (double)h));
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (distance) {
    case kBhattacharyya:
      return method == 0   ? dispatch_nlm<0, kBhattacharyya>(a, s)
             : method == 1 ? dispatch_nlm<1, kBhattacharyya>(a, s)
                           : dispatch_nlm<2, kBhattacharyya>(a, s);
    case kHellinger:
      return method == 0   ? dispatch_nlm<0, kHellinger>(a, s)
             : method == 1 ? dispatch_nlm<1, kHellinger>(a, s)
                           : dispatch_nlm<2, kHellinger>(a, s);
    case kRenyi:
      return method == 0 ? dispatch_nlm<0, kRenyi>(a, s) : dispatch_nlm<1, kRenyi>(a, s);
    default:
      return dispatch_nlm<0, kKullbackLeibler>(a, s);
  }
}

extern "C" int nlm_wishart(const float* z, int64_t H, int64_t W, int64_t ld, int radius,
                           float looks, float h, int method, float* z_out, void* stream) {
  return nlm_stochastic(z, H, W, ld, radius, looks, h, zinv::kBhattacharyya, 0.5f, method,
                        z_out, stream);
}
