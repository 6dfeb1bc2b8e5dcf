// pixel.cuh -- per-pixel device arithmetic: the adjugate inverse+det (Alg. 2 of
// the paper) in plain FP32, FMA-compensated FP32 and FP64; the Cholesky route
// (Alg. 1); status bits.  Nine packed reals per pixel in the paper's letter
// order (§2.1): x = {a, Re b, Im b, Re c, Im c, d, Re e, Im e, f}.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "zinv.h"

namespace zinv {

// ---------------------------------------------------------------------------
// Alg. 2 (§3.1): cofactors (Eq. adjoint_elements), det (Eq. detr), t = 1/det,
// Z^-1 = t adj(Z) (Eq. inv_adjoint).  T = float or double.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

template <typename T>
__device__ __forceinline__ void adjugate_inv_det(const T x[9], T w[9], T& det) {
  const T a = x[0], br = x[1], bi = x[2], cr = x[3], ci = x[4];
  const T d = x[5], er = x[6], ei = x[7], f = x[8];
  // real diagonal cofactors: a_c = d f - |e|^2, d_c = a f - |c|^2, f_c = a d - |b|^2
  const T ac = d * f - (er * er + ei * ei);
  const T dc = a * f - (cr * cr + ci * ci);
  const T fc = a * d - (br * br + bi * bi);
  // complex upper cofactors: b_c = c conj(e) - b f, c_c = b e - c d, e_c = c conj(b) - a e
  const T bcr = (cr * er + ci * ei) - br * f;
  const T bci = (ci * er - cr * ei) - bi * f;
  const T ccr = (br * er - bi * ei) - cr * d;
  const T cci = (br * ei + bi * er) - ci * d;
  const T ecr = (cr * br + ci * bi) - a * er;
  const T eci = (ci * br - cr * bi) - a * ei;
  // det = a a_c + Re(conj(b) b_c) + Re(conj(c) c_c)
  det = a * ac + br * bcr + bi * bci + cr * ccr + ci * cci;
  const T t = recip(det);
  w[0] = t * ac;
  w[1] = t * bcr;
  w[2] = t * bci;
  w[3] = t * ccr;
  w[4] = t * cci;
  w[5] = t * dc;
  w[6] = t * ecr;
  w[7] = t * eci;
  w[8] = t * fc;
}

// ---------------------------------------------------------------------------
// Compensated arithmetic (T = float for the compensated mode, T = double for
// the flagged-pixel recompute).  Error-free transforms: TwoProduct by FMA (the
// rounding error of a*b is fma(a, b, -p) exactly) and Knuth's TwoSum; Dot2 of
// Ogita, Rump and Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput.
// 2005) accumulates the products' and sums' errors separately, so the result is
// as accurate as if computed in twice the working precision.  The *_rn
// intrinsics keep nvcc from contracting or re-associating them.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float rcp_rn(float a) { return __frcp_rn(a); }
__device__ __forceinline__ double rcp_rn(double a) { return __drcp_rn(a); }

// Packed pairs (Blackwell's f32x2 instructions): each half rounds exactly as
// the scalar operation; a - b is fma(b, -1, a), one rounding of the exact
// difference.  With these the compensated routines below also run on float2,
// two pixels per instruction.
__device__ __forceinline__ float2 mul_rn(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add_rn(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub_rn(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
__device__ __forceinline__ float2 fma_rn(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 operator-(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 rcp_rn(float2 a) { return make_float2(__frcp_rn(a.x), __frcp_rn(a.y)); }

// 1 in the arithmetic type of x.
__device__ __forceinline__ float one_like(float) { return 1.0f; }
__device__ __forceinline__ double one_like(double) { return 1.0; }
__device__ __forceinline__ float2 one_like(float2) { return make_float2(1.0f, 1.0f); }

template <typename T>
struct dd {
  T hi, lo;  // value = hi + lo, |lo| <= ulp(hi)/2
};

template <typename T>
__device__ __forceinline__ void two_prod(T a, T b, T& p, T& e) {
  p = mul_rn(a, b);
  e = fma_rn(a, b, -p);
}

template <typename T>
__device__ __forceinline__ void two_sum(T a, T b, T& s, T& e) {
  s = add_rn(a, b);
  const T z = sub_rn(s, a);
  e = add_rn(sub_rn(a, sub_rn(s, z)), sub_rn(b, z));
}

// x0*y0 + x1*y1 + x2*y2 by Dot2, returned unevaluated as hi + lo.
template <typename T>
__device__ __forceinline__ dd<T> dot3(T x0, T y0, T x1, T y1, T x2, T y2) {
  T p, s, h, r, q;
  two_prod(x0, y0, p, s);
  two_prod(x1, y1, h, r);
  two_sum(p, h, p, q);
  s = add_rn(s, add_rn(q, r));
  two_prod(x2, y2, h, r);
  two_sum(p, h, p, q);
  s = add_rn(s, add_rn(q, r));
  dd<T> out;
  two_sum(p, s, out.hi, out.lo);
  return out;
}

// Alg. 2 with every cofactor and the det by Dot2 (the 2x2 products of Eq.
// adjoint_elements are formed exactly, so cancellation in them costs nothing).
template <typename T>
__device__ __forceinline__ void adjugate_inv_det_comp(const T x[9], T w[9], T& det) {
  const T a = x[0], br = x[1], bi = x[2], cr = x[3], ci = x[4];
  const T d = x[5], er = x[6], ei = x[7], f = x[8];
  const dd<T> ac = dot3(d, f, -er, er, -ei, ei);
  const dd<T> dc = dot3(a, f, -cr, cr, -ci, ci);
  const dd<T> fc = dot3(a, d, -br, br, -bi, bi);
  const dd<T> bcr = dot3(cr, er, ci, ei, -br, f);
  const dd<T> bci = dot3(ci, er, -cr, ei, -bi, f);
  const dd<T> ccr = dot3(br, er, -bi, ei, -cr, d);
  const dd<T> cci = dot3(br, ei, bi, er, -ci, d);
  const dd<T> ecr = dot3(cr, br, ci, bi, -a, er);
  const dd<T> eci = dot3(ci, br, -cr, bi, -a, ei);
  // det by Dot2 over the five products with the cofactors' high parts; the
  // products with their low parts are small and join the error accumulator.
  T p, s, h, r, q;
  two_prod(a, ac.hi, p, s);
  s = fma_rn(a, ac.lo, s);
  const T xs[4] = {br, bi, cr, ci};
  const dd<T> ys[4] = {bcr, bci, ccr, cci};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    two_prod(xs[k], ys[k].hi, h, r);
    two_sum(p, h, p, q);
    s = add_rn(s, add_rn(q, r));
    s = fma_rn(xs[k], ys[k].lo, s);
  }
  T dhi, dlo;
  two_sum(p, s, dhi, dlo);
  det = dhi;
  // t ~ 1/(dhi + dlo): the correctly rounded reciprocal plus one Newton-type
  // correction using its exact residual 1 - dhi*t and the det's low part.
  T t = rcp_rn(dhi);
  const T res = fma_rn(-dhi, t, one_like(dhi));
  t = fma_rn(t, fma_rn(-dlo, t, res), t);
  const dd<T> cof[9] = {ac, bcr, bci, ccr, cci, dc, ecr, eci, fc};
#pragma unroll
  for (int k = 0; k < 9; ++k) w[k] = fma_rn(cof[k].hi, t, mul_rn(cof[k].lo, t));
}

// det alone by the compensated route: the first-column cofactors a_c, b_c, c_c
// (Eq. adjoint_elements) and Eq. detr, all by Dot2; returned as hi + lo.
template <typename T>
__device__ __forceinline__ dd<T> det_comp(const T x[9]) {
  const T a = x[0], br = x[1], bi = x[2], cr = x[3], ci = x[4];
  const T d = x[5], er = x[6], ei = x[7], f = x[8];
  const dd<T> ac = dot3(d, f, -er, er, -ei, ei);
  const dd<T> bcr = dot3(cr, er, ci, ei, -br, f);
  const dd<T> bci = dot3(ci, er, -cr, ei, -bi, f);
  const dd<T> ccr = dot3(br, er, -bi, ei, -cr, d);
  const dd<T> cci = dot3(br, ei, bi, er, -ci, d);
  T p, s, h, r, q;
  two_prod(a, ac.hi, p, s);
  s = fma_rn(a, ac.lo, s);
  const T xs[4] = {br, bi, cr, ci};
  const dd<T> ys[4] = {bcr, bci, ccr, cci};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    two_prod(xs[k], ys[k].hi, h, r);
    two_sum(p, h, p, q);
    s = add_rn(s, add_rn(q, r));
    s = fma_rn(xs[k], ys[k].lo, s);
  }
  dd<T> out;
  two_sum(p, s, out.hi, out.lo);
  return out;
}

// det alone by Alg. 2's first-column cofactor expansion (the a_c, b_c, c_c of
// Eq. adjoint_elements in Eq. detr), plain FP32.  T = float, or float2 for two
// matrices at once; every operation is an explicit product or FMA, so both
// forms round alike.
template <typename T>
__device__ __forceinline__ T det_adjugate(const T x[9]) {
  const T a = x[0], br = x[1], bi = x[2], cr = x[3], ci = x[4];
  const T d = x[5], er = x[6], ei = x[7], f = x[8];
  const T ac = fma_rn(-er, er, fma_rn(-ei, ei, mul_rn(d, f)));   // d f - |e|^2
  const T bcr = fma_rn(-br, f, fma_rn(cr, er, mul_rn(ci, ei)));  // Re(c conj(e)) - Re(b) f
  const T bci = fma_rn(-bi, f, fma_rn(ci, er, mul_rn(-cr, ei)));
  const T ccr = fma_rn(-cr, d, fma_rn(br, er, mul_rn(-bi, ei)));
  const T cci = fma_rn(-ci, d, fma_rn(br, ei, mul_rn(bi, er)));
  return fma_rn(ci, cci, fma_rn(cr, ccr, fma_rn(bi, bci, fma_rn(br, bcr, mul_rn(a, ac)))));
}

// ln det, from hi + lo: ln(hi) + ln(1 + lo/hi) with |lo/hi| <= 2^-24.
__device__ __forceinline__ float log_dd(const dd<float>& d) {
  return logf(d.hi) + __fdividef(d.lo, d.hi);
}
__device__ __forceinline__ float2 log_dd(const dd<float2>& d) {
  return make_float2(log_dd(dd<float>{d.hi.x, d.lo.x}), log_dd(dd<float>{d.hi.y, d.lo.y}));
}

// ---------------------------------------------------------------------------
// Alg. 1 (§2.2), Cholesky route, FP32 with correctly rounded sqrt and
// reciprocal.  Z = L L^H, L lower triangular with real positive diagonal:
//   l00 = sqrt(a), l10 = conj(b)/l00, l20 = conj(c)/l00,
//   l11 = sqrt(d - |l10|^2), l21 = (conj(e) - l20 conj(l10)) / l11,
//   l22 = sqrt(f - |l20|^2 - |l21|^2);
// T = L^-1 (lower triangular), det = (l00 l11 l22)^2, Z^-1 = T^H T.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cholesky_inv_det(const float x[9], float w[9], float& det) {
  const float a = x[0], br = x[1], bi = x[2], cr = x[3], ci = x[4];
  const float d = x[5], er = x[6], ei = x[7], f = x[8];
  const float l00 = __fsqrt_rn(a);
  const float v0 = __frcp_rn(l00);
  const float l10r = br * v0, l10i = -bi * v0;
  const float l20r = cr * v0, l20i = -ci * v0;
  const float l11 = __fsqrt_rn(d - (l10r * l10r + l10i * l10i));
  const float v1 = __frcp_rn(l11);
  // conj(e) - l20 conj(l10)
  const float nr = er - (l20r * l10r + l20i * l10i);
  const float ni = -ei - (l20i * l10r - l20r * l10i);
  const float l21r = nr * v1, l21i = ni * v1;
  const float l22 = __fsqrt_rn(f - (l20r * l20r + l20i * l20i) - (l21r * l21r + l21i * l21i));
  const float v2 = __frcp_rn(l22);
  // T = L^-1: t00 = v0, t11 = v1, t22 = v2, t10 = -l10 v0 v1, t21 = -l21 v1 v2,
  // t20 = v2 v0 (l21 l10 v1 - l20)
  const float v01 = v0 * v1, v12 = v1 * v2, v02 = v0 * v2;
  const float t10r = -l10r * v01, t10i = -l10i * v01;
  const float t21r = -l21r * v12, t21i = -l21i * v12;
  const float pr = (l21r * l10r - l21i * l10i) * v1 - l20r;
  const float pi = (l21r * l10i + l21i * l10r) * v1 - l20i;
  const float t20r = pr * v02, t20i = pi * v02;
  const float ld = l00 * l11 * l22;
  det = ld * ld;
  // Z^-1 = T^H T (upper triangle)
  w[0] = v0 * v0 + (t10r * t10r + t10i * t10i) + (t20r * t20r + t20i * t20i);
  // conj(t10) t11 + conj(t20) t21
  w[1] = t10r * v1 + (t20r * t21r + t20i * t21i);
  w[2] = -t10i * v1 + (t20r * t21i - t20i * t21r);
  // conj(t20) t22
  w[3] = t20r * v2;
  w[4] = -t20i * v2;
  w[5] = v1 * v1 + (t21r * t21r + t21i * t21i);
  // conj(t21) t22
  w[6] = t21r * v2;
  w[7] = -t21i * v2;
  w[8] = v2 * v2;
}

// ---------------------------------------------------------------------------
// Flagged-pixel recompute (not in the paper; it follows its stability
// discussion in §3.3).  Hadamard's inequality gives det/(a d f) in (0, 1] for
// positive definite Z; a small ratio means cancellation ate the FP32 digits.
// !(>) also catches NaN and det <= 0.  A det whose magnitude is outside
// [2^-100, 2^100) is flagged too: det scales with the cube of the entries, so
// for entries beyond about 1e+-10 the terms of the expansion or det itself
// leave the FP32 normal range (underflow loses their digits; overflow or 1/det
// out of range ruins Z^-1, although Z^-1 is representable); FP64's range
// covers such pixels.  Inside the band every term is normal down to 2^-26 of
// det, so the FP32 results are exact multiples of the unscaled ones.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool needs_recompute(float det, const float x[9], float tau) {
  const unsigned e = (__float_as_uint(det) >> 23) & 0xffu;  // biased exponent of |det|
  return !(det > tau * (x[0] * x[5] * x[8])) || e - 27u >= 200u;
}

// The compensated route in FP64 on the FP32 inputs: their products and the
// Dot2 sums are exact enough that only the final FP32 rounding remains, even
// where the plain FP64 route would lose u64*cond^2.  Returns the pixel's status
// bits (RECOMPUTED, and NOT_PD from the FP64 det).
__device__ __forceinline__ uint32_t recompute_f64(const float x[9], float w[9], float& det) {
  double xd[9], wd[9], det64;
#pragma unroll
  for (int k = 0; k < 9; ++k) xd[k] = (double)x[k];
  adjugate_inv_det_comp<double>(xd, wd, det64);
#pragma unroll
  for (int k = 0; k < 9; ++k) w[k] = __double2float_rn(wd[k]);
  det = __double2float_rn(det64);
  uint32_t st = ZINV_PIX_RECOMPUTED;
  if (!(det64 > 0.0) || !isfinite(det64)) st |= ZINV_PIX_NOT_PD;
  return st;
}

// ---------------------------------------------------------------------------
// Dispatch over the algorithm variants; returns the pixel's ZINV_PIX_* bits.
// The FP64 variants recompute a flagged pixel inline here (one-pixel paths);
// the four-pixel kernel queues them instead (zinv_det.cu).
// ---------------------------------------------------------------------------
enum Alg : int { kPlain = 0, kComp = 1, kPlainF64 = 2, kCompF64 = 3, kChol = 4 };

// The FP32 route an algorithm variant starts from.
template <int ALG>
constexpr int kBaseAlg = ALG == kPlainF64 ? kPlain : (ALG == kCompF64 ? kComp : ALG);

template <int ALG>
constexpr bool kHasF64 = ALG == kPlainF64 || ALG == kCompF64;

template <int ALG>
__device__ __forceinline__ uint32_t pixel_inv_det(const float x[9], float w[9], float& det,
                                                  float tau) {
  if (ALG == kChol) {
    cholesky_inv_det(x, w, det);
  } else if (ALG == kComp || ALG == kCompF64) {
    adjugate_inv_det_comp<float>(x, w, det);
  } else {
    adjugate_inv_det<float>(x, w, det);
  }
  if (kHasF64<ALG> && needs_recompute(det, x, tau)) return recompute_f64(x, w, det);
  return (!(det > 0.0f) || !isfinite(det)) ? ZINV_PIX_NOT_PD : 0u;
}

// float4 lane access with a compile-time lane after unrolling
__device__ __forceinline__ float lane(const float4& v, int j) {
  return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}
__device__ __forceinline__ void set_lane(float4& v, int j, float x) {
  if (j == 0) v.x = x;
  else if (j == 1) v.y = x;
  else if (j == 2) v.z = x;
  else v.w = x;
}

// Warp-aggregated add of two per-thread counters into device counters.
__device__ __forceinline__ void add_counts(unsigned long long* counts, uint32_t c0, uint32_t c1) {
  const unsigned mask = __activemask();
  const uint32_t s0 = __reduce_add_sync(mask, c0);
  const uint32_t s1 = __reduce_add_sync(mask, c1);
  const int leader = __ffs(mask) - 1;
  if ((int)(threadIdx.x & 31) == leader) {
    if (s0) atomicAdd(counts, (unsigned long long)s0);
    if (s1) atomicAdd(counts + 1, (unsigned long long)s1);
  }
}

}  // namespace zinv
