// synth.cu -- GPU twin of the seeded input generators in synth/__init__.py.
//
// Same Philox4x32-10 counters and keys, same 53-bit uniforms, same series for
// log, exp and sin/cos, same order of every FP64 operation, so each pixel is
// bit-identical to the numpy twin.  This file must be compiled with
// -fmad=false (no fused multiply-add contraction); division and sqrt in FP64
// are IEEE correctly rounded on the GPU as in numpy.  It holds none of the
// method's arithmetic (no inverse, determinant, cofactor or window average).
#include <cuda_runtime.h>
#include <stdint.h>

#define SYNTH_OK 0
#define SYNTH_ERR_ARG (-1)
#define SYNTH_ERR_LAUNCH (-2)

namespace {

constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
constexpr uint32_t kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;
constexpr uint32_t kTagWishart = 1, kTagCond = 2, kTagRrh = 3, kTagSlc = 4;

__device__ __forceinline__ void philox(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += kW0;
      k1 += kW1;
    }
    const uint32_t hi0 = __umulhi(kM0, c[0]), lo0 = kM0 * c[0];
    const uint32_t hi1 = __umulhi(kM1, c[2]), lo1 = kM1 * c[2];
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

__device__ __forceinline__ double u53(uint32_t a, uint32_t b) {
  const uint64_t k = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
  return (double)(k + 1) * 0x1p-53;
}

// Uniform draws u_0, u_1, ... of one pixel; call d yields u_{2d}, u_{2d+1}.
struct Stream {
  uint32_t seed, tag, lo, hi, stream;
  int cached = -1;
  double u0 = 0, u1 = 0;
  __device__ Stream(uint32_t seed_, uint32_t tag_, uint64_t idx, uint32_t stream_)
      : seed(seed_), tag(tag_), lo((uint32_t)idx), hi((uint32_t)(idx >> 32)), stream(stream_) {}
  __device__ double u(int j) {
    const int d = j / 2;
    if (d != cached) {
      uint32_t c[4] = {lo, hi, (uint32_t)d, stream};
      philox(c, seed, tag);
      u0 = u53(c[0], c[1]);
      u1 = u53(c[2], c[3]);
      cached = d;
    }
    return (j & 1) ? u1 : u0;
  }
};

__constant__ double kLogC[13] = {
    0x1.0000000000000p+0, 0x1.5555555555555p-2, 0x1.999999999999ap-3, 0x1.2492492492492p-3,
    0x1.c71c71c71c71cp-4, 0x1.745d1745d1746p-4, 0x1.3b13b13b13b14p-4, 0x1.1111111111111p-4,
    0x1.e1e1e1e1e1e1ep-5, 0x1.af286bca1af28p-5, 0x1.8618618618618p-5, 0x1.642c8590b2164p-5,
    0x1.47ae147ae147bp-5};
__constant__ double kInvFact[24] = {
    0x1.0000000000000p+0, 0x1.0000000000000p+0, 0x1.0000000000000p-1, 0x1.5555555555555p-3,
    0x1.5555555555555p-5, 0x1.1111111111111p-7, 0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-13,
    0x1.a01a01a01a01ap-16, 0x1.71de3a556c734p-19, 0x1.27e4fb7789f5cp-22, 0x1.ae64567f544e4p-26,
    0x1.1eed8eff8d898p-29, 0x1.6124613a86d09p-33, 0x1.93974a8c07c9dp-37, 0x1.ae7f3e733b81fp-41,
    0x1.ae7f3e733b81fp-45, 0x1.952c77030ad4ap-49, 0x1.6827863b97d97p-53, 0x1.2f49b46814157p-57,
    0x1.e542ba4020225p-62, 0x1.71b8ef6dcf572p-66, 0x1.0ce396db7f853p-70, 0x1.761b413163819p-75};
constexpr double kLn2 = 0x1.62e42fefa39efp-1;
constexpr double kInvLn2 = 0x1.71547652b82fep+0;
constexpr double kHalfPi = 0x1.921fb54442d18p+0;
constexpr double kSqrtHalf = 0x1.6a09e667f3bcdp-1;

__device__ double dlog(double x) {
  int e;
  double m = frexp(x, &e);
  if (m < kSqrtHalf) {
    m = m * 2.0;
    e = e - 1;
  }
  const double z = (m - 1.0) / (m + 1.0);
  const double z2 = z * z;
  double p = kLogC[12];
  for (int k = 11; k >= 0; --k) p = p * z2 + kLogC[k];
  return (double)e * kLn2 + (2.0 * z) * p;
}

__device__ double dexp(double x) {
  const double k = rint(x * kInvLn2);
  const double r = x - k * kLn2;
  double p = kInvFact[17];
  for (int j = 16; j >= 0; --j) p = p * r + kInvFact[j];
  return ldexp(p, (int)k);
}

__device__ void dsincos_2pi(double u, double& sn, double& cs) {
  const double v = u * 4.0;
  const double q = floor(v);
  const double f = v - q;
  const double th = f * kHalfPi;
  const double t2 = th * th;
  double s = -kInvFact[23];
  for (int j = 21; j >= 1; j -= 2) s = s * t2 + ((((j - 1) / 2) % 2 == 0) ? kInvFact[j] : -kInvFact[j]);
  s = s * th;
  double c = -kInvFact[22];
  for (int j = 20; j >= 0; j -= 2) c = c * t2 + (((j / 2) % 2 == 0) ? kInvFact[j] : -kInvFact[j]);
  const int qi = ((int)q) % 4;
  if (qi == 0) { sn = s; cs = c; }
  else if (qi == 1) { sn = c; cs = -s; }
  else if (qi == 2) { sn = -s; cs = -c; }
  else { sn = -c; cs = s; }
}

__device__ void cnormal(double u1, double u2, double& re, double& im) {
  const double r = sqrt(-dlog(u1));
  double s, c;
  dsincos_2pi(u2, s, c);
  re = r * c;
  im = r * s;
}

struct C2 {
  double r, i;
};
__device__ __forceinline__ C2 cmul(C2 a, C2 b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
// a * conj(b)
__device__ __forceinline__ C2 cmulc(C2 a, C2 b) { return {a.r * b.r + a.i * b.i, a.i * b.r - a.r * b.i}; }

// Modified Gram-Schmidt on the columns of v (in place -> q), as the numpy twin.
__device__ void gram_schmidt(C2 v[3][3]) {
  for (int j = 0; j < 3; ++j) {
    const double nrm2 = (v[0][j].r * v[0][j].r + v[0][j].i * v[0][j].i) +
                        (v[1][j].r * v[1][j].r + v[1][j].i * v[1][j].i) +
                        (v[2][j].r * v[2][j].r + v[2][j].i * v[2][j].i);
    const double nrm = sqrt(nrm2);
    for (int i = 0; i < 3; ++i) {
      v[i][j].r = v[i][j].r / nrm;
      v[i][j].i = v[i][j].i / nrm;
    }
    for (int k = j + 1; k < 3; ++k) {
      const double pr = (v[0][j].r * v[0][k].r + v[0][j].i * v[0][k].i) +
                        (v[1][j].r * v[1][k].r + v[1][j].i * v[1][k].i) +
                        (v[2][j].r * v[2][k].r + v[2][j].i * v[2][k].i);
      const double pi = (v[0][j].r * v[0][k].i - v[0][j].i * v[0][k].r) +
                        (v[1][j].r * v[1][k].i - v[1][j].i * v[1][k].r) +
                        (v[2][j].r * v[2][k].i - v[2][j].i * v[2][k].r);
      for (int i = 0; i < 3; ++i) {
        const C2 t = cmul({pr, pi}, v[i][j]);
        v[i][k].r = v[i][k].r - t.r;
        v[i][k].i = v[i][k].i - t.i;
      }
    }
  }
}

__device__ __forceinline__ void store_packed(const C2 Z[3][3], float* z, int64_t ld, int64_t p) {
  z[0 * ld + p] = __double2float_rn(Z[0][0].r);
  z[1 * ld + p] = __double2float_rn(Z[0][1].r);
  z[2 * ld + p] = __double2float_rn(Z[0][1].i);
  z[3 * ld + p] = __double2float_rn(Z[0][2].r);
  z[4 * ld + p] = __double2float_rn(Z[0][2].i);
  z[5 * ld + p] = __double2float_rn(Z[1][1].r);
  z[6 * ld + p] = __double2float_rn(Z[1][2].r);
  z[7 * ld + p] = __double2float_rn(Z[1][2].i);
  z[8 * ld + p] = __double2float_rn(Z[2][2].r);
}

__device__ __forceinline__ void load_F(const double* F, int cls, C2 f[3][3]) {
  const double* b = F + cls * 18;
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) f[i][k] = {b[2 * (3 * i + k)], b[2 * (3 * i + k) + 1]};
}

__device__ __forceinline__ int pixel_class(int64_t y, int64_t x, int64_t W, int block,
                                           const int32_t* block_cls) {
  if (!block_cls) return 0;
  const int64_t bx = (W + block - 1) / block;
  return block_cls[(y / block) * bx + (x / block)];
}

__global__ void k_z_wishart(uint32_t seed, int64_t H, int64_t W, int N, const double* F,
                            const int32_t* block_cls, int block, float* z, int64_t ld) {
  const int64_t n = H * W;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    Stream st(seed, kTagWishart, (uint64_t)p, 0);
    int j = 0;
    double Td[3];
    for (int i = 0; i < 3; ++i) {
      double prod = 1.0;
      for (int l = 0; l < N - i; ++l) {
        prod = prod * st.u(j);
        ++j;
      }
      Td[i] = sqrt(-dlog(prod));
    }
    C2 t10, t20, t21;
    cnormal(st.u(j), st.u(j + 1), t10.r, t10.i);
    j += 2;
    cnormal(st.u(j), st.u(j + 1), t20.r, t20.i);
    j += 2;
    cnormal(st.u(j), st.u(j + 1), t21.r, t21.i);
    // B = T T^H
    C2 B[3][3];
    B[0][0] = {Td[0] * Td[0], 0.0};
    B[0][1] = {Td[0] * t10.r, -(Td[0] * t10.i)};
    B[0][2] = {Td[0] * t20.r, -(Td[0] * t20.i)};
    B[1][1] = {(t10.r * t10.r + t10.i * t10.i) + Td[1] * Td[1], 0.0};
    const C2 b12 = cmulc(t10, t20);
    B[1][2] = {b12.r + Td[1] * t21.r, b12.i - Td[1] * t21.i};
    B[2][2] = {((t20.r * t20.r + t20.i * t20.i) + (t21.r * t21.r + t21.i * t21.i)) + Td[2] * Td[2],
               0.0};
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < i; ++k) B[i][k] = {B[k][i].r, -B[k][i].i};
    C2 f[3][3];
    load_F(F, pixel_class(p / W, p % W, W, block, block_cls), f);
    C2 Cm[3][3];
    for (int i = 0; i < 3; ++i)
      for (int jj = 0; jj < 3; ++jj) {
        C2 s = cmul(f[i][0], B[0][jj]);
        for (int k = 1; k < 3; ++k) {
          const C2 t = cmul(f[i][k], B[k][jj]);
          s = {s.r + t.r, s.i + t.i};
        }
        Cm[i][jj] = s;
      }
    const double invN = 1.0 / (double)N;
    C2 Z[3][3];
    for (int i = 0; i < 3; ++i)
      for (int jj = i; jj < 3; ++jj) {
        C2 s = cmulc(Cm[i][0], f[jj][0]);
        for (int k = 1; k < 3; ++k) {
          const C2 t = cmulc(Cm[i][k], f[jj][k]);
          s = {s.r + t.r, s.i + t.i};
        }
        Z[i][jj] = {s.r * invN, s.i * invN};
      }
    store_packed(Z, z, ld, p);
  }
}

__global__ void k_z_cond(uint32_t seed, int64_t n, double ln_kmax, float* z, int64_t ld) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    Stream st(seed, kTagCond, (uint64_t)p, 0);
    const double lnk = st.u(0) * ln_kmax;
    const double kappa = dexp(lnk);
    const double lam[3] = {1.0, dexp(-(st.u(1) * lnk)), 1.0 / kappa};
    C2 q[3][3];
    int j = 2;
    for (int col = 0; col < 3; ++col)
      for (int row = 0; row < 3; ++row) {
        cnormal(st.u(j), st.u(j + 1), q[row][col].r, q[row][col].i);
        j += 2;
      }
    gram_schmidt(q);
    C2 Z[3][3];
    for (int i = 0; i < 3; ++i)
      for (int k = i; k < 3; ++k) {
        C2 s = cmulc(q[i][0], q[k][0]);
        s = {lam[0] * s.r, lam[0] * s.i};
        for (int m = 1; m < 3; ++m) {
          const C2 t = cmulc(q[i][m], q[k][m]);
          s = {s.r + lam[m] * t.r, s.i + lam[m] * t.i};
        }
        Z[i][k] = s;
      }
    store_packed(Z, z, ld, p);
  }
}

__global__ void k_z_rrh(uint32_t seed, int64_t n, float* z, int64_t ld) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    Stream st(seed, kTagRrh, (uint64_t)p, 0);
    C2 R[3][3];
    int j = 0;
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 3; ++k) {
        R[i][k] = {2.0 * st.u(j) - 1.0, 2.0 * st.u(j + 1) - 1.0};
        j += 2;
      }
    C2 Z[3][3];
    for (int i = 0; i < 3; ++i)
      for (int k = i; k < 3; ++k) {
        C2 s = cmulc(R[i][0], R[k][0]);
        for (int m = 1; m < 3; ++m) {
          const C2 t = cmulc(R[i][m], R[k][m]);
          s = {s.r + t.r, s.i + t.i};
        }
        Z[i][k] = s;
      }
    store_packed(Z, z, ld, p);
  }
}

__global__ void k_slc(uint32_t seed, int64_t H, int64_t W, const double* F,
                      const int32_t* block_cls, int block, int date, float2* s,
                      int64_t plane_ld) {
  const int64_t n = H * W;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    Stream st(seed, kTagSlc, (uint64_t)p, (uint32_t)date);
    C2 g[3];
    for (int i = 0; i < 3; ++i) cnormal(st.u(2 * i), st.u(2 * i + 1), g[i].r, g[i].i);
    C2 f[3][3];
    load_F(F, pixel_class(p / W, p % W, W, block, block_cls), f);
    for (int i = 0; i < 3; ++i) {
      C2 acc = cmul(f[i][0], g[0]);
      for (int k = 1; k < 3; ++k) {
        const C2 t = cmul(f[i][k], g[k]);
        acc = {acc.r + t.r, acc.i + t.i};
      }
      s[i * plane_ld + p] = make_float2(__double2float_rn(acc.r), __double2float_rn(acc.i));
    }
  }
}

__global__ void k_uniform(uint32_t seed, uint32_t tag, uint32_t stream_id, int64_t n, double lo,
                          double hi, float* out) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    Stream st(seed, tag, (uint64_t)p, stream_id);
    out[p] = __double2float_rn(lo + (hi - lo) * st.u(0));
  }
}

constexpr int kThreads = 128;

inline unsigned blocks_for(int64_t n) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 16;
  const int64_t need = (n + kThreads - 1) / kThreads;
  return (unsigned)(need < cap ? (need > 0 ? need : 1) : cap);
}

inline int done() { return cudaGetLastError() == cudaSuccess ? SYNTH_OK : SYNTH_ERR_LAUNCH; }

}  // namespace

extern "C" int synth_z_wishart(uint32_t seed, int64_t H, int64_t W, int N, const double* F,
                               const int32_t* block_cls, int block, float* z, int64_t ld,
                               void* stream) {
  if (H < 0 || W < 0 || N < 3 || !F || !z || ld < H * W || (block_cls && block < 1))
    return SYNTH_ERR_ARG;
  if (H * W == 0) return SYNTH_OK;
  k_z_wishart<<<blocks_for(H * W), kThreads, 0, (cudaStream_t)stream>>>(seed, H, W, N, F,
                                                                        block_cls, block, z, ld);
  return done();
}

extern "C" int synth_z_cond(uint32_t seed, int64_t n, double ln_kmax, float* z, int64_t ld,
                            void* stream) {
  if (n < 0 || !z || ld < n) return SYNTH_ERR_ARG;
  if (n == 0) return SYNTH_OK;
  k_z_cond<<<blocks_for(n), kThreads, 0, (cudaStream_t)stream>>>(seed, n, ln_kmax, z, ld);
  return done();
}

extern "C" int synth_z_rrh(uint32_t seed, int64_t n, float* z, int64_t ld, void* stream) {
  if (n < 0 || !z || ld < n) return SYNTH_ERR_ARG;
  if (n == 0) return SYNTH_OK;
  k_z_rrh<<<blocks_for(n), kThreads, 0, (cudaStream_t)stream>>>(seed, n, z, ld);
  return done();
}

extern "C" int synth_slc(uint32_t seed, int64_t H, int64_t W, const double* F,
                         const int32_t* block_cls, int block, int date, float* s,
                         int64_t plane_ld, void* stream) {
  if (H < 0 || W < 0 || !F || !s || plane_ld < H * W || (block_cls && block < 1))
    return SYNTH_ERR_ARG;
  if (H * W == 0) return SYNTH_OK;
  k_slc<<<blocks_for(H * W), kThreads, 0, (cudaStream_t)stream>>>(
      seed, H, W, F, block_cls, block, date, reinterpret_cast<float2*>(s), plane_ld);
  return done();
}

extern "C" int synth_uniform(uint32_t seed, uint32_t tag, uint32_t stream_id, int64_t n,
                             double lo, double hi, float* out, void* stream) {
  if (n < 0 || !out) return SYNTH_ERR_ARG;
  if (n == 0) return SYNTH_OK;
  k_uniform<<<blocks_for(n), kThreads, 0, (cudaStream_t)stream>>>(seed, tag, stream_id, n, lo,
                                                                  hi, out);
  return done();
}
