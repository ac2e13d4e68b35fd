// qcd_device.cuh -- device-side building blocks of the gauge sweep:
// complex numbers, SU(2) as unit quaternions, SU(3) as 3x3 complex matrices,
// Philox-4x32-10, lattice geometry on the even/odd layout, link storage.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "qcd_internal.h"

namespace qcd {

// ---------------------------------------------------------------------------
// Complex arithmetic
// ---------------------------------------------------------------------------
template <typename R>
struct Cx {
  R re, im;
};

template <typename R>
__device__ __forceinline__ Cx<R> cx(R re, R im) { return {re, im}; }
template <typename R>
__device__ __forceinline__ Cx<R> operator+(Cx<R> a, Cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R>
__device__ __forceinline__ Cx<R> operator-(Cx<R> a, Cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R>
__device__ __forceinline__ Cx<R> operator*(Cx<R> a, Cx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__device__ __forceinline__ Cx<R> conj(Cx<R> a) { return {a.re, -a.im}; }
template <typename R>
__device__ __forceinline__ Cx<R> scale(Cx<R> a, R s) { return {a.re * s, a.im * s}; }
// acc + a * b
template <typename R>
__device__ __forceinline__ Cx<R> cfma(Cx<R> a, Cx<R> b, Cx<R> acc) {
  return {fma(a.re, b.re, fma(-a.im, b.im, acc.re)), fma(a.re, b.im, fma(a.im, b.re, acc.im))};
}
// acc + a * conj(b)
template <typename R>
__device__ __forceinline__ Cx<R> cfma_nc(Cx<R> a, Cx<R> b, Cx<R> acc) {
  return {fma(a.re, b.re, fma(a.im, b.im, acc.re)), fma(a.im, b.re, fma(-a.re, b.im, acc.im))};
}
// acc + conj(a) * b
template <typename R>
__device__ __forceinline__ Cx<R> cfma_cn(Cx<R> a, Cx<R> b, Cx<R> acc) {
  return {fma(a.re, b.re, fma(a.im, b.im, acc.re)), fma(a.re, b.im, fma(-a.im, b.re, acc.im))};
}

// ---------------------------------------------------------------------------
// SU(2) as unit quaternions q0 + i (q1 s1 + q2 s2 + q3 s3), i.e. the matrix
// [[q0 + i q3, q2 + i q1], [-q2 + i q1, q0 - i q3]].  Real multiples of SU(2)
// (staple sums) use the same type.
// ---------------------------------------------------------------------------
template <typename R>
struct Quat {
  R q0, q1, q2, q3;
};

__device__ __forceinline__ float qfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double qfma(double a, double b, double c) { return fma(a, b, c); }

// acc + a b, a b the matrix product (a0 b0 - a.b,  a0 b + b0 a - a x b): each
// component one chain of four multiply-adds started from acc.  (Written as
// sums of differences, the compiler may not reassociate them and spends a
// multiply and an add more per component.)
template <typename R>
__device__ __forceinline__ Quat<R> qmul_add(const Quat<R>& acc, const Quat<R>& a, const Quat<R>& b) {
  Quat<R> c;
  c.q0 = qfma(a.q0, b.q0, qfma(-a.q1, b.q1, qfma(-a.q2, b.q2, qfma(-a.q3, b.q3, acc.q0))));
  c.q1 = qfma(a.q0, b.q1, qfma(a.q1, b.q0, qfma(-a.q2, b.q3, qfma(a.q3, b.q2, acc.q1))));
  c.q2 = qfma(a.q0, b.q2, qfma(a.q2, b.q0, qfma(-a.q3, b.q1, qfma(a.q1, b.q3, acc.q2))));
  c.q3 = qfma(a.q0, b.q3, qfma(a.q3, b.q0, qfma(-a.q1, b.q2, qfma(a.q2, b.q1, acc.q3))));
  return c;
}

// Matrix product a b: the chains above, each started from one product.
template <typename R>
__device__ __forceinline__ Quat<R> qmul(const Quat<R>& a, const Quat<R>& b) {
  Quat<R> c;
  c.q0 = qfma(a.q0, b.q0, qfma(-a.q1, b.q1, qfma(-a.q2, b.q2, -a.q3 * b.q3)));
  c.q1 = qfma(a.q0, b.q1, qfma(a.q1, b.q0, qfma(-a.q2, b.q3, a.q3 * b.q2)));
  c.q2 = qfma(a.q0, b.q2, qfma(a.q2, b.q0, qfma(-a.q3, b.q1, a.q1 * b.q3)));
  c.q3 = qfma(a.q0, b.q3, qfma(a.q3, b.q0, qfma(-a.q1, b.q2, a.q2 * b.q1)));
  return c;
}
// a (c + s k), the product with the quaternion (c, 0, 0, s) (the SU(2)
// background factor diag(e^{i phi}, e^{-i phi}) has c = cos phi, s = sin phi):
// the 8 multiply-adds of qmul whose other factor is not zero.
template <typename R>
__device__ __forceinline__ Quat<R> qmul_k(const Quat<R>& a, R c, R s) {
  return {a.q0 * c - a.q3 * s, a.q1 * c - a.q2 * s, a.q2 * c + a.q1 * s, a.q3 * c + a.q0 * s};
}
template <typename R>
__device__ __forceinline__ Quat<R> qdag(const Quat<R>& a) { return {a.q0, -a.q1, -a.q2, -a.q3}; }
template <typename R>
__device__ __forceinline__ Quat<R> qadd(const Quat<R>& a, const Quat<R>& b) {
  return {a.q0 + b.q0, a.q1 + b.q1, a.q2 + b.q2, a.q3 + b.q3};
}
template <typename R>
__device__ __forceinline__ Quat<R> qscale(const Quat<R>& a, R s) { return {a.q0 * s, a.q1 * s, a.q2 * s, a.q3 * s}; }
template <typename R>
__device__ __forceinline__ R qnorm2(const Quat<R>& a) { return a.q0 * a.q0 + a.q1 * a.q1 + a.q2 * a.q2 + a.q3 * a.q3; }

// ---------------------------------------------------------------------------
// SU(3) as full 3x3 complex matrices in registers.
// ---------------------------------------------------------------------------
template <typename R>
struct M3 {
  Cx<R> e[3][3];
};

template <typename R>
__device__ __forceinline__ void m3_zero(M3<R>& m) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) m.e[i][j] = {R(0), R(0)};
}

// a b
template <typename R>
__device__ __forceinline__ M3<R> m3_mul(const M3<R>& a, const M3<R>& b) {
  M3<R> c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Cx<R> acc = a.e[i][0] * b.e[0][j];
      acc = cfma(a.e[i][1], b.e[1][j], acc);
      acc = cfma(a.e[i][2], b.e[2][j], acc);
      c.e[i][j] = acc;
    }
  return c;
}
// a b^+
template <typename R>
__device__ __forceinline__ M3<R> m3_mul_nd(const M3<R>& a, const M3<R>& b) {
  M3<R> c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Cx<R> acc = {R(0), R(0)};
#pragma unroll
      for (int k = 0; k < 3; ++k) acc = cfma_nc(a.e[i][k], b.e[j][k], acc);
      c.e[i][j] = acc;
    }
  return c;
}
// acc += a^+ b
template <typename R>
__device__ __forceinline__ void m3_acc_dn(M3<R>& acc, const M3<R>& a, const M3<R>& b) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Cx<R> s = acc.e[i][j];
#pragma unroll
      for (int k = 0; k < 3; ++k) s = cfma_cn(a.e[k][i], b.e[k][j], s);
      acc.e[i][j] = s;
    }
}
// acc += a b^+
template <typename R>
__device__ __forceinline__ void m3_acc_nd(M3<R>& acc, const M3<R>& a, const M3<R>& b) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Cx<R> s = acc.e[i][j];
#pragma unroll
      for (int k = 0; k < 3; ++k) s = cfma_nc(a.e[i][k], b.e[j][k], s);
      acc.e[i][j] = s;
    }
}
template <typename R>
__device__ __forceinline__ M3<R> m3_dag(const M3<R>& a) {
  M3<R> c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) c.e[i][j] = conj(a.e[j][i]);
  return c;
}
template <typename R>
__device__ __forceinline__ R m3_retrace(const M3<R>& a) {
  return a.e[0][0].re + a.e[1][1].re + a.e[2][2].re;
}
// Re Tr(a b) without forming the product.
template <typename R>
__device__ __forceinline__ R m3_retrace_mul(const M3<R>& a, const M3<R>& b) {
  R s = R(0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) s = fma(a.e[i][k].re, b.e[k][i].re, fma(-a.e[i][k].im, b.e[k][i].im, s));
  return s;
}
// row 2 = conj(row0 x row1): the third row of an SU(3) matrix.
template <typename R>
__device__ __forceinline__ void m3_rebuild_row2(M3<R>& m) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
    Cx<R> v = m.e[0][c1] * m.e[1][c2] - m.e[0][c2] * m.e[1][c1];
    m.e[2][c] = conj(v);
  }
}

// ---------------------------------------------------------------------------
// Philox-4x32-10 (Salmon et al., SC11): 10 rounds, two 32x32->64 multiplies
// per round, key bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    // both halves of each 32x32 -> 64 product from one widening multiply
    const uint64_t p0 = uint64_t(0xD2511F53u) * c.x, p1 = uint64_t(0xCD9E8D57u) * c.z;
    const uint32_t lo0 = uint32_t(p0), hi0 = uint32_t(p0 >> 32);
    const uint32_t lo1 = uint32_t(p1), hi1 = uint32_t(p1 >> 32);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// ((w >> 9) + 1/2) 2^-23: a uniform in (0,1), exact in FP32 and FP64.  Built
// without an integer-to-float conversion (a slow pipe on this GPU): the 23
// bits become the mantissa of x = 1 + m 2^-23 in [1, 2), and
// x - (1 - 2^-24) = (2m + 1) 2^-24 is exact (at most 24 significant bits).
template <typename R>
__device__ __forceinline__ R u01(uint32_t w);
template <>
__device__ __forceinline__ float u01<float>(uint32_t w) {
  return __int_as_float(0x3F800000u | (w >> 9)) - 0.999999940395355224609375f;
}
template <>
__device__ __forceinline__ double u01<double>(uint32_t w) {
  return __longlong_as_double(0x3FF0000000000000ll | (static_cast<long long>(w >> 9) << 29)) -
         0.999999940395355224609375;
}

enum : uint32_t { KIND_TRY = 0u, KIND_DIR = 1u, KIND_START = 2u };
constexpr uint32_t START_SWEEP_WORD = 0xFFFFFFFFu;

struct Stream {
  uint32_t k0, k1, c0, c1, c2;
  template <typename R>
  __device__ __forceinline__ void uniforms(uint32_t block, R u[4]) const {
    uint4 w = philox4x32_10(make_uint4(c0, c1, c2, block), k0, k1);
    u[0] = u01<R>(w.x);
    u[1] = u01<R>(w.y);
    u[2] = u01<R>(w.z);
    u[3] = u01<R>(w.w);
  }
};

__device__ __forceinline__ Stream make_stream(uint32_t k0, uint32_t k1, uint32_t site, uint32_t sweep, int mu,
                                              int sub, uint32_t kind) {
  return Stream{k0, k1, site, sweep, uint32_t(mu) | (uint32_t(sub) << 2) | (kind << 4)};
}

// Transcendentals in the working precision.
__device__ __forceinline__ float q_log(float x) { return logf(x); }
__device__ __forceinline__ double q_log(double x) { return log(x); }
__device__ __forceinline__ float q_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double q_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float q_cospi(float x) { return cospif(x); }
__device__ __forceinline__ double q_cospi(double x) { return cospi(x); }
__device__ __forceinline__ void q_sincospi(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void q_sincospi(double x, double* s, double* c) { sincospi(x, s, c); }

// Kennedy-Pendleton draw with density ~ sqrt(1 - a0^2) exp(alpha a0),
// returned as delta = 1 - a0: try t uses block t,
// delta = (-ln u2 - ln u1 cos^2(2 pi u3)) / alpha, accepted when
// u4^2 <= 1 - delta / 2.  Returns false when all nhit tries fail.
template <typename R>
__device__ __forceinline__ bool kp_draw(R alpha, int nhit, const Stream& st, R& delta) {
  const R inv_alpha = R(1) / alpha;
  for (int t = 0; t < nhit; ++t) {
    R u[4];
    st.uniforms<R>(uint32_t(t), u);
    const R c = q_cospi(R(2) * u[2]);
    const R d = (-q_log(u[1]) - q_log(u[0]) * c * c) * inv_alpha;
    if (u[3] * u[3] <= R(1) - R(0.5) * d) {
      delta = d;
      return true;
    }
  }
  return false;
}

// FP32: the same draw with the hardware logarithm and cosine.  Their absolute
// errors (about 2^-21) move delta by less than 1e-7 / alpha, below the FP32
// resolution of a0 = 1 - delta; cos^2 is taken at 2 pi (u - 1/2), inside the
// fast cosine's accurate range, which leaves cos^2 unchanged.
// One FP32 try on the four uniforms of its block.
__device__ __forceinline__ bool kp_try_f32(const float u[4], float inv_alpha, float& delta) {
  const float c = __cosf(6.283185307179586f * (u[2] - 0.5f));
  const float d = (-__logf(u[1]) - __logf(u[0]) * c * c) * inv_alpha;
  delta = d;
  return u[3] * u[3] <= 1.f - 0.5f * d;
}

template <>
__device__ __forceinline__ bool kp_draw<float>(float alpha, int nhit, const Stream& st, float& delta) {
  const float inv_alpha = __fdividef(1.f, alpha);
  for (int t = 0; t < nhit; ++t) {
    float u[4];
    st.uniforms<float>(uint32_t(t), u);
    if (kp_try_f32(u, inv_alpha, delta)) return true;
  }
  return false;
}

// Unit quaternion with real part a0 = 1 - delta and a direction uniform on
// S^2 from block 0 of the direction stream: cos(theta) = 2 u1 - 1,
// phi = 2 pi u2.  The moduli use the cancellation-free forms
// sqrt(1 - a0^2) = sqrt(delta (2 - delta)) and
// sin(theta) = sqrt(1 - (2 u1 - 1)^2) = 2 sqrt(u1 (1 - u1)).
template <typename R>
__device__ __forceinline__ Quat<R> su2_with_delta(R delta, const Stream& dir) {
  R u[4];
  dir.uniforms<R>(0u, u);
  const R ct = R(2) * u[0] - R(1);
  const R st = R(2) * q_sqrt(u[0] * (R(1) - u[0]));
  R sp, cp;
  q_sincospi(R(2) * u[1], &sp, &cp);
  const R r = q_sqrt(delta * (R(2) - delta));
  return {R(1) - delta, r * st * cp, r * st * sp, r * ct};
}

// FP32: the azimuth's sine and cosine from the hardware pair at
// 2 pi (u - 1/2) (both change sign against 2 pi u), approximate square roots.
// ... from the direction block's uniforms u.
__device__ __forceinline__ Quat<float> su2_with_delta_u(float delta, const float u[4]) {
  // square roots as x rsqrt(x): both arguments are positive (u0 in (0, 1),
  // delta > 0 since -ln u > 0 for every uniform)
  const float ct = 2.f * u[0] - 1.f;
  const float q = u[0] * (1.f - u[0]);
  const float st = 2.f * q * rsqrtf(q);
  float sp, cp;
  __sincosf(6.283185307179586f * (u[1] - 0.5f), &sp, &cp);
  const float e = delta * (2.f - delta);
  const float r = e * rsqrtf(e);
  return {1.f - delta, -r * st * cp, -r * st * sp, r * ct};
}

template <>
__device__ __forceinline__ Quat<float> su2_with_delta<float>(float delta, const Stream& dir) {
  float u[4];
  dir.uniforms<float>(0u, u);
  return su2_with_delta_u(delta, u);
}

// FP32 draw of the unit quaternion X = (1 - delta, direction): the direction
// block does not depend on the tries, so it is drawn together with try 0 (two
// independent Philox chains interleave).  False when all nhit tries fail.
__device__ __forceinline__ bool kp_draw_dir_f32(float alpha, int nhit, const Stream& tries, const Stream& dir,
                                                Quat<float>& X) {
  const float inv_alpha = __fdividef(1.f, alpha);
  float u[4], v[4], delta;
  tries.uniforms<float>(0u, u);
  dir.uniforms<float>(0u, v);
  bool ok = kp_try_f32(u, inv_alpha, delta);
  for (int t = 1; !ok && t < nhit; ++t) {
    tries.uniforms<float>(uint32_t(t), u);
    ok = kp_try_f32(u, inv_alpha, delta);
  }
  if (ok) X = su2_with_delta_u(delta, v);
  return ok;
}

// Haar-random unit quaternion (Shoemake) from one block.
template <typename R>
__device__ __forceinline__ Quat<R> su2_haar(const Stream& st, uint32_t block) {
  R u[4];
  st.uniforms<R>(block, u);
  const R r1 = q_sqrt(R(1) - u[0]), r2 = q_sqrt(u[0]);
  R s1, c1, s2, c2;
  q_sincospi(R(2) * u[1], &s1, &c1);
  q_sincospi(R(2) * u[2], &s2, &c2);
  return {r1 * s1, r1 * c1, r2 * s2, r2 * c2};
}

// ---------------------------------------------------------------------------
// Geometry.  Site s = x + Ns (y + Ns (z + Ns t)); the even/odd layout keeps
// h = s >> 1 inside each parity (Ns even, so s and s^1 share y,z,t and differ
// in parity).
// ---------------------------------------------------------------------------
using Geom = GeomH;  // Ns, Nt, Vh = sites per parity, plane = vectors per plane

struct Site {
  int x, y, z, t;
};

// n / d for 0 <= n < 2^31 by the multiply-high of GeomH (m, s for d).
__device__ __forceinline__ int div_mh(int n, uint32_t m, int s) { return int(__umulhi(uint32_t(n), m) >> s); }

__device__ __forceinline__ Site site_of(const Geom& g, int parity, int h) {
  int r = 2 * h;
  Site c;
  int x0;
  if (g.pow2 & GEOM_POW2) {  // the same decoding by shifts and masks (uniform branch)
    const int ls = g.pow2 & 255, m = g.Ns - 1;
    x0 = r & m;
    c.y = (r >> ls) & m;
    c.z = (r >> (2 * ls)) & m;
    c.t = r >> (3 * ls);
  } else if (g.mNs) {  // by multiply-high (uniform branch)
    const int sN = (g.pow2 >> 17) & 31;
    int q = div_mh(r, g.mNs, sN);
    x0 = r - q * g.Ns;
    r = q;
    q = div_mh(r, g.mNs, sN);
    c.y = r - q * g.Ns;
    r = q;
    q = div_mh(r, g.mNs, sN);
    c.z = r - q * g.Ns;
    c.t = q;
  } else {
    x0 = r % g.Ns;
    r /= g.Ns;
    c.y = r % g.Ns;
    r /= g.Ns;
    c.z = r % g.Ns;
    c.t = r / g.Ns;
  }
  c.x = x0 + ((parity + c.y + c.z + c.t) & 1);
  return c;
}
__device__ __forceinline__ int lex(const Geom& g, const Site& c) {
  return c.x + g.Ns * (c.y + g.Ns * (c.z + g.Ns * c.t));
}
__device__ __forceinline__ int parity_of(const Site& c) { return (c.x + c.y + c.z + c.t) & 1; }
__device__ __forceinline__ Site step(const Geom& g, Site c, int mu, int d) {
  // d = +1 or -1, periodic
  if (mu == 0) {
    c.x += d;
    c.x = c.x < 0 ? g.Ns - 1 : (c.x >= g.Ns ? 0 : c.x);
  } else if (mu == 1) {
    c.y += d;
    c.y = c.y < 0 ? g.Ns - 1 : (c.y >= g.Ns ? 0 : c.y);
  } else if (mu == 2) {
    c.z += d;
    c.z = c.z < 0 ? g.Ns - 1 : (c.z >= g.Ns ? 0 : c.z);
  } else {
    c.t += d;
    c.t = c.t < 0 ? g.Nt - 1 : (c.t >= g.Nt ? 0 : c.t);
  }
  return c;
}

// Vector index of component comp of link (mu, parity, h).
__device__ __forceinline__ int64_t vidx(const Geom& g, int comp, int mu, int parity, int h) {
  return (int64_t(comp * 4 + mu) * 2 + parity) * g.plane + h;
}

// ---------------------------------------------------------------------------
// Neighbour stepping on the lexicographic index: a site carries its index and
// coordinates, and one step along a direction known at compile time is a
// stride plus a wrap correction.
// ---------------------------------------------------------------------------
// A site by its lexicographic index and coordinates.
struct LexSite {
  int s;
  int c[4];
};

template <int D>
__device__ __forceinline__ int lex_stride(const Geom& g) {
  return D == 0 ? 1 : D == 1 ? g.Ns : D == 2 ? g.Ns * g.Ns : g.Ns * g.Ns * g.Ns;
}
template <int D>
__device__ __forceinline__ int lex_extent(const Geom& g) {
  return D == 3 ? g.Nt : g.Ns;
}
// one step +1 / -1 along D with periodic wrap
template <int D, int STEP>
__device__ __forceinline__ LexSite lex_step(const Geom& g, LexSite x) {
  const int st = lex_stride<D>(g), ext = lex_extent<D>(g);
  if (STEP > 0) {
    const bool wrap = x.c[D] == ext - 1;
    x.s += wrap ? st - ext * st : st;
    x.c[D] = wrap ? 0 : x.c[D] + 1;
  } else {
    const bool wrap = x.c[D] == 0;
    x.s += wrap ? ext * st - st : -st;
    x.c[D] = wrap ? ext - 1 : x.c[D] - 1;
  }
  return x;
}

__device__ __forceinline__ LexSite lex_site(const Ctx& a, int parity, int h) {
  const Site sc = site_of(a.g, parity, h);
  LexSite x;
  x.c[0] = sc.x;
  x.c[1] = sc.y;
  x.c[2] = sc.z;
  x.c[3] = sc.t;
  x.s = 2 * h + (sc.x & 1);
  return x;
}

// Site of one parity for thread index i, enumerated x (in pairs) fastest, then
// y, then t, then z.  Each phase still visits every site once, but successive
// CTAs step through t before z, so the t-neighbour of a site is gathered a
// few CTAs after it was last read (not a whole Ns^3 volume later) and is still
// in L2: the longest reuse distance drops from Ns^3/2 to Ns^2 Nt/2 sites.
__device__ __forceinline__ LexSite lex_site_ytz(const Geom& g, int parity, int i) {
  int r = 2 * i;
  LexSite x;
  int x0;
  if (g.pow2 & GEOM_POW2) {  // the same decoding by shifts and masks (uniform branch)
    const int ls = g.pow2 & 255, lt = (g.pow2 >> 8) & 255, m = g.Ns - 1;
    x0 = r & m;
    x.c[1] = (r >> ls) & m;
    x.c[3] = (r >> (2 * ls)) & (g.Nt - 1);
    x.c[2] = r >> (2 * ls + lt);
  } else if (g.mNs) {  // by multiply-high (uniform branch)
    const int sN = (g.pow2 >> 17) & 31, sT = (g.pow2 >> 22) & 31;
    int q = div_mh(r, g.mNs, sN);
    x0 = r - q * g.Ns;
    r = q;
    q = div_mh(r, g.mNs, sN);
    x.c[1] = r - q * g.Ns;
    r = q;
    q = div_mh(r, g.mNt, sT);
    x.c[3] = r - q * g.Nt;
    x.c[2] = q;
  } else {
    x0 = r % g.Ns;
    r /= g.Ns;
    x.c[1] = r % g.Ns;
    r /= g.Ns;
    x.c[3] = r % g.Nt;
    x.c[2] = r / g.Nt;
  }
  x.c[0] = x0 + ((parity + x.c[1] + x.c[2] + x.c[3]) & 1);
  x.s = x.c[0] + g.Ns * (x.c[1] + g.Ns * (x.c[2] + g.Ns * x.c[3]));
  return x;
}

}  // namespace qcd
