// qcd_kernels.cuh -- templated kernels of the gauge sweep.  Each storage
// translation unit (su2_f32.cu, su2_f64.cu, su3_f32.cu, su3_f64.cu)
// instantiates them for one (group, precision) and exports a PolicyOps table.
//
// Link layout in device memory (the paper's sec. 3.3 scheme of 4-vectors with
// the site index fastest, split by checkerboard parity): 16-byte vectors,
// vector (comp, mu, parity, h) at ((comp * 4 + mu) * 2 + parity) * plane + h,
// h = s >> 1 the index inside the parity.  Per link:
//   SU(2) FP32  1 x float4   (q0, q1, q2, q3)
//   SU(2) FP64  2 x double2  (q0, q1) (q2, q3)
//   SU(3) FP32  3 x float4   rows 0-1: (u00, u01) (u02, u10) (u11, u12)
//   SU(3) FP64  9 x double2  u_rc, r-major
#pragma once

#include <algorithm>

#include "qcd_device.cuh"
#include "qcd_internal.h"

namespace qcd {

// ---------------------------------------------------------------------------
// Storage policies.  Loads go through the read-only path (ld.global.nc) when
// the links cannot change while the kernel runs (one phase per launch); a
// kernel that updates links between its own phases (the batched persistent
// kernel) loads with CG = true (ld.global.cg: cached in L2 only, never a stale
// L1 line).
// ---------------------------------------------------------------------------
template <bool CG, typename T>
__device__ __forceinline__ T ld16(const T* p) {
  if constexpr (CG) return __ldcg(p);
  else return __ldg(p);
}
template <typename R>
struct SU2Policy;

template <>
struct SU2Policy<float> {
  using Real = float;
  using Link = Quat<float>;
  static constexpr int N = 2, COMPS = 1;
  // CG (the batched kernel): the index in 32-bit arithmetic, exact because
  // qcd_batch_create admits FP32 lattices of fewer than 2^29 sites (8 arrays
  // of at most 2^28 float4); measured 6 % faster per sweep of the 64-lattice
  // scan than the 64-bit form, which the single-lattice kernels keep (there
  // the 32-bit form measured slower).
  template <bool CG = false>
  static __device__ __forceinline__ Link load(const void* base, const Geom& g, int mu, int par, int h) {
    const float4* p = reinterpret_cast<const float4*>(base);
    const float4 v = CG ? ld16<CG>(p + ((mu * 2 + par) * int(g.plane) + h)) : ld16<CG>(p + vidx(g, 0, mu, par, h));
    return {v.x, v.y, v.z, v.w};
  }
  static __device__ __forceinline__ void store(void* base, const Geom& g, int mu, int par, int h, const Link& u) {
    reinterpret_cast<float4*>(base)[vidx(g, 0, mu, par, h)] = make_float4(u.q0, u.q1, u.q2, u.q3);
  }
};

template <>
struct SU2Policy<double> {
  using Real = double;
  using Link = Quat<double>;
  static constexpr int N = 2, COMPS = 2;
  template <bool CG = false>
  static __device__ __forceinline__ Link load(const void* base, const Geom& g, int mu, int par, int h) {
    const double2* p = reinterpret_cast<const double2*>(base);
    const double2 a = ld16<CG>(p + vidx(g, 0, mu, par, h)), b = ld16<CG>(p + vidx(g, 1, mu, par, h));
    return {a.x, a.y, b.x, b.y};
  }
  static __device__ __forceinline__ void store(void* base, const Geom& g, int mu, int par, int h, const Link& u) {
    double2* p = reinterpret_cast<double2*>(base);
    p[vidx(g, 0, mu, par, h)] = make_double2(u.q0, u.q1);
    p[vidx(g, 1, mu, par, h)] = make_double2(u.q2, u.q3);
  }
};

template <typename R>
struct SU3Policy;

template <>
struct SU3Policy<float> {
  using Real = float;
  using Link = M3<float>;
  static constexpr int N = 3, COMPS = 3;
  template <bool CG = false>
  static __device__ __forceinline__ Link load(const void* base, const Geom& g, int mu, int par, int h) {
    const float4* p = reinterpret_cast<const float4*>(base);
    const float4 a = ld16<CG>(p + vidx(g, 0, mu, par, h));
    const float4 b = ld16<CG>(p + vidx(g, 1, mu, par, h));
    const float4 c = ld16<CG>(p + vidx(g, 2, mu, par, h));
    Link m;
    m.e[0][0] = {a.x, a.y};
    m.e[0][1] = {a.z, a.w};
    m.e[0][2] = {b.x, b.y};
    m.e[1][0] = {b.z, b.w};
    m.e[1][1] = {c.x, c.y};
    m.e[1][2] = {c.z, c.w};
    m3_rebuild_row2(m);
    return m;
  }
  static __device__ __forceinline__ void store(void* base, const Geom& g, int mu, int par, int h, const Link& m) {
    float4* p = reinterpret_cast<float4*>(base);
    p[vidx(g, 0, mu, par, h)] = make_float4(m.e[0][0].re, m.e[0][0].im, m.e[0][1].re, m.e[0][1].im);
    p[vidx(g, 1, mu, par, h)] = make_float4(m.e[0][2].re, m.e[0][2].im, m.e[1][0].re, m.e[1][0].im);
    p[vidx(g, 2, mu, par, h)] = make_float4(m.e[1][1].re, m.e[1][1].im, m.e[1][2].re, m.e[1][2].im);
  }
};

template <>
struct SU3Policy<double> {
  using Real = double;
  using Link = M3<double>;
  static constexpr int N = 3, COMPS = 9;
  template <bool CG = false>
  static __device__ __forceinline__ Link load(const void* base, const Geom& g, int mu, int par, int h) {
    const double2* p = reinterpret_cast<const double2*>(base);
    Link m;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const double2 v = ld16<CG>(p + vidx(g, k, mu, par, h));
      m.e[k / 3][k % 3] = {v.x, v.y};
    }
    return m;
  }
  static __device__ __forceinline__ void store(void* base, const Geom& g, int mu, int par, int h, const Link& m) {
    double2* p = reinterpret_cast<double2*>(base);
#pragma unroll
    for (int k = 0; k < 9; ++k) p[vidx(g, k, mu, par, h)] = make_double2(m.e[k / 3][k % 3].re, m.e[k / 3][k % 3].im);
  }
};

// ---------------------------------------------------------------------------
// Group algebra used by the generic staple / plaquette code
// ---------------------------------------------------------------------------
template <typename R>
struct Alg {
  // SU(2) (quaternions)
  static __device__ __forceinline__ void zero(Quat<R>& a) { a = {R(0), R(0), R(0), R(0)}; }
  static __device__ __forceinline__ Quat<R> mul(const Quat<R>& a, const Quat<R>& b) { return qmul(a, b); }
  static __device__ __forceinline__ Quat<R> mul_nd(const Quat<R>& a, const Quat<R>& b) { return qmul(a, qdag(b)); }
  static __device__ __forceinline__ void acc_nd(Quat<R>& acc, const Quat<R>& a, const Quat<R>& b) {
    acc = qmul_add(acc, a, qdag(b));
  }
  static __device__ __forceinline__ void acc_dn(Quat<R>& acc, const Quat<R>& a, const Quat<R>& b) {
    acc = qmul_add(acc, qdag(a), b);
  }
  // u B with B = diag(e^{i phi}, e^{-i phi}) = cos phi + i sin phi sigma3
  static __device__ __forceinline__ Quat<R> right_phase(const Quat<R>& u, R c, R s) {
    return qmul_k(u, c, s);
  }
  // Re Tr(a b^+) / N
  static __device__ __forceinline__ R retr_nd_over_n(const Quat<R>& a, const Quat<R>& b) {
    return a.q0 * b.q0 + a.q1 * b.q1 + a.q2 * b.q2 + a.q3 * b.q3;
  }

  // SU(3) (3x3 matrices)
  static __device__ __forceinline__ void zero(M3<R>& a) { m3_zero(a); }
  static __device__ __forceinline__ M3<R> mul(const M3<R>& a, const M3<R>& b) { return m3_mul(a, b); }
  static __device__ __forceinline__ M3<R> mul_nd(const M3<R>& a, const M3<R>& b) { return m3_mul_nd(a, b); }
  static __device__ __forceinline__ void acc_nd(M3<R>& acc, const M3<R>& a, const M3<R>& b) { m3_acc_nd(acc, a, b); }
  static __device__ __forceinline__ void acc_dn(M3<R>& acc, const M3<R>& a, const M3<R>& b) { m3_acc_dn(acc, a, b); }
  // u B with B = diag(e^{i phi}, e^{-i phi}, 1)
  static __device__ __forceinline__ M3<R> right_phase(M3<R> u, R c, R s) {
    const Cx<R> p{c, s}, pc{c, -s};
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      u.e[r][0] = u.e[r][0] * p;
      u.e[r][1] = u.e[r][1] * pc;
    }
    return u;
  }
  static __device__ __forceinline__ R retr_nd_over_n(const M3<R>& a, const M3<R>& b) {
    R s = R(0);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) s = fma(a.e[i][j].re, b.e[i][j].re, fma(a.e[i][j].im, b.e[i][j].im, s));
    return s * R(1.0 / 3.0);
  }
};

template <typename R>
__device__ __forceinline__ void load_phase(const Ctx& a, int x, R& c, R& s);
template <>
__device__ __forceinline__ void load_phase<float>(const Ctx& a, int x, float& c, float& s) {
  const float2 v = __ldg(a.phase32 + x);
  c = v.x;
  s = v.y;
}
template <>
__device__ __forceinline__ void load_phase<double>(const Ctx& a, int x, double& c, double& s) {
  const double2 v = __ldg(a.phase64 + x);
  c = v.x;
  s = v.y;
}

// The diagonal of the SU(3) y-link background at x: b[k] = e^{i theta_k(x)}.
template <typename R>
__device__ __forceinline__ void load_bdiag(const Ctx& a, int x, Cx<R> b[3]);
template <>
__device__ __forceinline__ void load_bdiag<float>(const Ctx& a, int x, Cx<float> b[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float2 v = __ldg(a.phase32 + a.g.Ns + 3 * x + k);
    b[k] = {v.x, v.y};
  }
}
template <>
__device__ __forceinline__ void load_bdiag<double>(const Ctx& a, int x, Cx<double> b[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double2 v = __ldg(a.phase64 + a.g.Ns + 3 * x + k);
    b[k] = {v.x, v.y};
  }
}

// u B for B = diag(b_0, b_1, b_2): column k times b_k.
template <typename R>
__device__ __forceinline__ M3<R> right_bdiag(M3<R> u, const Cx<R> b[3]) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) u.e[r][k] = u.e[r][k] * b[k];
  return u;
}

// Effective link Ut_mu(site) = U_mu(site) B_mu(site).
template <class P, int FIELD, bool CG = false>
__device__ __forceinline__ typename P::Link load_eff(const Ctx& a, int mu, const Site& c) {
  using R = typename P::Real;
  typename P::Link u = P::template load<CG>(a.links, a.g, mu, parity_of(c), lex(a.g, c) >> 1);
  if (FIELD == 1 && mu == 1) {  // lambda3 (sigma3): columns 0 and 1
    R ph_c, ph_s;
    load_phase<R>(a, c.x, ph_c, ph_s);
    u = Alg<R>::right_phase(u, ph_c, ph_s);
  }
  if constexpr (P::N == 3 && FIELD == 2) {  // lambda3 + lambda8: every column
    if (mu == 1) {
      Cx<R> b[3];
      load_bdiag<R>(a, c.x, b);
      u = right_bdiag(u, b);
    }
  }
  return u;
}

// Staple sum of U_mu(x) on effective links:
//   A = sum_{nu != mu} Ut_nu(x+mu) Ut_mu(x+nu)^+ Ut_nu(x)^+
//                    + (Ut_mu(x-nu) Ut_nu(x+mu-nu))^+ Ut_nu(x-nu)
template <class P, int FIELD, bool CG = false>
__device__ __forceinline__ typename P::Link staple(const Ctx& a, const Site& x, int mu) {
  using R = typename P::Real;
  using A = Alg<R>;
  typename P::Link acc;
  A::zero(acc);
  const Site xp = step(a.g, x, mu, +1);
#pragma unroll
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
    const Site xpn = step(a.g, x, nu, +1);
    const Site xmn = step(a.g, x, nu, -1);
    const Site xpmn = step(a.g, xp, nu, -1);
    {
      const auto u1 = load_eff<P, FIELD, CG>(a, nu, xp);
      const auto u2 = load_eff<P, FIELD, CG>(a, mu, xpn);
      const auto u3 = load_eff<P, FIELD, CG>(a, nu, x);
      A::acc_nd(acc, A::mul_nd(u1, u2), u3);
    }
    {
      const auto l1 = load_eff<P, FIELD, CG>(a, nu, xpmn);
      const auto l2 = load_eff<P, FIELD, CG>(a, mu, xmn);
      const auto l3 = load_eff<P, FIELD, CG>(a, nu, xmn);
      A::acc_dn(acc, A::mul(l2, l1), l3);
    }
  }
  return acc;
}

// ---------------------------------------------------------------------------
// SU(3) phase update: Cabibbo-Marinari heat-bath or overrelaxation over the
// SU(2) subgroups (0,1), (1,2), (0,2).
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ Quat<R> block_quat(const M3<R>& w, int i, int j) {
  return {R(0.5) * (w.e[i][i].re + w.e[j][j].re), R(0.5) * (w.e[i][j].im + w.e[j][i].im),
          R(0.5) * (w.e[i][j].re - w.e[j][i].re), R(0.5) * (w.e[i][i].im - w.e[j][j].im)};
}

// m <- R_emb m for the 2x2 matrix of quaternion r on rows (i, j).
template <typename R>
__device__ __forceinline__ void left_rotate(M3<R>& m, const Quat<R>& r, int i, int j) {
  const Cx<R> r00{r.q0, r.q3}, r01{r.q2, r.q1}, r10{-r.q2, r.q1}, r11{r.q0, -r.q3};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const Cx<R> mi = m.e[i][c], mj = m.e[j][c];
    m.e[i][c] = cfma(r01, mj, r00 * mi);
    m.e[j][c] = cfma(r11, mj, r10 * mi);
  }
}

// Register cap of the SU(3) phase kernels: fewer registers per thread let more
// warps stay resident to hide the latency of the 18-link gather.
#ifndef QCD_SU3_PHASE_MAXNREG
#define QCD_SU3_PHASE_MAXNREG 96
#endif

// Frozen-boundary mode: the spatial links of the t = 0 slice are not updated.
__device__ __forceinline__ bool frozen_link(const Ctx& a, int mu, int t) {
  return a.field_mode == 1 && mu < 3 && t == 0;
}

// Reunitarization of one link value (defined with the reunitarization kernels).
template <typename R>
__device__ __forceinline__ Quat<R> su2_reunit_value(const Quat<R>& u);
template <typename R>
__device__ __forceinline__ void su3_reunit_value(M3<R>& m);

template <typename R, int FIELD, int KIND>
__global__ void __maxnreg__(QCD_SU3_PHASE_MAXNREG) su3_phase_kernel(const Ctx a, int parity, int mu) {
  using P = SU3Policy<R>;
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= a.g.Vh) return;
  const Site x = site_of(a.g, parity, h);
  if (frozen_link(a, mu, x.t)) return;
  const M3<R> A = staple<P, FIELD>(a, x, mu);
  M3<R> U = P::load(a.links, a.g, mu, parity, h);
  M3<R> Ut = U;
  if (FIELD == 1 && mu == 1) {
    R bc, bs;
    load_phase<R>(a, x.x, bc, bs);
    Ut = Alg<R>::right_phase(U, bc, bs);
  } else if (FIELD == 2 && mu == 1) {
    Cx<R> b[3];
    load_bdiag<R>(a, x.x, b);
    Ut = right_bdiag(U, b);
  }
  M3<R> W = m3_mul(Ut, A);
  const uint32_t s = uint32_t(lex(a.g, x));
  uint32_t sweep = 0;
  if (KIND == KIND_HB) sweep = *a.sweep;
  unsigned exhausted = 0;
#pragma unroll
  for (int sub = 0; sub < 3; ++sub) {
    const int i = sub == 1 ? 1 : 0;
    const int j = sub == 0 ? 1 : 2;
    const Quat<R> w = block_quat(W, i, j);
    const R k = q_sqrt(qnorm2(w));
    Quat<R> r;
    if (KIND == KIND_HB) {
      const R alpha = R(2.0 / 3.0) * R(a.beta) * k;
      const Stream dir = make_stream(a.k0, a.k1, s, sweep, mu, sub, KIND_DIR);
      if (alpha == R(0)) {
        r = su2_haar<R>(dir, 0u);
      } else {
        const Stream tries = make_stream(a.k0, a.k1, s, sweep, mu, sub, KIND_TRY);
        R delta;
        if (!kp_draw<R>(alpha, a.nhit, tries, delta)) {
          ++exhausted;
          continue;
        }
        const Quat<R> X = su2_with_delta<R>(delta, dir);
        r = qmul(X, qdag(qscale(w, R(1) / k)));
      }
    } else {
      if (k == R(0)) continue;
      const Quat<R> vd = qdag(qscale(w, R(1) / k));
      r = qmul(vd, vd);
    }
    left_rotate(U, r, i, j);
    left_rotate(W, r, i, j);
  }
  if (exhausted) atomicAdd(a.exhausted, (unsigned long long)exhausted);
  if (KIND == KIND_OR_REUNIT) su3_reunit_value<R>(U);
  P::store(a.links, a.g, mu, parity, h, U);
}

// ---------------------------------------------------------------------------
// FP64 reunitarization of every link (one thread per link); optionally
// advances the sweep counter (the end of a sweep).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void advance_if(const Ctx& a, int advance) {
  if (advance && blockIdx.x == 0 && threadIdx.x == 0) *a.sweep_rw += 1u;
}

// 1 / sqrt(n) in FP64 for n near 1: an FP32 seed refined by one Newton step
// y <- y (3 - n y^2) / 2 (relative error 2.4e-7 -> ~1e-13; FP64 storage takes
// a second step).
__device__ __forceinline__ double rsqrt_fp64(double n) {
  const double y = double(rsqrtf(float(n)));
  return y * fma(-0.5 * n, y * y, 1.5);
}

// Exact dot products of FP32 vectors, finished in FP64 (Ogita, Rump & Oishi,
// "Accurate sum and dot product", SIAM J. Sci. Comput. 26 (2005), Dot2):
// every product x*y is split exactly into p + e with p = fl(x*y) and
// e = fma(x, y, -p); the p's are summed with Knuth's error-free TwoSum, the
// rounding errors collected, and the two FP32 parts are added in FP64.  The
// result carries ~2^-46 relative error, the same as an FP64 accumulation of
// the (exactly representable) FP64 products, with two FP32->FP64 conversions
// instead of one per input.
struct Dot2 {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x, float y) {
    const float p = x * y;
    const float e = fmaf(x, y, -p);
    const float t = s + p;
    const float bp = t - s;
    const float err = (s - (t - bp)) + (p - bp);
    s = t;
    c += err + e;
  }
  __device__ __forceinline__ double value() const { return double(s) + double(c); }
};

// u * (1 + d) rounded once: u + d u with d small.
__device__ __forceinline__ float scale1p(float u, float d) { return fmaf(d, u, u); }

// Near-unit norms: a Dot2 sum n = 1 + e with |e| small.  e = (s - 1) + c is
// formed in FP32 (s - 1 exact for s in [1/2, 2]; one rounding, relative
// 2^-24 of e), and (1 + e)^(-1/2) - 1 in FP64 by its series to e^3: for
// |e| <= 2^-8 the dropped terms are below 35/128 e^4 < 7e-11, far below the
// FP32 half-ulp of the corrected output.  Larger deviations take the full
// FP64 square root.
constexpr float REUNIT_SERIES_MAX = 0.00390625f;  // 2^-8
__device__ __forceinline__ float dot2_excess(const Dot2& n) { return (n.s - 1.f) + n.c; }
__device__ __forceinline__ double rsqrt1p_minus1(double e) {
  return e * fma(e, fma(e, -0.3125, 0.375), -0.5);
}

// 1/sqrt(n) - 1 in FP64 for a norm far from 1 (rare), out of line so that the
// hot code of the callers stays small (SU(2): batched scan 0.581 -> 0.575
// ms/sweep; the same for the SU(3) rows measured 1 % slower and is not done).
static __device__ __noinline__ float rsqrt_minus1_far(double n) { return float(rsqrt_fp64(n) - 1.0); }

template <typename R>
__device__ __forceinline__ Quat<R> su2_reunit_value(const Quat<R>& u) {
  if constexpr (sizeof(R) == 4) {
    // |q|^2 exactly, 1/|q| in FP64, q (1 + (1/|q| - 1)) rounded once in FP32
    Dot2 n;
    n.add(u.q0, u.q0);
    n.add(u.q1, u.q1);
    n.add(u.q2, u.q2);
    n.add(u.q3, u.q3);
    const float e = dot2_excess(n);
    const float d = fabsf(e) <= REUNIT_SERIES_MAX ? float(rsqrt1p_minus1(double(e))) : rsqrt_minus1_far(n.value());
    return Quat<R>{scale1p(u.q0, d), scale1p(u.q1, d), scale1p(u.q2, d), scale1p(u.q3, d)};
  } else {
    const double q0 = u.q0, q1 = u.q1, q2 = u.q2, q3 = u.q3;
    const double nn = fma(q0, q0, fma(q1, q1, fma(q2, q2, q3 * q3)));
    double inv = rsqrt_fp64(nn);
    inv *= fma(-0.5 * nn, inv * inv, 1.5);
    return Quat<R>{q0 * inv, q1 * inv, q2 * inv, q3 * inv};
  }
}

template <typename R, bool CG = false>
__device__ __forceinline__ void su2_reunit_link(const Ctx& a, int mu, int par, int h) {
  using P = SU2Policy<R>;
  P::store(a.links, a.g, mu, par, h, su2_reunit_value<R>(P::template load<CG>(a.links, a.g, mu, par, h)));
}

template <typename R>
__global__ void su2_reunit_kernel(const Ctx a, int advance) {
  advance_if(a, advance);
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= 8LL * a.g.Vh) return;
  const int plane = int(idx / a.g.Vh), h = int(idx % a.g.Vh);
  if (a.field_mode == 1 && frozen_link(a, plane >> 1, site_of(a.g, plane & 1, h).t)) return;
  su2_reunit_link<R>(a, plane >> 1, plane & 1, h);
}

// SU(3), FP32 storage (rows 1-2).  Gram-Schmidt written through three exact
// FP64 quantities of the stored rows r, t:
//   n1 = |r|^2,  c = <r, t> = sum conj(r_k) t_k,  m = |t|^2,
//   s1 = 1/sqrt(n1),  q = c / n1,  n2 = |t - q r|^2 = m - |c|^2 / n1,
//   s2 = 1/sqrt(n2),
//   row 1 = s1 r,  row 2 = s2 (t - q r) = t + ((s2 - 1) t - s2 q r),
// all scalars in FP64; each output element is its input plus an FP64-derived
// small correction, so it is rounded once, as an FP64 result stored in FP32.
__device__ __forceinline__ void su3f_reunit_rows(Cx<float> r[3], Cx<float> t[3]) {
  Dot2 n1, m, cre, cim;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    n1.add(r[k].re, r[k].re);
    n1.add(r[k].im, r[k].im);
    m.add(t[k].re, t[k].re);
    m.add(t[k].im, t[k].im);
    cre.add(r[k].re, t[k].re);  // Re conj(r) t = r.re t.re + r.im t.im
    cre.add(r[k].im, t[k].im);
    cim.add(r[k].re, t[k].im);  // Im conj(r) t = r.re t.im - r.im t.re
    cim.add(-r[k].im, t[k].re);
  }
  float d1, d2, bre, bim;
  const float e1 = dot2_excess(n1), em = dot2_excess(m);
  const float cr = cre.s + cre.c, ci = cim.s + cim.c;
  if (fmaxf(fmaxf(fabsf(e1), fabsf(em)), fmaxf(fabsf(cr), fabsf(ci))) <= REUNIT_SERIES_MAX) {
    // near-unitary rows (every sweep): series in the small FP64 quantities
    // e1 = n1 - 1, em = m - 1, c;  1/n1 = 1 - e1 + e1^2 (error c e1^3),
    // n2 - 1 = em - |c|^2 / n1
    const double E1 = e1, EM = em, Cr = cr, Ci = ci;
    const double w = fma(E1, E1 - 1.0, 1.0);
    const double qre = Cr * w, qim = Ci * w;
    const double E2 = fma(-Cr, qre, fma(-Ci, qim, EM));
    const double D2 = rsqrt1p_minus1(E2);
    d1 = float(rsqrt1p_minus1(E1));
    d2 = float(D2);
    bre = float(fma(D2, qre, qre));  // s2 q
    bim = float(fma(D2, qim, qim));
  } else {
    const double N1 = n1.value(), M = m.value(), Cre = cre.value(), Cim = cim.value();
    const double s1 = rsqrt_fp64(N1);
    const double inv_n1 = s1 * s1;
    const double qre = Cre * inv_n1, qim = Cim * inv_n1;
    const double n2 = M - fma(Cre, qre, Cim * qim);
    const double s2 = rsqrt_fp64(n2);
    d1 = float(s1 - 1.0);
    d2 = float(s2 - 1.0);
    bre = float(s2 * qre);  // s2 q
    bim = float(s2 * qim);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    // row 2: t + (d2 t - b r), b = s2 q (complex)
    const float cre_k = fmaf(d2, t[k].re, -fmaf(bre, r[k].re, -bim * r[k].im));
    const float cim_k = fmaf(d2, t[k].im, -fmaf(bre, r[k].im, bim * r[k].re));
    t[k] = {t[k].re + cre_k, t[k].im + cim_k};
    r[k] = {scale1p(r[k].re, d1), scale1p(r[k].im, d1)};
  }
}

// Rows 0-1 of an SU(3) link in FP64 storage.
template <bool CG>
__device__ __forceinline__ void load_rows_fp64(const Ctx& a, int mu, int par, int h, Cx<double> r[2][3]) {
  const double2* p = reinterpret_cast<const double2*>(a.links);
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const double2 v = ld16<CG>(p + vidx(a.g, k, mu, par, h));
    r[k / 3][k % 3] = {v.x, v.y};
  }
}

// Gram-Schmidt of rows 0-1 and row 2 = conj(row0 x row1), FP64 storage.
__device__ __forceinline__ void su3d_reunit(M3<double>& d) {
  double n1 = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) n1 = fma(d.e[0][c].re, d.e[0][c].re, fma(d.e[0][c].im, d.e[0][c].im, n1));
  double i1 = rsqrt_fp64(n1);
  i1 *= fma(-0.5 * n1, i1 * i1, 1.5);
#pragma unroll
  for (int c = 0; c < 3; ++c) d.e[0][c] = scale(d.e[0][c], i1);
  Cx<double> proj{0.0, 0.0};
#pragma unroll
  for (int c = 0; c < 3; ++c) proj = cfma_cn(d.e[0][c], d.e[1][c], proj);
#pragma unroll
  for (int c = 0; c < 3; ++c)
    d.e[1][c] = {fma(-proj.re, d.e[0][c].re, fma(proj.im, d.e[0][c].im, d.e[1][c].re)),
                 fma(-proj.re, d.e[0][c].im, fma(-proj.im, d.e[0][c].re, d.e[1][c].im))};
  double n2 = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) n2 = fma(d.e[1][c].re, d.e[1][c].re, fma(d.e[1][c].im, d.e[1][c].im, n2));
  double i2 = rsqrt_fp64(n2);
  i2 *= fma(-0.5 * n2, i2 * i2, 1.5);
#pragma unroll
  for (int c = 0; c < 3; ++c) d.e[1][c] = scale(d.e[1][c], i2);
  m3_rebuild_row2(d);
}

// Reunitarized link value: FP32 storage keeps rows 0-1 (row 2 is rebuilt on
// every load), FP64 storage all three rows.
template <typename R>
__device__ __forceinline__ void su3_reunit_value(M3<R>& m) {
  if constexpr (sizeof(R) == 4) {
    Cx<float> r[3] = {m.e[0][0], m.e[0][1], m.e[0][2]};
    Cx<float> t[3] = {m.e[1][0], m.e[1][1], m.e[1][2]};
    su3f_reunit_rows(r, t);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      m.e[0][c] = r[c];
      m.e[1][c] = t[c];
    }
  } else {
    su3d_reunit(m);
  }
}

template <typename R, bool CG = false>
__device__ __forceinline__ void su3_reunit_link(const Ctx& a, int mu, int par, int h) {
  using P = SU3Policy<R>;
  if constexpr (sizeof(R) == 4) {
    const float4* p = reinterpret_cast<const float4*>(a.links);
    const float4 x = ld16<CG>(p + vidx(a.g, 0, mu, par, h));
    const float4 y = ld16<CG>(p + vidx(a.g, 1, mu, par, h));
    const float4 z = ld16<CG>(p + vidx(a.g, 2, mu, par, h));
    Cx<float> r[3] = {{x.x, x.y}, {x.z, x.w}, {y.x, y.y}};
    Cx<float> t[3] = {{y.z, y.w}, {z.x, z.y}, {z.z, z.w}};
    su3f_reunit_rows(r, t);
    float4* q = reinterpret_cast<float4*>(a.links);
    q[vidx(a.g, 0, mu, par, h)] = make_float4(r[0].re, r[0].im, r[1].re, r[1].im);
    q[vidx(a.g, 1, mu, par, h)] = make_float4(r[2].re, r[2].im, t[0].re, t[0].im);
    q[vidx(a.g, 2, mu, par, h)] = make_float4(t[1].re, t[1].im, t[2].re, t[2].im);
  } else {
    M3<double> d;
    load_rows_fp64<CG>(a, mu, par, h, d.e);
    su3d_reunit(d);
    P::store(a.links, a.g, mu, par, h, d);
  }
}

template <typename R>
__global__ void su3_reunit_kernel(const Ctx a, int advance) {
  advance_if(a, advance);
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= 8LL * a.g.Vh) return;
  const int plane = int(idx / a.g.Vh), h = int(idx % a.g.Vh);
  if (a.field_mode == 1 && frozen_link(a, plane >> 1, site_of(a.g, plane & 1, h).t)) return;
  su3_reunit_link<R>(a, plane >> 1, plane & 1, h);
}

// ---------------------------------------------------------------------------
// Start: cold (unit links) or hot (Haar links; SU(2) Shoemake, SU(3)
// Mezzadri), generated in FP64 and rounded to the storage.
// ---------------------------------------------------------------------------
__device__ __forceinline__ M3<double> su3_haar_fp64(const Stream& st) {
  double u[20];
#pragma unroll
  for (int b = 0; b < 5; ++b) st.uniforms<double>(uint32_t(b), u + 4 * b);
  M3<double> z;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const double rad = sqrt(-2.0 * log(u[2 * k]));
    double sn, cs;
    sincospi(2.0 * u[2 * k + 1], &sn, &cs);
    z.e[k / 3][k % 3] = {rad * cs, rad * sn};
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int q = 0; q < r; ++q) {
      Cx<double> proj{0.0, 0.0};
#pragma unroll
      for (int c = 0; c < 3; ++c) proj = cfma_cn(z.e[q][c], z.e[r][c], proj);
#pragma unroll
      for (int c = 0; c < 3; ++c) z.e[r][c] = z.e[r][c] - proj * z.e[q][c];
    }
    double n = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) n += z.e[r][c].re * z.e[r][c].re + z.e[r][c].im * z.e[r][c].im;
    n = sqrt(n);
#pragma unroll
    for (int c = 0; c < 3; ++c) z.e[r][c] = {z.e[r][c].re / n, z.e[r][c].im / n};
  }
  // det, then multiply by det^(-1/3) on the principal branch
  const Cx<double> d = z.e[0][0] * (z.e[1][1] * z.e[2][2] - z.e[1][2] * z.e[2][1]) -
                       z.e[0][1] * (z.e[1][0] * z.e[2][2] - z.e[1][2] * z.e[2][0]) +
                       z.e[0][2] * (z.e[1][0] * z.e[2][1] - z.e[1][1] * z.e[2][0]);
  const double th = atan2(d.im, d.re);
  double fs, fc;
  sincos(-th / 3.0, &fs, &fc);
  const Cx<double> fix{fc, fs};
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) z.e[r][c] = z.e[r][c] * fix;
  return z;
}

template <class P>
__global__ void start_kernel(const Ctx a, int hot) {
  using R = typename P::Real;
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= 8LL * a.g.Vh) return;
  const int plane = int(idx / a.g.Vh), h = int(idx % a.g.Vh);
  const int mu = plane >> 1, par = plane & 1;
  const Site x = site_of(a.g, par, h);
  const Stream st = make_stream(a.k0, a.k1, uint32_t(lex(a.g, x)), START_SWEEP_WORD, mu, 0, KIND_START);
  typename P::Link u;
  if constexpr (P::N == 2) {
    const Quat<double> q = hot ? su2_haar<double>(st, 0u) : Quat<double>{1.0, 0.0, 0.0, 0.0};
    u = {R(q.q0), R(q.q1), R(q.q2), R(q.q3)};
  } else {
    M3<double> m;
    if (hot) {
      m = su3_haar_fp64(st);
    } else {
      m3_zero(m);
      m.e[0][0].re = m.e[1][1].re = m.e[2][2].re = 1.0;
    }
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) u.e[r][c] = {R(m.e[r][c].re), R(m.e[r][c].im)};
  }
  P::store(a.links, a.g, mu, par, h, u);
}

// Frozen-boundary mode: the spatial links of the t = 0 slice hold B (y-links
// diag(e^{i phi}, e^{-i phi}) for SU(2), the lambda3 + lambda8 diagonal for
// SU(3); x- and z-links unity).
template <class P>
__global__ void set_frozen_kernel(const Ctx a) {
  using R = typename P::Real;
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t V3 = int64_t(a.g.Ns) * a.g.Ns * a.g.Ns;
  if (idx >= 3 * V3) return;
  const int mu = int(idx / V3), s = int(idx % V3);  // t = 0: s is the spatial index
  const Site x{s % a.g.Ns, (s / a.g.Ns) % a.g.Ns, s / (a.g.Ns * a.g.Ns), 0};
  typename P::Link u;
  if constexpr (P::N == 2) {
    double c = 1.0, sn = 0.0;
    if (mu == 1) {
      const double2 ph = a.phase64[x.x];
      c = ph.x;
      sn = ph.y;
    }
    u = {R(c), R(0), R(0), R(sn)};
  } else {
    m3_zero(u);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double2 b = mu == 1 ? a.phase64[a.g.Ns + 3 * x.x + k] : make_double2(1.0, 0.0);
      u.e[k][k] = {R(b.x), R(b.y)};
    }
  }
  P::store(a.links, a.g, mu, parity_of(x), lex(a.g, x) >> 1, u);
}

// Sum of v over the block (any multiple of 32 threads), in a fixed order,
// written by thread 0; every thread of the block must call it.  No FP64
// arithmetic inside the warp (FP64 runs at a small fraction of the FP32 rate,
// and five dependent FP64 adds per thread at the end of every CTA held its
// warps): each shuffle level adds by Knuth's error-free TwoSum, t + e = s + s' exactly,
// and carries the errors in c; lane 0 adds s + c in FP64.  The warp sum keeps
// a relative error near 2^-48 (the rounding of c), as an FP64 sum of the
// FP32 inputs would; the warps are then added in FP64.
__device__ __forceinline__ void block_sum_f32(float v, double* out) {
  __shared__ double sh[32];
  float s = v, c = 0.f;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float so = __shfl_down_sync(0xffffffffu, s, off), co = __shfl_down_sync(0xffffffffu, c, off);
    const float t = s + so;
    const float bp = t - s;
    const float e = (s - (t - bp)) + (so - bp);
    s = t;
    c += co + e;
  }
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = double(s) + double(c);
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) r += sh[w];
    *out = r;
  }
}

// ---------------------------------------------------------------------------
// Measurements: plaquette (spatial / temporal split) and Polyakov loop.
// Products in the storage precision, sums in FP64: per-thread value, warp
// shuffle, per-block partial, then one block sums the partials in a fixed
// order (deterministic for a given lattice).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void block_sum2(double& v0, double& v1, double* partial_out) {
  __shared__ double sh[2][MEAS_THREADS / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    v0 += __shfl_down_sync(0xffffffffu, v0, off);
    v1 += __shfl_down_sync(0xffffffffu, v1, off);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    sh[0][warp] = v0;
    sh[1][warp] = v1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < MEAS_THREADS / 32; ++w) {
      s0 += sh[0][w];
      s1 += sh[1][w];
    }
    partial_out[0] = s0;
    partial_out[1] = s1;
  }
}

// Plaquettes of one site (index idx over both parities): spatial sum into v0,
// temporal sum into v1, (1/N) Re Tr each, FP64.
template <class P, int FIELD, bool CG = false>
__device__ __forceinline__ void plaquette_site(const Ctx& a, int64_t idx, double& v0, double& v1) {
  using R = typename P::Real;
  using A = Alg<R>;
  const int par = int(idx / a.g.Vh), h = int(idx % a.g.Vh);
  const Site x = site_of(a.g, par, h);
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const Site xpm = step(a.g, x, mu, +1);
    const auto umu = load_eff<P, FIELD, CG>(a, mu, x);
#pragma unroll
    for (int nu = mu + 1; nu < 4; ++nu) {
      const Site xpn = step(a.g, x, nu, +1);
      const auto ab = A::mul(umu, load_eff<P, FIELD, CG>(a, nu, xpm));
      const auto dc = A::mul(load_eff<P, FIELD, CG>(a, nu, x), load_eff<P, FIELD, CG>(a, mu, xpn));
      const double p = double(A::retr_nd_over_n(ab, dc));
      if (nu == 3) v1 += p;
      else v0 += p;
    }
  }
}

// Polyakov loop of spatial site idx: (1/N) Tr of the ordered t-product, FP64.
template <class P, bool CG = false>
__device__ __forceinline__ void polyakov_site(const Ctx& a, int64_t idx, double& v0, double& v1) {
  using R = typename P::Real;
  using A = Alg<R>;
  Site x;
  x.x = int(idx % a.g.Ns);
  x.y = int((idx / a.g.Ns) % a.g.Ns);
  x.z = int(idx / (int64_t(a.g.Ns) * a.g.Ns));
  x.t = 0;
  auto l = P::template load<CG>(a.links, a.g, 3, parity_of(x), lex(a.g, x) >> 1);
  for (int t = 1; t < a.g.Nt; ++t) {
    x.t = t;
    l = A::mul(l, P::template load<CG>(a.links, a.g, 3, parity_of(x), lex(a.g, x) >> 1));
  }
  if constexpr (P::N == 2) {
    v0 += double(l.q0);
  } else {
    v0 += (double(l.e[0][0].re) + double(l.e[1][1].re) + double(l.e[2][2].re)) / 3.0;
    v1 += (double(l.e[0][0].im) + double(l.e[1][1].im) + double(l.e[2][2].im)) / 3.0;
  }
}

template <class P, int FIELD>
__global__ void __launch_bounds__(MEAS_THREADS, 2) measure_kernel(const Ctx a, int n_plaq_blocks) {
  double v0 = 0.0, v1 = 0.0;
  if (int(blockIdx.x) < n_plaq_blocks) {
    const int64_t idx = int64_t(blockIdx.x) * MEAS_THREADS + threadIdx.x;
    if (idx < 2LL * a.g.Vh) plaquette_site<P, FIELD>(a, idx, v0, v1);
  } else {
    const int64_t idx = int64_t(int(blockIdx.x) - n_plaq_blocks) * MEAS_THREADS + threadIdx.x;
    if (idx < int64_t(a.g.Ns) * a.g.Ns * a.g.Ns) polyakov_site<P>(a, idx, v0, v1);
  }
  block_sum2(v0, v1, a.partials + 2 * blockIdx.x);
}

// Sums the per-block partials in a fixed order and normalises:
// out = {P, P_s, P_t, Re L, Im L}.
static __global__ void __launch_bounds__(FINAL_THREADS)
    measure_final_kernel(const Ctx a, int n_plaq_blocks, int n_poly_blocks) {
  __shared__ double sh[4][FINAL_THREADS];
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < n_plaq_blocks; b += FINAL_THREADS) {
    s[0] += a.partials[2 * b];
    s[1] += a.partials[2 * b + 1];
  }
  for (int b = threadIdx.x; b < n_poly_blocks; b += FINAL_THREADS) {
    s[2] += a.partials[2 * (n_plaq_blocks + b)];
    s[3] += a.partials[2 * (n_plaq_blocks + b) + 1];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] = s[k];
  __syncthreads();
  for (int w = FINAL_THREADS / 2; w > 0; w >>= 1) {
    if (int(threadIdx.x) < w) {
#pragma unroll
      for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double V = 2.0 * double(a.g.Vh);
    const double V3 = double(a.g.Ns) * a.g.Ns * a.g.Ns;
    a.meas_out[0] = (sh[0][0] + sh[1][0]) / (6.0 * V);
    a.meas_out[1] = sh[0][0] / (3.0 * V);
    a.meas_out[2] = sh[1][0] / (3.0 * V);
    a.meas_out[3] = sh[2][0] / V3;
    a.meas_out[4] = sh[3][0] / V3;
  }
}

// Final sums of a working sweep's fused measurement: the plaquette partials
// of the three plane-summing phases of the last pass (odd parity, mu = 1, 2,
// 3; `grid` block partials each) and the Polyakov-loop partials.  Writes
// meas_out = {P, P_s, P_t, Re L, Im L, P_1, P_2, P_3}, P_mu the mean plaquette
// of the planes phase mu sums: (y,x); (z,x), (z,y); (t,x), (t,y), (t,z).
// Two strided steps per loop keep six loads of the one block in flight; the
// per-thread sums are reduced by warp shuffles and then across the 32 warps,
// all in a fixed order.
// plane_scale multiplies the plane sums: 1 when the phase kernels summed
// (1/N) Re Tr, 1/N when they summed Re Tr.
static __global__ void __launch_bounds__(FINAL_THREADS) fused_final_kernel(const Ctx a, int grid, double plane_scale) {
  constexpr int NW = FINAL_THREADS / 32;
  __shared__ double sh[5][NW];
  const int nl = meas_poly_blocks(a.g);
  const double* p1 = a.partials + fused_plaq_offset(a.g, 1);
  const double* p2 = a.partials + fused_plaq_offset(a.g, 2);
  const double* p3 = a.partials + fused_plaq_offset(a.g, 3);
  double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  int b = threadIdx.x;
  for (; b + FINAL_THREADS < grid; b += 2 * FINAL_THREADS) {
    const double x1 = p1[b], x2 = p2[b], x3 = p3[b];
    const double y1 = p1[b + FINAL_THREADS], y2 = p2[b + FINAL_THREADS], y3 = p3[b + FINAL_THREADS];
    s[0] += x1;
    s[1] += x2;
    s[2] += x3;
    s[0] += y1;
    s[1] += y2;
    s[2] += y3;
  }
  for (; b < grid; b += FINAL_THREADS) {
    s[0] += p1[b];
    s[1] += p2[b];
    s[2] += p3[b];
  }
  for (int c = threadIdx.x; c < nl; c += FINAL_THREADS) {
    s[3] += a.partials[2 * c];
    s[4] += a.partials[2 * c + 1];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    double v = s[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) sh[k][warp] = v;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      double v = lane < NW ? sh[k][lane] : 0.0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      s[k] = v;
    }
    if (lane == 0) {
      const double V = 2.0 * double(a.g.Vh);
      const double V3 = double(a.g.Ns) * a.g.Ns * a.g.Ns;
      s[0] *= plane_scale;
      s[1] *= plane_scale;
      s[2] *= plane_scale;
      const double sp = s[0] + s[1];
      a.meas_out[0] = (sp + s[2]) / (6.0 * V);
      a.meas_out[1] = sp / (3.0 * V);
      a.meas_out[2] = s[2] / (3.0 * V);
      a.meas_out[3] = s[3] / V3;
      a.meas_out[4] = s[4] / V3;
      a.meas_out[5] = s[0] / V;
      a.meas_out[6] = s[1] / (2.0 * V);
      a.meas_out[7] = s[2] / (3.0 * V);
    }
  }
}

// ---------------------------------------------------------------------------
// Canonical FP64 layout [s][mu][row][col][re,im] <-> device storage
// ---------------------------------------------------------------------------
template <class P>
__global__ void to_canonical_kernel(const Ctx a, double* out) {
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t V = 2LL * a.g.Vh;
  if (idx >= 4 * V) return;
  const int s = int(idx >> 2), mu = int(idx & 3);
  Site x;
  x.x = s % a.g.Ns;
  x.y = (s / a.g.Ns) % a.g.Ns;
  x.z = (s / (a.g.Ns * a.g.Ns)) % a.g.Ns;
  x.t = s / (a.g.Ns * a.g.Ns * a.g.Ns);
  const auto u = P::load(a.links, a.g, mu, parity_of(x), s >> 1);
  constexpr int N = P::N;
  double* o = out + idx * (2 * N * N);
  if constexpr (N == 2) {
    const double q0 = u.q0, q1 = u.q1, q2 = u.q2, q3 = u.q3;
    o[0] = q0; o[1] = q3;    // u00 = q0 + i q3
    o[2] = q2; o[3] = q1;    // u01 = q2 + i q1
    o[4] = -q2; o[5] = q1;   // u10 = -q2 + i q1
    o[6] = q0; o[7] = -q3;   // u11 = q0 - i q3
  } else {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        o[2 * (3 * r + c)] = u.e[r][c].re;
        o[2 * (3 * r + c) + 1] = u.e[r][c].im;
      }
  }
}

template <class P>
__global__ void from_canonical_kernel(const Ctx a, const double* in) {
  using R = typename P::Real;
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t V = 2LL * a.g.Vh;
  if (idx >= 4 * V) return;
  const int s = int(idx >> 2), mu = int(idx & 3);
  Site x;
  x.x = s % a.g.Ns;
  x.y = (s / a.g.Ns) % a.g.Ns;
  x.z = (s / (a.g.Ns * a.g.Ns)) % a.g.Ns;
  x.t = s / (a.g.Ns * a.g.Ns * a.g.Ns);
  constexpr int N = P::N;
  const double* o = in + idx * (2 * N * N);
  typename P::Link u;
  if constexpr (N == 2) {
    // SU(2) projection of the 2x2 matrix
    u.q0 = R(0.5 * (o[0] + o[6]));
    u.q1 = R(0.5 * (o[3] + o[5]));
    u.q2 = R(0.5 * (o[2] - o[4]));
    u.q3 = R(0.5 * (o[1] - o[7]));
  } else {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) u.e[r][c] = {R(o[2 * (3 * r + c)]), R(o[2 * (3 * r + c) + 1])};
  }
  P::store(a.links, a.g, mu, parity_of(x), s >> 1, u);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
inline unsigned grid_for(int64_t n, int block) { return unsigned((n + block - 1) / block); }

template <class P, int FIELD, int KIND>
inline void launch_phase_t(const Ctx& a, int parity, int mu, int block, cudaStream_t st) {
  static_assert(P::N == 3, "SU(2) uses the kernels of qcd_su2c.cuh");
  su3_phase_kernel<typename P::Real, FIELD, KIND><<<grid_for(a.g.Vh, block), block, 0, st>>>(a, parity, mu);
}

template <class P, int KIND>
inline void launch_phase_level(const Ctx& a, int parity, int mu, int block, cudaStream_t st) {
  switch (su3_field_level(a)) {
    case 0: launch_phase_t<P, 0, KIND>(a, parity, mu, block, st); break;
    case 1: launch_phase_t<P, 1, KIND>(a, parity, mu, block, st); break;
    default: launch_phase_t<P, 2, KIND>(a, parity, mu, block, st); break;
  }
}

template <class P>
cudaError_t launch_phase(const Ctx& a, int kind, int parity, int mu, int block, cudaStream_t st) {
  if (kind == KIND_HB) launch_phase_level<P, KIND_HB>(a, parity, mu, block, st);
  else if (kind == KIND_OR) launch_phase_level<P, KIND_OR>(a, parity, mu, block, st);
  else launch_phase_level<P, KIND_OR_REUNIT>(a, parity, mu, block, st);  // (no fused measurement here)
  return cudaGetLastError();
}

template <class P>
cudaError_t launch_reunit(const Ctx& a, int advance, cudaStream_t st) {
  const int block = 256;
  if constexpr (P::N == 2)
    su2_reunit_kernel<typename P::Real><<<grid_for(8LL * a.g.Vh, block), block, 0, st>>>(a, advance);
  else
    su3_reunit_kernel<typename P::Real><<<grid_for(8LL * a.g.Vh, block), block, 0, st>>>(a, advance);
  return cudaGetLastError();
}

template <class P>
cudaError_t launch_start(const Ctx& a, int hot, cudaStream_t st) {
  const int block = 128;
  start_kernel<P><<<grid_for(8LL * a.g.Vh, block), block, 0, st>>>(a, hot);
  return cudaGetLastError();
}

template <class P>
cudaError_t launch_set_frozen(const Ctx& a, cudaStream_t st) {
  const int64_t n = 3LL * a.g.Ns * a.g.Ns * a.g.Ns;
  set_frozen_kernel<P><<<grid_for(n, 256), 256, 0, st>>>(a);
  return cudaGetLastError();
}

template <class P>
cudaError_t launch_measure(const Ctx& a, int effective, cudaStream_t st) {
  const int np = meas_plaq_blocks(a.g), nl = meas_poly_blocks(a.g);
  if constexpr (P::N == 2) {
    if (effective && phases_on_links(a)) measure_kernel<P, 1><<<np + nl, MEAS_THREADS, 0, st>>>(a, np);
    else measure_kernel<P, 0><<<np + nl, MEAS_THREADS, 0, st>>>(a, np);
  } else {
    switch (effective ? su3_field_level(a) : 0) {
      case 0: measure_kernel<P, 0><<<np + nl, MEAS_THREADS, 0, st>>>(a, np); break;
      case 1: measure_kernel<P, 1><<<np + nl, MEAS_THREADS, 0, st>>>(a, np); break;
      default: measure_kernel<P, 2><<<np + nl, MEAS_THREADS, 0, st>>>(a, np); break;
    }
  }
  measure_final_kernel<<<1, FINAL_THREADS, 0, st>>>(a, np, nl);
  return cudaGetLastError();
}

template <class P>
cudaError_t launch_to_canonical(const Ctx& a, double* out, cudaStream_t st) {
  to_canonical_kernel<P><<<grid_for(8LL * a.g.Vh, 256), 256, 0, st>>>(a, out);
  return cudaGetLastError();
}

template <class P>
cudaError_t launch_from_canonical(const Ctx& a, const double* in, cudaStream_t st) {
  from_canonical_kernel<P><<<grid_for(8LL * a.g.Vh, 256), 256, 0, st>>>(a, in);
  return cudaGetLastError();
}

template <class P, int FIELD, int KIND>
int phase_block_limit() {
  cudaFuncAttributes attr{};
  const cudaError_t e = cudaFuncGetAttributes(&attr, su3_phase_kernel<typename P::Real, FIELD, KIND>);
  return e == cudaSuccess ? attr.maxThreadsPerBlock : 0;
}

template <class P>
int max_phase_block() {
  int m = phase_block_limit<P, 0, KIND_HB>();
  m = std::min(m, phase_block_limit<P, 1, KIND_HB>());
  m = std::min(m, phase_block_limit<P, 2, KIND_HB>());
  m = std::min(m, phase_block_limit<P, 0, KIND_OR>());
  m = std::min(m, phase_block_limit<P, 1, KIND_OR>());
  m = std::min(m, phase_block_limit<P, 2, KIND_OR>());
  m = std::min(m, phase_block_limit<P, 0, KIND_OR_REUNIT>());
  m = std::min(m, phase_block_limit<P, 1, KIND_OR_REUNIT>());
  m = std::min(m, phase_block_limit<P, 2, KIND_OR_REUNIT>());
  return m;
}

template <class P>
constexpr PolicyOps make_ops(int precision) {
  return PolicyOps{P::N,
                   precision,
                   P::COMPS,
                   &launch_phase<P>,
                   &launch_reunit<P>,
                   &launch_start<P>,
                   &launch_measure<P>,
                   &launch_to_canonical<P>,
                   &launch_from_canonical<P>,
                   &launch_set_frozen<P>,
                   nullptr,
                   &max_phase_block<P>};
}

}  // namespace qcd
