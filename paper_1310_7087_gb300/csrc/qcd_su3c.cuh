// qcd_su3c.cuh -- phase kernel for SU(3) with FP32 12-real (two-row) links.
//
// Same update as su3_phase_kernel (Cabibbo-Marinari heat-bath or
// overrelaxation of one checkerboard phase), arranged for the compressed
// storage:
//   - the direction mu is a template parameter, so neighbour strides, the
//     parities of the 18 gathered links (odd distance: opposite parity, even
//     distance: same parity) and the links that carry the background phase are
//     all known at compile time;
//   - neighbour sites are reached by adding strides to the lexicographic site
//     index with a wrap correction, not by re-encoding coordinates;
//   - a product of SU(3) matrices is formed row 0-1 only and its row 2 is
//     rebuilt as conj(row0 x row1), which needs fewer multiplies than the full
//     3x3 product whenever a factor is only known by its stored rows;
//   - complex sums of products use the paired FP32 FMA of sm_100 and later
//     (one instruction, two lanes): a complex number is one register pair
//     (re, im), the other factor's real and imaginary parts are broadcast to
//     both lanes, so sum_k a_k b_k is accumulated as X = sum Re(b_k) a_k and
//     Y = sum Im(b_k) a_k and finished as (X.re - Y.im, X.im + Y.re) by one
//     more paired FMA on the swapped Y.  A three-term complex dot product
//     takes 7 paired instructions instead of 12 scalar FMAs.
#pragma once

#include "qcd_kernels.cuh"



namespace qcd {

// Rows 0 and 1 of an SU(3) matrix.
struct Rows2 {
  Cx<float> e[2][3];
};

// ---------------------------------------------------------------------------
// Paired FP32 complex arithmetic.  v2(a) is the register pair (re, im); bc(s)
// broadcasts a real to both lanes (free as an operand of the paired FMA).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 v2(Cx<float> a) { return make_float2(a.re, a.im); }
__device__ __forceinline__ Cx<float> cx2(float2 v) { return {v.x, v.y}; }
__device__ __forceinline__ float2 bc(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 swp(float2 v) { return make_float2(v.y, v.x); }
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// Accumulators of sum_k a_k b_k:  X += Re(b) a,  Y += Im(b) a.
struct XY {
  float2 x, y;
};
__device__ __forceinline__ XY xy_first(Cx<float> a, Cx<float> b) { return {fmul2(bc(b.re), v2(a)), fmul2(bc(b.im), v2(a))}; }
__device__ __forceinline__ void xy_add(XY& s, Cx<float> a, Cx<float> b) {
  s.x = ffma2(bc(b.re), v2(a), s.x);
  s.y = ffma2(bc(b.im), v2(a), s.y);
}
// ... - a b
__device__ __forceinline__ void xy_sub(XY& s, Cx<float> a, Cx<float> b) {
  s.x = ffma2(bc(-b.re), v2(a), s.x);
  s.y = ffma2(bc(-b.im), v2(a), s.y);
}
// sum a_k b_k = (X.re - Y.im, X.im + Y.re)
__device__ __forceinline__ Cx<float> xy_mul(const XY& s) { return cx2(ffma2(swp(s.y), make_float2(-1.f, 1.f), s.x)); }
// sum a_k conj(b_k) = (X.re + Y.im, X.im - Y.re); also sum conj(b_k) a_k
__device__ __forceinline__ Cx<float> xy_conj(const XY& s) { return cx2(ffma2(swp(s.y), make_float2(1.f, -1.f), s.x)); }
// conj(sum a_k b_k) = (X.re - Y.im, -X.im - Y.re)
__device__ __forceinline__ Cx<float> xy_mul_conj(const XY& s) {
  return cx2(ffma2(s.x, make_float2(1.f, -1.f), neg2(swp(s.y))));
}

// conj(a b - c d): one element of a rebuilt third row.
__device__ __forceinline__ Cx<float> cross2(Cx<float> a, Cx<float> b, Cx<float> c, Cx<float> d) {
  XY s = xy_first(a, b);
  xy_sub(s, c, d);
  return xy_mul_conj(s);
}

__device__ __forceinline__ Rows2 su3c_load(const void* base, const Geom& g, int mu, int par, int h) {
  const float4* p = reinterpret_cast<const float4*>(base);
  const float4 a = __ldg(p + vidx(g, 0, mu, par, h));
  const float4 b = __ldg(p + vidx(g, 1, mu, par, h));
  const float4 c = __ldg(p + vidx(g, 2, mu, par, h));
  Rows2 r;
  r.e[0][0] = {a.x, a.y};
  r.e[0][1] = {a.z, a.w};
  r.e[0][2] = {b.x, b.y};
  r.e[1][0] = {b.z, b.w};
  r.e[1][1] = {c.x, c.y};
  r.e[1][2] = {c.z, c.w};
  return r;
}

// (-x, x): with the swapped pair of a, x (i a) = (-x a.im, x a.re).
__device__ __forceinline__ float2 pm(float x) { return make_float2(-x, x); }
// a b for a complex factor b given as b.re and pm(b.im): b.re a + b.im (i a),
// one paired multiply of the swapped pair and one paired multiply-add (the
// accumulator form xy_mul(xy_first(a, b)) takes three).
__device__ __forceinline__ Cx<float> cmul_pm(Cx<float> a, float bre, float2 bim_pm) {
  return cx2(ffma2(bc(bre), v2(a), fmul2(swp(v2(a)), bim_pm)));
}
__device__ __forceinline__ Cx<float> cmul_pm(Cx<float> a, Cx<float> b) { return cmul_pm(a, b.re, pm(b.im)); }

// Right multiplication by B = diag(e^{i phi}, e^{-i phi}, 1).
__device__ __forceinline__ void su3c_phase(Rows2& r, float c, float s) {
  const float2 sp = pm(s), sm = pm(-s);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    r.e[i][0] = cmul_pm(r.e[i][0], c, sp);
    r.e[i][1] = cmul_pm(r.e[i][1], c, sm);
  }
}

__device__ __forceinline__ void su3c_rebuild(M3<float>& m) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
    m.e[2][c] = cross2(m.e[0][c1], m.e[1][c2], m.e[0][c2], m.e[1][c1]);
  }
}

__device__ __forceinline__ M3<float> su3c_full(const Rows2& r) {
  M3<float> m;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    m.e[0][c] = r.e[0][c];
    m.e[1][c] = r.e[1][c];
  }
  su3c_rebuild(m);
  return m;
}

// rows 0-1 of a b^+   (a by its rows 0-1, b full)
__device__ __forceinline__ Rows2 su3c_mul_nd(const Rows2& a, const M3<float>& b) {
  Rows2 c;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      XY s = xy_first(a.e[i][0], b.e[j][0]);
      xy_add(s, a.e[i][1], b.e[j][1]);
      xy_add(s, a.e[i][2], b.e[j][2]);
      c.e[i][j] = xy_conj(s);
    }
  return c;
}

// rows 0-1 of a b   (a by its rows 0-1, b full)
__device__ __forceinline__ Rows2 su3c_mul(const Rows2& a, const M3<float>& b) {
  Rows2 c;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      XY s = xy_first(a.e[i][0], b.e[0][j]);
      xy_add(s, a.e[i][1], b.e[1][j]);
      xy_add(s, a.e[i][2], b.e[2][j]);
      c.e[i][j] = xy_mul(s);
    }
  return c;
}

// a b   (both full)
__device__ __forceinline__ M3<float> su3c_mul3(const M3<float>& a, const M3<float>& b) {
  M3<float> c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      XY s = xy_first(a.e[i][0], b.e[0][j]);
      xy_add(s, a.e[i][1], b.e[1][j]);
      xy_add(s, a.e[i][2], b.e[2][j]);
      c.e[i][j] = xy_mul(s);
    }
  return c;
}

// rows 0-1 of a^+ b   (a, b full): sum_k conj(a_ki) b_kj
__device__ __forceinline__ Rows2 su3c_mul_dn(const M3<float>& a, const M3<float>& b) {
  Rows2 c;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      XY s = xy_first(b.e[0][j], a.e[0][i]);
      xy_add(s, b.e[1][j], a.e[1][i]);
      xy_add(s, b.e[2][j], a.e[2][i]);
      c.e[i][j] = xy_conj(s);
    }
  return c;
}

// m <- R_emb m for the 2x2 matrix of quaternion r on rows (i, j):
// row i' = r00 row i + r01 row j, row j' = r10 row i + r11 row j.
__device__ __forceinline__ void su3c_left_rotate(M3<float>& m, const Quat<float>& r, int i, int j) {
  const Cx<float> r00{r.q0, r.q3}, r01{r.q2, r.q1}, r10{-r.q2, r.q1}, r11{r.q0, -r.q3};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const Cx<float> mi = m.e[i][c], mj = m.e[j][c];
    XY si = xy_first(mi, r00);
    xy_add(si, mj, r01);
    XY sj = xy_first(mi, r10);
    xy_add(sj, mj, r11);
    m.e[i][c] = xy_mul(si);
    m.e[j][c] = xy_mul(sj);
  }
}

// Effective link of direction D at site x, whose parity PAR is known.
template <int FIELD, int D>
__device__ __forceinline__ Rows2 su3c_eff(const Ctx& a, int par, const LexSite& x) {
  Rows2 r = su3c_load(a.links, a.g, D, par, x.s >> 1);
  if (FIELD == 1 && D == 1) {
    const float2 ph = __ldg(a.phase32 + x.c[0]);
    su3c_phase(r, ph.x, ph.y);
  } else if (FIELD == 2 && D == 1) {
    Cx<float> b[3];
    load_bdiag<float>(a, x.c[0], b);
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) r.e[i][k] = cmul_pm(r.e[i][k], b[k]);
  }
  return r;
}

// acc += the SU(3) matrix whose rows 0-1 are t, for an accumulator whose row
// 2 is held conjugated: t's row 2 is conj(t0 x t1), so the conjugated row
// gains t0 x t1, which starts the chain of its products (one paired add less
// per element than su3c_acc).
__device__ __forceinline__ void su3c_acc_c(M3<float>& acc, const Rows2& t) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
    acc.e[0][c] = cx2(fadd2(v2(acc.e[0][c]), v2(t.e[0][c])));
    acc.e[1][c] = cx2(fadd2(v2(acc.e[1][c]), v2(t.e[1][c])));
    XY s{ffma2(bc(t.e[1][c2].re), v2(t.e[0][c1]), v2(acc.e[2][c])), fmul2(bc(t.e[1][c2].im), v2(t.e[0][c1]))};
    xy_sub(s, t.e[0][c2], t.e[1][c1]);
    acc.e[2][c] = xy_mul(s);
  }
}
__device__ __forceinline__ void su3c_conj_row2(M3<float>& m) {
#pragma unroll
  for (int c = 0; c < 3; ++c) m.e[2][c].im = -m.e[2][c].im;
}

// Staple sum of U_MU(x) (x of parity p) on effective links, full 3x3 (row 2
// accumulated conjugated, see su3c_acc_c).
// With SPLIT, *low receives the part of the sum over nu < MU.
template <int FIELD, int MU, bool SPLIT = false>
__device__ __forceinline__ M3<float> su3c_staple(const Ctx& a, int p, const LexSite& x, M3<float>* low = nullptr) {
  M3<float> A;
  m3_zero(A);
  const LexSite xp = lex_step<MU, +1>(a.g, x);
#pragma unroll
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == MU) {
      if (SPLIT) {
        *low = A;
        su3c_conj_row2(*low);
      }
      continue;
    }
    // Each branch of this switch is one static value of NU.
    switch (nu) {
#define QCD_SU3C_NU(NU)                                                                         \
  case NU: {                                                                                      \
    const LexSite xpn = lex_step<NU, +1>(a.g, x);                                                \
    const LexSite xmn = lex_step<NU, -1>(a.g, x);                                                \
    const LexSite xpmn = lex_step<NU, -1>(a.g, xp);                                              \
    /* upper: Ut_nu(x+mu) Ut_mu(x+nu)^+ Ut_nu(x)^+ */                                             \
    const Rows2 x1 = su3c_mul_nd(su3c_eff<FIELD, NU>(a, p ^ 1, xp),                               \
                                 su3c_full(su3c_eff<FIELD, MU>(a, p ^ 1, xpn)));                  \
    su3c_acc_c(A, su3c_mul_nd(x1, su3c_full(su3c_eff<FIELD, NU>(a, p, x))));                      \
    /* lower: (Ut_mu(x-nu) Ut_nu(x+mu-nu))^+ Ut_nu(x-nu) */                                      \
    const M3<float> y = su3c_full(su3c_mul(su3c_eff<FIELD, MU>(a, p ^ 1, xmn),                   \
                                           su3c_full(su3c_eff<FIELD, NU>(a, p, xpmn))));          \
    su3c_acc_c(A, su3c_mul_dn(y, su3c_full(su3c_eff<FIELD, NU>(a, p ^ 1, xmn))));                 \
    break;                                                                                        \
  }
      QCD_SU3C_NU(0)
      QCD_SU3C_NU(1)
      QCD_SU3C_NU(2)
      QCD_SU3C_NU(3)
#undef QCD_SU3C_NU
    }
  }
  su3c_conj_row2(A);
  return A;
}

// The first Kennedy-Pendleton try and the direction of each subgroup do not
// depend on the staple, so the heat-bath kernel draws them before it gathers
// the links, while the gather's first loads are in flight.  Six floats per
// subgroup stay live: alpha delta of try 0, u3^2 of its acceptance test, and
// sin(theta), cos(theta), sin(phi), cos(phi) of the direction, combined with
// the modulus in the order su2_with_delta_u uses, so the result is the same
// to the bit as drawing them after the staple.
struct KpFirst {
  float e, a3, st, ct, sp, cp;
};

__device__ __forceinline__ KpFirst su3c_kp_first(const Stream& tries, const Stream& dir) {
  float u[4], v[4];
  tries.uniforms<float>(0u, u);
  dir.uniforms<float>(0u, v);
  KpFirst f;
  // try 0 as kp_try_f32 forms it, before the division by alpha
  const float c = __cosf(6.283185307179586f * (u[2] - 0.5f));
  f.e = -__logf(u[1]) - __logf(u[0]) * c * c;
  f.a3 = u[3] * u[3];
  // the direction as su2_with_delta_u forms it
  f.ct = 2.f * v[0] - 1.f;
  const float q = v[0] * (1.f - v[0]);
  f.st = 2.f * q * rsqrtf(q);
  __sincosf(6.283185307179586f * (v[1] - 0.5f), &f.sp, &f.cp);
  return f;
}

// Tries 1 .. nhit - 1 after a failed first try (out of line: about 2 % of
// first tries fail at beta 6): delta of the first accepted one, -1 when all
// fail.
static __device__ __noinline__ float su3c_kp_retry(float inv_alpha, int nhit, Stream tries) {
  for (int t = 1; t < nhit; ++t) {
    float u[4], d;
    tries.uniforms<float>(uint32_t(t), u);
    if (kp_try_f32(u, inv_alpha, d)) return d;
  }
  return -1.f;
}

// The alpha = 0 case (Haar-random rotation), out of line: it is never taken at
// beta > 0 and would otherwise sit in the hot code.
static __device__ __noinline__ Quat<float> su3c_haar_rotation(Stream dir) { return su2_haar<float>(dir, 0u); }

// Heat-bath or overrelaxation of U_MU(x) given its staple sum A.
// Returns the link as stored (rows 0-1; row 2 not kept up to date).
template <int FIELD, int KIND, int MU>
__device__ __forceinline__ M3<float> su3c_update(const Ctx& a, int parity, int h, const LexSite& x,
                                                 const M3<float>& A, M3<float> U, const KpFirst* first = nullptr,
                                                 uint32_t sweep = 0) {
  M3<float> Ut = U;
  if (FIELD == 2 && MU == 1) {
    Cx<float> b[3];
    load_bdiag<float>(a, x.c[0], b);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int k = 0; k < 3; ++k) Ut.e[r][k] = cmul_pm(U.e[r][k], b[k]);
  } else if (FIELD == 1 && MU == 1) {
    const float2 ph = __ldg(a.phase32 + x.c[0]);
    const Cx<float> p{ph.x, ph.y}, pc{ph.x, -ph.y};
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      Ut.e[r][0] = cmul_pm(U.e[r][0], p);
      Ut.e[r][1] = cmul_pm(U.e[r][1], pc);
    }
  }
  M3<float> W = su3c_mul3(Ut, A);
  unsigned exhausted = 0;
#pragma unroll
  for (int sub = 0; sub < 3; ++sub) {
    const int i = sub == 1 ? 1 : 0;
    const int j = sub == 0 ? 1 : 2;
    const Quat<float> w = block_quat(W, i, j);
    const float n2 = qnorm2(w);
    Quat<float> r;
    if (KIND == KIND_HB) {
      const float rk = n2 > 0.f ? rsqrtf(n2) : 0.f;  // 1/k (approximate, ~2 ulp)
      const float k = n2 * rk;
      const float alpha = float(2.0 / 3.0) * float(a.beta) * k;
      const Stream dir = make_stream(a.k0, a.k1, uint32_t(x.s), sweep, MU, sub, KIND_DIR);
      if (alpha == 0.f) {
        r = su3c_haar_rotation(dir);
      } else {
        const Stream tries = make_stream(a.k0, a.k1, uint32_t(x.s), sweep, MU, sub, KIND_TRY);
        const float inv_alpha = __fdividef(1.f, alpha);
        float delta = first[sub].e * inv_alpha;
        if (!(first[sub].a3 <= 1.f - 0.5f * delta)) {
          delta = su3c_kp_retry(inv_alpha, a.nhit, tries);
          if (delta < 0.f) {
            ++exhausted;
            continue;
          }
        }
        const float e = delta * (2.f - delta);
        const float m = e * rsqrtf(e);
        const KpFirst& f = first[sub];
        r = qmul(Quat<float>{1.f - delta, -m * f.st * f.cp, -m * f.st * f.sp, m * f.ct}, qdag(qscale(w, rk)));
      }
    } else {
      if (n2 == 0.f) continue;
      const Quat<float> vd = qdag(qscale(w, rsqrtf(n2)));
      r = qmul(vd, vd);
    }
    su3c_left_rotate(U, r, i, j);
    if (sub < 2) su3c_left_rotate(W, r, i, j);
  }
  if (exhausted) atomicAdd(a.exhausted, (unsigned long long)exhausted);
  if (KIND == KIND_OR_REUNIT || KIND == KIND_OR_MEAS) su3_reunit_value<float>(U);
  SU3Policy<float>::store(a.links, a.g, MU, parity, h, U);
  return U;
}

// Register caps (64^3x16, per launch): overrelaxation QCD_SU3_PHASE_MAXNREG
// (96); heat-bath 128 (0.2291 ms; 80 / 96 / 112 / 160 / 200: 0.2581 / 0.2359 /
// 0.2392 / 0.2660 / 0.2640); the reunitarizing overrelaxation of the last
// pass 128 (its group 0.1921 -> 0.1908 ms per launch against 96; 112: 0.1940).
#ifndef QCD_SU3_HB_MAXNREG
#define QCD_SU3_HB_MAXNREG 128
#endif
#ifndef QCD_SU3_REUNIT_MAXNREG
#define QCD_SU3_REUNIT_MAXNREG 128
#endif

// Programmatic dependent launch between consecutive phases of a sweep: each
// CTA lets the next phase's grid be scheduled as soon as it starts (so the
// next grid is resident while this one's last wave finishes), and waits for
// the previous phase's grid to complete, with its stores visible, before it
// reads a link.  Without a programmatic predecessor the wait returns at once.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <int FIELD, int KIND, int MU>
__global__ void __maxnreg__(KIND == KIND_HB          ? QCD_SU3_HB_MAXNREG
                            : KIND == KIND_OR_REUNIT ? QCD_SU3_REUNIT_MAXNREG
                                                     : QCD_SU3_PHASE_MAXNREG) su3c_phase_kernel(const Ctx a, int parity) {
  pdl_launch_dependents();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.g.Vh) return;
  const LexSite x = lex_site_ytz(a.g, parity, i);
  if (frozen_link(a, MU, x.c[3])) return;
  pdl_wait();
  const int h = x.s >> 1;
  KpFirst first[3];
  uint32_t sweep = 0;
  if (KIND == KIND_HB) {
    sweep = *a.sweep;
#pragma unroll
    for (int sub = 0; sub < 3; ++sub)
      first[sub] = su3c_kp_first(make_stream(a.k0, a.k1, uint32_t(x.s), sweep, MU, sub, KIND_TRY),
                                 make_stream(a.k0, a.k1, uint32_t(x.s), sweep, MU, sub, KIND_DIR));
  }
  const M3<float> A = su3c_staple<FIELD, MU>(a, parity, x);
  su3c_update<FIELD, KIND, MU>(a, parity, h, x, A, su3c_full(su3c_load(a.links, a.g, MU, parity, h)), first,
                               sweep);
}

// Last-pass phase (odd parity, MU >= 1) of a working sweep: update and
// reunitarize as KIND_OR_REUNIT, and sum (1/3) Re Tr(Ut_new S) over the
// phase, S the staples of the planes (MU, nu < MU): the plaquettes of those
// planes, each once.  Not used in the frozen-boundary mode.
// The plane-summing phases keep the partial staple live through the update:
// 128 registers (measured 0.196 ms per launch at 64^3x16; 0.201 at 112, 0.207
// at 96 with spills).
#ifndef QCD_SU3_MEAS_MAXNREG
#define QCD_SU3_MEAS_MAXNREG 128
#endif

template <int FIELD, int MU>
__global__ void __maxnreg__(QCD_SU3_MEAS_MAXNREG) su3c_or_meas_kernel(const Ctx a, int parity) {
  pdl_launch_dependents();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float v = 0.f;
  if (i < a.g.Vh) {
    const LexSite x = lex_site_ytz(a.g, parity, i);
    pdl_wait();
    const int h = x.s >> 1;
    M3<float> low;
    const M3<float> A = su3c_staple<FIELD, MU, true>(a, parity, x, &low);
    M3<float> U = su3c_update<FIELD, KIND_OR_MEAS, MU>(a, parity, h, x, A,
                                                       su3c_full(su3c_load(a.links, a.g, MU, parity, h)));
    su3c_rebuild(U);  // row 2 as every later load rebuilds it
    if (FIELD == 1 && MU == 1) {
      const float2 ph = __ldg(a.phase32 + x.c[0]);
      const Cx<float> pp{ph.x, ph.y}, pc{ph.x, -ph.y};
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        U.e[r][0] = cmul_pm(U.e[r][0], pp);
        U.e[r][1] = cmul_pm(U.e[r][1], pc);
      }
    } else if (FIELD == 2 && MU == 1) {
      Cx<float> b[3];
      load_bdiag<float>(a, x.c[0], b);
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) U.e[r][k] = cmul_pm(U.e[r][k], b[k]);
    }
    v = m3_retrace_mul(U, low);  // Re Tr; the final sums take the 1/3
  }
  block_sum_f32(v, a.partials + fused_plaq_offset(a.g, MU) + blockIdx.x);
}

// Polyakov loop of a working sweep's fused measurement: (1/3) Tr of the
// ordered product over t of the t-links of each spatial site, one thread per
// site, products formed by rows 0-1 with row 2 rebuilt as for every FP32 link
// (with the final-sum kernel below: measurement tail 0.107 -> 0.077 ms per
// working sweep at 64^3x16, against the generic full-matrix product;
// splitting each product over 2 or 4 lanes with a shuffle tree measured
// slower, 0.094 / 0.127 ms, and so did unrolling the t-loop by 4, 0.091 ms).
// Block partials of Re and Im, FP64, in a fixed order.
static __global__ void __launch_bounds__(MEAS_THREADS) su3c_poly_kernel(const Ctx a) {
  const long long V3 = (long long)a.g.Ns * a.g.Ns * a.g.Ns;
  const long long site = (long long)blockIdx.x * MEAS_THREADS + threadIdx.x;
  double v0 = 0.0, v1 = 0.0;
  if (site < V3) {
    const int Ns = a.g.Ns;
    const int x = int(site % Ns), y = int((site / Ns) % Ns), z = int(site / ((long long)Ns * Ns));
    const int s0 = x + Ns * (y + Ns * z), xyz = x + y + z;
    Rows2 l = su3c_load(a.links, a.g, 3, xyz & 1, s0 >> 1);
#pragma unroll 1
    for (int t = 1; t < a.g.Nt; ++t)
      l = su3c_mul(l, su3c_full(su3c_load(a.links, a.g, 3, (xyz + t) & 1, int((s0 + (long long)t * V3) >> 1))));
    const Cx<float> l22 = cross2(l.e[0][0], l.e[1][1], l.e[0][1], l.e[1][0]);
    v0 = (double(l.e[0][0].re) + double(l.e[1][1].re) + double(l22.re)) / 3.0;
    v1 = (double(l.e[0][0].im) + double(l.e[1][1].im) + double(l22.im)) / 3.0;
  }
  block_sum2(v0, v1, a.partials + 2 * blockIdx.x);
}

inline cudaError_t su3c_measure_fused_tail(const Ctx& a, int block, cudaStream_t st) {
  su3c_poly_kernel<<<meas_poly_blocks(a.g), MEAS_THREADS, 0, st>>>(a);
  fused_final_kernel<<<1, FINAL_THREADS, 0, st>>>(a, int(grid_for(a.g.Vh, block)), 1.0 / 3.0);
  return cudaGetLastError();
}

// Launch with programmatic stream serialization: the kernel may be scheduled
// before its predecessor in the stream (or in the captured graph) completes;
// it waits in-kernel (pdl_wait) before touching the predecessor's results.
template <typename... P>
inline void launch_programmatic(void (*kernel)(P...), unsigned grid, int block, cudaStream_t st, const Ctx& a,
                                int parity) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(unsigned(block));
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, a, parity);
}

template <int FIELD, int KIND, int MU>
inline void su3c_launch_one(const Ctx& a, int parity, int block, cudaStream_t st) {
  launch_programmatic(su3c_phase_kernel<FIELD, KIND, MU>, grid_for(a.g.Vh, block), block, st, a, parity);
}

template <int FIELD, int KIND>
inline void su3c_launch_kind(const Ctx& a, int parity, int mu, int block, cudaStream_t st) {
  switch (mu) {
    case 0: su3c_launch_one<FIELD, KIND, 0>(a, parity, block, st); break;
    case 1: su3c_launch_one<FIELD, KIND, 1>(a, parity, block, st); break;
    case 2: su3c_launch_one<FIELD, KIND, 2>(a, parity, block, st); break;
    default: su3c_launch_one<FIELD, KIND, 3>(a, parity, block, st); break;
  }
}

template <int KIND>
inline void su3c_launch_level(const Ctx& a, int parity, int mu, int block, cudaStream_t st) {
  switch (su3_field_level(a)) {
    case 0: su3c_launch_kind<0, KIND>(a, parity, mu, block, st); break;
    case 1: su3c_launch_kind<1, KIND>(a, parity, mu, block, st); break;
    default: su3c_launch_kind<2, KIND>(a, parity, mu, block, st); break;
  }
}

// The overrelaxation kernels that also reunitarize (last pass of a sweep),
// with or without the fused plaquette sums, are compiled in their own
// translation unit.
cudaError_t su3c_launch_or_reunit(const Ctx& a, int parity, int mu, int block, cudaStream_t st);
cudaError_t su3c_launch_or_meas(const Ctx& a, int parity, int mu, int block, cudaStream_t st);

inline cudaError_t su3c_launch_phase(const Ctx& a, int kind, int parity, int mu, int block, cudaStream_t st) {
  if (kind == KIND_HB) su3c_launch_level<KIND_HB>(a, parity, mu, block, st);
  else if (kind == KIND_OR) su3c_launch_level<KIND_OR>(a, parity, mu, block, st);
  else if (kind == KIND_OR_MEAS && mu >= 1) return su3c_launch_or_meas(a, parity, mu, block, st);
  else return su3c_launch_or_reunit(a, parity, mu, block, st);
  return cudaGetLastError();
}

template <int FIELD, int KIND, int MU>
int su3c_block_limit() {
  cudaFuncAttributes attr{};
  return cudaFuncGetAttributes(&attr, su3c_phase_kernel<FIELD, KIND, MU>) == cudaSuccess ? attr.maxThreadsPerBlock
                                                                                        : 0;
}

template <int FIELD, int KIND>
int su3c_block_limit_mu() {
  return std::min(std::min(su3c_block_limit<FIELD, KIND, 0>(), su3c_block_limit<FIELD, KIND, 1>()),
                  std::min(su3c_block_limit<FIELD, KIND, 2>(), su3c_block_limit<FIELD, KIND, 3>()));
}

int su3c_or_reunit_max_block();

inline int su3c_max_phase_block() {
  int m = std::min(std::min(su3c_block_limit_mu<0, KIND_HB>(), su3c_block_limit_mu<1, KIND_HB>()),
                   std::min(su3c_block_limit_mu<0, KIND_OR>(), su3c_block_limit_mu<1, KIND_OR>()));
  m = std::min(m, std::min(su3c_block_limit_mu<2, KIND_HB>(), su3c_block_limit_mu<2, KIND_OR>()));
  return std::min(m, su3c_or_reunit_max_block());
}

}  // namespace qcd
