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
//     3x3 product whenever a factor is only known by its stored rows.
#pragma once

#include "qcd_kernels.cuh"



namespace qcd {

// Rows 0 and 1 of an SU(3) matrix.
struct Rows2 {
  Cx<float> e[2][3];
};

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

// Right multiplication by B = diag(e^{i phi}, e^{-i phi}, 1).
__device__ __forceinline__ void su3c_phase(Rows2& r, float c, float s) {
  const Cx<float> p{c, s}, pc{c, -s};
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    r.e[i][0] = r.e[i][0] * p;
    r.e[i][1] = r.e[i][1] * pc;
  }
}

__device__ __forceinline__ M3<float> su3c_full(const Rows2& r) {
  M3<float> m;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    m.e[0][c] = r.e[0][c];
    m.e[1][c] = r.e[1][c];
  }
  m3_rebuild_row2(m);
  return m;
}

// rows 0-1 of a b^+   (a by its rows 0-1, b full)
__device__ __forceinline__ Rows2 su3c_mul_nd(const Rows2& a, const M3<float>& b) {
  Rows2 c;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Cx<float> s{0.f, 0.f};
#pragma unroll
      for (int k = 0; k < 3; ++k) s = cfma_nc(a.e[i][k], b.e[j][k], s);
      c.e[i][j] = s;
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
      Cx<float> s = a.e[i][0] * b.e[0][j];
      s = cfma(a.e[i][1], b.e[1][j], s);
      s = cfma(a.e[i][2], b.e[2][j], s);
      c.e[i][j] = s;
    }
  return c;
}

// rows 0-1 of a^+ b   (a, b full)
__device__ __forceinline__ Rows2 su3c_mul_dn(const M3<float>& a, const M3<float>& b) {
  Rows2 c;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Cx<float> s{0.f, 0.f};
#pragma unroll
      for (int k = 0; k < 3; ++k) s = cfma_cn(a.e[k][i], b.e[k][j], s);
      c.e[i][j] = s;
    }
  return c;
}

// acc += the SU(3) matrix whose rows 0-1 are t
__device__ __forceinline__ void su3c_acc(M3<float>& acc, const Rows2& t) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
    acc.e[0][c] = acc.e[0][c] + t.e[0][c];
    acc.e[1][c] = acc.e[1][c] + t.e[1][c];
    const Cx<float> v = t.e[0][c1] * t.e[1][c2] - t.e[0][c2] * t.e[1][c1];
    acc.e[2][c] = acc.e[2][c] + conj(v);
  }
}

// Effective link of direction D at site x, whose parity PAR is known.
template <bool FIELD, int D>
__device__ __forceinline__ Rows2 su3c_eff(const Ctx& a, int par, const LexSite& x) {
  Rows2 r = su3c_load(a.links, a.g, D, par, x.s >> 1);
  if (FIELD && D == 1) {
    const float2 ph = __ldg(a.phase32 + x.c[0]);
    su3c_phase(r, ph.x, ph.y);
  }
  return r;
}

// Staple sum of U_MU(x) (x of parity p) on effective links, full 3x3.
template <bool FIELD, int MU>
__device__ __forceinline__ M3<float> su3c_staple(const Ctx& a, int p, const LexSite& x) {
  M3<float> A;
  m3_zero(A);
  const LexSite xp = lex_step<MU, +1>(a.g, x);
#pragma unroll
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == MU) continue;
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
    su3c_acc(A, su3c_mul_nd(x1, su3c_full(su3c_eff<FIELD, NU>(a, p, x))));                        \
    /* lower: (Ut_mu(x-nu) Ut_nu(x+mu-nu))^+ Ut_nu(x-nu) */                                      \
    const M3<float> y = su3c_full(su3c_mul(su3c_eff<FIELD, MU>(a, p ^ 1, xmn),                   \
                                           su3c_full(su3c_eff<FIELD, NU>(a, p, xpmn))));          \
    su3c_acc(A, su3c_mul_dn(y, su3c_full(su3c_eff<FIELD, NU>(a, p ^ 1, xmn))));                   \
    break;                                                                                        \
  }
      QCD_SU3C_NU(0)
      QCD_SU3C_NU(1)
      QCD_SU3C_NU(2)
      QCD_SU3C_NU(3)
#undef QCD_SU3C_NU
    }
  }
  return A;
}

// Heat-bath or overrelaxation of U_MU(x) given its staple sum A.
template <bool FIELD, int KIND, int MU>
__device__ __forceinline__ void su3c_update(const Ctx& a, int parity, int h, const LexSite& x, const M3<float>& A,
                                            M3<float> U) {
  M3<float> Ut = U;
  if (FIELD && MU == 1) {
    const float2 ph = __ldg(a.phase32 + x.c[0]);
    Ut = Alg<float>::right_phase(U, ph.x, ph.y);
  }
  M3<float> W = m3_mul(Ut, A);
  uint32_t sweep = 0;
  if (KIND == KIND_HB) sweep = *a.sweep;
  unsigned exhausted = 0;
#pragma unroll
  for (int sub = 0; sub < 3; ++sub) {
    const int i = sub == 1 ? 1 : 0;
    const int j = sub == 0 ? 1 : 2;
    const Quat<float> w = block_quat(W, i, j);
    const float n2 = qnorm2(w);
    Quat<float> r;
    if (KIND == KIND_HB) {
      const float k = sqrtf(n2);
      const float alpha = float(2.0 / 3.0) * float(a.beta) * k;
      const Stream dir = make_stream(a.k0, a.k1, uint32_t(x.s), sweep, MU, sub, KIND_DIR);
      if (alpha == 0.f) {
        r = su2_haar<float>(dir, 0u);
      } else {
        const Stream tries = make_stream(a.k0, a.k1, uint32_t(x.s), sweep, MU, sub, KIND_TRY);
        float delta;
        if (!kp_draw<float>(alpha, a.nhit, tries, delta)) {
          ++exhausted;
          continue;
        }
        const Quat<float> X = su2_with_delta<float>(delta, dir);
        r = qmul(X, qdag(qscale(w, 1.f / k)));
      }
    } else {
      if (n2 == 0.f) continue;
      const Quat<float> vd = qdag(qscale(w, rsqrtf(n2)));
      r = qmul(vd, vd);
    }
    left_rotate(U, r, i, j);
    if (sub < 2) left_rotate(W, r, i, j);
  }
  if (exhausted) atomicAdd(a.exhausted, (unsigned long long)exhausted);
  SU3Policy<float>::store(a.links, a.g, MU, parity, h, U);
}

template <bool FIELD, int KIND, int MU>
__global__ void __maxnreg__(QCD_SU3_PHASE_MAXNREG) su3c_phase_kernel(const Ctx a, int parity) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.g.Vh) return;
  const LexSite x = lex_site_ytz(a.g, parity, i);
  if (frozen_link(a, MU, x.c[3])) return;
  const int h = x.s >> 1;
  const M3<float> A = su3c_staple<FIELD, MU>(a, parity, x);
  su3c_update<FIELD, KIND, MU>(a, parity, h, x, A, su3c_full(su3c_load(a.links, a.g, MU, parity, h)));
}

template <bool FIELD, int KIND, int MU>
inline void su3c_launch_one(const Ctx& a, int parity, int block, cudaStream_t st) {
  const unsigned grid = grid_for(a.g.Vh, block);
  su3c_phase_kernel<FIELD, KIND, MU><<<grid, block, 0, st>>>(a, parity);
}

template <bool FIELD, int KIND>
inline void su3c_launch_kind(const Ctx& a, int parity, int mu, int block, cudaStream_t st) {
  switch (mu) {
    case 0: su3c_launch_one<FIELD, KIND, 0>(a, parity, block, st); break;
    case 1: su3c_launch_one<FIELD, KIND, 1>(a, parity, block, st); break;
    case 2: su3c_launch_one<FIELD, KIND, 2>(a, parity, block, st); break;
    default: su3c_launch_one<FIELD, KIND, 3>(a, parity, block, st); break;
  }
}

inline cudaError_t su3c_launch_phase(const Ctx& a, int kind, int parity, int mu, int block, cudaStream_t st) {
  const bool field = phases_on_links(a);
  if (kind == KIND_HB) {
    if (field) su3c_launch_kind<true, KIND_HB>(a, parity, mu, block, st);
    else su3c_launch_kind<false, KIND_HB>(a, parity, mu, block, st);
  } else {
    if (field) su3c_launch_kind<true, KIND_OR>(a, parity, mu, block, st);
    else su3c_launch_kind<false, KIND_OR>(a, parity, mu, block, st);
  }
  return cudaGetLastError();
}

template <bool FIELD, int KIND, int MU>
int su3c_block_limit() {
  cudaFuncAttributes attr{};
  return cudaFuncGetAttributes(&attr, su3c_phase_kernel<FIELD, KIND, MU>) == cudaSuccess ? attr.maxThreadsPerBlock
                                                                                        : 0;
}

template <bool FIELD, int KIND>
int su3c_block_limit_mu() {
  return std::min(std::min(su3c_block_limit<FIELD, KIND, 0>(), su3c_block_limit<FIELD, KIND, 1>()),
                  std::min(su3c_block_limit<FIELD, KIND, 2>(), su3c_block_limit<FIELD, KIND, 3>()));
}

inline int su3c_max_phase_block() {
  return std::min(std::min(su3c_block_limit_mu<false, KIND_HB>(), su3c_block_limit_mu<true, KIND_HB>()),
                  std::min(su3c_block_limit_mu<false, KIND_OR>(), su3c_block_limit_mu<true, KIND_OR>()));
}

}  // namespace qcd
