// qcd_su2c.cuh -- SU(2) phase update (Kennedy-Pendleton heat-bath or
// overrelaxation) with the direction MU as a template parameter: neighbour
// sites are reached by stride steps on the lexicographic index and the
// parities of the gathered links are known at compile time.  Used by the
// single-lattice phase kernels and by the batched persistent kernel (CG =
// true there: links change inside that launch, so they are read through L2).
#pragma once

#include "qcd_kernels.cuh"

namespace qcd {

template <typename R, bool FIELD, int D, bool CG>
__device__ __forceinline__ Quat<R> su2c_eff(const Ctx& a, int par, const LexSite& x) {
  Quat<R> u = SU2Policy<R>::template load<CG>(a.links, a.g, D, par, x.s >> 1);
  if (FIELD && D == 1) {
    R c, s;
    load_phase<R>(a, x.c[0], c, s);
    u = qmul(u, Quat<R>{c, R(0), R(0), s});
  }
  return u;
}

// Staple sum of U_MU(x), x of parity p, on effective links (quaternion form).
template <typename R, bool FIELD, int MU, bool CG>
__device__ __forceinline__ Quat<R> su2c_staple(const Ctx& a, int p, const LexSite& x) {
  Quat<R> A{R(0), R(0), R(0), R(0)};
  const LexSite xp = lex_step<MU, +1>(a.g, x);
#pragma unroll
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == MU) continue;
    switch (nu) {
#define QCD_SU2C_NU(NU)                                                                       \
  case NU: {                                                                                    \
    const LexSite xpn = lex_step<NU, +1>(a.g, x);                                               \
    const LexSite xmn = lex_step<NU, -1>(a.g, x);                                               \
    const LexSite xpmn = lex_step<NU, -1>(a.g, xp);                                             \
    /* upper: Ut_nu(x+mu) Ut_mu(x+nu)^+ Ut_nu(x)^+ */                                           \
    A = qadd(A, qmul(qmul(su2c_eff<R, FIELD, NU, CG>(a, p ^ 1, xp),                             \
                          qdag(su2c_eff<R, FIELD, MU, CG>(a, p ^ 1, xpn))),                     \
                     qdag(su2c_eff<R, FIELD, NU, CG>(a, p, x))));                               \
    /* lower: (Ut_mu(x-nu) Ut_nu(x+mu-nu))^+ Ut_nu(x-nu) */                                    \
    A = qadd(A, qmul(qdag(qmul(su2c_eff<R, FIELD, MU, CG>(a, p ^ 1, xmn),                       \
                               su2c_eff<R, FIELD, NU, CG>(a, p, xpmn))),                        \
                     su2c_eff<R, FIELD, NU, CG>(a, p ^ 1, xmn)));                               \
    break;                                                                                      \
  }
      QCD_SU2C_NU(0)
      QCD_SU2C_NU(1)
      QCD_SU2C_NU(2)
      QCD_SU2C_NU(3)
#undef QCD_SU2C_NU
    }
  }
  return A;
}

// One link update: A = k V (k = sqrt(det A)); heat-bath Ut_new = X V^+ with X
// drawn by Kennedy-Pendleton (Haar when alpha = beta k = 0), overrelaxation
// Ut_new = V^+ Ut^+ V^+; stored U = Ut_new B^+.
template <typename R, bool FIELD, int KIND, int MU, bool CG>
__device__ __forceinline__ void su2c_update(const Ctx& a, int parity, int h, uint32_t sweep) {
  using P = SU2Policy<R>;
  constexpr bool reunit = KIND == KIND_OR_REUNIT;
  const LexSite x = lex_site(a, parity, h);
  if (frozen_link(a, MU, x.c[3])) return;
  // a link left as it is still gets the reunitarization the pass carries
  auto keep = [&]() {
    if (reunit) P::store(a.links, a.g, MU, parity, h, su2_reunit_value<R>(P::template load<CG>(a.links, a.g, MU, parity, h)));
  };
  const Quat<R> A = su2c_staple<R, FIELD, MU, CG>(a, parity, x);
  const R k2 = qnorm2(A);
  constexpr bool phased = FIELD && MU == 1;
  R bc = R(1), bs = R(0);
  if (phased) load_phase<R>(a, x.c[0], bc, bs);
  const Quat<R> Bd{bc, R(0), R(0), -bs};  // B^+
  Quat<R> ut_new;
  if (KIND == KIND_HB) {
    const R k = q_sqrt(k2);
    const R alpha = R(a.beta) * k;
    const Stream dir = make_stream(a.k0, a.k1, uint32_t(x.s), sweep, MU, 0, KIND_DIR);
    if (alpha == R(0)) {
      ut_new = su2_haar<R>(dir, 0u);
    } else {
      const Stream tries = make_stream(a.k0, a.k1, uint32_t(x.s), sweep, MU, 0, KIND_TRY);
      R delta;
      if (!kp_draw<R>(alpha, a.nhit, tries, delta)) {
        atomicAdd(a.exhausted, 1ull);
        keep();
        return;  // keep the link
      }
      ut_new = qmul(su2_with_delta<R>(delta, dir), qdag(qscale(A, R(1) / k)));
    }
  } else {
    if (k2 == R(0)) {
      keep();
      return;
    }
    const Quat<R> Vd = qdag(qscale(A, R(1) / q_sqrt(k2)));
    Quat<R> ut = P::template load<CG>(a.links, a.g, MU, parity, h);
    if (phased) ut = qmul(ut, qdag(Bd));
    ut_new = qmul(qmul(Vd, qdag(ut)), Vd);
  }
  const Quat<R> u_new = phased ? qmul(ut_new, Bd) : ut_new;
  P::store(a.links, a.g, MU, parity, h, reunit ? su2_reunit_value<R>(u_new) : u_new);
}

template <typename R, bool FIELD, int KIND, int MU>
__global__ void su2c_phase_kernel(const Ctx a, int parity) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= a.g.Vh) return;
  su2c_update<R, FIELD, KIND, MU, false>(a, parity, h, KIND == KIND_HB ? *a.sweep : 0u);
}

template <typename R, bool FIELD, int KIND>
inline void su2c_launch_kind(const Ctx& a, int parity, int mu, int block, cudaStream_t st) {
  const unsigned grid = grid_for(a.g.Vh, block);
  switch (mu) {
    case 0: su2c_phase_kernel<R, FIELD, KIND, 0><<<grid, block, 0, st>>>(a, parity); break;
    case 1: su2c_phase_kernel<R, FIELD, KIND, 1><<<grid, block, 0, st>>>(a, parity); break;
    case 2: su2c_phase_kernel<R, FIELD, KIND, 2><<<grid, block, 0, st>>>(a, parity); break;
    default: su2c_phase_kernel<R, FIELD, KIND, 3><<<grid, block, 0, st>>>(a, parity); break;
  }
}

template <typename R>
cudaError_t su2c_launch_phase(const Ctx& a, int kind, int parity, int mu, int block, cudaStream_t st) {
  const bool field = phases_on_links(a);
  if (kind == KIND_HB) {
    if (field) su2c_launch_kind<R, true, KIND_HB>(a, parity, mu, block, st);
    else su2c_launch_kind<R, false, KIND_HB>(a, parity, mu, block, st);
  } else if (kind == KIND_OR) {
    if (field) su2c_launch_kind<R, true, KIND_OR>(a, parity, mu, block, st);
    else su2c_launch_kind<R, false, KIND_OR>(a, parity, mu, block, st);
  } else {  // KIND_OR_REUNIT (no fused measurement for SU(2))
    if (field) su2c_launch_kind<R, true, KIND_OR_REUNIT>(a, parity, mu, block, st);
    else su2c_launch_kind<R, false, KIND_OR_REUNIT>(a, parity, mu, block, st);
  }
  return cudaGetLastError();
}

template <typename R, bool FIELD, int KIND, int MU>
int su2c_limit() {
  cudaFuncAttributes attr{};
  return cudaFuncGetAttributes(&attr, su2c_phase_kernel<R, FIELD, KIND, MU>) == cudaSuccess ? attr.maxThreadsPerBlock
                                                                                          : 0;
}

template <typename R, bool FIELD, int KIND>
int su2c_limit_mu() {
  return std::min(std::min(su2c_limit<R, FIELD, KIND, 0>(), su2c_limit<R, FIELD, KIND, 1>()),
                  std::min(su2c_limit<R, FIELD, KIND, 2>(), su2c_limit<R, FIELD, KIND, 3>()));
}

template <typename R>
int su2c_max_phase_block() {
  const int m = std::min(std::min(su2c_limit_mu<R, false, KIND_HB>(), su2c_limit_mu<R, true, KIND_HB>()),
                         std::min(su2c_limit_mu<R, false, KIND_OR>(), su2c_limit_mu<R, true, KIND_OR>()));
  return std::min(m, std::min(su2c_limit_mu<R, false, KIND_OR_REUNIT>(), su2c_limit_mu<R, true, KIND_OR_REUNIT>()));
}

template <typename R>
PolicyOps su2c_ops(int precision) {
  using P = SU2Policy<R>;
  return PolicyOps{2,
                   precision,
                   P::COMPS,
                   &su2c_launch_phase<R>,
                   &launch_reunit<P>,
                   &launch_start<P>,
                   &launch_measure<P>,
                   &launch_to_canonical<P>,
                   &launch_from_canonical<P>,
                   &launch_set_frozen<P>,
                   nullptr,
                   &su2c_max_phase_block<R>};
}

}  // namespace qcd
