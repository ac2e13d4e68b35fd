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
    u = qmul_k(u, c, s);
  }
  return u;
}

// Staple sum of U_MU(x), x of parity p, on effective links (quaternion form);
// with SPLIT, *low receives the part over nu < MU.
template <typename R, bool FIELD, int MU, bool CG, bool SPLIT = false>
__device__ __forceinline__ Quat<R> su2c_staple(const Ctx& a, int p, const LexSite& x, Quat<R>* low = nullptr) {
  Quat<R> A{R(0), R(0), R(0), R(0)};
  const LexSite xp = lex_step<MU, +1>(a.g, x);
#pragma unroll
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == MU) {
      if (SPLIT) *low = A;
      continue;
    }
    switch (nu) {
#define QCD_SU2C_NU(NU)                                                                       \
  case NU: {                                                                                    \
    const LexSite xpn = lex_step<NU, +1>(a.g, x);                                               \
    const LexSite xmn = lex_step<NU, -1>(a.g, x);                                               \
    const LexSite xpmn = lex_step<NU, -1>(a.g, xp);                                             \
    /* upper: Ut_nu(x+mu) Ut_mu(x+nu)^+ Ut_nu(x)^+ */                                           \
    A = qmul_add(A, qmul(su2c_eff<R, FIELD, NU, CG>(a, p ^ 1, xp),                              \
                         qdag(su2c_eff<R, FIELD, MU, CG>(a, p ^ 1, xpn))),                      \
                 qdag(su2c_eff<R, FIELD, NU, CG>(a, p, x)));                                    \
    /* lower: (Ut_mu(x-nu) Ut_nu(x+mu-nu))^+ Ut_nu(x-nu) */                                    \
    A = qmul_add(A, qdag(qmul(su2c_eff<R, FIELD, MU, CG>(a, p ^ 1, xmn),                        \
                              su2c_eff<R, FIELD, NU, CG>(a, p, xpmn))),                         \
                 su2c_eff<R, FIELD, NU, CG>(a, p ^ 1, xmn));                                    \
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

// 1 / sqrt(k2) for k2 >= 0 (0 for k2 = 0).  FP32: the approximate reciprocal
// square root (about 2 ulp), as in the SU(3) FP32 update; its error moves the
// new link off the group by about 1e-7, which the reunitarization of the last
// pass removes.  FP64: correctly rounded.
__device__ __forceinline__ float su2_rnorm(float k2) { return k2 > 0.f ? rsqrtf(k2) : 0.f; }
__device__ __forceinline__ double su2_rnorm(double k2) { return k2 > 0.0 ? 1.0 / sqrt(k2) : 0.0; }
// k = sqrt(k2) and 1/k (0 for k2 = 0).
__device__ __forceinline__ void su2_norms(float k2, float& k, float& rk) {
  rk = su2_rnorm(k2);
  k = k2 * rk;
}
__device__ __forceinline__ void su2_norms(double k2, double& k, double& rk) {
  k = sqrt(k2);
  rk = k > 0.0 ? 1.0 / k : 0.0;
}

// One link update: A = k V (k = sqrt(det A)); heat-bath Ut_new = X V^+ with X
// drawn by Kennedy-Pendleton (Haar when alpha = beta k = 0), overrelaxation
// Ut_new = V^+ Ut^+ V^+; stored U = Ut_new B^+.  KIND_OR_REUNIT and
// KIND_OR_MEAS reunitarize the stored link; KIND_OR_MEAS (odd parity, MU >= 1
// of a working sweep's last pass) returns (1/2) Re Tr(Ut A_nu) summed over
// nu < MU for the final link, i.e. the plaquettes of the planes (MU, nu < MU)
// through it.
// x: the site, of parity `parity`, with its lexicographic index and coordinates.
template <typename R, bool FIELD, int KIND, int MU, bool CG>
__device__ __forceinline__ R su2c_update_at(const Ctx& a, int parity, const LexSite& x, uint32_t sweep) {
  using P = SU2Policy<R>;
  constexpr bool reunit = KIND == KIND_OR_REUNIT || KIND == KIND_OR_MEAS;
  constexpr bool meas = KIND == KIND_OR_MEAS;
  const int h = x.s >> 1;
  if (frozen_link(a, MU, x.c[3])) return R(0);
  Quat<R> low{R(0), R(0), R(0), R(0)};
  const Quat<R> A = su2c_staple<R, FIELD, MU, CG, meas>(a, parity, x, &low);
  const R k2 = qnorm2(A);
  constexpr bool phased = FIELD && MU == 1;
  R bc = R(1), bs = R(0);
  if (phased) load_phase<R>(a, x.c[0], bc, bs);
  Quat<R> u_new;
  bool keep = false;  // the link stays as it is (it still gets the reunitarization)
  if (KIND == KIND_HB) {
    R k, rk;  // sqrt(k2), 1/k
    su2_norms(k2, k, rk);
    const R alpha = R(a.beta) * k;
    const Stream dir = make_stream(a.k0, a.k1, uint32_t(x.s), sweep, MU, 0, KIND_DIR);
    Quat<R> ut_new;
    if (alpha == R(0)) {
      ut_new = su2_haar<R>(dir, 0u);
    } else {
      const Stream tries = make_stream(a.k0, a.k1, uint32_t(x.s), sweep, MU, 0, KIND_TRY);
      Quat<R> X;
      bool ok;
      if constexpr (sizeof(R) == 4) {
        ok = kp_draw_dir_f32(alpha, a.nhit, tries, dir, X);
      } else {
        R delta;
        ok = kp_draw<R>(alpha, a.nhit, tries, delta);
        if (ok) X = su2_with_delta<R>(delta, dir);
      }
      if (!ok) {
        atomicAdd(a.exhausted, 1ull);
        keep = true;
      } else {
        ut_new = qmul(X, qdag(qscale(A, rk)));
      }
    }
    if (keep) return R(0);  // heat-bath passes carry no reunitarization
    u_new = phased ? qmul_k(ut_new, bc, -bs) : ut_new;  // Ut_new B^+
  } else {
    const Quat<R> u = P::template load<CG>(a.links, a.g, MU, parity, h);
    if (k2 == R(0)) {
      if (!reunit) return R(0);
      u_new = u;
    } else {
      const Quat<R> Vd = qdag(qscale(A, su2_rnorm(k2)));
      const Quat<R> ut = phased ? qmul_k(u, bc, bs) : u;
      const Quat<R> ut_new = qmul(qmul(Vd, qdag(ut)), Vd);
      u_new = phased ? qmul_k(ut_new, bc, -bs) : ut_new;
    }
  }
  if (reunit) u_new = su2_reunit_value<R>(u_new);
  P::store(a.links, a.g, MU, parity, h, u_new);
  if (!meas) return R(0);
  const Quat<R> ut_final = phased ? qmul_k(u_new, bc, bs) : u_new;
  return qmul(ut_final, low).q0;  // (1/2) Re Tr(Ut low)
}

template <typename R, bool FIELD, int KIND, int MU, bool CG>
__device__ __forceinline__ R su2c_update(const Ctx& a, int parity, int h, uint32_t sweep) {
  return su2c_update_at<R, FIELD, KIND, MU, CG>(a, parity, lex_site(a, parity, h), sweep);
}

template <typename R, bool FIELD, int KIND, int MU>
__global__ void su2c_phase_kernel(const Ctx a, int parity) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= a.g.Vh) return;
  su2c_update<R, FIELD, KIND, MU, false>(a, parity, h, KIND == KIND_HB ? *a.sweep : 0u);
}

// Sum of v over the block (any multiple of 32 threads) in a fixed order.
__device__ __forceinline__ void su2c_block_sum(double v, double* out) {
  __shared__ double sh[32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) s += sh[w];
    *out = s;
  }
}

// Last-pass phase (odd parity, MU >= 1) of a working sweep: update,
// reunitarize and sum the plaquettes of the planes (MU, nu < MU).
template <typename R, bool FIELD, int MU>
__global__ void su2c_or_meas_kernel(const Ctx a, int parity) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  R v = R(0);
  if (h < a.g.Vh) v = su2c_update<R, FIELD, KIND_OR_MEAS, MU, false>(a, parity, h, 0u);
  if constexpr (sizeof(R) == 4) block_sum_f32(v, a.partials + fused_plaq_offset(a.g, MU) + blockIdx.x);
  else su2c_block_sum(v, a.partials + fused_plaq_offset(a.g, MU) + blockIdx.x);
}

template <typename R>
cudaError_t su2c_measure_fused_tail(const Ctx& a, int block, cudaStream_t st) {
  const int nl = meas_poly_blocks(a.g);
  measure_kernel<SU2Policy<R>, 0><<<nl, MEAS_THREADS, 0, st>>>(a, 0);  // Polyakov loop only
  fused_final_kernel<<<1, FINAL_THREADS, 0, st>>>(a, int(grid_for(a.g.Vh, block)), 1.0);
  return cudaGetLastError();
}

template <typename R, bool FIELD>
inline void su2c_launch_or_meas(const Ctx& a, int parity, int mu, int block, cudaStream_t st) {
  const unsigned grid = grid_for(a.g.Vh, block);
  switch (mu) {
    case 1: su2c_or_meas_kernel<R, FIELD, 1><<<grid, block, 0, st>>>(a, parity); break;
    case 2: su2c_or_meas_kernel<R, FIELD, 2><<<grid, block, 0, st>>>(a, parity); break;
    default: su2c_or_meas_kernel<R, FIELD, 3><<<grid, block, 0, st>>>(a, parity); break;
  }
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
  } else if (kind == KIND_OR_MEAS && mu >= 1) {
    if (field) su2c_launch_or_meas<R, true>(a, parity, mu, block, st);
    else su2c_launch_or_meas<R, false>(a, parity, mu, block, st);
  } else {
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
  cudaFuncAttributes f0{}, f1{};
  const int meas = cudaFuncGetAttributes(&f0, su2c_or_meas_kernel<R, false, 3>) == cudaSuccess &&
                           cudaFuncGetAttributes(&f1, su2c_or_meas_kernel<R, true, 1>) == cudaSuccess
                       ? std::min(f0.maxThreadsPerBlock, f1.maxThreadsPerBlock)
                       : 0;
  return std::min(std::min(m, meas),
                  std::min(su2c_limit_mu<R, false, KIND_OR_REUNIT>(), su2c_limit_mu<R, true, KIND_OR_REUNIT>()));
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
                   &su2c_measure_fused_tail<R>,
                   &su2c_max_phase_block<R>};
}

}  // namespace qcd
