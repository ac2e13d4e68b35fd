// qcd_internal.h -- interface between the host library (qcd_api.cu) and the
// per-storage kernel translation units.  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace qcd {

struct GeomH {
  int Ns, Nt;
  int Vh;
  int pow2;  // log2(Ns) | log2(Nt) << 8 | 1 << 16 when Ns and Nt are powers of two
             // (site decoding by shifts and masks); otherwise the shifts of
             // the divisions by Ns and Nt below in bits 17-21 and 22-26
  int64_t plane;
  // Division of 0 <= n < 2^31 by Ns (Nt) as a multiply-high and a shift:
  // n / d = umulhi(n, m) >> s with l = ceil(log2 d), s = l - 1 and
  // m = ceil(2^(31 + l) / d) < 2^32.  Exact: n m / 2^(31 + l) exceeds n / d
  // by less than n / 2^(31 + l) < 2^-l <= 1 / d, and the fraction of n / d is
  // at most 1 - 1 / d.  0: decode by division.
  uint32_t mNs, mNt;
};

constexpr int GEOM_POW2 = 1 << 16;

inline void geom_div_magic(uint32_t d, uint32_t* m, int* s) {
  int l = 0;
  while ((1u << l) < d) ++l;
  *m = uint32_t(((uint64_t(1) << (31 + l)) + d - 1) / d);
  *s = l - 1;
}

// Site-decoding fields of g for Ns, Nt >= 2: the power-of-two code, or the
// multiply-high divisions.
inline void geom_set_decode(GeomH& g) {
  auto lg = [](int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return (1 << l) == n ? l : -1;
  };
  const int ls = lg(g.Ns), lt = lg(g.Nt);
  g.mNs = g.mNt = 0;
  if (ls >= 0 && lt >= 0) {
    g.pow2 = ls | (lt << 8) | GEOM_POW2;
    return;
  }
  int sN = 0, sT = 0;
  geom_div_magic(uint32_t(g.Ns), &g.mNs, &sN);
  geom_div_magic(uint32_t(g.Nt), &g.mNt, &sT);
  g.pow2 = (sN << 17) | (sT << 22);
}

// Everything a kernel launch needs for one lattice.  Device pointers only.
struct Ctx {
  void* links;
  GeomH g;
  double beta;
  uint32_t k0, k1;              // Philox key of this call
  const uint32_t* sweep;        // device sweep counter (Philox counter word 1)
  uint32_t* sweep_rw;           // same counter, for the end-of-sweep advance
  int nhit;
  int flux;                     // 0: no background field
  int field_mode;               // 0: phase on every y-link (effective links U B);
                                // 1: field on the frozen spatial links of t = 0
  int flux8;                    // lambda8 flux quanta (SU(3)); 0: lambda3 only
  // Background tables, 4 Ns entries each: [x] = (cos phi, sin phi) with
  // phi = 2 pi n x / Ns^2, then [Ns + 3x + k] = e^{i theta_k(x)}, the diagonal
  // of the SU(3) y-link background diag(e^{i(p3+p8)}, e^{i(-p3+p8)}, e^{-2i p8}).
  // (The argument struct is kept at 120 bytes: growing it past 128 bytes
  // measurably slowed every kernel that takes it.)
  const double2* phase64;
  const float2* phase32;
  unsigned long long* exhausted;
  double* partials;             // measurement scratch, measure_partials() doubles
  double* meas_out;             // 5 doubles: P, P_s, P_t, Re L, Im L
};

static_assert(sizeof(Ctx) <= 128, "kernel argument struct grew past 128 bytes");

constexpr int MEAS_THREADS = 256;
constexpr int FINAL_THREADS = 1024;

inline int meas_plaq_blocks(const GeomH& g) { return int((2LL * g.Vh + MEAS_THREADS - 1) / MEAS_THREADS); }
__host__ __device__ inline int meas_poly_blocks(const GeomH& g) {
  return int(((long long)g.Ns * g.Ns * g.Ns + MEAS_THREADS - 1) / MEAS_THREADS);
}
inline size_t measure_partials(const GeomH& g) { return 2 * size_t(meas_plaq_blocks(g) + meas_poly_blocks(g)); }
// Measurement fused into a working sweep: the Polyakov-loop partials first,
// then one stretch per plane-summing phase (mu = 1, 2, 3) of one double per
// block of the phase kernel (blocks of at least 32 threads).
__host__ __device__ inline int fused_stride(const GeomH& g) { return (g.Vh + 31) / 32; }
__host__ __device__ inline int fused_plaq_offset(const GeomH& g, int mu) {
  return 2 * meas_poly_blocks(g) + (mu - 1) * fused_stride(g);
}
inline size_t fused_partials(const GeomH& g) { return size_t(fused_plaq_offset(g, 4)); }

// Phase kinds: heat-bath, overrelaxation, and overrelaxation whose kernel also
// reunitarizes each link it updates before storing it (the last pass of a
// sweep carries the reunitarization this way, with no pass of its own).
// KIND_OR_MEAS: as KIND_OR_REUNIT, and for phase (odd parity, mu >= 1) also
// sums the plaquettes of the planes (mu, nu < mu) through the updated links:
// after the last pass each plaquette of plane (mu, nu) has exactly one odd
// mu-link, so these three phases see every plaquette once.
enum { KIND_HB = 0, KIND_OR = 1, KIND_OR_REUNIT = 2, KIND_OR_MEAS = 3 };

// One table per (group, storage).
struct PolicyOps {
  int group;
  int precision;   // 0 = FP64 plain, 1 = FP32 compressed
  int comps;       // 16-byte vectors per link
  cudaError_t (*phase)(const Ctx&, int kind, int parity, int mu, int block, cudaStream_t);
  cudaError_t (*reunit)(const Ctx&, int advance_sweep, cudaStream_t);
  cudaError_t (*start)(const Ctx&, int hot, cudaStream_t);
  cudaError_t (*measure)(const Ctx&, int effective, cudaStream_t);
  cudaError_t (*to_canonical)(const Ctx&, double* dev_out, cudaStream_t);
  cudaError_t (*from_canonical)(const Ctx&, const double* dev_in, cudaStream_t);
  // Frozen-boundary mode: set the spatial links of the t = 0 slice to B.
  cudaError_t (*set_frozen)(const Ctx&, cudaStream_t);
  // Tail of a working sweep whose last pass ran KIND_OR_MEAS phases with
  // `block` threads: Polyakov loop and the final sums into meas_out.  Null when
  // the storage has no fused measurement.
  cudaError_t (*measure_fused_tail)(const Ctx&, int block, cudaStream_t);
  // Largest block the phase kernels of this storage can launch with (the
  // minimum over heat-bath / overrelaxation, with and without the field).
  int (*max_phase_block)();
};

// Effective-link phases are applied only in field mode 0 with a field.
inline bool phases_on_links(const Ctx& a) { return (a.flux != 0 || a.flux8 != 0) && a.field_mode == 0; }
// Which background multiply the SU(3) FP32 phase kernel instantiates:
// 0 none, 1 lambda3 only (columns 0, 1), 2 general diagonal (all columns).
inline int su3_field_level(const Ctx& a) { return !phases_on_links(a) ? 0 : (a.flux8 != 0 ? 2 : 1); }

// Record the message returned by qcd_last_error() on this thread; returns code.
int set_last_error(int code, const char* msg);

extern const PolicyOps kOpsSU2F64;
extern const PolicyOps kOpsSU2F32;
extern const PolicyOps kOpsSU3F64;
extern const PolicyOps kOpsSU3F32;

}  // namespace qcd
