/*
 * qcd_oracle.h -- FP64 CPU oracle for the checkerboard Monte Carlo sweep of
 * pure SU(2)/SU(3) Wilson lattice gauge theory at finite temperature in a
 * constant Abelian chromomagnetic background field.
 *
 * TEST INFRASTRUCTURE.  This is the slow, plain reference that the CUDA
 * library is checked against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no source with the
 * CUDA library and never calls it.  See qcd_oracle.c for what each routine
 * follows and for the pins that tie it to the mathematics.
 *
 * Conventions (shared with the CUDA library only through this written
 * definition, never through code):
 *   - directions mu = 0,1,2,3 are x,y,z,t; extents Ns (x,y,z) and Nt (t);
 *   - site s = x + Ns*(y + Ns*(z + Ns*t)), x fastest; parity (x+y+z+t) mod 2;
 *   - canonical link array: [s][mu][row][col][re,im], FP64, N*N complex
 *     entries per link;
 *   - U_mu(x) is the stored ("bare") link; the action and all updates use the
 *     effective link  Ut_mu(x) = U_mu(x) B_mu(x),  B = 1 except on y-links,
 *     B_y(x) = diag(e^{i phi}, e^{-i phi} [, 1]),  phi = 2 pi n x / Ns^2.
 */
#ifndef QCD_ORACLE_H
#define QCD_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct oracle_lattice oracle_lattice;

enum { ORACLE_HEATBATH = 0, ORACLE_OVERRELAX = 1 };
/* Where the background field lives: as a phase on every dynamical y-link
 * (effective links U B), or on the frozen spatial links of the t = 0 slice. */
enum { ORACLE_FIELD_LINKS = 0, ORACLE_FIELD_FROZEN = 1 };

/* Philox-4x32-10 block function (Salmon et al., SC11).  ctr[4], key[2] in,
 * out[4] out. */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                          uint32_t out[4]);
/* 32-bit word -> uniform in (0,1):  ((w >> 9) + 1/2) * 2^-23.  Every value is
 * exactly representable in FP32 and FP64. */
double oracle_uniform(uint32_t w);

/* Lattice life cycle.  N = 2 or 3; Ns, Nt even and >= 2; nhit >= 1 is the cap
 * on Kennedy-Pendleton tries per (link, subgroup).  NULL on bad arguments or
 * allocation failure. */
oracle_lattice *oracle_create(int N, int Ns, int Nt, double beta, int flux,
                              int nhit, uint32_t lattice_id);
/* flux8: flux quanta of the lambda8 component (SU(3) only; 0 for SU(2)). */
oracle_lattice *oracle_create_ex(int N, int Ns, int Nt, double beta, int flux,
                                 int flux8, int nhit, uint32_t lattice_id,
                                 int field_mode);
void oracle_destroy(oracle_lattice *L);
void oracle_set_threads(int n);
int oracle_get_threads(void);

void oracle_cold_start(oracle_lattice *L);
void oracle_hot_start(oracle_lattice *L, uint64_t seed);

/* n_hb times: one heat-bath pass, n_or overrelaxation passes, one
 * reunitarization; the sweep counter advances after each. */
void oracle_sweep(oracle_lattice *L, int n_hb, int n_or, uint64_t seed);
/* One checkerboard phase (all links of direction mu on sites of one parity). */
void oracle_phase(oracle_lattice *L, int kind, int parity, int mu,
                  uint64_t seed);
void oracle_reunitarize(oracle_lattice *L);
/* Reunitarize only the links of phase (parity, mu), as a sweep's last
 * overrelaxation pass does to each link right after updating it. */
void oracle_reunitarize_phase(oracle_lattice *L, int parity, int mu);
/* Reunitarize one N x N matrix in place ([row][col][re,im], FP64). */
void oracle_reunitarize_matrix(int N, double *m);

/* plaq[3] = {P, P_s, P_t} on effective links; poly[2] = {Re L, Im L}. */
void oracle_measure(const oracle_lattice *L, double plaq[3], double poly[2]);
/* Mean (1/N) Re Tr plaquette of each plane on effective links, planes in
 * the order (x,y), (x,z), (y,z), (x,t), (y,t), (z,t). */
void oracle_measure_planes(const oracle_lattice *L, double planes[6]);
/* plaq[3] = {P, P_s, P_t} on bare links. */
void oracle_measure_bare(const oracle_lattice *L, double plaq[3]);

void oracle_get_links(const oracle_lattice *L, double *out);
void oracle_set_links(oracle_lattice *L, const double *in);
uint32_t oracle_get_sweep(const oracle_lattice *L);
void oracle_set_sweep(oracle_lattice *L, uint32_t sweep);
long oracle_exhausted(const oracle_lattice *L);

/* Single-link helpers for pins and sampled parity (no state change). */
void oracle_staple(const oracle_lattice *L, long s, int mu, double *out);
double oracle_link_action(const oracle_lattice *L, long s, int mu);
int oracle_link_update(const oracle_lattice *L, int kind, long s, int mu,
                       uint64_t seed, double *out);

/* Distribution helpers: n independent draws, draw i using counter words
 * (i, 0, 0, try) under key (seed_lo, seed_hi). */
void oracle_kp_samples(double alpha, int nhit, uint64_t seed, long n,
                       double *a0, int *tries);
void oracle_su2_samples(double alpha, int nhit, uint64_t seed, long n,
                        double *x4);
void oracle_haar_samples(int N, uint64_t seed, long n, double *out);

#ifdef __cplusplus
}
#endif
#endif
