/*
 * on_oracle.h -- FP64 CPU oracle for the checkerboard Monte Carlo sweep of the
 * lattice O(N) model (N-component real scalar field on the sites, lambda
 * phi^4 self-interaction) by multi-hit ("improved") Metropolis.
 *
 * TEST INFRASTRUCTURE, like qcd_oracle.h: only the test suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load it; it shares no source
 * with the CUDA library.
 *
 * Conventions (the CUDA library follows the same written definition):
 *   - site s = x + Ns*(y + Ns*(z + Ns*t)), parity (x+y+z+t) mod 2;
 *   - canonical field array [s][c], c = 0..N-1, FP64;
 *   - action S = sum_x [ -2 kappa sum_mu phi_x . phi_{x+mu} + phi_x . phi_x
 *                        + lambda (phi_x . phi_x - 1)^2 ];
 *   - a visit of site x makes nhit Metropolis hits; hit h proposes
 *     phi'_c = phi_c + delta (2 u_c - 1), u_c = uniform(word c) of the Philox
 *     block (s, sweep, 3 << 4, h), and accepts iff dS <= 0 or
 *     u < exp(-dS), u = uniform(word h mod 4) of block (s, sweep, 4 << 4,
 *     h / 4); key = (seed_lo ^ lattice_id * 0x9E3779B9, seed_hi);
 *   - a sweep updates the even sites, then the odd ones; the sweep counter
 *     advances once per sweep;
 *   - hot start: phi_c = 2 u_c - 1 from block (s, 0xFFFFFFFF, 2 << 4, 0);
 *     cold start: phi = (1, 0, ..., 0).
 */
#ifndef ON_ORACLE_H
#define ON_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct on_lattice on_lattice;

/* N in 1..4; Ns, Nt even and >= 2; nhit >= 1; delta > 0.  NULL on bad
 * arguments.  The field starts cold. */
on_lattice *on_create(int N, int Ns, int Nt, double kappa, double lambda,
                      double delta, int nhit, uint32_t lattice_id);
void on_destroy(on_lattice *L);

void on_cold_start(on_lattice *L);
void on_hot_start(on_lattice *L, uint64_t seed);

/* One checkerboard phase (all sites of one parity) at the current sweep
 * counter; the counter does not move. */
void on_phase(on_lattice *L, int parity, uint64_t seed);
/* n sweeps: even phase, odd phase, counter + 1. */
void on_sweep(on_lattice *L, int n, uint64_t seed);

/* The value site s would take in this sweep's visit (all nhit hits), given the
 * current field; the field is not changed.  Returns the accepted hits. */
int on_site_update(const on_lattice *L, long s, uint64_t seed, double out[4]);

/* Local action of value phi[0..N-1] at site s in the field of its neighbours:
 * -2 kappa phi . F + phi . phi + lambda (phi . phi - 1)^2,
 * F = sum_mu (phi_{x+mu} + phi_{x-mu}). */
double on_local_action(const on_lattice *L, long s, const double *phi);
/* Total action S. */
double on_action(const on_lattice *L);

/* out[7] = { <phi.phi>, (1/4V) sum_{x,mu} phi_x . phi_{x+mu}, |M|,
 *            M_0, M_1, M_2, M_3 },  M = (1/V) sum_x phi_x (M_c = 0, c >= N). */
void on_measure(const on_lattice *L, double out[7]);

void on_get_field(const on_lattice *L, double *out); /* V*N doubles */
void on_set_field(on_lattice *L, const double *in);
uint32_t on_get_sweep(const on_lattice *L);
void on_set_sweep(on_lattice *L, uint32_t sweep);
/* Accepted Metropolis hits since creation. */
long long on_accepted(const on_lattice *L);

#ifdef __cplusplus
}
#endif
#endif
