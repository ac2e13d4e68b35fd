/*
 * on_oracle.c -- plain FP64 CPU oracle for the O(N) model sweep by multi-hit
 * Metropolis (TEST INFRASTRUCTURE; see on_oracle.h for the conventions).
 *
 * What it follows.  The paper simulates O(N) models next to SU(N)
 * gluodynamics (sec. 3.3, "SUNCL and ONCL Modules"): the field is an N-vector
 * on every lattice site, the sites are updated on the even/odd checkerboard,
 * and the update is an improved Metropolis algorithm; its benchmarks run
 * O(4) with NHIT = 100 tries per site (sec. 4, Table 1).  The paper prints no
 * action and no update formula, so this file implements these readings:
 *   R18  the lattice O(N) phi^4 action
 *          S = sum_x [ -2 kappa sum_mu phi_x.phi_{x+mu} + phi_x.phi_x
 *                      + lambda (phi_x.phi_x - 1)^2 ];
 *   R19  "improved" Metropolis = multi-hit: a visit makes NHIT successive
 *        Metropolis hits on the site with its neighbours fixed; hit h
 *        proposes phi' = phi + delta (2u - 1) componentwise and accepts with
 *        probability min(1, exp(-dS)), dS the change of the local action;
 *   R20  random numbers: Philox-4x32-10 as for the gauge sweep, proposal
 *        block (s, sweep, 3 << 4, h), acceptance uniform = word h mod 4 of
 *        block (s, sweep, 4 << 4, h / 4).
 * Pins (tests/test_oracle_on.py): the local action difference equals the
 * total action difference of a one-site change (brute force); lambda = 0 is
 * the free field, <phi.phi> = N G(0) with the lattice propagator; kappa = 0
 * decouples the sites, <phi.phi> is a ratio of one-dimensional integrals;
 * many hits on one site with fixed neighbours sample exp(-s(phi)).
 */
#include "on_oracle.h"
#include "qcd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

struct on_lattice {
    int N, Ns, Nt, nhit;
    long V;
    double kappa, lambda, delta;
    uint32_t lattice_id, sweep;
    long long accepted;
    double *phi; /* [s][c], c < N */
};

enum { KIND_START = 2, KIND_PROPOSE = 3, KIND_ACCEPT = 4 };

on_lattice *on_create(int N, int Ns, int Nt, double kappa, double lambda,
                      double delta, int nhit, uint32_t lattice_id)
{
    if (N < 1 || N > 4 || Ns < 2 || Nt < 2 || (Ns & 1) || (Nt & 1) ||
        nhit < 1 || !(delta > 0.0))
        return NULL;
    on_lattice *L = calloc(1, sizeof *L);
    if (!L) return NULL;
    L->N = N; L->Ns = Ns; L->Nt = Nt; L->nhit = nhit;
    L->V = (long)Ns * Ns * Ns * Nt;
    L->kappa = kappa; L->lambda = lambda; L->delta = delta;
    L->lattice_id = lattice_id;
    L->phi = calloc((size_t)L->V * N, sizeof(double));
    if (!L->phi) { free(L); return NULL; }
    on_cold_start(L);
    return L;
}

void on_destroy(on_lattice *L)
{
    if (!L) return;
    free(L->phi);
    free(L);
}

static void coords(const on_lattice *L, long s, int c[4])
{
    c[0] = (int)(s % L->Ns); s /= L->Ns;
    c[1] = (int)(s % L->Ns); s /= L->Ns;
    c[2] = (int)(s % L->Ns);
    c[3] = (int)(s / L->Ns);
}

static long index_of(const on_lattice *L, const int c[4])
{
    return c[0] + (long)L->Ns * (c[1] + (long)L->Ns * (c[2] + (long)L->Ns * c[3]));
}

/* neighbour of s one step along mu in direction d = +1 / -1 (periodic) */
static long neighbour(const on_lattice *L, long s, int mu, int d)
{
    int c[4];
    coords(L, s, c);
    int ext = mu == 3 ? L->Nt : L->Ns;
    c[mu] = (c[mu] + d + ext) % ext;
    return index_of(L, c);
}

static void block(const on_lattice *L, uint64_t seed, uint32_t c0, uint32_t c1,
                  uint32_t c2, uint32_t c3, uint32_t out[4])
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed ^ (L->lattice_id * 0x9E3779B9u),
                       (uint32_t)(seed >> 32)};
    oracle_philox4x32_10(ctr, key, out);
}

void on_cold_start(on_lattice *L)
{
    memset(L->phi, 0, sizeof(double) * (size_t)L->V * L->N);
    for (long s = 0; s < L->V; ++s) L->phi[s * L->N] = 1.0;
    L->sweep = 0;
}

void on_hot_start(on_lattice *L, uint64_t seed)
{
    for (long s = 0; s < L->V; ++s) {
        uint32_t w[4];
        block(L, seed, (uint32_t)s, 0xFFFFFFFFu, KIND_START << 4, 0, w);
        for (int c = 0; c < L->N; ++c)
            L->phi[s * L->N + c] = 2.0 * oracle_uniform(w[c]) - 1.0;
    }
    L->sweep = 0;
}

/* F = sum over the 8 neighbours of their field values */
static void neighbour_sum(const on_lattice *L, long s, double F[4])
{
    for (int c = 0; c < 4; ++c) F[c] = 0.0;
    for (int mu = 0; mu < 4; ++mu)
        for (int d = -1; d <= 1; d += 2) {
            long n = neighbour(L, s, mu, d);
            for (int c = 0; c < L->N; ++c) F[c] += L->phi[n * L->N + c];
        }
}

/* s(phi) = -2 kappa phi.F + phi.phi + lambda (phi.phi - 1)^2 */
static double local_action_F(const on_lattice *L, const double *phi, const double F[4])
{
    double pf = 0.0, pp = 0.0;
    for (int c = 0; c < L->N; ++c) {
        pf += phi[c] * F[c];
        pp += phi[c] * phi[c];
    }
    return -2.0 * L->kappa * pf + pp + L->lambda * (pp - 1.0) * (pp - 1.0);
}

double on_local_action(const on_lattice *L, long s, const double *phi)
{
    double F[4];
    neighbour_sum(L, s, F);
    return local_action_F(L, phi, F);
}

double on_action(const on_lattice *L)
{
    double S = 0.0;
    for (long s = 0; s < L->V; ++s) {
        const double *p = L->phi + s * L->N;
        double pp = 0.0, hop = 0.0;
        for (int c = 0; c < L->N; ++c) pp += p[c] * p[c];
        for (int mu = 0; mu < 4; ++mu) {
            const double *q = L->phi + neighbour(L, s, mu, +1) * L->N;
            for (int c = 0; c < L->N; ++c) hop += p[c] * q[c];
        }
        S += -2.0 * L->kappa * hop + pp + L->lambda * (pp - 1.0) * (pp - 1.0);
    }
    return S;
}

/* All nhit hits of one visit of site s, starting from phi[0..N-1] (updated in
 * place); neighbours are read from the field.  Returns the accepted hits. */
static int visit(const on_lattice *L, long s, uint64_t seed, double *phi)
{
    double F[4];
    neighbour_sum(L, s, F);
    double cur = local_action_F(L, phi, F);
    uint32_t acc[4] = {0, 0, 0, 0};
    int accepted = 0;
    for (int h = 0; h < L->nhit; ++h) {
        uint32_t w[4];
        block(L, seed, (uint32_t)s, L->sweep, KIND_PROPOSE << 4, (uint32_t)h, w);
        if ((h & 3) == 0)
            block(L, seed, (uint32_t)s, L->sweep, KIND_ACCEPT << 4, (uint32_t)(h >> 2), acc);
        double trial[4] = {0.0, 0.0, 0.0, 0.0};
        for (int c = 0; c < L->N; ++c)
            trial[c] = phi[c] + L->delta * (2.0 * oracle_uniform(w[c]) - 1.0);
        double next = local_action_F(L, trial, F);
        double dS = next - cur;
        if (dS <= 0.0 || oracle_uniform(acc[h & 3]) < exp(-dS)) {
            for (int c = 0; c < L->N; ++c) phi[c] = trial[c];
            cur = next;
            ++accepted;
        }
    }
    return accepted;
}

int on_site_update(const on_lattice *L, long s, uint64_t seed, double out[4])
{
    double phi[4] = {0.0, 0.0, 0.0, 0.0};
    for (int c = 0; c < L->N; ++c) phi[c] = L->phi[s * L->N + c];
    int a = visit(L, s, seed, phi);
    for (int c = 0; c < 4; ++c) out[c] = phi[c];
    return a;
}

void on_phase(on_lattice *L, int parity, uint64_t seed)
{
    long long acc = 0;
    /* sites of one parity are independent: their neighbours all have the
     * other parity, so the order of the visits does not matter */
#pragma omp parallel for schedule(static) reduction(+ : acc)
    for (long s = 0; s < L->V; ++s) {
        int c[4];
        coords(L, s, c);
        if (((c[0] + c[1] + c[2] + c[3]) & 1) != parity) continue;
        double phi[4] = {0.0, 0.0, 0.0, 0.0};
        for (int k = 0; k < L->N; ++k) phi[k] = L->phi[s * L->N + k];
        acc += visit(L, s, seed, phi);
        for (int k = 0; k < L->N; ++k) L->phi[s * L->N + k] = phi[k];
    }
    L->accepted += acc;
}

void on_sweep(on_lattice *L, int n, uint64_t seed)
{
    for (int i = 0; i < n; ++i) {
        on_phase(L, 0, seed);
        on_phase(L, 1, seed);
        L->sweep += 1;
    }
}

void on_measure(const on_lattice *L, double out[7])
{
    double pp = 0.0, hop = 0.0, M[4] = {0.0, 0.0, 0.0, 0.0};
    for (long s = 0; s < L->V; ++s) {
        const double *p = L->phi + s * L->N;
        for (int c = 0; c < L->N; ++c) {
            pp += p[c] * p[c];
            M[c] += p[c];
        }
        for (int mu = 0; mu < 4; ++mu) {
            const double *q = L->phi + neighbour(L, s, mu, +1) * L->N;
            for (int c = 0; c < L->N; ++c) hop += p[c] * q[c];
        }
    }
    double V = (double)L->V, m2 = 0.0;
    out[0] = pp / V;
    out[1] = hop / (4.0 * V);
    for (int c = 0; c < 4; ++c) {
        out[3 + c] = M[c] / V;
        m2 += out[3 + c] * out[3 + c];
    }
    out[2] = sqrt(m2);
}

void on_get_field(const on_lattice *L, double *out)
{
    memcpy(out, L->phi, sizeof(double) * (size_t)L->V * L->N);
}

void on_set_field(on_lattice *L, const double *in)
{
    memcpy(L->phi, in, sizeof(double) * (size_t)L->V * L->N);
}

uint32_t on_get_sweep(const on_lattice *L) { return L->sweep; }
void on_set_sweep(on_lattice *L, uint32_t sweep) { L->sweep = sweep; }
long long on_accepted(const on_lattice *L) { return L->accepted; }
