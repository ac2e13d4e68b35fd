/*
 * qcd_oracle.c -- FP64 CPU oracle for the checkerboard Monte Carlo sweep of
 * pure SU(2)/SU(3) Wilson lattice gauge theory at finite temperature in a
 * constant Abelian chromomagnetic background field.
 *
 * TEST INFRASTRUCTURE.  This is the plain, slow, obviously-correct reference
 * that the CUDA library is checked against.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * source with the CUDA library (its own Philox, its own matrix code, full
 * N x N complex matrices in FP64, no compression, no even/odd layout) and it
 * never calls the library.
 *
 * What it follows.  The paper (QCDGPU, Demchik & Kolomoyets) names the method
 * but prints no formula for it: SU(N) gluodynamics in an external field at
 * finite temperature (abstract, sec. 1); links are N x N complex matrices
 * updated by (pseudo)heat-bath on an even/odd checkerboard (sec. 3.3); runs use
 * a hot start, NHIT = 10 and reunitarization (sec. 5); plaquette and Polyakov
 * loop are the measured quantities (sec. 1, sec. 5).  The steps the paper
 * leaves out are the textbook ones, each named where it is used:
 *   Wilson action         S = beta sum_P (1 - Re Tr U_P / N)   (Wilson 1974)
 *   SU(2) heat-bath       Kennedy & Pendleton, Phys. Lett. B156 (1985) 393
 *   SU(3) heat-bath       Cabibbo & Marinari, Phys. Lett. B119 (1982) 387
 *   overrelaxation        Creutz, Phys. Rev. D36 (1987) 515
 *   random numbers        Philox-4x32-10, Salmon et al., SC11 (2011)
 *   Haar SU(2)            uniform unit quaternions, Shoemake (Graphics Gems III)
 *   Haar SU(3)            Gram-Schmidt of complex Gaussians, Mezzadri,
 *                         Notices AMS 54 (2007) 592, then det^(-1/3)
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes):
 *   R1 action normalisation as above, so the SU(2) single-link weight is
 *      exp(beta k a0) and an SU(3) subgroup weight is exp((2 beta/3) k a0);
 *   R2 phase order: parity even then odd, inside it mu = x, y, z, t;
 *   R3 NHIT caps the Kennedy-Pendleton tries per (link, subgroup); when all
 *      fail the SU(2) link is kept, the SU(3) subgroup step is skipped;
 *   R4 when alpha = beta k = 0 the heat-bath draw is Haar and replaces the
 *      link (SU(2)) or is the subgroup rotation (SU(3));
 *   R5 external field: U(1) phase along lambda3 (sigma3 for SU(2)) on y-links,
 *      phi(x) = 2 pi n x / Ns^2, applied on the right, Ut = U B; updates act on
 *      Ut and store U = Ut_new B^dagger (effective-link mode; a change of
 *      variables, so effective-link observables do not depend on n);
 *   R10 lambda8 component (SU(3) only): with the generator sqrt(3) lambda8 =
 *      diag(1, 1, -2), B_y(x) = diag(e^{i(p3 + p8)}, e^{i(-p3 + p8)},
 *      e^{-2 i p8}), p3 = 2 pi n x / Ns^2, p8 = 2 pi n8 x / Ns^2, so every
 *      diagonal phase is an integer multiple of 2 pi x / Ns^2;
 *   R9 frozen-boundary mode (the field imposed through fixed links, as in the
 *      background-field studies the paper cites): the spatial links of the
 *      time slice t = 0 hold B and are never updated or reunitarized, the
 *      other links carry no phase;
 *   R6 Polyakov loop: (1/N) Tr of the product t = 0 .. Nt-1, averaged over the
 *      Ns^3 spatial sites;
 *   R7 reunitarization after each heat-bath pass's overrelaxation block;
 *   R8 random-number keys: key = (seed_lo ^ lattice_id * 0x9E3779B9, seed_hi),
 *      counter = (site, sweep, mu | subgroup << 2 | kind << 4, block); kind 0 =
 *      Kennedy-Pendleton try, 1 = direction / Haar, 2 = start (sweep word
 *      0xFFFFFFFF); uniforms ((w >> 9) + 1/2) 2^-23.
 *
 * Pins (tests/test_oracle_*.py): Philox known-answer vectors; uniform grid;
 * Kennedy-Pendleton chi-square against sqrt(1-a0^2) e^(alpha a0); direction
 * isotropy; Haar moments (E|Tr U|^2 = 1, E (Tr U)^3 = 1 for SU(3)); cold-start
 * and background-field closed forms; staple / plaquette sum rule;
 * overrelaxation action conservation; unitarity and det = 1; beta = 0; strong
 * coupling (character expansion / Weyl integral); weak coupling; the
 * change-of-variables identity of the background field.
 */
#include "qcd_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define MAXN 3
typedef double complex cplx;
typedef struct { cplx e[MAXN][MAXN]; } mat;

struct oracle_lattice {
    int N, Ns, Nt;
    long V;
    double beta;
    int flux, flux8;
    int field_mode;     /* ORACLE_FIELD_LINKS or ORACLE_FIELD_FROZEN */
    int nhit;
    uint32_t lattice_id;
    uint32_t sweep;     /* heat-bath passes since the start */
    long exhausted;     /* (link, subgroup) draws that used up NHIT tries */
    cplx *U;            /* [V][4][N][N] */
};

/* ------------------------------------------------------------------------ */
/* Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC11).  Ten rounds of two     */
/* 32x32->64 multiplies; the key is bumped by the Weyl constants between     */
/* rounds.                                                                   */
/* ------------------------------------------------------------------------ */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                          uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

double oracle_uniform(uint32_t w)
{
    return ((double)(w >> 9) + 0.5) * 0x1p-23;
}

/* A random stream: fixed key and first three counter words; the fourth
 * counter word is the block index. */
typedef struct { uint32_t key[2]; uint32_t c0, c1, c2; } stream;

static void stream_uniforms(const stream *st, uint32_t block, double u[4])
{
    uint32_t ctr[4] = { st->c0, st->c1, st->c2, block }, w[4];
    oracle_philox4x32_10(ctr, st->key, w);
    for (int i = 0; i < 4; ++i) u[i] = oracle_uniform(w[i]);
}

enum { KIND_TRY = 0, KIND_DIR = 1, KIND_START = 2 };
#define START_SWEEP_WORD 0xFFFFFFFFu

static stream lattice_stream(const oracle_lattice *L, uint64_t seed,
                             uint32_t sweep, long s, int mu, int sub, int kind)
{
    stream st;
    st.key[0] = (uint32_t)seed ^ (L->lattice_id * 0x9E3779B9u);
    st.key[1] = (uint32_t)(seed >> 32);
    st.c0 = (uint32_t)s;
    st.c1 = sweep;
    st.c2 = (uint32_t)(mu | (sub << 2) | (kind << 4));
    return st;
}

static stream plain_stream(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2)
{
    stream st;
    st.key[0] = (uint32_t)seed;
    st.key[1] = (uint32_t)(seed >> 32);
    st.c0 = c0; st.c1 = c1; st.c2 = c2;
    return st;
}

/* ------------------------------------------------------------------------ */
/* N x N complex matrices                                                    */
/* ------------------------------------------------------------------------ */
static mat mat_zero(void)
{
    mat m;
    memset(&m, 0, sizeof m);
    return m;
}

static mat mat_identity(int N)
{
    mat m = mat_zero();
    for (int i = 0; i < N; ++i) m.e[i][i] = 1.0;
    return m;
}

static mat mat_mul(int N, const mat *a, const mat *b)
{
    mat c = mat_zero();
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            cplx acc = 0.0;
            for (int k = 0; k < N; ++k) acc += a->e[i][k] * b->e[k][j];
            c.e[i][j] = acc;
        }
    return c;
}

static mat mat_dag(int N, const mat *a)
{
    mat c = mat_zero();
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) c.e[i][j] = conj(a->e[j][i]);
    return c;
}

static mat mat_mul3(int N, const mat *a, const mat *b, const mat *c)
{
    mat ab = mat_mul(N, a, b);
    return mat_mul(N, &ab, c);
}

static void mat_add_to(int N, mat *acc, const mat *a)
{
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) acc->e[i][j] += a->e[i][j];
}

static cplx mat_trace(int N, const mat *a)
{
    cplx t = 0.0;
    for (int i = 0; i < N; ++i) t += a->e[i][i];
    return t;
}

static cplx mat_det(int N, const mat *a)
{
    if (N == 2) return a->e[0][0] * a->e[1][1] - a->e[0][1] * a->e[1][0];
    return a->e[0][0] * (a->e[1][1] * a->e[2][2] - a->e[1][2] * a->e[2][1])
         - a->e[0][1] * (a->e[1][0] * a->e[2][2] - a->e[1][2] * a->e[2][0])
         + a->e[0][2] * (a->e[1][0] * a->e[2][1] - a->e[1][1] * a->e[2][0]);
}

/* SU(2) element q0 + i (q1 sigma1 + q2 sigma2 + q3 sigma3) as a 2x2 matrix. */
static mat quat_to_mat(const double q[4])
{
    mat m = mat_zero();
    m.e[0][0] = q[0] + I * q[3];
    m.e[0][1] = q[2] + I * q[1];
    m.e[1][0] = -q[2] + I * q[1];
    m.e[1][1] = q[0] - I * q[3];
    return m;
}

/* Projection of the 2x2 block (rows/cols i, j) of w onto real multiples of
 * SU(2): the part that Re Tr(R w) sees for R in SU(2). */
static void block_to_quat(const mat *w, int i, int j, double q[4])
{
    cplx w11 = w->e[i][i], w12 = w->e[i][j], w21 = w->e[j][i], w22 = w->e[j][j];
    q[0] = 0.5 * creal(w11 + w22);
    q[1] = 0.5 * cimag(w12 + w21);
    q[2] = 0.5 * creal(w12 - w21);
    q[3] = 0.5 * cimag(w11 - w22);
}

/* The N x N identity with the 2x2 matrix r placed on rows/cols (i, j). */
static mat embed(int N, const mat *r, int i, int j)
{
    mat m = mat_identity(N);
    m.e[i][i] = r->e[0][0];
    m.e[i][j] = r->e[0][1];
    m.e[j][i] = r->e[1][0];
    m.e[j][j] = r->e[1][1];
    return m;
}

/* ------------------------------------------------------------------------ */
/* Geometry and links                                                        */
/* ------------------------------------------------------------------------ */
static void site_coords(const oracle_lattice *L, long s, int c[4])
{
    c[0] = (int)(s % L->Ns); s /= L->Ns;
    c[1] = (int)(s % L->Ns); s /= L->Ns;
    c[2] = (int)(s % L->Ns); s /= L->Ns;
    c[3] = (int)s;
}

static long site_index(const oracle_lattice *L, const int c[4])
{
    long Ns = L->Ns;
    return c[0] + Ns * (c[1] + Ns * (c[2] + Ns * (long)c[3]));
}

static long site_shift(const oracle_lattice *L, long s, int mu, int step)
{
    int c[4];
    site_coords(L, s, c);
    int ext = (mu == 3) ? L->Nt : L->Ns;
    c[mu] = ((c[mu] + step) % ext + ext) % ext;
    return site_index(L, c);
}

static int site_parity(const oracle_lattice *L, long s)
{
    int c[4];
    site_coords(L, s, c);
    return (c[0] + c[1] + c[2] + c[3]) & 1;
}

static cplx *link_ptr(const oracle_lattice *L, long s, int mu)
{
    return L->U + ((size_t)s * 4 + mu) * L->N * L->N;
}

static mat get_link(const oracle_lattice *L, long s, int mu)
{
    mat m = mat_zero();
    const cplx *p = link_ptr(L, s, mu);
    for (int i = 0; i < L->N; ++i)
        for (int j = 0; j < L->N; ++j) m.e[i][j] = p[i * L->N + j];
    return m;
}

static void put_link(oracle_lattice *L, long s, int mu, const mat *m)
{
    cplx *p = link_ptr(L, s, mu);
    for (int i = 0; i < L->N; ++i)
        for (int j = 0; j < L->N; ++j) p[i * L->N + j] = m->e[i][j];
}

/* Background field B_mu(x) (reading R5). */
static mat background(const oracle_lattice *L, long s, int mu)
{
    mat b = mat_identity(L->N);
    if (mu == 1 && (L->flux != 0 || L->flux8 != 0)) {
        int c[4];
        site_coords(L, s, c);
        double unit = 2.0 * M_PI * c[0] / ((double)L->Ns * L->Ns);
        double p3 = unit * L->flux, p8 = unit * L->flux8;
        b.e[0][0] = cexp(I * (p3 + p8));
        b.e[1][1] = cexp(I * (-p3 + p8));
        if (L->N == 3) b.e[2][2] = cexp(I * (-2.0 * p8));
    }
    return b;
}

/* The phase the dynamical link carries: B in the effective-link mode, unity
 * when the field lives on the frozen boundary links. */
static mat link_phase(const oracle_lattice *L, long s, int mu)
{
    if (L->field_mode == ORACLE_FIELD_FROZEN) return mat_identity(L->N);
    return background(L, s, mu);
}

/* Effective link Ut = U B (effective-link mode) or U (frozen mode). */
static mat eff_link(const oracle_lattice *L, long s, int mu)
{
    mat u = get_link(L, s, mu), b = link_phase(L, s, mu);
    return mat_mul(L->N, &u, &b);
}

/* Frozen-boundary mode: the spatial links of the time slice t = 0 hold the
 * background field B and are never updated. */
static int is_frozen(const oracle_lattice *L, long s, int mu)
{
    if (L->field_mode != ORACLE_FIELD_FROZEN || mu == 3) return 0;
    int c[4];
    site_coords(L, s, c);
    return c[3] == 0;
}

static void set_frozen_links(oracle_lattice *L)
{
    if (L->field_mode != ORACLE_FIELD_FROZEN) return;
    long V3 = (long)L->Ns * L->Ns * L->Ns;
    for (long s = 0; s < V3; ++s)
        for (int mu = 0; mu < 3; ++mu) {
            mat b = background(L, s, mu);
            put_link(L, s, mu, &b);
        }
}

/* Staple sum of U_mu(x) on effective links:
 *   A = sum_{nu != mu} [ Ut_nu(x+mu) Ut_mu(x+nu)^+ Ut_nu(x)^+
 *                      + Ut_nu(x+mu-nu)^+ Ut_mu(x-nu)^+ Ut_nu(x-nu) ]
 * so that Re Tr(Ut_mu(x) A) is the sum of the 2(d-1) plaquettes holding the
 * link. */
static mat staple(const oracle_lattice *L, long s, int mu)
{
    int N = L->N;
    mat a = mat_zero();
    long s_pmu = site_shift(L, s, mu, +1);
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        long s_pnu = site_shift(L, s, nu, +1);
        long s_mnu = site_shift(L, s, nu, -1);
        long s_pmu_mnu = site_shift(L, s_pmu, nu, -1);

        mat u1 = eff_link(L, s_pmu, nu);
        mat u2 = eff_link(L, s_pnu, mu), u2d = mat_dag(N, &u2);
        mat u3 = eff_link(L, s, nu), u3d = mat_dag(N, &u3);
        mat upper = mat_mul3(N, &u1, &u2d, &u3d);

        mat l1 = eff_link(L, s_pmu_mnu, nu), l1d = mat_dag(N, &l1);
        mat l2 = eff_link(L, s_mnu, mu), l2d = mat_dag(N, &l2);
        mat l3 = eff_link(L, s_mnu, nu);
        mat lower = mat_mul3(N, &l1d, &l2d, &l3);

        mat_add_to(N, &a, &upper);
        mat_add_to(N, &a, &lower);
    }
    return a;
}

/* ------------------------------------------------------------------------ */
/* Random SU(2) elements                                                     */
/* ------------------------------------------------------------------------ */

/* Kennedy-Pendleton draw of a0 = 1 - delta in [-1, 1] with density
 * proportional to sqrt(1 - a0^2) exp(alpha a0), alpha > 0.  Try t reads block
 * t of the stream as u1..u4; delta = (-ln u2 - ln u1 cos^2(2 pi u3)) / alpha is
 * a Gamma(3/2, 1/alpha) variate, accepted when u4^2 <= 1 - delta/2.  Returns
 * the number of tries used (delta in *delta), 0 if all nhit failed. */
static int kp_draw(double alpha, int nhit, const stream *st, double *delta)
{
    for (int t = 0; t < nhit; ++t) {
        double u[4];
        stream_uniforms(st, (uint32_t)t, u);
        double c = cos(2.0 * M_PI * u[2]);
        double d = (-log(u[1]) - log(u[0]) * c * c) / alpha;
        if (u[3] * u[3] <= 1.0 - 0.5 * d) {
            *delta = d;
            return t + 1;
        }
    }
    return 0;
}

/* Unit quaternion with real part a0 = 1 - delta and a direction uniform on
 * S^2, read from block 0 of the direction stream: cos(theta) = 2 u1 - 1,
 * phi = 2 pi u2.  The moduli are written without cancellation:
 * sqrt(1 - a0^2) = sqrt(delta (2 - delta)) and
 * sin(theta) = sqrt(1 - cos^2(theta)) = 2 sqrt(u1 (1 - u1)). */
static void su2_with_delta(double delta, const stream *dir, double x[4])
{
    double u[4];
    stream_uniforms(dir, 0, u);
    double ct = 2.0 * u[0] - 1.0;
    double st = 2.0 * sqrt(u[0] * (1.0 - u[0]));
    double ph = 2.0 * M_PI * u[1];
    double r = sqrt(delta * (2.0 - delta));
    x[0] = 1.0 - delta;
    x[1] = r * st * cos(ph);
    x[2] = r * st * sin(ph);
    x[3] = r * ct;
}

/* Haar-random unit quaternion (Shoemake) from one block of uniforms. */
static void su2_haar(const stream *st, uint32_t block, double x[4])
{
    double u[4];
    stream_uniforms(st, block, u);
    double r1 = sqrt(1.0 - u[0]), r2 = sqrt(u[0]);
    x[0] = r1 * sin(2.0 * M_PI * u[1]);
    x[1] = r1 * cos(2.0 * M_PI * u[1]);
    x[2] = r2 * sin(2.0 * M_PI * u[2]);
    x[3] = r2 * cos(2.0 * M_PI * u[2]);
}

/* Haar-random SU(3) (Mezzadri): 9 complex Gaussians from blocks 0..4 of the
 * stream by Box-Muller, z_k = sqrt(-2 ln u_{2k}) exp(2 pi i u_{2k+1}), laid out
 * row-major; Gram-Schmidt on the rows (this gives the positive-diagonal QR
 * factor, i.e. Mezzadri's phase fix); then multiply by det^(-1/3) on the
 * principal branch. */
static mat su3_haar(const stream *st)
{
    double u[20];
    for (uint32_t b = 0; b < 5; ++b) stream_uniforms(st, b, u + 4 * b);
    mat z = mat_zero();
    for (int k = 0; k < 9; ++k) {
        double rad = sqrt(-2.0 * log(u[2 * k]));
        z.e[k / 3][k % 3] = rad * cexp(I * 2.0 * M_PI * u[2 * k + 1]);
    }
    for (int r = 0; r < 3; ++r) {
        for (int q = 0; q < r; ++q) {
            cplx proj = 0.0;
            for (int c = 0; c < 3; ++c) proj += conj(z.e[q][c]) * z.e[r][c];
            for (int c = 0; c < 3; ++c) z.e[r][c] -= proj * z.e[q][c];
        }
        double n = 0.0;
        for (int c = 0; c < 3; ++c) n += creal(z.e[r][c] * conj(z.e[r][c]));
        n = sqrt(n);
        for (int c = 0; c < 3; ++c) z.e[r][c] /= n;
    }
    cplx d = mat_det(3, &z);
    cplx fix = cexp(-I * carg(d) / 3.0);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) z.e[r][c] *= fix;
    return z;
}

/* ------------------------------------------------------------------------ */
/* Link updates                                                              */
/* ------------------------------------------------------------------------ */

/* SU(2) heat-bath of one link (Kennedy-Pendleton).  A = k V with k = sqrt(det
 * A); Ut_new = X V^+ with X distributed as exp(beta k Re Tr X / 2).  Returns 1
 * if NHIT was exhausted (link kept). */
static int heatbath_su2(const oracle_lattice *L, uint64_t seed, long s, int mu,
                        mat *out)
{
    mat a = staple(L, s, mu);
    double det = creal(mat_det(2, &a));
    double k = sqrt(det > 0.0 ? det : 0.0);
    double alpha = L->beta * k;
    stream dir = lattice_stream(L, seed, L->sweep, s, mu, 0, KIND_DIR);
    mat b = link_phase(L, s, mu), bd = mat_dag(2, &b);
    double x[4];
    mat ut_new;
    if (alpha == 0.0) {
        su2_haar(&dir, 0, x);
        ut_new = quat_to_mat(x);
    } else {
        stream tries = lattice_stream(L, seed, L->sweep, s, mu, 0, KIND_TRY);
        double delta;
        if (!kp_draw(alpha, L->nhit, &tries, &delta)) {
            *out = get_link(L, s, mu);
            return 1;
        }
        su2_with_delta(delta, &dir, x);
        mat xm = quat_to_mat(x);
        mat v = a;
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) v.e[i][j] /= k;
        mat vd = mat_dag(2, &v);
        ut_new = mat_mul(2, &xm, &vd);
    }
    *out = mat_mul(2, &ut_new, &bd);
    return 0;
}

/* SU(2) overrelaxation: Ut_new = V^+ Ut^+ V^+, which keeps Re Tr(Ut A). */
static void overrelax_su2(const oracle_lattice *L, long s, int mu, mat *out)
{
    mat a = staple(L, s, mu);
    double det = creal(mat_det(2, &a));
    double k = sqrt(det > 0.0 ? det : 0.0);
    if (k == 0.0) {
        *out = get_link(L, s, mu);
        return;
    }
    mat v = a;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) v.e[i][j] /= k;
    mat vd = mat_dag(2, &v);
    mat ut = eff_link(L, s, mu), utd = mat_dag(2, &ut);
    mat ut_new = mat_mul3(2, &vd, &utd, &vd);
    mat b = link_phase(L, s, mu), bd = mat_dag(2, &b);
    *out = mat_mul(2, &ut_new, &bd);
}

/* Cabibbo-Marinari subgroups (rows/cols), updated in this order. */
static const int SUBGROUP[3][2] = { { 0, 1 }, { 1, 2 }, { 0, 2 } };

/* SU(3) heat-bath of one link: for each subgroup, W = Ut A, project its 2x2
 * block onto k V (V in SU(2)), draw X with weight exp((2 beta k / 3) x0) by
 * Kennedy-Pendleton and left-multiply the link by the embedded R = X V^+.
 * Returns the number of subgroups whose NHIT tries were exhausted. */
static int heatbath_su3(const oracle_lattice *L, uint64_t seed, long s, int mu,
                        mat *out)
{
    mat a = staple(L, s, mu);
    mat b = link_phase(L, s, mu);
    mat u = get_link(L, s, mu);
    int exhausted = 0;
    for (int sub = 0; sub < 3; ++sub) {
        int i = SUBGROUP[sub][0], j = SUBGROUP[sub][1];
        mat ut = mat_mul(3, &u, &b);
        mat w = mat_mul(3, &ut, &a);
        double q[4];
        block_to_quat(&w, i, j, q);
        double k = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        double alpha = 2.0 * L->beta * k / 3.0;
        stream dir = lattice_stream(L, seed, L->sweep, s, mu, sub, KIND_DIR);
        double x[4];
        mat r;
        if (alpha == 0.0) {
            su2_haar(&dir, 0, x);
            r = quat_to_mat(x);
        } else {
            stream tries = lattice_stream(L, seed, L->sweep, s, mu, sub, KIND_TRY);
            double delta;
            if (!kp_draw(alpha, L->nhit, &tries, &delta)) {
                ++exhausted;
                continue;
            }
            su2_with_delta(delta, &dir, x);
            double vq[4] = { q[0] / k, q[1] / k, q[2] / k, q[3] / k };
            mat xm = quat_to_mat(x), v = quat_to_mat(vq), vd = mat_dag(2, &v);
            r = mat_mul(2, &xm, &vd);
        }
        mat re = embed(3, &r, i, j);
        u = mat_mul(3, &re, &u);
    }
    *out = u;
    return exhausted;
}

/* SU(3) overrelaxation: for each subgroup R = (V^+)^2, which keeps
 * Re Tr(R W) and hence Re Tr(Ut A). */
static void overrelax_su3(const oracle_lattice *L, long s, int mu, mat *out)
{
    mat a = staple(L, s, mu);
    mat b = link_phase(L, s, mu);
    mat u = get_link(L, s, mu);
    for (int sub = 0; sub < 3; ++sub) {
        int i = SUBGROUP[sub][0], j = SUBGROUP[sub][1];
        mat ut = mat_mul(3, &u, &b);
        mat w = mat_mul(3, &ut, &a);
        double q[4];
        block_to_quat(&w, i, j, q);
        double k = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        if (k == 0.0) continue;
        double vq[4] = { q[0] / k, q[1] / k, q[2] / k, q[3] / k };
        mat v = quat_to_mat(vq), vd = mat_dag(2, &v);
        mat r = mat_mul(2, &vd, &vd);
        mat re = embed(3, &r, i, j);
        u = mat_mul(3, &re, &u);
    }
    *out = u;
}

static int update_link(const oracle_lattice *L, int kind, uint64_t seed, long s,
                       int mu, mat *out)
{
    if (is_frozen(L, s, mu)) {
        *out = get_link(L, s, mu);
        return 0;
    }
    if (kind == ORACLE_HEATBATH)
        return L->N == 2 ? heatbath_su2(L, seed, s, mu, out)
                         : heatbath_su3(L, seed, s, mu, out);
    if (L->N == 2) overrelax_su2(L, s, mu, out);
    else overrelax_su3(L, s, mu, out);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Reunitarization (sec. 5): SU(2) quaternion normalisation; SU(3)           */
/* Gram-Schmidt of rows 1, 2 and row 3 = conj(row1 x row2).                  */
/* ------------------------------------------------------------------------ */
static mat reunitarize_one(int N, const mat *m)
{
    if (N == 2) {
        double q[4];
        block_to_quat(m, 0, 1, q);
        double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        for (int i = 0; i < 4; ++i) q[i] /= n;
        return quat_to_mat(q);
    }
    mat u = *m;
    double n1 = 0.0;
    for (int c = 0; c < 3; ++c) n1 += creal(u.e[0][c] * conj(u.e[0][c]));
    n1 = sqrt(n1);
    for (int c = 0; c < 3; ++c) u.e[0][c] /= n1;
    cplx proj = 0.0;
    for (int c = 0; c < 3; ++c) proj += conj(u.e[0][c]) * u.e[1][c];
    for (int c = 0; c < 3; ++c) u.e[1][c] -= proj * u.e[0][c];
    double n2 = 0.0;
    for (int c = 0; c < 3; ++c) n2 += creal(u.e[1][c] * conj(u.e[1][c]));
    n2 = sqrt(n2);
    for (int c = 0; c < 3; ++c) u.e[1][c] /= n2;
    for (int c = 0; c < 3; ++c) {
        int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
        u.e[2][c] = conj(u.e[0][c1] * u.e[1][c2] - u.e[0][c2] * u.e[1][c1]);
    }
    return u;
}

/* ------------------------------------------------------------------------ */
/* Public API                                                                */
/* ------------------------------------------------------------------------ */
oracle_lattice *oracle_create(int N, int Ns, int Nt, double beta, int flux,
                              int nhit, uint32_t lattice_id)
{
    return oracle_create_ex(N, Ns, Nt, beta, flux, 0, nhit, lattice_id,
                            ORACLE_FIELD_LINKS);
}

oracle_lattice *oracle_create_ex(int N, int Ns, int Nt, double beta, int flux,
                                 int flux8, int nhit, uint32_t lattice_id,
                                 int field_mode)
{
    if ((N != 2 && N != 3) || Ns < 2 || Nt < 2 || (Ns & 1) || (Nt & 1) ||
        beta < 0.0 || nhit < 1 || (N == 2 && flux8 != 0) ||
        (field_mode != ORACLE_FIELD_LINKS && field_mode != ORACLE_FIELD_FROZEN))
        return NULL;
    oracle_lattice *L = calloc(1, sizeof *L);
    if (!L) return NULL;
    L->N = N; L->Ns = Ns; L->Nt = Nt;
    L->V = (long)Ns * Ns * Ns * Nt;
    L->beta = beta; L->flux = flux; L->flux8 = flux8; L->nhit = nhit;
    L->field_mode = field_mode;
    L->lattice_id = lattice_id;
    L->U = calloc((size_t)L->V * 4 * N * N, sizeof(cplx));
    if (!L->U) {
        free(L);
        return NULL;
    }
    oracle_cold_start(L);
    return L;
}

void oracle_destroy(oracle_lattice *L)
{
    if (!L) return;
    free(L->U);
    free(L);
}

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_cold_start(oracle_lattice *L)
{
    mat one = mat_identity(L->N);
    for (long s = 0; s < L->V; ++s)
        for (int mu = 0; mu < 4; ++mu) put_link(L, s, mu, &one);
    set_frozen_links(L);
    L->sweep = 0;
    L->exhausted = 0;
}

void oracle_hot_start(oracle_lattice *L, uint64_t seed)
{
#pragma omp parallel for schedule(static)
    for (long s = 0; s < L->V; ++s) {
        for (int mu = 0; mu < 4; ++mu) {
            stream st = lattice_stream(L, seed, START_SWEEP_WORD, s, mu, 0,
                                       KIND_START);
            mat u;
            if (L->N == 2) {
                double x[4];
                su2_haar(&st, 0, x);
                u = quat_to_mat(x);
            } else {
                u = su3_haar(&st);
            }
            put_link(L, s, mu, &u);
        }
    }
    set_frozen_links(L);
    L->sweep = 0;
    L->exhausted = 0;
}

/* One checkerboard phase.  Links of direction mu on sites of one parity do not
 * appear in one another's staples, so they are updated in place. */
void oracle_phase(oracle_lattice *L, int kind, int parity, int mu,
                  uint64_t seed)
{
    long exhausted = 0;
#pragma omp parallel for schedule(static) reduction(+ : exhausted)
    for (long s = 0; s < L->V; ++s) {
        if (site_parity(L, s) != parity) continue;
        mat u;
        exhausted += update_link(L, kind, seed, s, mu, &u);
        put_link(L, s, mu, &u);
    }
    L->exhausted += exhausted;
}

void oracle_reunitarize(oracle_lattice *L)
{
#pragma omp parallel for schedule(static)
    for (long s = 0; s < L->V; ++s)
        for (int mu = 0; mu < 4; ++mu) {
            if (is_frozen(L, s, mu)) continue;
            mat u = get_link(L, s, mu);
            mat r = reunitarize_one(L->N, &u);
            put_link(L, s, mu, &r);
        }
}

/* The links of one checkerboard phase only.  A sweep's reunitarization (R7)
 * can be carried by its last overrelaxation pass, each link reunitarized
 * right after its update there: every link is updated exactly once in a pass,
 * so after the pass every link has been reunitarized.  Following that pass
 * phase by phase needs the projection of just the phase's links. */
void oracle_reunitarize_phase(oracle_lattice *L, int parity, int mu)
{
#pragma omp parallel for schedule(static)
    for (long s = 0; s < L->V; ++s) {
        if (site_parity(L, s) != parity || is_frozen(L, s, mu)) continue;
        mat u = get_link(L, s, mu);
        mat r = reunitarize_one(L->N, &u);
        put_link(L, s, mu, &r);
    }
}

void oracle_reunitarize_matrix(int N, double *m)
{
    mat u = mat_zero();
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j)
            u.e[i][j] = m[2 * (i * N + j)] + I * m[2 * (i * N + j) + 1];
    mat r = reunitarize_one(N, &u);
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            m[2 * (i * N + j)] = creal(r.e[i][j]);
            m[2 * (i * N + j) + 1] = cimag(r.e[i][j]);
        }
}

void oracle_sweep(oracle_lattice *L, int n_hb, int n_or, uint64_t seed)
{
    for (int h = 0; h < n_hb; ++h) {
        for (int p = 0; p < 2; ++p)
            for (int mu = 0; mu < 4; ++mu)
                oracle_phase(L, ORACLE_HEATBATH, p, mu, seed);
        for (int o = 0; o < n_or; ++o)
            for (int p = 0; p < 2; ++p)
                for (int mu = 0; mu < 4; ++mu)
                    oracle_phase(L, ORACLE_OVERRELAX, p, mu, seed);
        oracle_reunitarize(L);
        L->sweep += 1;
    }
}

/* (1/N) Re Tr of the plaquette U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+. */
static double plaquette(const oracle_lattice *L, long s, int mu, int nu,
                        int effective)
{
    int N = L->N;
    long s_pmu = site_shift(L, s, mu, +1), s_pnu = site_shift(L, s, nu, +1);
    mat a = effective ? eff_link(L, s, mu) : get_link(L, s, mu);
    mat b = effective ? eff_link(L, s_pmu, nu) : get_link(L, s_pmu, nu);
    mat c = effective ? eff_link(L, s_pnu, mu) : get_link(L, s_pnu, mu);
    mat d = effective ? eff_link(L, s, nu) : get_link(L, s, nu);
    mat cd = mat_dag(N, &c), dd = mat_dag(N, &d);
    mat ab = mat_mul(N, &a, &b);
    mat abc = mat_mul(N, &ab, &cd);
    mat p = mat_mul(N, &abc, &dd);
    return creal(mat_trace(N, &p)) / N;
}

static void measure_plaquettes(const oracle_lattice *L, int effective,
                               double plaq[3])
{
    double *ps = malloc(sizeof(double) * (size_t)L->V);
    double *pt = malloc(sizeof(double) * (size_t)L->V);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < L->V; ++s) {
        double sp = 0.0, tp = 0.0;
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu) {
                double p = plaquette(L, s, mu, nu, effective);
                if (nu == 3) tp += p;
                else sp += p;
            }
        ps[s] = sp;
        pt[s] = tp;
    }
    double sum_s = 0.0, sum_t = 0.0;
    for (long s = 0; s < L->V; ++s) {
        sum_s += ps[s];
        sum_t += pt[s];
    }
    free(ps);
    free(pt);
    plaq[0] = (sum_s + sum_t) / (6.0 * L->V);
    plaq[1] = sum_s / (3.0 * L->V);
    plaq[2] = sum_t / (3.0 * L->V);
}

void oracle_measure(const oracle_lattice *L, double plaq[3], double poly[2])
{
    measure_plaquettes(L, 1, plaq);
    int N = L->N;
    long V3 = (long)L->Ns * L->Ns * L->Ns;
    cplx sum = 0.0;
    for (long sx = 0; sx < V3; ++sx) {
        mat p = mat_identity(N);
        for (int t = 0; t < L->Nt; ++t) {
            mat u = eff_link(L, sx + V3 * t, 3);
            p = mat_mul(N, &p, &u);
        }
        sum += mat_trace(N, &p) / N;
    }
    poly[0] = creal(sum) / V3;
    poly[1] = cimag(sum) / V3;
}

void oracle_measure_planes(const oracle_lattice *L, double planes[6])
{
    static const int PLANE[6][2] = { { 0, 1 }, { 0, 2 }, { 1, 2 },
                                     { 0, 3 }, { 1, 3 }, { 2, 3 } };
    for (int k = 0; k < 6; ++k) {
        double sum = 0.0;
        for (long s = 0; s < L->V; ++s)
            sum += plaquette(L, s, PLANE[k][0], PLANE[k][1], 1);
        planes[k] = sum / (double)L->V;
    }
}

void oracle_measure_bare(const oracle_lattice *L, double plaq[3])
{
    measure_plaquettes(L, 0, plaq);
}

void oracle_get_links(const oracle_lattice *L, double *out)
{
    size_t n = (size_t)L->V * 4 * L->N * L->N;
    for (size_t i = 0; i < n; ++i) {
        out[2 * i] = creal(L->U[i]);
        out[2 * i + 1] = cimag(L->U[i]);
    }
}

void oracle_set_links(oracle_lattice *L, const double *in)
{
    size_t n = (size_t)L->V * 4 * L->N * L->N;
    for (size_t i = 0; i < n; ++i) L->U[i] = in[2 * i] + I * in[2 * i + 1];
}

uint32_t oracle_get_sweep(const oracle_lattice *L) { return L->sweep; }
void oracle_set_sweep(oracle_lattice *L, uint32_t sweep) { L->sweep = sweep; }
long oracle_exhausted(const oracle_lattice *L) { return L->exhausted; }

static void mat_out(int N, const mat *m, double *out)
{
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            out[2 * (i * N + j)] = creal(m->e[i][j]);
            out[2 * (i * N + j) + 1] = cimag(m->e[i][j]);
        }
}

void oracle_staple(const oracle_lattice *L, long s, int mu, double *out)
{
    mat a = staple(L, s, mu);
    mat_out(L->N, &a, out);
}

double oracle_link_action(const oracle_lattice *L, long s, int mu)
{
    mat a = staple(L, s, mu), ut = eff_link(L, s, mu);
    mat p = mat_mul(L->N, &ut, &a);
    return creal(mat_trace(L->N, &p));
}

int oracle_link_update(const oracle_lattice *L, int kind, long s, int mu,
                       uint64_t seed, double *out)
{
    mat u;
    int ex = update_link(L, kind, seed, s, mu, &u);
    mat_out(L->N, &u, out);
    return ex;
}

void oracle_kp_samples(double alpha, int nhit, uint64_t seed, long n,
                       double *a0, int *tries)
{
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) {
        stream st = plain_stream(seed, (uint32_t)i, 0, KIND_TRY << 4);
        double d = 0.0;
        tries[i] = kp_draw(alpha, nhit, &st, &d);
        a0[i] = tries[i] ? 1.0 - d : 0.0;
    }
}

void oracle_su2_samples(double alpha, int nhit, uint64_t seed, long n,
                        double *x4)
{
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) {
        stream dir = plain_stream(seed, (uint32_t)i, 0, KIND_DIR << 4);
        double *x = x4 + 4 * i;
        if (alpha == 0.0) {
            su2_haar(&dir, 0, x);
            continue;
        }
        stream st = plain_stream(seed, (uint32_t)i, 0, KIND_TRY << 4);
        double delta;
        if (!kp_draw(alpha, nhit, &st, &delta)) {
            x[0] = x[1] = x[2] = x[3] = 0.0;
            continue;
        }
        su2_with_delta(delta, &dir, x);
    }
}

void oracle_haar_samples(int N, uint64_t seed, long n, double *out)
{
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) {
        stream st = plain_stream(seed, (uint32_t)i, START_SWEEP_WORD,
                                 KIND_START << 4);
        mat u;
        if (N == 2) {
            double x[4];
            su2_haar(&st, 0, x);
            u = quat_to_mat(x);
        } else {
            u = su3_haar(&st);
        }
        mat_out(N, &u, out + (size_t)2 * N * N * i);
    }
}
