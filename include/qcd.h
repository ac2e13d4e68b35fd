/*
 * qcd.h -- C ABI of libqcdgb300: the checkerboard Monte Carlo sweep of pure
 * SU(2)/SU(3) Wilson lattice gauge theory at finite temperature in a constant
 * Abelian chromomagnetic background field, on one NVIDIA GB300 (sm_103a).
 *
 * What the calls compute.  The paper (QCDGPU, Demchik & Kolomoyets) describes
 * SU(N) gluodynamics in an external field at finite temperature (abstract,
 * sec. 1), links stored as N x N matrices split into 4-vectors with the site
 * index fastest (sec. 3.3), (pseudo)heat-bath updates of the even and odd
 * checkerboard halves (sec. 3.3), hot start, NHIT = 10 tries and
 * reunitarization (sec. 5), and plaquette / Polyakov-loop measurements (sec. 1,
 * sec. 5).  It prints no formulas; the library implements the textbook methods
 * those passages name:
 *   - Wilson action S = beta sum_P (1 - Re Tr U_P / N);
 *   - SU(2): Kennedy-Pendleton heat-bath, k = sqrt(det A), weight
 *     exp(beta k a0);
 *   - SU(3): Cabibbo-Marinari heat-bath over the SU(2) subgroups (0,1),(1,2),
 *     (0,2), weight exp((2 beta / 3) k a0) per subgroup;
 *   - microcanonical overrelaxation (SU(2) reflection, per SU(3) subgroup
 *     R = (V^+)^2);
 *   - reunitarization (SU(2) quaternion normalisation; SU(3) Gram-Schmidt of
 *     rows 1, 2 and row 3 = conj(row1 x row2)), computed in FP64;
 *   - background field: U(1) phase along lambda3 (sigma3 for SU(2)) on y-links,
 *     B_y(x) = diag(e^{i phi}, e^{-i phi} [, 1]), phi = 2 pi n x / Ns^2, applied
 *     as the effective link Ut = U B.  Updates act on Ut and store U = Ut B^+;
 *   - random numbers: Philox-4x32-10 with key (seed_lo ^ lattice_id *
 *     0x9E3779B9, seed_hi) and counter (site, sweep, mu | subgroup << 2 |
 *     kind << 4, block), uniforms ((w >> 9) + 1/2) 2^-23.
 *
 * Conventions.
 *   - mu = 0,1,2,3 is x,y,z,t; site s = x + Ns (y + Ns (z + Ns t)).
 *   - Canonical host layout (get/set): FP64 [s][mu][row][col][re,im],
 *     N*N complex numbers per link, x fastest.  It does not depend on the
 *     device layout.
 *   - Return value: QCD_OK (0) or a negative QCD_ERR_* code; no error is fatal
 *     and qcd_last_error() gives a message for the calling thread.
 *   - Ownership: the library owns the device memory it allocates, the caller
 *     owns every host buffer it passes, the CUDA stream is borrowed.
 *   - Ordering: every call is ordered on the lattice's stream.  Calls that
 *     return host data (measure, get, counters) synchronize that stream.
 *   - A handle is not thread-safe; distinct handles may be used concurrently.
 */
#ifndef QCD_H
#define QCD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QCD_OK 0
#define QCD_ERR_INVALID_ARG (-1)   /* bad group, odd/small extents, beta < 0 ... */
#define QCD_ERR_OOM (-2)           /* device or host allocation failed          */
#define QCD_ERR_CUDA (-3)          /* a CUDA call failed; see qcd_last_error()  */
#define QCD_ERR_TIMEOUT (-4)       /* a bounded device wait ran out             */
#define QCD_ERR_NOT_SUPPORTED (-5) /* valid but unsupported request            */

/* Link storage. */
#define QCD_FP64_PLAIN 0      /* SU(2): 4 FP64 reals; SU(3): 18 FP64 reals       */
#define QCD_FP32_COMPRESSED 1 /* SU(2): 4 FP32 reals; SU(3): rows 1-2, 12 FP32
                                 reals, row 3 rebuilt as conj(row1 x row2)      */
/* Start. */
#define QCD_COLD 0 /* every link the unit matrix                             */
#define QCD_HOT 1  /* every link Haar-random: SU(2) Shoemake, SU(3) Mezzadri */
/* Field modes (sec. 1: lattice gauge theory in an external chromomagnetic
 * field; the paper gives no formula, so both are readings of that claim).
 * B_y(x) = diag(e^{i phi}, e^{-i phi} [, 1]), phi = 2 pi n x / Ns^2 along
 * lambda3 (sigma3 for SU(2)), times the lambda8 part of qcd_lattice_create_ex
 * for SU(3); B = 1 on x-, z- and t-links. */
#define QCD_FIELD_LINKS 0  /* effective links U B on every link: updates and
                              measurements act on U B, U = (U B)_new B^+ is
                              stored (a change of variables of the n = 0
                              theory for the effective-link observables)     */
#define QCD_FIELD_FROZEN 1 /* the spatial links of the time slice t = 0 are
                              set to B and never updated nor reunitarized;
                              every other link carries no phase (fixed-
                              boundary background field, physically visible) */
/* Update kinds for qcd_phase. */
#define QCD_HEATBATH 0
#define QCD_OVERRELAX 1
#define QCD_OVERRELAX_REUNIT 2  /* overrelaxation, then the FP64 reunitarization
                                   of each updated link: the kernels of the
                                   last pass of a sweep                      */
#define QCD_OVERRELAX_MEASURE 3 /* as QCD_OVERRELAX_REUNIT, and the plaquette
                                   sums of a working sweep's fused
                                   measurement (odd parity, mu >= 1 only)    */

typedef struct qcd_lattice qcd_lattice;

/* Create one lattice Ns^3 x Nt (finite temperature: sec. 4 singles out the
 * time extent) and apply the start (sec. 5 "hot" initialisation).
 *   out       receives the handle (NULL on failure).
 *   group     2 or 3.
 *   Ns, Nt    even, >= 2; Ns^3 Nt < 2^31.
 *   beta      >= 0.
 *   flux      flux quantum n of the background field (any integer, 0 = none).
 *   precision QCD_FP64_PLAIN or QCD_FP32_COMPRESSED.
 *   start     QCD_COLD or QCD_HOT.
 *   seed      Philox key for the hot start and the default for qcd_sweep.
 *   stream    cudaStream_t to order work on, or NULL for the default stream.
 * Allocates the links and a few KB of reduction scratch on the current
 * device.  NHIT defaults to 10 (sec. 5). */
int qcd_lattice_create(qcd_lattice **out, int group, int Ns, int Nt,
                       double beta, int flux, int precision, int start,
                       uint64_t seed, void *stream);
/* As qcd_lattice_create with a lambda8 flux and an explicit field mode.
 *   flux8       flux quanta of the lambda8 component (SU(3) only; nonzero for
 *               group 2 is QCD_ERR_INVALID_ARG).  With the generator
 *               sqrt(3) lambda8 = diag(1, 1, -2) the y-link background is
 *               B_y(x) = diag(e^{i(p3 + p8)}, e^{i(-p3 + p8)}, e^{-2 i p8}),
 *               p3 = 2 pi flux x / Ns^2, p8 = 2 pi flux8 x / Ns^2.
 *   field_mode  QCD_FIELD_LINKS or QCD_FIELD_FROZEN (anything else is
 *               QCD_ERR_INVALID_ARG).  In the frozen mode the start is applied
 *               to every link and then the t = 0 spatial links are overwritten
 *               with B; qcd_set_links stores what it is given, frozen links
 *               included (a checkpoint holds them as B).
 * qcd_lattice_create is this call with flux8 = 0 and QCD_FIELD_LINKS. */
int qcd_lattice_create_ex(qcd_lattice **out, int group, int Ns, int Nt,
                          double beta, int flux, int flux8, int field_mode,
                          int precision, int start, uint64_t seed,
                          void *stream);
/* A lattice divided into two parts along t (Sect. "Multi-GPU Mode and
 * Distributed Simulations": dividing the lattice is also the remedy when the
 * device memory is too small).  Arguments as for qcd_lattice_create_ex, plus
 *   nt_device   t-slices 0 .. nt_device-1 of every link array are placed in
 *               device memory and the rest in pinned host memory of the NUMA
 *               node next to the GPU; 0 <= nt_device <= Nt, else
 *               QCD_ERR_INVALID_ARG.  The device part is rounded up to the
 *               mapping granule (2 MB on GB300): qcd_get_residency reports
 *               what was placed.
 * Both parts sit behind one virtual address range, so every kernel, sweep,
 * measurement and copy behaves exactly as on a device-resident lattice and
 * gives bit-identical results; the host part is read and written by the GPU
 * over the CPU-GPU link, at that link's bandwidth.  Each link array is padded
 * to a whole number of granules.  Split lattices skip the launch-shape
 * autotuner (128 threads per block unless a tuned shape for the same
 * lattice is cached or qcd_set_block sets one).  qcd_get_links / qcd_set_links
 * (and the checkpoint calls built on them) stage the canonical FP64 copy in
 * device memory, so they need room for it there.  QCD_ERR_NOT_SUPPORTED when
 * the device cannot map host-NUMA memory; QCD_ERR_OOM when either part cannot
 * be allocated. */
int qcd_lattice_create_split(qcd_lattice **out, int group, int Ns, int Nt,
                             double beta, int flux, int flux8, int field_mode,
                             int precision, int start, uint64_t seed,
                             void *stream, int nt_device);
/* Bytes of link storage in device and in host memory (padding included) and
 * the number of leading t-slices wholly in device memory (Nt for an ordinary
 * lattice). */
int qcd_get_residency(qcd_lattice *lat, size_t *device_bytes,
                      size_t *host_bytes, int *nt_device);
int qcd_lattice_destroy(qcd_lattice *lat);
/* The field mode the lattice was created with. */
int qcd_get_field_mode(qcd_lattice *lat, int *field_mode);

/* Cap on Kennedy-Pendleton tries per (link, subgroup); >= 1.  When every try
 * is rejected the SU(2) link is kept and the SU(3) subgroup step is skipped
 * (both leave the target distribution invariant); such events are counted. */
int qcd_set_nhit(qcd_lattice *lat, int nhit);

/* Sweep (sec. 3.3, sec. 5): n_heatbath times { one heat-bath pass; n_overrelax
 * overrelaxation passes; FP64 reunitarization of every link }.  A pass visits
 * the 8 checkerboard phases: parity even then odd, inside it mu = x,y,z,t.
 * The reunitarization is applied by the last overrelaxation pass's kernels
 * to each link right after its update in that pass (each link is updated
 * once per pass), so it costs no separate pass over the links; with
 * n_overrelax = 0 a reunitarization kernel follows the heat-bath pass.
 * The sweep counter (Philox counter word 1) advances once per heat-bath pass.
 * seed is the Philox key of this call (pass the create seed to continue one
 * stream).  n_heatbath >= 0, n_overrelax >= 0. */
int qcd_sweep(qcd_lattice *lat, int n_heatbath, int n_overrelax, uint64_t seed);

/* A working sweep (sec. 4: a sweep followed by measurements): n_heatbath
 * sweeps as qcd_sweep, then the plaquette and Polyakov loop of the resulting
 * configuration into host_out[5] = {P, P_s, P_t, Re L, Im L} (as
 * qcd_measure).  With n_overrelax >= 1, FP32 SU(3) storage and the
 * effective-link field mode, the plaquette sums are fused into the last
 * overrelaxation pass: after the pass each plaquette of plane (mu, nu < mu)
 * contains exactly one odd mu-link, so the odd phases mu = 1, 2, 3 add
 * Re Tr(Ut A_nu) for nu < mu over their updated links (A_nu the staples of
 * plane (mu, nu); each warp adds its threads' FP32 values by error-free
 * TwoSum and finishes in FP64, the block adds its warps in FP64, and the final
 * sums take the 1/3) and no separate pass over the links is needed; otherwise
 * the measurement kernels run after the sweeps.  wait = 1: returns after the
 * results are on the host; wait = 0: host_out (page-locked for overlap) is
 * filled once the stream is synchronized. */
int qcd_working_sweep(qcd_lattice *lat, int n_heatbath, int n_overrelax,
                      uint64_t seed, double *host_out, int wait);

/* One checkerboard phase (parity 0/1, direction mu) at the current sweep
 * counter, with no counter change, launched as the sweep launches it.  For
 * tests and sampled checks of every kernel a sweep runs:
 *   QCD_HEATBATH, QCD_OVERRELAX   the heat-bath and the plain overrelaxation
 *                                 phases (no reunitarization);
 *   QCD_OVERRELAX_REUNIT          a phase of the last overrelaxation pass of a
 *                                 sweep: each updated link is reunitarized
 *                                 (sec. 5) in FP64 before it is stored;
 *   QCD_OVERRELAX_MEASURE         a plane-summing phase of a working sweep's
 *                                 last pass (parity 1, mu = 1, 2, 3; else
 *                                 QCD_ERR_INVALID_ARG): as QCD_OVERRELAX_REUNIT,
 *                                 and Re Tr of every plaquette of the planes
 *                                 (mu, nu < mu) is summed (SU(2): (1/2) Re Tr),
 *                                 through the updated link of each, into the
 *                                 lattice's measurement scratch (the SU(3)
 *                                 1/3 is taken in the final sums);
 *                                 QCD_ERR_NOT_SUPPORTED
 *                                 where qcd_working_sweep does not fuse its
 *                                 measurement (FP64 SU(3), frozen mode).
 * After the eight phases of a last pass run this way (QCD_OVERRELAX_REUNIT for
 * parity 0 and for (1, 0), QCD_OVERRELAX_MEASURE for (1, 1..3)),
 * qcd_measure_fused_finish returns the working sweep's measurement. */
int qcd_phase(qcd_lattice *lat, int kind, int parity, int mu, uint64_t seed);
/* The tail of a working sweep's fused measurement (sec. 5: working sweeps end
 * with measurements): the Polyakov loop and the final FP64 sums of the plane
 * sums left by the QCD_OVERRELAX_MEASURE phases (1, 1), (1, 2), (1, 3).
 * host_out[8] = {P, P_s, P_t, Re L, Im L, P_1, P_2, P_3}, P_mu the mean
 * plaquette of the planes phase (1, mu) summed: (x,y); (x,z), (y,z);
 * (x,t), (y,t), (z,t).  A plane (mu, nu < mu) holds no link of a later phase
 * of the pass, so each P_mu is also that of the configuration the pass ends
 * with.  The phases and this call must run with one launch shape (the block
 * size of qcd_set_block, or the tuned one: the plane sums are one per block
 * of the phase kernels).  QCD_ERR_NOT_SUPPORTED as for
 * QCD_OVERRELAX_MEASURE.  Host pointer; synchronizes the stream. */
int qcd_measure_fused_finish(qcd_lattice *lat, double *host_out);
/* FP64 reunitarization of every link. */
int qcd_reunitarize(qcd_lattice *lat);

/* Measurements on the effective links (sec. 1, sec. 5), FP64 sums:
 *   plaquette[3] = {P, P_s, P_t}: (1/N) Re Tr of the plaquette averaged over
 *     all 6V plaquettes, the 3V spatial ones (mu,nu < t) and the 3V temporal;
 *   polyakov[2] = {Re L, Im L}: (1/N) Tr of the ordered product of t-links
 *     t = 0..Nt-1, averaged over the Ns^3 spatial sites.
 * Either pointer may be NULL.  Host pointers; synchronizes the stream. */
int qcd_measure(qcd_lattice *lat, double *plaquette, double *polyakov);
/* The same plaquettes on the bare links U (they depend on the field). */
int qcd_measure_bare(qcd_lattice *lat, double *plaquette);
/* qcd_measure without the wait: enqueues the measurement and the copy of the
 * five results {P, P_s, P_t, Re L, Im L} into host_out (host double[5];
 * page-locked memory lets the copy overlap other work) on the lattice's
 * stream and returns.  host_out must stay valid, and is filled, once the
 * stream has been synchronized.  Not counted by the live profile.  For
 * pipelines that keep several lattices in flight on separate streams. */
int qcd_measure_async(qcd_lattice *lat, double *host_out);

/* Links in the canonical FP64 host layout (4 V N^2 complex numbers).
 * set_links rounds to the storage (FP32-12 keeps rows 1-2; SU(2) keeps the
 * SU(2)-projection q0 + i q.sigma of each 2x2 matrix). */
int qcd_get_links(qcd_lattice *lat, double *host_out);
int qcd_set_links(qcd_lattice *lat, const double *host_in);

/* Raw device storage to and from a host buffer of qcd_link_bytes() bytes
 * (pinned memory gives full copy speed).  Used for checkpoints and for
 * end-to-end runs that stage configurations on the host. */
int qcd_link_bytes(const qcd_lattice *lat, size_t *bytes);
int qcd_copy_links_in(qcd_lattice *lat, const void *host_in, size_t bytes);
int qcd_copy_links_out(qcd_lattice *lat, void *host_out, size_t bytes);

/* Sweep counter (heat-bath passes since the start) and NHIT-exhaustion
 * counter. */
int qcd_get_sweep(qcd_lattice *lat, uint32_t *sweep);
int qcd_set_sweep(qcd_lattice *lat, uint32_t sweep);
int qcd_get_exhausted(qcd_lattice *lat, unsigned long long *count);

/* Launch shape: threads per block of the phase kernels (0 = autotune on the
 * next sweep; otherwise a multiple of 32 in [32, 1024]). */
int qcd_set_block(qcd_lattice *lat, int threads);
int qcd_get_block(const qcd_lattice *lat, int *threads);

/* Checkpoint / resume (the paper's portable saved computation state, sec. 3.1
 * and sec. 6).  The random numbers are counter-based, so the state is the
 * links plus (seed, sweep counter, NHIT): resuming reproduces the
 * uninterrupted run bit for bit.  File: 80-byte little-endian header (magic
 * "QCDGB300", version 1, group, storage, Ns, Nt, flux, NHIT, lattice id, sweep
 * counter, seed, beta, NHIT-exhaustion count) followed by the links in the
 * canonical FP64 layout, so a file written with one storage loads into
 * either.
 *   qcd_save: writes `path` (overwrites); synchronizes the stream.
 *   qcd_lattice_load: creates a lattice from `path` with the given storage
 *   (QCD_FP64_PLAIN or QCD_FP32_COMPRESSED; FP32 rounds FP64 links) on
 *   `stream`.  QCD_ERR_INVALID_ARG for an unreadable or malformed file. */
int qcd_save(qcd_lattice *lat, const char *path);
int qcd_lattice_load(qcd_lattice **out, const char *path, int precision,
                     void *stream);

/* Live kernel timing (the paper's optional run-time profiling of kernels,
 * sec. 3.2).  When enabled, CUDA events are recorded on the lattice's stream
 * around every kernel the sweep and the measurements launch (inside the
 * captured sweep graph), and their durations are accumulated per category:
 *   QCD_PROF_HEATBATH  heat-bath phase kernels
 *   QCD_PROF_OVERRELAX overrelaxation phase kernels
 *   QCD_PROF_REUNIT    the last overrelaxation pass, whose kernels also
 *                      reunitarize the links they update, and the
 *                      sweep-counter advance (with n_overrelax = 0: the
 *                      reunitarization kernel)
 *   QCD_PROF_MEASURE   measurement kernels (block partials + final sum)
 * Events bracket groups of kernels (the heat-bath pass, the other
 * overrelaxation passes, the last pass, the measurement), and a group's time
 * is counted for all its kernels.  Enabling or disabling resets the totals.
 * Sweeps stay queued back to back: two instances of each captured sweep
 * alternate and one instance's events are read before its next launch.
 * qcd_get_profile fills ms[QCD_PROF_N] (total milliseconds) and
 * launches[QCD_PROF_N]; it synchronizes the stream. */
#define QCD_PROF_HEATBATH 0
#define QCD_PROF_OVERRELAX 1
#define QCD_PROF_REUNIT 2
#define QCD_PROF_MEASURE 3
#define QCD_PROF_N 4
int qcd_set_profiling(qcd_lattice *lat, int enable);
int qcd_get_profile(qcd_lattice *lat, double *ms, unsigned long long *launches);

/* Allocation-free measurement.  The paper has no counterpart: this entry point
 * exists for callers that cannot let the library allocate device memory, such
 * as code running inside a host framework that owns all device memory through
 * its own pool (an extra cudaMalloc would fail under the pool's cap or
 * synchronize the device mid-stream), or code that must have no allocation
 * failure path.  It computes what qcd_measure computes, on link storage the
 * caller already holds on the device, and calls no cudaMalloc, cudaFree or
 * allocating library routine.
 *   links       device pointer to the library's storage layout for (group,
 *               precision, Ns, Nt): the bytes qcd_copy_links_out produces.  Read
 *               only; owned by the caller.
 *   link_bytes  its size, as qcd_link_bytes reports it for the lattice it came
 *               from.  The padding of each link array differs between lattices
 *               made by qcd_lattice_create and by qcd_lattice_create_split, and
 *               is read off this size; a size that is not 8 x (vectors per
 *               link) arrays of at least Ns^3 Nt / 2 16-byte vectors is
 *               QCD_ERR_INVALID_ARG.
 *   flux, flux8 flux quanta of the background field (effective links U B), as
 *               given to qcd_lattice_create_ex (flux8 != 0 needs group 3).  For
 *               the storage of a lattice in the frozen field mode pass 0 and 0:
 *               its measurements use the links as stored.
 *   plaquette   host double[3] {P, P_s, P_t} or NULL;
 *   polyakov    host double[2] {Re L, Im L} or NULL.
 *   stream      cudaStream_t or NULL; the call synchronizes it.
 * Scratch: one file-scope device array of QCD_NOALLOC_SCRATCH_BYTES (512 KiB)
 * per GPU that loads the library, held until the process exits.  A lattice
 * needs 16 (ceil(V/256) + ceil(Ns^3/256)) bytes of block partials plus
 * at most 96 Ns + 320 bytes; every lattice of at most 4,194,304 sites (such as
 * 64^3 x 16) fits, a lattice that needs more returns QCD_ERR_INVALID_ARG with
 * the sizes in qcd_last_error().  The first call on a device looks up the
 * array's device address (with that device current) and keeps it; make that
 * first call before any stream capture.  The address belongs to the device's
 * CUDA context, so after a cudaDeviceReset of that device (which also ends
 * every lattice of this library on it) the call must not be used again in the
 * same process.  Every call on a device shares the array and overwrites what
 * the previous call left there (nothing in it needs to start at zero), so calls
 * that overlap on the GPU (different streams, or different host threads) race
 * and must not be issued. */
#define QCD_NOALLOC_SCRATCH_BYTES (512u * 1024u)
int qcd_measure_noalloc(const void *links, size_t link_bytes, int group,
                        int precision, int Ns, int Nt, int flux, int flux8,
                        double *plaquette, double *polyakov, void *stream);

/* ------------------------------------------------------------------------
 * Batched parameter scan.  The paper runs parameter scans as independent jobs
 * handed out by its dispatcher (sec. 4; its fastest mode, sec. 5); here many
 * independent SU(2) lattices of uneven sizes, each with its own beta and flux,
 * are swept together by one persistent cooperative kernel launch captured in
 * a CUDA graph.  Each lattice gets a group of CTAs in proportion to its
 * volume and synchronises only within that group; waits are bounded.
 * Lattice i uses Philox key (seed_lo ^ i * 0x9E3779B9, seed_hi): the same
 * random numbers as a single lattice created with lattice_id i.
 * ------------------------------------------------------------------------ */
typedef struct qcd_batch qcd_batch;

/* n lattices: Ns[i], Nt[i] even >= 2, beta[i] >= 0, flux[i]; group must be 2
 * (QCD_ERR_NOT_SUPPORTED otherwise); precision and start as for
 * qcd_lattice_create.  Each lattice has fewer than 2^29 sites (FP32) or 2^31
 * (FP64), else QCD_ERR_INVALID_ARG.  Arrays are host memory, read during the
 * call. */
int qcd_batch_create(qcd_batch **out, int n, int group, const int *Ns,
                     const int *Nt, const double *beta, const int *flux,
                     int precision, int start, uint64_t seed, void *stream);
int qcd_batch_destroy(qcd_batch *b);

/* n_sweeps sweeps of every lattice (each: 1 heat-bath pass, n_overrelax
 * overrelaxation passes, FP64 reunitarization, measurement) in one launch
 * per wave (see qcd_batch_set_wave_bytes; one launch when the links fit L2).
 * meas_out: host double[n][n_sweeps][5] = {P, P_s, P_t, Re L, Im L} after each
 * sweep, or NULL.  The first call chooses the launch shape (autotune over 128,
 * 256, 512 threads per CTA on a scratch copy).  Returns QCD_ERR_TIMEOUT if a
 * group's barrier wait ran out (the sweep is then abandoned part-way).
 * Synchronizes the stream. */
int qcd_batch_sweep(qcd_batch *b, int n_sweeps, int n_overrelax, uint64_t seed,
                    double *meas_out);
/* Links of lattice `index` in the canonical FP64 host layout. */
int qcd_batch_get_links(qcd_batch *b, int index, double *host_out);
int qcd_batch_set_links(qcd_batch *b, int index, const double *host_in);
int qcd_batch_get_sweep(qcd_batch *b, uint32_t *sweep);
int qcd_batch_link_bytes(const qcd_batch *b, size_t *bytes);
/* Launch shape: threads per CTA (0 = autotune, or 64 / 128 / 256 / 512) and the
 * resulting number of CTAs. */
int qcd_batch_set_block(qcd_batch *b, int threads);
int qcd_batch_get_shape(qcd_batch *b, int *threads, int *ctas);
/* Waves.  A scan whose links outgrow L2 is swept in waves of consecutive
 * lattices whose links fit `bytes` (default: the device's L2 size, 0 = one
 * wave): each wave is one persistent launch that runs all the sweeps of the
 * call on its lattices, so their links stay in L2 across the sweeps; the
 * waves run one after another.  The lattices are independent, so the links
 * are the same for any wave size; the measurement sums of a lattice follow
 * its CTA group's size (equal to rounding).  get returns the number of waves
 * and the budget. */
int qcd_batch_set_wave_bytes(qcd_batch *b, size_t bytes);
int qcd_batch_get_waves(qcd_batch *b, int *waves, size_t *bytes);
/* Bound of every barrier wait, in seconds (default 2, at most 60). */
int qcd_batch_set_wait(qcd_batch *b, double seconds);
/* Test hook: lattice `lattice`'s barriers wait for one arrival that never
 * comes, so the wait runs out and qcd_batch_sweep returns QCD_ERR_TIMEOUT;
 * -1 switches it off. */
int qcd_batch_inject_stall(qcd_batch *b, int lattice);

/* ------------------------------------------------------------------------
 * O(N) model (sec. 3.3 "SUNCL and ONCL Modules": an N-vector field on the
 * sites, checkerboard updates by an improved Metropolis algorithm; sec. 4,
 * Table 1: O(4) with NHIT = 100 tries per site).  The paper gives no formula;
 * readings:
 *   action  S = sum_x [ -2 kappa sum_mu phi_x.phi_{x+mu} + phi_x.phi_x
 *                       + lambda (phi_x.phi_x - 1)^2 ],  phi_x in R^N;
 *   update  a visit of a site makes nhit Metropolis hits with the eight
 *           neighbours fixed: hit h proposes phi' = phi + delta (2u - 1) per
 *           component (Philox block (s, sweep, 3 << 4, h)) and accepts iff
 *           dS <= 0 or u < exp(-dS), u = word h mod 4 of block
 *           (s, sweep, 4 << 4, h / 4); key = (seed_lo, seed_hi);
 *   sweep   even sites, then odd sites; the sweep counter advances once.
 * Field storage on the device: one 16-byte vector per site (FP32 float4 or
 * FP64 two double2), even/odd halves; canonical host order [s][c], N doubles
 * per site, s = x + Ns (y + Ns (z + Ns t)).
 * ------------------------------------------------------------------------ */
typedef struct qcd_on qcd_on;

/* N in 1..4; Ns, Nt even >= 2, Ns^3 Nt < 2^31; delta > 0; precision
 * QCD_FP64_PLAIN (FP64 field and arithmetic) or QCD_FP32_COMPRESSED (FP32
 * field and arithmetic, FP64 sums in measurements); start QCD_COLD
 * (phi = (1, 0, .., 0)) or QCD_HOT (phi_c = 2u - 1 from Philox block
 * (s, 0xFFFFFFFF, 2 << 4, 0)).  nhit defaults to 100.  Allocates the field
 * (32 B per site FP32, 64 B FP64) and a few KB on the current device. */
int qcd_on_create(qcd_on **out, int N, int Ns, int Nt, double kappa,
                  double lambda, double delta, int precision, int start,
                  uint64_t seed, void *stream);
int qcd_on_destroy(qcd_on *m);
int qcd_on_set_nhit(qcd_on *m, int nhit);
/* Threads per block of the phase kernel: 64, 128 (default), 256 or 512. */
int qcd_on_set_block(qcd_on *m, int threads);
/* n_sweeps sweeps (one CUDA graph per sweep: even phase, odd phase, counter
 * advance); seed is the Philox key of the call.  Stream-ordered. */
int qcd_on_sweep(qcd_on *m, int n_sweeps, uint64_t seed);
/* One checkerboard phase at the current sweep counter (no advance). */
int qcd_on_phase(qcd_on *m, int parity, uint64_t seed);
/* out[7] (host) = { <phi.phi>, (1/4V) sum_{x,mu} phi_x.phi_{x+mu}, |M|,
 * M_0, M_1, M_2, M_3 },  M = (1/V) sum_x phi_x; FP64 sums in a fixed order.
 * Synchronizes the stream. */
int qcd_on_measure(qcd_on *m, double *out);
/* Field in the canonical FP64 host layout (V N doubles); set rounds to the
 * storage precision. */
int qcd_on_get_field(qcd_on *m, double *host_out);
int qcd_on_set_field(qcd_on *m, const double *host_in);
int qcd_on_get_sweep(qcd_on *m, uint32_t *sweep);
int qcd_on_set_sweep(qcd_on *m, uint32_t sweep);
/* Accepted Metropolis hits since creation. */
int qcd_on_get_accepted(qcd_on *m, unsigned long long *accepted);

/* Measured FP64 arithmetic rate of the current device, for the roofline of
 * the FP64-plain sweep (sec. 5 compares single and double precision; on this
 * GPU the FP64 path is bound by the FP64 pipe, not by memory).  A kernel of
 * independent FP64 fused multiply-add chains filling every SM is timed with
 * CUDA events on `stream` (best of five launches after one warm-up);
 * *flops_per_s receives 2 flops per FMA over that time.  Changes no clock or
 * other device setting; synchronizes the stream. */
int qcd_probe_fp64_rate(double *flops_per_s, void *stream);

/* Message of the last failed call on this thread ("" if none). */
const char *qcd_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
