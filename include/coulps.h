/*
 * coulps — lattice path-integral Coulomb energy sampler for one GB300 GPU.
 *
 * The method (Sugihara, Higo & Nakamura, JPSJ 2014): the N-body Coulomb energy
 * Eq. (s1) is written, through the two-point function of a free scalar field
 * (Eqs. (2body), (path)), as the lattice expectation value Eq. (nsum)
 *
 *     E_N ~ < (sum_i q_i phi_{n_i})^2 - sum_i (q_i phi_{n_i})^2 >,
 *
 * taken under exp(-H_L), H_L = 1/2 sum_<m,n> (phi_m - phi_n)^2 (Eq. (proplat)),
 * with phi = 0 outside the box (the paper's open-boundary modification of
 * Eq. (phi)).  The expectation is estimated by Markov-chain Monte Carlo:
 * heatbath updates Eq. (phi), optionally over-relaxation reflections, and the
 * sample mean Eq. (nsum2).
 *
 * Conventions for every entry point:
 *   - Return value: COULPS_OK (0) or a negative status below.  No C++
 *     exception ever crosses this interface.  On error nothing is left half
 *     done unless the description says otherwise.
 *   - Sites are 0-based (x, y, z) with 0 <= x < Lx etc.; x is the fastest
 *     index of every natural-order host array, i.e. element x + Lx*(y + Ly*z).
 *   - The library owns every device buffer it allocates.  Device memory comes
 *     from the allocator installed with coulps_set_allocator (for example a
 *     framework's caching allocator) or, by default, from cudaMallocAsync on
 *     the handle's stream.  Host pointers passed in are only read or written
 *     during the call; the caller keeps ownership.
 *   - Work is queued asynchronously on the handle's CUDA stream unless a call
 *     says it synchronises.  Device-side failures (a timed-out wait, a
 *     non-finite sample) are recorded in a per-lattice error word and reported
 *     by the next synchronising call.
 *   - A handle must not be used from two host threads at once.
 *   - One GPU per process (several processes for several GPUs): each kernel's
 *     shared-memory size and per-SM occupancy are set up once, for the device
 *     current at its first launch, and are not repeated for another device.
 */
#ifndef COULPS_H
#define COULPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define COULPS_OK 0
#define COULPS_EINVAL (-1)       /* bad argument (sizes, pointers, ranges)      */
#define COULPS_ENOMEM (-2)       /* device or host allocation failed            */
#define COULPS_ECUDA (-3)        /* a CUDA runtime call failed                  */
#define COULPS_ETIMEOUT (-4)     /* a device-side bounded wait gave up          */
#define COULPS_ENONFINITE (-5)   /* a sample or running sum became non-finite   */
#define COULPS_EIO (-6)          /* checkpoint file could not be read/written   */
#define COULPS_ECORRUPT (-7)     /* checkpoint checksum / header mismatch       */
#define COULPS_EUNSUPPORTED (-8) /* shape or mode the library does not handle   */

#define COULPS_F32 0 /* field and sweeps in FP32, estimator sums in FP64 */
#define COULPS_F64 1 /* field, sweeps and estimator in FP64              */

typedef struct coulps_lattice *coulps_lattice_t;
typedef struct coulps_charges *coulps_charges_t;

/* Human-readable text for a status code (static storage, never NULL). */
const char *coulps_error_string(int status);

/* Library version as 10000*major + 100*minor + patch. */
int coulps_version(void);

/* ---- device memory ----------------------------------------------------- */
/* Allocation hooks.  alloc(bytes, stream, ctx) returns device memory usable on
 * `stream` or NULL; free(ptr, stream, ctx) releases it.  Passing two NULLs
 * restores the default (cudaMallocAsync / cudaFreeAsync).  Affects handles
 * created afterwards; each handle remembers the hooks it was created with. */
typedef void *(*coulps_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*coulps_free_fn)(void *ptr, void *stream, void *ctx);
int coulps_set_allocator(coulps_alloc_fn alloc, coulps_free_fn free_fn, void *ctx);

/* ---- lattice ----------------------------------------------------------- */
/* Create n_chains independent Markov chains of the field phi on an
 * Lx x Ly x Lz box (Eq. (proplat)'s lattice, phi = 0 outside), cold start
 * phi = 0, on the current CUDA device.
 *   precision: COULPS_F32 or COULPS_F64.
 *   seed:      Philox key (low word, high word) of every random draw.
 *   stream:    cudaStream_t to queue work on (NULL = legacy default stream).
 * Limits: 1 <= Lx <= 512, 1 <= Ly, Lz <= 65535, 1 <= n_chains <= 65535,
 * and the quad index (z*Ly + y)*ceil(Lx/8) must fit in 32 bits.  Two copies
 * of the field are allocated (fused passes, see coulps_set_fused).
 * Errors: EINVAL, ENOMEM, ECUDA. */
int coulps_lattice_create(int Lx, int Ly, int Lz, int n_chains, int precision,
                          uint64_t seed, void *stream, coulps_lattice_t *out);

/* Release a lattice (queues the frees on its stream).  NULL is ignored.
 * Charge sets created on it must be destroyed first. */
void coulps_lattice_destroy(coulps_lattice_t lat);

/* Change the stream later work is queued on. */
int coulps_set_stream(coulps_lattice_t lat, void *stream);

/* info[0..12] = Lx, Ly, Lz, n_chains, precision, row stride W (elements),
 * pass counter, device bytes held, tile rows TY, slab depth DZ, fused-pass
 * mode (0, 1, 2), fused-pass tile rows, fused-pass slab depth. */
int coulps_lattice_info(coulps_lattice_t lat, int64_t info[13]);

/* Tile shape of the half-sweep kernel: ty rows of y per CTA, dz planes of z
 * per CTA (0 = keep).  Used by the autotuner; results do not depend on it.
 * Errors: EINVAL (ty*W/4 > 256 threads, ty < 1, dz < 1). */
int coulps_set_tile(coulps_lattice_t lat, int ty, int dz);

/* Copy chain `chain`'s field to / from a host array of Lx*Ly*Lz doubles in
 * natural order.  Synchronises the stream.  field_set does not change the
 * pass counter.  Errors: EINVAL, ECUDA, and any recorded device error. */
int coulps_field_get(coulps_lattice_t lat, int chain, double *host_xyz);
int coulps_field_set(coulps_lattice_t lat, int chain, const double *host_xyz);

/* n_compound compound sweeps on every chain.  A compound sweep is n_hb
 * heatbath passes (Eq. (phi) at every site) followed by n_or over-relaxation
 * passes (phi -> S/3 - phi, S the sum of the six neighbours); a pass is the
 * red half-sweep ((x+y+z) even) then the black one.  Each pass advances the
 * pass counter by one; heatbath pass p of chain k draws its uniforms from
 * Philox4x32-10 with counter (quad, p, k, colour).  Asynchronous.
 * Errors: EINVAL (negative counts), ECUDA. */
int coulps_sweep(coulps_lattice_t lat, int n_compound, int n_hb, int n_or);

/* Wait for the lattice's stream and report any recorded device error. */
int coulps_sync(coulps_lattice_t lat);

/* Failure detection.  Every wait inside the library's kernels (mbarrier
 * phases of the TMA rings) is bounded by %globaltimer time; a wait that
 * gives up records COULPS_ETIMEOUT in the lattice's error word, lets its
 * copies in flight land and returns, so the context stays usable and the
 * next coulps_sync / coulps_estimate reports the error.  The word stays set
 * (the fields may be partly updated) until coulps_clear_error, typically after
 * restoring a checkpoint.
 * coulps_selftest_wait queues, on the lattice's stream, a kernel that waits
 * for a flag nothing sets and gives up after limit_ns (1 us .. 1 s) exactly
 * like those waits: it exercises the failure path without touching the
 * fields.  Errors: EINVAL, ECUDA. */
int coulps_selftest_wait(coulps_lattice_t lat, int64_t limit_ns);
int coulps_clear_error(coulps_lattice_t lat);

/* ---- charge sets and the estimator ------------------------------------- */
/* Register n point charges q[i] at sites site_xyz[3i..3i+2] of lattice `lat`
 * (copied; the arrays are the caller's).  All chains of the lattice are
 * measured against this set.  Coincident sites are allowed.  log_capacity
 * samples of (Q, P, e) per chain are kept on the device for
 * coulps_samples (0 = keep none).  Errors: EINVAL (site outside the box,
 * n < 0, non-finite q), EUNSUPPORTED (a chain's field holds more than 2^32
 * elements: sites are kept as 32-bit offsets), ENOMEM, ECUDA. */
int coulps_charges_create(coulps_lattice_t lat, int64_t n, const int32_t *site_xyz,
                          const double *q, int64_t log_capacity, coulps_charges_t *out);

void coulps_charges_destroy(coulps_charges_t ch);

/* Take one sample per chain of the current fields (one term of Eq. (nsum2)):
 *   Q = sum_i q_i phi(r_i),  P = sum_i (q_i phi(r_i))^2,  e = Q^2 - P,
 * Q and P summed in FP64 in a fixed order (bitwise reproducible), e formed in
 * FP64; then update the per-chain running sums of e and e^2 and the batch
 * sums.  Asynchronous.  Errors: EINVAL (charges of another lattice), ECUDA. */
int coulps_measure(coulps_lattice_t lat, coulps_charges_t ch);

/* n_therm unmeasured compound sweeps, then n_meas measured ones, each
 * followed by one sample per chain as coulps_measure takes it.  In the
 * measured sweeps the sample is gathered by the last half-sweep itself (the
 * charge gather fused into the sweep); the per-CTA partial sums are then
 * added in a fixed order.  The measured loop is captured once into a CUDA
 * graph and replayed (not on the legacy default stream, nor while profiling).  Asynchronous.  Errors: EINVAL, ECUDA. */
int coulps_run(coulps_lattice_t lat, coulps_charges_t ch, int n_therm, int n_meas,
               int n_hb, int n_or);

/* Synchronise and return the estimate of E_N pooled over all chains:
 *   mean      = sum of all samples / their number (Eq. (nsum2)),
 *   stderr_bm = batch-means standard error (chains give independent batches;
 *               the batch length doubles as samples accumulate so that
 *               between 32 and 64 batches per chain are kept),
 *   tau_int   = integrated autocorrelation time in samples, from the ratio of
 *               the batch-mean variance to the per-sample variance,
 *   n         = number of samples (all chains).
 * Any pointer may be NULL.  Errors: ECUDA, ETIMEOUT, ENONFINITE. */
int coulps_estimate(coulps_charges_t ch, double *mean, double *stderr_bm, double *tau_int,
                    int64_t *n);

/* Pipelined estimates, for callers that read a result after every step
 * without stalling the GPU on each read.  coulps_estimate_post queues, on the
 * lattice's stream, a copy of the estimator state and of the lattice's error
 * word as they will be after everything queued so far, into one of two
 * pinned slots the set owns; it returns at once.  coulps_estimate_take waits
 * for the oldest posted copy and returns what coulps_estimate would have
 * returned at that point (the same pooling, and ETIMEOUT / ENONFINITE if the
 * error word was set then).  At most two posts may be outstanding (EINVAL
 * otherwise); take without an outstanding post is EINVAL.  A loop of
 * (queue step k; post; take the result of step k - 1) keeps the next step
 * queued while the host pools the last one.  Errors: EINVAL, ENOMEM (first
 * post), ECUDA, ETIMEOUT, ENONFINITE (take). */
int coulps_estimate_post(coulps_charges_t ch);
int coulps_estimate_take(coulps_charges_t ch, double *mean, double *stderr_bm, double *tau_int,
                         int64_t *n);

/* Synchronise and copy the logged samples: QPe[(s*n_chains + k)*3 + {0,1,2}]
 * = (Q, P, e) of sample s of chain k, for s < min(samples taken, cap,
 * log_capacity).  *n receives the number of samples copied per chain. */
int coulps_samples(coulps_charges_t ch, double *QPe, int64_t cap, int64_t *n);

/* Forget all samples (running sums, batches and log). Asynchronous. */
int coulps_reset_stats(coulps_charges_t ch);

/* Several charge sets on the same samples.  A sample of the field does not
 * depend on where the charges sit (the paper's argument for reusing one
 * sample set), so any number of charge sets of one lattice can be measured
 * on every sample: coulps_measure_sets takes one sample of every set from the
 * current fields (one gather launch and one finalize launch per 32 sets);
 * coulps_run_sets runs n_therm unmeasured and n_meas measured compound
 * sweeps, each measured one followed by a sample of every set (captured once
 * per call as a CUDA graph when n_meas >= 4).  Each set keeps its own
 * statistics and log (coulps_estimate etc. per set).  Asynchronous.
 * Errors: EINVAL (no sets, a set of another lattice), ECUDA. */
int coulps_measure_sets(coulps_lattice_t lat, const coulps_charges_t *sets, int n_sets);
int coulps_run_sets(coulps_lattice_t lat, const coulps_charges_t *sets, int n_sets, int n_therm,
                    int n_meas, int n_hb, int n_or);

/* Replace the positions and values of the ch's n charges (same n as at
 * creation) from host arrays, asynchronously: the arrays are converted and
 * staged in library-owned pinned memory before the call returns, so the
 * caller may reuse them at once.  Running sums are kept.  Errors: EINVAL
 * (site outside the box, non-finite q), ECUDA. */
int coulps_charges_update(coulps_charges_t ch, const int32_t *site_xyz, const double *q);

/* Off-lattice charges (the paper's closing remarks: a particle between sites
 * is modelled through the eight sites around it, and forces follow by the
 * same interpolation).  Particle i sits at pos_xyz[3i..3i+2] (doubles,
 * 0 <= x <= Lx - 1 etc.; every dimension of the lattice >= 2) with charge
 * q[i].  With base b = floor(r) clipped to L - 2 and f = r - b, the eight
 * corners b + c (c in {0,1}^3) carry the trilinear weights
 *   w_c = prod_mu (c_mu ? f_mu : 1 - f_mu),
 * so a sample reads phi~_i = sum_c w_c phi(b + c) and takes, as Eq. (nsum2)
 * does for lattice charges, Q = sum_i q_i phi~_i, P = sum_i (q_i phi~_i)^2,
 * e = Q^2 - P (all in FP64; mean = sum_{i != j} q_i q_j G~(r_i, r_j) with the
 * interpolated Green function).  With forces != 0 every sample also adds, per
 * chain and particle,
 *   f_i = -de/dr_i = -2 q_i (Q - q_i phi~_i) grad phi~_i,
 *   grad phi~_i = sum_c (grad w_c) phi(b + c),
 * to running sums (the measure does not depend on the positions, so their
 * mean is the force on particle i).  Weights and gradients are formed once
 * on the host in FP64.  The set works with coulps_measure, coulps_run (the
 * gather is a separate launch after the sweep), coulps_measure_sets,
 * coulps_run_sets, coulps_estimate, coulps_samples, coulps_chain_stats and
 * coulps_reset_stats (which also clears the force sums); coulps_charges_update
 * and coulps_gcv_create return EUNSUPPORTED.  Errors: EINVAL (a position
 * outside the box or not finite, a dimension < 2, non-finite q, n < 0),
 * EUNSUPPORTED (a chain's field holds more than 2^32 elements), ENOMEM,
 * ECUDA. */
int coulps_charges_create_off(coulps_lattice_t lat, int64_t n, const double *pos_xyz,
                              const double *q, int64_t log_capacity, int forces,
                              coulps_charges_t *out);

/* Near-field direct correction of an off-lattice set (the paper's closing
 * remarks: close particles are better computed directly than through the
 * lattice, whose Green function misses the steep core of the potential).
 * The near set N = {(i, j): i < j, |r_i - r_j| < rc} is fixed by this call
 * (rc = 0: none).  From then on every sample leaves N's pairs out,
 *   s_N = 2 sum_{(i,j) in N} q_i q_j phi~_i phi~_j,
 *   P -> P + s_N, e = Q^2 - P - s_N  (the logged P includes s_N),
 * and, with forces on, f_i = -2 q_i (Q - q_i phi~_i - sum_{j near i} q_j
 * phi~_j) grad phi~_i; the pairs come back with the continuum kernel of
 * Eq. (s1), returned here in FP64:
 *   *e_direct = 2 sum_{(i,j) in N} q_i q_j / (4 pi r_ij),
 *   f_direct[3i + mu] = 2 q_i sum_{j near i} q_j (r_i - r_j)_mu / (4 pi r_ij^3)
 * (any of the three outputs may be NULL; f_direct holds 3 n doubles).  The
 * energy is then coulps_estimate's mean + *e_direct and the force
 * coulps_forces' mean + f_direct.  Pairs are found on the host by a cell grid;
 * the list is kept on the device as CSR (both directions, ascending).
 * Synchronises; drops the set's samples, force sums and captured graphs.
 * Errors: EINVAL (rc < 0 or not finite), EUNSUPPORTED (not an off-lattice
 * set), ENOMEM, ECUDA. */
int coulps_charges_near(coulps_charges_t ch, double rc, int64_t *n_pairs, double *e_direct,
                        double *f_direct);

/* Pure host helpers behind coulps_charges_create_off and coulps_charges_near
 * (no device, no lattice; host arrays owned by the caller).
 * coulps_near_pairs: for n particles at pos_xyz, the near partners
 * (|r_i - r_j| < rc, j != i) as CSR, both directions, each list ascending:
 * ptr[0..n] and nbr[0..ptr[n]).  *n_entries always receives ptr[n]; if it
 * exceeds cap (nbr may then be NULL) nothing else is written and EINVAL is
 * returned, so a first call with cap = 0 sizes the array.
 * coulps_offlattice_corners: for each particle its eight corner sites
 * (c = 4 cx + 2 cy + cz, base site floor(r) clipped to L - 2) as offsets in
 * one chain's field of a lattice of this shape and precision
 * (colour * colour_elems + (z * Ly + y) * W + x / 2, the layout of
 * coulps_field_get's storage), their trilinear weights (8 n doubles) and
 * weight gradients (24 n doubles, [8 i + c][mu]).
 * Errors: EINVAL (bad sizes or pointers, non-finite or out-of-box positions,
 * a dimension < 2), ENOMEM. */
int coulps_near_pairs(int64_t n, const double *pos_xyz, double rc, int64_t *ptr, uint32_t *nbr,
                      int64_t cap, int64_t *n_entries);
int coulps_offlattice_corners(int Lx, int Ly, int Lz, int precision, int64_t n,
                              const double *pos_xyz, uint32_t *offset, double *weight,
                              double *grad);

/* Synchronise and return the mean force on each particle of an off-lattice
 * set created with forces != 0: mean[3i + mu] = (sum over all chains' samples
 * of f_i,mu) / (number of samples), and, if stderr_chains is not NULL, the
 * standard error from the spread of the chains' own means (chains are
 * independent).  Errors: EINVAL, EUNSUPPORTED (not an off-lattice set with
 * forces), ECUDA, ETIMEOUT. */
int coulps_forces(coulps_charges_t ch, double *mean, double *stderr_chains);

/* Per-chain estimator state, COULPS_STAT_STRIDE doubles per chain:
 *   [0] samples n, [1] sum e, [2] sum e^2, [3] open batch sum, [4] open batch
 *   count, [5] batch length b, [6] completed batches m (32 <= m < 64 once
 *   n >= 32 b), [7] the most recent sample e, [8 + j] sum of e over completed
 *   batch j.
 * coulps_chain_stats synchronises and copies n_chains rows into out (cap =
 * doubles available).  coulps_pool_stats is pure host arithmetic: it pools
 * any number of such rows (for example gathered from several processes, each
 * running its own chains with its own seed) exactly as coulps_estimate does,
 * summing in row order.  Rows must share one batch length.  Errors: EINVAL. */
#define COULPS_STAT_STRIDE 72
int coulps_chain_stats(coulps_charges_t ch, double *out, int64_t cap);
int coulps_pool_stats(const double *stats, int64_t n_rows, double *mean, double *stderr_bm,
                      double *tau_int, int64_t *n);

/* ---- schedule of the measured phase ------------------------------------ */
/* COULPS_SCHEDULE_ALIGNED (default): every chain does the same kind of pass in
 * the same launch.  COULPS_SCHEDULE_PHASED: in coulps_run's measured phase
 * (n_hb > 0, n_or > 0, n_hb + n_or <= 8, n_meas >= 2, n_chains >= n_hb + n_or),
 * chain k is delayed by k mod (n_hb + n_or) passes, so each launch mixes
 * heatbath tiles (ALU-bound) of some chains with over-relaxation tiles
 * (memory-bound) of the others.  Every chain does exactly the same passes,
 * Philox draws and samples as with the aligned schedule (results are
 * bitwise identical); only the order across chains changes. */
/* Several streams (n = 2 .. 4): every compound sweep runs chain k on stream
 * k % n, stream 0 being the lattice's and the others the library's own,
 * forked from the lattice's stream at the start of the sweep and joined back
 * at its end (also inside captured graphs), so that the groups' heatbath
 * (instruction-bound) and over-relaxation (memory-bound) kernels can run at
 * the same time.  Every chain's passes, Philox draws and samples are
 * unchanged (bitwise identical results); all work still completes in order
 * on the lattice's stream.  n = 1 (default): one stream.  At most n_chains
 * streams are used.  Not used by the phased schedule.
 * Errors: EINVAL, ECUDA. */
int coulps_set_streams(coulps_lattice_t lat, int n);

/* COULPS_SCHEDULE_SHIFTED: with two streams (coulps_set_streams(lat, 2)),
 * fused modes 1 and 3, n_hb >= 1 and n_or >= 1, coulps_run's measured phase
 * (n_meas >= 2, on-lattice charge set) runs the odd chains half a compound
 * sweep behind the even ones: a prologue (even chains: the first sweep; odd
 * chains: its heatbath passes), n_meas - 1 steady steps (even: the next
 * sweep; odd: the over-relaxation passes and sample of their previous sweep,
 * then the heatbath passes of the next), an epilogue (odd: the rest of their
 * last sweep), each captured as a CUDA graph.  One group's heatbath
 * half-sweeps then run beside the other's over-relaxation kernels.  Every
 * chain does exactly the passes, Philox draws and samples of the aligned
 * schedule (bitwise identical results); after the call all chains have
 * finished the same sweeps.  Otherwise it runs as ALIGNED. */
#define COULPS_SCHEDULE_ALIGNED 0
#define COULPS_SCHEDULE_PHASED 1
#define COULPS_SCHEDULE_SHIFTED 2
int coulps_set_schedule(coulps_lattice_t lat, int schedule);

/* Fused passes.  A fused pass (both half-sweeps) runs as one kernel that
 * reads the field once and writes it once (8 bytes per site in FP32 instead
 * of 12 for over-relaxation), from the field into a second copy of it or
 * back: the lattice then holds two copies (twice the field memory).  Within
 * a compound sweep one block of consecutive passes is fused, and the sweep
 * starts and ends in the lattice's field: enable = 1 fuses the
 * over-relaxation passes (all of them when n_or is even or n_hb >= 1: with
 * an odd n_or the first heatbath pass writes the second copy, at no extra
 * traffic, and the fused block ends in the field; all but the last when
 * n_or is odd and n_hb = 0), enable = 2 all passes (an even number of them),
 * enable = 3 (default) over-relaxation pass pairs: two consecutive passes in one
 * kernel that reads the field once and writes it once for both (4 bytes per
 * site and pass in FP32); the heatbath passes run as half-sweeps, the
 * over-relaxation passes as n_or / 2 pairs and n_or mod 2 single fused
 * passes (an odd number of these kernels after a heatbath pass: that pass
 * writes the second copy as in enable = 1; with no heatbath pass one pair
 * becomes two single passes, and a lone pass runs as half-sweeps).
 * enable = 4 all passes as pairs, heatbath ones included, followed by single
 * fused passes so that the number of kernels is even (n = 1 pass: two
 * half-sweeps; n mod 4 = 0: n / 2 pairs; 1: (n - 3) / 2 pairs + 3 singles;
 * 2: n / 2 - 1 pairs + 2 singles; 3: (n - 1) / 2 pairs + 1 single).  Rows
 * too wide for a pair CTA (fewer than 4 rows fit) run enable = 3 as 1 and
 * 4 as 2.  enable = 0 none (and frees the second copy).  Results are bitwise those of
 * the half-sweep path (same arithmetic per site, same Philox counters).  The
 * sample of a measured compound sweep is gathered by its last kernel.  Not
 * used by the phased schedule.  coulps_set_pass_tile: ty rows of y per CTA
 * (the CTA also computes one halo row each side: (ty + 2) * W / 4 threads
 * <= 512), dz planes of z per CTA (0 = keep).  Errors: EINVAL, ENOMEM,
 * ECUDA. */
int coulps_set_fused(coulps_lattice_t lat, int enable);
int coulps_set_pass_tile(coulps_lattice_t lat, int ty, int dz);

/* Pass-pair tile (enable = 3, 4): ty rows of y per CTA, which also computes
 * three halo rows each side ((ty + 6) * W / 4 threads <= 512 in FP32, 256 in
 * FP64; ty + 8 <= 256; shared memory within 227 KiB), dz planes of z per CTA
 * (0 = keep).  coulps_pair_tile writes the current (ty, dz), (0, 0) when the
 * lattice has no pair tile.  Errors: EINVAL. */
int coulps_set_pair_tile(coulps_lattice_t lat, int ty, int dz);
int coulps_pair_tile(coulps_lattice_t lat, int32_t out[2]);

/* ---- kernel timing ----------------------------------------------------- */
/* With profiling on, every half-sweep and fused pass launched by
 * coulps_sweep (and by coulps_run, which then launches directly instead of
 * replaying its graph) is bracketed by CUDA events on the stream it runs on
 * (the lattice's, or with coulps_set_streams the chain group's; launches of
 * different groups then overlap, so their durations do not isolate one
 * kernel: time kernels on one stream).  coulps_kernel_times
 * synchronises and returns, since profiling was enabled or last read:
 *   out[0] total ms of heatbath half-sweeps, out[1] their count,
 *   out[2] total ms of over-relaxation half-sweeps, out[3] their count,
 *   out[4] total ms of mixed half-sweeps (phased schedule), out[5] their count,
 *   out[6] total ms of fused heatbath passes, out[7] their count,
 *   out[8] total ms of fused over-relaxation passes, out[9] their count,
 * and restarts the accumulation.  coulps_kernel_times_n writes the first n
 * of these and further kinds, zero past the last one:
 *   out[10] total ms of pass pairs with a heatbath pass, out[11] their count,
 *   out[12] total ms of over-relaxation pass pairs, out[13] their count. */
int coulps_set_profiling(coulps_lattice_t lat, int enable);
int coulps_kernel_times(coulps_lattice_t lat, double out[10]);
int coulps_kernel_times_n(coulps_lattice_t lat, double *out, int n);

/* ---- checkpoint -------------------------------------------------------- */
/* Save / restore the full sampler state: fields of all chains, the pass
 * counter, seed and shape, and (if ch != NULL) the estimator state of the
 * charge set (statistics, sample log, control-variate statistics and, for an
 * off-lattice set with forces, the force sums), with a checksum.  Restoring
 * then continuing gives bitwise the same samples as an uninterrupted run.
 * The charge set itself (sites or positions, near pairs) is not stored: load
 * into a set created the same way.  Files of the first format (no
 * control-variate state or force sums) still load.  Synchronises.
 * Errors: EIO, ECORRUPT (checksum or shape mismatch, or force sums present in
 * only one of file and set), ECUDA. */
int coulps_checkpoint_save(coulps_lattice_t lat, coulps_charges_t ch, const char *path);
int coulps_checkpoint_load(coulps_lattice_t lat, coulps_charges_t ch, const char *path);

/* ---- many independent systems ----------------------------------------- */
/* A batch holds n_systems independent lattices of (possibly) different
 * shapes, each with one chain and its own charge set and estimator, and
 * sweeps them all with one launch per half-sweep: a persistent grid walks a
 * work list of (system, y tile, z slab) tiles.  System s uses Philox counter
 * word 2 = s (its "chain" id), so each system reproduces a one-chain lattice
 * with that chain id.  Storage, boundary, update rules and estimator are those
 * of the lattice API above; the measured compound sweep gathers Q, P in its
 * last kernel and is replayed as one CUDA graph.  By default the
 * over-relaxation passes run as pass pairs (coulps_batch_set_fused). */
typedef struct coulps_batch *coulps_batch_t;

/* dims[3s..3s+2] = (Lx, Ly, Lz) of system s, limits as coulps_lattice_create.
 * Errors: EINVAL, ENOMEM, ECUDA. */
int coulps_batch_create(int n_systems, const int32_t *dims, int precision, uint64_t seed,
                        void *stream, coulps_batch_t *out);
void coulps_batch_destroy(coulps_batch_t b);

/* Tile shape of every system: ty_dz[2s] rows, ty_dz[2s+1] planes (0 = keep).
 * Results do not depend on it.  Errors: EINVAL (more than 256 threads, box
 * rows > 256, shared memory > 227 KiB). */
int coulps_batch_set_tiles(coulps_batch_t b, const int32_t *ty_dz);
int coulps_batch_system_tile(coulps_batch_t b, int system, int32_t *ty_dz);

/* info[0..9] = n_systems, work-list tiles, persistent CTAs, shared memory
 * bytes per CTA, pass counter, field bytes, total sites, fused-pass CTAs,
 * pass-pair CTAs and threads per pair CTA (0 without pass pairs). */
int coulps_batch_info(coulps_batch_t b, int64_t *info);

/* Fused over-relaxation passes, between the fields and a second copy of
 * them (twice the field memory).  enable = 1: the over-relaxation passes of
 * a compound sweep run as fused passes (both half-sweeps of a pass in one
 * z-march, each site read and written once, 8 bytes per site in FP32
 * instead of 12), one persistent launch per pass over a list of pass tiles.
 * enable = 2 (the default when every system admits a pair tile): they run
 * as pass pairs (two passes in one z-march, 4 bytes per site and pass), one
 * persistent launch per pair over a list of pair tiles, largest first, and
 * a fused pass for an odd remainder.  The heatbath passes stay half-sweeps,
 * written into the second copy when the number of out-of-place kernels is
 * odd (with no heatbath pass, a pair becomes two fused passes, or the last
 * pass runs as half-sweeps); the sweep ends in the fields.  enable = 3: all
 * passes, heatbath ones included, as pass pairs and fused passes (an even
 * number of kernels: by n = n_hb + n_or mod 4, n / 2 pairs; (n - 3) / 2
 * pairs and 3 fused passes; n / 2 - 1 and 2; (n - 1) / 2 and 1; a single
 * pass as half-sweeps).  enable = 0:
 * half-sweeps only (frees the copy).  Results are bitwise those of the
 * half-sweeps in every mode.  EINVAL for enable >= 2 if some system admits no
 * pair tile.
 * Pass tile of every system: ty_dz[2s] rows, ty_dz[2s+1] planes (0 = keep;
 * (ty + 2) * W / 4 <= 256 threads, ty + 4 <= 256, shared memory <= 227 KiB).
 * Pair tile of every system: the same form ((ty + 6) * W / 4 <= 512
 * threads in FP32, 256 in FP64, ty + 8 <= 256, shared memory <= 227 KiB;
 * ty = 0 in coulps_batch_system_pair_tile: no pair tile fits).
 * coulps_batch_fused returns the mode (-1 for a null handle).
 * Errors: EINVAL, ENOMEM, ECUDA. */
int coulps_batch_set_fused(coulps_batch_t b, int enable);
int coulps_batch_fused(coulps_batch_t b);
int coulps_batch_set_pass_tiles(coulps_batch_t b, const int32_t *ty_dz);
int coulps_batch_system_pass_tile(coulps_batch_t b, int system, int32_t *ty_dz);
int coulps_batch_set_pair_tiles(coulps_batch_t b, const int32_t *ty_dz);
int coulps_batch_system_pair_tile(coulps_batch_t b, int system, int32_t *ty_dz);

/* Charges of all systems: those of system s are entries offsets[s] ..
 * offsets[s+1]-1 of site_xyz (3 per charge, inside that system's box) and q.
 * Replaces any previous set and resets the estimators.  log_capacity samples
 * of (Q, P, e) per system are kept.  Errors: EINVAL, ENOMEM, ECUDA. */
int coulps_batch_charges(coulps_batch_t b, const int64_t *offsets, const int32_t *site_xyz,
                         const double *q, int64_t log_capacity);

/* Unmeasured compound sweeps of all systems (asynchronous). */
int coulps_batch_sweep(coulps_batch_t b, int n_compound, int n_hb, int n_or);

/* n_therm unmeasured then n_meas measured compound sweeps of all systems.
 * Errors: EINVAL (no charges, or a measured sweep with no pass), ECUDA. */
int coulps_batch_run(coulps_batch_t b, int n_therm, int n_meas, int n_hb, int n_or);

int coulps_batch_sync(coulps_batch_t b);

/* Per-system estimates (arrays of n_systems; any pointer may be NULL), as
 * coulps_estimate for a one-chain lattice.  Synchronises. */
int coulps_batch_estimate(coulps_batch_t b, double *mean, double *stderr_bm, double *tau_int,
                          int64_t *n);

/* Logged samples: QPe[(k*n_systems + s)*3 + {0,1,2}] = (Q, P, e) of sample k
 * of system s, for k < min(samples, cap, log_capacity).  Synchronises. */
int coulps_batch_samples(coulps_batch_t b, double *QPe, int64_t cap, int64_t *n);

/* System s's field as Lx*Ly*Lz doubles in natural order.  Synchronises. */
int coulps_batch_field_get(coulps_batch_t b, int system, double *host_xyz);
/* Sets system s's field from host_xyz (natural order x fastest, Lx Ly Lz
 * doubles; rounded to the precision).  Synchronises. */
int coulps_batch_field_set(coulps_batch_t b, int system, const double *host_xyz);
/* Raw per-system statistics of the plain samples: out[s * COULPS_STAT_STRIDE
 * + k] as coulps_chain_stats (cap >= n_systems * COULPS_STAT_STRIDE);
 * coulps_batch_reset_stats clears them (asynchronous).  Errors: EINVAL, ECUDA. */
int coulps_batch_stats(coulps_batch_t b, double *out, int64_t cap);
int coulps_batch_reset_stats(coulps_batch_t b);

/* ---- global control variate of every system of a batch ---------------- */
/* Not in the paper.  The control variate of coulps_gcv_create for each
 * system s of a batch: g = Q_s h_s (h_s = -G rho_s by n_iter red/black SOR
 * iterations of the system's box, rounded so that A h_s is exact in FP32),
 * plus for R in 1..4 the local term of P; T g = h_s . rho_s - Q_s (A h_s) .
 * phi_s (+ k(0) sum q^2 - sum_i q_i^2 phi_i w_i), mean 0 for any h and kernel.
 * h_s is bitwise the one coulps_gcv_create makes for the same box, charges
 * and n_iter.  create reads the batch's charges (re-create it after
 * coulps_batch_charges) and synchronises; it needs charges (EINVAL).
 * info: out[2 s] = h_s . rho_s, out[2 s + 1] = |A u_s + rho_s| / |rho_s|.
 * h: h_s (FP32, natural order) of one system.  eval: T g of every system's
 * current field into tg (device, n_systems doubles; NULL = internal),
 * asynchronous.  run: n_meas measured compound sweeps of all systems (one
 * CUDA graph each on a non-default stream), each recording the plain sample
 * (coulps_batch_estimate) and e - c T g per system (coulps_batch_gcv_estimate,
 * raw sums by coulps_batch_gcv_stats, cleared by coulps_batch_gcv_reset).
 * Errors: EINVAL, ENOMEM, ECUDA. */
typedef struct coulps_batch_gcv *coulps_batch_gcv_t;
int coulps_batch_gcv_create(coulps_batch_t b, int n_iter, int R, coulps_batch_gcv_t *out);
void coulps_batch_gcv_destroy(coulps_batch_gcv_t g);
int coulps_batch_gcv_info(coulps_batch_gcv_t g, double *out);
int coulps_batch_gcv_h(coulps_batch_gcv_t g, int system, float *host_xyz);
int coulps_batch_gcv_eval(coulps_batch_gcv_t g, double *tg);
int coulps_batch_gcv_run(coulps_batch_gcv_t g, int n_meas, int n_hb, int n_or, double c);
int coulps_batch_gcv_reset(coulps_batch_gcv_t g);
int coulps_batch_gcv_stats(coulps_batch_gcv_t g, double *out, int64_t cap);
int coulps_batch_gcv_estimate(coulps_batch_gcv_t g, double *mean, double *stderr_bm,
                              double *tau_int, int64_t *n);

/* ---- Stein control variate kernels -------------------------------------- */
/* Building blocks of the learned control variate (not in the paper): a small
 * 3D conv net g(phi) whose Stein term sum_x (dg_x/dphi_x - g_x (A phi)_x) has
 * zero mean under exp(-H_L) (integration by parts; A phi = grad H_L).
 *
 * coulps_cv_pack_weights (host only): PyTorch conv3d weights w[co][ci][kz][ky][kx]
 * (16 x 16 x 3 x 3 x 3 floats) -> 27 x 256 BF16 (round to nearest even) in the
 * order coulps_cv_conv3d reads them.
 *
 * coulps_cv_conv3d: h = conv3d(a, w) + bias, 3x3x3, zero padding, 16 -> 16
 * channels, on the tensor cores (BF16 operands, FP32 accumulation).
 *   in_bf16 device [nb][Lz][Ly][Lx][16] BF16, channels last (16-byte aligned)
 *   wpack   device, the 27 x 256 BF16 of coulps_cv_pack_weights
 *   bias    device, 16 floats;  out device [nb][Lz][Ly][Lx][16] FP32
 *   x_period 0, or P > 0: the output columns x with x % P == P - 1 are set to
 *           0 (the gutters of the interleaved box layout, see
 *           coulps_cv_pack_region, stay 0 from layer to layer)
 *   err     device int; a timed-out wait ORs COULPS_ERR bit 1 into it
 * Asynchronous on stream.  Errors: EINVAL, ECUDA. */
int coulps_cv_pack_weights(const float *w, uint16_t *wpack);
int coulps_cv_conv3d(const void *in_bf16, const void *wpack, const float *bias, float *out,
                     int nb, int Lx, int Ly, int Lz, int x_period, int *err, void *stream);
/* Same convolution with the activation fused into its epilogue: writes
 * a = tanh(h) and s = 1 - a^2 as BF16 [nb][Lz][Ly][Lx][16] (16-byte aligned);
 * gutter columns get a = 0, s = 1. */
int coulps_cv_conv3d_tanh(const void *in_bf16, const void *wpack, const float *bias,
                          void *a_bf16, void *s_bf16, int nb, int Lx, int Ly, int Lz,
                          int x_period, int *err, void *stream);
/* The same for the output rows y in [y0, y1) and planes z in [z0, z1) only
 * (all x of them; the input is read one row and one plane around them, zero
 * outside the box).  Other outputs are not written.  For layers whose
 * consumers read only part of the box, such as the region terms below.
 * Errors: EINVAL (an empty or out-of-box range), ECUDA. */
int coulps_cv_conv3d_tanh_rows(const void *in_bf16, const void *wpack, const float *bias,
                               void *a_bf16, void *s_bf16, int nb, int Lx, int Ly, int Lz,
                               int x_period, int y0, int y1, int z0, int z1, int *err,
                               void *stream);

/* coulps_cv_conv3d_wgrad: weight gradient of coulps_cv_conv3d,
 *   dW[co][ci][o] = sum_{b, p} dh[b, p, co] a[b, p + o, ci]   (a = 0 outside),
 * o = 9 kz + 3 ky + kx, i.e. dW has PyTorch's [co][ci][kz][ky][kx] order.
 * a, dh: device BF16 [nb][Lz][Ly][Lx][16]; dW device 16*16*27 floats;
 * scratch: device, >= min(1024, ceil(T / 32)) * 27 * 256 floats, T = nb*Lz*Ly*ceil(Lx/64).
 * Summed in a fixed order (reproducible).  Asynchronous. */
int coulps_cv_conv3d_wgrad(const void *a_bf16, const void *dh_bf16, float *dW, int nb, int Lx,
                           int Ly, int Lz, float *scratch, int64_t scratch_floats, void *stream);

/* coulps_cv_pack_field: the net's input for every chain of an FP32 lattice,
 * on the lattice's stream: act[chain][z][y][x][16] BF16 = (phi, rho, rho phi,
 * 0, ...) and Aphi[chain][z][y][x] = (A phi) = 6 phi - (sum of the six neighbours),
 * phi = 0 outside the box (the gradient of H_L).  rho: device Lz*Ly*Lx floats
 * (charge density per site).  act must be 16-byte aligned.
 * coulps_cv_activate: a = tanh(h), s = 1 - a^2 (BF16) for n floats h. */
int coulps_cv_pack_field(coulps_lattice_t lat, const float *rho, void *act_bf16, float *Aphi);
int coulps_cv_activate(const float *h, void *a_bf16, void *s_bf16, int64_t n, void *stream);
/* coulps_cv_pack_region: the same for the sub-box E = [origin, origin + dims)
 * (x, y, z order) of every chain, in E's own coordinates; A phi is taken from
 * the full field (neighbours outside E but inside the box count).  interleave
 * 0: act[chain][ez][ey][ex][16], Aphi[chain][ez][ey][ex].  interleave 1: the
 * chains' boxes side by side along x, each followed by one zero column:
 * act[ez][ey][chain][ex + 1][16], Aphi likewise, i.e. one lattice of
 * n_chains (ex + 1) x ey x ez sites on which coulps_cv_conv3d with
 * x_period = ex + 1 and nb = 1 convolves every box with its own zero padding
 * (the small boxes then fill the tensor-core tiles).  rho is the full
 * box's density.  Errors: EINVAL (E not inside the box), EUNSUPPORTED (FP64). */
int coulps_cv_pack_region(coulps_lattice_t lat, const float *rho, const int32_t *origin,
                          const int32_t *dims, int interleave, void *act_bf16, float *Aphi);

/* coulps_cv_stein_sum: per chain b, the Stein term of the net,
 *   out[b] = sum_x (dg_x/dphi_x - g_x (A phi)_x)
 *          = sum_q sum_c s2[c, q] D[c, q] - sum_x g_x Aphi_x
 *            + sum_{q on a face} sum_c2 s2[c2, q] sum_{c1, e} dK_b(q)[c2][c1][e] s1[c1, q + e]
 * with D = conv(s1, K) (coulps_cv_conv3d with the divergence kernel K), g =
 * channel 0 of g16 ([b][site][16] FP32), s1, s2 BF16 [b][site][16], and dK
 * (device, 64 x 16 x 16 x 27 floats) the face corrections indexed by
 * class b = cx + 4 cy + 16 cz, c = 0 low face, 1 inside, 2 high face, 3 both
 * (edge 1).  Sums in FP64, fixed order.  scratch: >= 128 * nb doubles.  out:
 * device nb doubles. */
int coulps_cv_stein_sum(const float *g16, const float *D, const void *s2_bf16, const float *Aphi,
                        const void *s1_bf16, const float *dK, int nb, int Lx, int Ly, int Lz,
                        double *scratch, int64_t scratch_doubles, double *out, void *stream);

/* coulps_cv_region_pack: the class kernels of coulps_cv_stein_region in the
 * form its tensor-core kernel reads them, formed once per set of weights.
 * Ktab (device, 216 x 27 x 16 x 16 floats, 16-byte aligned:
 * K[class][e][c2][c1]) holds one divergence kernel per class ix + 6 iy + 36 iz
 * (see below); kpack (device, 216 x 41472 bytes, 16-byte aligned) receives,
 * per class, K split into three BF16 parts K = hi + mid + lo (each part the
 * BF16 rounding of what the parts before it leave; together they hold K's
 * FP32 value), stored as the tensor core's K-major operand without swizzle:
 * the byte of row n = 16 p + c2 (part p), channel c1 and offset e at
 * e 1536 + (n / 8) 128 + (c1 / 8) 768 + (n % 8) 16 + (c1 % 8) 2.
 * Asynchronous on stream.  Errors: EINVAL, ECUDA. */
int coulps_cv_region_pack(const float *Ktab, void *kpack, void *stream);

/* coulps_cv_stein_region: the Stein term of a net g that is kept inside the
 * box R = [lo, hi) and set to 0 elsewhere (still a smooth field of phi, so the
 * term keeps mean 0), evaluated on a sub-box E (edims = x, y, z sizes) that
 * holds R and its 3-site halo, with R in E's coordinates:
 *   out[b] = sum_{q in R+1} sum_c2 s2[c2, q] sum_{c1, e} K_q[c2][c1][e] s1[c1, q + e]
 *            - sum_{x in R} g_x Aphi_x
 * where K_q is the divergence kernel summed over the offsets f of the last
 * layer with q - f inside R (per axis a subset of {-1, 0, 1}).  One K per
 * class ix + 6 iy + 36 iz, the per-axis index of the allowed set {-1} 0,
 * {0} 1, {-1, 0} 2, {1} 3, {0, 1} 4, {-1, 0, 1} 5 (f = -1 is bit 0), given as
 * kpack, the output of coulps_cv_region_pack.  g_x, the net's output, is
 * formed at the sites of R from the second layer's activations a2 (BF16
 * [b][E][16], 16-byte aligned, 0 outside E as in the convs' zero padding)
 * and the last layer: w3g (device, 27 x 16 floats [o][ci], o = 9 kz + 3 ky +
 * kx, the weights of PyTorch layout W3[0][ci][kz][ky][kx], as the tensor-core
 * convs use them: BF16 values) and bias b3g, summed in FP32.  s1, s2 BF16
 * [b][E][16] (16-byte aligned), Aphi [b][E], all in the layout `interleave`
 * of coulps_cv_pack_region (gutters are not read).  The
 * sums over c1 and e run on the tensor cores (tcgen05, BF16 operands, K in its
 * three parts, FP32 accumulation): one FP32 value per (chain, site); the sums
 * over sites are FP64 in a fixed order.  scratch >= nb * (|(R + 1) within E|
 * + |R|) doubles; out device nb doubles (overwritten); err: device int, as for
 * coulps_cv_conv3d (a bounded wait for the tensor cores or their copies that
 * gave up ORs bit 1 into it and leaves out unspecified).  Asynchronous.
 * Errors: EINVAL, ECUDA. */
int coulps_cv_stein_region(const void *a2_bf16, const float *w3g, float b3g,
                           const void *s1_bf16, const void *s2_bf16,
                           const float *Aphi, const void *kpack, int nb, const int32_t *edims,
                           int interleave, const int32_t *lo, const int32_t *hi, double *scratch,
                           int64_t scratch_doubles, double *out, int *err, void *stream);

/* coulps_cv_charge_term: the part of the divergence that comes through the
 * net's third input channel rho phi (coulps_cv_pack_field writes
 * act = (phi, rho, rho phi, 0, ...)), which the kernels above leave out:
 *   out[b] += sum_k rho_k sum_p sum_c2 s2[c2, x_k + f_p]
 *                         sum_c1 M[p][c2][c1] s1[c1, x_k + f_p + e_p]
 * with M[p][c2][c1] = W3[c2][f_p] W2[c2][c1][e_p] W1[c1][2][-(f_p + e_p)]
 * over the 343 pairs p = 49 az + 7 ay + ax, per axis a = 0..6 standing for
 * (f, e) = (-1,0) (-1,1) (0,-1) (0,0) (0,1) (1,-1) (1,0); positions outside
 * the box (edims = x, y, z sizes) count as 0.  q_xyz (device, n_q x 3
 * int32, inside the box, box coordinates) and q_rho (device, n_q floats) are
 * the charge sites whose g is kept (all of them, or those inside R for
 * coulps_cv_stein_region) and their density.  M device 343 x 16 x 16 floats;
 * s1, s2 in the layout `interleave` (s1, s2 and M 16-byte aligned).  The sum
 * over the 7 pairs of one (ay, az) class is FP32 per chain and charge; those
 * 49 n_q partials are summed in FP64, charges in order.  scratch >= 49 * nb *
 * n_q doubles.  Asynchronous.
 * Errors: EINVAL, ECUDA. */
int coulps_cv_charge_term(const void *s1_bf16, const void *s2_bf16, const float *M,
                          const int32_t *q_xyz, const float *q_rho, int n_q, int nb,
                          const int32_t *edims, int interleave, double *scratch,
                          int64_t scratch_doubles, double *out, void *stream);

/* Control-variate estimator, kept beside the plain one of a charge set:
 * coulps_cv_record adds to chain b's CV statistics the sample
 *   y_b = e_b - c * tg[b],
 * e_b the chain's most recent Eq. (nsum2) sample (stat [7]) and tg device
 * n_chains doubles (for example coulps_cv_stein_region's out).  Call it after
 * each measurement whose field tg was computed from.  coulps_cv_chain_stats,
 * coulps_cv_estimate and coulps_cv_reset mirror coulps_chain_stats,
 * coulps_estimate and coulps_reset_stats for these samples (same layout, same
 * pooling).  Checkpoints do not hold them.  Asynchronous except the readers. */
int coulps_cv_record(coulps_charges_t ch, const double *tg, double c);
int coulps_cv_chain_stats(coulps_charges_t ch, double *out, int64_t cap);
int coulps_cv_estimate(coulps_charges_t ch, double *mean, double *stderr_bm, double *tau_int,
                       int64_t *n);
int coulps_cv_reset(coulps_charges_t ch);

/* ---- global control variate ------------------------------------------- */
/* Not in the paper.  g_x = Q(phi) h_x with Q = sum_i q_i phi(r_i) and a fixed
 * field h of the charge set: its Stein term
 *   T g = h . rho - Q (A h) . phi            (rho = charge density)
 * has mean 0 under exp(-H_L) for any h, and with h = -G rho it equals
 * Q^2 - rho.G.rho, which removes from e = Q^2 - P all of its variance except
 * that of P.  coulps_gcv_create solves A u = -rho by n_iter red/black SOR
 * iterations (FP64, the optimal factor of the box) on the lattice's stream,
 * rounds u to the fixed-point grid 2^-k with 13 max|u| 2^k < 2^24 (h), so
 * that v = A h is exact in FP32 (kept in the field's layout) and h . rho is
 * formed in FP64: E[T g] = 0 holds for the h actually used.  Per sample
 * v . phi adds FP32 products in FP32 over 16 sites and those in FP64.
 * R in 1..4 adds the local term of P: g^P_x = sum_i q_i^2 phi(r_i) k(x - r_i)
 * with k the Dirichlet Green function of the (2R+1)^3 cube at its centre
 * (FP32), whose Stein term k(0) sum q^2 - sum_i q_i^2 phi(r_i) w_i,
 * w_i = sum_d k(d) (A phi)(r_i + d), also has mean 0 and removes most of the
 * variance of P; T g then denotes the sum of both terms.  R = 0: Q term only.
 * Synchronises.  The object reads the charge set's positions at creation
 * (re-create it after coulps_charges_update; destroy it before the set).
 * coulps_gcv_info: out[0] = h . rho, out[1] = |A u + rho| / |rho| (synchronises).
 * coulps_gcv_h: h (fp32) in natural order (synchronises).
 * coulps_gcv_eval: per chain T g of the current fields into tg (device,
 *   n_chains doubles; NULL = internal buffer); asynchronous.
 * coulps_gcv_run: n_meas measured compound sweeps; each records the plain
 *   Eq. (nsum2) sample and the control-variate sample e - c T g
 *   (coulps_cv_estimate reads the latter).  Synchronises at the end.
 * Errors: EINVAL, ENOMEM, ECUDA. */
typedef struct coulps_gcv *coulps_gcv_t;
int coulps_gcv_create(coulps_charges_t ch, int n_iter, int R, coulps_gcv_t *out);
void coulps_gcv_destroy(coulps_gcv_t gcv);
int coulps_gcv_info(coulps_gcv_t gcv, double out[2]);
int coulps_gcv_h(coulps_gcv_t gcv, float *host_xyz);
int coulps_gcv_eval(coulps_gcv_t gcv, double *tg);
int coulps_gcv_run(coulps_gcv_t gcv, int n_meas, int n_hb, int n_or, double c);

/* ---- allocation-free measurement --------------------------------------- */
/* The paper has no counterpart to this entry point.  It serves callers that
 * cannot allocate device memory when they measure: code running while a CUDA
 * stream is being captured (cudaMalloc is not allowed there), real-time or
 * embedded controllers that forbid allocation after start-up, and plugins
 * whose host application has reserved all device memory.  It computes, for
 * each of n_chains fields the caller owns, the same (Q, P, e) as
 * coulps_measure, and allocates nothing: no cudaMalloc, no cudaFree, no
 * allocating library call.  Its only working memory is a file-scope device
 * array of COULPS_STATIC_SCRATCH_DOUBLES doubles (512 KiB) and a one-word
 * counter of out-of-range offsets (cleared by each call) that every GPU
 * loading this library holds until the process exits.
 *   field      device pointer to n_chains fields in the library's storage
 *              layout: field[chain][colour][z][y][h] with colour (x+y+z)&1,
 *              h = x>>1, row stride W = 4*ceil(Lx/8) rounded up to a
 *              multiple of 8 (FP32) or 4 (FP64) elements, every other element
 *              0; one chain is 2*Lz*Ly*W elements (float or double by
 *              precision).  This is the layout coulps_lattice_create uses.
 *   site_index device pointer to n uint32 offsets within one chain's field:
 *              colour*(Lz*Ly*W) + (z*Ly + y)*W + (x>>1).  An offset of
 *              2*Lz*Ly*W or more is not read: it makes every chain's
 *              (Q, P, e) NaN.
 *   q          device pointer to n doubles.
 *   QPe        device pointer to 3*n_chains doubles, written as
 *              (Q, P, e) of chain k at QPe[3k..3k+2], bitwise the values
 *              coulps_measure gives for the same fields and charges.
 *   stream     cudaStream_t the work is queued on (asynchronous); it must
 *              belong to the current device (EINVAL otherwise; checked when
 *              the stream is not being captured into a graph).
 * Limit: n_chains * b * 2 <= COULPS_STATIC_SCRATCH_DOUBLES, where
 * b = min(64, max(1, ceil(n / 1024))) CTAs per chain; e.g. any n with up to
 * 512 chains, or up to 32768 chains when n <= 1024.  Larger requests return
 * COULPS_EINVAL and queue nothing.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  All calls share the one array and it keeps the
 * last call's contents; every slot a call reads is first written by that same
 * call, so nothing needs clearing, but calls that overlap on the GPU (for
 * example on two streams at once) race on it and must be serialised by the
 * caller.  A device reset while the library is loaded is not supported.
 * Errors: EINVAL, ECUDA, EUNSUPPORTED (device ordinal >= 64). */
#define COULPS_STATIC_SCRATCH_DOUBLES 65536
int coulps_measure_static(const void *field, int Lx, int Ly, int Lz, int n_chains, int precision,
                          const uint32_t *site_index, const double *q, int64_t n, double *QPe,
                          void *stream);

/* The random term of the heatbath update Eq. (phi), exactly as the sweep
 * kernels form it: out[i] = -erfc^-1(2 r_i) / sqrt(3) with
 * r_i = (w[i] + 1/2) 2^-32, for n 32-bit words w (device arrays; out holds
 * floats for COULPS_F32, doubles for COULPS_F64).  FP64 uses CUDA's erfcinv;
 * FP32 uses the library's own erfc^-1 (polynomials in Giles' variable, in
 * base 2: v = -log2(u (2 - u)), with both u and 1 - u formed from the
 * integer word), a few FP32 ulps from the exact value.  Asynchronous on `stream`.
 * Errors: EINVAL (bad precision, NULL arrays with n > 0), ECUDA. */
int coulps_heatbath_noise(int precision, const uint32_t *w, void *out, int64_t n, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* COULPS_H */
