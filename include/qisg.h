/*
 * qisg.h -- C ABI of the GB300 library for the MCQSG hot path: checkerboard
 * Metropolis sweeps plus parallel tempering for the 2D +-J quantum Ising spin
 * glass in Trotter-Suzuki form (an L x L x L_tau classical Ising prism).
 *
 * Paper: "The QISG suite: high-performance codes for studying Quantum Ising
 * Spin Glasses" (Bernaschi, Gonzalez-Adalid Pemartin, Martin-Mayor, Parisi).
 *   Sec. 1, Eq. (2)-(3)   the classical model: p(S) ~ exp(-k E(S)), E sums the
 *                         spatial bonds J S S and the imaginary-time bonds S S.
 *                         Here each ladder slot carries its own (k, k_tau)
 *                         with exp(-2 k_tau) = tanh(k Gamma); k_tau = k is the
 *                         paper's equal-coupling case.
 *   Sec. 2.1              red/blue checkerboard Metropolis with precomputed
 *                         Metropolis factors; multispin coding; parallel
 *                         tempering with P = min(1, exp((k_a-k_b)(E_a-E_b))).
 *   Sec. 2.1.1            counter-based Philox4x32-10 random numbers, one
 *                         counter per clone, reproducible for any work split.
 *   Appendix A            EMCS = ptfr sweeps + one PT update; an online energy
 *                         measurement every mesfr EMCS.
 *   Appendix E.1          the replica overlap q.
 *
 * Conventions (all entry points):
 *   - Return 0 (QISG_OK) or a negative QISG_E* code; qisg_last_error() gives
 *     a message for the calling thread's most recent failure.
 *   - Host arrays are owned by the caller; sizes are stated per call.  The
 *     handle owns all device memory it allocates.
 *   - Work is stream-ordered on opts.cuda_stream (a cudaStream_t; NULL means
 *     the legacy default stream).  Getters synchronise that stream.
 *   - A handle must not be used from two threads at once.
 *   - Sites are indexed site = x + L*y + L*L*tau; colour (x+y+tau) mod 2;
 *     red (0) is updated first.  Samples a, replicas r, ladder slots s,
 *     walkers w (walker w starts at slot w).
 *   - Results depend only on (L, L_tau, ladder, n_replicas, n_samples, seed,
 *     sweep count, pt_every), never on the packing, word width or schedule.
 */
#ifndef QISG_H
#define QISG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QISG_OK        0
#define QISG_EINVAL   (-1)   /* bad argument (see each call)                  */
#define QISG_ENOMEM   (-2)   /* device allocation failed or over mem_budget   */
#define QISG_ECUDA    (-3)   /* a CUDA call failed                            */
#define QISG_ETIMEOUT (-4)   /* a bounded device wait expired                 */
#define QISG_ECORRUPT (-5)   /* a state buffer failed its consistency check   */
#define QISG_ESTATE   (-6)   /* call not valid in the current state           */

/* Packings of independent systems into one word (Sec. 2.1, multispin coding).
 * LANES: a word holds the n_replicas x n_slots systems of ONE sample (lane =
 *   replica-in-word * n_slots + walker); every lane draws its own random
 *   number; PT swaps the slot labels, not the spins (Sec. 2.1).
 * SAMPLES: a word holds 32 or 64 SAMPLES at one (replica, slot); the draw of
 *   a (replica, slot, site, sweep) is shared by the 64 samples of a sample
 *   block, as in Ito-Kanada's multi-sample coding (Sec. 2.1.1); PT moves the
 *   spin bits of each sample between slot words.
 * SITES: the paper's own multi-site coding with its update rule (Sec. 2.1,
 *   Sec. 2.1.1, Appendices B and C): a 32-bit word holds 32 imaginary-time
 *   sites of ONE system (site (x, y, tau) is bit tau / M of word-site
 *   x + L y + L^2 (tau mod M), M = L_tau / 32), and a site with u of its 6
 *   bonds unsatisfied flips iff u + d >= 3, d its two-bit daemon, whose
 *   bits come from Philox4x32-10 + one xoroshiro128++ state step + the
 *   inverse-cumulative bytes of Sec. 2.1.1 (the words b4, b8, b12 of
 *   word-site ws of system (a, r, slot s) in sweep t: Philox counter
 *   {ws, t, s | r << 16, 5 << 28 | which << 24 | a}, which = 0, 1, 2).  This
 *   is a different Markov chain from the threshold rule of LANES and
 *   SAMPLES (the same distribution, another random stream).  Needs word_bits
 *   0 or 32, k_tau = k <= 16 at every slot (the rule prices a flip with one
 *   coupling), L_tau a multiple of 64 and n_samples < 2^24; never chosen by
 *   AUTO.  PT swaps the slot labels, as in LANES.                          */
#define QISG_LAYOUT_AUTO    0
#define QISG_LAYOUT_LANES   1
#define QISG_LAYOUT_SAMPLES 2
#define QISG_LAYOUT_SITES   3

typedef struct qisg_handle qisg_handle;

/* One ladder slot: spatial coupling k and imaginary-time coupling k_tau. */
typedef struct {
    double k;
    double k_tau;
} qisg_slot;

typedef struct {
    int word_bits;          /* 32 | 64; 0 = choose                                */
    void *cuda_stream;      /* cudaStream_t, NULL = legacy default stream          */
    size_t mem_budget;      /* bytes of device memory the handle may take; 0 = any */
    int pt_every;           /* sweeps per PT pass (the paper's ptfr); 0 = never    */
    int measure_every;      /* sweeps per measurement (mesfr); 0 = never           */
    int layout;             /* QISG_LAYOUT_*                                       */
    int per_sample_launch;  /* LANES only: 1 = one kernel launch per sample per
                               half sweep (the plain per-instance form)            */
    int tau_antiperiodic;   /* 1 = antiperiodic boundary along tau (Sec. 1: the
                               bond from tau = L_tau-1 to tau = 0 counts -S S in
                               B); 0 = periodic                                    */
    int history_len;        /* PT walk history (Appendix A's history_betas): keep
                               the slot of every walker at the last history_len
                               measurements; 0 = none                              */
    int maxit;              /* measurements per block average (Appendix A); 0 =
                               none                                                */
    int blocks_len;         /* block sums kept when maxit > 0 (>= 1)               */
} qisg_opts;

/* Fill *opts with defaults: word_bits 0, NULL stream, no budget, pt_every 1,
 * measure_every 0, layout AUTO, per_sample_launch 0, tau_antiperiodic 0,
 * no walk history, no block sums. */
void qisg_opts_default(qisg_opts *opts);

/* Linear ladder (k_s = lo + (hi-lo) s/(n-1), both ends included; k_s = lo for
 * n = 1) with k_tau,s = -1/2 log tanh(k_s Gamma), the separate-coupling form
 * of Sec. 1's relation between k and Gamma.  out: caller array of n slots.
 * EINVAL: n < 1, gamma <= 0, lo <= 0 or a non-finite k_tau. */
int qisg_ladder_linear(double lo, double hi, int n, double gamma, qisg_slot *out);

/* The tables of the SITES daemon rule for coupling k (Sec. 2.1.1, Appendix
 * C), computed on the host: cum[0..254] = cumulative(n), the truncation of
 * 2^64 sum_{m <= n} p^pop(m) (1-p)^(8-pop(m)) with p = e^{-4k} (fixed point
 * with 126 fractional bits; the paper uses 128-bit floats); lut (NULL =
 * skip): 2^lut_bits entries, entry h = n_min | (n_max - n_min) << 8, where
 * [n_min, n_max] holds n* of every 64-bit word whose top lut_bits bits are
 * h.  The caller owns both arrays (255 and 2^lut_bits entries).  EINVAL:
 * k outside [0, 16], cum NULL, lut_bits outside 1..16. */
int qisg_daemon_tables(double k, int lut_bits, uint64_t *cum, uint16_t *lut);

/* Create an instance: n_samples disorder samples (J = +-1, p = 1/2), each
 * with n_replicas independent replicas of an n_slots PT ladder, on an
 * L x L x L_tau prism periodic in all three directions (Sec. 1, Sec. 2.1).
 * Couplings and the start configuration are drawn from Philox under `seed`
 * (the paper's separate J / start / Monte Carlo seeds, Appendix A, become
 * counter domains).  Walker w starts at slot w.  The uint32 Metropolis table
 * and the PT bases are built once here, on the host, in FP64 (Sec. 2.1:
 * Metropolis factors precomputed for every possible value).
 *   ladder: host array of n_slots slots (copied).  opts may be NULL.
 * EINVAL: L odd or < 2; L_tau odd or < 2; n_slots < 1; n_replicas < 1;
 *   n_samples < 1; a k or k_tau negative or non-finite; a packing that cannot
 *   hold the systems (LANES needs n_slots <= word bits and n_replicas <=
 *   2 * (word bits / n_slots); SAMPLES needs n_slots <= 32).
 * ENOMEM: allocation failed or the state exceeds opts->mem_budget.        */
int qisg_create(qisg_handle **out, int L, int L_tau, const qisg_slot *ladder, int n_slots,
                int n_replicas, int64_t n_samples, uint64_t seed, const qisg_opts *opts);

/* Run n_sweeps sweeps.  Sweep t (0-based count of sweeps done before it):
 * red half sweep, blue half sweep (the blue pass also counts the integer
 * energies of every system), then a PT pass when pt_every > 0 and
 * (t+1) % pt_every == 0, then a measurement when measure_every > 0 and
 * (t+1) % measure_every == 0 (Appendix A's EMCS cadence).  Asynchronous.
 * EINVAL: n_sweeps < 0.                                                     */
int qisg_sweep(qisg_handle *h, int64_t n_sweeps);

/* One explicit PT pass on the current configurations (Sec. 2.1), drawing the
 * numbers a PT pass after the last completed sweep would draw, so that
 * pt_every = 0 plus one qisg_pt_swap per sweep reproduces pt_every = 1.
 * ESTATE: no sweep has run yet.                                             */
int qisg_pt_swap(qisg_handle *h);

/* Integer energies of the configurations now at each slot, by slot:
 * A = sum over spatial bonds of J S S, B = sum over tau bonds of S S
 * (Eq. (3): -E = A + B at k_tau = k).  A, B: host int64
 * [n_samples][n_replicas][n_slots].  Synchronises.                          */
int qisg_energies(qisg_handle *h, int64_t *A, int64_t *B);

/* Replica overlaps of the configurations now at each slot (Appendix E.1):
 * q[a][s][p] = sum_i S^{r1}_i S^{r2}_i over pairs p = (r1 < r2) in
 * lexicographic order.  q: host int64 [n_samples][n_slots][n_pairs],
 * n_pairs = n_replicas (n_replicas-1) / 2.  Synchronises.
 * Limits: the LANES and SITES overlap kernels keep one 8-byte counter per
 * pair in shared memory (48 KB), so they take n_replicas <= 111; beyond
 * that this call and the cadenced measurement return QISG_ECUDA.  The
 * SAMPLES packing takes up to 65535 (word group, slot, pair) sets (EINVAL
 * beyond).                                                               */
int qisg_overlaps(qisg_handle *h, int64_t *q);

/* PT permutation: walker_at[a][r][s] = walker now at slot s.  Host int32
 * [n_samples][n_replicas][n_slots].  Synchronises.                        */
int qisg_permutation(qisg_handle *h, int32_t *walker_at);

/* Unpacked +-1 spins of samples a_lo .. a_lo+n_a-1, by walker:
 * S[a - a_lo][r][w][site], host int8, n_a*n_replicas*n_slots*L*L*L_tau
 * bytes.  EINVAL: the sample range is outside [0, n_samples).  Synchronises.
 * Unpacked on the device through a temporary staging buffer of at most
 * 256 MB (or one sample's spins, if larger), allocated outside the memory
 * budget and freed before returning; ENOMEM if it cannot be allocated.    */
int qisg_get_spins(qisg_handle *h, int64_t a_lo, int64_t n_a, int8_t *S);

/* Couplings of samples a_lo .. a_lo+n_a-1: J[a - a_lo][x + L*y][dir], int8
 * +-1, dir 0 = bond to (x+1, y), dir 1 = bond to (x, y+1). */
int qisg_get_couplings(qisg_handle *h, int64_t a_lo, int64_t n_a, int8_t *J);

/* Replace the couplings of every sample (host int8 [n_samples][L*L][2],
 * entries +-1; EINVAL otherwise).  Energies are recomputed. */
int qisg_set_couplings(qisg_handle *h, const int8_t *J);

/* Replace the state: spins by walker (host int8 [n_samples][n_replicas]
 * [n_slots][N], entries +-1), the permutation (host int32
 * [n_samples][n_replicas][n_slots], each row a permutation of 0..n_slots-1)
 * and the sweep counter.  Measurement sums are cleared; energies are
 * recomputed.  Because every draw is a function of the counters, resuming
 * from a saved state is bit-exact with the uninterrupted run.
 * ECORRUPT: a row of walker_at is not a permutation or a spin is not +-1;
 * nothing of the handle changes then.  Packed on the device through a
 * temporary staging buffer, allocated outside the memory budget and freed
 * before returning: in the SAMPLES packing the whole state when it is at
 * most 256 MB (one copy, the +-1 check on the device), else up to 256 MB of
 * one word group's samples at a time (at least one replica's, word_bits *
 * n_slots * N bytes; the check on the host); in the other packings at most
 * 256 MB, or one sample's spins if larger.                                 */
int qisg_set_state(qisg_handle *h, const int8_t *S, const int32_t *walker_at, uint64_t sweep);

/* Test entry: one explicit PT pass (Sec. 2.1) of every chain through the
 * handle's own PT kernel, on integer energies given by the caller instead of
 * the ones counted from its configurations -- so that tests can place the
 * acceptance test u < P wherever they choose (at, just inside and just
 * outside the kernel's float shortcut margin) and compare the permutation
 * with an independent evaluation of the rule.
 *   U          host int64 [n_samples][n_replicas][n_slots][2]: the
 *              unsatisfied spatial and tau bond counts (u_s, u_t) of the
 *              configuration of walker w (last-but-one index), i.e.
 *              A = 2N - 2 u_s and B = N - 2 u_t; only differences enter.
 *   walker_at  host int32 [n_samples][n_replicas][n_slots]: in, the
 *              permutation before the pass; out, the one after it.
 *   t          the pass draws the numbers of a PT pass after sweep t.
 *   wide       0: energy differences in the width the lattice size selects
 *              (32 bits when 2N < 2^30), 1: 64-bit differences.
 * Afterwards the handle's energies and permutation no longer describe its
 * configurations: qisg_sweep and qisg_pt_swap return ESTATE until
 * qisg_set_state.  Synchronises.
 * EINVAL: a count outside [0, 2^38) (or [0, 2^29) with 32-bit differences),
 *   more than 32 slots; ECORRUPT: a row of walker_at is not a permutation. */
int qisg_pt_given(qisg_handle *h, const int64_t *U, int32_t *walker_at, uint64_t t, int wide);

/* Checkpoint files.  The paper writes the configurations at every block of
 * measurements and they serve as backups to restart from (Sec. 2.1,
 * Appendix A); here a checkpoint holds everything a bit-exact resume needs,
 * with a CRC over all of it.  Byte layout (little-endian integers):
 *   offset 0    "QISGCKP1"; u32 version = 1; u32 header bytes = 128
 *          16   i32 L, L_tau, n_slots, n_replicas; i64 n_samples; u64 seed;
 *               u64 sweep; i64 n_meas; i32 pt_every, measure_every,
 *               tau_antiperiodic, rule (0 threshold table, 1 daemon bits);
 *               zeros up to byte 128
 *   then        the ladder, n_slots x (f64 k, f64 k_tau) (IEEE bits)
 *               couplings int8 [n_samples][L*L][2], +-1
 *               spins by walker, one bit each (1 <=> -1), bit i of the
 *                 sequence [n_samples][n_replicas][n_slots][N] at bit
 *                 i % 8 of byte i / 8, padded with zero bits to a byte
 *               walker_at i32 [n_samples][n_replicas][n_slots]
 *               measurement sums i64: sumA, sumB [n_samples][n_replicas]
 *                 [n_slots]; sumq, sumq2 [n_samples][n_slots][n_pairs]
 *   last        u32 CRC-32 (IEEE 802.3: reflected polynomial 0xEDB88320,
 *               initial value and final complement 0xFFFFFFFF) of every
 *               byte before it
 * The walk history and block sums are not stored: after a load they hold
 * the measurements taken from then on. */
typedef struct {
    int L, L_tau, n_slots, n_replicas;
    int64_t n_samples;
    uint64_t seed, sweep;
    int64_t n_meas;
    int pt_every, measure_every, tau_antiperiodic, rule;
} qisg_checkpoint_info;

/* Write the handle's state to `path` (through path.tmp, renamed when
 * complete).  The spins are read back in chunks of at most 256 MB.
 * Synchronises.  EINVAL: the file cannot be written. */
int qisg_checkpoint_save(qisg_handle *h, const char *path);

/* Check a checkpoint file on the host only (no device work): header, sizes
 * and CRC; fills *info (may be NULL).  ECORRUPT: bad magic or version,
 * inconsistent sizes, truncated or extended file, CRC mismatch; EINVAL: the
 * file cannot be opened. */
int qisg_checkpoint_verify(const char *path, qisg_checkpoint_info *info);

/* Resume from a checkpoint: the file is checked first (ECORRUPT as above,
 * before the handle is touched), must describe this handle's problem (same
 * lattice, ladder bits, replicas, samples, seed, cadences, boundary and
 * rule; EINVAL otherwise; any packing or word width), and then replaces the
 * couplings, spins, permutation, sweep counter and measurement sums, so the
 * run continues bit for bit as if uninterrupted.  Unpacks the spins into a
 * host buffer of one byte per spin.  Synchronises. */
int qisg_checkpoint_load(qisg_handle *h, const char *path);

/* Measurement sums since creation (or the last qisg_set_state), by slot:
 *   sumA, sumB  [n_samples][n_replicas][n_slots]  sums of A and B
 *   sumq, sumq2 [n_samples][n_slots][n_pairs]     sums of q and q^2
 *   n_meas      number of measurements taken.
 * Any output pointer may be NULL.  Synchronises.                           */
int qisg_measurements(qisg_handle *h, int64_t *sumA, int64_t *sumB, int64_t *sumq,
                      int64_t *sumq2, int64_t *n_meas);

/* FP64 per-slot means over samples, replicas (pairs) and measurements:
 * e_s[s] = <A>/(2N), e_t[s] = <B>/N, q2[s] = <q^2>/N^2, N = L*L*L_tau;
 * the integer sums are added in the fixed order sample, replica (pair).
 * Host double arrays of n_slots.  ESTATE: no measurement yet.             */
int qisg_slot_means(qisg_handle *h, double *e_s, double *e_t, double *q2);

/* PT walk history (Appendix A: at every measurement the state of the
 * parallel-tempering random walk, i.e. the value of k of every system copy,
 * is collected in history_betas for the equilibration test):
 * slot_of[i][a][r][w] = the ladder slot of walker w of chain (a, r) at
 * measurement first + i (measurements counted from creation or the last
 * qisg_set_state / qisg_checkpoint_load).  Host uint8
 * [n][n_samples][n_replicas][n_slots].  Synchronises.
 * ESTATE: history_len = 0, or a requested measurement is not (yet, or no
 * longer) among the last history_len.                                       */
int qisg_walk_history(qisg_handle *h, int64_t first, int64_t n, uint8_t *slot_of);

/* Block sums (Appendix A: maxit consecutive energy measurements are
 * averaged and written out): sumA[i][a][r][s] and sumB[i][a][r][s], by slot,
 * over the measurements first_block*maxit ... of blocks first .. first+n-1.
 * Host int64 [n][n_samples][n_replicas][n_slots].  Only complete blocks
 * among the last blocks_len are available (ESTATE otherwise, or when
 * maxit = 0).  Synchronises.                                                */
int qisg_block_sums(qisg_handle *h, int64_t first, int64_t n, int64_t *sumA, int64_t *sumB);

/* FP64 block averages per slot: e_s[i][s] = <A>/(2N), e_t[i][s] = <B>/N over
 * the samples, replicas and maxit measurements of block first + i, the
 * integer sums added in the fixed order sample, replica.  Host double
 * [n][n_slots].  Errors as qisg_block_sums.                                 */
int qisg_block_means(qisg_handle *h, int64_t first, int64_t n, double *e_s, double *e_t);

/* Imaginary-time observables (Appendix E.1: the tau-resolved overlaps
 * Q_2(tau), Q_4(tau), F(tau) and the Euclidean correlation C(tau) of the
 * analysis programs), computed on the configurations now at each slot.
 * With q~_x(tau_1, tau) = S_{x,tau_1} S_{x,tau_1+tau} (tau_1 + tau taken
 * modulo L_tau, as the paper does for both boundaries) and
 * Q~(tau_1, tau) = sum_x q~_x, for every sample a_lo .. a_lo+n_a-1,
 * replica r, slot s and lag tau = 0 .. L_tau-1, sums over tau_1:
 *   S1 = sum Q~  (= L^2 L_tau times the site average of C_x(tau))
 *   S2 = sum Q~^2, S4 = sum Q~^4   (L_tau Q_2(tau), L_tau Q_4(tau) of one
 *                                   configuration)
 *   SF = sum (|sum_x e^{i 2pi x_1/L} q~_x|^2 + |sum_x e^{i 2pi x_2/L} q~_x|^2)
 *        (2 L_tau F(tau)); FP64 from the column and row sums of q~, x in
 *        order 0 .. L-1, with a cos / sin table from the host's libm.
 * Averages over measurements and replicas are the caller's.  Host arrays
 * [n_a][n_replicas][n_slots][L_tau] (int64, int64, int64, double).  Spins
 * are unpacked on the device in chunks through a temporary buffer of at
 * most 256 MB (or one sample's spins), allocated outside the memory budget.
 * EINVAL: sample range, L > 32, or 8 L L_tau bytes above 227 KB of shared
 * memory.  Synchronises. */
int qisg_tau_observables(qisg_handle *h, int64_t a_lo, int64_t n_a, int64_t *S1, int64_t *S2, int64_t *S4,
                         double *SF);

/* The uint32 Metropolis table in use: T[s][u_s][u_t] (u_s unsatisfied
 * spatial bonds 0..4, u_t unsatisfied tau bonds 0..2); a spin flips iff
 * T == 0xFFFFFFFF or its draw R < T.  Host uint32 [n_slots][5][3].         */
int qisg_thresholds(qisg_handle *h, uint32_t *T);

/* Sweeps done so far. */
int qisg_sweep_count(qisg_handle *h, uint64_t *t);

/* Layout and word width the handle chose (QISG_LAYOUT_LANES or _SAMPLES). */
int qisg_layout(qisg_handle *h, int *layout, int *word_bits);

/* Kernel launches this handle has issued since creation (diagnostics). */
int qisg_launch_count(qisg_handle *h, int64_t *n);

/* Kernel kinds for qisg_profile_read. */
#define QISG_KERNEL_SWEEP   0   /* the red and blue half-sweep kernels            */
#define QISG_KERNEL_PT      1   /* the PT pass                                    */
#define QISG_KERNEL_MEASURE 2   /* overlaps and measurement sums                  */
#define QISG_KERNEL_PERMUTE 3   /* SAMPLES: moving spin bits after a PT pass       */
#define QISG_KERNEL_BLUE    4   /* read only: the blue half sweeps (in SWEEP too)  */
#define QISG_KERNEL_RED     5   /* read only: the red half sweeps (in SWEEP too)   */

/* Start (enable = 1, counters reset) or stop (0) timing every launch of the
 * kernels above with CUDA events recorded on the handle's stream, around the
 * launch, at most 65536 launches per kind (later launches are counted, not
 * timed).  enable = QISG_PROFILE_ONLY | (1 << kind) | ... times only the
 * kinds named.  An event pair waits for the work before it, so a timed
 * launch no longer overlaps its neighbours' launch latency: profiled runs
 * are slower than plain ones.  Diagnostics for roofline figures; off by
 * default. */
#define QISG_PROFILE_ONLY 0x100
int qisg_profile(qisg_handle *h, int enable);

/* Total device time (ms) of the timed launches of one kind, how many were
 * timed and how many were launched since qisg_profile(h, 1); kinds BLUE and
 * RED split QISG_KERNEL_SWEEP by colour.  Synchronises.  EINVAL: unknown
 * kind. */
int qisg_profile_read(qisg_handle *h, int kind, double *total_ms, int64_t *n_timed,
                      int64_t *n_launched);

/* Sweeps are replayed from a CUDA graph of one cycle of lcm(pt_every,
 * measure_every) sweeps whenever the sweep count is at a multiple of the
 * cycle (captured once on an internal stream, launched on the handle's
 * stream).  enable = 0 launches every kernel directly instead.  Results are
 * the same either way. */
int qisg_set_graphs(qisg_handle *h, int enable);

/* SAMPLES packing: launch the kernels of a sweep with programmatic dependent
 * launch (enable = 1, the default): each kernel is launched as the blocks of
 * the one before it leave, and waits for it on the device before it reads
 * its results, which hides part of the gaps between the red, blue, PT and
 * measurement launches (38.6 against 38.9 us per sweep at L = 16,
 * L_tau = 256, 32 samples x 4 replicas x 16 slots, on a GB300).  Results
 * are the same either way.  Synchronises. */
int qisg_set_launch_overlap(qisg_handle *h, int enable);

/* SAMPLES packing with 32-bit words: run each sweep's PT pass (Sec. 2.1) in
 * the last blocks of the blue pass instead of a launch of its own (enable =
 * 1, the default).  Each block of the blue pass takes a ticket once its bond
 * counts are added; the last P = ceil(n_samples * n_rep / 4) blocks wait
 * until every block has, then decide the chains as the PT pass does, a warp
 * per chain.  Used when P is at most half the blue pass's blocks and half
 * its resident blocks, 2N < 2^30 and n_slots <= 32; otherwise the PT pass
 * has its own launch.  The wait is bounded by wait_ns nanoseconds (0: the
 * default, 5 s; the bound is shared with qisg_set_persistent's barriers): a
 * wait that runs out ends the pass without PT and the next synchronising
 * call returns ETIMEOUT (the handle's state is then undefined: destroy it).
 * Results are the same either way.  EINVAL: wait_ns < 0.  Synchronises. */
int qisg_set_pt_in_blue(qisg_handle *h, int enable, int64_t wait_ns);

/* The persistent form of the batched sweep (SAMPLES packing, 32-bit words,
 * PT every sweep; Sec. 2.1's red / blue / PT cycle): enable = 1 runs every
 * stretch of sweeps up to the next measurement (or 64 sweeps when nothing
 * is measured) as ONE cooperative kernel launch -- fused red pass with the
 * pending PT exchanges, grid barrier, blue pass with the bond counts,
 * barrier, PT pass, barrier, per sweep -- and replays those launches (and
 * the measurements) from a captured CUDA graph.  The trajectory is the
 * same as with separate launches.  Each grid-barrier wait is bounded by
 * wait_ns nanoseconds (0: the default, 5 s); a wait that runs out ends the
 * launch and the next synchronising call returns ETIMEOUT (the handle's
 * state is then undefined: destroy it).  qisg_autotune then chooses the red
 * pass's threads per site and the sites each blue thread walks along tau
 * for this form.  EINVAL: another packing or word width, pt_every != 1,
 * 2N >= 2^30, or wait_ns < 0.  Synchronises. */
int qisg_set_persistent(qisg_handle *h, int enable, int64_t wait_ns);

/* Choose the SAMPLES sweep schedule by timing sweeps_per_candidate real
 * sweeps per candidate on the handle's own state; the red and blue passes are
 * timed and tuned separately.  Candidates: tiles 1, 2, 4, ..., 64 and the
 * default (0) and, for 32-bit words, the three blue kernel variants of each.
 * The tile is, for 64-bit words, the site groups of 4 each thread walks along
 * tau; for 32-bit words it selects the red pass's threads per site (1: four,
 * 2: two, 0: four while one thread per site would fill fewer than four waves
 * of 2048 threads per SM, else one) and the blue pass's sites per thread
 * (variants 0 and 2, a thread per replica quad walking at most `tile` sites,
 * the L_tau / 2 sites of a column split into ceil(L_tau / 2 / tile) segments
 * whose lengths differ by at most one; 2 with its registers bounded to four
 * blocks per SM and no prefetch of the next site) or site groups of 4 per
 * thread (variant 1, a thread per replica).  The default of variants 0 and 2 picks the segment
 * count that fills whole waves of resident blocks.  The simulation advances
 * by C * (1 + sweeps_per_candidate) sweeps meanwhile, C = 24 candidates for
 * 32-bit words and 8 for 64-bit words (results never depend on the schedule,
 * so the trajectory is the one an untuned run would follow); with the
 * persistent form on, C = 21 (3 red x 7 blue tiles, the default among them).
 * chosen: the blue pass's tile (0 for LANES, which has nothing to tune).
 * Synchronises. */
int qisg_autotune(qisg_handle *h, int sweeps_per_candidate, int *chosen);

/* Read or pin the SAMPLES sweep schedule: tile[c] and variant[c] of the red
 * (c = 0) and blue (c = 1) pass as qisg_autotune chooses them (tile 0 = the
 * default, else 1..64 as there; variant 0, 1 or 2).  Results never depend on
 * the schedule.  EINVAL: tile outside 0..64, variant not 0..2. */
int qisg_get_tiles(qisg_handle *h, int tile[2], int variant[2]);
int qisg_set_tiles(qisg_handle *h, const int tile[2], const int variant[2]);

/* Block until the handle's stream is idle; reports any device error flag. */
int qisg_sync(qisg_handle *h);

/* Free the handle and its device memory (NULL is a no-op). */
void qisg_destroy(qisg_handle *h);

/* Text of a QISG_E* code; a message for the last failure on this thread. */
const char *qisg_strerror(int code);
const char *qisg_last_error(void);

/* Philox4x32-10 on the device (Sec. 2.1.1): out[4i..4i+3] = Philox of
 * counter ctr[4i..4i+3] under key key[2i..2i+1], i < n.  All pointers are
 * DEVICE pointers; stream as in qisg_opts.  Used to check the device
 * generator against others.  EINVAL: n < 0 or a NULL pointer with n > 0. */
int qisg_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t n,
                       void *cuda_stream);

/* ------------------------------------------------------------------------ */
/* Batched form: many independent single-sample instances of uneven size in  */
/* one persistent kernel (and the building block of the serving loop).       */
/* ------------------------------------------------------------------------ */

typedef struct qisg_batch qisg_batch;

/* One instance: an L x L x L_tau prism with its own ladder, n_replicas
 * replicas, one disorder sample drawn from `seed`, a sweep target (0 = no
 * limit) and its boundary along tau (tau_antiperiodic 1: the bond from
 * tau = L_tau-1 to tau = 0 counts -S S, Sec. 1; 0: periodic).  Its
 * trajectory is that of qisg_create(L, L_tau, ladder, n_slots, n_replicas,
 * 1, seed) with pt_every = 1 and the same tau_antiperiodic. */
typedef struct {
    int L, L_tau, n_slots, n_replicas;
    const qisg_slot *ladder;    /* host array of n_slots (copied at admission) */
    uint64_t seed;
    int64_t n_sweeps;
    int tau_antiperiodic;
} qisg_instance_desc;

/* A batch with `capacity` instance slots whose device state lives in one
 * arena of mem_budget bytes (0: half of the free device memory), work ordered
 * on cuda_stream.  ENOMEM if the arena cannot be allocated. */
int qisg_batch_create(qisg_batch **out, int capacity, size_t mem_budget, void *cuda_stream);

/* Admit an instance into a free slot: its state is allocated from the arena
 * and initialised on the device (Sec. 2.1 start: random spins, walker w at
 * slot w).  EINVAL: bad descriptor (L even 2..128, L_tau even, 1..32 slots,
 * 1 .. 2*(64/n_slots) replicas, tau_antiperiodic 0 or 1); ENOMEM: no free slot or the arena has no room -- the
 * caller keeps the request queued.  Synchronises. */
int qisg_batch_admit(qisg_batch *b, const qisg_instance_desc *d, int *slot);

/* Free a slot and its arena memory.  Synchronises. */
int qisg_batch_retire(qisg_batch *b, int slot);

/* Advance every admitted instance by n_sweeps sweeps (an instance stops at
 * its target).  One cooperative persistent kernel runs all of them: red and
 * blue half sweeps over a work-list of (instance, site range) tiles, a PT
 * pass with one warp per (instance, replica) chain, and the counter advance,
 * separated by grid barriers whose waits are bounded (ETIMEOUT at the next
 * synchronising call if one gives up).  Asynchronous. */
int qisg_batch_run(qisg_batch *b, int64_t n_sweeps);

/* Tile rows of 256 sites per work item (1..16) and tile order (0: admission order, 1:
 * largest instances first).  Results never depend on either. */
int qisg_batch_set_schedule(qisg_batch *b, int tile_rows, int schedule);

/* Bound of each grid-barrier wait of the batch kernel, in nanoseconds (0:
 * the default, 5 s).  A wait that runs out sets the batch's error flag and
 * every block of the launch returns; the next synchronising call on the
 * batch returns ETIMEOUT, and the batch's state is then undefined (destroy
 * it).  For tests of that path and for callers that want a tighter watchdog.
 * EINVAL: wait_ns < 0. */
int qisg_batch_set_wait_limit(qisg_batch *b, int64_t wait_ns);

/* Time sweeps_per_candidate sweeps of each (tile rows, order) candidate on the
 * live batch and keep the fastest; the batch advances meanwhile. */
int qisg_batch_autotune(qisg_batch *b, int sweeps_per_candidate, int *tile_rows, int *schedule);

/* Sweeps done by a slot and whether it reached its target. */
int qisg_batch_status(qisg_batch *b, int slot, uint64_t *sweeps_done, int *done);

/* Results of a slot (any pointer may be NULL): A, B by slot int64
 * [n_replicas][n_slots], walker_at int32 [n_replicas][n_slots], spins by
 * walker int8 [n_replicas][n_slots][L*L*L_tau].  Synchronises. */
int qisg_batch_results(qisg_batch *b, int slot, int64_t *A, int64_t *B, int32_t *walker_at, int8_t *S);

/* Free arena bytes, free slots, kernel launches so far. */
int qisg_batch_info(qisg_batch *b, size_t *free_bytes, int *free_slots, int64_t *launches);

/* Arena bytes an instance would take (0 for an invalid descriptor). */
size_t qisg_batch_instance_bytes(const qisg_instance_desc *d);

int qisg_batch_sync(qisg_batch *b);
void qisg_batch_destroy(qisg_batch *b);

/* The transfer-matrix product of the exact-diagonalisation code (Sec. 2.2,
 * Eq. (transfer-matrix) and Appendix D), the matrix-vector product its
 * Lanczos iteration is built on: out = T in on the even (parity = +1) or
 * odd (parity = -1) sector of the transfer matrix
 *   T = e^{-k H0/2} prod_j [jP 1 + jM sigma^X_j] e^{-k H0/2},
 *   jP = e^{k_tau} / (e^{k_tau} + e^{-k_tau}), jM = e^{-k_tau} / (...),
 * of the L x L sample with couplings J (host int8 [L*L][2], +-1: bond 0 of
 * site x1 + L x2 to (x1+1, x2), bond 1 to (x1, x2+1), periodic; at L = 2
 * the two bonds between a pair of sites are distinct, as in the sweeps).
 * k_tau = k is the paper's case (its Gamma from exp(-2k) = tanh(k Gamma));
 * other pairs are the separate-coupling form of the rest of this library.
 * in, out: DEVICE arrays of 2^{L^2-1} doubles in the parity-aware basis
 * |n>_{e,o} = (|n> +- |2^{L^2}-1-n>)/sqrt 2, n < 2^{L^2-1} (bit j of n set
 * <=> S_j = -1); they may be the same array.  The L^2-1 bit-flip rounds
 * j = 0 .. L^2-2 are applied in order, then the last factor of Eq. (lr);
 * the results are those of that order with IEEE double arithmetic.  One GPU
 * holds L <= 5 (2^24 doubles); the paper splits L = 6 over 256 GPUs.
 * Allocates nothing; asynchronous on cuda_stream.  EINVAL: NULL pointer,
 * L outside 2..5, parity not +-1, a coupling not +-1 or a k, k_tau negative
 * or not finite, vectors not 8-byte aligned. */
int qisg_transfer_matvec(const double *in, double *out, int L, double k, double k_tau, const int8_t *J,
                         int parity, void *cuda_stream);

/* Replica overlaps of a caller-owned configuration, computed without
 * allocating device memory.  (The paper has no counterpart: this is a
 * deployment aid.)  It serves callers that cannot call cudaMalloc -- a host
 * whose allocator owns all device memory under a fixed budget, a serving loop
 * that must not stall on the device-wide synchronisation an allocation can
 * cause -- by counting in a scratch array compiled into the library (a
 * static __device__ array of QISG_NOALLOC_MAX_COUNTS 64-bit counters, 2 MiB,
 * which every GPU that loads the library holds until the process exits).
 *
 *   spins  DEVICE pointer to the SAMPLES packing: words of word_bits (32 or
 *          64) bits, [b][s][q][site][4] with b = sample / word_bits,
 *          q = replica / 4, the last index replica % 4, site = x + L*y +
 *          L*L*tau, bit (sample % word_bits) set <=> spin -1; b runs over
 *          ceil(n_samples / word_bits) blocks, q over ceil(n_replicas / 4).
 *          Each word at [..][s][..] holds the configuration now at slot s.
 *   q      DEVICE pointer, int64 [n_samples][n_slots][n_pairs], written with
 *          q = sum_i S^{r1}_i S^{r2}_i for pairs r1 < r2 in lexicographic
 *          order (the quantity qisg_overlaps reports).
 *   cuda_stream  cudaStream_t the work is ordered on (NULL: legacy default).
 * The scratch array's device address is looked up (cudaGetSymbolAddress)
 * on the first call made with a given device and CUDA context current, and
 * cached per (device, context); a call whose stream is being captured uses
 * the cache only, so make the first call on each device and context before
 * any stream capture (ESTATE otherwise).  The call allocates nothing (no
 * cudaMalloc, no cudaFree, no allocating library routine).  All calls share
 * the scratch array, which keeps the last call's counts; each call clears the
 * part it uses first.  Calls that overlap on the GPU race on the array:
 * serialise them.
 * EINVAL (checked before any device work): NULL pointer; word_bits not
 *   32/64; spins not aligned to its word or q to 8 bytes; L or L_tau odd or
 *   < 2; more than 2^31 sites; n_slots < 1, n_replicas < 2 or n_samples < 1;
 *   n_samples * n_slots * n_pairs > QISG_NOALLOC_MAX_COUNTS.
 * Asynchronous: errors of the kernels themselves surface at the next sync. */
#define QISG_NOALLOC_MAX_COUNTS (1 << 18)
int qisg_overlaps_noalloc(const void *spins, int word_bits, int L, int L_tau, int n_slots,
                          int n_replicas, int64_t n_samples, int64_t *q, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* QISG_H */
