/*
 * spinrp.h -- C ABI of the GB300 random-phase spin-dynamics library.
 *
 * The library evolves ONE pure state of M spins-1/2 (2^M amplitudes, resident
 * on the GPU) with the method of Alvarez, Danieli, Levstein & Pastawski,
 * "Quantum parallelism as a tool for ensemble spin dynamics calculations"
 * (arXiv:0710.3747):
 *
 *   - the state is the entangled random-phase state of the paper's "Testing the
 *     quantum parallelism" section, spin 1 up and every Zeeman basis state |r>
 *     of spins 2..M with weight 2^{-(M-1)/2} and an independent phase, which
 *     stands for the infinite-temperature ensemble of Eq. 1 (p_i = 1/2^{M-1});
 *   - the Hamiltonian is the secular spin-spin Hamiltonian of the "Spin systems
 *     with different coupling networks" section,
 *        H = sum_{i<j} [ a_ij S^z_i S^z_j + 1/2 b_ij (S^+_i S^-_j + S^-_i S^+_j) ];
 *   - the evolution is the symmetric second-order Trotter-Suzuki product the
 *     paper names (introduction, summary), with the splitting
 *        U(dt) = e^{-i dt/2 D} F_1 .. F_B F_B .. F_1 e^{-i dt/2 D},
 *     D = sum a_ij S^z_i S^z_j and F_k = exp(-i dt/2 b_k (S^x S^x + S^y S^y))
 *     on flip-flop bond k, bonds in canonical order (all pairs i<j with
 *     b_ij != 0, lexicographic);
 *   - after every step the library records the local polarization
 *     P_11(t) = 2 [W_11(t) - 1/2] of Eq. 2 with m = m' = 1 (computed as
 *     (N_up - N_dn)/(N_up + N_dn) of spin 1) and the norm, in FP64.
 *
 * Conventions: spins are numbered 1..M in the API; coupling matrices are M x M
 * row-major FP64, symmetric, zero diagonal; hbar = 1.  Amplitudes exchanged
 * with the host are in LOGICAL order (bit n-1 of the index = spin n, set = up)
 * as interleaved (re, im) FP64 pairs; on the device the library may store
 * them with its own bit permutation.
 *
 * Errors: every call returns SPINRP_OK (0) or a positive SPINRP_E* code and
 * never aborts; spinrp_last_error() gives a message for the calling thread.
 * Ownership: the caller owns the handles it creates and destroys them; the
 * library never frees caller memory.  Device work is asynchronous on the
 * stream given at state creation, except where a call says it synchronizes.
 * Handles are not thread-safe: one thread at a time per handle.
 */
#ifndef SPINRP_H
#define SPINRP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPINRP_OK 0
#define SPINRP_EINVAL 1       /* bad argument (size, index, type, capacity) */
#define SPINRP_ENOMEM 2       /* host or device allocation failed */
#define SPINRP_ECUDA 3        /* a CUDA runtime call or kernel launch failed */
#define SPINRP_ETIMEOUT 4     /* a bounded device-side wait gave up */
#define SPINRP_EUNSUPPORTED 5 /* valid request this build does not implement */
#define SPINRP_ESTATE 6       /* call out of order (e.g. evolve before init) */

/* Hamiltonian families of the paper ("Spin systems with different coupling
 * networks"): b/a = 0 Ising, a/b = 0 XY, a/b = 1 isotropic, a/b = -2 secular
 * dipolar truncated by a field along z.  For a coupling matrix J:
 *   XY:        a = 0,   b = J          (H = sum J (SxSx + SySy))
 *   DIPOLAR:   a = 2J,  b = -J         (H = sum J [2 SzSz - (SxSx + SySy)])
 *   ISOTROPIC: a = J,   b = J
 *   ISING:     a = J,   b = 0
 *   GENERIC:   a = a_generic, b = J                                         */
#define SPINRP_XY 0
#define SPINRP_DIPOLAR 1
#define SPINRP_ISOTROPIC 2
#define SPINRP_ISING 3
#define SPINRP_GENERIC 4

/* Amplitude precision on the device: complex64 (FP32 gate arithmetic) or
 * complex128 (FP64).  Gate coefficients, diagonal phases' integer tables and
 * all reductions are generated / accumulated in FP64 in both cases. */
#define SPINRP_C64 0
#define SPINRP_C128 1

typedef struct spinrp_system spinrp_system; /* host-side spin system (couplings, plan) */
typedef struct spinrp_state spinrp_state;   /* one device-resident state + P(t) series */

/* Message describing the last error on the calling thread ("" if none). */
const char *spinrp_last_error(void);

/* Library version string. */
const char *spinrp_version(void);

/* ---- spin systems (host only, no GPU needed) ---------------------------- */

/* Create a spin system of M spins (2 <= M <= 34) from the coupling matrix J
 * (M*M doubles, row-major) and Hamiltonian family htype (SPINRP_XY ..
 * SPINRP_GENERIC); a_generic is read only for SPINRP_GENERIC (else may be
 * NULL).  Only the upper triangle i<j is read.  The system copies its inputs.
 * The paper's problem statement: H of "Spin systems with different coupling
 * networks".  On success *out receives a handle to free with
 * spinrp_system_destroy.  Errors: SPINRP_EINVAL (M, htype, NULL, non-finite
 * coupling), SPINRP_ENOMEM. */
int spinrp_system_create(int M, const double *J, int htype, const double *a_generic,
                         spinrp_system **out);

/* The paper's two coupling networks ("Spin systems with different coupling
 * networks"), built in the library:
 * the open two-leg ladder of M = 2L spins, legs 1..L and L+1..2L with
 * neighbour coupling j_leg, rungs (n, n+L) with j_rung, XY Hamiltonian
 * (a = 0, b = J; the paper's b_x = j_leg, b_y = j_rung). */
int spinrp_ladder_create(int L, double j_leg, double j_rung, spinrp_system **out);

/* The star of M spins with truncated dipolar couplings: spin 1 at the origin,
 * spins 2..M uniform in the unit ball and at least rmin (0..0.5) apart, drawn
 * by rejection from Philox4x32-10 with key (lo32, hi32 of geom_seed) --
 * candidate n takes x, y from the words of counter (n, 0, 0, 2) and z from
 * counter (n, 1, 0, 2), each the top 53 bits of two words scaled to [-1, 1);
 * J_ij = (1 - 3 cos^2 theta_ij)/r_ij^3 (theta from the z axis) rescaled to unit
 * rms over pairs; Hamiltonian J [2 S^zS^z - (S^xS^x + S^yS^y)] (a = 2J, b = -J,
 * the a/b = -2 of the paper).  Errors: SPINRP_EINVAL. */
int spinrp_star_dipolar_create(int M, uint64_t geom_seed, double rmin, spinrp_system **out);

/* Copy the M x M coupling matrices of H (row-major, symmetric, zero diagonal):
 * a (S^zS^z) and b (flip-flop); either pointer may be NULL. */
int spinrp_system_couplings(const spinrp_system *sys, double *a, double *b);

/* The order in which the evolution applies the flip-flop bonds of the
 * forward half step, as indices into spinrp_system_bonds: 0, 1, ..., B-1.
 * The device reorders only gates on disjoint spins (they commute exactly),
 * so this is the product an external checker must replay.  Writes
 * min(B, cap) indices; *n receives B. */
int spinrp_schedule(const spinrp_system *sys, int32_t *bond_order, int cap, int *n);

/* Free a system (NULL is ignored).  States created from it stay valid. */
void spinrp_system_destroy(spinrp_system *sys);

/* Number of spins. */
int spinrp_system_num_spins(const spinrp_system *sys);

/* Flip-flop bonds in the canonical order of the forward half step: pairs
 * (i, j), 1-based, i < j, b_ij != 0, lexicographic.  Writes min(n, cap)
 * pairs (2 ints each) to pairs (may be NULL when cap = 0) and the total count
 * to *n.  Errors: SPINRP_EINVAL. */
int spinrp_system_bonds(const spinrp_system *sys, int32_t *pairs, int cap, int *n);

/* Choose the shared-memory tile width K (number of spins a tile spans, 2^K
 * amplitudes per tile) used for precision prec by states created afterwards;
 * K = 0 restores the built-in default (complex128: the widest K <= 12 that
 * leaves at least 128 tiles, at least 8; complex64: the width
 * among 12, 13 and 14 with the fewest modelled sweep-time units, sweeps per
 * step x max(2^K, jobs x 2^M / 152), ties to 13, then 12; states of up to 12
 * spins are one tile).  Valid K: 1..14 for SPINRP_C64, 1..13 for
 * SPINRP_C128 (clipped to M).  This is the autotuner's knob.
 * Errors: SPINRP_EINVAL. */
int spinrp_system_set_tile(spinrp_system *sys, int prec, int K);

/* Register bits per phase of the complex64 tile kernel: each thread keeps the
 * 2^rb amplitudes spanned by rb tile bits in registers while it applies every
 * ready gate on those bits (rb = 5 or 6; 0 restores the default: 6 for
 * tiles of 13+ spins, else 5).  Wider register sets apply more gates per
 * shared-memory round trip with fewer threads per tile.  The second autotuner knob; affects states and batches
 * created afterwards.  The complex128 tile kernel always keeps 2^5 amplitudes
 * per thread (tiles of 10+ spins; narrower tiles run the per-gate kernel).
 * Errors: SPINRP_EINVAL. */
int spinrp_system_set_regbits(spinrp_system *sys, int rb);

/* Storage orientation of complex64 states (no counterpart in the paper; a
 * storage choice of the register-blocked kernel).  When the flip-flop bonds
 * of the system form a bipartite graph (ladders, chains), its spins are
 * 2-coloured so that every bond joins the two colours, and a complex64 state
 * may store each amplitude whose basis index has an odd number of
 * first-colour spins up with its real and imaginary parts swapped, (Im, Re):
 * the two amplitudes every gate mixes are then stored in opposite orders and
 * the gate is applied to the stored words as they are.  mode 1: states are
 * oriented when the system is bipartite and the register-blocked program can
 * keep its colour pattern; mode 0 (default): never.  (On GB300 the oriented
 * sweep issues 10 % fewer instructions but runs a few per cent slower: its
 * back-to-back shared-memory loads throttle the shared-memory queue.)  Every readout of the
 * library (P, norms, spinrp_state_read, sector weights) returns the plain
 * values; only direct access to the amplitude buffer sees the swap (see
 * spinrp_state_orientation).  Takes effect for states created afterwards.
 * Errors: SPINRP_EINVAL. */
int spinrp_system_set_orientation(spinrp_system *sys, int mode);

/* The storage orientation a state of precision prec created now would have:
 * *black receives its mask of first-colour spins (bit q-1 = spin q), or 0 when
 * it would be stored plainly.  Host only (plans the system).  Errors:
 * SPINRP_EINVAL. */
int spinrp_system_orientation(const spinrp_system *sys, int prec, uint64_t *black);

/* Describe the sweep plan the library would use for precision prec: number
 * of segments the forward half step is cut into (*segments), device sweeps
 * per Trotter step in the steady state (*sweeps_per_step) and the tile width
 * (*K).  Any output pointer may be NULL.  Host only. */
int spinrp_system_plan_info(const spinrp_system *sys, int prec, int *segments,
                            int *sweeps_per_step, int *K);

/* Export the plan: the flip-flop gates of one forward half step in the order
 * the device applies them, as 1-based pairs (2 ints each), with the index of
 * the segment (sweep tile) each one runs in.  Writes min(n, cap) entries and
 * the total to *n.  For checking that the device order is the canonical one
 * up to exchanges of gates on disjoint spins. */
int spinrp_system_plan_gates(const spinrp_system *sys, int prec, int32_t *pairs,
                             int32_t *segment, int cap, int *n);

/* ---- states ----------------------------------------------------------- */

/* Device memory a state of system sys at precision prec needs: *psi_bytes
 * for the 2^M amplitudes and *work_bytes for everything else (FP64 P/norm
 * series of series_cap entries, reduction partials, gate tables, plan). */
int spinrp_state_bytes(const spinrp_system *sys, int prec, int64_t series_cap,
                       size_t *psi_bytes, size_t *work_bytes);

/* Create a state on the current CUDA device.  stream is a cudaStream_t (NULL
 * = default stream).  series_cap is the number of P(t) entries the state can
 * record (init records one, each Trotter step one).  psi and work are device
 * buffers of at least the sizes spinrp_state_bytes reports, 256-byte aligned,
 * owned by the caller and kept alive until spinrp_state_destroy; either may be
 * NULL, and the library then allocates (and later frees) that buffer itself
 * with cudaMalloc.  The state copies what it needs from sys.
 * Errors: SPINRP_EINVAL, SPINRP_ENOMEM, SPINRP_ECUDA. */
int spinrp_state_create(const spinrp_system *sys, int prec, void *stream, int64_t series_cap,
                        void *psi, void *work, spinrp_state **out);

/* Free a state and any memory the library allocated for it (NULL ignored).
 * Synchronizes the state's stream first. */
void spinrp_state_destroy(spinrp_state *st);

/* Set the state to the paper's entangled random-phase state
 *   |Psi> = 2^{-(M-1)/2} sum_r e^{i phi_r} |up>_1 (x) |r>,
 * phi_r = 2 pi u, u = top 53 bits of the first two output words of
 * Philox4x32-10(counter = (lo32 r, hi32 r, 0, 0), key = (lo32 seed, hi32 seed))
 * times 2^-53, r = the basis index of spins 2..M (spin n at bit n-2).  Resets
 * the series and records P(0).  Asynchronous. */
int spinrp_state_init_random_phase(spinrp_state *st, uint64_t seed);

/* Set the state to the paper's product (unentangled) random state of the
 * "Testing the quantum parallelism" section,
 *   |Psi> = |up>_1 (x) prod_{l=2..M} (|down>_l + e^{-i phi_l} |up>_l)/sqrt 2,
 * i.e. psi_x = 2^{-(M-1)/2} exp(-i sum_{l up in x} phi_l) for spin 1 up, 0
 * otherwise: only M-1 independent phases.  phi_l = 2 pi u_l, u_l = top 53 bits
 * of the first two output words of Philox4x32-10(counter = (l-1, 0, 0, 1),
 * key = (lo32 seed, hi32 seed)) times 2^-53 (the counter's last word keeps
 * these draws apart from the entangled state's).  Resets the series and
 * records P(0).  Asynchronous. */
int spinrp_state_init_product_phase(spinrp_state *st, uint64_t seed);

/* Load an arbitrary state from the host: 2^M complex amplitudes in logical
 * order as interleaved FP64 (re, im).  Resets the series and records P(0).
 * Synchronizes. */
int spinrp_state_load(spinrp_state *st, const double *amps);

/* Evolve by `steps` second-order Trotter steps of size dt (order must be 2;
 * dt may be negative), appending P and the norm after every step to the
 * series.  Asynchronous on the state's stream.  Errors: SPINRP_ESTATE before
 * init/load, SPINRP_EINVAL if the series would exceed its capacity or dt is
 * not finite, SPINRP_EUNSUPPORTED for order != 2, SPINRP_ECUDA. */
int spinrp_evolve(spinrp_state *st, double dt, int64_t steps, int order);

/* Number of entries recorded so far (1 after init, +1 per step). */
int64_t spinrp_series_length(const spinrp_state *st);

/* Copy the recorded polarization series P_{site,1}(t_k), k = 0..len-1 (the
 * local polarization of spin `site` given spin 1 polarized at t = 0, the
 * paper's Eq. 2 with m = 1 and P = 2W - 1) to the host buffer out
 * (min(len, cap) doubles); *n receives len.  Site 1 is always recorded;
 * sites 2..M need the all-site readout (spinrp_state_set_sites) enabled at
 * the last init / load, else SPINRP_ESTATE.  Sites outside 1..M give
 * SPINRP_EINVAL.  Synchronizes the state's stream. */
int spinrp_polarization(spinrp_state *st, int site, double *out, int64_t cap, int64_t *n);

/* Request (all_sites != 0) or drop the all-site readout from the next
 * spinrp_state_init_* / spinrp_state_load on: after every Trotter step the
 * reducing sweep also sums, per block, the weight with each spin up, and a
 * fixed-order column reduction records P_{q1}(t) = (2 N_up(q) - N)/N of every
 * spin q (M doubles per entry, in the work buffer spinrp_state_bytes sizes).
 * No extra pass over the state; one small kernel per step. */
int spinrp_state_set_sites(spinrp_state *st, int all_sites);

/* All-site series: out[k * M + (q - 1)] = P_{q1}(t_k) for k = 0..min(len,
 * cap)-1, q = 1..M; *n receives len.  SPINRP_ESTATE unless the all-site
 * readout was enabled at the last init / load.  Synchronizes. */
int spinrp_site_series(spinrp_state *st, double *out, int64_t cap, int64_t *n);

/* Same for the norm sum_x |psi_x|^2 after each step. */
int spinrp_norm_series(spinrp_state *st, double *out, int64_t cap, int64_t *n);

/* Weights of the total-S^z sectors of the current state: out[k] = sum of
 * |psi_x|^2 over the basis states with k spins up, k = 0..M (the
 * magnetization distribution; the paper's secular Hamiltonian, section
 * "Spin systems with different coupling networks", commutes with the total
 * S^z, so every family conserves it, and the random-phase state of
 * "Ensemble vs. pure entangled state" starts at out[k] = C(M-1, k-1) /
 * 2^(M-1)).
 * FP64 sums in a fixed order (reproducible).  Writes min(cap, M+1) values
 * and M+1 to *n; reads the whole state once on the state's stream and
 * synchronizes it.  Errors: SPINRP_EINVAL, SPINRP_ESTATE (not initialized),
 * SPINRP_ECUDA. */
int spinrp_sector_norms(spinrp_state *st, double *out, int cap, int *n);

/* Read n amplitudes with LOGICAL basis indices idx[k] (0 <= idx < 2^M) into
 * out (2n doubles, re/im).  Synchronizes. */
int spinrp_state_read(spinrp_state *st, const int64_t *idx, int64_t n, double *out);

/* Device pointer of the amplitude buffer and the device-side bit layout:
 * layout[q] receives the physical bit position of spin q+1 (M ints).  The
 * layout is the same after every complete spinrp_evolve call. */
int spinrp_state_layout(const spinrp_state *st, int32_t *layout, void **psi);

/* Storage orientation of the state (see spinrp_system_set_orientation):
 * *black receives the mask of first-colour spins (bit q-1 = spin q) of an
 * oriented state, whose amplitudes with an odd number of those spins up are
 * stored (Im, Re) in the buffer spinrp_state_layout reports, or 0 for a
 * state stored plainly.  Host only. */
int spinrp_state_orientation(const spinrp_state *st, uint64_t *black);

/* Pipelined sweeps (no counterpart in the paper; the same second-order
 * Trotter-Suzuki steps, the product the introduction and summary name,
 * scheduled differently).  A complex64 state whose plan uses 13-spin tiles
 * and six register bits, plainly stored, with at least four tiles per SM
 * (M >= 23 on GB300), runs each sweep as one persistent launch of one block
 * per SM: a producer warpgroup gathers tiles into three shared-memory buffers
 * and writes them back while two compute warpgroups apply the sweep's gates,
 * so the state's streaming through HBM overlaps the arithmetic.
 * on = 1 (the default) uses it where the plan takes it, on = 0 the
 * one-tile-per-block sweep; the amplitudes and series are the same bit for
 * bit.  Takes effect at the next evolve.  Host only.  Errors: SPINRP_EINVAL.
 * The pipeline's hand-over waits are bounded (2 s each); one that gives up
 * records NaN for that step's P and norm and sets the state's error word,
 * which spinrp_polarization (site 1) and spinrp_norm_series then report as
 * SPINRP_ETIMEOUT. */
int spinrp_state_set_pipeline(spinrp_state *st, int on);

/* *on = 1 when the state's sweeps run pipelined (the setting is on and the
 * plan takes it), else 0.  Host only.  Errors: SPINRP_EINVAL. */
int spinrp_state_pipeline(const spinrp_state *st, int *on);

/* Diagnostic of the pipelined sweep's bounded waits (no counterpart in the
 * paper): one launch in which the producer issues no copies, so every wait
 * gives up after its time limit and every block returns; reports
 * SPINRP_ETIMEOUT (with the launch's duration in *seconds, if not NULL) --
 * SPINRP_ECUDA if no wait ran out -- and clears the error word again.  The
 * amplitudes and the series are untouched.  SPINRP_ESTATE when the state's
 * plan does not take the pipelined sweep.  Synchronizes. */
int spinrp_state_pipeline_timeout_check(spinrp_state *st, double *seconds);

/* ---- batches of independent jobs ------------------------------------------ */

/* A batch evolves many independent random-phase states at once: disorder
 * realizations and phase seeds, the average over N_alpha realizations of the
 * paper's Eq. 4 (each job is one W^{alpha}, its P_11 one term of the mean).
 * Jobs may differ in M and couplings; jobs with the same sweep plan (same M
 * and bond structure) form a group whose sweeps run as one launch over all
 * its jobs, and the steady-state Trotter steps of all groups are replayed as
 * one CUDA graph.  A group without an explicit tile width takes the default
 * tile model's width for its job count (see spinrp_system_set_tile), which
 * for large groups can be wider than a single state's.  Device memory
 * (states, tables, series) is allocated by the library with cudaMalloc. */
typedef struct spinrp_batch spinrp_batch;

/* Create a batch of njobs jobs: systems[k] (copied; the caller may destroy it
 * afterwards) with phase seed seeds[k], precision prec, room for series_cap
 * P(t) entries per job, all work on `stream`.  Errors: SPINRP_EINVAL,
 * SPINRP_ENOMEM, SPINRP_ECUDA. */
int spinrp_batch_create(int njobs, const spinrp_system *const *systems, const uint64_t *seeds,
                        int prec, int64_t series_cap, void *stream, spinrp_batch **out);

/* Free a batch (synchronizes its stream; NULL ignored). */
void spinrp_batch_destroy(spinrp_batch *b);

/* Device bytes the batch holds, and the number of plan groups. */
int spinrp_batch_info(const spinrp_batch *b, size_t *device_bytes, int *groups);

/* Random-phase state of every job (seeds from create); records P(0). */
int spinrp_batch_init_random_phase(spinrp_batch *b);

/* Product random state (as spinrp_state_init_product_phase) of every job. */
int spinrp_batch_init_product_phase(spinrp_batch *b);

/* `steps` second-order Trotter steps of size dt for every job (order 2). */
int spinrp_batch_evolve(spinrp_batch *b, double dt, int64_t steps, int order);

/* Launch mode of the batch's multi-tile groups.  on = 1: one persistent
 * launch per spinrp_batch_evolve call, replayed from a CUDA graph captured
 * for its step count, whose blocks pull work items -- one tile of one sweep
 * of one job -- from a device queue in sweep order and wait (on a per-job
 * counter of finished tiles, about a second at most) until the job's previous
 * sweep is complete; it reads tiles through L2 only (other SMs wrote them
 * earlier in the same launch).  Groups with complex64 register programs of
 * six register bits on 13- or 14-spin tiles take part (those of the batch's
 * most common width); the others, and the groups whose whole state fits one
 * tile (kept in shared memory for every step), run as with on = 0.  on = 0
 * (the default, 8 % faster on GB300 for the 4096-star batch): one launch per
 * sweep, steady steps replayed from CUDA graphs.  Results are the same bit
 * for bit.  A persistent wait that gives up sets an error word that
 * spinrp_batch_polarization and spinrp_batch_ensemble report as
 * SPINRP_ETIMEOUT.  Errors: SPINRP_EINVAL. */
int spinrp_batch_set_persistent(spinrp_batch *b, int on);

/* Pipelined sweeps for a batch's multi-tile groups (no counterpart in the
 * paper; the same steps scheduled differently, see spinrp_state_set_pipeline):
 * a group of complex64 jobs with 13-spin tiles and six register bits, plainly
 * stored, with at least four (job, tile) units per SM, runs each sweep as one
 * persistent launch over all its jobs' tiles.  on = 1 (the default) uses it
 * where a group takes it, on = 0 one tile per block; the series are the same
 * bit for bit.  Groups in the persistent launch (spinrp_batch_set_persistent)
 * keep it.  A hand-over wait that gives up marks the step NaN and sets an
 * error word that spinrp_batch_polarization and spinrp_batch_ensemble report
 * as SPINRP_ETIMEOUT.  Host only.  Errors: SPINRP_EINVAL. */
int spinrp_batch_set_pipeline(spinrp_batch *b, int on);

/* *groups receives the number of the batch's plan groups whose sweeps run
 * pipelined.  Host only.  Errors: SPINRP_EINVAL. */
int spinrp_batch_pipeline(const spinrp_batch *b, int *groups);

/* Diagnostic of the persistent launch's bounded waits (no counterpart in the
 * paper): runs the launch for a `steps`-step plan with its queue started past
 * the first sweep, so every item waits for tiles that never run; each wait
 * gives up after its poll limit, the blocks return, and the call reports
 * SPINRP_ETIMEOUT (with the launch's duration in *seconds, if not NULL) --
 * SPINRP_ECUDA if no wait ran out.  No tile is processed: the batch's states
 * and series are unchanged, and its next evolve runs normally.  Needs a
 * batch with persistent groups, initialized.  Synchronizes. */
int spinrp_batch_persist_timeout_check(spinrp_batch *b, int64_t steps, double *seconds);

/* P(t) series of job k (site 1) to the host; synchronizes. */
int spinrp_batch_polarization(spinrp_batch *b, int job, double *out, int64_t cap, int64_t *n);

/* Mean and standard deviation over all jobs of P(t_k), k = 0..len-1 (the
 * N_alpha average of Eq. 4 and its spread), reduced on the device in FP64;
 * either output may be NULL.  Synchronizes. */
int spinrp_batch_ensemble(spinrp_batch *b, double *mean, double *stddev, int64_t cap, int64_t *n);

/* ---- allocation-free readout (no counterpart in the paper) --------------- */

/* The paper has no counterpart to this call.
 *
 * Polarization P = (N_up - N_dn)/(N_up + N_dn) of spin `site` (1-based) and
 * the norm N_up + N_dn of a device state the caller owns, written to out[0]
 * and out[1] (a device buffer of 2 doubles the caller owns), asynchronously on
 * `stream` (a cudaStream_t; NULL = default stream).
 *
 * For callers that cannot allocate device memory (code inside a host
 * application that owns every device allocation, or a loop that must not let
 * an allocation synchronize the device): this call allocates nothing.  Its
 * only scratch, 1216 FP64 partial pairs and a counter (about 19.5 KiB), is a
 * fixed array in device memory that every GPU loading the library holds until
 * the process exits.
 *
 * psi: 2^M amplitudes, complex64 (prec = SPINRP_C64) or complex128, interleaved
 * re/im.  layout: NULL when bit n-1 of the index is spin n, else M ints giving
 * the bit position of each spin (as spinrp_state_layout reports for a
 * library state).  blocks: reduction blocks, 0 = automatic; more than 1216 is
 * rejected (SPINRP_EINVAL).  Errors: SPINRP_EINVAL for bad arguments or M > 34,
 * SPINRP_ECUDA if a CUDA call fails.
 *
 * The first call on a device (with that device current) looks up the
 * scratch array's device address; make that first call before any stream
 * capture.  The address is cached per device with the unique ID of the
 * context it was looked up in, and looked up again when a call runs in
 * another context (after the device was reset and its context recreated).
 * Every call shares the one array and clears its counter itself;
 * calls that overlap on the GPU (different streams, no ordering between them)
 * race on it and must not be issued. */
int spinrp_polarization_noalloc(const void *psi, int M, int prec, int site, const int32_t *layout,
                                int blocks, double *out, void *stream);

/* ---- measurement (no counterpart in the paper) ------------------------- */

/* Kernel kinds for spinrp_profile_read. */
#define SPINRP_KERNEL_SWEEP 0  /* tile sweeps (gates, diagonal phase, reduction) */
#define SPINRP_KERNEL_INIT 1   /* random-phase initialization */
#define SPINRP_KERNEL_TABLES 2 /* FP64 gate / phase table generation */

/* enable != 0: from now on bracket every kernel this state launches with a
 * pair of CUDA events on the state's stream (clearing earlier records);
 * enable == 0: stop recording (records are kept for spinrp_profile_read). */
int spinrp_profile(spinrp_state *st, int enable);

/* Total device time (ms) and number of launches recorded for one kernel
 * kind.  Synchronizes the state's stream. */
int spinrp_profile_read(spinrp_state *st, int kind, double *total_ms, int64_t *launches);

/* Number of kernels the library has launched in this process (all states). */
int64_t spinrp_launch_count(void);

/* Bytes this state has copied host->device and device->host so far. */
int spinrp_state_transfer_bytes(const spinrp_state *st, int64_t *h2d, int64_t *d2h);

/* Host self-check of the device program for precision prec (no GPU): every
 * sweep's register-blocked phase program is executed on a random host tile
 * and compared with the sweep's plain op list, and the element-wise ops are
 * checked to stay in order.  Also reports the mean number of phases per sweep
 * and of gates per phase (either pointer may be NULL).  SPINRP_OK when every
 * sweep agrees, SPINRP_EINVAL with a message otherwise. */
int spinrp_system_plan_check(const spinrp_system *sys, int prec, double *phases_per_sweep,
                             double *gates_per_phase);

#ifdef __cplusplus
}
#endif

#endif /* SPINRP_H */
