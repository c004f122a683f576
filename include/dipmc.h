/*
 * dipmc.h -- C ABI of the B300 dipolar Heisenberg Monte Carlo sweep library
 * (libdipmc.so), after Stamps & Ambrose, arXiv:1211.6234.
 *
 * One lattice handle holds R independent replicas of an L x L periodic square
 * lattice of unit 3-vector spins (Sec. 2.1) that share L, the update spacing l,
 * the seed and the site schedule; each replica has its own J, C_D, K2, K4, T.
 *
 * Energy (Sec. 4 total energy, with these readings of the printed signs):
 *   E = -J sum_bonds s_i.s_j + sum_i (-K2 s_iz^2 - K4 s_iz^4) + (C_D/2) sum_n s_n.h_n
 *   h_n = sum_m W~(n - m) s_m          (m = n included through W~(0))
 * W~ is the dipole tensor summed over periodic images (Sec. 2.1, Eq. 2).
 *
 * Conventions for every entry point:
 *   - Return 0 (MC_OK) on success, a negative MC_E* code otherwise; nothing
 *     throws across the ABI.  mc_last_error() gives a one-line reason (per thread).
 *   - Handles are opaque and owned by the library (create/destroy).  Buffers
 *     passed in are owned by the caller; the library never keeps a pointer to
 *     them past the call.  A handle is not safe for concurrent calls: call the
 *     functions of one handle from one host thread at a time (different handles
 *     may be driven from different threads).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Device work of a call is enqueued on that stream; calls that return host
 *     data synchronise it.
 *   - Spin and field arrays are FP32, replica-major SoA: [R][3][L][L]
 *     (component x, y, z; row y; column x).  W~ arrays are [4][L][L] (xx, xy,
 *     yy, zz) indexed by the displacement rho = (rho_x, rho_y) in [0, L)^2.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11) keyed by the 64-bit seed
 * (key = {lo32, hi32}).  Counter layouts (word 3 carries a tag in its top byte):
 *   attempt at site q of replica r, sweep t, sub-step k: {q, r, t, k | 1<<24};
 *       words 0, 1 draw the proposal, word 2 the acceptance uniform
 *   sweep schedule round keys: {t, 0, 0, 2<<24}; paper's draw: {t, k, 0, 3<<24}
 *   random initial spins: {site, r, 0, 4<<24}
 * A uniform is u = (word >> 8) * 2^-24.
 */
#ifndef DIPMC_H
#define DIPMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MC_OK 0
#define MC_EINVAL (-1)    /* bad argument */
#define MC_ENOMEM (-2)    /* device allocation failed / over budget */
#define MC_ENOTREADY (-3) /* a prerequisite step was not done (e.g. W~ not computed) */
#define MC_ETIMEOUT (-4)  /* a bounded device wait gave up */
#define MC_ECUDA (-5)     /* a CUDA call failed; the message names it */
#define MC_ENOSYS (-6)    /* no field path supports this (L, l) in this library */

/* Observable indices (per sample, once per measured sweep). */
#define MC_OBS_ABS_M 0  /* |m| = |sum s| / N                        */
#define MC_OBS_MZ 1     /* m_z                                       */
#define MC_OBS_ABS_MZ 2 /* |m_z|                                     */
#define MC_OBS_MPAR 3   /* M_par = sqrt(M_x^2 + M_y^2)  (Sec. 4.1)   */
#define MC_OBS_E 4      /* energy per spin E/N                       */
#define MC_OBS_MST 5    /* staggered magnetisation m_st (Appendix B): sqrt(m_h^2 + m_v^2) from the z
                           components of the four 2 x 2 sub-lattices, m_h = m1 + m2 - m3 - m4,
                           m_v = m1 + m4 - m3 - m2, m_lambda = (1/N) sum over sub-lattice lambda;
                           1 = (x, y even), 2 = (x odd, y even), 3 = (x, y odd), 4 = (x even, y odd) */
#define MC_OBS_WALL 6   /* wall density (n_v^z + n_h^z)/(4N), n_v^a = sum_i 1 - sgn(s_i^a s_{i+y}^a),
                           n_h^a likewise with i+x (Sec. 4.1 domain-wall equations) */
#define MC_OBS_OX 7     /* orientational order of one state |n_h^x - n_v^x| / (n_h^x + n_v^x) (0 without walls); */
#define MC_OBS_OY 8     /*   its mean is O_x of Sec. 4.1; likewise y and z */
#define MC_OBS_OZ 9
#define MC_OBS_CONE 10  /* cone angle of one state (2/pi)(1/N) sum_i |theta_i - pi/2| (the per-site
                           average inside eta is over time; this one is per state, for its variance) */
#define MC_NOBS 11

/* Field paths (mc_set_field_path). */
#define MC_PATH_AUTO 0
#define MC_PATH_DIRECT 1      /* FP32 CUDA-core Toeplitz sum, one CTA per replica */
#define MC_PATH_WINDOW_F32 2  /* windowed sweep, stale field from the FP32 full field */
#define MC_PATH_TENSOR 3      /* windowed sweep, stale field on tcgen05 tensor cores, split-BF16x3 */
#define MC_PATH_FFT 4         /* full field per sub-step by 2D FFT convolution (L a power of two) */
#define MC_PATH_SPECTRAL 5    /* field at the sub-step's sites from sub-lattice spectra (L/l <= 32) */
#define MC_PATH_INCREMENTAL 6 /* field kept at every site, rank-n update per sub-step (L <= 64, (L/l)^2 <= 64) */
#define MC_PATH_FFT_CLUSTER 7 /* 2D transform of each replica held in a 16-CTA cluster's shared memory (L a power
                                 of two, 16 <= L <= 256, L/l a power of two <= 16) */

typedef struct mc_lattice mc_lattice;

/* Statistics of one replica since the last reset. */
typedef struct mc_obs {
    int64_t samples;            /* measured sweeps */
    double mean[MC_NOBS];       /* sample means */
    double var[MC_NOBS];        /* sample variances (1/n) */
    double err_naive[MC_NOBS];  /* sqrt(var / (n - 1)) */
    double err[MC_NOBS];        /* autocorrelation-corrected error of the mean: the largest error of
                                   the means of blocks of 2^k sweeps over the levels k >= 1 that
                                   still hold >= 32 blocks, and never below err_naive.  It reaches
                                   the true error only when a block of 2^k sweeps is long against
                                   tau_int (a run of about 320 tau_int sweeps or more); shorter runs
                                   underestimate it */
    double tau_int[MC_NOBS];    /* 0.5 (err / err_naive)^2, in sweeps between samples */
    double eta;                 /* cone angle (Sec. 4.1): (1/N) sum_i sqrt((2/pi)^2 <(theta_i - pi/2)^2>) */
    double energy;              /* current energy per spin (tracked exactly, FP64) */
    int64_t accepted;           /* accepted single-site moves */
    int64_t attempted;          /* attempted single-site moves */
} mc_obs;

/* One-line description of the last error on this thread ("" if none). */
const char *mc_last_error(void);

/* ABI version (incremented on incompatible changes). */
int mc_version(void);

/*
 * Create a handle for `replicas` lattices of size L x L with update spacing l
 * (Sec. 3.1: simultaneous update sites o + l(a, b), n = (L/l)^2 of them).
 * Requires L >= 2, 2 <= l <= L, L % l == 0 (l = L is exact sequential
 * Metropolis, Appendix B), replicas >= 1.  Allocates device state on the
 * current device.  Defaults: J = 1, C_D = 0.1, K2 = 0.8, K4 = 0, T = 0.6 for all
 * replicas; cap proposal of 0.5 rad; permutation schedule; spins +z; W~ not
 * computed.  *out is NULL on failure.
 */
int mc_create_lattice(int L, int l, int replicas, uint64_t seed, mc_lattice **out);

/* Free the handle and its device memory (synchronises the device). NULL is a no-op. */
int mc_destroy(mc_lattice *lat);

/* Couplings of one replica (replica = -1: all).  T > 0.  Energies are in units of
 * k_B = 1 (Sec. 2.2).  Invalidates the tracked energy (recomputed at the next sweep). */
int mc_set_params(mc_lattice *lat, int replica, double J, double C_D, double K2, double K4,
                  double T);

/* Proposal (Sec. 3.1): kind 0 = uniform on the spherical cap of half-angle
 * cone_rad around the current spin (0 < cone_rad <= pi); kind 1 = uniform on S^2
 * (the paper's choice; cone_rad ignored); kind 2 = complete reversal S = -s, the
 * dipolar Ising variant of Appendix B when the spins are (0, 0, +-1) (init mode 3). */
int mc_set_proposal(mc_lattice *lat, int kind, double cone_rad);

/* Site schedule: kind 0 = every sweep visits the l^2 offsets in a pseudo-random
 * permutation (each site attempted once per sweep); kind 1 = each sub-step draws
 * its offset uniformly with replacement (Sec. 3.1 host loop). */
int mc_set_schedule(mc_lattice *lat, int kind);

/* Field path for the sweep (MC_PATH_*).  MC_PATH_AUTO picks the fastest supported.
 * The windowed paths (2, 3) process the l^2 sub-steps of a sweep in windows of B
 * consecutive sub-steps: the field at every site a window visits is evaluated once
 * on the state at the window's start (for all replicas together), and each
 * sub-step adds the exact change from the moves accepted earlier in the window,
 * so the sweep is the same simultaneous-flip update (Sec. 3.1, 3.2) up to
 * rounding.  MC_PATH_TENSOR needs L % 8 == 0 and B*(L/l)^2 % 128 == 0.
 * MC_PATH_FFT evaluates the full field of every replica by FFT convolution before
 * each sub-step (L a power of two, 8 <= L <= 1024, spins in global memory); it is
 * the path for large lattices, where mc_get_field and mc_energy also use the FFT.
 * MC_PATH_SPECTRAL splits the field at a sub-step's sites into l^2 circular
 * convolutions on the (L/l) x (L/l) grid of each cell offset and keeps the DFT of
 * every offset's spin sub-lattice on the device: a sub-step is an O(L^2)
 * contraction of those spectra with the transforms of W~, an inverse DFT, the
 * update and the DFT of the updated sub-lattice (2 <= L/l <= 32, any L).  The FFT
 * and spectral paths measure the energy afresh from the full field at each
 * measured sweep.  MC_PATH_INCREMENTAL keeps the field at every site in shared
 * memory and adds W~ * delta of the accepted moves after each sub-step, so the
 * energy of a measured sweep is an O(L^2) sum over the kept field; the field is
 * re-evaluated from scratch every 8 sweeps.  MC_PATH_FFT_CLUSTER runs each
 * replica in a cluster of 16 CTAs that keeps the replica's 2D Fourier transform
 * (S^, and W^, the transform of W~) in shared memory, each CTA a sixteenth of the
 * wave vectors and of the rows: the field at a sub-step's n sites is a partial
 * inverse transform (h = W~ * s is a convolution, Sec. 2.1, Eq. 2), the accepted
 * moves update S^ exactly, and S^ is taken afresh by a 2D DFT before every sweep;
 * the energy is measured afresh at measured sweeps.  It is meant for one or a
 * few large lattices.  MC_PATH_AUTO order: tensor (where its
 * window fits: L % 8 == 0, L/l in {1, 2, 4}, the spins of a replica in shared
 * memory, i.e. L up to about 100), direct, spectral, FFT, windowed FP32 (the
 * incremental and cluster paths are chosen explicitly or by mc_autotune). */
int mc_set_field_path(mc_lattice *lat, int path);

/* Sub-steps per window of the windowed paths (must divide l^2; 0 = automatic). */
int mc_set_window(mc_lattice *lat, int B);

/* Initial spins: mode 0 = random uniform on S^2 from the seed; 1 = all +z;
 * 2 = copy `user` (host pointer, [R][3][L][L] FP32, used as given); 3 = random
 * Ising spins (0, 0, +-1) from the seed (+1 where the site's first uniform is
 * below 1/2).  Resets the sweep counter to 0, clears observables and the energy
 * histogram, invalidates the tracked energy. */
int mc_init_spins(mc_lattice *lat, int mode, const float *user);

/* Replica-summed dipole tensor (Sec. 2.1, Eq. 2), computed on the GPU in FP64:
 * W~(rho) = sum_{|a|,|b| <= image_cutoff} W(rho_c + (aL, bL)) over r != 0, where
 * rho_c is the minimum-image representative of each component (both +-L/2 averaged
 * when a component is L/2), plus, if tail_correction, the continuum tail outside
 * the square of half-width (A + 1/2) L: zz += 4 sqrt(2) / ((A + 1/2) L^3), xx and
 * yy -= half of that.  image_cutoff in [0, 4096]. */
int mc_precompute_W(mc_lattice *lat, int image_cutoff, int tail_correction);

/*
 * Run nsweeps sweeps of the simultaneous-flip Metropolis update (Sec. 3.1, 3.2)
 * on every replica.  One sweep = l^2 sub-steps; sub-step k of sweep t uses offset
 * o = schedule(t, k); every site q = o + l(a, b) gets a proposal and is accepted
 * iff u < exp(-dE/T) with dE computed from the state before the sub-step; all
 * accepted moves are then applied together.  If measure_every > 0, observables
 * are sampled after every measure_every-th sweep.  Requires mc_precompute_W.
 * Asynchronous on `stream` (errors of the launch itself are reported).
 */
int mc_sweep(mc_lattice *lat, int nsweeps, int measure_every, void *stream);

/*
 * Uneven lattices in one launch: run nsweeps sweeps of every replica of `count`
 * handles of possibly different L as ONE persistent launch of the direct kernel
 * (one CTA per replica for the whole call), e.g. requests or parameter ladders of
 * L = 32, 48, 64, 96 together.  The handles must all resolve to the direct path
 * (MC_PATH_DIRECT), share C = L / l (the number of simultaneous sites per
 * sub-step, Sec. 3.1), the proposal, cone and schedule, have W~ computed, keep no
 * energy histogram and appear once each.  Every replica gets exactly the
 * arithmetic of mc_sweep on its own handle (the same cell offsets per thread and
 * reduction orders), so its spins, observables and tracked energy are those of
 * that call, bit for bit; each handle's sweep counter advances by nsweeps.
 * Asynchronous on `stream`.  MC_EINVAL for a handle that breaks a rule above.
 */
int mc_sweep_group(mc_lattice *const *lats, int count, int nsweeps, int measure_every, void *stream);

/*
 * As mc_sweep (no measurement), and also record every attempt into `trace`
 * (device pointer, caller-owned, FP32).  Record layout, MC_TRACE_W floats per
 * attempt, ordered [replica][sweep][sub-step][site d] with d = Dy*(L/l) + Dx:
 *   q (site index y*L + x, exact), h_x, h_y, h_z (field at q before the step),
 *   dE, u, accepted (0/1), S_x, S_y, S_z (proposal).
 * trace_floats must be >= R * nsweeps * L * L * MC_TRACE_W.
 */
#define MC_TRACE_W 10
int mc_sweep_trace(mc_lattice *lat, int nsweeps, float *trace, size_t trace_floats,
                   void *stream);

/* Statistics of one replica (synchronises the lattice's last stream). */
int mc_observables(mc_lattice *lat, int replica, mc_obs *out);

/* Statistics of replicas [first, first + count) into out[0 .. count-1]
 * (caller-owned host array), exactly as mc_observables gives them one by one,
 * with one synchronisation and one device-to-host copy for the whole range.
 * MC_EINVAL for a range outside [0, R) or a null out. */
int mc_observables_batch(mc_lattice *lat, int first, int count, mc_obs *out);

/* Histogram of the energy per spin E/N over the measured sweeps (Appendix B,
 * energy distributions near the transition): nbins equal bins on [lo, hi) per
 * replica; samples outside are not counted.  Setting it clears the counts;
 * nbins = 0 turns it off.  mc_get_histogram copies nbins counts of one replica
 * to a host array (synchronises the lattice's last stream). */
int mc_set_histogram(mc_lattice *lat, double lo, double hi, int nbins);
int mc_get_histogram(mc_lattice *lat, int replica, int64_t *counts);

/* Clear all observable accumulators (binning, cone angle, acceptance). */
int mc_reset_observables(mc_lattice *lat);

/* Copy spins [R][3][L][L] FP32 into dst (dst_on_device: 1 = device pointer,
 * 0 = host pointer).  Synchronises `stream`. */
int mc_get_spins(mc_lattice *lat, float *dst, int dst_on_device, void *stream);

/* Full dipole field h = W~ * s at every site of every replica, [R][3][L][L] FP32,
 * computed directly in FP32 on the GPU.  Synchronises `stream`. */
int mc_get_field(mc_lattice *lat, float *dst, int dst_on_device, void *stream);

/* W~ by the Ewald/Harris split of Sec. 2.1 (real-space erfc sum plus the
 * reciprocal-lattice sum of the erf part; FP64 on the GPU): the exact infinite
 * image sum, which the image window plus continuum tail of mc_precompute_W
 * approximates.  eta is the splitting width (<= 0: L/4); the result does not
 * depend on it.  mc_precompute_W_ewald installs it in a handle (as
 * mc_precompute_W does, recorded with image_cutoff -1).  mc_wtilde_ewald gives
 * the tensor between two layers a height z apart (the quasi-3D case of the
 * Sec. 2.1 footnote; z = 0 is the lattice itself), [6][L][L] FP64 to a host
 * pointer: xx, xy, yy, zz, xz, yz, rho = (x, y) at [y][x].  |z| <= L. */
int mc_precompute_W_ewald(mc_lattice *lat, double eta);
int mc_wtilde_ewald(int L, double z, double eta, double *dst_host);

/* W~ in FP64, [4][L][L], to a host pointer.  MC_ENOTREADY before mc_precompute_W. */
int mc_get_W(mc_lattice *lat, double *dst_host);

/* Total energy of every replica from a full field evaluation (FP32 field, FP64
 * sums), [R] doubles to a host pointer.  Synchronises `stream`. */
int mc_energy(mc_lattice *lat, double *dst_host, void *stream);

/* Per-kernel device time, measured with CUDA events recorded on the launching
 * stream around every launch while timing is enabled.  Kernel classes: */
#define MC_K_SWEEP_DIRECT 0  /* the direct sweep kernel (one launch per mc_sweep) */
#define MC_K_TC_FIELD 1      /* tensor-core window field (one launch per window) */
#define MC_K_WINDOW_STEPS 2  /* sequential sub-steps of a window */
#define MC_K_FULL_FIELD 3    /* FP32 full field (energy anchor, windowed FP32 path) */
#define MC_K_SPEC_FIELD 4    /* spectral path: field spectra of a window's offsets (one launch per window) */
#define MC_K_SPEC_UPDATE 5   /* spectral path: a window's sub-steps (inverse DFT, update, DFT of the updated sub-lattice) */
#define MC_K_TC_REDUCE 6     /* retired: the split-K sum now runs inside the sub-step kernel (no launches) */
#define MC_NKCLASS 7
typedef struct mc_timing {
    int64_t launches[MC_NKCLASS];
    double ms[MC_NKCLASS];
} mc_timing;

/* Enable (1) or disable (0) kernel timing; both reset the accumulated times. */
int mc_set_timing(mc_lattice *lat, int enable);

/* Accumulated kernel times since the last mc_set_timing (synchronises the device). */
int mc_get_timing(mc_lattice *lat, mc_timing *out);

/* SM clock cycles of the windowed paths' sub-step kernel while timing was enabled,
 * averaged over its CTAs and launches: out[0] per decision block of 16 sites (the
 * sequential part), out[1] the set-up before the first block, out[2] the tail
 * after the last block (write-back, spectra, energy, observables), out[3] blocks
 * per launch.  Zeros when nothing was timed.  Synchronises the device. */
int mc_get_window_cycles(mc_lattice *lat, double *out);

/*
 * Update spacing for a stated error (Sec. 3.2).  The flip probability of the
 * simultaneous update errs by about eps/T with eps = 2 C_D sum_{v != 0} |l v|^-3
 * = 2 C_D 9.033621683 / l^3 (D = 2, summed over the update sublattice l Z^2 and
 * its images).  Returns in *l_out the smallest l >= 2 dividing L with
 * eps/T_min <= max_error (most simultaneous sites), or L if none is smaller.
 */
int mc_choose_spacing(int L, double C_D, double T_min, double max_error, int *l_out);

/*
 * Autotuner: times every supported field path (and, for the tensor path, window
 * sizes of 32, 64 and 128 sub-steps) for nsweeps_trial sweeps on this handle,
 * restoring the state after each trial (checkpoint/restore), and keeps the
 * fastest.  When the tensor path wins, its launch shapes (mc_tuning: split-K
 * K-blocks per unit, N-tile, sub-step warp layout) are then tuned one at a time
 * the same way.  The chosen path and window are returned (either pointer may be
 * NULL); mc_get_tuning gives the rest.  Synchronises the device.
 */
int mc_autotune(mc_lattice *lat, int nsweeps_trial, void *stream, int *path_out, int *window_out);

/*
 * Launch shapes of the windowed tensor path (none changes what is computed; the
 * split-K shape changes the FP32 summation order, so trajectories under
 * different shapes agree to rounding, not bit for bit):
 *   window        sub-steps per window (as mc_set_window; 0 = automatic)
 *   tc_kblocks    K-blocks of 32 per split-K unit of the tensor-core contraction
 *                 (0 = automatic: the fewest whose units fit one wave of SMs)
 *   tc_ntile      replicas per N-tile of the contraction, a multiple of 16 in
 *                 [16, 256] (0 = automatic: 256, or all replicas when fewer)
 *   steps_layout  warp roles of the sub-step kernel under the permutation
 *                 schedule: 0 = one decider warp and seven helper warps; 1 = the
 *                 helper that shares the decider's SM sub-partition stays idle
 *                 during the blocks (six helpers); 2 = as 1, and the CTAs of every
 *                 second wave of SMs decide on another sub-partition, so that two
 *                 CTAs sharing an SM do not decide on the same one
 * mc_set_tuning checks the fields and keeps them; mc_get_tuning returns them.
 * mc_autotune searches them for the tensor path and leaves the fastest set.
 */
typedef struct mc_tuning {
    int window;
    int tc_kblocks;
    int tc_ntile;
    int steps_layout;
} mc_tuning;
int mc_set_tuning(mc_lattice *lat, const mc_tuning *t);
int mc_get_tuning(mc_lattice *lat, mc_tuning *out);

/* Sweep counter (index of the next sweep; the RNG counters depend on it). */
int mc_get_sweep_counter(mc_lattice *lat, uint64_t *out);

/*
 * Checkpoint: serialise the complete state (sizes, seed, sweep counter,
 * parameters, spins, tracked energy, observable accumulators) into buf.  Call
 * with buf = NULL to get the size in *len.  Resuming with mc_restore on a handle
 * of the same L, l, R continues the run bit-exactly (the RNG is counter-based).
 * mc_restore replaces the handle's seed, sweep counter, parameters, proposal kind,
 * cone and site schedule with the checkpoint's, whatever the handle ran before;
 * the handle's W~ must already match the checkpoint's (mc_precompute_W with the
 * same cutoff and tail, else MC_ENOTREADY).  A buffer that is too short or not a
 * checkpoint of this library gives MC_EINVAL and leaves the handle unchanged.
 */
int mc_checkpoint(mc_lattice *lat, void *buf, size_t *len);
int mc_restore(mc_lattice *lat, const void *buf, size_t len);

/*
 * Total energy of caller-provided spin states without allocating device memory.
 * The paper has no counterpart: this entry point exists for callers that cannot
 * call cudaMalloc -- code that runs inside a device-memory budget owned by
 * someone else (a framework's caching allocator, a serving process that reserves
 * all device memory up front) or on latency-critical paths where an allocation
 * would synchronise the device.  It computes the same energies as mc_energy, but
 * needs no lattice handle and allocates nothing: the field it needs between its
 * two kernels lives in a fixed 4 MiB array in device memory that every GPU which
 * loads the library holds until the process exits.
 *   L, R       lattice size and number of states, 2 <= L <= 4096, 1 <= R <= 65535,
 *              with R * 3 * L * L <= 1048576 (e.g. R <= 85 at L = 64, R <= 5 at
 *              L = 256); larger requests fail with MC_EINVAL, whose message names
 *              the bound that was exceeded (and the largest R for this L).
 *   W32        device, [4][L][L] FP32 replica-summed tensor (as from mc_get_W, cast).
 *   spins      device, [R][3][L][L] FP32.
 *   couplings  device, [R][4] FP32: J, C_D, K2, K4 of each state.
 *   energy     device, [R] FP64 output: total energy of each state.
 *   stream     cudaStream_t (NULL = legacy default stream); work is enqueued, not
 *              synchronised.
 * The first call on a device looks up the array's device address; make that
 * first call before any stream capture.  All calls share the one array: calls
 * whose work overlaps on the GPU (different streams, or several threads) race
 * and must be serialised by the caller.  Nothing from an earlier call is read.
 */
int mc_energy_noalloc(int L, int R, const float *W32, const float *spins, const float *couplings,
                      double *energy, void *stream);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of simulation requests.  The paper runs one    */
/* lattice at a time and has no counterpart; a request is one run of Sec. 4's  */
/* model (L, couplings, temperature, sweeps) with its own seed.                */
/* ------------------------------------------------------------------------ */
#define MC_REQ_QUEUED 0
#define MC_REQ_RUNNING 1
#define MC_REQ_DONE 2
#define MC_REQ_FAILED 3
#define MC_REQ_RELEASED 4

typedef struct mc_request {
    int L, l;                /* l = 0: chosen by mc_choose_spacing at the server's error bound */
    int replicas;            /* < 1 means 1; replica r draws the counters of replica r of a lone handle */
    double J, C_D, K2, K4, T;
    int64_t sweeps;
    int measure_every;       /* observables every this many sweeps (0 = none); results match a lone
                                run whose mc_sweep calls are multiples of it */
    uint64_t seed;
    int init_mode;           /* 0 random on S^2 from the seed, 1 all +z, 3 random Ising (as mc_init_spins) */
    int image_cutoff;        /* A of mc_precompute_W; 0 = 64 (tail correction on) */
    int proposal;            /* 0 cap of half-angle cone (0 = 0.5 rad), 1 uniform on S^2, 2 reversal */
    double cone;
} mc_request;

typedef struct mc_request_info {
    int state, l, path;
    int packed;                         /* 1 = shares packed launches with other requests */
    int64_t sweeps_done;
    double t_submit, t_admit, t_done;   /* seconds on the host's monotonic clock */
    size_t bytes;                       /* device bytes attributed to it while admitted */
    char error[160];
} mc_request_info;

typedef struct mc_server_stats {
    int queued, running, done, failed;
    int packs, lone;                    /* device handles held: packs and lone handles */
    int64_t completed;
    size_t bytes_in_use, budget;
    int64_t grouped_launches;           /* launches that ran direct packs of different L together */
} mc_server_stats;

typedef struct mc_server mc_server;

/* Device bytes of a handle of `replicas` lattices L x L at spacing l on the path
 * that (L, l) resolves to automatically (the server's admission estimate). */
int mc_footprint(int L, int l, int replicas, size_t *bytes);

/*
 * Requests whose (L, l) the direct path serves, with L < 128, share packed launches: one handle
 * whose replica slots belong to different requests, each slot with its own seed,
 * sweep counter and sweep budget, so that a request's result is bit-identical to
 * the same request run alone on a lone handle (mc_create_lattice with its seed,
 * mc_set_params, mc_precompute_W(A, 1), mc_init_spins, mc_sweep).  Direct packs of
 * different L with the same L / l, proposal and measurement interval whose busy
 * slots fit one resident wave together run as one launch (as mc_sweep_group),
 * still bit-identical to each request's lone run.  Other lattices (L >= 128, or
 * (L, l) outside the direct path) share spectral packs, else FFT packs, whose
 * launches run all slots' sub-steps together, again bit-identical to each request's
 * lone run on that path.  A request that fits no pack gets a lone handle of its own.
 * Packs and lone handles run on separate streams and overlap.
 *
 * Requests are admitted in arrival order while the device bytes of the handles
 * they need fit hbm_budget_bytes and fewer than max_active are running; a packed
 * request waits only for free slots.  Sweeps are issued in quanta of at most
 * quantum_sweeps; a request joins or leaves a pack between quanta.  max_error is
 * the flip-probability error bound (Sec. 3.2) used when a request leaves l = 0: the
 * smallest l within the bound that the direct pack serves, else the smallest that
 * any pack serves (a larger l only lowers the error).
 * The server is single-threaded: call every function from one host thread.
 */
int mc_server_create(size_t hbm_budget_bytes, int max_active, int quantum_sweeps, double max_error,
                     mc_server **out);
/* Queue a request (copied).  MC_EINVAL for bad fields, MC_ENOMEM if it can never fit. */
int mc_server_submit(mc_server *srv, const mc_request *req, uint64_t *id);
/* One scheduling pass: retire finished launches (finished requests are read back
 * to host memory and free their device memory), admit waiting requests, launch
 * the next quantum everywhere idle.  Does not wait for the GPU except to read the
 * results of a request that just finished; call it repeatedly. */
int mc_server_step(mc_server *srv);
/* State (MC_REQ_*) and sweeps completed of a request; either pointer may be NULL.
 * MC_EINVAL for an id the server never handed out. */
int mc_server_poll(mc_server *srv, uint64_t id, int *state, int64_t *sweeps_done);
/* State, chosen spacing and path, packing, submit/admit/done times (steady clock, s),
 * device bytes and the failure reason of a request. */
int mc_server_request_info(mc_server *srv, uint64_t id, mc_request_info *out);
/* Observables of one replica of a DONE request (as mc_observables).  MC_ENOTREADY otherwise. */
int mc_server_collect(mc_server *srv, uint64_t id, int replica, mc_obs *out);
/* Final spins of a DONE request, [replicas][3][L][L] FP32, to a host pointer. */
int mc_server_get_spins(mc_server *srv, uint64_t id, float *dst_host);
/* Drop a request in any state: a queued or running one stops (its slots are
 * refilled only behind the launch that still carries it); its results and its record
 * are freed.  Its id then polls as MC_REQ_RELEASED with 0 sweeps done, collecting from
 * it gives MC_ENOTREADY, and releasing it again is a no-op. */
int mc_server_release(mc_server *srv, uint64_t id);
/* Counts of requests by state, packs and lone handles held, device bytes in use. */
int mc_server_get_stats(mc_server *srv, mc_server_stats *out);
/* Wait for the server's launches, free its handles and memory.  NULL is a no-op. */
int mc_server_destroy(mc_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* DIPMC_H */
