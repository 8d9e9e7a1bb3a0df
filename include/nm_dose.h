/*
 * nm_dose.h -- C ABI of the GB300 (sm_103a) Monte Carlo internal-dosimetry
 * engine for 18F PET/CT, after ARCHER-NM (Peng et al., arXiv 2111.11687).
 *
 * The engine simulates positron-emitter decays drawn from a PET-derived
 * activity map (§2.1: linear PET -> decay PDF), each giving two back-to-back
 * 0.511 MeV photons (§2.1) plus a locally deposited positron kinetic energy
 * (or, as an option, a positron drawn from the beta+ spectrum and tracked),
 * transports the photons through a CT-derived density/material voxel grid with
 * Compton (Klein-Nishina) and photoelectric events and a 10 keV photon cutoff
 * (§2.1), tallies deposited energy per voxel, and reports the dose-rate map
 * of Eq. 1, its batch uncertainty, and the organ means of Eq. 2 and Eq. 3.
 *
 * Conventions for every entry point:
 *  - Voxel arrays are [nz][ny][nx] with x fastest; spacing is in cm; the grid
 *    origin is its corner; the outside of the grid is vacuum.
 *  - A pointer argument may be host or device memory: the library asks the
 *    CUDA runtime which it is.  Inputs are copied before the call returns, so
 *    the caller may free them afterwards.  Outputs are allocated by the caller.
 *  - Every call returns an nm_status; nothing aborts, traps or asserts.  On an
 *    error, nm_last_error() returns a message for the calling thread.
 *  - Device work is ordered on the stream given in nm_options (NULL = the
 *    legacy default stream); calls that return data synchronise that stream.
 *  - Energies are tallied in int64 fixed point, one unit = 2^-6 eV, and each
 *    deposit is a difference of fixed-point energies, so a fixed seed gives
 *    bit-identical tallies run to run whatever the scheduling.
 */
#ifndef NM_DOSE_H
#define NM_DOSE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NM_MAX_MATERIALS 8  /* material ids 0..7 */
#define NM_MAX_LABELS 31    /* organ labels 1..31; 0 = outside every organ */
#define NM_UNITS_PER_MEV 64000000.0 /* tally unit: 2^-6 eV */

typedef struct nm_dose nm_dose; /* opaque handle; owns all its device memory */

typedef enum {
  NM_OK = 0,
  NM_ERR_ARG = 1,      /* invalid argument: sizes, NaN/negative inputs, ... */
  NM_ERR_CUDA = 2,     /* a CUDA runtime call failed */
  NM_ERR_OOM = 3,      /* device allocation failed */
  NM_ERR_OVERFLOW = 4, /* the int64 tallies could overflow */
  NM_ERR_TIMEOUT = 5,  /* a bounded device wait gave up */
  NM_ERR_STATE = 6,    /* call not valid in the handle's state */
  NM_ERR_DEVICE = 7    /* a device-side check failed (see nm_last_error) */
} nm_status;

enum { NM_SOURCE_DECAY = 0, NM_SOURCE_POINT = 1 };

/* Voxel phantom (§2.1: CT -> mass density and material per voxel). */
typedef struct {
  int32_t nx, ny, nz;        /* voxels; nx*ny*nz < 2^31 */
  float dx, dy, dz;          /* voxel size, cm, > 0 */
  const float* density;      /* g/cm^3, finite, > 0, [nz][ny][nx] */
  const uint8_t* material;   /* material id < materials.n, [nz][ny][nx] */
} nm_grid;

/* Photon interaction data (§2.1: photoelectric and Compton explicit, pair
 * production absent below 1.02 MeV).  Per material m:
 *   mu_compton = rho N_A (Z/A)_m sigma_KN(E)           (Klein-Nishina)
 *   mu_photo   = rho pe_coeff Zeff_m^pe_exp / E^3       (E in MeV)
 *   mu_rayl    = rho rayleigh_coeff Zeff_m^2 / E^2      (only if rayleigh != 0)
 * with linear attenuation in 1/cm. */
typedef struct {
  int32_t n;                 /* materials, 1..NM_MAX_MATERIALS */
  const double* z_over_a;    /* [n] host pointer */
  const double* zeff;        /* [n] host pointer */
  double pe_coeff;           /* cm^2/g MeV^3 */
  double pe_exp;             /* 3.8 */
  double rayleigh_coeff;     /* cm^2/g MeV^2 */
  int32_t rayleigh;          /* 0 = off (the paper's physics) */
  double photon_cut_mev;     /* 0.010 (§2.1) */
  double electron_cut_mev;   /* 0.200 (§2.1); recorded, electrons deposit locally */
} nm_materials;

typedef struct {
  int32_t source_mode;       /* NM_SOURCE_DECAY (activity map) or NM_SOURCE_POINT */
  float point[3];            /* cm, point mode: one photon per history from here */
  double photon_mev;         /* 0.511 */
  double positron_mev;       /* positron energy deposited at the decay, 0.25 */
  int32_t batches;           /* batches per nm_dose_run call, >= 1 (default 10); the uncertainty
                                needs two batches in total, over one call or several */
  double activity_bq;        /* A(t_s) of Eq. 1, Bq */
  int32_t n_labels;          /* organs 1..n_labels in the label map (0 = none) */
  int32_t block_threads;     /* transport CTA size; 0 = autotuned */
  int32_t chunk;             /* histories per warp work grab; 0 = autotuned */
  int32_t warp_aggregate;    /* warp-aggregated tally atomics: -1 auto, 0 off, 1 on */
  int32_t regroup;           /* event regrouping in the transport: -1 auto, 0 off, 1 on */
  int32_t regroup_lanes;     /* lanes of a warp that must wait for a Compton or a
                                new-history pass before it runs (1..32); 0 = auto */
  int32_t max_steps;         /* per-photon flight-step limit (bounded loops) */
  void* stream;              /* cudaStream_t; NULL = legacy default stream */
  int32_t history_sigma;     /* 1: also keep history-by-history statistics (the paper's
                                uncertainty method, §2.1; +16 B per voxel, no warp
                                aggregation); read with nm_dose_get_history_sigma */
  double beta_max_mev;       /* decay mode.  0 (default): positron_mev is deposited in the
                                decay voxel (§2.1's positron, locally absorbed).  > 0
                                (< 20): the positron's kinetic energy T is drawn from the
                                allowed beta+ spectrum with this endpoint (18F: 0.6335),
                                N(T) ~ F(Z, E) p E (T_max - T)^2 with the non-relativistic
                                Fermi function of a positron, and the positron runs a
                                straight track in an isotropic direction whose mass range
                                (g/cm^2) is Katz-Penfold's R(T) = 0.412 T^(1.265 - 0.0954
                                ln T), each voxel keeping the energy lost in it (the energy
                                at the remaining range), and both photons start where the
                                track ends; a track that leaves the grid takes its energy
                                and both photons out with it.  Not in nm_dose_tally_noalloc. */
  int32_t beta_z;            /* atomic number of the daughter for the Fermi function
                                (18F -> 18O: 8, the default), 0..100 */
  int32_t kn_sampler;        /* Compton angle (Klein-Nishina, §2.1): 0 (default) = inverse
                                CDF tabulated in FP64 at 64 energies x 257 probabilities
                                and interpolated (one draw, CDF error < 2e-5); 1 = Kahn's
                                rejection sampler.  Batched runs need one value for all. */
  /* Other radionuclides (§4 names 177Lu and 131I as the next ones), decay mode.
   * The fields below describe one decay; zero (the default) gives 18F as
   * above.  Not in nm_dose_run_batch or nm_dose_tally_noalloc. */
  int32_t no_annihilation;   /* 0 (default): the positron of each decay annihilates into two
                                back-to-back photons of photon_mev (where its track ends);
                                1: no annihilation photons (a beta- emitter) */
  int32_t beta_electron;     /* 0 (default): the beta particle is a positron; 1: an electron
                                (the Fermi function's sign in its spectrum) */
  int32_t n_beta;            /* 0 (default): one branch with endpoint beta_max_mev; 1..8:
                                branch b has endpoint beta_endpoint_mev[b] (0 < E < 20 MeV)
                                and is taken by a fraction beta_intensity[b] (>= 0, positive
                                sum, normalised) of the decays; the particle is tracked as
                                described under beta_max_mev.  Host arrays. */
  const double* beta_endpoint_mev;
  const double* beta_intensity;
  int32_t n_gamma;           /* 0..8 gamma lines: line j of gamma_mev[j] MeV (above the
                                photon cutoff, at most 1 MeV) leaves the decay site (the
                                nucleus, not the end of the beta track) with probability
                                gamma_yield[j] (0..1) per decay, independently of the other
                                lines, in an isotropic direction.  Host arrays. */
  const double* gamma_mev;
  const double* gamma_yield;
} nm_options;

typedef struct {
  uint64_t histories;        /* histories simulated so far */
  uint64_t batches;          /* batches folded so far */
  int64_t emitted;           /* energy units emitted by all histories */
  int64_t deposited;         /* energy units in the tally */
  int64_t escaped;           /* energy units carried out of the grid */
  int64_t killed;            /* energy units of photons stopped by max_steps */
  uint64_t steps;            /* flight steps (real + virtual) */
  uint64_t compton, photo, rayleigh, cutoff, escapes;
  double transport_ms;       /* device time of the transport launches: per run call, from the first
                                batch's start to the last transport's end (consecutive batches
                                overlap on two streams, folds between them inside the span) */
  double fold_ms;            /* device time of the batch folds (a fold waits for SMs while the other
                                stream's transport holds them: an upper bound) */
  uint32_t device_status;    /* OR of NM_DEV_* flags seen */
  int32_t block_threads, chunk, warp_aggregate, regroup, regroup_lanes, grid_blocks; /* tuning used */
  uint64_t history_splits;   /* history_sigma: histories whose deposits touched more voxels
                                than a lane keeps (their totals were squared in parts) */
} nm_counters;

#define NM_DEV_STEP_LIMIT 1u   /* a photon hit max_steps */
#define NM_DEV_KAHN_LIMIT 2u   /* Kahn sampling hit its trial limit */
#define NM_DEV_BAD_VOXEL 4u    /* material id out of range, density not > 0 */
#define NM_DEV_BAD_ACTIVITY 8u /* activity negative or not finite */
#define NM_DEV_TIMEOUT 16u     /* a bounded wait on the tensor cores gave up */
#define NM_DEV_RAYLEIGH_LIMIT 32u /* the Rayleigh (Thomson) angle hit its trial limit */

/* Fills *o with the defaults: decay mode, 0.511 MeV photons, 0.25 MeV positron,
 * 10 batches, A(t_s) = 8.0 mCi decayed 60 min with T1/2 = 109.77 min (§2.2),
 * autotuned launch shape, max_steps 100000, legacy default stream. */
void nm_options_default(nm_options* o);

/* §2.1 CT -> phantom: HU to mass density by the piecewise-linear curve through
 * (HU, g/cm^3) = (-1000, 0.0012), (-750, 0.26), (-100, 0.95), (40, 1.03),
 * (1000, 1.85), clamped at both ends, computed in FP32; material = the node
 * nearest in HU, ties to the lower node (0 air, 1 lung, 2 adipose, 3 soft
 * tissue, 4 bone), decided in integer arithmetic.  hu[n] in; density[n],
 * material[n] out (host or device).  n >= 0. */
nm_status nm_ct_to_phantom(const int16_t* hu, int64_t n, float* density, uint8_t* material,
                           void* stream);

/* Creates a simulation handle (§2.1).  grid, materials: as above.  activity:
 * [V] decay density (the PET value, Bq/mL; linear -> decay PDF), >= 0 and
 * finite with a positive sum, required in decay mode, ignored (may be NULL) in
 * point mode.  labels: [V] organ ids 0..opts->n_labels, or NULL.  opts: NULL =
 * defaults.  The activity is turned into an alias table on the device in FP64.
 * All inputs are copied.  Errors: NM_ERR_ARG for invalid sizes or values,
 * NM_ERR_OOM, NM_ERR_CUDA; *out is NULL on error. */
nm_status nm_dose_create(nm_dose** out, const nm_grid* grid, const nm_materials* materials,
                         const float* activity, const uint8_t* labels, const nm_options* opts);

/* Simulates n_decays more histories (§2.1-2.2) in opts.batches batches of
 * near-equal size, folding each batch into the statistics.  History ids
 * continue across calls and every history's random numbers depend only on
 * (seed, history id) (Philox4x32-10), so the tally after run(a) + run(b) is
 * bit-identical to run(a + b); the batch uncertainty depends on the split.
 * NM_ERR_OVERFLOW if the cumulative tally could exceed 2^63 units;
 * NM_ERR_DEVICE if a device check fired (the batch is still folded). */
nm_status nm_dose_run(nm_dose* h, uint64_t n_decays, uint64_t seed);

/* Many patients in one launch (the paper runs one patient at a time; this is
 * the batched form of nm_dose_run).  Runs n_decays[i] more histories on each
 * handle hs[i] (i < n <= 64) with seed `seed`, in the handles' common number
 * of batches: per batch one persistent transport launch whose warps drain
 * per-patient work queues, moving to the next patient when one runs dry, then
 * every patient's fold; all batches are captured into one CUDA graph and
 * launched once on the first handle's stream.  Handles must be distinct and
 * share materials, energies, batches, max_steps and device; grids may differ.
 * Each handle's tally is bit-identical to nm_dose_run(hs[i], n_decays[i],
 * seed).  The launch shape is the first handle's explicit options, else
 * chosen by timed trials on the batch (cached per batch geometry).  Errors as
 * for nm_dose_run; NM_ERR_ARG for mismatched handles. */
nm_status nm_dose_run_batch(nm_dose* const* hs, int32_t n, const uint64_t* n_decays, uint64_t seed);

/* Eq. 1: dose rate D/N_evts * A(t_s) per voxel (Gy/s) into dose[V], and the
 * batch standard deviation of that mean into sigma[V] (Gy/s); either may be
 * NULL.  organ_dose[n_labels + 1]: Eq. 2 organ means (index = label; index 0
 * is the mean outside all organs), may be NULL.  NM_ERR_STATE before any run
 * (and, when sigma or organ_dose is asked for, before two batches).  The dose
 * alone (sigma and organ_dose NULL) takes one streaming pass and is
 * bit-identical to the dose written with them. */
nm_status nm_dose_get(nm_dose* h, float* dose, float* sigma, double* organ_dose);

/* Per organ label 0..n_labels (arrays of n_labels + 1 doubles, any may be
 * NULL): Eq. 2 mean dose rate (Gy/s), Eq. 3 RMS of the voxels' relative
 * uncertainties (a voxel with zero dose counts as 1), batch standard deviation
 * of the organ mean (Gy/s), and the organ's voxel count.  Without eps_rms (and
 * with a label map) no pass over the voxels is made: the mean and its sigma
 * come from the per-organ batch sums the fold keeps (the same FP32 voxel
 * doses, summed per batch in FP64), equal to the full pass's to ~1e-7
 * relative; cheap enough to poll while a run converges. */
nm_status nm_dose_get_organs(nm_dose* h, double* mean, double* eps_rms, double* sigma_mean,
                             int64_t* voxels);

/* Eq. 2 over any dose map of the handle's grid (e.g. a denoised one): the
 * unweighted mean of dose[V] (host or device FP32) over each label's voxels,
 * into mean[n_labels + 1] (host or device).  NM_ERR_STATE without labels. */
nm_status nm_dose_map_organs(nm_dose* h, const float* dose, double* mean);

/* Multi-time-point dosimetry (§4: dose over time from activity measured at
 * several time points).  act[k] (k < n_points <= 16) are activity maps [V]
 * (Bq per voxel, host or device) measured at times t_h[k] (hours, 0 <= t_0 <
 * t_1 < ...); out[V] (host or device) receives each voxel's time-integrated
 * activity, the number of decays from injection (t = 0) on, in Bq s:
 *   uptake before t_0 as a linear rise from 0:   A_0 t_0 / 2,
 *   between time points by the trapezoid rule:   (A_k + A_k+1)(t_k+1 - t_k) / 2,
 *   after the last point by physical decay only: A_n T_1/2 / ln 2,
 * times 3600 s/h, in FP64, rounded to FP32 at the end.  *total (may be NULL)
 * is the FP64 sum over voxels.  Used as a decay map with activity_bq =
 * *total, nm_dose_get then gives the absorbed dose (Gy) instead of the dose
 * rate.  NM_ERR_ARG for negative or non-finite activities, times out of
 * order, or a half-life that is not > 0. */
nm_status nm_time_integrated_activity(const float* const* act, const double* t_h, int32_t n_points, int64_t V,
                                      double half_life_h, float* out, double* total, void* stream);

/* Exact cumulative tally, int64 energy units per voxel, into tally[V]. */
nm_status nm_dose_get_tally(nm_dose* h, int64_t* tally);

/* History-by-history sigma of the mean dose rate (Gy/s, [V], host or device),
 * §2.1's method (Walters et al. 2002): every history's total deposit per voxel
 * is squared into an exact 128-bit integer sum, and
 *   sigma = sqrt((S2/N - (T/N)^2) / (N - 1)) in dose-rate units.
 * Needs a handle created with history_sigma = 1 (else NM_ERR_STATE).  A
 * history that deposits in more than 16 voxels has its totals squared in
 * parts (counted in nm_counters.history_splits). */
nm_status nm_dose_get_history_sigma(nm_dose* h, float* sigma);

/* Sets the id of the next history (default 0; nm_dose_run and
 * nm_dose_run_batch continue from it).  A history's random numbers depend
 * only on (seed, id), so shards of one run on several devices or processes
 * take disjoint id ranges [first, first + n) and their merged statistics
 * (nm_dose_merge) equal those of one handle that ran the ranges in turn: the
 * tally and counters bit for bit.  Ids above 2^62 are reserved
 * (NM_ERR_ARG).  Nothing checks that ranges do not overlap. */
nm_status nm_dose_seek(nm_dose* h, uint64_t next_history_id);

/* Checkpoints of a handle's statistics (the exact cumulative tally of Eq. 1,
 * the batch sums behind the uncertainty, the organ sums, counters, the
 * history count, the next history id and, with history_sigma, the 128-bit
 * sums of squared history totals) as one flat byte image that the caller
 * owns, in host or device memory (found with pointer attributes).
 * nm_dose_checkpoint_size gives its size for h; nm_dose_checkpoint writes it
 * (NM_ERR_ARG if `bytes` is smaller).  The image holds no pointers: it can be
 * written to a file or sent to another process. */
nm_status nm_dose_checkpoint_size(const nm_dose* h, uint64_t* bytes);
nm_status nm_dose_checkpoint(nm_dose* h, void* buf, uint64_t bytes);

/* Replaces h's statistics by an image from a handle with the same grid,
 * label slots and history_sigma option (else NM_ERR_ARG; nothing changes);
 * runs then continue exactly as on the handle that wrote it. */
nm_status nm_dose_restore(nm_dose* h, const void* buf, uint64_t bytes);

/* Adds another shard's image (same grid and options, disjoint history ids)
 * to h: tallies, counters and 128-bit sums add exactly, the FP64 batch and
 * organ sums add (the shards' batches are batches of the combined run),
 * history and batch counts add, the next id becomes the larger of the two.
 * A host image is staged through a temporary device buffer.  NM_ERR_ARG on a
 * mismatched image, NM_ERR_OVERFLOW if the merged tally could exceed 2^63
 * units. */
nm_status nm_dose_merge(nm_dose* h, const void* buf, uint64_t bytes);

/* Counters and the launch shape in use. */
nm_status nm_dose_counters(nm_dose* h, nm_counters* c);

/* Forgets all histories and statistics (history ids restart at 0). */
nm_status nm_dose_reset(nm_dose* h);

/* Frees the handle and its device memory.  NULL is allowed. */
void nm_dose_destroy(nm_dose* h);

/* Message of the last error on the calling thread ("" if none). */
const char* nm_last_error(void);

/* ---- Checks of the device building blocks (used by the test suite) ------- */

/* Philox4x32-10 (Salmon et al., SC'11) evaluated by the device code for n
 * (counter, key) pairs: ctr[4n], key[2n] in, out[4n] out; host pointers. */
nm_status nm_check_philox(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out);

/* n Klein-Nishina scattering cosines at energy e_mev drawn by the device's
 * Kahn sampler with key (seed) and counters 0..n-1; cos_out[n] host. */
nm_status nm_check_kahn(double e_mev, int64_t n, uint64_t seed, float* cos_out);

/* n scattering cosines at energy e_mev drawn by the transport's tabulated
 * Klein-Nishina sampler (kn_sampler = 0) built for photons between cut_mev
 * and e0_mev, key (seed), counters 0..n-1; cos_out[n] host. */
nm_status nm_check_kn_table(double e_mev, double cut_mev, double e0_mev, int64_t n, uint64_t seed,
                            float* cos_out);

/* Device memory released by destroyed handles and by the library's per-call
 * temporaries is kept (up to 8 GiB, per device and buffer size) and handed to
 * the next allocation of the same size on the same device, so that a handle
 * created after one of the same grid maps no new memory.  This call returns
 * every kept buffer to the device (cudaFree); buffers of live handles are not
 * affected.  A failed allocation releases them by itself before it retries.
 * Safe to call at any time from any thread.  Kept buffers belong to the
 * device's context: destroy the handles and call this before cudaDeviceReset
 * or anything else that ends the primary context, whose memory (kept buffers
 * included) does not outlive it. */
void nm_release_cached_memory(void);

/* Fault injection: the n-th device allocation made by the library from now
 * on (nm_dose_create and the calls it makes) fails as if the device were out
 * of memory; 0 switches it off.  The failing call returns NM_ERR_OOM and frees
 * what it had allocated. */
void nm_debug_fail_alloc(int32_t n);

/* Runs one bounded device wait on an mbarrier that nothing completes (the
 * wait of the tensor-core kernels) with a limit of max_cycles SM clocks:
 * returns NM_ERR_TIMEOUT once it gives up; the context stays usable. */
nm_status nm_check_wait_timeout(int64_t max_cycles);

/* n positron kinetic energies (MeV) as the transport draws them in the beta+
 * spectrum mode (beta_max_mev = t_max_mev, beta_z = z), for histories 0..n-1
 * with key (seed): inverse-CDF table built in FP64 on the host, linear between
 * its kBetaTable = 1024 nodes.  t_out[n] host. */
nm_status nm_check_beta(double t_max_mev, int32_t z, int64_t n, uint64_t seed, float* t_out);

/* The handle's alias table: n_active entries of (prob, voxel, alias voxel).
 * Pass NULL arrays to query *n_active only.  Host pointers. */
nm_status nm_dose_alias_table(nm_dose* h, int64_t* n_active, float* prob, int32_t* voxel,
                              int32_t* alias_voxel);

/* Decay sites of histories first..first+n-1 with the handle's source sampler:
 * voxel[n], pos[3n] (cm), dir[3n] (first photon); host pointers. */
nm_status nm_check_source(nm_dose* h, uint64_t first, int64_t n, uint64_t seed, int32_t* voxel,
                          float* pos, float* dir);

/* ---- Ceilings of this GPU for the transport's roofline --------------------
 *
 * The paper has no counterpart (it quotes wall times only); these measure
 * the two hardware rates the transport's memory traffic is bounded by, for
 * which no published GB300 figure exists.  Each allocates its own buffer,
 * runs one untimed warm-up launch and one launch timed with CUDA events on a
 * private stream of the current device, and frees the buffer. */

/* L2 read bandwidth: every thread streams 16-byte words of a bytes-long
 * buffer (1 MiB .. 2 GiB, a multiple of 16; below the L2's size for an L2
 * figure) reps times (1..1000) with L2-only loads.  *gb_per_s = bytes * reps
 * / time / 1e9. */
nm_status nm_probe_l2_read(int64_t bytes, int32_t reps, double* gb_per_s);

/* Scattered 64-bit atomic adds with unused results (the form of the tally
 * deposits): about `ops` adds (2^20 .. 2^34) of 1 to slots of a buffer of
 * `slots` 8-byte words (a power of two, 2^10 .. 2^28) picked by a per-thread
 * xorshift generator.  *ops_per_s = adds / time. */
nm_status nm_probe_atomic_add_u64(int64_t slots, int64_t ops, double* ops_per_s);

/* ---- 3x3x3 convolutions of the dose denoiser (tensor cores, BF16 in, FP32 accumulate)
 *
 * The denoiser (a 3D U-Net) is not in the paper; these are its building blocks.
 * Volumes are channels-last BF16 (raw 16-bit patterns), [n][d][h][w][c].  The
 * input of a convolution is the channel concatenation of source 0 (c0
 * channels; at half resolution, read with nearest upsampling, when
 * src0_coarse != 0) and source 1 (c1 channels, full resolution, may be
 * absent with c1 = 0).  Stride 1, zero padding 1.  Weights are BF16
 * [cout][nm_conv3d_kpad(c0 + c1)] with column k = tap * (c0 + c1) + ci,
 * tap = (dz+1)*9 + (dy+1)*3 + (dx+1), and zeros past 27 taps.  All pointers are
 * device memory and 16-byte aligned; c0, c1 multiples of 8; cout one of
 * 16, 32, 48, 64, 96, 128, 192 (weight gradients: 16, 32, 64, 128).  The
 * calls run on `stream` and synchronise it; NM_ERR_DEVICE on a tensor-core
 * wait time-out. */
typedef struct {
  int32_t n, d, h, w;   /* output grid: batch and (fine) spatial size */
  int32_t c0, c1;       /* input channels from source 0 and source 1 */
  int32_t src0_coarse;  /* source 0 is at half resolution */
  int32_t cout;         /* output channels */
} nm_conv3d_desc;

/* Padded GEMM depth of a convolution with cin input channels (27 cin rounded
 * up to a multiple of 128). */
int32_t nm_conv3d_kpad(int32_t cin);

/* y = act(conv(x) + bias): act = ReLU if relu != 0; bias [cout] FP32 or NULL. */
nm_status nm_conv3d_fwd(const nm_conv3d_desc* desc, const uint16_t* x0, const uint16_t* x1,
                        const uint16_t* w, const float* bias, uint16_t* y, int32_t relu,
                        void* stream);

/* Input gradient: dx[n][d][h][w][c0 + c1] (BF16, before any mask) of the
 * convolution `desc` for the output gradient dy[n][d][h][w][cout]; dx is at
 * full resolution for both sources (the caller sums source 0 back to half
 * resolution).  c0 + c1 must be one of the output channel counts above. */
nm_status nm_conv3d_dgrad(const nm_conv3d_desc* desc, const uint16_t* dy, const uint16_t* w,
                          uint16_t* dx, void* stream);

/* Weight and bias gradients: dw[cout][kpad] (FP32) = sum over voxels of the
 * im2col rows of the input times dy; db[cout] (FP32, may be NULL) = sum of
 * dy.  Deterministic: split over voxel ranges, summed in a fixed order. */
nm_status nm_conv3d_wgrad(const nm_conv3d_desc* desc, const uint16_t* x0, const uint16_t* x1,
                          const uint16_t* dy, float* dw, float* db, void* stream);

/* ---- Dose denoiser: 3D U-Net trained and applied on the GPU ------------------
 *
 * Not in the paper.  A U-Net of `levels` levels with widths base_width * 2^i
 * (default 4 levels, 16..128), two 3x3x3 convolutions with ReLU per level,
 * 2x2x2 average pooling down, nearest upsampling concatenated with the skip
 * up, and a 1x1x1 head added to input channel 0.  Inputs are BF16 [batch][P]
 * [P][P][8]: channel 0 = low-count dose / s, 1 = density, 2 = activity / a,
 * 3 = activity / (a max(density, 0.1)), 4..7 = 0, where s and a are the body
 * means (density >= 0.1) of the low-count dose and of the activity; the output
 * and training target are dose / s (linear, so that the squared-error optimum
 * is the conditional mean and organ means are not biased).  Weights: FP32 master copy updated by Adam,
 * BF16 copy for the convolutions; all convolutions on the tensor cores. */
typedef struct {
  int32_t patch;       /* P, a multiple of 2^(levels-1) (default 64) */
  int32_t batch;       /* patches per step (default 2) */
  int32_t levels;      /* 2..4 (default 4) */
  int32_t base_width;  /* 16 or 32 (default 16) */
  float lr, beta1, beta2, eps;  /* Adam (defaults 1e-3, 0.9, 0.999, 1e-8) */
  uint64_t seed;       /* weight initialisation */
  void* stream;        /* cudaStream_t; NULL = legacy default stream */
  int64_t infer_voxels;  /* voxels of one whole-volume inference pass (default 2^25, >= 4096) */
} nm_denoise_options;

typedef struct nm_denoiser nm_denoiser;

void nm_denoise_options_default(nm_denoise_options* o);
nm_status nm_denoise_create(nm_denoiser** out, const nm_denoise_options* opts);
void nm_denoise_destroy(nm_denoiser* h);

/* Number of FP32 parameters in the flat parameter vector, and the layout of
 * layer i (0 .. 2*(2*levels-1)-1 in forward order e0a e0b e1a ... d0a d0b; i =
 * that count is the head): weights at w_offset as [cout][kpad] with column
 * k = tap * cin + ci, biases at b_offset. */
int64_t nm_denoise_param_count(const nm_denoiser* h);
nm_status nm_denoise_layer(const nm_denoiser* h, int32_t i, int32_t* cin, int32_t* cout, int32_t* kpad,
                           int64_t* w_offset, int64_t* b_offset);

/* Copies the parameters out (get), in (set, also refreshes the BF16 copy)
 * and/or the last step's gradients out (grads); any may be NULL; host or
 * device pointers of nm_denoise_param_count floats. */
nm_status nm_denoise_params(nm_denoiser* h, float* get, const float* set, float* grads);

/* Adam's state (Kingma and Ba, 2015): the first and second moment estimates
 * (nm_denoise_param_count floats each, host or device; either may be NULL) and
 * the number of updates made so far.  After update t with gradient g:
 * m1 = beta1 m1 + (1 - beta1) g, m2 = beta2 m2 + (1 - beta2) g^2, and
 * w -= lr (m1 / (1 - beta1^t)) / (sqrt(m2 / (1 - beta2^t)) + eps). */
nm_status nm_denoise_adam_state(nm_denoiser* h, float* m1, float* m2, int64_t* step);

/* Test support for checking the network layer by layer.  With on != 0 every
 * later train step keeps, for each convolution layer i (0 .. 2*(2*levels-1)-1,
 * forward order), three BF16 tensors: kind 0 its input [batch][s]^3[cin]
 * (s = P >> level; a decoder layer's input as the channel concatenation
 * [nearest-upsampled coarse | skip]), kind 1 its output activation after
 * ReLU [batch][s]^3[cout], kind 2 the loss gradient at its output after the
 * ReLU mask [batch][s]^3[cout].  on = 0 frees them.  nm_denoise_captured
 * copies one out (host or device; NM_ERR_ARG if `bytes` is too small,
 * NM_ERR_STATE with capture off). */
nm_status nm_denoise_capture(nm_denoiser* h, int32_t on);
nm_status nm_denoise_captured(nm_denoiser* h, int32_t layer, int32_t kind, uint16_t* out, int64_t bytes);

/* One training step on device tensors: x [batch][P]^3[8] BF16, target
 * [batch][P]^3 FP32, weight [batch][P]^3 FP32 or NULL (= 1); loss = mean of
 * weight * (y - target)^2 over all voxels (written to *loss, host).  Forward,
 * backward (tensor-core input and weight gradients) and, if lr > 0, an Adam
 * update with learning rate lr. */
nm_status nm_denoise_train_step(nm_denoiser* h, const uint16_t* x, const float* target, const float* weight,
                                float lr, float* loss);

/* Forward only: y [batch][P]^3 FP32 (device). */
nm_status nm_denoise_forward(nm_denoiser* h, const uint16_t* x, float* y);

/* Network inputs (and optionally targets and body weights) for n_patches
 * patches at corners[3*i..] (x, y, z; may lie partly outside the volume,
 * which reads as zero) of whole volumes [nz][ny][nx] (device FP32). */
nm_status nm_denoise_make_patches(const float* dose, const float* density, const float* activity,
                                  const float* dose_high, int32_t nx, int32_t ny, int32_t nz, float dose_scale,
                                  float act_scale, const int32_t* corners, int32_t n_patches, int32_t patch,
                                  uint16_t* x, float* target, float* weight, void* stream);

/* Body means (density >= 0.1) of a dose map and an activity map (device). */
nm_status nm_denoise_scales(const float* dose, const float* activity, const float* density, int64_t n,
                            float* dose_scale, float* act_scale, void* stream);

/* Denoises a whole low-count dose-rate map (device FP32 [nz][ny][nx]) into
 * dose_out (device, same units; may equal dose).  The bounding box of the body
 * (density >= 0.1) plus 8 voxels of context on every side runs through the
 * network as one volume (in slabs along z, each with its own context, when it
 * exceeds infer_voxels); voxels outside the body box keep the input value.  Allocates
 * the forward buffers of that volume once and keeps them with the handle. */
nm_status nm_denoise_apply(nm_denoiser* h, const float* dose, const float* density, const float* activity,
                           int32_t nx, int32_t ny, int32_t nz, float* dose_out);

/* The same over the bounding box of the non-zero voxels of roi (device
 * uint8 [nz][ny][nx], e.g. the organ label map; NULL = the body) plus the 8
 * voxels of context; the scales are still the body means.  Outside that box
 * dose_out keeps the input. */
nm_status nm_denoise_apply_roi(nm_denoiser* h, const float* dose, const float* density, const float* activity,
                               const uint8_t* roi, int32_t nx, int32_t ny, int32_t nz, float* dose_out);

/* ---- Tally without device allocation ---------------------------------------
 *
 * For callers that cannot call cudaMalloc -- code running inside another
 * framework's memory pool or arena, real-time or safety-constrained services
 * that forbid allocation after start-up, hosts that hand the library only
 * pre-allocated buffers.  The paper has no counterpart: it is a deployment
 * variant of nm_dose_create + nm_dose_run + nm_dose_get_tally.
 *
 * Computes the cumulative tally of histories 0..n_decays-1 (seed as in
 * nm_dose_run; bit-identical to a handle's tally after nm_dose_run(n_decays,
 * seed)) into tally[V] (int64 energy units, device memory, overwritten).
 * grid->density, grid->material, activity (decay mode) and tally must be
 * memory of the current device (or managed memory); materials and opts are
 * host structs, checked as nm_dose_create checks them (NM_ERR_ARG before any
 * device work); labels and batch statistics are not part of this call; the
 * beta+ spectrum option is refused.  counters may be NULL; its deposited
 * field is emitted - escaped - killed.
 *
 * All working memory (packed voxels, alias table and its FP64 scans, physics
 * tables, counters) lives in one fixed device array of 24 MiB that every GPU
 * which loads the library holds until the process exits; grids above 2^18
 * voxels (64^3) are rejected with NM_ERR_ARG.  The call allocates no device
 * memory.  Its first call on a device looks up that array's device address
 * (with the device current) and keeps it, keyed by the device's context, so
 * a call after cudaDeviceReset looks it up again; make that first call
 * before any stream capture.  Every call uses the same array, so calls that overlap on
 * the GPU (other streams or threads, the same device) race and must be
 * serialised by the caller; nothing in the array needs clearing between
 * calls.  The call synchronises opts->stream. */
nm_status nm_dose_tally_noalloc(const nm_grid* grid, const nm_materials* materials,
                                const float* activity, const nm_options* opts,
                                uint64_t n_decays, uint64_t seed, int64_t* tally,
                                nm_counters* counters);

#ifdef __cplusplus
}
#endif

#endif /* NM_DOSE_H */
