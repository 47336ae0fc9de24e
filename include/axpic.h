/*
 * axpic.h - C ABI of the GB300 (sm_103a) axion Monte-Carlo operators for
 * particle-in-cell plasmas.
 *
 * The library implements, per cell and per macroparticle, the three axion
 * channels of the paper "An axion framework for Particle-in-Cell codes with
 * Monte-Carlo sampling": screened Primakoff conversion (Sec. II.F), Compton-like
 * photoproduction (Sec. II.G) and electron-ion / electron-electron
 * bremsstrahlung (Sec. II.H), their detailed-balance inverse operators
 * (Sec. II.I), Poisson macro-event sampling with cap-and-rescale variance
 * control (Sec. II.D), and the conservative cell-local energy/momentum
 * feedback with temperature evolution (Sec. II.J).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Units: energies in keV, momenta in m_e c, times in seconds, densities in
 *   cm^-3, volumes in cm^3, couplings g_agg in GeV^-1 and g_ae dimensionless.
 * - Particles live in cell-sorted slabs. Species s of cell c occupies slots
 *   [c*capacity, c*capacity + count[c]) of its two arrays of 16-byte records:
 *   wp holds each slot's weight and momentum {w, px, py, pz}, xyz its
 *   position {x, y, z, unused} as fractions of the cell in [0, 1). capacity
 *   must be a multiple of 4 and both arrays 16-byte aligned.
 * - Pointers marked "device" are CUDA device pointers owned by the caller; the
 *   library never frees them. Pointers marked "host" are read or written
 *   synchronously before the call returns. The library owns only its scratch
 *   (cell records, feedback buffers, counters, tallies) and its sampling
 *   tables, allocated by axpic_init_plasma and released by axpic_destroy.
 * - Step calls (axpic_absorb, axpic_emit, axpic_feedback, axpic_step,
 *   axpic_update_cells, axpic_sample_plasma) only enqueue kernels on the
 *   context's stream: they neither allocate nor synchronise, so a sequence of
 *   them can be captured in a CUDA graph. Arguments are validated on the host
 *   first; an invalid call returns AXPIC_E_INVALID and launches nothing.
 * - Errors found on the device (slab capacity exceeded, non-finite values)
 *   are latched in a device flag and reported by the next synchronising call
 *   (axpic_sync, axpic_tally_spectrum, axpic_destroy).
 * - Random numbers: one Philox4x32-10 stream keyed by the 64-bit seed, with
 *   counter (step, global cell index, particle, stream << 24 | sub), so a
 *   result does not depend on launch shape or on how cells are sharded.
 */
#ifndef AXPIC_H
#define AXPIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct axpic_ctx axpic_ctx; /* opaque; owned by the library */

typedef enum {
  AXPIC_OK = 0,
  AXPIC_E_INVALID = 1,  /* bad argument; nothing was launched */
  AXPIC_E_CAPACITY = 2, /* a slab overflowed; the excess products were dropped */
  AXPIC_E_CUDA = 3,     /* a CUDA runtime call failed */
  AXPIC_E_TIMEOUT = 4,  /* a bounded device wait gave up */
  AXPIC_E_NUMERIC = 5   /* a non-finite value was produced */
} axpic_status;

/* Channel mask bits. */
enum {
  AXPIC_CH_PRIMAKOFF = 1, /* gamma + Z <-> a + Z (Sec. II.F) */
  AXPIC_CH_COMPTON = 2,   /* gamma + e -> a + e in a blackbody bath (Sec. II.G) */
  AXPIC_CH_BREMS = 4,     /* e + Z -> e + Z + a and e + e -> e + e + a (Sec. II.H) */
  AXPIC_CH_ALL = 7
};

/* One particle species in cell-sorted slabs (Sec. II.D.1: weighted
 * macroparticles; Sec. II.B: p in m_e c). Device pointers: wp and xyz hold
 * ncells*capacity records of 4 binary32 values each, {w, px, py, pz} and
 * {x, y, z, unused} (slot i at [4 i .. 4 i + 3]); count holds ncells int32.
 * A slot's weight and momentum share one record because every decision
 * reads them together, and its position is one more record because every
 * event, streaming and merging step moves the three coordinates together.
 * The library writes 0 into the unused word of the positions it writes. */
typedef struct {
  float *wp;
  float *xyz;
  int32_t *count;
  int32_t capacity;
} axpic_species;

/* The plasma (Sec. II.E, Eqs. rho_def, qn_def). */
typedef struct {
  int32_t ncells;          /* cells owned by this context */
  int32_t nspecies;        /* ion species, 1..8 */
  int64_t cell_index_base; /* global index of cell 0 (keys the RNG; sharding) */
  double *T_keV;           /* device [ncells] electron temperature, read/write */
  const double *n_ion;     /* device [ncells*nspecies] ion densities, cm^-3 */
  const double *Z;         /* host [nspecies] charge states */
  const double *A;         /* host [nspecies] mass numbers */
  double cell_volume_cm3;  /* volume represented by one cell */
  axpic_species electrons, photons, axions;
} axpic_plasma_desc;

/* Operator options. Defaults (axpic_default_params) are the readings listed
 * beside each field. */
typedef struct {
  double g_agg_GeV_inv;     /* axion-photon coupling, GeV^-1 (Eq. prim_xs) */
  double g_ae;              /* axion-electron coupling (Eqs. epsC, eps_eZ) */
  double dt_phys_s;         /* physical step, s (Eq. dt_phys) */
  double w_a;               /* axion macroparticle weight (Eq. lambda_macro) */
  double w_gamma_ref;       /* weight of photons made by a->gamma; <= 0: w_a */
  double lambda_cap;        /* Poisson-mean cap (Eq. lambda_eff); <= 0: off.
                               A ceiling of 64 always applies. */
  int32_t kappa_mode;       /* 0 Debye (Eq. kappa_debye), 1 fixed kappa */
  double kappa_fixed_keV;   /* used when kappa_mode == 1 */
  int32_t prim_targets;     /* 0: sum_i Z_i^2 n_i over ions (Sec. II.F);
                               1: all charges, n_eff */
  double prim_inverse_mult; /* a->gamma rate = mult * gamma->a rate (1) */
  int32_t eq_stats;         /* absorption target: 0 Maxwell-Boltzmann,
                               1 Bose-Einstein (Sec. II.I) */
  int32_t brems_ee;         /* 1: add e-e bremsstrahlung (Eq. eps_ee) */
  int32_t absorb_mode;      /* 0 Bernoulli deletion, 1 weight reduction
                               (Sec. II.I, P_abs) */
  double brems_gamma_shape; /* Gamma(a) energy sampler shape (1.70) */
  double relax_r;           /* temperature relaxation r (Eq. Te_relax) */
  double T_floor_keV;       /* temperature clamp */
  double T_ceil_keV;
  int32_t T_mode;           /* 0 fixed, 1 prescribed field, 2 evolved (Sec. II.E) */
  uint64_t seed;            /* Philox key */
  int32_t tally_nbins;      /* emitted-spectrum histogram bins (160) */
  double tally_Emax_keV;    /* histogram range [0, Emax) (80 keV) */
  int32_t tally_enable;     /* 1: step calls accumulate the emitted spectrum */
  int32_t diag_enable;      /* 1: feedback writes per-cell diagnostics */
  int32_t threads_per_block;/* threads per CTA of the event kernel (32..128, one
                               warp per cell); 0: default 128 */
  int32_t decide_chunk;     /* cells per chunk of a decision warp: 4, 8, 16 or
                               32; 0: the largest of 32, 16 and 8 that still
                               gives every resident decision warp a chunk of
                               the plasma's cells, else 4 (launch shape, see
                               axpic_autotune) */
  int32_t rate_model;       /* 0: closed forms (default); 1: exact FP32 table:
                               the full decisions' Primakoff and absorption
                               rates and the emission energies from per-cell
                               spectral records interpolated from the table;
                               2: surrogate network (axpic_set_surrogate):
                               where it is trusted its per-cell emissivity
                               constants set the prefactors of every rate's
                               closed functional form (emission, absorption,
                               Primakoff both ways) and its quantiles the
                               emission energies, evaluated by the network
                               kernel (sr_cells_kernel) right after each
                               temperature update; the table's records
                               elsewhere. Models 1 and 2 need
                               one ion species with Z in {1, 2}, Debye
                               screening and ions as Primakoff targets. Not
                               part of the paper's method. */
  int32_t sr_table_nkt;     /* table nodes in ln(kappa/T) (0: 128) */
  int32_t sr_table_nne;     /* table nodes in log10 n_e (0: 64) */
  int32_t step_branches;    /* axpic_run_steps: the cells run as 1, 2, 4 or
                               8 independent ranges on forked streams of the
                               graph, each chaining 32 steps with its own step
                               counter, so that one range's decisions overlap
                               another's events (0: 8 up to 2^20 cells, else
                               1; with rate models 1 and 2 each range also
                               rebuilds its own records). Results do not
                               depend on it. Not part of the paper's method. */
  int32_t reserved[2];
  double axion_mass_keV;    /* m_a c^2 (Sec. II.B: E = sqrt(p^2 + m_a^2)); 0
                               (default): massless. Axions are absorbed and
                               convert a->gamma at the massless rates of their
                               total energy E (the a->gamma photon takes E
                               along p); emission needs E > m_a and is thinned
                               with acceptance beta = p/E (thermal-bath events
                               by their channel uniform rescaled in its
                               channel's interval; gamma->a at beta(omega)
                               times the rate, the axion taking momentum
                               beta p_gamma); the thermal-bath feedback
                               exchanges E and p. Streaming takes its own
                               mass argument (axpic_stream_axions). */
} axpic_params;

/* Number of doubles written by axpic_tally_spectrum into totals_out. */
#define AXPIC_TOTALS_LEN 32
/* Layout of totals_out. */
enum {
  AXPIC_T_NEMIT_P = 0, AXPIC_T_NEMIT_C, AXPIC_T_NEMIT_B, /* sum w' of emitted axions */
  AXPIC_T_UEMIT_P, AXPIC_T_UEMIT_C, AXPIC_T_UEMIT_B,     /* sum w'E, keV */
  AXPIC_T_EVENTS_P, AXPIC_T_EVENTS_C, AXPIC_T_EVENTS_B,  /* macro-events */
  AXPIC_T_EVENTS_PINV,                                   /* a->gamma events */
  AXPIC_T_ABSORBED_C, AXPIC_T_ABSORBED_B,                /* Bernoulli absorptions */
  AXPIC_T_CAP_HITS, AXPIC_T_CLAMP_HITS, AXPIC_T_DROPPED,
  AXPIC_T_N_AXIONS, AXPIC_T_U_AXIONS,                    /* alive: sum w, sum wE (keV) */
  AXPIC_T_MACRO_AXIONS, AXPIC_T_MACRO_PHOTONS,
  AXPIC_T_RESIDUAL_E,                                    /* sum of carried energy, keV */
  AXPIC_T_N_PHOTONS, AXPIC_T_U_PHOTONS,
  AXPIC_T_U_ELECTRONS,                                   /* NR kinetic, keV */
  AXPIC_T_REMAPS,                                        /* cell remaps applied */
  AXPIC_T_PART_E, AXPIC_T_PART_G, AXPIC_T_PART_A,        /* sum over step calls of the
                                                            particles present at the start */
  AXPIC_T_REMAP_E,                                       /* electrons in remapped cells */
  AXPIC_T_CALLS                                          /* cell-steps processed */
};

/* Per-cell FP64 quantities returned by axpic_get_cell_info (Sec. II.E-II.H). */
#define AXPIC_CELL_INFO_LEN 16
enum {
  AXPIC_CI_RHO = 0, AXPIC_CI_XH, AXPIC_CI_NE, AXPIC_CI_NEFF, AXPIC_CI_SZ,
  AXPIC_CI_KAPPA, AXPIC_CI_QC, AXPIC_CI_QB, AXPIC_CI_GAMMA_C, AXPIC_CI_GAMMA_B,
  AXPIC_CI_GAMMA0_P, AXPIC_CI_ETA, AXPIC_CI_T
};

/* Per-cell FP64 feedback diagnostics of the last feedback (Sec. II.J). */
#define AXPIC_CELL_DIAG_LEN 16
enum {
  AXPIC_CD_DE = 0, AXPIC_CD_DPX, AXPIC_CD_DPY, AXPIC_CD_DPZ, /* this step's exchange */
  AXPIC_CD_S_MINUS_1, AXPIC_CD_BX, AXPIC_CD_BY, AXPIC_CD_BZ,
  AXPIC_CD_VAR, AXPIC_CD_VAR_NEW, AXPIC_CD_W,
  AXPIC_CD_APPLIED_E, AXPIC_CD_RES_E, AXPIC_CD_RES_PX, AXPIC_CD_RES_PY, AXPIC_CD_RES_PZ
};

/* Fill *p with the default options. Never fails for a non-NULL p. */
void axpic_default_params(axpic_params *p);

/* Create a context for one plasma (Sec. II.E): validate the description,
 * allocate the library's scratch, build the energy-sampling tables
 * (Sec. II.G, II.H) and compute every cell's rate record (Sec. II.E-II.I).
 * The particle slabs are used as they are (see axpic_sample_plasma).
 * stream: a cudaStream_t (NULL: the legacy default stream) on which every
 * later call of this context is enqueued. The only call that allocates,
 * besides axpic_destroy which frees. Returns AXPIC_E_INVALID for a NULL or
 * inconsistent description, AXPIC_E_CUDA if an allocation fails. */
axpic_status axpic_init_plasma(axpic_ctx **out, const axpic_plasma_desc *desc,
                               const axpic_params *params, void *stream);

/* Fill the slabs with the synthetic initial plasma: per cell n_el
 * non-relativistic Maxwellian electrons of weight n_e V/n_el, n_ph Planck
 * photons at T_e of weight n_gamma V/n_ph (Sec. II.G, blackbody bath) and
 * n_ax Maxwell-Boltzmann-equilibrium axions of weight w_a, with isotropic
 * directions and uniform positions; counts are set. AXPIC_E_INVALID if a
 * count exceeds its capacity. */
axpic_status axpic_sample_plasma(axpic_ctx *ctx, int32_t n_el, int32_t n_ph, int32_t n_ax);

/* Recompute every cell's rate record after the caller changed T_keV or
 * n_ion (temperature mode "prescribed field", Sec. II.E). */
axpic_status axpic_update_cells(axpic_ctx *ctx);

/* Composition from the deposited electron density (Sec. II.E, Eqs. rho_def
 * and qn_def: n_e and rho inferred from the deposited charge density with
 * the hydrogen mass fraction under quasi-neutrality, or the densities bound
 * to one ion species). Each cell's free-electron density is that of its own
 * electron macroparticles, n_e = sum w / cell_volume_cm3 (summed in
 * compensated binary32 pairs per lane, then in FP64: within about
 * (count/32) 2^-48 of the exact sum). Then,
 * for every cell:
 * - bind_species = -1: mass fractions mass_frac (host [nspecies], finite,
 *   >= 0, summing to 1 within 1e-9; X_H and 1 - X_H for hydrogen-helium)
 *   with n_e = sum_i Z_i n_i: n_i = X_i (rho/m_u) / A_i,
 *   rho/m_u = n_e / sum_i Z_i X_i / A_i;
 * - bind_species = k in [0, nspecies): n_k = n_e / Z_k, the others 0
 *   (mass_frac unused).
 * Writes n_ion_out (device [ncells*nspecies], cm^-3). When n_ion_out is the
 * context's own n_ion array, the rate records are then rebuilt from it as by
 * axpic_update_cells; the cached electron moments are unchanged, since the
 * deposit moves no electron. Asynchronous. AXPIC_E_INVALID (nothing written)
 * for a bad bind_species, a bound species with Z <= 0, missing or invalid
 * mass fractions, or a null n_ion_out with cells. */
axpic_status axpic_deposit_composition(axpic_ctx *ctx, int32_t bind_species, const double *mass_frac,
                                       double *n_ion_out);

/* Axion free streaming and cell migration: every axion moves by
 * (p / E) c dt_s, E = sqrt(p^2 + m_a^2) with m_a c^2 = mass_keV (Sec. II.B:
 * massless axions at c, massive ones sub-luminal; the axions' transport
 * between steps) on a
 * regular grid of nx x ny x nz cubic cells of edge h_cm [cm], cell index
 * (k ny + j) nx + i (nx ny nz must equal ncells). Positions are fractions of
 * the cell; a dimension of one cell is not streamed. c dt_s must stay below
 * h_cm (at most one cell per dimension and step). boundary 0: periodic;
 * 1: open (axions leaving the box are removed and counted, see
 * axpic_stream_stats). The position update is binary32 with each rounding
 * fixed: E = sqrt(((px px + py py) + pz pz) + mu mu) with mu =
 * binary32(mass_keV / m_e c^2), d = (kappa / E) p_dim with kappa =
 * binary32(c dt / h), t = x + d, shift floor(t), fraction t - shift (the
 * largest binary32 below 1 where that rounds up to 1); E = 0 does not move. Each cell's arrivals, ordered by the source cell's position
 * relative to it ((dz, dy, dx) ascending lexicographic over {-1, 0, 1}^3)
 * and then by source slot, take the slots its leaving axions freed
 * (ascending), then the slots after the old count; freed slots left over are
 * closed by the tail fill (the slot rule of a full step's axions). Staying
 * axions keep their slots unless the tail fill moves them. Axions beyond the
 * capacity are dropped, counted and latch AXPIC_E_CAPACITY. Asynchronous on the context's stream; the first
 * call allocates scratch (33 bytes per axion slot plus 216 per cell), later
 * calls allocate nothing. AXPIC_E_INVALID (nothing launched) for a grid
 * that does not match, h_cm <= 0, dt_s < 0, c dt_s >= h_cm or another
 * boundary value, or a negative mass. */
axpic_status axpic_stream_axions(axpic_ctx *ctx, int32_t nx, int32_t ny, int32_t nz, double h_cm, double dt_s,
                                 double mass_keV, int32_t boundary);

/* Axion merging for population control: in every cell holding more than
 * n_target axions, each group of three or more axions with the same octant
 * of p (signs of px, py, pz; zero counts as positive) and the same |p|^2 bin
 * becomes two axions with the group's weight W, momentum P and energy E
 * (massless: each of weight W/2 and |p| = E/W, on either side of P at
 * cos theta = |P|/E; Vranic et al., Comput. Phys. Commun. 191, 65 (2015);
 * the method merges axions as a species of the PIC code, Sec. II.A, and names
 * no algorithm). The bin of an axion is the number of the nedges (<= 30)
 * ascending binary32 thresholds edges_p2 [(m_e c)^2] at or below
 * |p|^2 = (px px + py py) + pz pz in binary32. Arithmetic is binary32 with
 * every step rounded, the sums compensated (Kahan) in slot order;
 * the new axions take the group's first two slots at the weighted mean
 * position, the other slots are freed and closed by the tail fill. One pass;
 * a cell may stay above n_target. Asynchronous; the first call allocates 1
 * byte per axion slot. AXPIC_E_INVALID (nothing launched) for n_target < 0,
 * more than 30 thresholds, or thresholds not finite, >= 0 and ascending. */
axpic_status axpic_merge_axions(axpic_ctx *ctx, int32_t n_target, int32_t nedges, const float *edges_p2);
/* Axions removed by every merge so far (host, 1 double). Synchronises. */
axpic_status axpic_merge_stats(axpic_ctx *ctx, double *removed);

/* Checkpoint and resume. The state a context owns between steps, besides
 * the caller's slabs and T_keV: the cells' rate records and cached electron
 * moments, the FP64 exchange and residual-carry buffers, the per-cell
 * diagnostics, the tallies and counters, the decision masks, the latched
 * error flag and, for rate models 1 and 2, the spectral records (not the
 * surrogate's network or trust map: axpic_set_surrogate sets those). Philox
 * is stateless, so a context of the same geometry and parameters whose
 * caller arrays and loaded state are a save's continues bit for bit from
 * the next step index. axpic_state_bytes gives the size; save and load copy
 * it to and from host memory (bytes must equal it, else AXPIC_E_INVALID).
 * Save and load synchronise. */
axpic_status axpic_state_bytes(axpic_ctx *ctx, uint64_t *bytes);
axpic_status axpic_save_state(axpic_ctx *ctx, void *host_out, uint64_t bytes);
axpic_status axpic_load_state(axpic_ctx *ctx, const void *host_in, uint64_t bytes);

/* nsteps steps as axpic_run_steps runs them, each followed by the axions'
 * streaming of axpic_stream_axions with these parameters (the transport
 * between steps, Sec. II.B), replayed from CUDA graphs of 32 steps. Each
 * step's cell branches are joined before the streaming, which crosses
 * them. Graphs are kept per channel mask for the last streaming parameters.
 * Asynchronous; results are identical to nsteps pairs of axpic_step and
 * axpic_stream_axions. AXPIC_E_INVALID as for either call. */
axpic_status axpic_run_steps_streamed(axpic_ctx *ctx, int64_t first_step, int32_t nsteps, int32_t channel_mask,
                                      int32_t nx, int32_t ny, int32_t nz, double h_cm, double dt_stream_s,
                                      double mass_keV, int32_t boundary);

/* Totals of every streaming so far (axpic_stream_axions and the streaming of
 * axpic_run_steps_streamed), to out (host, 4
 * doubles): axions that left an open box (number, weight, weight x energy
 * [keV], the total energy sqrt(p^2 + m_a^2)) and axions dropped at a full
 * slab (number). Zeros before the first
 * call. Synchronises. */
axpic_status axpic_stream_stats(axpic_ctx *ctx, double *out);

/* Inverse operators on the axions present when the call starts (Sec. II.F.1
 * last paragraph; Sec. II.I): Primakoff a->gamma conversion with weight
 * depletion (photon products appended) and detailed-balance absorption of the
 * thermal-bath channels, P_abs = 1 - exp(-Gamma_abs dt). Absorbed energy and
 * momentum go to the cell exchange buffer (Sec. II.J). */
axpic_status axpic_absorb(axpic_ctx *ctx, int64_t step, int32_t channel_mask);

/* Forward operators (Sec. II.D, II.F-II.H): Primakoff gamma->a on the
 * photons present before this step's axpic_absorb, Compton-like and
 * bremsstrahlung emission on electrons, with Poisson macro-events, capping
 * and inverse-CDF energy sampling; new axions are appended (stream
 * compaction) and the emitted energy and momentum go to the exchange buffer. */
axpic_status axpic_emit(axpic_ctx *ctx, int64_t step, int32_t channel_mask);

/* Conservative feedback (Sec. II.J, Eqs. cell_moments to b_def): affine
 * remap of the electron momenta with the cell's exchange buffer plus the
 * energy carried from earlier steps, then the temperature update
 * (Eqs. Te_est, Te_relax) in temperature mode "evolved". Clears the buffer. */
axpic_status axpic_feedback(axpic_ctx *ctx, int64_t step);

/* One step, absorb -> emit -> feedback: the three calls above enqueued
 * together (identical results). */
axpic_status axpic_step(axpic_ctx *ctx, int64_t step, int32_t channel_mask);
/* One full step, as axpic_step, over the cells [first_cell, first_cell +
 * ncells) only. Cells are independent within a step (every operator is
 * cell-local, Sec. II.D), so steps of one index over disjoint ranges that
 * cover the context, in any order, leave the particles, temperatures and
 * records bit for bit as one axpic_step does (tallies are FP64 sums whose
 * rounding follows the order). This lets a caller overlap the copies of
 * one range with the step of another. Asynchronous on the context's
 * stream. AXPIC_E_INVALID (nothing launched) for a range outside the
 * context, a step index outside [0, 2^32 - 1) or unknown channel bits. */
axpic_status axpic_step_cells(axpic_ctx *ctx, int64_t step, int32_t channel_mask, int32_t first_cell,
                              int32_t ncells);

/* Emitted-spectrum tally (App. B): H_out (host, 3*nbins doubles, channel-
 * major: Primakoff, Compton-like, bremsstrahlung) receives
 * H_k = sum w'E (keV) of the axions emitted since the previous call, and
 * totals_out (host, AXPIC_TOTALS_LEN doubles, may be NULL) the counters
 * listed above; both accumulators are then cleared. nbins must equal the
 * context's tally_nbins. Synchronises the stream and reports latched errors. */
axpic_status axpic_tally_spectrum(axpic_ctx *ctx, int32_t nbins, double *H_out,
                                  double *totals_out);

/* Deterministic rates for one cell, for checking (Eqs. prim_prob,
 * gamma_abs): for each of n energies E_keV[i] (device) writes four binary32
 * values to out[4*i..4*i+3] (device): P_{gamma->a} (of a photon of energy
 * E; times beta(E) for a massive axion), P_{a->gamma} and Gamma_abs,C dt,
 * Gamma_abs,B dt (of an axion of total energy E), from the cell record's
 * prefactors (the closed forms; the network's where rate model 2 trusts
 * it; spectral records are not consulted). Enqueued on the stream. */
axpic_status axpic_eval_rates(axpic_ctx *ctx, int32_t cell, const float *E_keV, int32_t n,
                              float *out);

/* Copy AXPIC_CELL_INFO_LEN doubles per cell for cells [first, first+count)
 * into host_out. Synchronises the stream. */
axpic_status axpic_get_cell_info(axpic_ctx *ctx, int32_t first, int32_t count, double *host_out);

/* Copy AXPIC_CELL_DIAG_LEN doubles per cell of the last feedback (written
 * only with diag_enable) into host_out. Synchronises the stream. */
axpic_status axpic_get_cell_diag(axpic_ctx *ctx, int32_t first, int32_t count, double *host_out);

/* Copy the carried (not yet applied) energy and momentum per cell, 4 doubles
 * per cell (keV, m_e c), into host_out. Synchronises the stream. */
axpic_status axpic_get_residuals(axpic_ctx *ctx, int32_t first, int32_t count, double *host_out);

/* One step (the same kernels as axpic_step) for callers that cannot
 * allocate device memory: a host code whose memory manager owns the whole GPU
 * heap, or a real-time loop where a cudaMalloc could stall or fail. It needs
 * no context and calls no cudaMalloc, cudaFree or other allocating routine.
 * The paper has no counterpart: this is an interface convenience.
 *
 * Its scratch (rate records, electron moments, sampling tables, counters,
 * exchange buffer, photon counts, decision bit masks and records, error
 * flag; about 23 MB) is a file-scope device array of the library, held by
 * every GPU that loads the library until the process exits. It limits a call
 * to 16384 cells, to ncells * (sum of the three capacities) / 8 <= 4 MiB of
 * bit masks and to ncells * (16 (axion + photon capacity) + 4 electron
 * capacity) <= 16 MiB of decision records (about 1300 cells with capacities
 * 512/384/384); larger requests return AXPIC_E_INVALID without launching.
 * The first call on a device does a set-up: with that device current it
 * looks up the array's device address and uploads the sampling tables; make
 * that first call before any stream capture. Later calls reupload the tables
 * only when brems_gamma_shape changes.
 *
 * desc, params: as for axpic_init_plasma (read during the call, and checked
 *   the same way: AXPIC_E_INVALID, nothing launched, for what
 *   axpic_init_plasma rejects; rate_model must be 0).
 * carry: device [ncells*4] FP64, owned by the caller, read and written: the
 *   energy (keV) and momentum (m_e c) not yet applied by the remap, which
 *   axpic_step keeps inside its context; zero it before the first step.
 * Rates are recomputed from T_keV and n_ion, and electron moments from the
 * electrons, on every call; no tally or per-cell diagnostics are produced.
 * Every call shares the one scratch array (it keeps the last call's
 * contents; what must start at zero is cleared by each call), so calls that
 * overlap on the GPU, on different streams or threads, race. Every call
 * waits for the stream before it returns, and returns AXPIC_E_CAPACITY or
 * AXPIC_E_NUMERIC found on the device. */
axpic_status axpic_step_noalloc(const axpic_plasma_desc *desc, const axpic_params *params, int64_t step,
                                int32_t channel_mask, double *carry, void *stream);

/* Runs nsteps full steps (as axpic_step with steps first_step,
 * first_step + 1, ...) by replaying CUDA graphs of 32 steps and of one step
 * (for the remainder): the decision, event and feedback kernels (and, with
 * evolved T, the rate model's record kernel), with the step index read from
 * device counters that the feedback kernels advance.
 * Inside a graph the cells run as step_branches independent ranges on forked
 * streams, each range with its own counter, joined at the graph's end. Both
 * graphs are captured on the first call for a channel mask, whatever its
 * nsteps (on private streams of the context, ordered after the context's
 * stream), so later calls launch without capturing; they are kept until the
 * launch shape changes. Asynchronous; results are identical to nsteps calls of
 * axpic_step. AXPIC_E_INVALID for
 * nsteps < 0, a step range outside [0, 2^32 - 1) or unknown channel bits.
 * Not part of the paper's method: batching of many small boxes in one
 * context (each cell carries its own plasma record) and launch by graph. */
axpic_status axpic_run_steps(axpic_ctx *ctx, int64_t first_step, int32_t nsteps, int32_t channel_mask);

/* The context's launch shape: cells per decision chunk, warps per event CTA
 * and the branches a replayed step runs its cells as (each may be NULL).
 * A replayed step launches 4 x branches kernels (decision, event, the event
 * kernel of the cells with more flagged slots than a lane takes, feedback per
 * branch; 5 x branches with a rate model's record kernel) and one 4-byte
 * memset per branch. AXPIC_E_INVALID for a NULL context. Not part of the
 * paper's method. */
axpic_status axpic_launch_shape(const axpic_ctx *ctx, int32_t *decide_chunk, int32_t *event_warps,
                                int32_t *step_branches);

/* Picks the launch shape (cells per decision chunk, 4/8/16/32, and warps per
 * event CTA, 2 or 4) by timing trial_steps steps of the context's own state
 * for each shape (CUDA events, after one untimed step), with the step index
 * `step` and channel_mask. The context's device state (the slabs and counts
 * of the three species, T, rates, moments, exchange and carried buffers,
 * tallies and counters) is saved to scratch first and restored after every
 * trial, so the state afterwards is bit for bit what it was. Needs device
 * memory for one copy of that state. Synchronises. Writes the best shape's
 * ms per step to *best_ms_out (may be NULL) and its parameters to
 * *chunk_out and *warps_out (may be NULL). AXPIC_E_INVALID for
 * trial_steps < 1. Not part of the paper's method. */
axpic_status axpic_autotune(axpic_ctx *ctx, int64_t step, int32_t trial_steps, int32_t channel_mask,
                            double *best_ms_out, int32_t *chunk_out, int32_t *warps_out);

/* Measurement of the step's kernels. axpic_profile_begin (synchronises)
 * prepares CUDA events for the next max_steps calls of axpic_step, which then
 * record an event on the context's stream before and after each kernel they
 * launch (recording adds no kernel work). axpic_profile_end (synchronises)
 * writes to ms_out (host, AXPIC_PROFILE_SLOTS doubles) the summed device time
 * of each kernel over the recorded steps, in the order that
 * axpic_step_kernel_names gives (unused slots are 0), sets *steps_out (may be
 * NULL) to the number of steps recorded, and releases the events. Not part of
 * the paper's method. */
#define AXPIC_PROFILE_SLOTS 4
axpic_status axpic_profile_begin(axpic_ctx *ctx, int32_t max_steps);
axpic_status axpic_profile_end(axpic_ctx *ctx, double *ms_out, int32_t *steps_out);

/* Comma-separated names of the profiled kernels of one axpic_step, in
 * launch order: decisions, events (its slot also times event_heavy_kernel,
 * launched right after it for the cells with more flagged slots than a lane
 * takes), feedback, then, with evolved T, the rate model's record kernel
 * (sr_table_kernel for the table model, sr_cells_kernel for the surrogate).
 * The string is static; "" for a NULL context. */
const char *axpic_step_kernel_names(const axpic_ctx *ctx);

/* ---------------------------------------------------------------------------
 * The spectral surrogate's network: MLP 4 -> 64 -> 64 -> 96 with tanh hidden
 * layers (the hardware's binary32 tanh approximation, relative error below
 * 1e-5, in training, validation and inference), FP32 master parameters, bfloat16 tensor-core products with FP32
 * accumulation (layers 2 and 3 and every backward product; layer 1, K = 4,
 * on the CUDA cores). Not part of the paper's method: a learned stand-in for
 * the per-channel spectral emissivity and inverse CDF (see
 * axpic_surrogate_targets). The model's output o at the normalised features
 * f = (ln x, ln(kappa/T), log10 n_e, Z) of axpic_surrogate_features is
 *   y_o = shape_o(x, kappa/T) + mu_o + sum_{i=1..3} S_oi f_i + sigma_o z_o,
 * z the network's output at the cell features (0, f_1, f_2, f_3): shape_o
 * carries every x-dependence, so the learned part is a function of the cell,
 * and a cell's three ln-emissivity constants c_o = y_o - shape_o (o = 0, 32,
 * 64) are all the step needs from the network for its rates.
 * S is an FP32 linear map (axpic_mlp_set_skip; its column i = 0 multiplies
 * zero) and shape_o is fixed: for the ln-emissivity outputs (o = 0, 32, 64)
 * the channel's exact x-dependence at fixed cell,
 *   Primakoff      3 ln x - ln(e^x - 1) + ln F(s), s = 4 x^2 / (kappa/T)^2,
 *                  F the screening function of Sec. II.F,
 *   Compton-like   5 ln x - ln(e^x - 1),
 *   bremsstrahlung a ln x - x (a = brems_gamma_shape);
 * zero for the quantiles. After S the Primakoff and Compton-like rates are
 * exact; the network carries the bremsstrahlung brackets and the Primakoff
 * quantiles. axpic_mlp_forward and axpic_mlp_gradients take the network's
 * own inputs (callers pass cell features). Calls are ordered on the stream
 * given at creation; those that return host data synchronise it.
 * ------------------------------------------------------------------------- */
typedef struct axpic_mlp axpic_mlp;
#define AXPIC_MLP_PARAMS 10720 /* W1[4][64], b1[64], W2[64][64], b2[64], W3[64][96], b3[96] */

/* Creates a network with zero parameters on `stream` (a cudaStream_t). */
axpic_status axpic_mlp_create(axpic_mlp **out, void *stream);
/* Copies AXPIC_MLP_PARAMS host floats in (and resets the Adam state) or out. */
axpic_status axpic_mlp_set_params(axpic_mlp *m, const float *params);
axpic_status axpic_mlp_get_params(axpic_mlp *m, float *params);
/* Z[n][96] (device) = network(X[n][4]) (device); asynchronous. */
axpic_status axpic_mlp_forward(axpic_mlp *m, const float *X, int32_t n, float *Z);
/* Gradients of loss = sum over samples and outputs of (z - Zt)^2 / n with
 * respect to every parameter, written to grads (host, AXPIC_MLP_PARAMS, may
 * be NULL) with the loss to *loss_out (may be NULL). X, Zt: device. */
axpic_status axpic_mlp_gradients(axpic_mlp *m, const float *X, const float *Zt, int32_t n, double *loss_out,
                                 float *grads);
/* One training step: gradients on (X, Zt), then Adam (beta 0.9, 0.999,
 * eps 1e-8, bias-corrected) with learning rate lr. *loss_out (may be NULL,
 * which keeps the call asynchronous) gets the loss before the update. */
axpic_status axpic_mlp_train_step(axpic_mlp *m, const float *X, const float *Zt, int32_t n, float lr,
                                  double *loss_out);
axpic_status axpic_mlp_destroy(axpic_mlp *m);
const char *axpic_mlp_last_error(const axpic_mlp *m);

/* Output normalisation of the network (mu, sigma of the model above), 96
 * floats each; set by axpic_surrogate_fit. sigma must be >= 0 (0: the
 * output is the constant mu). */
axpic_status axpic_mlp_set_norm(axpic_mlp *m, const float *mu, const float *sigma);
axpic_status axpic_mlp_get_norm(axpic_mlp *m, float *mu, float *sigma);
/* The linear map S of the model above, 96 x 4 floats, S[o][i] at o * 4 + i
 * (zero on creation; fitted by least squares in axpic_surrogate_fit).
 * AXPIC_E_INVALID for a non-finite entry. */
axpic_status axpic_mlp_set_skip(axpic_mlp *m, const float *skip);
axpic_status axpic_mlp_get_skip(axpic_mlp *m, float *skip);

/* The function the surrogate stands in for, in binary64 on the host: for
 * each of n rows (x = omega/T, kappa/T, n_e [cm^-3], Z in {1, 2}) of `in`,
 * 96 values to `out`: per channel (Primakoff, Compton-like, bremsstrahlung)
 * ln(dQ/dx) [erg cm^-3 s^-1 per unit x] at unit coupling (g_agg = 1 GeV^-1,
 * g_ae = 1; Eqs. prim_xs/prim_rate with Planck photons, epsC, eps_eZ/eps_ee
 * with the [1 - c eta] brackets floored at 1e-3), then the quantiles x(u_j),
 * u_j = j/32, j = 1..31, of its number spectrum on [0.05, 20]. Single-ion
 * plasma (n_i = n_e / Z), Debye screening, ions as Primakoff targets. */
axpic_status axpic_surrogate_targets(const double *in, int32_t n, double brems_shape, double *out);
/* The network's input features of n rows (x, kappa/T, n_e, Z): ln x,
 * ln(kappa/T), log10 n_e and Z, each mapped onto [-1, 1] over the domain
 * x in [0.05, 20], kappa/T in [0.012, 41], n_e in [1e23, 1e26]. */
axpic_status axpic_surrogate_features(const double *in, int32_t n, float *out);
/* Trains the network from scratch on the GPU: ncells random cells of the
 * domain (T uniform in [0.5, 10] keV, n_e log-uniform in [1e23, 1e26],
 * Z in {1, 2}; only cells where both bremsstrahlung brackets 1 - c eta are
 * at least 0.05, the region where that fit holds) with x_per_cell
 * log-uniform x each (the learned part does not depend on x: 1 suffices),
 * targets from axpic_surrogate_targets. mu and S by least squares, sigma
 * the residual spread (floors 1e-4 on rates, 1e-5 on quantiles; rates
 * weighted 16 in the loss) set on the handle; the Compton-like and
 * bremsstrahlung quantiles, which do not depend on the cell, are the exact
 * knots in mu with sigma and S zero. The weight gradients are summed in a
 * fixed order, so a fit is reproducible bit for bit. `steps` Adam steps on
 * consecutive batches of `batch` rows with a cosine learning rate from lr to
 * lr / 100. *loss_out (may be NULL): final loss on the whole set
 * (normalised units). Synchronises. */
axpic_status axpic_surrogate_fit(axpic_mlp *m, int32_t ncells, int32_t x_per_cell, int32_t steps, int32_t batch,
                                 float lr, uint64_t seed, double brems_shape, double *loss_out);
/* Error of the trained network on a grid of nT temperatures (log-uniform in
 * [0.5, 10] keV) x nne densities (log-uniform in [1e23, 1e26]) x Z in {1, 2}
 * (node (Z-1, j, i) at index ((Z-1) nne + j) nT + i; nT, nne in [2, 4096]),
 * each at 8 x values log-spaced on [0.05, 20] (the learned part depends on
 * the cell alone): err_out[3 node] = largest
 * |ln(dQ/dx) error| over x and channels (the relative rate error),
 * err_out[3 node + 1] = largest relative error of the Compton-like and
 * bremsstrahlung quantiles (those the step samples emission energies from),
 * err_out[3 node + 2] = that of the Primakoff quantiles (which the step does
 * not use: gamma->a products inherit the photon's momentum). Synchronises. */
axpic_status axpic_surrogate_validate(axpic_mlp *m, int32_t nT, int32_t nne, double brems_shape, float *err_out);

/* Gives a context with rate_model 2 its network: the parameters, output
 * model and a trust map from axpic_surrogate_validate's err_out (nT x nne x
 * 2 nodes, 3 floats each). A node passes where its rate error is <= tol_rate
 * and its sampled-quantile error <= tol_quantile; it is trusted where it and
 * its eight neighbours in (T, n_e) at its Z pass (the grid's edge nodes
 * count their neighbours inside it). A cell uses the network where the four
 * nodes around its (T, n_e) at its Z are trusted, the table elsewhere. The
 * error between nodes can exceed the nodes', most where it rises steeply:
 * the neighbours' test keeps the trusted cells away from failing nodes, and
 * a finer grid and a tolerance below the bound wanted leave a margin. Copies everything (the network may be destroyed
 * afterwards) and rebuilds the cells' records: trusted cells get the
 * network's prefactors (one tensor-core row per cell), the others the
 * table's spectral record. Synchronises. AXPIC_E_INVALID for another rate
 * model, grid sizes outside [2, 4096], negative tolerances, or a network
 * whose Compton-like or bremsstrahlung quantiles depend on the cell. */
axpic_status axpic_set_surrogate(axpic_ctx *ctx, axpic_mlp *m, const float *err_map, int32_t nT, int32_t nne,
                                 float tol_rate, float tol_quantile);
/* The cell records of cells [first, first + count), AXPIC_REC_LEN floats per
 * cell to rec_out (host), and (src_out: host, may be NULL) one byte per cell:
 * 1 where the cell's rates come from its spectral record (rate model 1; rate
 * model 2 where the network is not trusted), 0 otherwise. Record slots:
 * [0] T [keV], [1] 1/T, [2] 4/kappa^2, [3] lambda_C/w_e and [4] lambda_B/w_e
 * (emission Poisson means per unit electron weight), [5] and [6] the
 * Compton-like and bremsstrahlung absorption prefactors (tau_C = [5] x^2
 * e^x/(e^x - 1) and tau_B = [6] x^(a-3) for Maxwell-Boltzmann targets),
 * [7] Gamma_0 dt of gamma->a (Gamma dt = [7] F(s)), [8] m [7] as the
 * composition gives it, [9] n_e and [10] n_eff (1e24 cm^-3), [11] rho
 * [g cm^-3], [12] X_H, [13] the Primakoff target sum (1e24 cm^-3).
 * Synchronises. */
#define AXPIC_REC_LEN 16
axpic_status axpic_get_cell_records(axpic_ctx *ctx, int32_t first, int32_t count, float *rec_out,
                                    uint8_t *src_out);
/* The spectral records of cells [first, first + count) (rate models 1 and 2;
 * under model 2 only the cells the network is not trusted for have one, see
 * axpic_get_cell_records): 192 floats per cell to out (host): ln(dQ_c/dx) +
 * x_k at unit coupling on x_k = 0.05 e^((k - 1) h), h = ln(400) / 29,
 * k = 0..31 (c * 32 + k; c = Primakoff, Compton-like, brems), the
 * quantiles x(j/32) (96 + c * 31 + j - 1), then ln(g_agg^2 dt pi^2 (hbar c)^3
 * / (T^4 keV)), ln(g_ae^2 dt 2 pi^2 (hbar c)^3 / (T^4 keV)) and T.
 * Synchronises. */
axpic_status axpic_get_spectral_records(axpic_ctx *ctx, int32_t first, int32_t count, float *out);

/* Wait for the stream and return the first latched device error, if any. */
axpic_status axpic_sync(axpic_ctx *ctx);

/* Wait for the stream, free the library's scratch and the context. */
axpic_status axpic_destroy(axpic_ctx *ctx);

/* Message of the last error on this context (never NULL; static for NULL ctx). */
const char *axpic_last_error(const axpic_ctx *ctx);

/* Library version string. */
const char *axpic_version(void);

#ifdef __cplusplus
}
#endif

#endif /* AXPIC_H */
