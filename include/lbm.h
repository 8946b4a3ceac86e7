/*
 * lbm.h - C ABI of the GB300 Shan-Chen bubble-merging lattice Boltzmann
 * library (method of Barzegari, Bayani & Mirbagheri, "A criterion for bubble
 * merging in liquid metal", arXiv 1708.01608).
 *
 * One context = one periodic lattice on one CUDA device.  Device memory is
 * owned by the context (allocated through the caller's allocator callbacks
 * when given, else cudaMalloc); every host buffer is owned by the caller.
 * Work is enqueued on the stream given in the configuration (NULL = the
 * legacy default stream).  A context is not thread-safe.  No function throws
 * across the ABI: each returns an lbm_status, and lbm_last_error() gives a
 * message for the calling thread's last failure.
 *
 * Lattice conventions (shared by every call that takes or returns fields):
 *   cell (x, y, z) has linear index x + nx*(y + ny*z); nz = 1 for D2Q9.
 *   Scalar fields are nx*ny*nz doubles in that order.
 *   Populations f_i(x, t) ("after streaming": the value that has arrived at
 *   x) are Q fields, population-major: f[i*N + cell].
 *   Velocity order, D2Q9 (weights 4/9, 1/9 x4, 1/36 x4):
 *     0 (0,0) 1 (1,0) 2 (0,1) 3 (-1,0) 4 (0,-1) 5 (1,1) 6 (-1,1) 7 (-1,-1) 8 (1,-1)
 *   D3Q19 (weights 1/3, 1/18 x6, 1/36 x12):
 *     0 (0,0,0) 1 (1,0,0) 2 (-1,0,0) 3 (0,1,0) 4 (0,-1,0) 5 (0,0,1) 6 (0,0,-1)
 *     7 (1,1,0) 8 (-1,-1,0) 9 (1,-1,0) 10 (-1,1,0) 11 (1,0,1) 12 (-1,0,-1)
 *     13 (1,0,-1) 14 (-1,0,1) 15 (0,1,1) 16 (0,-1,-1) 17 (0,1,-1) 18 (0,-1,1)
 *
 * The time step (Sec. 3.1 of the paper: Shan-Chen model, single relaxation
 * time, "streams and collisions"):
 *   rho = sum_i f_i, j = sum_i f_i c_i
 *   psi = rho0 (1 - exp(-rho/rho0))           (Sec. 3.1, rho0 = 1 in the paper)
 *   F   = -G psi(x) sum_i w_i psi(x + c_i) c_i (long-range attraction, Sec. 3.1)
 *   u   = (j + tau F)/rho                      (velocity-shift forcing)
 *   f*_i = f_i - (f_i - f_eq_i(rho, u))/tau
 *   f*_i(x_s) += w_i dm_s at injection sites   (virtual blowing agent, Sec. 3)
 *   f_i(x + c_i, t+1) = f*_i(x)                (periodic)
 * EOS pressure p = rho/3 + (G/6) psi^2 (Sec. 3.1; the printed 0.166 = cs^2/2).
 */
#ifndef SCLBM_LBM_H
#define SCLBM_LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx; /* opaque */

typedef enum {
  LBM_OK = 0,
  LBM_EINVAL = 1,   /* bad argument or configuration; nothing was changed */
  LBM_ENOMEM = 2,   /* device allocation failed */
  LBM_ECUDA = 3,    /* a CUDA call failed; the context should be destroyed */
  LBM_ESTATE = 4,   /* call not valid in the current state (e.g. not seeded) */
  LBM_ENUMERIC = 5, /* a non-finite density was found by a diagnostic */
  LBM_ETIMEOUT = 6  /* a bounded device wait gave up; results are invalid */
} lbm_status;

typedef enum { LBM_D2Q9 = 0, LBM_D3Q19 = 1 } lbm_lattice;

/* storage precision of the populations; arithmetic is FP64 for LBM_F64 and
 * FP32 otherwise.  The 16-bit forms store f_i - w_i*rho_ref. */
typedef enum {
  LBM_F64 = 0,
  LBM_F32 = 1,
  LBM_F16_OFFSET = 2,
  LBM_BF16_OFFSET = 3
} lbm_storage;

/* fields for lbm_read; every field is returned as doubles */
typedef enum {
  LBM_RHO = 0,  /* N: density */
  LBM_PSI = 1,  /* N: pseudopotential */
  LBM_P = 2,    /* N: EOS pressure */
  LBM_U = 3,    /* 3N: physical velocity (j + F/2)/rho, components x, y, z */
  LBM_F = 4,    /* Q*N: populations f_i(x, t) */
  LBM_LAPP = 5  /* N: periodic 5-point (2-D) / 7-point (3-D) Laplacian of p */
} lbm_field;

/* step kernel selection */
typedef enum {
  LBM_KERNEL_AUTO = 0,    /* fused kernel with the tuned tile */
  LBM_KERNEL_FUSED = 1,   /* one pass: TMA-staged tiles, psi halo in smem */
  LBM_KERNEL_TWO_PASS = 2 /* psi field pass + collide/stream pass */
} lbm_kernel;

/* Optional device allocator.  alloc returns device memory of `bytes` usable
 * on `stream` (NULL on failure); free releases it. */
typedef void *(*lbm_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*lbm_free_fn)(void *ptr, size_t bytes, void *stream, void *user);

typedef struct {
  int32_t lattice;      /* lbm_lattice */
  int32_t storage;      /* lbm_storage */
  int64_t nx, ny, nz;   /* periodic extents; nz must be 1 for D2Q9 */
  double tau;           /* BGK relaxation time, > 0.5 */
  double G;             /* Shan-Chen interaction strength (G < -4 separates) */
  double rho0;          /* psi scale; 1 reproduces the paper's psi */
  double rho_ref;       /* reference density of the 16-bit offset storage */
  double gas_threshold; /* cells with rho < threshold are gas (labelling) */
  int32_t kernel;       /* lbm_kernel */
  int32_t tile;         /* fused-kernel tile id; 0 = pick automatically */
  void *stream;         /* cudaStream_t, may be NULL */
  lbm_alloc_fn alloc;   /* NULL: cudaMalloc/cudaFree */
  lbm_free_fn free;
  void *alloc_user;
  int32_t debug_flags;  /* 0 in normal use.  LBM_DEBUG_WITHHOLD_TMA: every
                           fused-kernel CTA skips the TMA copies of its
                           second staged plane, so that its bounded wait
                           (1 s) expires and lbm_sync reports LBM_ETIMEOUT;
                           exercises the timeout path without a fault.
                           LBM_DEBUG_CONVERT_BEFORE_FMA and
                           LBM_DEBUG_SMALL_FILM_QUEUE: see below */
  double nucleus_radius; /* radius of the nuclei lbm_seed_bubbles samples
                            when given no bubble list (Sec. 3: random
                            nucleation sites); default 3 cells */
  int32_t mass_residual; /* 16-bit storages only; 0 (default) or 1.  With
                            1 every cell keeps an FP32 rounding residual:
                            what the rounding of its stored populations took
                            off in the last step (the blowing agent's deposit
                            included) joins the cell's mass in its next
                            collision, so stored mass plus residuals is
                            conserved to FP32 rounding, and a deposit far
                            below a 16-bit quantum is kept (Sec. 3: gas is
                            added every step until the agent is finished).
                            The residual is part of population 0 in every
                            read-back and diagnostic; it costs 8 bytes per
                            lattice update on top of 2 Q x 2 */
} lbm_config;

#define LBM_DEBUG_WITHHOLD_TMA 1
/* 16-bit storages: the x-pair kernels convert each stored value to FP32
   before the relaxation's FMA even where 1 - omega is itself a 16-bit value
   (they otherwise widen it inside the FMA); the results are the same bits,
   which a test checks by comparing the two forms */
#define LBM_DEBUG_CONVERT_BEFORE_FMA 2
/* The film test's midpoint queue holds 16 entries, so that the line walks
   take most midpoints themselves (the path of a lattice with more than
   2^20 midpoints); the results are the same */
#define LBM_DEBUG_SMALL_FILM_QUEUE 4

typedef struct {
  double x, y, z, r; /* centre (cell coordinates; z = 0 in 2-D) and radius */
} lbm_bubble;

/* Fill *cfg with defaults: D3Q19, F32, 64^3, tau 1, G -5, rho0 1,
 * rho_ref 1, threshold 1, automatic kernel, default stream, cudaMalloc,
 * nucleus radius 3. */
void lbm_config_default(lbm_config *cfg);

/* Create a context on the current CUDA device and allocate its two
 * population lattices: the lattice on which the Shan-Chen model of Sec. 3.1
 * runs its "streams and collisions" (the paper runs it in OpenLB; the
 * lattice type, extents, tau, G and the psi scale rho0 of psi = rho0 (1 -
 * exp(-rho/rho0)) are this call's configuration).  Populations are stored
 * as f[i][z][y][x] with the x extent padded to a multiple of 8 elements;
 * lbm_read and lbm_write_f convert to the unpadded layout above.  Errors:
 * EINVAL (extents < 1, nz != 1 for D2Q9, an extent above 2^20 or more than
 * 2^31 - 1 padded cells, tau not finite and > 0.5, rho0 <= 0, G not
 * finite, unknown enum, alloc without free), ENOMEM, ECUDA.  *out is NULL
 * on failure. */
lbm_status lbm_create(const lbm_config *cfg, lbm_ctx **out);

/* Release all device memory of the context (after synchronising its
 * stream).  NULL is ignored. */
void lbm_destroy(lbm_ctx *ctx);

/* Random nucleation sites (Sec. 3: nucleation positions from a random
 * function) drawn by rejection sampling from SplitMix64 keyed by
 * seed ^ 0x7369746573000000.  Candidate m uses outputs 4m..4m+3 (as doubles
 * (u >> 11) * 2^-53): centre (floor(u0 nx), floor(u1 ny), floor(u2 nz)),
 * radius r_min + (r_max - r_min) u3; it is accepted when its minimum-image
 * distance to every accepted centre is >= max(min_spacing, r_a + r_b +
 * min_gap).  Pure host function; writes n bubbles to out.  Errors: EINVAL
 * (bad sizes), ESTATE (fewer than n accepted within max_tries; *out holds
 * the accepted ones and *got their count). */
lbm_status lbm_sample_sites(int64_t nx, int64_t ny, int64_t nz, int32_t n,
                            double r_min, double r_max, double min_spacing,
                            double min_gap, uint64_t seed, int64_t max_tries,
                            lbm_bubble *out, int32_t *got);

/* Initial state (Sec. 3.1: a time-random model places the nucleation
 * sites; every other lattice point is filled with liquid).  b is a host
 * array of n bubbles, or NULL: then n nuclei of radius cfg.nucleus_radius
 * are drawn from `seed` exactly as lbm_sample_sites(nx, ny, nz, n, r, r,
 * min_spacing, 0, seed) draws them (min_spacing is used only in that case;
 * lbm_read_sites returns the drawn list).  With s = min over bubbles of
 * (minimum-image distance - r),
 *   rho = rho_g + (rho_l - rho_g)/2 (1 + tanh(2 s / width))
 * (rho = rho_l when n = 0), plus noise_amp*(2u - 1) with u the SplitMix64
 * output at the cell's linear index keyed by seed ^ 0x6E6F697365000000, then
 * f_i = w_i rho (equilibrium at rest).  The bubble centres, rounded to the
 * nearest cell, become the injection sites (in order).  Resets the step
 * counter, disables injection and clears the label history.  Errors:
 * EINVAL (n < 0, non-finite values, width <= 0, min_spacing < 0 when
 * sampling), ESTATE (fewer than n nuclei fit the spacing rule; nothing is
 * seeded). */
lbm_status lbm_seed_bubbles(lbm_ctx *ctx, const lbm_bubble *b, int32_t n,
                            double rho_l, double rho_g, double width,
                            double noise_amp, double min_spacing, uint64_t seed);

/* The bubbles of the last lbm_seed_bubbles call (given or drawn), in site
 * order; n must equal their number.  Host only.  Errors: EINVAL, ESTATE
 * (not seeded). */
lbm_status lbm_read_sites(const lbm_ctx *ctx, lbm_bubble *out, int32_t n);

/* Virtual blowing agent (Sec. 3: gas added to each bubble every step until
 * the agent is finished).  rate[s] and budget[s] (host, n = number of seeded
 * bubbles) set, per site s, the mass added per step and the total left:
 * each step dm = min(rate, budget), budget -= dm (FP64), and w_i*dm is added
 * to f*_i at the site cell after collision.  n = 0 disables injection.
 * Errors: EINVAL (n not 0 or the seeded count, negative values). */
lbm_status lbm_inject(lbm_ctx *ctx, const double *rate, const double *budget,
                      int32_t n);

/* Copy the remaining FP64 budgets (n = number of sites) to host. */
lbm_status lbm_read_budgets(lbm_ctx *ctx, double *budget, int32_t n);

/* Where the blowing agent goes.  mode 0 (default): w_i dm into the site
 * cell's post-collision populations inside the step.  mode 1: spread over
 * the site's bubble, the gas component holding the site cell at the start
 * of each lbm_step call: after every step, the dm of the bubble's sites
 * (taken in increasing site order from their FP64 budgets) is divided
 * evenly over the bubble's cells, each getting w_i dm / n on its
 * post-streaming populations; a site whose cell is liquid deposits at that
 * cell.  In mode 1 lbm_step labels the gas of its starting state and
 * synchronises once to read the sites' labels.  Mode 1 needs FP64 or FP32
 * storage (a deposit per cell is below a 16-bit offset's resolution).
 * Errors: EINVAL. */
lbm_status lbm_set_injection_mode(lbm_ctx *ctx, int32_t mode);

/* Advance nsteps time steps (asynchronous on the context stream).  Errors:
 * ESTATE (not seeded), EINVAL (nsteps < 0), ECUDA, or a sticky ETIMEOUT from
 * an earlier step. */
lbm_status lbm_step(lbm_ctx *ctx, int64_t nsteps);

/* Autotuner: time every fused-kernel tile that fits this lattice and storage,
 * each with the planned number of z chunks (fewest staged planes per CTA
 * slot when CTAs run in waves), half and double it, and the number that
 * fills the resident CTA slots once (two warm-up steps, then the best of
 * two rounds of `steps` timed steps, starting from the current state), and
 * keep the fastest for later lbm_step calls.  The populations, budgets and
 * step counter are restored afterwards, so the call has no effect on
 * results.  *best_tile and *best_ms (either may be NULL) receive the chosen
 * tile id and its time per step.  Errors: ESTATE (not seeded), EINVAL
 * (two-pass context, steps < 1), ENOMEM, ECUDA. */
lbm_status lbm_autotune(lbm_ctx *ctx, int32_t steps, int32_t *best_tile, double *best_ms);

/* Launch plan of the step kernel: out = {kernel (lbm_kernel), tile id,
 * tile x extent, tile y extent, z chunks, CTAs per step}; tile
 * fields are 0 for the two-pass kernel. */
lbm_status lbm_plan_info(const lbm_ctx *ctx, int32_t out[6]);

/* Number of steps taken since seeding. */
int64_t lbm_step_count(const lbm_ctx *ctx);

/* Wait for all work of the context; reports device-side timeouts. */
lbm_status lbm_sync(lbm_ctx *ctx);

/* Rupture criterion of Sec. 3.1 / Sec. 4: second derivative of the EOS
 * pressure (computed in FP64 from the current populations).  line == NULL:
 * out receives the full periodic Laplacian (count must be N).  Otherwise
 * line = {x, y, z, axis, len}: out[m] = p(x+e) - 2p(x) + p(x-e) at the len
 * cells (x, y, z) + m*e_axis (periodic; axis 0, 1 or 2; count must be len).
 * Synchronous.  Errors: EINVAL, ESTATE, ENUMERIC (non-finite density). */
lbm_status lbm_pressure_laplacian(lbm_ctx *ctx, double *out, int64_t count,
                                  const int64_t *line);

/* Film between two bubbles (Sec. 3.1 / Sec. 4: the second derivative of the
 * pressure across the film is the rupture criterion).  line = {x, y, z,
 * axis, len}: len cells from (x,y,z) along the axis, starting inside bubble
 * A and ending inside bubble B.  With rho_mid the density separating gas
 * from liquid: x1 = first upward crossing of rho_mid along the line, x2 =
 * the next downward crossing (linear interpolation between cells, in cells
 * from the start), h = x2 - x1 the film thickness, d2p_mid = p(c+e) - 2p(c)
 * + p(c-e) at the line cell c nearest to (x1+x2)/2 (FP64 EOS pressure; the
 * mean of the two cells when the midpoint is exactly half-way), r_d = half
 * the number of rows along the next axis ((axis+1) mod dims), contiguous
 * with the midpoint row, whose liquid run along the axis through the
 * midpoint column is no thicker than h + 2 (the film disc radius of Sec. 3).
 * found = 0 when no such film exists (the bubbles have merged).
 * Synchronous. */
typedef struct {
  int32_t found;
  double x1, x2, h, d2p_mid, r_d;
} lbm_film;
lbm_status lbm_film_probe(lbm_ctx *ctx, const int64_t *line, double rho_mid, lbm_film *out);

/* Rupture criterion of Sec. 3.1 (eta_m switches when d2p/dn2 = 0 across the
 * film; Sec. 4: rupture starts at that point).  Advance in chunks of
 * diag_every steps, probing the film after each chunk (lbm_film_probe).
 * Exact zeros do not occur in floating point, and a thick film's liquid
 * plateau has d2p/dn2 ~ 0 trivially (acoustic transients swing it either
 * way), so the criterion applies to a thin film, h <= h_max: it is armed
 * once the midpoint value has been below -eps_arm, disarmed whenever the
 * film is thicker than h_max, and fires at the first probe of a thin film
 * where it is >= 0.  Stops when it fires, when a probe finds no film
 * (merged = 1: the bubbles joined before the criterion), or after
 * max_steps.  On firing: fired = 1; h_c = the film thickness where
 * d2p/dn2 crosses zero, interpolated linearly in d2p between the previous
 * probe (d2p < 0) and the firing probe (d2p >= 0):
 *   h_c = h_prev + (h - h_prev) * (-d_prev) / (d - d_prev),
 * which removes the dependence on diag_every (the film thins by ~0.01
 * cells per step near rupture); h_probe and r_d are those of the firing
 * probe.  out->steps = steps taken by this call.  Synchronous. */
typedef struct {
  int32_t fired, merged;
  int64_t steps;
  double h_c, h_probe, r_d;
} lbm_rupture;
lbm_status lbm_run_until_rupture(lbm_ctx *ctx, const int64_t *line, double rho_mid,
                                  double eps_arm, double h_max, int64_t diag_every,
                                  int64_t max_steps, lbm_rupture *out);

/* Gas connected-component labelling, the bubble identification behind the
 * paper's count of merging defects (Sec. 4) and the merge events of its
 * foam runs (Sec. 3: bubbles merge by film rupture): gas cells are
 * rho < gas_threshold (FP64 density), face-connected (4 in 2-D, 6 in 3-D)
 * with periodic wrap; each gas cell gets the smallest linear index of its
 * component, liquid cells -1.  labels: host array of N int32 or NULL;
 * *ncomp receives the number of components (may be NULL).  Synchronous.
 * Errors: EINVAL, ESTATE (not seeded), ENUMERIC, ECUDA. */
lbm_status lbm_label_gas(lbm_ctx *ctx, int32_t *labels, int64_t *ncomp);

/* The record of one diagnostic interval in a single pass over the
 * populations: FP64 totals as lbm_totals (totals may be NULL), gas labels as
 * lbm_label_gas (labels: host array of N int32 or NULL; *ncomp may be NULL),
 * per-site labels and merge events updated as by lbm_label_gas.
 * Synchronous. */
lbm_status lbm_diagnose(lbm_ctx *ctx, double totals[4], int32_t *labels, int64_t *ncomp);

/* Label of each injection site's cell after the last labelling (-1 when
 * the cell is liquid), and the number of merge events so far: a merge event
 * is a pair of sites whose labels differed at the previous labelling and
 * are equal now (both gas).  site_labels may be NULL. */
lbm_status lbm_site_labels(lbm_ctx *ctx, int32_t *site_labels, int32_t n,
                           int64_t *merge_events);

/* Bubble census (Sec. 4 counts bubbles and merging defects; Fig. 4 compares
 * bubble areas): labels the gas of the current state as lbm_label_gas does
 * (site labels and merge events included), then measures every component.
 * roots[q] / sizes[q] (q < min(ncomp, cap); either array may be NULL) are
 * the label (smallest linear cell index) and the size in cells of the
 * components, in increasing order of the label; *ncomp (may be NULL) is the
 * number of components; hist[b] (b < nbins, 1 <= nbins <= 63; may be NULL)
 * counts components of size 2^b <= s < 2^(b+1), the last bin open-ended.
 * Synchronous.  Errors: EINVAL, ESTATE, ENOMEM, ECUDA. */
lbm_status lbm_bubble_sizes(lbm_ctx *ctx, int64_t *roots, int64_t *sizes, int64_t cap,
                            int64_t *ncomp, int64_t *hist, int32_t nbins);

/* Film test at every lattice point (Sec. 4: the rupture criterion applied
 * "at each lattice point" of a foam).  Labels the gas and computes the FP64
 * EOS pressure of the current state, then for every liquid cell and every
 * lattice axis a (0 = x, 1 = y, 2 = z in user coordinates): walking from the
 * cell along +e_a and -e_a for at most h_max cells to the first gas cell
 * (labels L+ and L-, distances d+ and d-), the cell lies in a film along a
 * when both exist, L+ != L- and the liquid run t = d+ + d- - 1 <= h_max; it
 * is a midpoint of that film when |d+ - d-| <= 1.  At a midpoint,
 * d2p = p(x+e_a) - 2 p(x) + p(x-e_a) drives the two-bubble criterion per
 * (cell, axis): armed when d2p < -eps_arm, fired when armed and d2p >= 0
 * (arming cleared); a (cell, axis) that is not a film midpoint is disarmed.
 * The arming state lives in the context (cleared by lbm_seed_bubbles and
 * lbm_write_f) and carries over between calls.  out receives the counts;
 * fired[q] (q < min(out->fired, cap); may be NULL) the fired (cell, axis)
 * records in increasing (cell, axis) order.  When more than cap fire, which
 * cap of them are returned is unspecified; the counts are exact.
 * Synchronous.  Errors: EINVAL, ESTATE, ENOMEM, ECUDA. */
typedef struct {
  int64_t film;      /* (cell, axis) pairs lying in a film */
  int64_t midpoints; /* ... of them film midpoints */
  int64_t armed;     /* (cell, axis) pairs armed after this call */
  int64_t fired;     /* (cell, axis) pairs whose criterion fired in this call */
} lbm_film_census;
typedef struct {
  int64_t cell;                   /* linear index x + nx (y + ny z) */
  int32_t axis;                   /* 0, 1, 2 */
  int32_t label_minus, label_plus; /* bubbles on the -axis and +axis sides */
  int32_t thickness;              /* liquid cells between them */
  double d2p;                     /* second difference of p along the axis */
} lbm_film_cell;
lbm_status lbm_film_cells(lbm_ctx *ctx, int32_t h_max, double eps_arm, lbm_film_census *out,
                          lbm_film_cell *fired, int64_t cap);

/* The same film test (same arming state, same census), reported per pair
 * of bubbles that meet in a film: the criterion "at each lattice point" of
 * a foam (Sec. 4) gives each pair's film disc and critical thickness, the
 * two quantities of Fig. 3.  For a pair (gas labels label_a < label_b) and a
 * lattice axis, the lines along the axis holding a film midpoint of the
 * pair are its film's area in cells (a film of even thickness has two
 * midpoints on a line).  The pair's film lies across the axis with the most
 * lines (the lower axis on a tie); r_d = sqrt(lines / pi) in 3-D, lines / 2
 * in 2-D; h_min is the thinnest liquid run there.  fired counts the pair's
 * midpoints whose criterion fired in this call (any axis) and h_c is their
 * mean thickness (0 when none fired).  pairs[q] for q < min(*npairs, cap),
 * in increasing (label_a, label_b) order; *npairs (may be NULL) = all pairs.
 * Use either this call or lbm_film_cells per diagnostic interval: each
 * advances the arming state.  Synchronous.  Errors: EINVAL, ESTATE, ENOMEM,
 * ECUDA. */
typedef struct {
  int32_t label_a, label_b; /* the two bubbles, label_a < label_b */
  int32_t axis;             /* 0, 1, 2: the axis the film lies across */
  int32_t h_min;            /* thinnest liquid run of the film along axis */
  int64_t lines;            /* lattice lines along axis through the film */
  int64_t midpoints;        /* film midpoints of the pair along axis */
  int64_t fired;            /* midpoints of the pair that fired in this call */
  double r_d;               /* film disc radius */
  double h_c;               /* mean thickness of the fired midpoints */
} lbm_film_pair;
lbm_status lbm_film_pairs(lbm_ctx *ctx, int32_t h_max, double eps_arm, lbm_film_census *census,
                          lbm_film_pair *pairs, int64_t cap, int64_t *npairs);

/* One diagnostic interval in one call and one synchronisation: the FP64
 * totals and gas labels of the current state (lbm_diagnose; labels[N] to
 * host when labels is not NULL), the site
 * labels and merge events (read afterwards with lbm_site_labels), the film
 * test at every lattice point (lbm_film_cells: fired[q] for q < nfired, in
 * (cell, axis) order) and the bubble census (lbm_bubble_sizes: roots[q],
 * sizes[q] for q < nsizes in increasing root order, hist[nbins]).  Results
 * are those of the separate calls on the same state; any output array may
 * be NULL (its cap is then ignored).  Errors: EINVAL, ESTATE, ENOMEM,
 * ECUDA. */
typedef struct {
  double totals[4];      /* as lbm_totals */
  int64_t ncomp;         /* gas components */
  int64_t merge_events;  /* cumulative, as lbm_site_labels */
  lbm_film_census film;  /* as lbm_film_cells */
  int64_t nfired;        /* fired records written */
  int64_t nsizes;        /* census entries written */
} lbm_interval_report;
lbm_status lbm_diagnostic_interval(lbm_ctx *ctx, int32_t h_max, double eps_arm, int32_t *labels,
                                   lbm_film_cell *fired, int64_t fired_cap, int64_t *roots,
                                   int64_t *sizes, int64_t sizes_cap, int64_t *hist,
                                   int32_t nbins, lbm_interval_report *out);

/* FP64 totals: out[0] = sum rho, out[1..3] = sum j over all cells, with a
 * fixed-order block reduction (repeated calls give identical bits).  FP64
 * storage sums every population in FP64; the FP32-arithmetic storages sum
 * the offsets f_i - w_i rho_ref of a cell in FP32 and the cells in
 * compensated FP32 / FP64 (mass = N rho_ref + sum of offsets).
 * Synchronous. */
lbm_status lbm_totals(lbm_ctx *ctx, double out[4]);

/* Copy a field (doubles, see lbm_field) to host: the density, pressure and
 * velocity fields are the quantities whose profiles Fig. 2 plots across the
 * film (Sec. 4), with p the EOS of Sec. 3.1 and psi its pseudopotential;
 * LBM_F returns the populations themselves.  bytes must be exactly the
 * field's size.  Synchronous.  Errors: EINVAL (NULL, unknown field, wrong
 * size), ESTATE (not seeded), ENUMERIC (non-finite density), ECUDA. */
lbm_status lbm_read(lbm_ctx *ctx, int32_t field, double *host_dst, size_t bytes);

/* Overwrite the populations with host data f[i*N + cell] (doubles, rounded
 * to the storage precision); marks the context seeded.  bytes = Q*N*8. */
lbm_status lbm_write_f(lbm_ctx *ctx, const double *host_src, size_t bytes);

/* ---- batched ensemble of independent two-bubble D2Q9 domains ------------
 * The bubble-size sweep of Sec. 4 (Fig. 3: critical film thickness h_c
 * against the film-disc radius R_d) runs many uneven lattices at once, and
 * every diag_every steps a probe measures each domain's film
 * (lbm_film_probe) and advances its rupture state machine
 * (lbm_run_until_rupture) on the device.  Domains whose criterion fired, or
 * whose film is gone, stop.  Storage is FP32 offset form
 * (f_i - w_i rho_ref), arithmetic FP32, probes FP64.  The steps run as one
 * launch per time step and tile class over every active domain, or as
 * persistent launches (lbm_ensemble_set_launch); the results do not depend
 * on which. */
typedef struct {
  int64_t nx, ny;          /* extents: 8..4096, nx a multiple of 4 */
  double tau, G, rho0, rho_ref;
  double rho_l, rho_g, width, noise_amp; /* initial state as lbm_seed_bubbles */
  uint64_t seed;
  int32_t nbubbles;        /* 0..4 */
  lbm_bubble bubbles[4];   /* centres (x, y, 0) and radii */
  int64_t line[5];         /* film probe line {x, y, 0, axis 0/1, len} */
  double rho_mid;          /* gas / liquid separating density of the probe */
} lbm_domain;

typedef struct lbm_ensemble lbm_ensemble; /* opaque */

/* Create an ensemble of n domains on the current device (one arena; the
 * allocator callbacks as in lbm_config, NULL for cudaMalloc) and seed every
 * domain.  diag_every must be even.  Errors: EINVAL, ENOMEM, ECUDA. */
lbm_status lbm_ensemble_create(const lbm_domain *dom, int32_t n, double eps_arm,
                               double h_max, int32_t diag_every, lbm_alloc_fn alloc,
                               lbm_free_fn free, void *alloc_user, lbm_ensemble **out);
void lbm_ensemble_destroy(lbm_ensemble *ens);

/* Run until every domain has stopped or max_steps more steps were taken
 * (whole diagnostic intervals).  *steps_done (may be NULL) receives the
 * steps taken.  Synchronous. */
lbm_status lbm_ensemble_run(lbm_ensemble *ens, int64_t max_steps, int64_t *steps_done);

/* Per domain: fired / merged flags, the step at which it stopped (or the
 * steps so far), h_c (interpolated zero crossing), h_probe and r_d at
 * firing, as lbm_run_until_rupture. */
lbm_status lbm_ensemble_results(const lbm_ensemble *ens, lbm_rupture *out, int32_t n);

/* out = {steps taken, lattice updates performed (sum over domains of cells x
 * steps while active), active domains, kernel launches}. */
lbm_status lbm_ensemble_stats(const lbm_ensemble *ens, double out[4]);

/* Current populations of one domain as doubles f[i*N + x + nx*y]. */
lbm_status lbm_ensemble_read_f(lbm_ensemble *ens, int32_t domain, double *host, size_t bytes);

/* How lbm_ensemble_run launches the steps (not in the paper, which gives no
 * implementation); the results do not depend on it.
 * LBM_ENS_GRAPH: one launch per step and tile class over every active
 *   domain, captured with the probe in a CUDA graph per interval.
 * LBM_ENS_TEMPORAL: one launch per S steps (S = 2 or 5, diag_every a
 *   multiple of 2 S): a CTA takes a tile of one domain with a halo of 2 S
 *   cells through S steps in shared memory.
 * LBM_ENS_PERSISTENT: per-step launches until the active domains' work
 *   items (tiles of 128 columns x chunks of rows) fit in one wave of CTAs,
 *   then one cooperative launch per ten intervals, in which every CTA keeps
 *   its work item, waits between steps only for the items at most two
 *   chunks and two tiles away, and the domain's first CTA runs the probe.
 * LBM_ENS_AUTO (the default): the per-interval launches chosen by measured
 *   time as the active set shrinks.
 * LBM_ENS_DEBUG_WITHHOLD_FLAG (tests only): as PERSISTENT, but the first
 *   CTA of every persistent launch never releases its step flag, so the
 *   bounded waits (1 s) expire and lbm_ensemble_run returns LBM_ETIMEOUT;
 *   exercises the timeout path without a fault.
 * Errors: EINVAL (NULL, unknown mode), ETIMEOUT (after a timed-out launch),
 * ECUDA. */
#define LBM_ENS_AUTO 0
#define LBM_ENS_GRAPH 1
#define LBM_ENS_DEBUG_WITHHOLD_FLAG 2
#define LBM_ENS_PERSISTENT 3
#define LBM_ENS_TEMPORAL 4
lbm_status lbm_ensemble_set_launch(lbm_ensemble *ens, int32_t mode);

/* ---- multi-lattice Shan-Chen model (Sec. 3.1, Fig. 1) -------------------
 * The paper's modified model puts each phase on its own lattice: every
 * bubble on one, the fluid on another (Fig. 1 steps 3-5); the lattices are
 * coupled and their interactions computed (step 6); eta_m switches the
 * barrier algorithm off when d2p/dn2 = 0 across the film, and the bubbles
 * merge (Sec. 3.1; lattices merged, steps 8-9).  The paper gives no
 * equations for it; this library's reading: lattice 0 holds the fluid and
 * lattice k = 1 .. nl-1 the gas of bubble k, coupled by the multicomponent
 * Shan-Chen force
 *   F_s(x) = -psi_s(x) sum_t Gm[s][t] sum_i w_i psi_t(x + c_i) c_i,
 * psi_s = rho0 (1 - exp(-rho_s/rho0)), with Gm[0][0] = G (the fluid's own
 * attraction: nl = 1 is the single-component model of lbm_step), Gm[0][k] =
 * Gm[k][0] = G_x (fluid and gas), Gm[k][k] = 0 and, between two bubbles,
 * Gm[k][l] = eta_m(k, l) G_b (the barrier; eta_m = 1 until the criterion
 * fires).  Every lattice relaxes with tau towards f_eq(rho_s, u_s),
 *   u' = sum_s j_s / sum_s rho_s,  u_s = u' + tau F_s / rho_s
 * (u_s = u' where rho_s = 0: an empty lattice has f_eq = 0), then streams.  Populations are plain FP64 or FP32 values f[s][i][cell] (same
 * cell order and velocity order as above).  The pressure of the coupled
 * lattices is p = rho_total/3 + 1/6 sum_s sum_t Gm[s][t] psi_s psi_t (the
 * EOS of Sec. 3.1 for nl = 1). */
typedef struct lbm_ml_ctx lbm_ml_ctx; /* opaque */
typedef struct {
  int32_t lattice;       /* LBM_D2Q9 or LBM_D3Q19 */
  int32_t storage;       /* LBM_F64 or LBM_F32 */
  int64_t nx, ny, nz;    /* periodic extents; nz = 1 for D2Q9 */
  int32_t nl;            /* lattices, 1..8: the fluid and nl - 1 bubbles */
  double tau, rho0;
  double G, G_x, G_b;    /* fluid self-coupling, fluid-gas, inter-bubble barrier */
  void *stream;          /* cudaStream_t, may be NULL */
  lbm_alloc_fn alloc;    /* NULL: cudaMalloc/cudaFree */
  lbm_free_fn free;
  void *alloc_user;
} lbm_ml_config;

/* Defaults: D2Q9, FP64, 128^2, nl 3, tau 1, rho0 1, G -5, G_x 1, G_b 0. */
void lbm_ml_config_default(lbm_ml_config *cfg);
/* Create on the current device.  Errors: EINVAL (as lbm_create; nl outside
 * 1..8, storage not FP64/FP32, non-finite couplings), ENOMEM. */
lbm_status lbm_ml_create(const lbm_ml_config *cfg, lbm_ml_ctx **out);
void lbm_ml_destroy(lbm_ml_ctx *ctx);
/* The coupling matrix in use (nl x nl, row-major): it changes only when a
 * pair merges. */
lbm_status lbm_ml_coupling(const lbm_ml_ctx *ctx, double *Gm);
/* Initial state (Sec. 3.1: bubbles at the nucleation sites, the fluid
 * elsewhere): b holds the nl - 1 bubbles (x, y, z, r).  The fluid lattice
 * gets the profile of lbm_seed_bubbles over all bubbles (liquid rho_l, its
 * vapour rho_v inside, noise from seed); bubble k's lattice gets rho_gas
 * inside bubble k with the same tanh profile (zero far outside, no noise);
 * f = w rho at rest.  The bubble centres, rounded, are the injection
 * sites, site k depositing into lattice k.  Every barrier is switched on
 * (eta_m = 1).  Synchronous.  Errors: EINVAL. */
lbm_status lbm_ml_seed(lbm_ml_ctx *ctx, const lbm_bubble *b, double rho_l, double rho_v,
                       double rho_gas, double width, double noise_amp, uint64_t seed);
/* Populations as doubles f[(s*Q + i)*N + cell] (bytes = nl*Q*N*8), written
 * (rounded to the storage) or read.  Synchronous. */
lbm_status lbm_ml_write_f(lbm_ml_ctx *ctx, const double *f, size_t bytes);
lbm_status lbm_ml_read_f(lbm_ml_ctx *ctx, double *f, size_t bytes);
/* Virtual blowing agent (Sec. 3), one site per bubble: each step dm =
 * min(rate[k], budget[k]) leaves the FP64 budget and w_i dm joins lattice
 * k + 1's post-collision populations at the site.  n = nl - 1, or 0 to
 * stop.  Errors: EINVAL, ESTATE. */
lbm_status lbm_ml_inject(lbm_ml_ctx *ctx, const double *rate, const double *budget, int32_t n);
lbm_status lbm_ml_read_budgets(lbm_ml_ctx *ctx, double *budget, int32_t n);
/* Advance nsteps (asynchronous on the stream).  Errors: EINVAL, ESTATE, ECUDA. */
lbm_status lbm_ml_step(lbm_ml_ctx *ctx, int64_t nsteps);
int64_t lbm_ml_step_count(const lbm_ml_ctx *ctx);
/* eta_m(k, l) = 0 (Sec. 3.1): bubble l's lattice is merged into bubble k's
 * (f_k += f_l, f_l = 0) and their barrier coupling removed.  Synchronous. */
lbm_status lbm_ml_merge(lbm_ml_ctx *ctx, int32_t k, int32_t l);
/* FP64 fields to host: rho (nl*N: every lattice's density, may be NULL) and
 * p (N: the pressure of the coupled lattices, may be NULL).  Synchronous. */
lbm_status lbm_ml_fields(lbm_ml_ctx *ctx, double *rho, double *p);
/* The rupture criterion of lbm_run_until_rupture (Sec. 3.1 / Sec. 4) on
 * this model: the film is found on the fluid lattice's density, its
 * d2p/dn2 on the coupled pressure.  When it fires, eta_m of the pair (k, l)
 * becomes 0 and their lattices merge (lbm_ml_merge); a film that vanishes
 * first is reported as merged.  Synchronous. */
lbm_status lbm_ml_run_until_rupture(lbm_ml_ctx *ctx, const int64_t *line, double rho_mid,
                                     double eps_arm, double h_max, int64_t diag_every,
                                     int64_t max_steps, int32_t k, int32_t l, lbm_rupture *out);

/* Allocation-free time step.  The paper has no counterpart: this entry point
 * serves callers that cannot allocate device memory - a host framework that
 * owns the whole device-memory pool and forbids allocations behind its
 * back, a time loop that must not stall on the allocator (cudaMalloc and
 * cudaFree can synchronise the device), a program held to a fixed
 * device-memory budget.  It advances FP32 populations f_in -> f_out by one
 * step of the two-pass kernels (no injection).  Layout: Q fields of
 * nx*ny*nz floats, f[i*N + cell], cell = x + nx*(y + ny*z), the
 * post-streaming form lbm_read(LBM_F) returns, plain values (no offset).
 * The psi field passed between the two kernels lives in a file-scope device
 * array of 2,097,152 floats (8 MB) that every GPU loading the library holds
 * until the process exits; lattices of more cells are rejected with
 * LBM_EINVAL (the product is bounded without overflow).  The first call in
 * each CUDA context (the current one: the device's primary context, or a
 * driver context the caller made current) looks up that array's device
 * address and caches it under the context's process-unique id; make that
 * first call before any stream capture.  Every call uses the same array,
 * which keeps the last call's psi: calls that overlap on the GPU (other
 * streams or threads without ordering) race on it.  f_in and f_out are
 * distinct device buffers owned by the caller; stream may be NULL.
 * Asynchronous; no memory is allocated or freed.  Errors: EINVAL (unknown
 * lattice, extents < 1 or nz != 1 for D2Q9, more than 2,097,152 cells, tau
 * not finite and > 0.5, rho0 not finite and > 0, G not finite, NULL or
 * aliased buffers), ECUDA. */
lbm_status lbm_step_static_f32(int32_t lattice, int64_t nx, int64_t ny, int64_t nz, double tau,
                               double G, double rho0, const float *f_in, float *f_out,
                               void *stream);

/* FP64 fused multiply-add rate of the current device, measured: a kernel
 * of independent chains of dependent FMAs (8 per thread, `iters` rounds)
 * over every SM, the fastest of three timed launches (CUDA events, after one
 * warm-up launch).  *tflops = 2 * FMAs / seconds / 1e12.  The paper has no
 * counterpart: this is the denominator of the FP64 storage form's roofline,
 * whose step kernel is bound by the FP64 pipe.  Synchronous (legacy default
 * stream).  Errors: EINVAL, ECUDA. */
lbm_status lbm_fp64_rate(int32_t iters, double *tflops);

/* Message of the calling thread's last failure ("" if none). */
const char *lbm_last_error(void);

/* Library version string. */
const char *lbm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SCLBM_LBM_H */
