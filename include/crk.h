/* crk.h -- C ABI of the GB300 CRKSPH neighbor-sum library (libcrk).
 *
 * The library evaluates the hydrodynamic hot path of CRK-HACC (arXiv
 * 2511.21921) for gas particles in periodic boxes:
 *
 *   crk_cell_build  -- Morton sort, bucket tree and per-particle neighbor
 *                      lists (the paper's GPU tree with few rebuilds, Sec. 2.9).
 *   crk_moments     -- gas volume V (App. A.2, Eq. Vg), geometric moments and
 *                      reproducing-kernel coefficients A, B, grad A, grad B
 *                      (App. A.1, Eq. RK; closed forms from the reproducing
 *                      conditions of the CRKSPH formulation the paper cites).
 *   crk_rates       -- RK density (Sec. 2.5.1, Eq. rhow, gas only), velocity
 *                      gradient (App. A.1, Eq. gradv), ideal-gas EOS with
 *                      gamma from the parameters (5/3, Sec. 2.4.1), relaxation
 *                      flag (App. A.1), and pairwise momentum and compatible
 *                      energy rates with limited artificial viscosity (Sec. 2.1).
 *   crk_adjoint     -- vector-Jacobian product of the rates with respect to
 *                      positions, velocities, internal energies and smoothing
 *                      lengths (no counterpart in the paper; it gives the
 *                      subgrid calibration of Sec. 3 a gradient).
 *   crk_set_species, crk_volume_gw
 *                   -- wind particles in the gas density (Sec. 2.5.1).
 *   crk_leaf_mark, crk_time_bins, crk_moments_active, crk_rates_active
 *                   -- active-set evaluation: passive particles reuse their
 *                      stored coefficients and fields (App. A.1).
 *   crk_hdot, crk_kick, crk_kick_refined, crk_drift
 *                   -- the time step around the rates: smoothing-length rate
 *                      and exponential drifts (App. A.3), kick-drift-kick with
 *                      refined kicks and parabolic passive drifts (App. A.4).
 *   crk_cool_exact  -- exact integration of radiative cooling and heating over
 *                      a step (Sec. 2.3.2).
 *   crk_subgrid_volume, crk_subgrid_deposit
 *                   -- subgrid particles over the gas: scatter volumes (App.
 *                      A.2) and normalised kernel deposits (Secs. 2.5-2.7).
 *
 * Conventions shared by every entry point:
 *  - Device pointers are owned by the caller; the library never allocates
 *    device or pinned memory.  All scratch lives in the caller's workspace
 *    `ws` of at least crk_workspace_size() bytes (256-byte aligned).
 *  - Arrays are structure-of-arrays in the caller's particle order:
 *    a vector field of n particles is [3][n] (component-major); n <= 2^30.
 *  - Element type: positions `x` and box sides are always double.  Every other
 *    real array is double when params.precision == CRK_FP64 and float when
 *    params.precision == CRK_MIXED32.
 *  - Calls are asynchronous on `stream` and never synchronise the host, so a
 *    sequence of them can be captured in a CUDA graph -- except
 *    crk_status_poll, crk_stats and crk_neighbors_csr, which synchronise.
 *  - Argument errors are returned immediately.  Data errors found on the
 *    device (x outside [0, L), h >= L/2, non-finite input, singular second
 *    moment, list capacity exceeded) set a device status word that
 *    crk_status_poll returns (and clears; crk_cell_build also clears it when
 *    it starts); outputs of a call that set it are undefined.
 *    No kernel traps or waits without a bound.
 */
#ifndef CRK_H
#define CRK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* crk_stream_t; /* a cudaStream_t; NULL = legacy default */

typedef enum {
  CRK_OK = 0,
  CRK_EINVAL = 1,      /* bad argument (NULL pointer, size, parameter) */
  CRK_ENOMEM = 2,      /* workspace too small or neighbor-list capacity exceeded */
  CRK_ECUDA = 3,       /* a CUDA runtime call failed */
  CRK_EDOMAIN = 4,     /* some x outside [0, L) or h outside (0, L/2) */
  CRK_ENONFINITE = 5,  /* NaN or Inf in an input */
  CRK_ESINGULAR = 6,   /* second moment m2 singular for some particle (it falls back to A=1, B=0) */
  CRK_ETIMEOUT = 7,    /* a bounded device wait gave up */
  CRK_ESTATE = 8,      /* call out of order (e.g. crk_rates before crk_moments) */
  CRK_EBOUNDS = 9      /* bounds-checked build only: a kernel met an index out of range
                          (the access was skipped; outputs are undefined) */
} crk_status;

typedef enum {
  CRK_FP64 = 0,    /* every sum and pair term in double (the plain FP64 form) */
  CRK_MIXED32 = 1  /* float pair arithmetic and accumulation; double-equivalent
                      minimum-image separations; double 3x3 inverse of m2 */
} crk_precision;

typedef struct {
  double gamma;     /* adiabatic index; 5/3 for a monatomic ideal gas (Sec. 2.4.1) */
  double Cl, Cq;    /* linear / quadratic artificial-viscosity coefficients */
  double eps2;      /* softening of the viscosity denominator |eta|^2 + eps2 */
  double eta_crit;  /* near-field damping applies when min(r/h_i, r/h_j) < eta_crit */
  double eta_fold;  /* width of the near-field damping exp(-((eta-eta_crit)/eta_fold)^2) */
  double relax_dt;  /* relaxation time step (App. A.1); 0 turns relaxation off */
  int32_t limiter;  /* 1: velocity-gradient limiter on the viscosity; 0: off */
  int32_t precision;/* crk_precision */
  int32_t nbr_cap;  /* neighbor-list slots per particle reserved in the workspace; 0 = 192 */
  int32_t block_threads; /* threads per block of the pair sweeps; 0 = autotuned default */
  int32_t blocks_per_sm; /* resident blocks per SM for the persistent sweeps; 0 = default */
  int32_t prefetch;      /* sweeps prefetch the neighbor record this many list entries ahead
                            into L1; 0 = off */
  int32_t energy_split;  /* compatible energy split of the pair work E_ij = m_i a_ij.(v_j - v_i)
                            (Sec. 2.1): 0 = halves, f_ij = 1/2; 1 = weighted by the specific
                            energies, f_ij = (1 + sgn(E_ij)(u_j - u_i)/(u_i + u_j))/2, so heating
                            goes mostly to the colder particle and cooling is drawn mostly from
                            the hotter one; f_ij + f_ji = 1 either way */
  int32_t q_side;        /* viscosity in the momentum rate: 0 = (P_i + P_j + Q_ij + Q_ji) with
                            (G_ij - G_ji); 1 = per side, (P_i + P_j)(G_ij - G_ji) +
                            2 (Q_ij G_ij - Q_ji G_ji), each Q with its own side's gradient */
} crk_params;

typedef struct crk_plan crk_plan;

/* Fill `p` with the library defaults: gamma = 5/3, Cl = 2, Cq = 1, eps2 = 0.01,
 * eta_crit = 1/n_h for n_h = (3*100/(4 pi))^(1/3), eta_fold = 0.2, relaxation
 * off, limiter on, energy halves, viscosity with the pressures, CRK_MIXED32.
 * Host only. */
void crk_params_default(crk_params* p);

/* Create a plan for up to n_max particles in up to n_boxes_max boxes.  The plan
 * owns host metadata only (sizes, tuned launch shapes, the state of the
 * workspace it last built).  Host only; CRK_EINVAL on bad sizes/parameters. */
crk_status crk_plan_create(const crk_params* params, int64_t n_max, int32_t n_boxes_max,
                           crk_plan** out);
void crk_plan_destroy(crk_plan* plan);

/* Bytes of workspace needed for n particles in n_boxes boxes.  Host only. */
crk_status crk_workspace_size(const crk_plan* plan, int64_t n, int32_t n_boxes, size_t* bytes);

/* (a) Cell-list build.  box_off: device int64[n_boxes+1], box_off[0] = 0,
 * box_off[n_boxes] = n, non-decreasing: particles of box b are
 * [box_off[b], box_off[b+1]).  box_L: device double[n_boxes], side of each
 * periodic box [0, L)^3.  x: device double[3][n].  h: device real[n],
 * 0 < h < L/2.  Sorts the particles by (box, Morton key), builds the bucket
 * tree and the union neighbor lists U(i) = {j != i, |x_ij| < max(h_i, h_j)}
 * with flags for the gather set (|x_ij| < h_i).  Stores everything in ws. */
crk_status crk_cell_build(crk_plan* plan, crk_stream_t stream, void* ws, size_t ws_bytes,
                          int64_t n, int32_t n_boxes, const int64_t* box_off,
                          const double* box_L, const double* x, const void* h);

/* (b) Volume and reproducing-kernel coefficients.  m: device real[n] masses.
 * V_out: optional device real[n].  coef_out: optional device real[16][n]
 * holding A, B[3], gradA[3], gradB[3][3] (gradB[g][a] = d B^a / d x^g). */
crk_status crk_moments(crk_plan* plan, crk_stream_t stream, void* ws, const void* m,
                       void* V_out, void* coef_out);

/* (c) Rates.  v: device real[3][n], u: device real[n] (specific internal
 * energy, >= 0).  Outputs dvdt: real[3][n], dudt: real[n]; optional rho_out:
 * real[n]; optional gradv_out: real[9][n] with gradv[a*3+b] = d v^a / d x^b. */
crk_status crk_rates(crk_plan* plan, crk_stream_t stream, void* ws, const void* v, const void* u,
                     void* dvdt, void* dudt, void* rho_out, void* gradv_out);

/* (d) Adjoint.  Given cotangents g_dvdt real[3][n] and g_dudt real[n] of the
 * rates, accumulate nothing and write the vector-Jacobian products
 * g_x real[3][n], g_v real[3][n], g_u real[n], g_h real[n].  Neighbor sets,
 * image shifts, relaxation flags and limiter branches are held at the primal
 * point.  recompute = 1 re-evaluates the per-particle forward state (volume,
 * coefficients, density, velocity gradient) from v, u and the masses of the
 * last crk_moments; recompute = 0 reuses the state the last crk_rates left in
 * ws (same inputs).  No per-pair data is stored. */
crk_status crk_adjoint(crk_plan* plan, crk_stream_t stream, void* ws, const void* v, const void* u,
                       const void* g_dvdt, const void* g_dudt, void* g_x, void* g_v, void* g_u,
                       void* g_h, int32_t recompute);

/* (d') Rates and their vector-Jacobian product in one pass structure, for
 * cotangents known before the rates (a loss linear in the rates, or lagged
 * cotangents): the density sweep, then the adjoint's pair sweep accumulates
 * the forward rates from the same pair forces it differentiates, then the
 * other reverse sweeps.  Outputs as crk_rates (dvdt, dudt) and crk_adjoint
 * (g_x, g_v, g_u, g_h); the rates agree with crk_rates' to rounding (the pair
 * expressions are the same, the compiler may contract them differently).
 * Requires crk_moments (not the active-set or wind configurations). */
crk_status crk_rates_adjoint(crk_plan* plan, crk_stream_t stream, void* ws, const void* v,
                             const void* u, const void* g_dvdt, const void* g_dudt, void* dvdt,
                             void* dudt, void* g_x, void* g_v, void* g_u, void* g_h);

/* ---- Gas and wind (Sec. 2.5.1, Eq. rhow; App. A.2) -----------------------------
 * Wind particles live in the same boxes, tree and lists as the gas but take
 * part in the density only: the gas density sums over gas and wind neighbors
 * with the volume over gas and wind, V_{g+w}; volume, coefficients, velocity
 * gradient and pair rates stay gas-only; winds get zero rates and, as the
 * subgrid particles they are, are skipped by crk_subgrid_*.  A wind particle's
 * coefficients are reproduced over its gas neighbors (a wind far from gas falls
 * back to the uncorrected kernel without setting CRK_ESINGULAR) and its V is
 * its V_{g+w}. */

/* (o) Species of the particles of the last crk_cell_build: device uint8[n],
 * caller order, 0 gas, nonzero wind; NULL returns to all gas.  Call after
 * every crk_cell_build (a build clears it) and before crk_moments.  With winds
 * present crk_adjoint and the active-set calls return CRK_ESTATE. */
crk_status crk_set_species(crk_plan* plan, crk_stream_t stream, void* ws,
                           const uint8_t* species);

/* (p) The volume over gas and wind of the last crk_moments, device real[n],
 * caller order (equal to crk_moments' V_out when there are no winds). */
crk_status crk_volume_gw(crk_plan* plan, crk_stream_t stream, void* ws, void* Vgw_out);

/* ---- Active-set evaluation (App. A.1; Sec. 2 power-of-two time bins) --------
 * On a step of a time-bin hierarchy only the active particles update their
 * forces; passive particles keep the correction coefficients (and volume,
 * density, velocity gradient) of their last active step.  flags: device
 * uint8[n], caller order; bit 0 (1) active; bit 1 (2) recompute volume and
 * coefficients (implied by bit 0); bit 2 (4) transformed (species conversion,
 * see crk_leaf_mark).  The sweeps run over compacted lists of the flagged
 * particles; the records of the others are packed from the caller's state
 * arrays, which persist between steps in the caller's order. */

/* (l) Leaf marking: set bit 1 on every particle sharing a tree leaf (a bucket
 * of 8 consecutive Morton-sorted particles) with a transformed particle (bit
 * 2), in place, so that the leaf recomputes its coefficients (App. A.1).
 * leaf_out: optional device int32[n], the leaf of every particle.  Requires a
 * built workspace. */
crk_status crk_leaf_mark(crk_plan* plan, crk_stream_t stream, void* ws, uint8_t* flags,
                         int32_t* leaf_out);

/* (l') Power-of-two time bins per leaf (Sec. 2; App. A.4): each leaf takes
 * the level k = the smallest k >= 0 with dt_max / 2^k <= min over its members
 * of dt (device real[n], caller order, a particle's own time-step limit),
 * capped at max_level (0..40); level_out (optional device uint8[n], caller
 * order) receives it.  On sub-step `substep` (0 <= substep < 2^max_level) of
 * the finest level a leaf is active when substep is a multiple of
 * 2^(max_level - k); bit 0 of flags (optional device uint8[n], in/out) is set
 * accordingly and the other bits are kept.  Requires a built workspace. */
crk_status crk_time_bins(crk_plan* plan, crk_stream_t stream, void* ws, const void* dt,
                         double dt_max, int32_t max_level, int64_t substep, uint8_t* level_out,
                         uint8_t* flags);

/* (m) Volume and coefficients of the flagged particles (bit 0 or 1).
 * V_state: device real[n], coef_state: device real[16][n] (layout of
 * crk_moments' coef_out), caller order, in/out: written for flagged particles,
 * read for the others.  Sets up the active list that crk_rates_active uses. */
crk_status crk_moments_active(crk_plan* plan, crk_stream_t stream, void* ws, const void* m,
                              const uint8_t* flags, void* V_state, void* coef_state);

/* (n) Density, velocity gradient and pair rates of the active particles (bit 0
 * of the flags given to the last crk_moments_active).  rho_state: device
 * real[n], gradv_state: device real[9][n], in/out (written for active
 * particles, read for passive ones, whose pressure, sound speed and relaxation
 * flag follow from them as for a fresh evaluation).  dvdt real[3][n], dudt
 * real[n]: written for active particles only.  CRK_ESTATE unless the last
 * moments call on this workspace was crk_moments_active.  crk_hdot may follow;
 * crk_adjoint then needs recompute = 1. */
crk_status crk_rates_active(crk_plan* plan, crk_stream_t stream, void* ws, const void* v,
                            const void* u, void* rho_state, void* gradv_state, void* dvdt,
                            void* dudt);

/* ---- Time step around the rates (App. A.3 and A.4) -------------------------
 * A kick-drift-kick step is: crk_kick (half kick with the rates of the last
 * evaluation), crk_drift (positions, smoothing lengths), crk_cell_build,
 * crk_moments, crk_rates at the new positions, crk_hdot, crk_kick (second
 * half kick).  These four calls are one pass over the particles each; they
 * neither read nor write the workspace except crk_hdot, which reads it.
 * Element types follow params.precision as everywhere else. */

/* (e) Smoothing-length rate (App. A.3, Smoothing Length Integration):
 *   hdot_i = (h^T_i - h_i) / dt_a + h_i (div v)_i / 3,
 *   h^T_i  = h_i (1 - lambda + lambda Delta_N),  Delta_N = n_h V_i^(1/3) / h_i,
 * with V_i the volume of the last crk_moments, (div v)_i the trace of the
 * velocity gradient of the last crk_rates and h_i the smoothing length of the
 * last crk_cell_build.  dt_a > 0: the active time step; lambda: the Thacker
 * weight; n_h > 0: target particles per kernel radius (4 for the paper's
 * gas).  Optional outputs, device real[n] in caller order: hdot_out;
 * hrate_out = hdot_i / h_i (the logarithmic rate that crk_drift takes);
 * div_out = (div v)_i.  CRK_ESTATE before a crk_rates on this workspace. */
crk_status crk_hdot(crk_plan* plan, crk_stream_t stream, void* ws, double dt_a, double lambda,
                    double n_h, void* hdot_out, void* hrate_out, void* div_out);

/* (f) Kick (App. A.4, K): v_out = v0 + dt a and, when u_out is given,
 * u_out = u0 + dt dudt.  dt is the kick length (dt_a/2 for a half kick; the
 * refined first half kick of App. A.4 is this call from v0 with dt_b/2).
 * active: optional device uint8[n]; particles with active[i] == 0 keep v0 (and
 * u0).  v0, a, v_out: device real[3][n]; u0, dudt, u_out: device real[n].
 * Outputs may alias inputs (in-place kicks).  n <= the plan's n_max. */
crk_status crk_kick(crk_plan* plan, crk_stream_t stream, int64_t n, double dt,
                    const uint8_t* active, const void* v0, const void* a, void* v_out,
                    const void* u0, const void* dudt, void* u_out);

/* (g) Completion of a refined step (App. A.4, Adaptive Kick Corrections):
 *   v_out = v0 + a0 (dt_b - dt_c) + (a0 + a1) dt_c / 2
 * (and likewise u from u0, du0, du1 when u_out is given): constant a0 until
 * the last dt_c of the refined interval dt_b, then a plain kick-drift-kick
 * average.  0 <= dt_c <= dt_b.  Layouts and `active` as for crk_kick. */
crk_status crk_kick_refined(crk_plan* plan, crk_stream_t stream, int64_t n, double dt_b,
                            double dt_c, const uint8_t* active, const void* v0, const void* a0,
                            const void* a1, void* v_out, const void* u0, const void* du0,
                            const void* du1, void* u_out);

/* (h) Drift by dt >= 0 (App. A.4, D), in place, and the drifts of App. A.3.
 *   x: device double[3][n], updated in double as x + v dt and wrapped into the
 *      particle's box [0, L) (box_off/box_L as for crk_cell_build); a particle
 *      that moves more than one box side is left outside and the next
 *      crk_cell_build reports CRK_EDOMAIN.
 *   v is v_half (device real[3][n]) or, when a0 (device real[3][n]) is given,
 *      the local half-step velocity of a passive sub-step
 *      v_half + a0 [t_elapse_i + (dt - dt_a_i)/2]; dt_a and t_elapse are
 *      optional device double[n] (the particle's active interval and the time
 *      of it already drifted; defaults dt and 0, an active particle).
 *   h, hrate: optional pair, device real[n]: h <- h exp(hrate dt) with hrate
 *      the logarithmic rate from crk_hdot.
 *   V: optional device real[n] (needs h and n_h > 0): V <- (h / n_h)^3.
 *   rho, div: optional pair, device real[n]: rho <- rho exp(-div dt).
 * In the mixed form the displacement v dt is a float, added in double. */
crk_status crk_drift(crk_plan* plan, crk_stream_t stream, int64_t n, int32_t n_boxes,
                     const int64_t* box_off, const double* box_L, double dt, double* x,
                     const void* v_half, const void* a0, const double* dt_a,
                     const double* t_elapse, void* h, const void* hrate, double n_h, void* V,
                     void* rho, const void* div);

/* ---- Subgrid particles over the gas (App. A.2; Secs. 2.5.3, 2.6.3, 2.7.4) -----
 * Stars, winds and black holes interact with the gas of the last
 * crk_cell_build through its bucket tree.  Subgrid arrays are in the caller's
 * order: box_off_s: device int64[n_boxes+1] (same boxes, same order as the
 * build), x_s: device double[3][n_s] inside their box, h_s: device real[n_s].
 * One warp per subgrid particle; no workspace beyond the built one. */

/* (j) Scatter volume (App. A.2, Eq. Vsg): V_s = 1 / (sum over gas j with
 * r_sj < h_j of W(r_sj, h_j) + W(0, h_s)); optional h_out = n_h V_s^(1/3)
 * (the smoothing length the volume determines; n_h = 2.25 for stars and black
 * holes, 4 for winds in the paper).  V_out, h_out: device real[n_s]. */
crk_status crk_subgrid_volume(crk_plan* plan, crk_stream_t stream, void* ws, int64_t n_s,
                              const int64_t* box_off_s, const double* x_s, const void* h_s,
                              double n_h, void* V_out, void* h_out);

/* (k) Normalised kernel deposit (Eqs. windmetal with Anorm, starmetal, AGNE):
 * each subgrid particle s shares q_s (device real[n_comp][n_s], n_comp <= 64)
 * among the eligible gas j with r_sj < h_s in proportion to V_j W(r_sj, h_s),
 * V_j the gas volume of the last crk_moments, normalised by
 * A_s = 1 / sum_j V_j W(r_sj, h_s).  eligible: optional device uint8[n] in the
 * gas's caller order (0 excludes a gas particle from both the normalisation
 * and the deposit, as the paper does for metal-rich or overweight gas).
 * dq: device real[n_comp][n] in the gas's caller order, ACCUMULATED into
 * (atomic adds; the caller zeroes it); A_out: optional device real[n_s]
 * (0 when no eligible gas is in reach: nothing is deposited).
 * CRK_ESTATE before a crk_moments on this workspace. */
crk_status crk_subgrid_deposit(crk_plan* plan, crk_stream_t stream, void* ws, int64_t n_s,
                               const int64_t* box_off_s, const double* x_s, const void* h_s,
                               int32_t n_comp, const void* q_s, const uint8_t* eligible,
                               void* A_out, void* dq);

/* ---- Radiative cooling and heating (Sec. 2.3.2, Exact Integration) ----------
 * The source function of du/dt = -Lambda(u; rho)/rho is tabulated as
 * lam_k = Lambda(u_k)/rho^2 at n_nodes energies u_k = 10^(log10_u_min +
 * k dlog10_u) (lam > 0 cools, lam < 0 heats; the rho^2 scaling is that of the
 * self-similar power-law test of App. B) and interpolated with a power law in
 * every bin (Eq. L). */
typedef struct {
  int32_t n_nodes;       /* >= 2 */
  int32_t reserved;
  double log10_u_min;    /* log10 of the first node */
  double dlog10_u;       /* node spacing in dex, > 0 (the paper uses 0.004) */
  const double* lambda;  /* device double[n_nodes], owned by the caller */
} crk_cool_table;

/* (i) Exact integration over a step dt >= 0 with rho held fixed (Eqs. intcool,
 * Iu, Iinv): every particle walks the table bins from its own energy (the
 * anchor u_a = u0) and inverts the power-law integral in the bin where rho dt
 * runs out.  A bin whose edge values differ in sign holds the equilibrium: it
 * is crossed at the constant rate max(|lam_k|, |lam_k+1|) and the energy stops
 * at the linearly interpolated zero crossing.  The table ends are a floor and a
 * ceiling; an energy outside [u_min, u_max] is returned unchanged.
 * rho, u0, u1: device real[n] (u1 may alias u0); n <= the plan's n_max.
 * One pass over the particles; no workspace. */
crk_status crk_cool_exact(crk_plan* plan, crk_stream_t stream, int64_t n,
                          const crk_cool_table* table, double dt, const void* rho,
                          const void* u0, void* u1);

/* Autotuner for the launch shapes of the eight neighbor sweeps (volume,
 * moments, density, rates and the four adjoint sweeps).  Each sweep is
 * compiled in CRK_TUNE_VARIANTS variants: three minimum numbers of resident
 * blocks per SM (so three register caps and occupancies; variant % 3), each
 * with the neighbor records read straight from global memory when the pair is
 * evaluated (variants 0-2), copied one list entry ahead through a per-thread
 * shared-memory ring with cp.async, each lane its own record (variants 3-5),
 * loaded one list entry ahead into a register double buffer (variants 6-8),
 * copied into the ring by the whole warp, consecutive lanes taking consecutive
 * 16-byte pieces of one record (variants 9-11 densely, 15-17 in power-of-two
 * lane groups per record), or loaded into rotating register buffers with
 * several entries in flight (variants 12-14: four buffers for the light
 * sweeps, three for the heavy ones).
 * This call runs crk_moments, crk_rates and, when g_dvdt and g_dudt are given,
 * crk_adjoint on the caller's data with each variant `repeats` times, times
 * every sweep with CUDA events and keeps the fastest variant per sweep in the
 * plan.  Outputs of the trial runs go to the workspace; afterwards the
 * workspace holds the state of a complete crk_moments + crk_rates call.
 * choice_out (optional, host int32[8]) receives the chosen variant per sweep,
 * ms_out (optional, host float[8][CRK_TUNE_VARIANTS]) the mean milliseconds of
 * every variant.  Synchronises.  Requires a built workspace. */
#define CRK_TUNE_VARIANTS 18
crk_status crk_autotune(crk_plan* plan, crk_stream_t stream, void* ws, const void* m,
                        const void* v, const void* u, const void* g_dvdt, const void* g_dudt,
                        int32_t repeats, int32_t* choice_out, float* ms_out);

/* Set the launch variant of each of the eight sweeps (host int32[8], in the
 * order of crk_autotune's choice_out, each in [0, CRK_TUNE_VARIANTS)) without
 * timing anything: to replay a stored autotuner choice or to test a variant.
 * Host only; CRK_EINVAL on a value out of range (nothing is changed then). */
crk_status crk_tune_set(crk_plan* plan, const int32_t* choice);

/* Test/inspection: the neighbor sets of the last build as CSR in caller order.
 * mode 0: gather set G(i) without the particle itself; mode 1: union set U(i).
 * row_ptr: device int64[n+1]; col: device int32[cap], sorted within a row.
 * *nnz (host) receives the total; CRK_ENOMEM if it exceeds cap.  Synchronises. */
crk_status crk_neighbors_csr(crk_plan* plan, crk_stream_t stream, void* ws, int32_t mode,
                             int64_t* row_ptr, int32_t* col, int64_t cap, int64_t* nnz);

typedef struct {
  int64_t n, n_boxes;
  int64_t gather_pairs;   /* sum_i |G(i)| - n: ordered pairs j != i with r < h_i */
  int64_t union_pairs;    /* sum_i |U(i)| */
  int64_t list_slots;     /* longest per-particle union list found by the build */
  int64_t list_capacity;  /* list slots reserved per particle (params.nbr_cap) */
  int64_t tree_nodes;
  int64_t launches;       /* kernels this plan has launched since it was created (host count) */
  int64_t tree_tests;     /* tree nodes tested by the last list build (counting pass) */
  int64_t bucket_tests;   /* candidate buckets (8 particles each) tested by that pass */
  int32_t status;         /* device status word (not cleared) */
  int32_t reserved;
} crk_stats;

/* Statistics of the last build.  Synchronises `stream`. */
crk_status crk_stats_get(crk_plan* plan, crk_stream_t stream, void* ws, crk_stats* out);

/* Copy `bytes` from src to dst on `stream` with the SMs (16-byte loads and
 * stores from every SM at once) instead of a copy engine: the staging copy of a
 * step's inputs into device memory and of its results back.  On GB300 a copy
 * engine translates host addresses one page at a time, and right after a step
 * has walked tens of GB of device memory a 1 GiB transfer through it was
 * measured at 21-27 GB/s; this call moved the same bytes at 211 GB/s in and
 * 191 GB/s out.  src and dst: device memory of the current device, managed
 * memory, or host memory allocated page-locked or registered through CUDA
 * (mapped at its own address), each range within one allocation; the ranges
 * must not overlap.  bytes == 0 is a no-op.  CRK_EINVAL for a null pointer,
 * overlapping ranges or memory the device cannot reach (checked on the host
 * before anything is launched, so pageable host memory is refused rather than
 * touched); CRK_ECUDA when a launch fails.  Asynchronous: the caller keeps
 * both buffers alive until the stream has passed the copy. */
crk_status crk_copy(crk_stream_t stream, void* dst, const void* src, size_t bytes);

/* Synchronise `stream`, return the device status word in *device_status and
 * clear it. */
crk_status crk_status_poll(crk_plan* plan, crk_stream_t stream, void* ws,
                           crk_status* device_status);

const char* crk_status_string(crk_status s);

/* Per-kernel timing.  While enabled, every neighbor sweep and build phase the
 * plan launches is bracketed by CUDA events on its stream (up to 256 records,
 * oldest first).  crk_timing_read synchronises on the last event, writes up to
 * `cap` records (name, milliseconds) and clears the list.  Host only apart
 * from the event records; enabling adds two event records per launch. */
typedef struct {
  char name[24];
  float ms;
} crk_kernel_time;
crk_status crk_timing_enable(crk_plan* plan, int32_t enable);
crk_status crk_timing_read(crk_plan* plan, crk_kernel_time* out, int32_t cap, int32_t* count);

/* Measured arithmetic peak of the current device: a grid of 8 blocks of 256
 * threads per SM, each thread running 8 independent chains of fused
 * multiply-adds (2 flops each) in float (fp64 = 0) or double (fp64 = 1), `iters`
 * rounds of 16 per chain.  One warm-up launch, then three timed launches on
 * `stream` (CUDA events); *flops_per_s receives the best rate and *ms
 * (optional, host) that launch's duration.  The pair sweeps are bound by the
 * FP32 pipes: this is the measured counterpart of their derived FP32 peak
 * (SMs x 128 lanes x 2 flops x clock).  Allocates and frees a small device
 * buffer and synchronises `stream`; not capturable.  CRK_EINVAL for iters <= 0
 * or fp64 outside {0, 1}. */
crk_status crk_alu_peak(crk_stream_t stream, int32_t fp64, int32_t iters, double* flops_per_s,
                        double* ms);

/* Gas volume V_i = m_i / sum_j m_j W(|x_ij|, h_i) of one periodic box without a
 * workspace.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory -- for example a subgrid operator
 * called from inside a simulation framework whose device-memory pool owns all
 * allocations, or a host loop that must not call cudaMalloc/cudaFree because
 * they can synchronise the device.  For particles that are all gas (no
 * species) and all inside [0, L) it gives the volume of crk_cell_build
 * followed by crk_moments (V_out), to rounding (the summation order differs),
 * for at most CRK_STATIC_MAX_PARTICLES particles, using a fixed scratch area of
 * about 2.6 MB that is compiled into the library and that every GPU loading
 * the library keeps until exit.
 *   precision: CRK_FP64 (h, m, V_out double) or CRK_MIXED32 (float).
 *   n: particles, 0 <= n <= CRK_STATIC_MAX_PARTICLES, else CRK_ENOMEM.
 *   L: box side; x: device double[3][n] in [0, L); h, m, V_out: device real[n].
 *   h_bound: host upper estimate of max h; it only sets the cell size (at most
 *   32 cells per axis), any positive value gives the same result to rounding.
 * A particle with x outside [0, L) gets V = NaN and enters no other
 * particle's sum; a particle with h outside (0, L/2) gets V = NaN and still
 * enters its neighbors' sums.  The call allocates nothing and is asynchronous
 * on `stream`.  The first call on each device looks up the scratch address
 * (cudaGetSymbolAddress), so make that first call before any stream capture;
 * the address is kept for the life of the process, so a cudaDeviceReset of
 * that device must not come between two calls.  All calls share the scratch,
 * which keeps the last call's contents (each call clears what it needs), so
 * calls whose kernels overlap on the GPU -- on different streams or host
 * threads -- race and must be serialised by the caller. */
#define CRK_STATIC_MAX_PARTICLES 65536
crk_status crk_volume_static(crk_stream_t stream, int32_t precision, int64_t n, double L,
                             double h_bound, const double* x, const void* h, const void* m,
                             void* V_out);

#ifdef __cplusplus
}
#endif
#endif /* CRK_H */
