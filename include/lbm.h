/*
 * lbm.h -- C ABI of the GB300 two-component pseudo-potential lattice
 * Boltzmann step (D3Q19) with the multiscale models of arXiv 2512.21696,
 * "Enhanced numerical models for two-component fluid flow in multiscale
 * porous structures".
 *
 * One time step (lbm_step) does, for every non-solid cell:
 *   - pull streaming of both components with halfway bounce-back at solid
 *     cells (LB equation, Eq. 2);
 *   - moments: component densities rho^A, rho^B and momentum j;
 *   - residual-component update in gray cells (Sec. II, Eq. 5, Fig. 6);
 *   - forces: Shan-Chen inter-component force with psi = rho (Sec. II),
 *     CSF surface-tension control (Eq. 4), the multiscale capillary and
 *     viscous force of Eq. 1 with the tensorial resistivity of Eqs. 6-7,
 *     and a constant body acceleration;
 *   - collision projected on the second-order Hermite basis with the force
 *     term of Eq. 3 (velocity u = (j + F/2)/rho; in gray cells u solves
 *     (rho I + R/2) u = j + F_other/2 with the resistivity tensor R).
 *
 * Conventions
 *   - Grids are nx*ny*nz cells, x fastest: cell (x,y,z) has linear index
 *     x + nx*(y + ny*z).  Per-cell arrays are dense in that order; vector
 *     fields are stored component-major, u[d*ncell + cell].
 *   - Cell types: LBM_CELL_PORE (resolved fluid), LBM_CELL_SOLID,
 *     LBM_CELL_GRAY (under-resolved porous cell with porosity 0 < phi < 1),
 *     LBM_CELL_INLET / LBM_CELL_OUTLET (pressure reservoirs, lbm_set_pressure).
 *   - Every call returns LBM_OK (0) or a negative LBM_ERR_* code and never
 *     throws; lbm_strerror() turns a code into text.  After an error the
 *     context stays valid unless the code is LBM_ERR_CUDA from a sticky CUDA
 *     fault, in which case only lbm_destroy() may follow.
 *   - Ownership: the context owns all device memory it allocates.  Array
 *     arguments are read (or written) during the call only; the caller keeps
 *     ownership.  `mem` says whether an array pointer is host memory
 *     (LBM_MEM_HOST) or device memory of the context's device
 *     (LBM_MEM_DEVICE, e.g. a torch tensor's data_ptr()).
 *   - Streams: all device work is enqueued on lbm_params.stream (NULL = the
 *     legacy default stream).  lbm_step and lbm_set_* calls are asynchronous
 *     with respect to the host except that host-memory inputs are copied
 *     before the call returns.  lbm_observables, lbm_get_fields (host output),
 *     lbm_get_static and lbm_save_state synchronise the stream.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define LBM_API __attribute__((visibility("default")))
#else
#define LBM_API
#endif

#define LBM_ABI_VERSION 1
#define LBM_MAX_PORE_TYPES 16

enum lbm_status {
    LBM_OK = 0,
    LBM_ERR_ARG = -1,      /* invalid argument, size or ordering of calls */
    LBM_ERR_CUDA = -2,     /* a CUDA runtime call failed */
    LBM_ERR_OOM = -3,      /* device or host allocation failed */
    LBM_ERR_NUMERIC = -4,  /* non-finite or negative density detected */
    LBM_ERR_TIMEOUT = -5,  /* a bounded device-side wait gave up */
    LBM_ERR_STATE = -6     /* call out of order (e.g. step before geometry) */
};

enum lbm_mem { LBM_MEM_HOST = 0, LBM_MEM_DEVICE = 1 };

/* Velocity set.  D3Q19 (default) is the method's lattice.  D2Q9 runs the same
 * step on one plane (nz = 1; the paper's two-dimensional experiments of
 * Sec. III) with weights 4/9, 1/9, 1/36: F32 storage only, two launches per
 * step, not in batches or the adjoint (LBM_ERR_ARG there). */
enum lbm_lattice { LBM_LATTICE_D3Q19 = 0, LBM_LATTICE_D2Q9 = 1 };

enum lbm_cell {
    LBM_CELL_PORE = 0,
    LBM_CELL_SOLID = 1,
    LBM_CELL_GRAY = 2,
    LBM_CELL_INLET = 3,  /* reservoir held at the inlet densities */
    LBM_CELL_OUTLET = 4  /* reservoir held at the outlet densities */
};

/* Population storage.  F32: the rest population f_0 and the deviations
 * f_i - 3 w_i f_0 (i >= 1) of each cell, in FP32.  F16S / BF16S: the shifted
 * deviations f_i - w_i rho0 (rho0 = (rho_hi + rho_lo)/2, i = 0..18) in
 * FP16 / BF16, half the bytes per cell.  All storages compute in FP32; the
 * 16-bit storages always run the fused one-launch kernel (lbm_set_kernel's
 * path choice applies to F32) and their checkpoints hold 16-bit slots.
 * F16R / BF16R: the F32 layout's rest population (int32) with the 18
 * deviations f_i - 3 w_i f_0(source) in FP16 (scaled by 2^12) / BF16: the
 * stored numbers are only the velocity and non-equilibrium parts, 80 bytes
 * per cell, fused kernel with the default tile. */
enum lbm_storage {
    LBM_STORAGE_F32 = 0,
    LBM_STORAGE_F16S = 1,
    LBM_STORAGE_BF16S = 2,
    LBM_STORAGE_F16R = 3,
    LBM_STORAGE_BF16R = 4
};

/* Model and run parameters.  Index 0 is component A, 1 is component B. */
typedef struct lbm_params {
    int nx, ny, nz;
    int periodic[3];        /* 1: periodic axis; 0: the outside is solid wall */
    double tau[2];          /* relaxation times; viscosity nu = (tau - 1/2)/3 */
    double G;               /* Shan-Chen coupling: F^a = -G psi^a grad psi^other */
    double kappa_csf;       /* Eq. 4 coefficient (negative lowers sigma) */
    double phi_avg[2];      /* Eq. 4 characteristic average of phi^a */
    double phi_max[2];      /* Eq. 4 characteristic maximum of phi^a */
    int csf_everywhere;     /* 0: Eq. 4 only in gray cells; 1: in all cells */
    double rho_wall[2];     /* virtual densities seen at solid cells (wetting) */
    double body_accel[2][3];/* body acceleration per component; F = rho g */
    int wet_idx;            /* index of the wetting component (water) */
    double rho_hi, rho_lo;  /* bulk majority / minority densities */
    double s_lo, s_hi;      /* residual hysteresis thresholds on s */
    double at_cut;          /* H(At) = |grad At|/2 only where |At| <= at_cut */
    double eps_n;           /* floor of |grad| in unit normals (default 1e-4 rho_hi:
                               keeps Eq. 4's normals well defined in FP32) */
    double kr_min;          /* floor of relative permeabilities */
    double c_g;             /* weight of grad(phi) grad(phi)^T in the axis tensor */
    int storage;            /* enum lbm_storage */
    void *stream;           /* cudaStream_t for all work of this context */
    double probe_center[3]; /* pressure probe for lbm_obs.dp */
    double probe_r_in;      /* inside: distance < probe_r_in */
    double probe_r_out;     /* outside: distance > probe_r_out */
    int lattice;            /* enum lbm_lattice */
} lbm_params;

/* Constitutive curves of one pore type (Appendix: Kozeny-Carman K0,
 * capillary pressure and Corey relative permeabilities; Eq. 5 scaling).
 *   K0(phi)  = kc_d^2 phi^3 / (180 (1 - phi)^2)
 *   Pc(Sw)   = Pe Se^(-1/lambda) (Brooks-Corey, thomeer_g = 0), or
 *              Pe 10^min(-thomeer_g / ln(1 - Se), 1) (Thomeer's hyperbola
 *              log10(Pc/Pe) ln(1 - Se) = -G, the form the Appendix fits,
 *              capped at 10 Pe), with Pe = lamL(phi) pd and
 *              Se = (Sw - swr)/(1 - swr) in [1e-2, 1]
 *   lamL     = sqrt((K0(phi_ref)/phi_ref) / (K0(phi)/phi))        (Leverett)
 *   Kr_w     = Se^nw,  Kr_n = (1 - Se)^nn                          (Se in [0, 1])
 *   residual water Sw_irr = Sw at Pc = pc_ref_max_f * pd; residual oil
 *   So_res = 1 - Sw at Pc = pc_ref_min_f * pd (Fig. 6 crossings)
 *   aniso    = ratio a >= 1 of the principal permeabilities of Eq. 7:
 *              K^D = diag(K0/a, K0, K0) along the principal axis e1. */
typedef struct lbm_constitutive {
    double kc_d, pd, lambda, swr, nw, nn, phi_ref, pc_ref_max_f, pc_ref_min_f, aniso;
    double thomeer_g; /* Thomeer pore-geometrical factor G > 0, or 0 for Brooks-Corey */
} lbm_constitutive;

/* Observables of the current fields: deterministic float-float sums (about
 * 48 bits, counts exact), reported in FP64. */
typedef struct lbm_obs {
    double mass[2];      /* sum of rho^a over non-solid cells */
    double sat;          /* sum(phi_c Sw)/sum(phi_c); phi_c = 1 pore, phi gray */
    double flux_out;     /* mean u_x over the plane x = nx-1 (solid counts 0) */
    double flux_vol[3];  /* mean of u over all cells (solid counts 0) */
    double max_u;        /* max |u| over non-solid cells */
    double dp;           /* mean p inside probe_r_in minus outside probe_r_out,
                            p = (rhoA + rhoB)/3 + G rhoA rhoB */
    long long nan_count; /* non-finite density or velocity values */
    long long step;      /* steps taken since lbm_init_fields */
} lbm_obs;

/* Accumulated device time of one kernel, filled by lbm_profile_read. */
typedef struct lbm_kernel_stat {
    char name[32];
    long long launches;
    double total_ms;
} lbm_kernel_stat;

typedef struct lbm_ctx lbm_ctx;

/* Text of a status code (static storage). */
LBM_API const char *lbm_strerror(int code);

/* Text of the last CUDA runtime error seen by the library in the calling
 * thread ("" if none); valid until the next failing call in that thread. */
LBM_API const char *lbm_last_cuda_error(void);

/* sizeof of the ABI structures, for binding layout checks: which = 0
 * lbm_params, 1 lbm_constitutive, 2 lbm_obs, 3 lbm_kernel_stat; 0 otherwise. */
LBM_API size_t lbm_struct_size(int which);

/* LBM_ABI_VERSION of the loaded library. */
LBM_API int lbm_abi_version(void);

/* Fill p with defaults for an nx*ny*nz periodic grid: tau = 1, G = 0,
 * kappa_csf = 0, rho_hi/lo = 1/0.03, phi_avg = (rho_hi+rho_lo)/2,
 * phi_max = rho_hi, rho_wall = (rho_hi+rho_lo)/2 (neutral wetting),
 * wet_idx = 1, s_lo/s_hi = 0.1/0.9, at_cut = 0.95, eps_n = 1e-4 rho_hi,
 * kr_min = 1e-6, c_g = 1, F32 storage, NULL stream, probe at the grid
 * centre with r_in = 0, r_out = +inf.  LBM_ERR_ARG if p is NULL or a size
 * is < 1. */
LBM_API int lbm_default_params(lbm_params *p, int nx, int ny, int nz);

/* Fill c with the default curves: kc_d = 1, pd = 0.02, lambda = 2,
 * swr = 0.15, nw = 3, nn = 2, phi_ref = 0.35, pc_ref_max_f = 3.5,
 * pc_ref_min_f = 0.575 (midpoints of the ranges in Sec. II), aniso = 1. */
LBM_API int lbm_default_constitutive(lbm_constitutive *c);

/* Create a context on the current CUDA device.  Validates p (sizes >= 1,
 * tau > 1/2, 4 >= rho_hi > rho_lo > 0 ... ; LBM_ERR_ARG otherwise) and allocates
 * the population, density, field and geometry buffers (LBM_ERR_OOM if the
 * device is too small).  *out is NULL on failure.  Every pore type starts
 * with the default curves. */
LBM_API int lbm_create(lbm_ctx **out, const lbm_params *p);

/* Free every device buffer and the handle.  NULL is accepted. */
LBM_API int lbm_destroy(lbm_ctx *ctx);

/* Curves of pore type `pore_type` in [0, LBM_MAX_PORE_TYPES).  Takes effect
 * at the next lbm_set_geometry.  LBM_ERR_ARG on an out-of-range type or
 * invalid curve (pd <= 0, lambda <= 0, swr outside [0,1), aniso < 1, ...). */
LBM_API int lbm_set_constitutive(lbm_ctx *ctx, int pore_type, const lbm_constitutive *c);

/* Geometry: type[ncell] (enum lbm_cell), phi[ncell] porosity of gray cells
 * (values at other cells are ignored and taken as 1, 0 at solid cells),
 * pore_type[ncell]
 * (may be NULL = all type 0).  Runs the FP64 geometry precompute on the
 * device: gradient and Hessian of phi, principal axis of
 * M = H H + c_g grad(phi) grad(phi)^T (Eqs. 6-7 and the abstract), K0,
 * Leverett factor and residual amounts (Eq. 5, Fig. 6) of every gray cell.
 * LBM_ERR_ARG on unknown cell codes or gray phi outside (0,1). */
LBM_API int lbm_set_geometry(lbm_ctx *ctx, const uint8_t *type, const float *phi,
                     const uint8_t *pore_type, int mem);

/* Equilibrium initial state of densities rhoA, rhoB [ncell] and velocity u
 * [3][ncell] (NULL = at rest).  The residual flag of each cell starts wet
 * when its normalised wetting density s >= 1/2, with no residual amount.
 * Requires lbm_set_geometry first (LBM_ERR_STATE). */
LBM_API int lbm_init_fields(lbm_ctx *ctx, const float *rhoA, const float *rhoB, const float *u, int mem);

/* Advance nsteps >= 0 time steps (asynchronous).  The fields read back by
 * lbm_get_fields / lbm_observables are those of the last step.  On lattices
 * of at most 2^18 cells (not batch runs, not while profiling) a call of more
 * than 33 steps replays CUDA graphs of 32 steps, captured on first use per
 * buffer parity and dropped by every call that changes a parameter
 * (lbm_set_constitutive, lbm_set_geometry, lbm_set_pressure, lbm_set_mss,
 * lbm_init_fields, lbm_load_state, lbm_set_kernel, lbm_profile); the
 * replayed kernels are the same launches, so the result is bit-identical and
 * lbm_launch_count counts them.  A failed capture falls back to direct
 * launches for the rest of the context's life; while the caller's stream is
 * being captured (the caller's own graph) the steps are launched directly. */
LBM_API int lbm_step(lbm_ctx *ctx, int nsteps);

/* Pressure boundaries: the densities held in the LBM_CELL_INLET and
 * LBM_CELL_OUTLET cells (the imbibition set-ups of Sec. I and of the
 * Appendix drive the flow by a pressure difference between two boundaries
 * and lower it in steps; the paper does not say how the boundary is
 * imposed).  A reservoir cell holds the given component densities at rest:
 * in every step it takes them as its moments, so that the force stencils of
 * its neighbours see them, carries no force and no velocity, and leaves the
 * collision as their rest equilibrium, which streams into the domain.  Its
 * pressure is p = (rhoA + rhoB)/3 + G rhoA rhoB.
 *   rho_in[2], rho_out[2]: host arrays, densities (A, B) of the inlet and of
 *   the outlet cells, finite, >= 0 with a positive sum; copied.
 * Takes effect from the next step (also for a run of a batch, whose next
 * step re-reads its runs).  Until called both hold (rho_hi, rho_lo).
 * LBM_ERR_ARG on a NULL pointer or invalid densities.  No device work. */
LBM_API int lbm_set_pressure(lbm_ctx *ctx, const double rho_in[2], const double rho_out[2]);

/* Mass-sink-source (the Appendix's relative-permeability runs inject water
 * around the oil-water interface to move between saturation stages; the
 * paper defines it in its refs. [12, 15]).  Reading: in every fluid cell that
 * is not a reservoir, each step's collision moves dm = rate * I from the
 * non-wetting to the wetting component as rest equilibrium (w_i dm per
 * population; cell mass and momentum unchanged), with the interface
 * indicator I = max(0, (4 r_w r_n - I_b) / (1 - I_b)), r = rho^a / rho,
 * I_b = 4 r_lo r_hi its value in either bulk (r_lo = rho_lo/(rho_hi +
 * rho_lo)): zero in the bulks, one in the middle of an interface.
 * rate (lattice density per step; negative drains water) takes effect from
 * the next step; 0 switches the term off (and the plain march runs again).
 * Works on a run of a batch.  LBM_ERR_ARG for a non-finite rate.  No device
 * work. */
LBM_API int lbm_set_mss(lbm_ctx *ctx, double rate);

/* Saturation controller around the mass-sink-source: every check_every
 * steps the rate is set to clamp(gain (target - S), -max_rate, max_rate)
 * (0 within tol), S = lbm_obs.sat, until S is within tol of the target at a
 * check or max_steps steps ran; the rate is 0 on return.  *steps_done
 * receives the steps taken.  LBM_OK when the target was reached,
 * LBM_ERR_TIMEOUT otherwise, LBM_ERR_ARG on invalid arguments (target in
 * [0, 1], gain > 0, max_rate > 0, tol > 0, check_every >= 1, max_steps >= 1).
 * Synchronous. */
LBM_API int lbm_mss_to_saturation(lbm_ctx *ctx, double target, double gain, double max_rate, double tol,
                                  int check_every, int max_steps, int *steps_done);

/* Stepped-pressure protocol of the imbibition set-ups (Sec. I: the pressure
 * difference between the two boundaries is lowered level by level and a
 * steady state is recorded at each level; the Appendix evaluates Pc(Sw) the
 * same way).  For level k = 0 .. nlevels-1: hold rho_in[2k..2k+1] and
 * rho_out[2k..2k+1] (as lbm_set_pressure), then step check_every steps at a
 * time until the saturation (lbm_obs.sat, which leaves the reservoirs out)
 * changed by at most sat_tol over the last check, or max_steps steps ran.
 * sat[k] receives the saturation at the end of the level and steps[k] the
 * steps it took.  The capillary pressure of a level is the reservoirs'
 * pressure difference, p = (rhoA + rhoB)/3 + G rhoA rhoB at each end.
 *   nlevels >= 1, check_every >= 1, sat_tol >= 0, max_steps >= 1; host arrays.
 * Returns LBM_OK when every level became steady, LBM_ERR_TIMEOUT when some
 * level ran out of steps (outputs still filled), LBM_ERR_STATE without
 * reservoir cells or fields, LBM_ERR_ARG on invalid arguments (checked
 * before the first step).  Synchronous. */
LBM_API int lbm_pressure_levels(lbm_ctx *ctx, int nlevels, const double *rho_in, const double *rho_out,
                                int check_every, double sat_tol, int max_steps, double *sat, int *steps);

/* Reductions of the current fields into *out (synchronises).
 * Returns LBM_ERR_NUMERIC when nan_count > 0 (out is still filled). */
LBM_API int lbm_observables(lbm_ctx *ctx, lbm_obs *out);

/* Asynchronous observables for monitoring loops: enqueues the reductions of
 * the current fields and the copy of their raw sums into raw[0..15] on the
 * context's stream and returns; raw[16] receives the step count at once.
 * raw: LBM_OBS_RAW doubles of host memory (pinned, so that the copy does not
 * wait) that stays valid until the stream has passed the copy; several calls
 * may be in flight, each with its own raw.  lbm_obs_decode turns raw into
 * lbm_obs (host arithmetic only) after the stream passed the copy, and
 * returns LBM_ERR_NUMERIC when nan_count > 0 as lbm_observables does. */
#define LBM_OBS_RAW 17
LBM_API int lbm_observables_async(lbm_ctx *ctx, double *raw);
LBM_API int lbm_obs_decode(lbm_ctx *ctx, const double *raw, lbm_obs *out);

/* Current fields: rhoA, rhoB [ncell], u [3][ncell], sw [ncell] (effective
 * water saturation incl. residual amounts); any pointer may be NULL.  Solid
 * cells read 0. */
LBM_API int lbm_get_fields(lbm_ctx *ctx, float *rhoA, float *rhoB, float *u, float *sw, int mem);

/* Geometry results of gray cells (zero elsewhere): kinv [6][ncell] = K^-1
 * entries xx, yy, zz, xy, xz, yz (Eq. 7 inverse permeability, 1/length^2);
 * pc_scale [ncell] = lamL(phi) pd; sw_irr, so_res [ncell]. */
LBM_API int lbm_get_static(lbm_ctx *ctx, float *kinv, float *pc_scale, float *sw_irr,
                   float *so_res, int mem);

/* Checkpoint of the populations, residual state and step counter. */
LBM_API int lbm_state_size(lbm_ctx *ctx, size_t *bytes);
LBM_API int lbm_save_state(lbm_ctx *ctx, void *host_buf, size_t bytes);
LBM_API int lbm_load_state(lbm_ctx *ctx, const void *host_buf, size_t bytes);

/* Per-kernel CUDA-event timing of every launch while enabled (adds two
 * event records per launch).  lbm_profile(ctx, 1) clears the counters.
 * lbm_profile_read synchronises and writes up to max entries. */
LBM_API int lbm_profile(lbm_ctx *ctx, int enable);
LBM_API int lbm_profile_read(lbm_ctx *ctx, lbm_kernel_stat *out, int max, int *count);

/* Kernel path of lbm_step: path 0 (default) = one fused launch per step
 * (rolling z-window with shared-memory halos), path 1 = two launches
 * (densities, then forces + collision).  tile selects the fused tile:
 * 0 = 32x8 columns, 1 = 32x16, 2 = 32x8 with two CTAs per SM, 3 = 32x12,
 * 4 = 64x8, 7 = 64x7, 8 = chosen per grid among 2, 4 and 7 (the one whose
 * z-chunked columns best fill the resident CTA slots; 4 and 7 only where nx
 * is a multiple of 64; the shifted 16-bit storages run 2 or 7, the
 * rest-referenced ones 2, 4 or 7, other tiles there running 2), 5 and 6 = the
 * published-density march on 32x8 and 32x7 tiles
 * (every CTA resident, one cooperative launch per step: each tile publishes
 * its densities and reads its ring from its neighbours instead of
 * recomputing it; no CUDA-graph replay).  The march runs the plain F32 step;
 * with reservoir cells, a mass-sink-source rate, a 16-bit storage or more
 * tile columns than resident CTAs, tiles 5 and 6 run tile 2.  Default: 8.
 * Both paths and all tiles compute
 * identical states.  A march whose bounded wait for a neighbouring tile gave
 * up (1 s) makes the next lbm_observables or lbm_get_fields return
 * LBM_ERR_TIMEOUT.  LBM_ERR_ARG on unknown values. */
LBM_API int lbm_set_kernel(lbm_ctx *ctx, int path, int tile);

/* The kernel path and the fused tile a step of ctx runs (*path, *tile: host
 * ints): tile 8 resolved to the shape chosen for this grid (2, 4 or 7), a
 * shape the storage does not have reported as the 2 it runs; on path 1 the
 * requested tile.  Tiles 5 and 6 are reported as requested (whether the march
 * applies is decided per launch).  Resolves the launch configurations on the
 * device on first use; no device work.  LBM_ERR_ARG on NULL pointers. */
LBM_API int lbm_get_kernel(lbm_ctx *ctx, int *path, int *tile);

/* Testing hook for the error path of lbm_step (no counterpart in the paper):
 * the next count step launches are issued with a zero-size thread block, a
 * configuration the CUDA runtime rejects on the host before any device work.
 * lbm_step then returns LBM_ERR_CUDA and the context keeps the state of the
 * last step that ran (buffer parity, step count, fields).  count = 0 cancels.
 * LBM_ERR_ARG on a NULL context or a negative count.  No device work. */
LBM_API int lbm_inject_launch_failures(lbm_ctx *ctx, int count);

/* ---- Porosity gradient (discrete adjoint) ---------------------------------
 * Loss on the fields of the last step (outlet flux and saturation mismatch):
 *   L = (q - q_target)^2 / q_target^2 + (S - s_target)^2,
 *   q = mean of u_x over the plane x = nx - 1 (solid cells count 0),
 *   S = sum(phi_c Sw) / sum(phi_c) over non-solid cells (phi_c = 1 in pores). */
typedef struct lbm_loss {
    double q_target;  /* nonzero */
    double s_target;
} lbm_loss;

/* Runs nsteps forward steps from the current state (F32 storage, not a batch
 * run), evaluates L, and computes dL/dphi for every cell (0 outside gray
 * cells) with the hand-written adjoint of the step: the forward keeps a
 * checkpoint every ckpt steps; the backward recomputes each segment from its
 * checkpoint and runs the adjoint step backwards through it, then chains the
 * gray-cell constants to phi through the geometry precompute (Kozeny-Carman
 * K0, Leverett factor, residual crossings of Eq. 5 / Fig. 6, the principal
 * axis of Eqs. 6-7 via d e1 = sum_{k != 1} e_k (e_k^T dM e1)/(mu1 - mu_k)).
 * Piecewise-constant parts (residual hysteresis, the H(At) cut-off, clamps)
 * contribute their active branch.  dL_dphi: n floats, host or device (mem).
 * out3 (may be NULL): L, q, S.  Ends at the forward's final state (as
 * lbm_step(nsteps) would).  Device memory: (nsteps/ckpt + ckpt + 5)
 * population buffers.  Synchronous.  LBM_ERR_ARG for a geometry with
 * pressure (inlet / outlet) cells, which the adjoint step does not model.  The paper does not differentiate its
 * model; this is the calibration use of it. */
LBM_API int lbm_adjoint_run(lbm_ctx *ctx, const lbm_loss *L, int nsteps, int ckpt, float *dL_dphi, int mem,
                            double *out3);

/* ---- Batches of lattices (REV library runs, workflow step ii) -----------
 * A batch advances many independent lattices of uneven size together: one
 * persistent launch per step (and tile shape in use) takes (run, column,
 * z-chunk) items from a device work counter, k steps are captured once into
 * a CUDA graph and replayed.  The paper runs its REV library one simulation
 * at a time; batching is this library's own scheduling and changes no
 * arithmetic (a run advanced in a batch equals the run advanced alone).
 *
 * lbm_batch_create: runs[nruns] give each lattice's shape, body acceleration
 *   and probe; all other fields must be equal (LBM_ERR_ARG otherwise), and
 *   storage must be F32, F16R or BF16R.  Device buffers are owned by the
 *   batch.  The runs also share run 0's constitutive curves: set the same
 *   curves on every run (lbm_batch_step and lbm_batch_tune return
 *   LBM_ERR_STATE while they differ); reservoir densities and
 *   mass-sink-source rates are per run.
 * lbm_batch_run: the context of one run, a view of the batch's buffers: use
 *   it with lbm_set_constitutive, lbm_set_geometry, lbm_init_fields,
 *   lbm_observables, lbm_get_fields, lbm_get_static and checkpoints (and
 *   lbm_step to advance that run alone).  lbm_destroy refuses it; it lives
 *   until lbm_batch_destroy.
 * lbm_batch_step: nsteps steps of every run (LBM_ERR_STATE unless every run
 *   has fields at the same step parity).  Asynchronous; the first call with a
 *   given nsteps and parity captures the graph.
 * lbm_batch_tune: for the runs of each x extent, times trial_steps steps
 *   (rounded up to even) of every tile shape (0 = 32x8, 1 = 16x16,
 *   2 = 32x16) and keeps the fastest; the state is restored afterwards.
 *   tiles_out (nruns entries, may be NULL) receives the choice per run.
 *   Synchronous.
 * lbm_batch_observables: lbm_observables of every run into out[nruns]
 *   (synchronous); LBM_ERR_NUMERIC if any run has non-finite fields, with
 *   every entry filled.
 * lbm_batch_step_to_steady: steps the batch check_every steps at a time
 *   until, for every run, the mean velocity changed by at most rel_tol of its
 *   largest component over the last chunk (steady flow: the permeability
 *   K = <u> nu / g is then read at steady state), or until max_steps; returns
 *   LBM_OK when steady, LBM_ERR_TIMEOUT when max_steps ran out; steps_done
 *   (may be NULL) receives the steps taken.  Runs whose fields turned
 *   non-finite are left out of the test.  Synchronous.
 * lbm_batch_info: total cells, steps taken, kernels launched by
 *   lbm_batch_step, and the number of launches per step. */
typedef struct lbm_batch lbm_batch;
LBM_API int lbm_batch_create(lbm_batch **out, int nruns, const lbm_params *runs);
LBM_API int lbm_batch_destroy(lbm_batch *b);
LBM_API int lbm_batch_run(lbm_batch *b, int run, lbm_ctx **view);
LBM_API int lbm_batch_step(lbm_batch *b, int nsteps);
LBM_API int lbm_batch_tune(lbm_batch *b, int trial_steps, int *tiles_out);
LBM_API int lbm_batch_info(lbm_batch *b, long long *cells, long long *steps, long long *launches, int *ngroups);
LBM_API int lbm_batch_observables(lbm_batch *b, lbm_obs *out);
LBM_API int lbm_batch_step_to_steady(lbm_batch *b, int check_every, double rel_tol, int max_steps, int *steps_done);

/* lbm_mss_to_saturation for every run of a batch at once, targets[nruns]
 * (host array): each run has its own rate; the batch steps until every run
 * is within tol of its target at a check (LBM_OK) or max_steps ran
 * (LBM_ERR_TIMEOUT).  Runs whose fields turned non-finite are left out (rate
 * 0; lbm_batch_observables reports them).  All rates are 0 on return.
 * Synchronous. */
LBM_API int lbm_batch_mss_to_saturation(lbm_batch *b, const double *targets, double gain, double max_rate,
                                        double tol, int check_every, int max_steps, int *steps_done);

/* Number of kernels the context has launched since creation. */
LBM_API int lbm_launch_count(lbm_ctx *ctx, long long *count);

/* Observables of caller-provided fields, without allocating.  The paper has
 * no counterpart: this is a service for callers that cannot call cudaMalloc
 * (host callbacks and allocator hooks, plug-ins whose host application owns
 * the device memory pool, loops that must not risk an allocation's implicit
 * synchronisation).  It computes what lbm_observables computes, from
 *   fields    device [6][ncell] float: rhoA, rhoB, ux, uy, uz, Sw (the layout
 *             lbm_get_fields writes when given one buffer's consecutive rows),
 *   type      device [ncell] cell codes, phi device [ncell] porosity,
 *   probe     host {cx, cy, cz, r_in, r_out} of the pressure probe, G the
 *             Shan-Chen coupling of the pressure p = (rhoA+rhoB)/3 + G rhoA rhoB,
 * on `stream` (cudaStream_t, NULL = legacy default), and writes *out (host;
 * out->step is 0).  Synchronises the stream.
 * Scratch: a file-scope device array of 58,496 bytes that every GPU loading
 * this library holds until exit.  Every call resolves that array's address
 * in the context current to the calling thread (cudaGetSymbolAddress: the
 * device's primary context, a context the caller made current, a primary
 * context re-created after cudaDeviceReset).  All calls share the array:
 * calls that overlap on the GPU race.  Nothing is
 * allocated, freed, or needs clearing between calls.  The call synchronises
 * its stream and so cannot be captured into a CUDA graph.
 * Errors: LBM_ERR_ARG for NULL pointers, sizes < 1 or more than
 * LBM_NOALLOC_MAX_CELLS cells, or a stream that is being captured (checked
 * before any work); LBM_ERR_CUDA; LBM_ERR_NUMERIC when non-finite values were
 * found (out is still filled). */
#define LBM_NOALLOC_MAX_CELLS (1LL << 28)
LBM_API int lbm_observables_noalloc(const float *fields, const uint8_t *type, const float *phi, int nx, int ny,
                                    int nz, double G, const double probe[5], void *stream, lbm_obs *out);

#ifdef __cplusplus
}
#endif
#endif
