/*
 * sp.h -- C ABI of libsp, a GB300 (sm_103a) implementation of the per-time-
 * step particle pipeline of the hybrid stochastic-particle Shakhov / DSMC
 * method of Jin, Liu, Yang, Cao, Zhuo, Zhong, arXiv:2506.23917.
 *
 * One call of sp_step() advances every flow instance of a context by one
 * global time step, following Sec. III.B of the paper:
 *   Step 3  index particles into cells and form the per-cell moments
 *           n, U, T, Q with the unbiased estimators of Step 3;
 *   Step 4  local observation time dt_c (Eq. "local time step"), relaxation
 *           time tau = mu/p, the split of the step into a DSMC part and a
 *           Shakhov part (Eqs. "tDSMC", "tShakhov"), the NTC/VHS collisions
 *           of Sec. II.A, the Shakhov resampling of Sec. II.B (Eqs.
 *           "Ncol_SBGK", "Maxwell", "A_cal") and the conservation rescale;
 *   Step 5  time-averaged sums after N_steady;
 *   Step 2  free flight (Eq. "free transport") with specular / diffuse
 *           walls, a diffuse circle (2-D) or sphere (3-D) body, removal at
 *           open faces, and injection from ghost-cell reservoirs at inflow
 *           faces; the global step of the next interval is
 *           Delta t_G = cfl * min_k dt_c,k (Eq. "global time step").
 * The state between calls is "indexed and sorted by cell, not yet
 * collided".  All random numbers come from Philox4x32-10 streams keyed by
 * (seed) and counted by (step, cell or reservoir cell, slot, purpose), so
 * the FP64 mode reproduces the CPU oracle particle for particle.
 *
 * Conventions
 *  - Every function returns an sp_status; no exception crosses the ABI.
 *  - All pointers in this header are HOST pointers unless stated otherwise.
 *    Caller buffers are read or written before the call returns (the call
 *    synchronises the context's stream when it copies data to the host).
 *  - The library owns all device memory of a context; it allocates it in
 *    sp_init() and frees it in sp_free().
 *  - Device work is enqueued on the CUDA stream given to sp_init() (NULL
 *    selects the legacy default stream of the current device).
 *  - A device-side failure (particle capacity overflow, a bounce or
 *    acceptance-rejection cap) sets a sticky flag that
 *    the next synchronising call reports as SP_ERR_DEVICE or
 *    SP_ERR_CAPACITY; sp_errors() reads the individual counters.
 */
#ifndef SP_H
#define SP_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SP_OK = 0,
  SP_ERR_ARG = -1,      /* invalid argument or configuration              */
  SP_ERR_CUDA = -2,     /* a CUDA runtime call failed                      */
  SP_ERR_CAPACITY = -3, /* particle capacity (or a static-sort limit) exceeded */
  SP_ERR_DEVICE = -4,   /* sticky device error flag set                    */
  SP_ERR_STATE = -5     /* call out of order (e.g. sp_step before particles) */
} sp_status;

/* Precision modes (sp_init):
 *   SP_FP64         particle state and all arithmetic in FP64 (matches the
 *                   CPU oracle particle for particle);
 *   SP_FP32         particle state and per-particle arithmetic (free flight,
 *                   pair collisions, Maxwellian sampling) in FP32; per-cell
 *                   sums accumulated in FP64, and the per-cell arithmetic
 *                   (U, T, q, tau, dt_c, the split, N_col, exp(-dt/tau), the
 *                   conservation rescale) and the time averages in FP64;
 *   SP_FP32_CELL32  opt-in variant of SP_FP32 whose per-cell sums and
 *                   per-cell arithmetic are FP32 too (only the exp(-dt/tau)
 *                   weight, the rescale factor and the time averages stay
 *                   FP64).  Faster; checked statistically like SP_FP32. */
typedef enum { SP_FP64 = 0, SP_FP32 = 1, SP_FP32_CELL32 = 2 } sp_precision;
typedef enum { SP_BC_SPECULAR = 0, SP_BC_DIFFUSE = 1, SP_BC_OUTFLOW = 2, SP_BC_INFLOW = 3 } sp_bc;
typedef enum { SP_BODY_NONE = 0, SP_BODY_CIRCLE = 1, SP_BODY_SPHERE = 2 } sp_body;
typedef enum { SP_MODE_HYBRID = 0, SP_MODE_DSMC = 1, SP_MODE_SHAKHOV = 2 } sp_mode;

/* One flow instance on a uniform Cartesian grid.  Units are any consistent
 * set (SI or nondimensional).  Faces are numbered 2*axis + side, side 0 is
 * the lower face. */
typedef struct sp_config {
  int32_t dim;            /* spatial dimensions 1..3 (velocities are 3-D)    */
  int32_t n[3];           /* cells per axis; unused axes are forced to 1     */
  double lo[3], hi[3];    /* domain box; unused axes give the unit depth     */
  double m;               /* molecular mass                                  */
  double R;               /* specific gas constant k/m                       */
  double gamma;           /* ratio of specific heats (local time step)       */
  double Pr;              /* Prandtl number of the Shakhov target g^S        */
  double omega;           /* VHS exponent: mu = mu_ref (T/T_ref)^omega       */
  double T_ref, mu_ref;   /* VHS reference temperature and viscosity         */
  double d_ref;           /* VHS reference diameter (cross-section)          */
  double Fn;              /* real molecules per simulated particle           */
  double cfl;             /* Delta t_G = cfl * min_k dt_c,k                  */
  double dt_fixed;        /* > 0: constant Delta t_G                         */
  int32_t face_bc[6];     /* sp_bc per face                                  */
  double face_T[6];       /* wall temperature (diffuse) / reservoir T (inflow) */
  double face_n[6];       /* reservoir number density (inflow)               */
  double face_u[6][3];    /* reservoir drift velocity (inflow)               */
  int32_t ghost_layers;   /* reservoir cell layers outside each inflow face  */
  int32_t body;           /* sp_body; diffuse at body_Tw                     */
  double body_c[3], body_r, body_Tw;
  const double* cell_volume; /* host [ncells] fluid volume per cell, or NULL
                                (uniform); read during sp_init only        */
  double sigc_T0;         /* (sigma_T c_r)_max starts at 2 sigma_T(cbar) cbar,
                             cbar = 4 sqrt(R sigc_T0 / pi)                   */
  int32_t n_steady;       /* first step index that is time-averaged          */
  uint64_t seed;          /* Philox key of this instance                     */
  int32_t mode;           /* sp_mode: hybrid, or one sub-step forced         */
  int32_t ar_max;         /* cap on Shakhov acceptance-rejection attempts    */
  int32_t n_surf;         /* surface elements of the body for wall tallies
                             (0: none); see sp_get_surface()                 */
  /* Open window of each outflow / inflow face (an orifice): on the face's
   * tangential axes (the other axes below dim, in increasing order) the face
   * is open where win_lo <= x <= win_hi; an axis with win_lo >= win_hi is
   * unrestricted (all zeros: the whole face is open).  The rest of the face
   * is a diffuse wall at face_T, and the reservoir of a windowed inflow face
   * spans the window plus ghost_layers cells on each side. */
  double win_lo[6][2], win_hi[6][2];
  /* Fractional part of the NTC candidate count (Sec. II.A leaves it open):
   * 0 = stochastic rounding with one uniform per cell and step (default);
   * 1 = Bird's carried remainder, kept per cell from 0 and added to the
   * next step's count (deterministic; no draw). */
  int32_t ntc_carry;
  /* Bird's sub-cells (Sec. II.A selects a candidate pair anywhere in the
   * cell; this is the usual DSMC refinement, off by default): 0 or 1 = off;
   * s >= 2 splits every cell into s equal parts per axis (s^dim sub-cells,
   * at most 8).  A cell's particles are then ordered by sub-cell (stable)
   * before its step, the first particle of a candidate pair is uniform over
   * the cell and its partner uniform over the other particles of the first
   * one's sub-cell (over the cell when it is alone there). */
  int32_t subcells;
  /* Body-fitted O-grid about a circular body (2-D; the paper's cylinder
   * meshes are body-fitted, Sec. IV.B).  0 = the uniform Cartesian grid
   * above.  1 = n[0] radial layers x n[1] angular sectors (n[1] >= 3) of
   * straight-edged quadrilaterals between the body polygon (nodes on the
   * circle body_r about body_c; a diffuse wall at body_Tw) and the outer
   * polygon (radius mesh_r_out): node radii r_0 = body_r,
   * r_{i+1} = r_i + dr_i with dr_{i+1} = mesh_growth * dr_i and the first
   * n[0] spacings summing to mesh_r_out - body_r; node angles 2 pi j / n[1];
   * cell k = i + n[0] j.  The outer polygon is face 1: face_bc[1] (inflow =
   * a freestream reservoir of ghost_layers rings continuing the radial
   * spacing, at face_n/T/u[1]; outflow; specular; diffuse at face_T[1]).
   * Particles find their cell by face crossing; the local observation time
   * uses each cell's shortest edge; lo/hi[0..1] must be a non-empty box but
   * are not used (the bounding box of the outer polygon is customary), and
   * hi[2] - lo[2] is the depth.  Requires body = SP_BODY_CIRCLE,
   * subcells <= 1; SP_ERR_ARG otherwise. */
  int32_t mesh;
  double mesh_r_out, mesh_growth;
} sp_config;

typedef struct sp_ctx sp_ctx;

/* Moment fields, laid out [field][cell] in sp_moments() output. */
enum {
  SP_F_N = 0, SP_F_n, SP_F_ux, SP_F_uy, SP_F_uz, SP_F_T, SP_F_qx, SP_F_qy, SP_F_qz,
  SP_F_tau, SP_F_dtc, SP_F_ratio, SP_NFIELDS
};

/* Create a context holding n_instances independent flows (cfgs[0..n)), all
 * with the same dim, stored and advanced in one set of kernels.  This is the
 * set-up part of Step 1 of Sec. III.B (the input data: grid, gas, boundary
 * conditions); the particles of Step 1 come with sp_set_particles().
 * precision: an sp_precision mode (SP_FP64, SP_FP32, SP_FP32_CELL32).
 * capacity: device particle slots over all instances (<= 2^31).
 * stream: a cudaStream_t or NULL.  Errors: SP_ERR_ARG for an invalid
 * config, SP_ERR_CUDA if device memory cannot be had. */
sp_status sp_init(const sp_config* cfgs, int n_instances, int precision, int64_t capacity,
                  void* stream, sp_ctx** out);

/* Step 1 of the paper: give instance `inst` its particles.  pos is
 * [dim][n] (SoA, row d holds coordinate d), vel is [3][n]; both host FP64.
 * The data is copied to a device staging area on the context's stream
 * (asynchronously when the host memory is page-locked: keep it unchanged
 * until the next synchronising call).  At the next sp_step / query every
 * instance's staged particles are converted to the context's precision,
 * indexed and stably sorted by cell (input order within a cell), and
 * Delta t of the next step is set to cfl * min dt_c of that state (on an
 * O-grid, particles outside the mesh -- inside the body polygon or beyond
 * the outer polygon -- are dropped).  Calling
 * it again restarts every instance from its staged particles; sampling sums
 * and the step counter are kept.  Errors: SP_ERR_CAPACITY if n exceeds the
 * capacity. */
sp_status sp_set_particles(sp_ctx* ctx, int inst, const double* pos, const double* vel, int64_t n);
/* sp_set_particles with host FP32 arrays (same layout and behaviour): half
 * the host-to-device bytes for FP32 contexts, whose state is FP32 anyway.
 * In an FP64 context the values are widened exactly. */
sp_status sp_set_particles_f32(sp_ctx* ctx, int inst, const float* pos, const float* vel, int64_t n);

/* Advance all instances by n_steps global steps (asynchronous): each step
 * is Steps 2-5 of Sec. III.B -- per cell the Step 3 moments, the Step 4
 * collision split into the DSMC part (Sec. II.A) and the Shakhov part
 * (Sec. II.B) with the rescale, the Step 5 sampling, then the free flight
 * of Step 2 and the indexing of Step 3 for the next step -- launched as one
 * CUDA graph per step. */
sp_status sp_step(sp_ctx* ctx, int n_steps);

/* kind 0: moments of the current state (fields SP_F_*); kind 1: time-
 * averaged fields of Step 6 (N, n, ux, uy, uz, T and the mean DSMC ratio in
 * SP_F_ratio; the other fields are 0).  out: host [n_fields][ncells(inst)].
 * In reproducible runs (FP64, or sp_set_reproducible on) kind 0 sums each
 * cell in source order, so the fields are bit-identical from run to run;
 * it puts the cells' particles in that order on the device first, which is
 * the order the next step would restore anyway (no later result changes).
 * With an FP32 state, kind 0 forms the per-cell quotients as products of
 * reciprocals (a few ulps from the FP64 mode's quotients).  When out is
 * page-locked host memory mapped for the device (cudaHostAlloc,
 * cudaHostRegister) and n_fields = SP_NFIELDS, the kernel writes the
 * fields into it directly; otherwise they are copied from a device buffer.
 * The call returns when out holds the fields. */
sp_status sp_moments(sp_ctx* ctx, int inst, int kind, double* out, int n_fields);

/* Current particles of instance inst in sorted order (host FP64, SoA).
 * Any pointer may be NULL.  *n receives the count; with pos == vel == cell
 * == NULL only the count is returned. */
sp_status sp_get_particles(sp_ctx* ctx, int inst, double* pos, double* vel, uint32_t* cell,
                           int64_t* n);

/* Record of the last step of instance inst, for parity checks: cell4 host
 * int64 [4][ncells] = (candidates, accepted, resampled, AR attempts) per cell
 * of the collided state; resampled host uint8 [n_old] per particle of that
 * state; perm host uint32 [n] = source index (in the moved sequence, injected
 * particles appended) of each slot of the new state.  Recording must be
 * enabled with sp_set_record(ctx, 1) before the step. */
sp_status sp_set_record(sp_ctx* ctx, int on);
sp_status sp_get_step_record(sp_ctx* ctx, int inst, int64_t* cell4, uint8_t* resampled,
                             uint32_t* perm, int64_t* n_old);

/* Conservation record of the last step of instance inst (record mode, FP64
 * and FP32 modes): out host double [6][ncells].  For every cell whose
 * velocities were rescaled (Sec. II.B: after a Shakhov resampling all
 * velocities of the cell are mapped to c' = U + (c - U_p) sqrt(T / T_p)),
 * with U, T the cell's Step 3 moments and the sums taken in FP64 over the
 * rescaled velocities before they are stored in the state's precision:
 * [0..2] sum c'_d - N U_d, [3] sum |c' - U|^2 - 3 R (N-1) T,
 * [4] 3 R (N-1) T (> 0; the energy scale), [5] N sqrt(|U|^2 + 3 R T) (the
 * momentum scale).  Cells without a rescale hold zeros.  SP_ERR_STATE
 * unless recording was on during the step (sp_set_record). */
sp_status sp_get_conservation(sp_ctx* ctx, int inst, double* out);
/* Cell offsets of the current state of instance inst: host uint32
 * [ncells+1], relative to the instance's first particle. */
sp_status sp_get_cell_start(sp_ctx* ctx, int inst, uint32_t* start);
/* Per-cell (sigma_T c_r)_max of instance inst: host double [ncells]. */
sp_status sp_get_sigc_max(sp_ctx* ctx, int inst, double* out);
/* Delta t of the next step of instance inst, and the global step index. */
sp_status sp_get_dt(sp_ctx* ctx, int inst, double* dt, int64_t* step);
/* Surface tallies of instance inst's body, summed over the sampled steps
 * (step index >= n_steady): out host [7][n_surf] = (hits, momentum given to
 * the wall x, y, z, energy given to the wall, momentum given along the
 * inward normal, momentum given along e_theta), each hit weighted by F_N m;
 * *time = sampled physical time.  Element b of a circle covers the polar
 * angle theta = atan2(n_y, n_x) in [-pi + 2 pi b/n_surf,
 * -pi + 2 pi (b+1)/n_surf); of a sphere, theta = acos(n_x) in
 * [pi b/n_surf, pi (b+1)/n_surf).  e_theta is the unit direction of
 * increasing theta at the hit point (zero on a sphere's axis).  Divided by
 * element area and time these are the wall stress and heat flux behind the
 * paper's surface pressure, shear, heat flux and force coefficients
 * (Sec. IV.B-E); sp_surface_coefficients() forms them. */
sp_status sp_get_surface(sp_ctx* ctx, int inst, double* out, double* time);
/* Surface and body coefficients from wall tallies (host arithmetic only; no
 * context or GPU needed).  cfg: the instance's configuration (its body,
 * n_surf and domain box); tallies: host [7][n_surf] as returned by
 * sp_get_surface; time: the sampled time; rho_inf, u_inf, p_inf: free-stream
 * density, speed (along +x) and pressure, with q_inf = rho_inf u_inf^2 / 2.
 * elem (host [4][n_surf], caller-owned): A_b = area of element b inside the
 * domain box (2-D: arc length times the z extent), found by sub-sampling
 * the element; Cp = (p_b - p_inf)/q_inf with p_b the normal momentum flux
 * into the wall; Cf = tau_b/q_inf with tau_b the momentum flux along
 * e_theta; Ch = (energy flux into the wall)/(q_inf u_inf).  Elements with
 * no area inside the box get zeros.  body (host [4]): Cd = F_x/(q_inf A_ref),
 * CL = F_y/(q_inf A_ref), Ch over the whole in-domain surface, and
 * A_ref = half the integral of |n_x| over the in-domain surface (the frontal
 * area of that part of a convex body).  SP_ERR_ARG for a missing body,
 * n_surf < 1, time <= 0 or q_inf <= 0. */
sp_status sp_surface_coefficients(const sp_config* cfg, const double* tallies, double time,
                                  double rho_inf, double u_inf, double p_inf, double* elem,
                                  double* body);
/* Device error counters: [0] capacity overflow, [1] reserved (always 0:
 * cells of any occupancy are processed, those above 1024 particles by one
 * thread block each), [2] bounce cap, [3] AR cap, [4] NTC candidate cap.
 * Clears nothing. */
sp_status sp_errors(sp_ctx* ctx, int64_t* out5);
/* Advance n_steps steps, each as the step graph of sp_step with CUDA event
 * nodes at the boundaries of its kernel groups; ms[0..min(n_slots,4))
 * receives the summed device time of (0) the batch plan and the collision +
 * free-flight kernels, (1) what of the reservoir injection (a branch beside
 * them) is left when they end, (2) the histogram scan and bookkeeping,
 * (3) the scatter.  Synchronises after every step (for measurement only). */
sp_status sp_step_profiled(sp_ctx* ctx, int n_steps, double* ms, int n_slots);
/* Within-cell order of the particles.  on = 1 (default): every step restores
 * the source order inside each cell (a stable counting sort overall), so a
 * run is bit-reproducible and FP64 mode matches the CPU oracle particle for
 * particle.  on = 0 (FP32 mode only; SP_ERR_ARG in FP64 mode): cells keep
 * the order in which the scatter's atomics placed them; every draw is still
 * an independent uniform per slot and pair selection is still uniform, so
 * results are statistically the same but differ bit-wise from run to run. */
sp_status sp_set_reproducible(sp_ctx* ctx, int on);
/* Collision-kernel schedule: `cap` particles of shared-memory staging per
 * warp (a warp takes consecutive cells whose particles fit; cells above it
 * go to a one-warp-per-cell launch) and `warps` warps per block (1..8).
 * The schedule changes no result.  SP_ERR_ARG if it does not fit. */
sp_status sp_set_schedule(sp_ctx* ctx, int cap, int warps);
/* Autotuner: for each candidate schedule (warps in 2, 4, 8; cap in 128,
 * 256, 384, 512, 768, 1024 and, per block size, the largest cap at each
 * number of resident blocks per SM; those that fit) advance one untimed
 * step and then steps_per_trial ordinary steps, each as the step graph with
 * CUDA event nodes around the plan and collision launches, and sum their
 * times; time the three fastest once more the same way and keep the one
 * with the least total.  The trial steps are part of the run (results do
 * not depend on the schedule); call it once the flow is developed.
 * *cap_out / *warps_out (may be NULL) receive the choice. */
sp_status sp_autotune(sp_ctx* ctx, int steps_per_trial, int* cap_out, int* warps_out);
/* Wait for the context's stream. */
sp_status sp_sync(sp_ctx* ctx);
/* Number of kernel launches one sp_step() issues (for launch accounting). */
int sp_launches_per_step(sp_ctx* ctx);
/* Release a context: waits for its stream, frees its device memory and
 * graphs.  (The end of the run of Sec. III.B: the fields of Step 6 are read
 * with sp_moments() before this call.) */
sp_status sp_free(sp_ctx* ctx);

/* Stable counting sort of cell keys that allocates no device memory.  The
 * paper has no counterpart: this is the indexing step (Step 3) offered as a
 * standalone call for callers that cannot call cudaMalloc -- code that runs
 * where the device memory plan is fixed (between CUDA-graph captures, under
 * a hard memory quota) or hosts that own every device buffer and forbid the
 * library to allocate.
 *   d_keys  device uint32 [n]: cell of each particle; keys >= ncells drop
 *           the particle (0xFFFFFFFF marks a removed particle)
 *   d_start device uint32 [ncells+1] (out): cell offsets, d_start[ncells]
 *           = number of particles kept
 *   d_perm  device uint32 [n] (out): d_perm[d_start[c] + r] = index of the
 *           r-th kept particle of cell c, in ascending index order
 *   stream  cudaStream_t or NULL; the call is asynchronous on it.
 * Scratch lives in a file-scope __device__ array sized for ncells <=
 * 1,048,576 (8 MiB, held by every GPU that loads the library until exit);
 * larger ncells, or n > 2^30 keys, return SP_ERR_CAPACITY with a message.
 * Cells of up to 1024 entries are put in order by one warp each, larger
 * ones by a block each (a cell of 2^20 entries takes a few tenths of a
 * second).  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture.  Every call shares the one
 * array and clears the counters it needs, so calls whose work overlaps on
 * the GPU (different streams, or different host threads) race: serialise
 * them.  Calls no cudaMalloc, cudaFree or other allocating routine. */
sp_status sp_sort_cells_static(const uint32_t* d_keys, int64_t n, int64_t ncells, uint32_t* d_start,
                               uint32_t* d_perm, void* stream);
const char* sp_status_str(int status);

#ifdef __cplusplus
}
#endif
#endif
