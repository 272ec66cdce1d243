/*
 * oracle.h -- plain FP64 CPU oracle of the hybrid stochastic-particle Shakhov /
 * DSMC time step (Jin, Liu, Yang, Cao, Zhuo, Zhong, "A hybrid numerical
 * algorithm based on the stochastic particle Shakhov and DSMC method",
 * arXiv:2506.23917).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library; it
 * is slow on purpose, single threaded, and written as a direct restatement
 * of the paper's steps (Sec. III.B, Steps 1-6).  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares
 * no code, header or constant table with the CUDA library.
 *
 * One context = one flow instance on a uniform Cartesian grid or a
 * body-fitted O-grid (the mesh option below).
 */
#ifndef SP_ORACLE_H
#define SP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_OK = 0, OR_ERR_ARG = -1, OR_ERR_CAPACITY = -3 };
enum { OR_BC_SPECULAR = 0, OR_BC_DIFFUSE = 1, OR_BC_OUTFLOW = 2, OR_BC_INFLOW = 3 };
enum { OR_BODY_NONE = 0, OR_BODY_CIRCLE = 1, OR_BODY_SPHERE = 2 };
enum { OR_MODE_HYBRID = 0, OR_MODE_DSMC = 1, OR_MODE_SHAKHOV = 2 };

typedef struct or_config {
  int32_t dim;            /* spatial dimensions 1..3; velocities are always 3-D */
  int32_t n[3];           /* cells per axis (1 on unused axes)                    */
  double lo[3], hi[3];    /* domain box (unused axes: a unit extent)              */
  double m;               /* molecular mass                                       */
  double R;               /* specific gas constant k/m                            */
  double gamma;           /* ratio of specific heats                              */
  double Pr;              /* Prandtl number of the Shakhov target                 */
  double omega;           /* VHS viscosity-temperature exponent                   */
  double T_ref, mu_ref;   /* mu = mu_ref (T/T_ref)^omega                          */
  double d_ref;           /* VHS reference diameter                               */
  double Fn;              /* real molecules per simulated particle                */
  double cfl;             /* Delta t_G = cfl * min_k Delta t_c,k                  */
  double dt_fixed;        /* > 0: constant step                                   */
  int32_t face_bc[6];     /* face 2*axis+side (side 0 = lo)                       */
  double face_T[6];       /* wall / reservoir temperature                         */
  double face_n[6];       /* reservoir number density (inflow)                    */
  double face_u[6][3];    /* reservoir drift velocity (inflow)                    */
  int32_t ghost_layers;   /* reservoir layers outside each inflow face            */
  int32_t body;           /* OR_BODY_*                                            */
  double body_c[3], body_r, body_Tw;
  const double* cell_volume; /* [ncells] or NULL (uniform)                        */
  double sigc_T0;         /* temperature that seeds (sigma_T c_r)_max             */
  int32_t n_steady;       /* first sampled step                                   */
  uint64_t seed;
  int32_t mode;           /* OR_MODE_*                                            */
  int32_t ar_max;         /* Shakhov acceptance-rejection attempt cap             */
  int32_t n_surf;         /* surface elements of the body (0: no surface tallies) */
  /* Open part of each outflow / inflow face: on the face's tangential axes
   * (the other axes below dim, in increasing order) the face is open where
   * win_lo <= x <= win_hi; an axis with win_lo >= win_hi is not restricted.
   * Elsewhere the face is a diffuse wall at face_T (an orifice with lips). */
  double win_lo[6][2], win_hi[6][2];
  /* Fractional part of the NTC candidate count: 0 = stochastic rounding
   * with one uniform per cell and step; 1 = Bird's carried remainder (the
   * fraction is kept per cell, starting at 0, and added to the next step's
   * count). */
  int32_t ntc_carry;
  /* Bird's sub-cells (an option; Sec. II.A selects pairs anywhere in the
   * cell): 0 or 1 = off; s >= 2 splits each cell into s parts per axis
   * (s^dim sub-cells, at most 8) and takes a candidate's partner from the
   * first particle's sub-cell when it holds another particle. */
  int32_t subcells;
  /* Body-fitted O-grid about a circular body (an option, 2-D only; the
   * paper's cylinder meshes are body-fitted, Sec. IV.B).  0 = the Cartesian
   * grid above.  1 = n[0] radial layers x n[1] sectors of straight-edged
   * quadrilaterals between the body polygon (nodes on the circle of radius
   * body_r about body_c) and the outer polygon (radius about mesh_r_out):
   * node radii r_0 = body_r, r_{i+1} = r_i + dr_i with dr_{i+1} =
   * mesh_growth * dr_i, the sum of the first n[0] spacings being
   * mesh_r_out - body_r; node angles 2 pi j / n[1].  Cell k = i + n[0] j.
   * The body polygon is a diffuse wall at body_Tw; the outer polygon is
   * face 1 (face_bc[1], and for an inflow boundary face_n/T/u[1] and
   * ghost_layers reservoir layers continuing the radial spacing).  Particles
   * find their cell by face crossing.  lo/hi[2] give the depth. */
  int32_t mesh;
  double mesh_r_out, mesh_growth;
} or_config;

typedef struct or_ctx or_ctx;

/* Moment fields, [field][cell]: */
enum {
  OR_F_N = 0, OR_F_n, OR_F_ux, OR_F_uy, OR_F_uz, OR_F_T, OR_F_qx, OR_F_qy, OR_F_qz,
  OR_F_tau, OR_F_dtc, OR_F_ratio, OR_NFIELDS
};

int or_init(const or_config* cfg, or_ctx** out);
/* pos: [dim][M] SoA, vel: [3][M] SoA.  Indexes and sorts the particles
 * (state S_0) and sets Delta t^0 from the moments of S_0. */
int or_set_particles(or_ctx* c, const double* pos, const double* vel, int64_t M);
int or_step(or_ctx* c, int nsteps);
int64_t or_num_particles(const or_ctx* c);
int or_get_particles(const or_ctx* c, double* pos, double* vel, uint32_t* cell);
/* kind 0: moments of the current state; kind 1: time-averaged (Step 6). */
int or_moments(const or_ctx* c, int kind, double* out, int nfields);
/* Records of the last step: per cell of S_n (cand, acc, nres, ar_attempts),
 * per particle of S_n the resample flag, and the stable-sort permutation
 * that produced S_{n+1} (old index of each new slot). */
int or_get_step_record(const or_ctx* c, int64_t* cell4, uint8_t* resampled,
                       uint32_t* perm, int64_t* n_old);
int or_get_cell_start(const or_ctx* c, uint32_t* start);
int or_get_sigc_max(const or_ctx* c, double* out);
int or_get_sample(const or_ctx* c, double* out /* [8][ncells] */, int64_t* nsamp);
double or_dt(const or_ctx* c);
int64_t or_step_index(const or_ctx* c);
/* Surface tallies of the body over the sampled steps: out [7][n_surf] =
 * (hits, momentum given to the wall x, y, z, energy given to the wall,
 * momentum given along the inward normal, momentum given along e_theta),
 * time = sampled time.  Element b of a circle spans polar angle
 * theta = atan2(n_y, n_x) in [-pi + 2 pi b/n, -pi + 2 pi (b+1)/n); of a
 * sphere, theta = acos(n_x) in [pi b/n, pi (b+1)/n).  e_theta is the unit
 * direction of increasing theta at the hit point (zero on a sphere's axis). */
int or_get_surface(const or_ctx* c, double* out, double* time);
/* counters over the whole run: removed, injected, move_capped, ar_capped */
int or_get_totals(const or_ctx* c, int64_t* out4);
/* Threads of the per-cell loop (Steps 3-5) of or_step: cells are
 * independent, so any count gives results identical to 1 (the default).
 * Without OpenMP the count stays 1. */
int or_set_threads(or_ctx* c, int n);
/* The pair of one NTC candidate from its two uniforms (the selection the
 * step uses): soff = NULL, or the sub-cell offsets of the cell's slots. */
int or_select_pair(int64_t N, const int64_t* soff, double u1, double u2, int64_t* i, int64_t* j);
/* The stable order by sub-cell of N particles of cell `cell` (pos [dim][N])
 * that a step with cfg->subcells >= 2 uses: order[r] = input index of slot
 * r, soff[0..nsub] the sub-cell offsets. */
int or_subcell_order(const or_config* cfg, int64_t cell, const double* pos, int64_t N, int64_t* order,
                     int64_t* soff);
int or_get_threads(const or_ctx* c);
/* O-grid option: the cell containing each of n points (pos [2][n]) found
 * by face crossing from a first guess, -1 outside the mesh (inside the
 * body polygon or beyond the outer polygon). */
int or_mesh_locate(const or_ctx* c, const double* pos, int64_t n, int64_t* cell);
/* O-grid option: node coordinates [(n[0] + ghost_layers + 1) * n[1]][2]
 * (node (i, j) at row i * n[1] + j), per-cell faces [ncells][4][3] (unit
 * outward normal and offset n.x = d of faces inner, outer, theta_j,
 * theta_j+1) and per-cell size L (the shortest edge). */
int or_mesh_geometry(const or_ctx* c, double* nodes, double* faces, double* L);
/* Cell volumes [ncells] (O-grid: quadrilateral area x depth). */
int or_get_volumes(const or_ctx* c, double* vol);
void or_free(or_ctx* c);

/* Building blocks exported for the pin tests. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_u01_from_words(uint32_t a, uint32_t b);
double or_sigc(const or_config* cfg, double cr);   /* sigma_T(c_r) * c_r */
/* one homogeneous collision step on a single cell's velocities (no transport);
 * vel is [3][N] SoA, updated in place; returns the cell record. */
int or_collide_cell(const or_config* cfg, int64_t step, uint32_t cell, double volume,
                    double dt_G, double* sigc_max, double* vel, int64_t N,
                    int64_t rec[4], uint8_t* resampled);

#ifdef __cplusplus
}
#endif
#endif
