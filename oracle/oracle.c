/*
 * oracle.c -- plain FP64 CPU oracle of the hybrid SP-Shakhov / DSMC step of
 * arXiv:2506.23917 (Jin et al.).  TEST INFRASTRUCTURE ONLY: it is the
 * yardstick the CUDA library is checked against and is never part of the
 * library's compute path.
 *
 * Everything here is a direct, unoptimised restatement of the paper:
 *   Step 1  initial particles are given by the caller (Sec. III.B Step 1).
 *   Step 2  free transport r <- r + c dt (Eq. "free transport", Sec. II.A),
 *           specular / diffuse walls, removal at open faces (Step 2).
 *   Step 3  indexing into cells (stable counting sort) and the per-cell
 *           moments n, U, T, Q with the unbiased estimators of Step 3.
 *   Step 4  local observation time dt_c (Eq. "local time step"), relaxation
 *           time tau = mu/p (Sec. II.B), split of the step into a DSMC part
 *           and a Shakhov part (Eqs. "tDSMC", "tShakhov"); NTC collisions
 *           (Eq. "Ncol_DSMC", Sec. II.A) with VHS isotropic scattering;
 *           Shakhov resampling with probability 1-exp(-dt/tau)
 *           (Eq. "Ncol_SBGK"), Box-Muller Maxwellian (Eq. "Maxwell") and the
 *           acceptance-rejection weight A (Eq. "A_cal"); conservation rescale
 *           (Sec. II.B, the equation after "A_cal").
 *   Step 5  time-averaged sums N, c, c^2 after N_steady.
 * Sums are plain left-to-right loops in slot order.
 *
 * Readings where the paper is silent or garbled (each is also listed in the
 * design notes of the repository):
 *   - Shakhov polynomial uses (C^2/(RT) - 5); the printed C^2/(2RT) would not
 *     conserve momentum.
 *   - Q enters only through Q/(pRT) = q_s/(RT)^2 with the unbiased
 *     q_s = 1/2 * N/((N-1)(N-2)) * sum |C|^2 C (the paper's 1/V and m cancel
 *     against p; its missing F_N is restored by p = n m R T).
 *   - Diffuse normal speed c_n = sqrt(-2 R T_w ln R1) (the printed "cos" is a
 *     typo), tangential components Box-Muller at T_w.
 *   - A_max = A at |C| = 5 sqrt(RT), C parallel to q_s.
 *   - N_col fractional part: stochastic rounding with one uniform; with
 *     ntc_carry, Bird's carried remainder per cell (starting at 0).
 *   - VHS cross-section (Bird): sigma_T c_r = pi d_ref^2 (4 R T_ref)^(w-1/2)
 *     / Gamma(5/2 - w) * c_r^(2-2w).
 *   - Rescale targets U, T of Step 3; skipped when nothing was resampled.
 *   - Delta t^{n+1} = cfl * min_k dt_c,k on the state of step n; the collision
 *     and the move of step n both use Delta t^n.
 *   - The step is ordered collide -> sample -> move -> inject -> index, so the
 *     state between steps is "indexed, not yet collided".
 *   - Open (inflow) faces: a reservoir of ghost cells outside the face is
 *     refilled each step at the face state and its particles that cross the
 *     face within the step are kept (the paper's ghost cells of Sec. IV.A).
 *     Where two inflow faces meet, each face's reservoir also covers the
 *     corner block beyond the other; a particle is kept only by the face it
 *     crosses first, so no phase-space region is injected twice.
 *   - A face may be open only on a window (an orifice); the rest of it is a
 *     diffuse wall at the face temperature, and the reservoir of a windowed
 *     inflow face spans the window plus ghost_layers cells on each side.
 *   - Body-fitted meshes (Sec. IV.B-E, not available) are stood in for by a
 *     synthetic O-grid of straight-edged quadrilaterals about the body
 *     polygon; particles find their cell by crossing faces; the local
 *     observation time uses each cell's shortest edge; the freestream
 *     enters from reservoir rings beyond the outer polygon.
 */
#define _GNU_SOURCE
#include "oracle.h"

#include <math.h>
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#include <stdlib.h>
#include <string.h>

#define PURP_NTC 1u
#define PURP_SHK 2u
#define PURP_WALL 3u
#define PURP_INJ 4u
#define PURP_INJWALL 5u
#define MAX_BOUNCE 16
#define NCOL_CAP (1LL << 24)
#define SENTINEL 0xFFFFFFFFu

typedef struct {
  double x[3];
  double v[3];
} part;

struct or_ctx {
  or_config cfg;
  int64_t ncells;
  double *vol;
  double inv_d[3], dl[3], Lmin;
  double sigc_coef, sigc_exp;
  uint32_t key[2];
  /* state S_n */
  part *p;
  int64_t M, cap;
  uint32_t *start; /* [ncells+1] */
  double *smax;
  double *rem; /* carried NTC remainder per cell (ntc_carry) */
  double *samp; /* [8][ncells] */
  int64_t nsamp;
  double dt;
  int64_t step;
  /* record of the last step */
  int64_t *rec;      /* [4][ncells] */
  uint8_t *resamp;   /* [M_old] */
  int64_t rec_n;
  uint32_t *perm;    /* [M] */
  int64_t totals[4];
  /* surface tallies (Step 5 sampling of wall fluxes) */
  double *surf; /* [7][n_surf] */
  double surf_time;
  int sampling_now;
  int nthreads; /* threads of the per-cell loop of a step (OpenMP; 1 = sequential) */
  double *Lc;   /* [ncells] cell size L of Delta t_c (uniform grid: L_min) */
  /* body-fitted O-grid (cfg.mesh == 1) */
  int mnr, mnt, mnl; /* radial layers, sectors, reservoir layers */
  double *mrad;      /* [mnr + mnl + 1] node radii */
  double *mnode;     /* [(mnr + mnl + 1) * mnt][2] node coordinates */
  double *mrel;      /* the same relative to the body centre (areas) */
  double *mface;     /* [ncells][4][3] outward unit normal, offset */
};

/* ---------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random
 * numbers: as easy as 1, 2, 3").  Round: two 32x32->64 products of the
 * counter words 0 and 2 with the round multipliers; key schedule bumped by
 * the Weyl constants between rounds.
 * ------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in (0,1) from two 32-bit words: 52 random bits k, u = (2k+1)/2^53. */
double or_u01_from_words(uint32_t a, uint32_t b) {
  uint64_t k = ((uint64_t)(a >> 6) << 26) | (uint64_t)(b >> 6);
  return (double)(2 * k + 1) * 0x1p-53;
}

/* q-th uniform of the stream (step, a, b, purpose, subbase + q/2). */
static double uq(const or_ctx* c, uint32_t a, uint32_t b, uint32_t purpose, uint32_t subbase, int q) {
  uint32_t ctr[4] = {(uint32_t)c->step, a, b, (purpose << 24) | (subbase + (uint32_t)(q / 2))};
  uint32_t o[4];
  or_philox4x32_10(ctr, c->key, o);
  return (q % 2 == 0) ? or_u01_from_words(o[0], o[1]) : or_u01_from_words(o[2], o[3]);
}

/* VHS: sigma_T(c_r) c_r (Sec. II.A; Bird's VHS diameter law, see header). */
double or_sigc(const or_config* g, double cr) {
  double coef = M_PI * g->d_ref * g->d_ref * pow(4.0 * g->R * g->T_ref, g->omega - 0.5) /
                tgamma(2.5 - g->omega);
  return coef * pow(cr, 2.0 - 2.0 * g->omega);
}

static double sigc_fast(const or_ctx* c, double cr) { return c->sigc_coef * pow(cr, c->sigc_exp); }

static int64_t cell_of(const or_ctx* c, const double* x) {
  const or_config* g = &c->cfg;
  int64_t idx[3] = {0, 0, 0};
  for (int d = 0; d < g->dim; ++d) {
    double f = floor((x[d] - g->lo[d]) * c->inv_d[d]);
    int64_t i = (int64_t)f;
    if (f < 0) i = 0;
    if (i > g->n[d] - 1) i = g->n[d] - 1;
    idx[d] = i;
  }
  return idx[0] + (int64_t)g->n[0] * (idx[1] + (int64_t)g->n[1] * idx[2]);
}

/* ---------------------------------------------------------------------
 * Step 3: per-cell moments with the unbiased estimators.
 * ------------------------------------------------------------------- */
typedef struct {
  int64_t N;
  double U[3], T, q[3], n, p, tau, dtc;
} mom;

static void moments_of(const or_ctx* c, int64_t k, const part* ps, int64_t N, mom* o) {
  const or_config* g = &c->cfg;
  memset(o, 0, sizeof *o);
  o->N = N;
  o->tau = INFINITY;
  o->dtc = INFINITY;
  if (N == 0) return;
  double s[3] = {0, 0, 0};
  for (int64_t i = 0; i < N; ++i)
    for (int d = 0; d < 3; ++d) s[d] += ps[i].v[d];
  for (int d = 0; d < 3; ++d) o->U[d] = s[d] / (double)N;
  o->n = (double)N * g->Fn / c->vol[k];
  if (N < 2) return;
  double S2 = 0, S3[3] = {0, 0, 0};
  for (int64_t i = 0; i < N; ++i) {
    double C0 = ps[i].v[0] - o->U[0], C1 = ps[i].v[1] - o->U[1], C2 = ps[i].v[2] - o->U[2];
    double c2 = C0 * C0 + C1 * C1 + C2 * C2;
    S2 += c2;
    S3[0] += c2 * C0;
    S3[1] += c2 * C1;
    S3[2] += c2 * C2;
  }
  o->T = S2 / (3.0 * g->R * (double)(N - 1));
  if (N >= 3)
    for (int d = 0; d < 3; ++d)
      o->q[d] = 0.5 * (double)N * S3[d] / ((double)(N - 1) * (double)(N - 2));
  double umag = sqrt(o->U[0] * o->U[0] + o->U[1] * o->U[1] + o->U[2] * o->U[2]);
  if (o->T > 0) {
    o->p = o->n * g->m * g->R * o->T;
    double mu = g->mu_ref * pow(o->T / g->T_ref, g->omega);
    o->tau = mu / o->p;
    o->dtc = c->Lc[k] / (umag + sqrt(g->gamma * g->R * o->T));
  } else if (umag > 0) {
    o->dtc = c->Lc[k] / umag;
  }
}

/* Split of the global step into DSMC and Shakhov parts (Eqs. tDSMC, tShakhov). */
static void split(const or_config* g, const mom* mm, double dtG, double* dsmc, double* sbgk) {
  if (g->mode == OR_MODE_DSMC) { *dsmc = dtG; *sbgk = 0; return; }
  if (g->mode == OR_MODE_SHAKHOV) { *dsmc = 0; *sbgk = dtG; return; }
  if (mm->dtc <= mm->tau) { *dsmc = dtG; *sbgk = 0; return; }
  double r = mm->tau / mm->dtc;
  *dsmc = r * dtG;
  *sbgk = (1.0 - r) * dtG;
}

static double ratio_of(const or_config* g, const mom* mm) {
  if (g->mode == OR_MODE_DSMC) return 1.0;
  if (g->mode == OR_MODE_SHAKHOV) return 0.0;
  if (mm->N < 2 || !(mm->T > 0) || mm->dtc <= mm->tau) return 1.0;
  return mm->tau / mm->dtc;
}

/* ---------------------------------------------------------------------
 * Bird's sub-cells (option).  The sub-cell of a particle of cell k: on each
 * axis the cell coordinate u = (x - lo) n / L (the expression of cell_of),
 * its fractional part within the cell split into s equal parts.  Before its
 * step, a cell's particles are put in a stable order by sub-cell, so that
 * every sub-cell is a run of consecutive slots: soff[t] .. soff[t+1].
 * ------------------------------------------------------------------- */
static int nsub_of(const or_config* g) {
  int ns = g->subcells > 1 ? g->subcells : 1, m = 1;
  for (int d = 0; d < g->dim; ++d) m *= ns;
  return m;
}

static int subcell_of(const or_ctx* c, int64_t k, const double* x) {
  const or_config* g = &c->cfg;
  const int ns = g->subcells;
  int64_t kk = k;
  int sub = 0, mul = 1;
  for (int d = 0; d < g->dim; ++d) {
    int64_t id = kk % g->n[d];
    kk /= g->n[d];
    double u = (x[d] - g->lo[d]) * c->inv_d[d];
    double f = floor((u - (double)id) * (double)ns);
    int t = (int)f;
    if (f < 0) t = 0;
    if (t > ns - 1) t = ns - 1;
    sub += mul * t;
    mul *= ns;
  }
  return sub;
}

/* The pair of an NTC candidate (Sec. II.A: "selected randomly within the
 * cell"): i uniform over the N slots, j uniform over the other N - 1; with
 * sub-cells, j uniform over the other particles of i's sub-cell (slots
 * soff[t] .. soff[t+1]) when it holds one. */
static void select_pair(int64_t N, const int64_t* soff, double u1, double u2, int64_t* pi, int64_t* pj) {
  int64_t i = (int64_t)(u1 * (double)N);
  if (i > N - 1) i = N - 1;
  int64_t a0 = 0, b0 = N;
  if (soff) {
    int t = 0;
    while (soff[t + 1] <= i) ++t;
    if (soff[t + 1] - soff[t] >= 2) {
      a0 = soff[t];
      b0 = soff[t + 1];
    }
  }
  int64_t j = a0 + (int64_t)(u2 * (double)(b0 - a0 - 1));
  if (j > b0 - 2) j = b0 - 2;
  if (j >= i) j += 1;
  *pi = i;
  *pj = j;
}

static void order_by_subcell(const or_ctx* c, int64_t k, part* ps, int64_t N, int64_t* soff) {
  const int m = nsub_of(&c->cfg);
  int64_t cnt[9] = {0};
  if (N == 0) { /* an empty cell: nothing to order (ps is the next cell's) */
    for (int t = 0; t <= m; ++t) soff[t] = 0;
    return;
  }
  int* sub = (int*)malloc(sizeof(int) * N);
  part* tmp = (part*)malloc(sizeof(part) * N);
  for (int64_t i = 0; i < N; ++i) {
    sub[i] = subcell_of(c, k, ps[i].x);
    cnt[sub[i] + 1] += 1;
  }
  for (int t = 0; t < m; ++t) cnt[t + 1] += cnt[t];
  for (int t = 0; t <= m; ++t) soff[t] = cnt[t];
  for (int64_t i = 0; i < N; ++i) tmp[cnt[sub[i]]++] = ps[i];
  memcpy(ps, tmp, sizeof(part) * N);
  free(tmp);
  free(sub);
}

/* ---------------------------------------------------------------------
 * Step 4 on one cell: NTC DSMC part, Shakhov part, rescale.
 * ps[0..N) are the cell's particles in slot order; k is the cell's index.
 * ------------------------------------------------------------------- */
static void collide_cell(or_ctx* c, int64_t k, double V, part* ps, int64_t N, const mom* mm,
                         double dtG, double* smax, double* rem, int64_t rec[4], uint8_t* res,
                         const int64_t* soff) {
  const or_config* g = &c->cfg;
  rec[0] = rec[1] = rec[2] = rec[3] = 0;
  if (N < 2 || !(mm->T > 0)) return;
  double dsmc, sbgk;
  split(g, mm, dtG, &dsmc, &sbgk);
  uint32_t kc = (uint32_t)k;

  /* DSMC, NTC scheme (Sec. II.A). */
  if (dsmc > 0) {
    double ncr = 0.5 * (double)N * (double)(N - 1) * g->Fn * (*smax) * dsmc / V;
    int64_t ncol;
    if (g->ntc_carry) {
      /* Bird's carried remainder */
      double x = ncr + *rem;
      ncol = (int64_t)floor(x);
      *rem = x - (double)ncol;
    } else {
      double ur = uq(c, kc, SENTINEL, PURP_NTC, 0, 0);
      ncol = (int64_t)floor(ncr + ur);
    }
    if (ncol > NCOL_CAP) ncol = NCOL_CAP;
    for (int64_t kk = 0; kk < ncol; ++kk) {
      double u1 = uq(c, kc, (uint32_t)kk, PURP_NTC, 0, 0);
      double u2 = uq(c, kc, (uint32_t)kk, PURP_NTC, 0, 1);
      double u3 = uq(c, kc, (uint32_t)kk, PURP_NTC, 0, 2);
      double u4 = uq(c, kc, (uint32_t)kk, PURP_NTC, 0, 3);
      double u5 = uq(c, kc, (uint32_t)kk, PURP_NTC, 0, 4);
      int64_t i, j;
      select_pair(N, soff, u1, u2, &i, &j);
      double* a = ps[i].v;
      double* b = ps[j].v;
      double g0 = a[0] - b[0], g1 = a[1] - b[1], g2 = a[2] - b[2];
      double cr = sqrt(g0 * g0 + g1 * g1 + g2 * g2);
      double sc = sigc_fast(c, cr);
      if (sc > *smax) *smax = sc;
      rec[0] += 1;
      if (u3 < sc / *smax) {
        rec[1] += 1;
        double cchi = 2.0 * u4 - 1.0;
        double schi = sqrt(1.0 - cchi * cchi);
        double th = 2.0 * M_PI * u5;
        double w0 = cchi, w1 = schi * cos(th), w2 = schi * sin(th);
        double m0 = a[0] + b[0], m1 = a[1] + b[1], m2 = a[2] + b[2];
        a[0] = 0.5 * (m0 - cr * w0);
        a[1] = 0.5 * (m1 - cr * w1);
        a[2] = 0.5 * (m2 - cr * w2);
        b[0] = 0.5 * (m0 + cr * w0);
        b[1] = 0.5 * (m1 + cr * w1);
        b[2] = 0.5 * (m2 + cr * w2);
      }
    }
  }

  /* Shakhov relaxation (Sec. II.B), only where q_s is defined (N >= 3). */
  if (sbgk > 0 && N >= 3) {
    double P = 1.0 - exp(-sbgk / mm->tau);
    double RT = g->R * mm->T;
    double s2RT = sqrt(2.0 * RT);
    double qn = sqrt(mm->q[0] * mm->q[0] + mm->q[1] * mm->q[1] + mm->q[2] * mm->q[2]);
    double Amax = 1.0 + 20.0 * (1.0 - g->Pr) * qn / (RT * sqrt(RT));
    int64_t nres = 0;
    for (int64_t s = 0; s < N; ++s) {
      double u0 = uq(c, kc, (uint32_t)s, PURP_SHK, 0, 0);
      if (!(u0 < P)) continue;
      if (res) res[s] = 1;
      nres += 1;
      double C0 = 0, C1 = 0, C2 = 0;
      for (int t = 0; t < g->ar_max; ++t) {
        double R1 = uq(c, kc, (uint32_t)s, PURP_SHK, 0, 1 + 5 * t);
        double R2 = uq(c, kc, (uint32_t)s, PURP_SHK, 0, 2 + 5 * t);
        double R3 = uq(c, kc, (uint32_t)s, PURP_SHK, 0, 3 + 5 * t);
        double R4 = uq(c, kc, (uint32_t)s, PURP_SHK, 0, 4 + 5 * t);
        double R5 = uq(c, kc, (uint32_t)s, PURP_SHK, 0, 5 + 5 * t);
        double r2 = sqrt(-log(R2)), r4 = sqrt(-log(R4));
        C0 = s2RT * cos(2.0 * M_PI * R1) * r2;
        C1 = s2RT * cos(2.0 * M_PI * R3) * r4;
        C2 = s2RT * sin(2.0 * M_PI * R3) * r4;
        double qC = mm->q[0] * C0 + mm->q[1] * C1 + mm->q[2] * C2;
        double CC = C0 * C0 + C1 * C1 + C2 * C2;
        double A = 1.0 + (1.0 - g->Pr) * qC / (5.0 * RT * RT) * (CC / RT - 5.0);
        rec[3] += 1;
        if (R5 * Amax < A) break;
        if (t == g->ar_max - 1) {
#ifdef _OPENMP
#pragma omp atomic
#endif
          c->totals[3] += 1;
        }
      }
      ps[s].v[0] = mm->U[0] + C0;
      ps[s].v[1] = mm->U[1] + C1;
      ps[s].v[2] = mm->U[2] + C2;
    }
    rec[2] = nres;
    /* Conservation rescale: c' = U + (c_p - U_p) sqrt(T/T_p). */
    if (nres > 0) {
      double s[3] = {0, 0, 0};
      for (int64_t i = 0; i < N; ++i)
        for (int d = 0; d < 3; ++d) s[d] += ps[i].v[d];
      double Up[3] = {s[0] / (double)N, s[1] / (double)N, s[2] / (double)N};
      double S2 = 0;
      for (int64_t i = 0; i < N; ++i) {
        double C0 = ps[i].v[0] - Up[0], C1 = ps[i].v[1] - Up[1], C2 = ps[i].v[2] - Up[2];
        S2 += C0 * C0 + C1 * C1 + C2 * C2;
      }
      double Tp = S2 / (3.0 * g->R * (double)(N - 1));
      if (Tp > 0) {
        double f = sqrt(mm->T / Tp);
        for (int64_t i = 0; i < N; ++i)
          for (int d = 0; d < 3; ++d) ps[i].v[d] = mm->U[d] + (ps[i].v[d] - Up[d]) * f;
      }
    }
  }
}

/* ---------------------------------------------------------------------
 * Step 2: free flight with walls.  Returns 1 if the particle left the
 * domain.  Draw stream: (purpose, a, b, subbase + 2*bounce + blk).
 * ------------------------------------------------------------------- */
static void diffuse_sample(const or_ctx* c, double Tw, uint32_t purpose, uint32_t a, uint32_t b,
                           uint32_t sub, double* cn, double* t1, double* t2) {
  double R1 = uq(c, a, b, purpose, sub, 0);
  double R3 = uq(c, a, b, purpose, sub, 1);
  double R4 = uq(c, a, b, purpose, sub, 2);
  double RTw = c->cfg.R * Tw;
  *cn = sqrt(-2.0 * RTw * log(R1));
  double r4 = sqrt(-log(R4));
  double s = sqrt(2.0 * RTw);
  *t1 = s * cos(2.0 * M_PI * R3) * r4;
  *t2 = s * sin(2.0 * M_PI * R3) * r4;
}

/* Whether the crossing point x of face f lies in the face's open window. */
static int face_open(const or_config* g, int f, const double* x) {
  int ax = f / 2, i = 0;
  for (int d = 0; d < g->dim; ++d) {
    if (d == ax) continue;
    if (g->win_lo[f][i] < g->win_hi[f][i] && (x[d] < g->win_lo[f][i] || x[d] > g->win_hi[f][i]))
      return 0;
    ++i;
  }
  return 1;
}

/* Surface tallies of one body hit (Step 5 sampling of the wall fluxes):
 * the momentum and energy the wall receives, binned by the polar angle of
 * the inward normal nv at the hit point. */
static void tally_hit(or_ctx* c, const double* nv, const double* vin, const double* v) {
  const or_config* g = &c->cfg;
  if (!(c->sampling_now && g->n_surf > 0)) return;
  int ns = g->n_surf;
  double th, frac;
  if (g->body == OR_BODY_CIRCLE) {
    th = atan2(nv[1], nv[0]);
    frac = (th + M_PI) / (2.0 * M_PI);
  } else {
    double cx = nv[0] < -1.0 ? -1.0 : (nv[0] > 1.0 ? 1.0 : nv[0]);
    th = acos(cx);
    frac = th / M_PI;
  }
  int bin = (int)floor(frac * (double)ns);
  if (bin < 0) bin = 0;
  if (bin > ns - 1) bin = ns - 1;
  double w = g->Fn * g->m;
  double ein = vin[0] * vin[0] + vin[1] * vin[1] + vin[2] * vin[2];
  double eout = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  double dp[3], et[3] = {0, 0, 0};
  for (int d = 0; d < 3; ++d) dp[d] = w * (vin[d] - v[d]);
  /* direction of increasing polar angle at the hit point */
  if (g->body == OR_BODY_CIRCLE) {
    et[0] = -nv[1];
    et[1] = nv[0];
  } else {
    double sn = sqrt(nv[1] * nv[1] + nv[2] * nv[2]);
    if (sn > 0) {
      et[0] = -sn;
      et[1] = nv[0] * nv[1] / sn;
      et[2] = nv[0] * nv[2] / sn;
    }
  }
  c->surf[0 * ns + bin] += 1.0;
  for (int d = 0; d < 3; ++d) c->surf[(1 + d) * ns + bin] += dp[d];
  c->surf[4 * ns + bin] += 0.5 * w * (ein - eout);
  c->surf[5 * ns + bin] -= dp[0] * nv[0] + dp[1] * nv[1] + dp[2] * nv[2];
  c->surf[6 * ns + bin] += dp[0] * et[0] + dp[1] * et[1] + dp[2] * et[2];
}

static int move_particle(or_ctx* c, double* x, double* v, double trem, uint32_t purpose, uint32_t a,
                         uint32_t b, uint32_t subbase) {
  const or_config* g = &c->cfg;
  for (int bounce = 0;; ++bounce) {
    if (bounce >= MAX_BOUNCE) { c->totals[2] += 1; return 0; }
    /* earliest domain face */
    double tf = INFINITY;
    int fa = -1, fs = 0;
    for (int d = 0; d < g->dim; ++d) {
      double t;
      if (v[d] > 0) { t = (g->hi[d] - x[d]) / v[d]; if (t < tf) { tf = t; fa = d; fs = 1; } }
      else if (v[d] < 0) { t = (g->lo[d] - x[d]) / v[d]; if (t < tf) { tf = t; fa = d; fs = 0; } }
    }
    /* body */
    double tb = INFINITY;
    if (g->body != OR_BODY_NONE) {
      int D = g->body == OR_BODY_CIRCLE ? 2 : 3;
      double bb = 0, aa = 0, cc = 0;
      for (int d = 0; d < D; ++d) {
        double dx = x[d] - g->body_c[d];
        bb += v[d] * dx;
        aa += v[d] * v[d];
        cc += dx * dx;
      }
      cc -= g->body_r * g->body_r;
      if (bb < 0 && aa > 0) {
        double disc = bb * bb - aa * cc;
        if (disc >= 0) {
          double t = (-bb - sqrt(disc)) / aa;
          tb = t < 0 ? 0 : t;
        }
      }
    }
    double th = tf < tb ? tf : tb;
    if (!(th < trem)) {
      for (int d = 0; d < g->dim; ++d) x[d] += v[d] * trem;
      return 0;
    }
    uint32_t sub = subbase + 2u * (uint32_t)bounce;
    if (tb <= tf) {
      for (int d = 0; d < g->dim; ++d) x[d] += v[d] * tb;
      trem -= tb;
      double nv[3] = {0, 0, 0};
      int D = g->body == OR_BODY_CIRCLE ? 2 : 3;
      for (int d = 0; d < D; ++d) nv[d] = (x[d] - g->body_c[d]) / g->body_r;
      double e1[3], e2[3];
      if (g->body == OR_BODY_CIRCLE) {
        e1[0] = -nv[1]; e1[1] = nv[0]; e1[2] = 0;
        e2[0] = 0; e2[1] = 0; e2[2] = 1;
      } else {
        double ax[3] = {0, 0, 0};
        if (fabs(nv[0]) < 0.9) ax[0] = 1; else ax[1] = 1;
        double cx = nv[1] * ax[2] - nv[2] * ax[1];
        double cy = nv[2] * ax[0] - nv[0] * ax[2];
        double cz = nv[0] * ax[1] - nv[1] * ax[0];
        double cn = sqrt(cx * cx + cy * cy + cz * cz);
        e1[0] = cx / cn; e1[1] = cy / cn; e1[2] = cz / cn;
        e2[0] = nv[1] * e1[2] - nv[2] * e1[1];
        e2[1] = nv[2] * e1[0] - nv[0] * e1[2];
        e2[2] = nv[0] * e1[1] - nv[1] * e1[0];
      }
      double cn, t1, t2;
      diffuse_sample(c, g->body_Tw, purpose, a, b, sub, &cn, &t1, &t2);
      double vin[3] = {v[0], v[1], v[2]};
      for (int d = 0; d < 3; ++d) v[d] = cn * nv[d] + t1 * e1[d] + t2 * e2[d];
      tally_hit(c, nv, vin, v);
      continue;
    }
    for (int d = 0; d < g->dim; ++d)
      if (d != fa) x[d] += v[d] * tf;
    x[fa] = fs ? g->hi[fa] : g->lo[fa];
    trem -= tf;
    int f = 2 * fa + fs;
    int bc = g->face_bc[f];
    if ((bc == OR_BC_OUTFLOW || bc == OR_BC_INFLOW) && !face_open(g, f, x)) bc = OR_BC_DIFFUSE;
    if (bc == OR_BC_SPECULAR) {
      v[fa] = -v[fa];
    } else if (bc == OR_BC_DIFFUSE) {
      double cn, t1, t2;
      diffuse_sample(c, g->face_T[f], purpose, a, b, sub, &cn, &t1, &t2);
      v[fa] = fs ? -cn : cn;
      v[(fa + 1) % 3] = t1;
      v[(fa + 2) % 3] = t2;
    } else {
      return 1;
    }
  }
}

/* ---------------------------------------------------------------------
 * Body-fitted O-grid (option, 2-D): straight-edged quadrilaterals between
 * the body polygon and the outer polygon.  A particle carries its cell and
 * finds the next one by face crossing: from its position it leaves the
 * cell through the face whose line its straight path meets first among
 * the faces it moves towards (exit times below zero count as zero, so a
 * point that rounding left just outside a face leaves at once), crosses
 * into the neighbour, and repeats until the remaining time ends inside the
 * current cell.
 * ------------------------------------------------------------------- */
#define MESH_TWO_PI (2.0 * 3.14159265358979323846)
#define MAX_CROSS 4096

static const double* mesh_node(const or_ctx* c, int i, int j) {
  int jj = j % c->mnt;
  return c->mnode + 2 * ((int64_t)i * c->mnt + jj);
}
static const double* mesh_rel(const or_ctx* c, int i, int j) {
  int jj = j % c->mnt;
  return c->mrel + 2 * ((int64_t)i * c->mnt + jj);
}

/* Shoelace area of the quadrilateral p0 p1 p2 p3 (counter-clockwise). */
static double quad_area(const double* p0, const double* p1, const double* p2, const double* p3) {
  return 0.5 * ((p0[0] * p1[1] - p1[0] * p0[1]) + (p1[0] * p2[1] - p2[0] * p1[1]) +
                (p2[0] * p3[1] - p3[0] * p2[1]) + (p3[0] * p0[1] - p0[0] * p3[1]));
}
static double tri_area(const double* p0, const double* p1, const double* p2) {
  return 0.5 * ((p1[0] - p0[0]) * (p2[1] - p0[1]) - (p2[0] - p0[0]) * (p1[1] - p0[1]));
}

/* Unit outward normal and offset (n.x = d on the line) of the edge p -> q
 * of a counter-clockwise cell; returns the edge length. */
static double edge_line(const double* p, const double* q, double* f) {
  double tx = q[0] - p[0], ty = q[1] - p[1];
  double len = sqrt(tx * tx + ty * ty);
  f[0] = ty / len;
  f[1] = -tx / len;
  f[2] = f[0] * p[0] + f[1] * p[1];
  return len;
}

static int mesh_build(or_ctx* c) {
  or_config* g = &c->cfg;
  if (g->dim != 2 || g->body != OR_BODY_CIRCLE || g->n[0] < 1 || g->n[1] < 3 || !(g->body_r > 0) ||
      !(g->mesh_r_out > g->body_r) || !(g->mesh_growth > 0) || g->subcells > 1)
    return OR_ERR_ARG;
  int nr = g->n[0], nt = g->n[1], nl = g->ghost_layers > 0 ? g->ghost_layers : 0;
  c->mnr = nr;
  c->mnt = nt;
  c->mnl = nl;
  int nrad = nr + nl + 1;
  c->mrad = (double*)malloc(sizeof(double) * nrad);
  /* spacing dr_0 with dr_0 (1 + q + ... + q^(nr-1)) = r_out - r_0 */
  double q = g->mesh_growth, geo = 0.0, qp = 1.0;
  for (int i = 0; i < nr; ++i) {
    geo += qp;
    qp *= q;
  }
  double dr = (g->mesh_r_out - g->body_r) / geo;
  c->mrad[0] = g->body_r;
  for (int i = 0; i + 1 < nrad; ++i) {
    c->mrad[i + 1] = c->mrad[i] + dr;
    dr *= q;
  }
  c->mnode = (double*)malloc(sizeof(double) * 2 * (size_t)nrad * nt);
  c->mrel = (double*)malloc(sizeof(double) * 2 * (size_t)nrad * nt);
  for (int i = 0; i < nrad; ++i)
    for (int j = 0; j < nt; ++j) {
      double th = MESH_TWO_PI * (double)j / (double)nt;
      double rx = c->mrad[i] * cos(th), ry = c->mrad[i] * sin(th);
      int64_t o = 2 * ((int64_t)i * nt + j);
      c->mrel[o] = rx;
      c->mrel[o + 1] = ry;
      c->mnode[o] = g->body_c[0] + rx;
      c->mnode[o + 1] = g->body_c[1] + ry;
    }
  c->mface = (double*)malloc(sizeof(double) * 12 * (size_t)c->ncells);
  double depth = g->hi[2] - g->lo[2];
  for (int j = 0; j < nt; ++j)
    for (int i = 0; i < nr; ++i) {
      int64_t k = i + (int64_t)nr * j;
      const double *A = mesh_node(c, i, j), *B = mesh_node(c, i + 1, j);
      const double *C = mesh_node(c, i + 1, j + 1), *D = mesh_node(c, i, j + 1);
      double* f = c->mface + 12 * k;
      double l0 = edge_line(D, A, f + 0);  /* inner */
      double l1 = edge_line(B, C, f + 3);  /* outer */
      double l2 = edge_line(A, B, f + 6);  /* theta_j */
      double l3 = edge_line(C, D, f + 9);  /* theta_j+1 */
      double L = l0;
      if (l1 < L) L = l1;
      if (l2 < L) L = l2;
      if (l3 < L) L = l3;
      c->Lc[k] = L;
      c->vol[k] = quad_area(mesh_rel(c, i, j), mesh_rel(c, i + 1, j), mesh_rel(c, i + 1, j + 1),
                            mesh_rel(c, i, j + 1)) * depth;
    }
  return OR_OK;
}

/* Walk of one particle of cell *k for time trem (O-grid): interior faces
 * hand it to the neighbour, the body polygon re-emits it diffusely at
 * body_Tw, the outer polygon removes it (inflow, outflow), reflects it
 * (specular) or re-emits it (diffuse at face_T[1]).  locate != 0: the
 * point location walk (boundary faces end it with -1 instead).  Draws of
 * wall event b: (step, a, bb, purpose<<24 | subbase + 2b), as for the
 * Cartesian walls.  Returns 1 when the particle left the domain. */
static int mesh_walk(or_ctx* c, int64_t* k, double* x, double* v, double trem, uint32_t purpose,
                     uint32_t a, uint32_t bb, uint32_t subbase, int locate) {
  const or_config* g = &c->cfg;
  int nr = c->mnr, nt = c->mnt, bounce = 0;
  for (int cross = 0;; ++cross) {
    if (cross >= MAX_CROSS) {
      if (locate) return 1;
      c->totals[2] += 1;
      return 0;
    }
    const double* f = c->mface + 12 * *k;
    double tmin = INFINITY;
    int fm = -1;
    for (int e = 0; e < 4; ++e) {
      double nvv = f[3 * e] * v[0] + f[3 * e + 1] * v[1];
      if (nvv > 0) {
        double t = (f[3 * e + 2] - (f[3 * e] * x[0] + f[3 * e + 1] * x[1])) / nvv;
        if (t < 0) t = 0;
        if (t < tmin) {
          tmin = t;
          fm = e;
        }
      }
    }
    if (!(tmin < trem)) {
      x[0] += v[0] * trem;
      x[1] += v[1] * trem;
      return 0;
    }
    x[0] += v[0] * tmin;
    x[1] += v[1] * tmin;
    trem -= tmin;
    int i = (int)(*k % nr), j = (int)(*k / nr);
    if (fm == 2) { *k = i + (int64_t)nr * ((j + nt - 1) % nt); continue; }
    if (fm == 3) { *k = i + (int64_t)nr * ((j + 1) % nt); continue; }
    if (fm == 0 && i > 0) { *k -= 1; continue; }
    if (fm == 1 && i < nr - 1) { *k += 1; continue; }
    if (locate) return 1;
    if (bounce >= MAX_BOUNCE) { c->totals[2] += 1; return 0; }
    uint32_t sub = subbase + 2u * (uint32_t)bounce;
    ++bounce;
    /* a boundary face: normal into the domain */
    double nv[3] = {-f[3 * fm], -f[3 * fm + 1], 0};
    double Tw;
    if (fm == 1) {
      int bc = g->face_bc[1];
      if (bc == OR_BC_OUTFLOW || bc == OR_BC_INFLOW) return 1;
      if (bc == OR_BC_SPECULAR) {
        double vn = f[3] * v[0] + f[4] * v[1];
        v[0] -= 2.0 * vn * f[3];
        v[1] -= 2.0 * vn * f[4];
        continue;
      }
      Tw = g->face_T[1];
    } else {
      Tw = g->body_Tw;
    }
    double e1[3] = {-nv[1], nv[0], 0}, e2[3] = {0, 0, 1};
    double cn, t1, t2;
    diffuse_sample(c, Tw, purpose, a, bb, sub, &cn, &t1, &t2);
    double vin[3] = {v[0], v[1], v[2]};
    for (int d = 0; d < 3; ++d) v[d] = cn * nv[d] + t1 * e1[d] + t2 * e2[d];
    if (fm == 0) tally_hit(c, nv, vin, v);
  }
}

/* The cell of point x (O-grid): a first guess from the point's polar
 * coordinates, then the walk from that cell's centroid to x; -1 outside. */
static int64_t mesh_locate(const or_ctx* c, const double* x) {
  const or_config* g = &c->cfg;
  int nr = c->mnr, nt = c->mnt;
  double dx = x[0] - g->body_c[0], dy = x[1] - g->body_c[1];
  double r = sqrt(dx * dx + dy * dy), th = atan2(dy, dx);
  if (th < 0) th += MESH_TWO_PI;
  int j = (int)floor(th * (double)nt / MESH_TWO_PI);
  if (j < 0) j = 0;
  if (j > nt - 1) j = nt - 1;
  int i = 0;
  while (i < nr - 1 && c->mrad[i + 1] <= r) ++i;
  int64_t k = i + (int64_t)nr * j;
  const double *A = mesh_node(c, i, j), *B = mesh_node(c, i + 1, j);
  const double *C = mesh_node(c, i + 1, j + 1), *D = mesh_node(c, i, j + 1);
  double p[2] = {0.25 * (A[0] + B[0] + C[0] + D[0]), 0.25 * (A[1] + B[1] + C[1] + D[1])};
  double w[3] = {x[0] - p[0], x[1] - p[1], 0};
  if (mesh_walk((or_ctx*)c, &k, p, w, 1.0, 0, 0, 0, 0, 1)) return -1;
  return k;
}


/* ---------------------------------------------------------------------
 * Context
 * ------------------------------------------------------------------- */
int or_init(const or_config* cfg, or_ctx** out) {
  if (!cfg || !out || cfg->dim < 1 || cfg->dim > 3) return OR_ERR_ARG;
  or_ctx* c = (or_ctx*)calloc(1, sizeof *c);
  c->cfg = *cfg;
  c->nthreads = 1;
  if (nsub_of(cfg) > 8) {
    free(c);
    return OR_ERR_ARG;
  }
  or_config* g = &c->cfg;
  for (int d = 0; d < 3; ++d) {
    if (d >= g->dim) { g->n[d] = 1; }
    if (g->n[d] < 1 || !(g->hi[d] > g->lo[d])) { free(c); return OR_ERR_ARG; }
    c->dl[d] = (g->hi[d] - g->lo[d]) / (double)g->n[d];
    c->inv_d[d] = (double)g->n[d] / (g->hi[d] - g->lo[d]);
  }
  c->Lmin = INFINITY;
  for (int d = 0; d < g->dim; ++d)
    if (c->dl[d] < c->Lmin) c->Lmin = c->dl[d];
  c->ncells = (int64_t)g->n[0] * g->n[1] * g->n[2];
  c->vol = (double*)malloc(sizeof(double) * c->ncells);
  c->Lc = (double*)malloc(sizeof(double) * (c->ncells > 0 ? c->ncells : 1));
  double v0 = c->dl[0] * c->dl[1] * c->dl[2];
  for (int64_t k = 0; k < c->ncells; ++k) {
    c->vol[k] = cfg->cell_volume ? cfg->cell_volume[k] : v0;
    c->Lc[k] = c->Lmin;
  }
  g->cell_volume = NULL;
  if (g->mesh == 1) {
    if (mesh_build(c) != OR_OK) {
      or_free(c);
      return OR_ERR_ARG;
    }
  } else if (g->mesh != 0) {
    or_free(c);
    return OR_ERR_ARG;
  }
  c->sigc_coef = M_PI * g->d_ref * g->d_ref * pow(4.0 * g->R * g->T_ref, g->omega - 0.5) /
                 tgamma(2.5 - g->omega);
  c->sigc_exp = 2.0 - 2.0 * g->omega;
  c->key[0] = (uint32_t)g->seed;
  c->key[1] = (uint32_t)(g->seed >> 32);
  c->start = (uint32_t*)calloc(c->ncells + 1, sizeof(uint32_t));
  c->smax = (double*)malloc(sizeof(double) * c->ncells);
  c->rem = (double*)calloc((size_t)(c->ncells > 0 ? c->ncells : 1), sizeof(double));
  /* (sigma_T c_r)_max seeded at 2 sigma_T(cbar_r) cbar_r, cbar_r = 4 sqrt(R T0 / pi). */
  double crb = 4.0 * sqrt(g->R * g->sigc_T0 / M_PI);
  double s0 = 2.0 * sigc_fast(c, crb);
  for (int64_t k = 0; k < c->ncells; ++k) c->smax[k] = s0;
  c->samp = (double*)calloc(8 * c->ncells, sizeof(double));
  c->rec = (int64_t*)calloc(4 * c->ncells, sizeof(int64_t));
  if (g->ar_max < 1) g->ar_max = 1;
  if (g->n_surf < 0) g->n_surf = 0;
  c->surf = (double*)calloc(7 * (g->n_surf > 0 ? g->n_surf : 1), sizeof(double));
  *out = c;
  return OR_OK;
}

void or_free(or_ctx* c) {
  if (!c) return;
  free(c->vol); free(c->p); free(c->start); free(c->smax); free(c->rem); free(c->samp);
  free(c->rec); free(c->resamp); free(c->perm); free(c->surf);
  free(c->Lc); free(c->mrad); free(c->mnode); free(c->mrel); free(c->mface);
  free(c);
}

/* Stable counting sort by cell; keys[i] == SENTINEL are dropped. */
static void sort_into_cells(or_ctx* c, part* src, const uint32_t* keys, int64_t M) {
  int64_t nc = c->ncells;
  memset(c->start, 0, sizeof(uint32_t) * (nc + 1));
  for (int64_t i = 0; i < M; ++i)
    if (keys[i] != SENTINEL) c->start[keys[i] + 1] += 1;
  for (int64_t k = 0; k < nc; ++k) c->start[k + 1] += c->start[k];
  int64_t Mn = c->start[nc];
  part* dst = (part*)malloc(sizeof(part) * (Mn ? Mn : 1));
  uint32_t* fill = (uint32_t*)calloc(nc, sizeof(uint32_t));
  free(c->perm);
  c->perm = (uint32_t*)malloc(sizeof(uint32_t) * (Mn ? Mn : 1));
  for (int64_t i = 0; i < M; ++i) {
    uint32_t k = keys[i];
    if (k == SENTINEL) continue;
    int64_t slot = c->start[k] + fill[k]++;
    dst[slot] = src[i];
    c->perm[slot] = (uint32_t)i;
  }
  free(fill);
  free(c->p);
  c->p = dst;
  c->M = Mn;
}

static double min_dtc(const or_ctx* c) {
  double mn = INFINITY;
  for (int64_t k = 0; k < c->ncells; ++k) {
    mom mm;
    int64_t N = c->start[k + 1] - c->start[k];
    moments_of(c, k, c->p + c->start[k], N, &mm);
    if (N >= 2 && mm.dtc < mn) mn = mm.dtc;
  }
  return mn;
}

int or_set_particles(or_ctx* c, const double* pos, const double* vel, int64_t M) {
  const or_config* g = &c->cfg;
  part* src = (part*)calloc(M ? M : 1, sizeof(part));
  uint32_t* keys = (uint32_t*)malloc(sizeof(uint32_t) * (M ? M : 1));
  for (int64_t i = 0; i < M; ++i) {
    for (int d = 0; d < g->dim; ++d) src[i].x[d] = pos[d * M + i];
    for (int d = 0; d < 3; ++d) src[i].v[d] = vel[d * M + i];
    if (g->mesh) {
      int64_t k = mesh_locate(c, src[i].x);
      keys[i] = k < 0 ? SENTINEL : (uint32_t)k;
    } else {
      keys[i] = (uint32_t)cell_of(c, src[i].x);
    }
  }
  sort_into_cells(c, src, keys, M);
  free(src);
  free(keys);
  c->step = 0;
  if (g->dt_fixed > 0) c->dt = g->dt_fixed;
  else {
    double mn = min_dtc(c);
    if (!(mn < INFINITY)) return OR_ERR_ARG;
    c->dt = g->cfl * mn;
  }
  return OR_OK;
}

static void append(part** buf, uint32_t** keys, int64_t* n, int64_t* cap, const part* q, uint32_t key) {
  if (*n == *cap) {
    *cap = *cap ? 2 * *cap : 1024;
    *buf = (part*)realloc(*buf, sizeof(part) * *cap);
    *keys = (uint32_t*)realloc(*keys, sizeof(uint32_t) * *cap);
  }
  (*buf)[*n] = *q;
  (*keys)[*n] = key;
  *n += 1;
}

/* Reservoir injection through the inflow faces, in face order, ghost-cell
 * order, particle order. */
static void inject(or_ctx* c, part** buf, uint32_t** keys, int64_t* n, int64_t* cap) {
  const or_config* g = &c->cfg;
  double dt = c->dt;
  for (int f = 0; f < 6; ++f) {
    int ax = f / 2, side = f % 2;
    if (ax >= g->dim || g->face_bc[f] != OR_BC_INFLOW) continue;
    /* tangential extent of the reservoir: the face's cells, plus the corner
     * blocks beyond every neighbouring face that is itself an inflow face */
    int ta[2], nt = 0, elo[2] = {0, 0}, ntc[2] = {1, 1};
    for (int d = 0; d < g->dim; ++d)
      if (d != ax) ta[nt++] = d;
    int64_t ntan = 1;
    for (int i = 0; i < nt; ++i) {
      int d = ta[i];
      int64_t i0 = g->face_bc[2 * d] == OR_BC_INFLOW ? -(int64_t)g->ghost_layers : 0;
      int64_t i1 = g->n[d] + (g->face_bc[2 * d + 1] == OR_BC_INFLOW ? g->ghost_layers : 0);
      /* a windowed face: only the cells within ghost_layers of its window */
      if (g->win_lo[f][i] < g->win_hi[f][i]) {
        int64_t w0 = (int64_t)floor((g->win_lo[f][i] - g->lo[d]) / c->dl[d]) - g->ghost_layers;
        int64_t w1 = (int64_t)ceil((g->win_hi[f][i] - g->lo[d]) / c->dl[d]) + g->ghost_layers;
        if (w0 > i0) i0 = w0;
        if (w1 < i1) i1 = w1;
        if (i1 < i0) i1 = i0;
      }
      elo[i] = (int)-i0;
      ntc[i] = (int)(i1 - i0);
      ntan *= ntc[i];
    }
    int64_t nghost = ntan * g->ghost_layers;
    double RT = g->R * g->face_T[f];
    double s2RT = sqrt(2.0 * RT);
    double face = side ? g->hi[ax] : g->lo[ax];
    for (int64_t gc = 0; gc < nghost; ++gc) {
      int64_t layer = gc / ntan, t = gc % ntan;
      double blo[3], bhi[3];
      for (int d = 0; d < 3; ++d) { blo[d] = g->lo[d]; bhi[d] = g->hi[d]; }
      int64_t tt = t;
      for (int i = 0; i < nt; ++i) {
        int d = ta[i];
        int64_t id = tt % ntc[i] - elo[i];
        tt /= ntc[i];
        blo[d] = g->lo[d] + (double)id * c->dl[d];
        bhi[d] = g->lo[d] + (double)(id + 1) * c->dl[d];
      }
      if (side == 0) {
        blo[ax] = g->lo[ax] - (double)(layer + 1) * c->dl[ax];
        bhi[ax] = g->lo[ax] - (double)layer * c->dl[ax];
      } else {
        blo[ax] = g->hi[ax] + (double)layer * c->dl[ax];
        bhi[ax] = g->hi[ax] + (double)(layer + 1) * c->dl[ax];
      }
      double Vg = (bhi[0] - blo[0]) * (bhi[1] - blo[1]) * (bhi[2] - blo[2]);
      double lam = g->face_n[f] * Vg / g->Fn;
      uint32_t sb = (uint32_t)f * 16u;
      int64_t ng = (int64_t)floor(lam + uq(c, (uint32_t)gc, SENTINEL, PURP_INJ, sb, 0));
      for (int64_t m = 0; m < ng; ++m) {
        part q;
        memset(&q, 0, sizeof q);
        for (int d = 0; d < g->dim; ++d)
          q.x[d] = blo[d] + uq(c, (uint32_t)gc, (uint32_t)m, PURP_INJ, sb, d) * (bhi[d] - blo[d]);
        double R1 = uq(c, (uint32_t)gc, (uint32_t)m, PURP_INJ, sb, 3);
        double R2 = uq(c, (uint32_t)gc, (uint32_t)m, PURP_INJ, sb, 4);
        double R3 = uq(c, (uint32_t)gc, (uint32_t)m, PURP_INJ, sb, 5);
        double R4 = uq(c, (uint32_t)gc, (uint32_t)m, PURP_INJ, sb, 6);
        double r2 = sqrt(-log(R2)), r4 = sqrt(-log(R4));
        q.v[0] = g->face_u[f][0] + s2RT * cos(2.0 * M_PI * R1) * r2;
        q.v[1] = g->face_u[f][1] + s2RT * cos(2.0 * M_PI * R3) * r4;
        q.v[2] = g->face_u[f][2] + s2RT * sin(2.0 * M_PI * R3) * r4;
        double vn = q.v[ax];
        if (side == 0 ? !(vn > 0) : !(vn < 0)) continue;
        double te = (face - q.x[ax]) / vn;
        if (!(te < dt)) continue;
        int ok = 1;
        for (int i = 0; i < nt; ++i) {
          int d = ta[i];
          double y = q.x[d] + q.v[d] * te;
          if (y < g->lo[d]) {
            if (g->face_bc[2 * d] != OR_BC_SPECULAR) { ok = 0; break; }
            y = 2.0 * g->lo[d] - y;
            q.v[d] = -q.v[d];
          } else if (y > g->hi[d]) {
            if (g->face_bc[2 * d + 1] != OR_BC_SPECULAR) { ok = 0; break; }
            y = 2.0 * g->hi[d] - y;
            q.v[d] = -q.v[d];
          }
          if (y < g->lo[d] || y > g->hi[d]) { ok = 0; break; }
          q.x[d] = y;
        }
        if (!ok) continue;
        q.x[ax] = face;
        if (!face_open(g, f, q.x)) continue; /* blocked by the face's wall part */
        if (move_particle(c, q.x, q.v, dt - te, PURP_INJWALL, (uint32_t)gc, (uint32_t)m,
                          (uint32_t)f << 16))
          continue;
        append(buf, keys, n, cap, &q, (uint32_t)cell_of(c, q.x));
        c->totals[1] += 1;
      }
    }
  }
}

/* Reservoir injection through the outer polygon of the O-grid (face 1 an
 * inflow boundary): ghost_layers rings of reservoir quadrilaterals beyond
 * it, continuing the radial spacing, refilled each step with
 * floor(n V / F_N + u) particles at the face state, uniform in each
 * quadrilateral (its two triangles A B C and A C D chosen by area).  A
 * particle whose straight path enters the outer polygon within the step
 * through one of the ghost_layers + 1 outer edges on either side of its
 * sector (the same truncation as the Cartesian reservoir's depth) enters
 * at the crossing and walks the rest of the step.  Order: layer, sector,
 * particle. */
static void inject_mesh(or_ctx* c, part** buf, uint32_t** keys, int64_t* n, int64_t* cap) {
  const or_config* g = &c->cfg;
  if (g->face_bc[1] != OR_BC_INFLOW) return;
  int nr = c->mnr, nt = c->mnt, nl = c->mnl, w = nl + 1;
  double dt = c->dt, depth = g->hi[2] - g->lo[2];
  double RT = g->R * g->face_T[1];
  double s2RT = sqrt(2.0 * RT);
  uint32_t sb = 1u * 16u;
  for (int64_t gc = 0; gc < (int64_t)nl * nt; ++gc) {
    int L = (int)(gc / nt), j = (int)(gc % nt), i0 = nr + L;
    double a1 = tri_area(mesh_rel(c, i0, j), mesh_rel(c, i0 + 1, j), mesh_rel(c, i0 + 1, j + 1));
    double a2 = tri_area(mesh_rel(c, i0, j), mesh_rel(c, i0 + 1, j + 1), mesh_rel(c, i0, j + 1));
    const double *A = mesh_node(c, i0, j), *B = mesh_node(c, i0 + 1, j);
    const double *C = mesh_node(c, i0 + 1, j + 1), *D = mesh_node(c, i0, j + 1);
    double lam = g->face_n[1] * (a1 + a2) * depth / g->Fn;
    int64_t ng = (int64_t)floor(lam + uq(c, (uint32_t)gc, SENTINEL, PURP_INJ, sb, 0));
    for (int64_t m = 0; m < ng; ++m) {
      part q;
      memset(&q, 0, sizeof q);
      double u0 = uq(c, (uint32_t)gc, (uint32_t)m, PURP_INJ, sb, 0);
      double s = uq(c, (uint32_t)gc, (uint32_t)m, PURP_INJ, sb, 1);
      double t = uq(c, (uint32_t)gc, (uint32_t)m, PURP_INJ, sb, 2);
      if (s + t > 1.0) {
        s = 1.0 - s;
        t = 1.0 - t;
      }
      const double* P1 = B;
      const double* P2 = C;
      if (!(u0 * (a1 + a2) < a1)) {
        P1 = C;
        P2 = D;
      }
      q.x[0] = A[0] + s * (P1[0] - A[0]) + t * (P2[0] - A[0]);
      q.x[1] = A[1] + s * (P1[1] - A[1]) + t * (P2[1] - A[1]);
      double R1 = uq(c, (uint32_t)gc, (uint32_t)m, PURP_INJ, sb, 3);
      double R2 = uq(c, (uint32_t)gc, (uint32_t)m, PURP_INJ, sb, 4);
      double R3 = uq(c, (uint32_t)gc, (uint32_t)m, PURP_INJ, sb, 5);
      double R4 = uq(c, (uint32_t)gc, (uint32_t)m, PURP_INJ, sb, 6);
      double r2 = sqrt(-log(R2)), r4 = sqrt(-log(R4));
      q.v[0] = g->face_u[1][0] + s2RT * cos(2.0 * M_PI * R1) * r2;
      q.v[1] = g->face_u[1][1] + s2RT * cos(2.0 * M_PI * R3) * r4;
      q.v[2] = g->face_u[1][2] + s2RT * sin(2.0 * M_PI * R3) * r4;
      /* first crossing of an outer edge within the step */
      double best = INFINITY;
      int jb = -1;
      for (int o = -w; o <= w; ++o) {
        int jj = ((j + o) % nt + nt) % nt;
        const double* f = c->mface + 12 * ((nr - 1) + (int64_t)nr * jj) + 3;
        double nvv = f[0] * q.v[0] + f[1] * q.v[1];
        if (!(nvv < 0)) continue;
        double sx = f[0] * q.x[0] + f[1] * q.x[1];
        if (!(sx > f[2])) continue;
        double te = (f[2] - sx) / nvv;
        if (!(te < dt) || !(te < best)) continue;
        const double *E0 = mesh_node(c, nr, jj), *E1 = mesh_node(c, nr, jj + 1);
        double ex = E1[0] - E0[0], ey = E1[1] - E0[1];
        double xc = q.x[0] + q.v[0] * te, yc = q.x[1] + q.v[1] * te;
        double u = ((xc - E0[0]) * ex + (yc - E0[1]) * ey) / (ex * ex + ey * ey);
        if (u < 0.0 || u > 1.0) continue;
        best = te;
        jb = jj;
      }
      if (jb < 0) continue;
      q.x[0] += q.v[0] * best;
      q.x[1] += q.v[1] * best;
      int64_t k = (nr - 1) + (int64_t)nr * jb;
      if (mesh_walk(c, &k, q.x, q.v, dt - best, PURP_INJWALL, (uint32_t)gc, (uint32_t)m, 1u << 16, 0))
        continue;
      append(buf, keys, n, cap, &q, (uint32_t)k);
      c->totals[1] += 1;
    }
  }
}

int or_step(or_ctx* c, int nsteps) {
  const or_config* g = &c->cfg;
  for (int it = 0; it < nsteps; ++it) {
    int64_t Mn = c->M;
    double dtG = c->dt;
    double mn = INFINITY;
    free(c->resamp);
    c->resamp = (uint8_t*)calloc(Mn ? Mn : 1, 1);
    c->rec_n = Mn;
    int sample = c->step >= g->n_steady;
    /* Steps 3-5 per cell.  Cells are independent (every draw is keyed by
     * the cell, each cell writes only its own slots and records), so with
     * nthreads > 1 they are spread over threads with results identical to
     * the sequential loop (the minimum is exact in any order). */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) reduction(min : mn) num_threads(c->nthreads > 0 ? c->nthreads : 1)
#endif
    for (int64_t k = 0; k < c->ncells; ++k) {
      int64_t s0 = c->start[k], N = c->start[k + 1] - s0;
      int64_t soff[9];
      const int64_t* so = NULL;
      if (g->subcells > 1) {
        order_by_subcell(c, k, c->p + s0, N, soff);
        so = soff;
      }
      mom mm;
      moments_of(c, k, c->p + s0, N, &mm);
      if (N >= 2 && mm.dtc < mn) mn = mm.dtc;
      int64_t rec[4];
      collide_cell(c, k, c->vol[k], c->p + s0, N, &mm, dtG, &c->smax[k], &c->rem[k], rec, c->resamp + s0, so);
      for (int i = 0; i < 4; ++i) c->rec[i * c->ncells + k] = rec[i];
      if (sample) {
        double* S = c->samp;
        int64_t nc = c->ncells;
        double sv[3] = {0, 0, 0}, sq[3] = {0, 0, 0};
        for (int64_t i = 0; i < N; ++i)
          for (int d = 0; d < 3; ++d) {
            sv[d] += c->p[s0 + i].v[d];
            sq[d] += c->p[s0 + i].v[d] * c->p[s0 + i].v[d];
          }
        S[0 * nc + k] += (double)N;
        for (int d = 0; d < 3; ++d) {
          S[(1 + d) * nc + k] += sv[d];
          S[(4 + d) * nc + k] += sq[d];
        }
        S[7 * nc + k] += ratio_of(g, &mm);
      }
    }
    if (sample) {
      c->nsamp += 1;
      c->surf_time += dtG;
    }
    c->sampling_now = sample;
    /* Step 2 of the next interval: move, remove, inject. */
    int64_t cap = Mn + 1024, n = 0;
    part* buf = (part*)malloc(sizeof(part) * cap);
    uint32_t* keys = (uint32_t*)malloc(sizeof(uint32_t) * cap);
    for (int64_t k = 0; k < c->ncells; ++k) {
      int64_t s0 = c->start[k], N = c->start[k + 1] - s0;
      for (int64_t s = 0; s < N; ++s) {
        part q = c->p[s0 + s];
        int gone;
        uint32_t key;
        if (g->mesh) {
          int64_t k2 = k;
          gone = mesh_walk(c, &k2, q.x, q.v, dtG, PURP_WALL, (uint32_t)k, (uint32_t)s, 0, 0);
          key = gone ? SENTINEL : (uint32_t)k2;
        } else {
          gone = move_particle(c, q.x, q.v, dtG, PURP_WALL, (uint32_t)k, (uint32_t)s, 0);
          key = gone ? SENTINEL : (uint32_t)cell_of(c, q.x);
        }
        if (gone) c->totals[0] += 1;
        append(&buf, &keys, &n, &cap, &q, key);
      }
    }
    if (g->mesh)
      inject_mesh(c, &buf, &keys, &n, &cap);
    else
      inject(c, &buf, &keys, &n, &cap);
    sort_into_cells(c, buf, keys, n);
    free(buf);
    free(keys);
    if (g->dt_fixed > 0) c->dt = g->dt_fixed;
    else if (mn < INFINITY) c->dt = g->cfl * mn;
    c->step += 1;
  }
  return OR_OK;
}

int64_t or_num_particles(const or_ctx* c) { return c->M; }
double or_dt(const or_ctx* c) { return c->dt; }
int64_t or_step_index(const or_ctx* c) { return c->step; }

int or_get_particles(const or_ctx* c, double* pos, double* vel, uint32_t* cell) {
  int64_t M = c->M;
  for (int64_t k = 0; k < c->ncells; ++k)
    for (uint32_t i = c->start[k]; i < c->start[k + 1]; ++i) {
      if (pos) for (int d = 0; d < c->cfg.dim; ++d) pos[d * M + i] = c->p[i].x[d];
      if (vel) for (int d = 0; d < 3; ++d) vel[d * M + i] = c->p[i].v[d];
      if (cell) cell[i] = (uint32_t)k;
    }
  return OR_OK;
}

int or_moments(const or_ctx* c, int kind, double* out, int nfields) {
  const or_config* g = &c->cfg;
  int64_t nc = c->ncells;
  if (nfields > OR_NFIELDS) nfields = OR_NFIELDS;
  for (int64_t k = 0; k < nc; ++k) {
    double f[OR_NFIELDS];
    memset(f, 0, sizeof f);
    if (kind == 0) {
      mom mm;
      int64_t N = c->start[k + 1] - c->start[k];
      moments_of(c, k, c->p + c->start[k], N, &mm);
      f[OR_F_N] = (double)N; f[OR_F_n] = mm.n;
      f[OR_F_ux] = mm.U[0]; f[OR_F_uy] = mm.U[1]; f[OR_F_uz] = mm.U[2];
      f[OR_F_T] = mm.T; f[OR_F_qx] = mm.q[0]; f[OR_F_qy] = mm.q[1]; f[OR_F_qz] = mm.q[2];
      f[OR_F_tau] = mm.tau; f[OR_F_dtc] = mm.dtc; f[OR_F_ratio] = ratio_of(g, &mm);
    } else {
      const double* S = c->samp;
      double sN = S[k];
      if (c->nsamp > 0) {
        f[OR_F_N] = sN / (double)c->nsamp;
        f[OR_F_n] = c->vol[k] > 0 ? f[OR_F_N] * g->Fn / c->vol[k] : 0.0;
        f[OR_F_ratio] = S[7 * nc + k] / (double)c->nsamp;
      }
      if (sN > 0) {
        double U[3], e = 0;
        for (int d = 0; d < 3; ++d) {
          U[d] = S[(1 + d) * nc + k] / sN;
          e += S[(4 + d) * nc + k] / sN - U[d] * U[d];
        }
        f[OR_F_ux] = U[0]; f[OR_F_uy] = U[1]; f[OR_F_uz] = U[2];
        f[OR_F_T] = e / (3.0 * g->R);
      }
    }
    for (int i = 0; i < nfields; ++i) out[(int64_t)i * nc + k] = f[i];
  }
  return OR_OK;
}

int or_get_step_record(const or_ctx* c, int64_t* cell4, uint8_t* resampled, uint32_t* perm,
                       int64_t* n_old) {
  if (cell4) memcpy(cell4, c->rec, sizeof(int64_t) * 4 * c->ncells);
  if (resampled && c->resamp) memcpy(resampled, c->resamp, c->rec_n);
  if (perm && c->perm) memcpy(perm, c->perm, sizeof(uint32_t) * c->M);
  if (n_old) *n_old = c->rec_n;
  return OR_OK;
}

int or_get_cell_start(const or_ctx* c, uint32_t* start) {
  memcpy(start, c->start, sizeof(uint32_t) * (c->ncells + 1));
  return OR_OK;
}
int or_get_sigc_max(const or_ctx* c, double* out) {
  memcpy(out, c->smax, sizeof(double) * c->ncells);
  return OR_OK;
}
int or_get_sample(const or_ctx* c, double* out, int64_t* nsamp) {
  memcpy(out, c->samp, sizeof(double) * 8 * c->ncells);
  if (nsamp) *nsamp = c->nsamp;
  return OR_OK;
}
int or_get_surface(const or_ctx* c, double* out, double* time) {
  int ns = c->cfg.n_surf;
  if (out && ns > 0) memcpy(out, c->surf, sizeof(double) * 7 * ns);
  if (time) *time = c->surf_time;
  return OR_OK;
}

int or_set_threads(or_ctx* c, int n) {
  if (!c || n < 1) return OR_ERR_ARG;
#ifdef _OPENMP
  c->nthreads = n;
#else
  c->nthreads = 1;
#endif
  return OR_OK;
}

int or_get_threads(const or_ctx* c) { return c ? c->nthreads : 0; }

int or_select_pair(int64_t N, const int64_t* soff, double u1, double u2, int64_t* i, int64_t* j) {
  if (N < 2 || !i || !j) return OR_ERR_ARG;
  select_pair(N, soff, u1, u2, i, j);
  return OR_OK;
}

int or_subcell_order(const or_config* cfg, int64_t cell, const double* pos, int64_t N, int64_t* order,
                     int64_t* soff) {
  or_ctx* c;
  if (or_init(cfg, &c) != OR_OK || cfg->subcells < 2) return OR_ERR_ARG;
  part* ps = (part*)calloc(N ? N : 1, sizeof(part));
  for (int64_t i = 0; i < N; ++i) {
    for (int d = 0; d < cfg->dim; ++d) ps[i].x[d] = pos[d * N + i];
    ps[i].v[0] = (double)i; /* carries the input index through the reorder */
  }
  order_by_subcell(c, cell, ps, N, soff);
  for (int64_t i = 0; i < N; ++i) order[i] = (int64_t)ps[i].v[0];
  free(ps);
  or_free(c);
  return OR_OK;
}

int or_get_totals(const or_ctx* c, int64_t* out4) {
  memcpy(out4, c->totals, sizeof c->totals);
  return OR_OK;
}

/* Homogeneous collision step on one cell (no transport), for the pin tests. */
int or_collide_cell(const or_config* cfg, int64_t step, uint32_t cell, double volume, double dt_G,
                    double* sigc_max, double* vel, int64_t N, int64_t rec[4], uint8_t* resampled) {
  or_config g = *cfg;
  g.dim = 1; g.n[0] = g.n[1] = g.n[2] = 1;
  g.lo[0] = g.lo[1] = g.lo[2] = 0; g.hi[0] = g.hi[1] = g.hi[2] = 1;
  g.cell_volume = NULL; g.body = OR_BODY_NONE;
  or_ctx* c;
  if (or_init(&g, &c) != OR_OK) return OR_ERR_ARG;
  c->vol[0] = volume;
  c->step = step;
  part* ps = (part*)calloc(N ? N : 1, sizeof(part));
  for (int64_t i = 0; i < N; ++i)
    for (int d = 0; d < 3; ++d) ps[i].v[d] = vel[d * N + i];
  mom mm;
  /* the homogeneous cell uses its own volume and index for the draw stream */
  moments_of(c, 0, ps, N, &mm);
  double rem = 0.0;
  collide_cell(c, (int64_t)cell, volume, ps, N, &mm, dt_G, sigc_max, &rem, rec, resampled, NULL);
  for (int64_t i = 0; i < N; ++i)
    for (int d = 0; d < 3; ++d) vel[d * N + i] = ps[i].v[d];
  free(ps);
  or_free(c);
  return OR_OK;
}

int or_mesh_locate(const or_ctx* c, const double* pos, int64_t n, int64_t* cell) {
  if (!c || c->cfg.mesh != 1 || n < 0) return OR_ERR_ARG;
  for (int64_t i = 0; i < n; ++i) {
    double x[2] = {pos[i], pos[n + i]};
    cell[i] = mesh_locate(c, x);
  }
  return OR_OK;
}

int or_mesh_geometry(const or_ctx* c, double* nodes, double* faces, double* L) {
  if (!c || c->cfg.mesh != 1) return OR_ERR_ARG;
  int64_t nn = (int64_t)(c->mnr + c->mnl + 1) * c->mnt;
  if (nodes) memcpy(nodes, c->mnode, sizeof(double) * 2 * nn);
  if (faces) memcpy(faces, c->mface, sizeof(double) * 12 * c->ncells);
  if (L) memcpy(L, c->Lc, sizeof(double) * c->ncells);
  return OR_OK;
}

int or_get_volumes(const or_ctx* c, double* vol) {
  if (!c) return OR_ERR_ARG;
  memcpy(vol, c->vol, sizeof(double) * c->ncells);
  return OR_OK;
}
