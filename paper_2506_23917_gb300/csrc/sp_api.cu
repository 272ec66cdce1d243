// sp_api.cu -- host driver and C ABI of libsp (see include/sp.h).
//
// Per step the driver enqueues, on the context's stream:
//   1. k_plan + k_collide (batches of cells per warp) and its
//      big-cell launch (one warp per cell with a large staging area):
//      gather through perm in stable order -> Step 3 moments -> Step 4
//      DSMC / Shakhov / rescale -> Step 5 sums -> Step 2 free flight of the
//      next interval, new key and histogram;
//   2. reservoir injection at inflow faces (count, scan, write);
//   3. exclusive scan of the histogram -> cell offsets of the new state;
//   4. bookkeeping (particle count, Delta t of the next step, step index);
//   5. scatter of source indices into the new cell order (the histogram is
//      the cursor and ends at zero, ready for the next step).
// The sequence is captured once per buffer parity as a CUDA graph and
// replayed by sp_step().
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/sp.h"
#include "sp_internal.h"

namespace sp {
// Sort each cell's perm segment ascending (sp_noalloc.cu).
void launch_order_cells(const uint32_t* start, int64_t ncells, uint32_t* perm, cudaStream_t s);
}  // namespace sp

using namespace sp;

namespace {
constexpr double kPiHost = 3.14159265358979323846;
// Blocks of the big-cell launches (one warp per cell up to kHugeCell
// particles; one block per larger cell), persistent over the big-cell list.
constexpr int kBigGridPerSm = 2;
}  // namespace

struct sp_ctx {
  int n_inst = 0, dim = 0, prec = 0;
  size_t tsize = 8;
  const KernelSet* K = nullptr;  // the kernels of this precision mode
  std::vector<InstParams> hP;
  std::vector<sp_config> cfg;
  InstParams* dP = nullptr;
  int64_t NC = 0, cap = 0;
  // device buffers
  void* pos[2][3] = {{nullptr}};
  void* vel[2][3] = {{nullptr}};
  uint32_t *key = nullptr, *perm = nullptr, *count = nullptr, *start = nullptr;
  uint32_t *cell_inst = nullptr, *scan_part = nullptr, *big_list = nullptr, *big_count = nullptr;
  uint32_t* ticket = nullptr;
  uint2* batches = nullptr;
  uint32_t* nbatch = nullptr;         // [kBatchClasses] batches of the plan per class
  uint8_t* cost = nullptr;            // [NC] cost bytes of the last step (batch plan)
  unsigned long long* cyc = nullptr;  // [3] batch-cycle sum, particle sum, cost unit per particle
  int collide_grid = 1;
  int nsm = 1;
  int sched_cap = kCapSmall, sched_warps = kWarpsDefault;
  int stable = 1;
  double* surf = nullptr;       // [elements][kSurfFields] wall tallies
  double* surf_time = nullptr;  // [n_inst] sampled time
  int64_t n_surf_tot = 0;
  double *vol = nullptr, *smax = nullptr, *samp = nullptr;
  double *ivol = nullptr, *rcp = nullptr;  // 1 / vol per cell; 1 / k for k <= kHugeCell
  double* rem = nullptr;  // [NC] carried NTC remainders
  double* mom = nullptr;  // [SP_NFIELDS][largest instance] output of sp_moments kind 0
  double* msum = nullptr; // [7][NC] scratch of the moments kernels
  int64_t mom_cells = 0;
  int32_t* rec = nullptr;
  double* cons = nullptr;  // [6][NC] rescale conservation record
  uint8_t* resamp = nullptr;
  double* dt_cur = nullptr;
  unsigned long long* dt_min = nullptr;
  uint32_t *step_d = nullptr, *Mcur = nullptr, *Mtot = nullptr;
  unsigned long long* err = nullptr;
  GhostCell* ghosts = nullptr;
  int64_t n_ghost = 0;
  uint32_t *gcount = nullptr, *goff = nullptr, *gscan_part = nullptr;
  cudaStream_t stream = nullptr;
  int cur = 0;
  int64_t step_host = 0;
  bool uploaded = false, dirty = false, record = false;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t pgraph[2] = {nullptr, nullptr};  // the same steps with timing events
  cudaEvent_t pev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  bool graph_ok = false;
  cudaStream_t side = nullptr;       // capture-time branches of the step graph (injection,
  cudaStream_t side2 = nullptr;      // big-cell launch, huge-cell launch)
  cudaStream_t side3 = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr, fork2_ev = nullptr, join2_ev = nullptr;
  cudaEvent_t fork3_ev = nullptr, join3_ev = nullptr;
  int launches = 0;
  std::vector<double*> dstage;    // per instance: FP64 [dim][n] then [3][n], device
  std::vector<int64_t> stage_n, stage_cap;
  std::vector<int> stage_f32;     // per instance: the staged data is FP32
  uint32_t* part_inst = nullptr;  // [cap] instance of each uploaded particle
  std::vector<uint32_t> prev_start;  // [NC+1] of the state before the last step (record mode)
  std::vector<unsigned long long> hinf, hmin;  // host mirrors used by upload()
  std::vector<double> hdt;
  uint32_t hM = 0;
  // body-fitted O-grid instances (all instances share the mesh kind)
  int mesh = 0;
  double *Lc = nullptr, *iLc = nullptr, *mrad = nullptr;  // [NC], [NC], radii
  void *mface = nullptr, *mnode = nullptr;                 // state type
};

namespace {

sp_status cuda_fail(cudaError_t e) {
  if (e == cudaSuccess) return SP_OK;
  fprintf(stderr, "libsp: CUDA error %s\n", cudaGetErrorString(e));
  return SP_ERR_CUDA;
}
#define CK(x)                                     \
  do {                                            \
    cudaError_t e_ = (x);                         \
    if (e_ != cudaSuccess) return cuda_fail(e_);  \
  } while (0)

template <class P>
cudaError_t dalloc(P** p, size_t bytes) {
  return cudaMalloc((void**)p, bytes ? bytes : 16);
}

void fill_params(const sp_config& c, InstParams* P, int64_t cell_off) {
  memset(P, 0, sizeof *P);
  P->dim = c.dim;
  for (int d = 0; d < 3; ++d) {
    P->n[d] = d < c.dim ? c.n[d] : 1;
    P->lo[d] = c.lo[d];
    P->hi[d] = c.hi[d];
    P->dl[d] = (c.hi[d] - c.lo[d]) / (double)P->n[d];
    P->inv_d[d] = (double)P->n[d] / (c.hi[d] - c.lo[d]);
  }
  P->Lmin = INFINITY;
  for (int d = 0; d < c.dim; ++d) P->Lmin = std::min(P->Lmin, P->dl[d]);
  P->m = c.m;
  P->R = c.R;
  P->gamma = c.gamma;
  P->Pr = c.Pr;
  P->omega = c.omega;
  P->T_ref = c.T_ref;
  P->mu_ref = c.mu_ref;
  P->Fn = c.Fn;
  P->cfl = c.cfl;
  P->dt_fixed = c.dt_fixed;
  // VHS (Bird): sigma_T c_r = pi d^2 (4 R T_ref)^(w - 1/2) / Gamma(5/2 - w) c_r^(2 - 2w)
  P->sigc_coef = kPiHost * c.d_ref * c.d_ref * pow(4.0 * c.R * c.T_ref, c.omega - 0.5) /
                 tgamma(2.5 - c.omega);
  P->sigc_exp = 2.0 - 2.0 * c.omega;
  for (int f = 0; f < 6; ++f) {
    P->face_bc[f] = c.face_bc[f];
    P->face_T[f] = c.face_T[f];
  }
  P->body = c.body;
  for (int d = 0; d < 3; ++d) P->body_c[d] = c.body_c[d];
  P->body_r = c.body_r;
  P->body_Tw = c.body_Tw;
  P->n_steady = c.n_steady;
  P->key0 = (uint32_t)c.seed;
  P->key1 = (uint32_t)(c.seed >> 32);
  P->mode = c.mode;
  P->ar_max = c.ar_max < 1 ? 1 : c.ar_max;
  P->ntc_carry = c.ntc_carry ? 1 : 0;
  P->subcells = c.subcells > 1 ? c.subcells : 1;
  P->nsub = 1;
  for (int d = 0; d < c.dim; ++d) P->nsub *= P->subcells;
  P->cell_off = cell_off;
  P->ncells = (int64_t)P->n[0] * P->n[1] * P->n[2];
  P->n_surf = (c.body != SP_BODY_NONE && c.n_surf > 0) ? c.n_surf : 0;
  P->FnM = c.Fn * c.m;
  P->inv3R = 1.0 / (3.0 * c.R);
  P->sqrt_gamma = sqrt(c.gamma);
  P->tau_k = c.mu_ref * pow(c.T_ref, -c.omega) / (c.m * c.R);
  P->inv_tau_k = 1.0 / P->tau_k;
  P->omf = (float)(1.0 - c.omega);
  P->inv_Lmin = 1.0 / P->Lmin;
  P->inv_Fn = 1.0 / c.Fn;
  for (int d = 0; d < 3; ++d) {
    P->g64.lo[d] = P->lo[d];
    P->g64.hi[d] = P->hi[d];
    P->g64.inv_d[d] = P->inv_d[d];
    P->g64.body_c[d] = P->body_c[d];
  }
  P->g64.body_r = P->body_r;
  for (int d = 0; d < 3; ++d) {
    const double span = fabs(P->hi[d]) + fabs(P->lo[d]) + (P->hi[d] - P->lo[d]);
    P->g64.eps[d] = 1e-12 * span;
    P->g32.eps[d] = (float)(1e-5 * span);
  }
  for (int f = 0; f < 6; ++f) P->g64.face_RT[f] = c.R * c.face_T[f];
  P->g64.body_RT = c.R * c.body_Tw;
  P->g64.sigc_coef = P->sigc_coef;
  P->g64.sigc_exp = P->sigc_exp;
  for (int d = 0; d < 3; ++d) {
    P->g32.lo[d] = (float)P->g64.lo[d];
    P->g32.hi[d] = (float)P->g64.hi[d];
    P->g32.inv_d[d] = (float)P->g64.inv_d[d];
    P->g32.body_c[d] = (float)P->g64.body_c[d];
  }
  P->g32.body_r = (float)P->g64.body_r;
  for (int f = 0; f < 6; ++f) P->g32.face_RT[f] = (float)P->g64.face_RT[f];
  P->g32.body_RT = (float)P->g64.body_RT;
  P->g32.sigc_coef = (float)P->sigc_coef;
  P->g32.sigc_exp = (float)P->sigc_exp;
  P->face_win = 0;
  for (int f = 0; f < 6; ++f)
    for (int i = 0; i < 2; ++i) {
      P->g64.win_lo[f][i] = c.win_lo[f][i];
      P->g64.win_hi[f][i] = c.win_hi[f][i];
      P->g32.win_lo[f][i] = (float)c.win_lo[f][i];
      P->g32.win_hi[f][i] = (float)c.win_hi[f][i];
      if (i < c.dim - 1 && c.win_lo[f][i] < c.win_hi[f][i]) P->face_win |= 1 << f;
    }
}

bool valid(const sp_config& c, int dim) {
  if (c.dim != dim || c.dim < 1 || c.dim > 3) return false;
  for (int d = 0; d < 3; ++d) {
    if (d < c.dim && c.n[d] < 1) return false;
    if (!(c.hi[d] > c.lo[d])) return false;
  }
  if (!(c.R > 0) || !(c.m > 0) || !(c.Fn > 0) || !(c.mu_ref > 0) || !(c.T_ref > 0)) return false;
  if (c.body == SP_BODY_CIRCLE && c.dim != 2) return false;
  if (c.subcells > 1) {
    int64_t m = 1;
    for (int d = 0; d < c.dim; ++d) m *= c.subcells;
    if (m > kMaxSub) return false;
  }
  if (c.body == SP_BODY_SPHERE && c.dim != 3) return false;
  if (c.mesh != 0) {
    if (c.mesh != 1 || c.dim != 2 || c.body != SP_BODY_CIRCLE || c.n[1] < 3 || !(c.body_r > 0) ||
        !(c.mesh_r_out > c.body_r) || !(c.mesh_growth > 0) || c.subcells > 1)
      return false;
  }
  return true;
}

// Body-fitted O-grid of one instance (sp_config.mesh = 1): node radii r_0 =
// body_r, r_{i+1} = r_i + dr_i, dr_{i+1} = q dr_i with the first n[0]
// spacings summing to r_out - r_0, continued over the reservoir rings;
// nodes at angles 2 pi j / n[1]; per cell k = i + n[0] j (corners A =
// (i, j), B = (i+1, j), C = (i+1, j+1), D = (i, j+1), counter-clockwise)
// the four face lines inner D->A, outer B->C, theta_j A->B, theta_j+1
// C->D as unit outward normal and offset, the shortest edge L and the area
// (shoelace on coordinates about the centre) times the depth.
struct MeshHost {
  std::vector<double> rad;    // [nr + nl + 1]
  std::vector<double> node;   // [(nr + nl + 1) nt][2]
  std::vector<double> rel;    // the same about the centre
  std::vector<double> face;   // [ncells][12]
  std::vector<double> L, vol; // [ncells]
};

double edge_line(const double* p, const double* q, double* f) {
  const double tx = q[0] - p[0], ty = q[1] - p[1];
  const double len = sqrt(tx * tx + ty * ty);
  f[0] = ty / len;
  f[1] = -tx / len;
  f[2] = f[0] * p[0] + f[1] * p[1];
  return len;
}

double quad_area(const double* p0, const double* p1, const double* p2, const double* p3) {
  return 0.5 * ((p0[0] * p1[1] - p1[0] * p0[1]) + (p1[0] * p2[1] - p2[0] * p1[1]) +
                (p2[0] * p3[1] - p3[0] * p2[1]) + (p3[0] * p0[1] - p0[0] * p3[1]));
}

double tri_area(const double* p0, const double* p1, const double* p2) {
  return 0.5 * ((p1[0] - p0[0]) * (p2[1] - p0[1]) - (p2[0] - p0[0]) * (p1[1] - p0[1]));
}

void build_mesh(const sp_config& c, MeshHost& m) {
  const int nr = c.n[0], nt = c.n[1], nl = c.ghost_layers > 0 ? c.ghost_layers : 0;
  const int nrad = nr + nl + 1;
  m.rad.assign(nrad, 0.0);
  double q = c.mesh_growth, geo = 0.0, qp = 1.0;
  for (int i = 0; i < nr; ++i) {
    geo += qp;
    qp *= q;
  }
  double dr = (c.mesh_r_out - c.body_r) / geo;
  m.rad[0] = c.body_r;
  for (int i = 0; i + 1 < nrad; ++i) {
    m.rad[i + 1] = m.rad[i] + dr;
    dr *= q;
  }
  m.node.assign(2 * (size_t)nrad * nt, 0.0);
  m.rel.assign(2 * (size_t)nrad * nt, 0.0);
  const double two_pi = 2.0 * 3.14159265358979323846;
  for (int i = 0; i < nrad; ++i)
    for (int j = 0; j < nt; ++j) {
      const double th = two_pi * (double)j / (double)nt;
      const double rx = m.rad[i] * cos(th), ry = m.rad[i] * sin(th);
      const size_t o = 2 * ((size_t)i * nt + j);
      m.rel[o] = rx;
      m.rel[o + 1] = ry;
      m.node[o] = c.body_c[0] + rx;
      m.node[o + 1] = c.body_c[1] + ry;
    }
  auto nd = [&](const std::vector<double>& v, int i, int j) { return &v[2 * ((size_t)i * nt + j % nt)]; };
  const int64_t ncell = (int64_t)nr * nt;
  m.face.assign(12 * (size_t)ncell, 0.0);
  m.L.assign(ncell, 0.0);
  m.vol.assign(ncell, 0.0);
  const double depth = c.hi[2] - c.lo[2];
  for (int j = 0; j < nt; ++j)
    for (int i = 0; i < nr; ++i) {
      const int64_t k = i + (int64_t)nr * j;
      const double *A = nd(m.node, i, j), *B = nd(m.node, i + 1, j);
      const double *C = nd(m.node, i + 1, j + 1), *D = nd(m.node, i, j + 1);
      double* f = &m.face[12 * (size_t)k];
      const double l0 = edge_line(D, A, f + 0);
      const double l1 = edge_line(B, C, f + 3);
      const double l2 = edge_line(A, B, f + 6);
      const double l3 = edge_line(C, D, f + 9);
      double L = l0;
      if (l1 < L) L = l1;
      if (l2 < L) L = l2;
      if (l3 < L) L = l3;
      m.L[k] = L;
      m.vol[k] = quad_area(nd(m.rel, i, j), nd(m.rel, i + 1, j), nd(m.rel, i + 1, j + 1),
                           nd(m.rel, i, j + 1)) * depth;
    }
}

// Reservoir quadrilaterals of an O-grid inflow boundary, in (ring, sector)
// order: expected count n V / F_N with V the area times the depth.
void build_ghosts_mesh(const sp_config& c, const MeshHost& m, int inst, std::vector<GhostCell>& out) {
  if (c.face_bc[1] != SP_BC_INFLOW) return;
  const int nr = c.n[0], nt = c.n[1], nl = c.ghost_layers > 0 ? c.ghost_layers : 0;
  const double depth = c.hi[2] - c.lo[2];
  const double s2RT = sqrt(2.0 * (c.R * c.face_T[1]));
  auto rl = [&](int i, int j) { return &m.rel[2 * ((size_t)i * nt + j % nt)]; };
  for (int64_t gc = 0; gc < (int64_t)nl * nt; ++gc) {
    GhostCell G;
    memset(&G, 0, sizeof G);
    G.inst = inst;
    G.face = 1;
    G.gc = (uint32_t)gc;
    G.mlay = (int)(gc / nt);
    G.msec = (int)(gc % nt);
    const int i0 = nr + G.mlay, j = G.msec;
    G.a1 = tri_area(rl(i0, j), rl(i0 + 1, j), rl(i0 + 1, j + 1));
    G.a2 = tri_area(rl(i0, j), rl(i0 + 1, j + 1), rl(i0, j + 1));
    G.lam = c.face_n[1] * (G.a1 + G.a2) * depth / c.Fn;
    G.s2RT = s2RT;
    for (int d = 0; d < 3; ++d) G.u[d] = c.face_u[1][d];
    out.push_back(G);
  }
}

// Reservoir cells in (face, layer-major, tangential) order with the same
// arithmetic as the reference definition of their boxes.
void build_ghosts(const sp_config& c, const InstParams& P, int inst, std::vector<GhostCell>& out) {
  for (int f = 0; f < 6; ++f) {
    const int ax = f / 2, side = f % 2;
    if (ax >= c.dim || c.face_bc[f] != SP_BC_INFLOW) continue;
    // tangential cells: the face's own, plus the corner blocks beyond each
    // neighbouring inflow face (a particle is kept by the face it crosses)
    int ta[2], nt = 0, elo[2] = {0, 0}, ntc[2] = {1, 1};
    for (int d = 0; d < c.dim; ++d)
      if (d != ax) ta[nt++] = d;
    int64_t ntan = 1;
    for (int i = 0; i < nt; ++i) {
      const int d = ta[i];
      int64_t i0 = c.face_bc[2 * d] == SP_BC_INFLOW ? -(int64_t)c.ghost_layers : 0;
      int64_t i1 = P.n[d] + (c.face_bc[2 * d + 1] == SP_BC_INFLOW ? c.ghost_layers : 0);
      if (c.win_lo[f][i] < c.win_hi[f][i]) {  // windowed face: near the window only
        const int64_t w0 = (int64_t)floor((c.win_lo[f][i] - c.lo[d]) / P.dl[d]) - c.ghost_layers;
        const int64_t w1 = (int64_t)ceil((c.win_hi[f][i] - c.lo[d]) / P.dl[d]) + c.ghost_layers;
        i0 = std::max(i0, w0);
        i1 = std::min(i1, w1);
        if (i1 < i0) i1 = i0;
      }
      elo[i] = (int)-i0;
      ntc[i] = (int)(i1 - i0);
      ntan *= ntc[i];
    }
    const int64_t ng = ntan * c.ghost_layers;
    const double RT = c.R * c.face_T[f];
    const double s2RT = sqrt(2.0 * RT);
    for (int64_t gc = 0; gc < ng; ++gc) {
      const int64_t layer = gc / ntan, t = gc % ntan;
      GhostCell G;
      memset(&G, 0, sizeof G);
      G.inst = inst;
      G.face = f;
      G.gc = (uint32_t)gc;
      for (int d = 0; d < 3; ++d) {
        G.blo[d] = c.lo[d];
        G.bhi[d] = c.hi[d];
      }
      int64_t tt = t;
      for (int i = 0; i < nt; ++i) {
        const int d = ta[i];
        const int64_t id = tt % ntc[i] - elo[i];
        tt /= ntc[i];
        G.blo[d] = c.lo[d] + (double)id * P.dl[d];
        G.bhi[d] = c.lo[d] + (double)(id + 1) * P.dl[d];
      }
      if (side == 0) {
        G.blo[ax] = c.lo[ax] - (double)(layer + 1) * P.dl[ax];
        G.bhi[ax] = c.lo[ax] - (double)layer * P.dl[ax];
      } else {
        G.blo[ax] = c.hi[ax] + (double)layer * P.dl[ax];
        G.bhi[ax] = c.hi[ax] + (double)(layer + 1) * P.dl[ax];
      }
      const double Vg = (G.bhi[0] - G.blo[0]) * (G.bhi[1] - G.blo[1]) * (G.bhi[2] - G.blo[2]);
      G.lam = c.face_n[f] * Vg / c.Fn;
      G.s2RT = s2RT;
      for (int d = 0; d < 3; ++d) G.u[d] = c.face_u[f][d];
      out.push_back(G);
    }
  }
}

StepArgs make_step_args(sp_ctx* c, int par) {
  StepArgs a;
  memset(&a, 0, sizeof a);
  for (int d = 0; d < 3; ++d) {
    a.Apos[d] = c->pos[par][d];
    a.Bpos[d] = c->pos[1 - par][d];
    a.Avel[d] = c->vel[par][d];
    a.Bvel[d] = c->vel[1 - par][d];
  }
  a.key = c->key;
  a.perm = c->perm;
  a.start = c->start;
  a.count = c->count;
  a.cell_inst = c->cell_inst;
  a.vol = c->vol;
  a.ivol = c->ivol;
  a.rcp = c->rcp;
  a.smax = c->smax;
  a.rem = c->rem;
  a.samp = c->samp;
  a.rec = c->record ? c->rec : nullptr;
  a.cons = c->record ? c->cons : nullptr;
  a.resamp = c->record ? c->resamp : nullptr;
  a.P = c->dP;
  a.dt_cur = c->dt_cur;
  a.dt_min = c->dt_min;
  a.step = c->step_d;
  a.big_list = c->big_list;
  a.big_count = c->big_count;
  a.ticket = c->ticket;
  a.batches = c->batches;
  a.nbatch = c->nbatch;
  a.cost = c->cost;
  a.cyc = c->cyc;
  a.err = c->err;
  a.NC = c->NC;
  a.mesh = c->mesh;
  a.Lc = c->Lc;
  a.iLc = c->iLc;
  a.mface = c->mface;
  a.mnode = c->mnode;
  a.mrad = c->mrad;
  a.msum = c->msum;
  a.cap = c->cap;
  a.big_cap = kHugeCell;
  a.cap_small = c->sched_cap;
  a.stable = c->stable;
  a.surf = c->n_surf_tot > 0 ? c->surf : nullptr;
  a.one = c->n_inst == 1 ? 1 : 0;
  a.P0 = c->hP[0];
  return a;
}

InjectArgs make_inject_args(sp_ctx* c, int par) {
  InjectArgs a;
  memset(&a, 0, sizeof a);
  a.ghosts = c->ghosts;
  a.n_ghost = c->n_ghost;
  a.gcount = c->gcount;
  a.goff = c->goff;
  for (int d = 0; d < 3; ++d) {
    a.Bpos[d] = c->pos[1 - par][d];
    a.Bvel[d] = c->vel[1 - par][d];
  }
  a.key = c->key;
  a.count = c->count;
  a.P = c->dP;
  a.dt_cur = c->dt_cur;
  a.step = c->step_d;
  a.Mcur = c->Mcur;
  a.err = c->err;
  a.cap = c->cap;
  a.surf = c->n_surf_tot > 0 ? c->surf : nullptr;
  a.mface = c->mface;
  a.mnode = c->mnode;
  return a;
}

// Persistent launch: enough blocks to fill every SM, never more than one
// warp per possible batch.
int small_grid(const sp_ctx* c) {
  const int64_t need = (c->NC + c->sched_warps - 1) / c->sched_warps;
  return (int)std::max<int64_t>(1, std::min<int64_t>(need, c->collide_grid));
}

void launch_collide_p(sp_ctx* c, const StepArgs& a, bool big, int grid, cudaStream_t s) {
  const int warps = big ? 1 : c->sched_warps;
  c->K->collide(c->dim, a, big, grid, warps, s);
}

// Collision-kernel schedule: staging capacity per warp and warps per block.
// Returns false if it does not fit the shared memory or the block limits.
bool apply_schedule(sp_ctx* c, int cap, int warps) {
  if (cap < 32 || cap > kHugeCell || warps < 1 ||
      warps > kMaxWarpsPerBlock)
    return false;
  const size_t smem = c->K->collide_smem(warps, cap);
  if (smem > (size_t)kMaxDynSmem) return false;
  const bool one = c->n_inst == 1;
  const int per_sm = c->K->collide_blocks_per_sm(c->dim, warps, cap, one, c->mesh != 0);
  if (per_sm < 1) return false;
  c->sched_cap = cap;
  c->sched_warps = warps;
  c->collide_grid = c->nsm * per_sm;
  return true;
}

// Enqueue one step reading buffer `par` and writing buffer 1 - par, for
// capture into a step graph.  With ev != nullptr, event-record nodes
// ev[0..4] bracket the four kernel groups (the plan and collision
// launches; what is left of the injection branch when they end; the scan
// and bookkeeping; the scatter), so that the host can time them.
int enqueue_step(sp_ctx* c, int par, cudaEvent_t* ev = nullptr) {
  int n = 0;
  const StepArgs a = make_step_args(c, par);
  const auto rec = [&](int k) {
    if (ev) cudaEventRecordWithFlags(ev[k], c->stream, cudaEventRecordExternal);
  };
  rec(0);
  // The reservoir injection reads nothing the collision kernel writes (the
  // previous step's particle count and Delta t; its particles go after the
  // current ones, its histogram counts are atomics), so in the step graph
  // it is a branch that runs beside the collision kernel, in the issue
  // slots and SMs that kernel leaves free; the cell scan joins the two.
  const bool fork = c->n_ghost > 0;
  if (fork) {
    cudaEventRecord(c->fork_ev, c->stream);
    cudaStreamWaitEvent(c->side, c->fork_ev, 0);
    const InjectArgs ia = make_inject_args(c, par);
    c->K->inject(c->dim, ia, 0, c->side);
    launch_scan(c->gcount, c->goff, c->n_ghost, c->gscan_part, c->side);
    c->K->inject(c->dim, ia, 1, c->side);
    cudaEventRecord(c->join_ev, c->side);
    n += 4;
  }
  launch_plan(c->start, c->cost, c->NC, c->sched_cap, (c->prec != SP_FP64 && c->dim == 2) ? kSplitLanes : 0,
              c->batches, c->nbatch, c->big_list, c->big_count, c->stream);
  ++n;
  // the big-cell launch (cells disjoint from the batches') is a branch
  // beside the main launch: its blocks start as SMs free up at the end of
  // the main launch instead of after all of it
  cudaEventRecord(c->fork2_ev, c->stream);
  cudaStreamWaitEvent(c->side2, c->fork2_ev, 0);
  cudaStreamWaitEvent(c->side3, c->fork2_ev, 0);
  launch_collide_p(c, a, true, kBigGridPerSm * c->nsm, c->side2); ++n;
  cudaEventRecord(c->join2_ev, c->side2);
  c->K->collide_huge(c->dim, a, kBigGridPerSm * c->nsm, c->side3); ++n;
  cudaEventRecord(c->join3_ev, c->side3);
  launch_collide_p(c, a, false, small_grid(c), c->stream); ++n;
  cudaStreamWaitEvent(c->stream, c->join2_ev, 0);
  cudaStreamWaitEvent(c->stream, c->join3_ev, 0);
  rec(1);
  if (fork) cudaStreamWaitEvent(c->stream, c->join_ev, 0);
  rec(2);
  launch_scan(c->count, c->start, c->NC, c->scan_part, c->stream); n += 2;
  launch_step_finalize(c->dP, c->n_inst, c->dt_cur, c->dt_min, c->step_d, c->Mcur, c->Mtot, c->start,
                       c->NC, c->goff, c->gcount, c->n_ghost, c->big_count, c->ticket, c->nbatch,
                       c->surf_time, c->cyc, c->stream); ++n;
  rec(3);
  launch_scatter(c->key, c->start, c->count, c->perm, c->Mtot, c->cap, c->stream); ++n;
  rec(4);
  return n;
}

void destroy_graphs(sp_ctx* c) {
  for (int i = 0; i < 2; ++i) {
    if (c->graph[i]) {
      cudaGraphExecDestroy(c->graph[i]);
      c->graph[i] = nullptr;
    }
    if (c->pgraph[i]) {
      cudaGraphExecDestroy(c->pgraph[i]);
      c->pgraph[i] = nullptr;
    }
  }
  c->graph_ok = false;
}

sp_status build_graphs(sp_ctx* c) {
  destroy_graphs(c);
  if (!c->side) {
    CK(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming));
    CK(cudaStreamCreateWithFlags(&c->side2, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c->fork2_ev, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->join2_ev, cudaEventDisableTiming));
    CK(cudaStreamCreateWithFlags(&c->side3, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c->fork3_ev, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->join3_ev, cudaEventDisableTiming));
    for (int k = 0; k < 5; ++k) CK(cudaEventCreate(&c->pev[k]));
  }
  // per parity: the step graph, and the same graph with timing events at
  // the kernel groups' boundaries (sp_step_profiled)
  for (int prof = 0; prof < 2; ++prof)
    for (int par = 0; par < 2; ++par) {
      cudaStream_t cs;
      CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      cudaStream_t saved = c->stream;
      c->stream = cs;
      cudaGraph_t g;
      cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        const int n = enqueue_step(c, par, prof ? c->pev : nullptr);
        if (!prof) c->launches = n;
        e = cudaStreamEndCapture(cs, &g);
      }
      c->stream = saved;
      cudaStreamDestroy(cs);
      CK(e);
      e = cudaGraphInstantiate(prof ? &c->pgraph[par] : &c->graph[par], g, 0);
      cudaGraphDestroy(g);
      CK(e);
    }
  c->graph_ok = true;
  return SP_OK;
}

sp_status check_errors(sp_ctx* c) {
  unsigned long long h[kNumErr];
  CK(cudaMemcpyAsync(h, c->err, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (h[kErrCapacity] || h[kErrCellCap]) return SP_ERR_CAPACITY;
  return SP_OK;
}

// Convert the staged particles of every instance into the state buffers,
// index and sort them, and set Delta t of the next step from their moments.
sp_status upload(sp_ctx* c) {
  int64_t M = 0;
  for (int i = 0; i < c->n_inst; ++i) M += c->stage_n[i];
  if (M > c->cap) return SP_ERR_CAPACITY;
  const int dim = c->dim;
  int64_t off = 0;
  for (int i = 0; i < c->n_inst; ++i) {
    const int64_t n = c->stage_n[i];
    if (n > 0) {
      const double* sp = c->dstage[i];
      const float* sf = (const float*)c->dstage[i];
      if (c->stage_f32[i])
        c->K->stage_in32(dim, sf, sf + dim * n, n, c->pos[c->cur], c->vel[c->cur], off, c->part_inst,
                         (uint32_t)i, c->stream);
      else
        c->K->stage_in(dim, sp, sp + dim * n, n, c->pos[c->cur], c->vel[c->cur], off, c->part_inst,
                       (uint32_t)i, c->stream);
    }
    off += n;
  }
  CK(cudaMemsetAsync(c->count, 0, sizeof(uint32_t) * c->NC, c->stream));
  const void* P3[3] = {c->pos[c->cur][0], c->pos[c->cur][1], c->pos[c->cur][2]};
  if (c->mesh)
    c->K->keys_mesh(P3, M, c->part_inst, c->dP, c->mface, c->mnode, c->mrad, c->key, c->count, c->stream);
  else
    c->K->keys(dim, P3, M, c->part_inst, c->dP, c->key, c->count, c->stream);
  launch_scan(c->count, c->start, c->NC, c->scan_part, c->stream);
  c->hM = (uint32_t)M;
  CK(cudaMemcpyAsync(c->Mtot, &c->hM, 4, cudaMemcpyHostToDevice, c->stream));
  // the state holds the located particles only: an O-grid drops those
  // outside the mesh (sentinel keys), so its size is start[NC], not M
  CK(cudaMemcpyAsync(c->Mcur, c->start + c->NC, 4, cudaMemcpyDeviceToDevice, c->stream));
  launch_scatter(c->key, c->start, c->count, c->perm, c->Mtot, c->cap, c->stream);
  // the scatter's atomics leave each cell's order arbitrary: reproducible
  // runs restore the source order, so that the moments below (and the first
  // step's Delta t) sum each cell in the same order on every run
  if (c->stable) launch_order_cells(c->start, c->NC, c->perm, c->stream);
  // Delta t from the moments of this state
  for (int i = 0; i < c->n_inst; ++i) c->hinf[i] = 0x7FF0000000000000ull;
  CK(cudaMemcpyAsync(c->dt_min, c->hinf.data(), 8 * c->n_inst, cudaMemcpyHostToDevice, c->stream));
  StepArgs a = make_step_args(c, c->cur);
  c->K->moments(a, 0, c->NC, nullptr, c->stream);
  CK(cudaMemcpyAsync(c->hmin.data(), c->dt_min, 8 * c->n_inst, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (int i = 0; i < c->n_inst; ++i) {
    if (c->hP[i].dt_fixed > 0) c->hdt[i] = c->hP[i].dt_fixed;
    else if (c->hmin[i] != 0x7FF0000000000000ull) {
      double v;
      memcpy(&v, &c->hmin[i], 8);
      c->hdt[i] = c->hP[i].cfl * v;
    } else {
      return SP_ERR_ARG;  // no cell with two particles and no fixed step
    }
  }
  CK(cudaMemcpyAsync(c->dt_cur, c->hdt.data(), 8 * c->n_inst, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->dt_min, c->hinf.data(), 8 * c->n_inst, cudaMemcpyHostToDevice, c->stream));
  c->uploaded = true;
  c->dirty = false;
  return SP_OK;
}

sp_status ensure_ready(sp_ctx* c) {
  if (c->dirty) {
    sp_status s = upload(c);
    if (s != SP_OK) return s;
  }
  if (!c->uploaded) return SP_ERR_STATE;
  return SP_OK;
}

// host copy of start[] over an instance's cell range
sp_status host_starts(sp_ctx* c, int inst, std::vector<uint32_t>& st) {
  const InstParams& P = c->hP[inst];
  st.resize(P.ncells + 1);
  CK(cudaMemcpyAsync(st.data(), c->start + P.cell_off, sizeof(uint32_t) * (P.ncells + 1),
                     cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return SP_OK;
}

// perm over an instance's range, each cell's entries in ascending order
// (the stable order the collision kernel restores).
sp_status host_perm_sorted(sp_ctx* c, const std::vector<uint32_t>& st, std::vector<uint32_t>& pm) {
  const int64_t s0 = st[0], n = (int64_t)st.back() - s0;
  pm.resize(std::max<int64_t>(n, 1));
  if (n > 0)
    CK(cudaMemcpyAsync(pm.data(), c->perm + s0, 4 * n, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (size_t k = 0; k + 1 < st.size(); ++k) std::sort(pm.begin() + (st[k] - s0), pm.begin() + (st[k + 1] - s0));
  pm.resize(n);
  return SP_OK;
}

}  // namespace

extern "C" {

const char* sp_status_str(int s) {
  switch (s) {
    case SP_OK: return "ok";
    case SP_ERR_ARG: return "invalid argument";
    case SP_ERR_CUDA: return "CUDA runtime error";
    case SP_ERR_CAPACITY: return "capacity exceeded";
    case SP_ERR_DEVICE: return "device error flag set";
    case SP_ERR_STATE: return "call out of order";
    default: return "unknown status";
  }
}

sp_status sp_init(const sp_config* cfgs, int n_instances, int precision, int64_t capacity,
                  void* stream, sp_ctx** out) {
  if (!cfgs || n_instances < 1 || !out || capacity < 1 || capacity > (int64_t(1) << 31)) return SP_ERR_ARG;
  if (precision != SP_FP64 && precision != SP_FP32 && precision != SP_FP32_CELL32) return SP_ERR_ARG;
  const int dim = cfgs[0].dim;
  for (int i = 0; i < n_instances; ++i)
    if (!valid(cfgs[i], dim)) return SP_ERR_ARG;
  sp_ctx* c = new (std::nothrow) sp_ctx;
  if (!c) return SP_ERR_ARG;
  c->n_inst = n_instances;
  c->dim = dim;
  c->prec = precision;
  c->tsize = precision == SP_FP64 ? 8 : 4;
  c->K = precision == SP_FP64 ? &kernels_f64() : precision == SP_FP32 ? &kernels_f32() : &kernels_f32c();
  c->stream = (cudaStream_t)stream;
  c->cap = capacity;
  c->cfg.assign(cfgs, cfgs + n_instances);
  c->hP.resize(n_instances);
  int64_t off = 0, soff = 0;
  for (int i = 0; i < n_instances; ++i) {
    fill_params(cfgs[i], &c->hP[i], off);
    off += c->hP[i].ncells;
    c->hP[i].surf_off = soff;
    soff += c->hP[i].n_surf;
  }
  c->n_surf_tot = soff;
  c->NC = off;
  if (c->NC >= (int64_t)0xFFFFFFF0) { delete c; return SP_ERR_ARG; }
  c->dstage.assign(n_instances, nullptr);
  c->stage_n.assign(n_instances, 0);
  c->stage_cap.assign(n_instances, 0);
  c->stage_f32.assign(n_instances, 0);
  c->hinf.assign(n_instances, 0x7FF0000000000000ull);
  c->hmin.assign(n_instances, 0);
  c->hdt.assign(n_instances, 0.0);
  // body-fitted O-grid instances: every instance of a context has the same
  // mesh kind (one kernel variant per launch)
  c->mesh = cfgs[0].mesh;
  for (int i = 0; i < n_instances; ++i)
    if (cfgs[i].mesh != c->mesh) { delete c; return SP_ERR_ARG; }
  std::vector<MeshHost> meshes(c->mesh ? n_instances : 0);
  int64_t node_off = 0, rad_off = 0;
  for (int i = 0; i < (int)meshes.size(); ++i) {
    build_mesh(cfgs[i], meshes[i]);
    InstParams& P = c->hP[i];
    P.mesh = 1;
    P.mnl = cfgs[i].ghost_layers > 0 ? cfgs[i].ghost_layers : 0;
    P.mnode_off = node_off;
    P.mrad_off = rad_off;
    node_off += (int64_t)meshes[i].node.size() / 2;
    rad_off += (int64_t)meshes[i].rad.size();
  }
  std::vector<GhostCell> gh;
  for (int i = 0; i < n_instances; ++i) {
    if (c->mesh) build_ghosts_mesh(cfgs[i], meshes[i], i, gh);
    else build_ghosts(cfgs[i], c->hP[i], i, gh);
  }
  c->n_ghost = (int64_t)gh.size();

  sp_status st = [&]() -> sp_status {
    CK(c->K->configure());
    const int64_t NC = c->NC, cap = c->cap;
    for (int b = 0; b < 2; ++b)
      for (int d = 0; d < 3; ++d) {
        if (d < dim) CK(dalloc(&c->pos[b][d], cap * c->tsize));
        CK(dalloc(&c->vel[b][d], cap * c->tsize));
      }
    CK(dalloc(&c->key, 4 * cap));
    CK(dalloc(&c->part_inst, 4 * cap));
    CK(dalloc(&c->perm, 4 * cap));
    CK(dalloc(&c->count, 4 * NC));
    CK(dalloc(&c->start, 4 * (NC + 1)));
    CK(dalloc(&c->cell_inst, 4 * NC));
    CK(dalloc(&c->scan_part, 4 * scan_partial_size(NC)));
    CK(dalloc(&c->big_list, 4 * NC));
    CK(dalloc(&c->big_count, 4));
    CK(dalloc(&c->ticket, 4));
    CK(dalloc(&c->batches, sizeof(uint2) * kBatchClasses * NC));
    CK(dalloc(&c->nbatch, 4 * kBatchClasses));
    CK(dalloc(&c->cost, std::max<int64_t>(NC, 1)));
    CK(dalloc(&c->cyc, 24));
    CK(dalloc(&c->vol, 8 * NC));
    CK(dalloc(&c->ivol, 8 * NC));
    CK(dalloc(&c->rcp, 8 * (kHugeCell + 1)));
    CK(dalloc(&c->smax, 8 * NC));
    CK(dalloc(&c->rem, 8 * std::max<int64_t>(NC, 1)));
    CK(dalloc(&c->samp, 8 * 8 * NC));
    CK(dalloc(&c->msum, 8 * 7 * NC));
    CK(dalloc(&c->dP, sizeof(InstParams) * n_instances));
    CK(dalloc(&c->dt_cur, 8 * n_instances));
    CK(dalloc(&c->dt_min, 8 * n_instances));
    CK(dalloc(&c->surf, 8 * kSurfFields * std::max<int64_t>(c->n_surf_tot, 1)));
    CK(dalloc(&c->surf_time, 8 * n_instances));
    CK(dalloc(&c->step_d, 4));
    CK(dalloc(&c->Mcur, 4));
    CK(dalloc(&c->Mtot, 4));
    CK(dalloc(&c->err, 8 * kNumErr));
    CK(dalloc(&c->ghosts, sizeof(GhostCell) * std::max<int64_t>(c->n_ghost, 1)));
    CK(dalloc(&c->gcount, 4 * std::max<int64_t>(c->n_ghost, 1)));
    CK(dalloc(&c->goff, 4 * (std::max<int64_t>(c->n_ghost, 1) + 1)));
    CK(dalloc(&c->gscan_part, 4 * scan_partial_size(std::max<int64_t>(c->n_ghost, 1))));
    cudaStream_t s = c->stream;
    CK(cudaMemcpyAsync(c->dP, c->hP.data(), sizeof(InstParams) * n_instances, cudaMemcpyHostToDevice, s));
    if (c->n_ghost)
      CK(cudaMemcpyAsync(c->ghosts, gh.data(), sizeof(GhostCell) * c->n_ghost, cudaMemcpyHostToDevice, s));
    std::vector<uint32_t> ci(NC);
    std::vector<double> vol(NC), ivol(NC), sm(NC), rcp(kHugeCell + 1, 0.0);
    for (int k = 1; k <= kHugeCell; ++k) rcp[k] = 1.0 / (double)k;
    for (int i = 0; i < n_instances; ++i) {
      const InstParams& P = c->hP[i];
      const sp_config& g = cfgs[i];
      const double v0 = P.dl[0] * P.dl[1] * P.dl[2];
      const double crb = 4.0 * sqrt(g.R * g.sigc_T0 / kPiHost);
      const double s0 = 2.0 * (P.sigc_coef * pow(crb, P.sigc_exp));
      for (int64_t k = 0; k < P.ncells; ++k) {
        ci[P.cell_off + k] = (uint32_t)i;
        vol[P.cell_off + k] = c->mesh ? meshes[i].vol[k] : (g.cell_volume ? g.cell_volume[k] : v0);
        ivol[P.cell_off + k] = 1.0 / vol[P.cell_off + k];
        sm[P.cell_off + k] = s0;
      }
    }
    CK(cudaMemcpyAsync(c->cell_inst, ci.data(), 4 * NC, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->vol, vol.data(), 8 * NC, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->ivol, ivol.data(), 8 * NC, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->rcp, rcp.data(), 8 * (kHugeCell + 1), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->smax, sm.data(), 8 * NC, cudaMemcpyHostToDevice, s));
    if (c->mesh) {
      // faces and nodes in the state's type, cell sizes and radii in FP64
      std::vector<double> L(NC), iL(NC), face(12 * (size_t)NC), node(2 * (size_t)node_off), rad(rad_off);
      for (int i = 0; i < n_instances; ++i) {
        const InstParams& P = c->hP[i];
        const MeshHost& m = meshes[i];
        for (int64_t k = 0; k < P.ncells; ++k) {
          L[P.cell_off + k] = m.L[k];
          iL[P.cell_off + k] = 1.0 / m.L[k];
        }
        std::copy(m.face.begin(), m.face.end(), face.begin() + 12 * P.cell_off);
        std::copy(m.node.begin(), m.node.end(), node.begin() + 2 * P.mnode_off);
        std::copy(m.rad.begin(), m.rad.end(), rad.begin() + P.mrad_off);
      }
      CK(dalloc(&c->Lc, 8 * NC));
      CK(dalloc(&c->iLc, 8 * NC));
      CK(dalloc(&c->mrad, 8 * std::max<int64_t>(rad_off, 1)));
      CK(dalloc(&c->mface, c->tsize * face.size()));
      CK(dalloc(&c->mnode, c->tsize * std::max<size_t>(node.size(), 1)));
      CK(cudaMemcpy(c->Lc, L.data(), 8 * NC, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(c->iLc, iL.data(), 8 * NC, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(c->mrad, rad.data(), 8 * rad.size(), cudaMemcpyHostToDevice));
      if (c->tsize == 8) {
        CK(cudaMemcpy(c->mface, face.data(), 8 * face.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->mnode, node.data(), 8 * node.size(), cudaMemcpyHostToDevice));
      } else {
        std::vector<float> f32(face.begin(), face.end()), n32(node.begin(), node.end());
        CK(cudaMemcpy(c->mface, f32.data(), 4 * f32.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->mnode, n32.data(), 4 * n32.size(), cudaMemcpyHostToDevice));
      }
    }
    CK(cudaMemsetAsync(c->rem, 0, 8 * std::max<int64_t>(NC, 1), s));
    CK(cudaMemsetAsync(c->samp, 0, 8 * 8 * NC, s));
    CK(cudaMemsetAsync(c->surf, 0, 8 * kSurfFields * std::max<int64_t>(c->n_surf_tot, 1), s));
    CK(cudaMemsetAsync(c->surf_time, 0, 8 * n_instances, s));
    CK(cudaMemsetAsync(c->step_d, 0, 4, s));
    CK(cudaMemsetAsync(c->big_count, 0, 4, s));
    CK(cudaMemsetAsync(c->ticket, 0, 4, s));
    CK(cudaMemsetAsync(c->nbatch, 0, 4 * kBatchClasses, s));
    CK(cudaMemsetAsync(c->cost, 0, std::max<int64_t>(c->NC, 1), s));
    CK(cudaMemsetAsync(c->cyc, 0, 16, s));
    CK(cudaMemsetAsync(c->cyc + 2, 0xFF, 8, s));
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev));
    if (!apply_schedule(c, kCapSmall, kWarpsDefault) && !apply_schedule(c, 256, 2)) return SP_ERR_CUDA;
    CK(cudaMemsetAsync(c->err, 0, 8 * kNumErr, s));
    CK(cudaMemsetAsync(c->count, 0, 4 * NC, s));
    CK(cudaStreamSynchronize(s));
    return SP_OK;
  }();
  if (st != SP_OK) {
    sp_free(c);
    return st;
  }
  *out = c;
  return SP_OK;
}

sp_status sp_set_particles(sp_ctx* c, int inst, const double* pos, const double* vel, int64_t n) {
  if (!c || inst < 0 || inst >= c->n_inst || n < 0 || (n > 0 && (!pos || !vel))) return SP_ERR_ARG;
  if (n > c->cap) return SP_ERR_CAPACITY;
  const int64_t need = (int64_t)(c->dim + 3) * n;
  if (need > c->stage_cap[inst]) {
    CK(cudaStreamSynchronize(c->stream));
    if (c->dstage[inst]) CK(cudaFree(c->dstage[inst]));
    c->dstage[inst] = nullptr;
    CK(dalloc(&c->dstage[inst], 8 * need));
    c->stage_cap[inst] = need;
  }
  if (n > 0) {
    CK(cudaMemcpyAsync(c->dstage[inst], pos, 8 * c->dim * n, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->dstage[inst] + c->dim * n, vel, 8 * 3 * n, cudaMemcpyHostToDevice, c->stream));
  }
  c->stage_n[inst] = n;
  c->stage_f32[inst] = 0;
  c->dirty = true;
  return SP_OK;
}

sp_status sp_set_particles_f32(sp_ctx* c, int inst, const float* pos, const float* vel, int64_t n) {
  if (!c || inst < 0 || inst >= c->n_inst || n < 0 || (n > 0 && (!pos || !vel))) return SP_ERR_ARG;
  if (n > c->cap) return SP_ERR_CAPACITY;
  const int64_t need = (int64_t)(c->dim + 3) * n;  // floats; the staging area counts doubles
  if ((need + 1) / 2 > c->stage_cap[inst]) {
    CK(cudaStreamSynchronize(c->stream));
    if (c->dstage[inst]) CK(cudaFree(c->dstage[inst]));
    c->dstage[inst] = nullptr;
    CK(dalloc(&c->dstage[inst], 4 * need + 8));
    c->stage_cap[inst] = (need + 1) / 2;
  }
  if (n > 0) {
    float* f = (float*)c->dstage[inst];
    CK(cudaMemcpyAsync(f, pos, 4 * c->dim * n, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(f + c->dim * n, vel, 4 * 3 * n, cudaMemcpyHostToDevice, c->stream));
  }
  c->stage_n[inst] = n;
  c->stage_f32[inst] = 1;
  c->dirty = true;
  return SP_OK;
}

sp_status sp_set_record(sp_ctx* c, int on) {
  if (!c) return SP_ERR_ARG;
  const bool want = on != 0;
  if (want && !c->rec) {
    CK(dalloc(&c->rec, 4 * 4 * c->NC));
    CK(dalloc(&c->cons, 8 * 6 * c->NC));
    CK(dalloc(&c->resamp, c->cap));
  }
  if (want != c->record) {
    c->record = want;
    destroy_graphs(c);
  }
  return SP_OK;
}

sp_status sp_step(sp_ctx* c, int n_steps) {
  if (!c || n_steps < 0) return SP_ERR_ARG;
  sp_status s = ensure_ready(c);
  if (s != SP_OK) return s;
  if (!c->graph_ok) {
    s = build_graphs(c);
    if (s != SP_OK) return s;
  }
  for (int i = 0; i < n_steps; ++i) {
    if (c->record) {
      c->prev_start.resize(c->NC + 1);
      CK(cudaMemcpyAsync(c->prev_start.data(), c->start, 4 * (c->NC + 1), cudaMemcpyDeviceToHost, c->stream));
      CK(cudaMemsetAsync(c->resamp, 0, c->cap, c->stream));
      CK(cudaMemsetAsync(c->cons, 0, 8 * 6 * c->NC, c->stream));
      CK(cudaStreamSynchronize(c->stream));
    }
    CK(cudaGraphLaunch(c->graph[c->cur], c->stream));
    c->cur ^= 1;
    c->step_host += 1;
  }
  return SP_OK;
}

sp_status sp_step_profiled(sp_ctx* c, int n_steps, double* ms, int n_slots) {
  if (!c || n_steps < 0 || !ms || n_slots < 1) return SP_ERR_ARG;
  sp_status s = ensure_ready(c);
  if (s != SP_OK) return s;
  if (!c->graph_ok) {
    s = build_graphs(c);
    if (s != SP_OK) return s;
  }
  double acc[4] = {0, 0, 0, 0};
  for (int it = 0; it < n_steps; ++it) {
    CK(cudaGraphLaunch(c->pgraph[c->cur], c->stream));
    CK(cudaEventSynchronize(c->pev[4]));
    for (int k = 0; k < 4; ++k) {
      float t = 0;
      CK(cudaEventElapsedTime(&t, c->pev[k], c->pev[k + 1]));
      acc[k] += t;
    }
    c->cur ^= 1;
    c->step_host += 1;
  }
  for (int k = 0; k < n_slots && k < 4; ++k) ms[k] = acc[k];
  CK(cudaGetLastError());
  return SP_OK;
}

sp_status sp_set_reproducible(sp_ctx* c, int on) {
  if (!c) return SP_ERR_ARG;
  if (c->prec == SP_FP64 && !on) return SP_ERR_ARG;  // FP64 mode always keeps the source order
  if ((on != 0) != (c->stable != 0)) {
    c->stable = on != 0;
    destroy_graphs(c);
  }
  return SP_OK;
}

sp_status sp_set_schedule(sp_ctx* c, int cap, int warps) {
  if (!c) return SP_ERR_ARG;
  if (!apply_schedule(c, cap, warps)) return SP_ERR_ARG;
  destroy_graphs(c);
  return SP_OK;
}

sp_status sp_autotune(sp_ctx* c, int steps_per_trial, int* cap_out, int* warps_out) {
  if (!c || steps_per_trial < 1) return SP_ERR_ARG;
  sp_status s = ensure_ready(c);
  if (s != SP_OK) return s;
  static const int caps[] = {128, 256, 384, 512, 768, 1024};
  static const int warps[] = {2, 4, 8};
  const int cap0 = c->sched_cap, w0 = c->sched_warps;
  // collision-group time of steps_per_trial steps of the step graph (its
  // copy with timing events), after one untimed step (the batch partition
  // changes with the schedule, and the cost bytes of the old one are stale)
  auto trial = [&](int ci, int wi, float* tot) -> sp_status {
    *tot = 0;
    sp_status bs = build_graphs(c);
    if (bs != SP_OK) return bs;
    for (int it = 0; it <= steps_per_trial; ++it) {
      CK(cudaGraphLaunch(c->pgraph[c->cur], c->stream));
      CK(cudaEventSynchronize(c->pev[4]));
      float t = 0;
      CK(cudaEventElapsedTime(&t, c->pev[0], c->pev[1]));
      if (it > 0) *tot += t;
      c->cur ^= 1;
      c->step_host += 1;
    }
    return SP_OK;
  };
  struct Cand { int cap, warps; float t; };
  std::vector<Cand> cand;
  // the fixed capacities, and for each block size the largest capacity at
  // each residency level (blocks per SM from the occupancy calculator):
  // more resident warps with slightly smaller batches can win (on the
  // developed cylinder 864 x 2 at 6 blocks beat 1024 x 2 at 5 by 2 %)
  std::vector<std::pair<int, int>> sched;
  for (int wi : warps) {
    for (int ci : caps) sched.push_back({ci, wi});
    int last = -1;
    for (int ci = kHugeCell; ci >= 128; ci -= 32) {
      const int per = c->K->collide_blocks_per_sm(c->dim, wi, ci, c->n_inst == 1, c->mesh != 0);
      if (per != last && per > 0 &&
          std::find(sched.begin(), sched.end(), std::make_pair(ci, wi)) == sched.end())
        sched.push_back({ci, wi});
      last = per;
    }
  }
  for (const auto& sw : sched) {
    const int ci = sw.first, wi = sw.second;
    if (!apply_schedule(c, ci, wi)) continue;
    float t = 0;
    sp_status st = trial(ci, wi, &t);
    if (st != SP_OK) return st;
    cand.push_back({ci, wi, t});
  }
  // second pass over the three fastest: the flow drifts between trials
  std::sort(cand.begin(), cand.end(), [](const Cand& x, const Cand& y) { return x.t < y.t; });
  if (cand.size() > 3) cand.resize(3);
  for (Cand& k : cand) {
    if (!apply_schedule(c, k.cap, k.warps)) continue;
    float t = 0;
    sp_status st = trial(k.cap, k.warps, &t);
    if (st != SP_OK) return st;
    k.t += t;
  }
  int best_cap = cap0, best_w = w0;
  float best = 3.4e38f;
  for (const Cand& k : cand)
    if (k.t < best) {
      best = k.t;
      best_cap = k.cap;
      best_w = k.warps;
    }
  if (!apply_schedule(c, best_cap, best_w)) apply_schedule(c, cap0, w0);
  destroy_graphs(c);
  if (cap_out) *cap_out = c->sched_cap;
  if (warps_out) *warps_out = c->sched_warps;
  CK(cudaGetLastError());
  return check_errors(c);
}

sp_status sp_sync(sp_ctx* c) {
  if (!c) return SP_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaGetLastError());
  return check_errors(c);
}

int sp_launches_per_step(sp_ctx* c) {
  if (!c) return 0;
  if (!c->graph_ok && c->uploaded) build_graphs(c);
  return c->launches;
}

sp_status sp_moments(sp_ctx* c, int inst, int kind, double* out, int n_fields) {
  if (!c || inst < 0 || inst >= c->n_inst || !out || n_fields < 1) return SP_ERR_ARG;
  sp_status s = ensure_ready(c);
  if (s != SP_OK) return s;
  const InstParams& P = c->hP[inst];
  const int64_t nc = P.ncells;
  const int nf = std::min(n_fields, (int)SP_NFIELDS);
  if (kind == 0) {
    // page-locked host memory the device can address: the fields kernel
    // writes its rows straight into it (the link transfer overlaps the
    // FP64 work); otherwise a device buffer and one copy
    cudaPointerAttributes pa;
    double* direct = nullptr;
    if (nf == SP_NFIELDS && cudaPointerGetAttributes(&pa, out) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
        pa.devicePointer)
      direct = (double*)pa.devicePointer;
    cudaGetLastError();  // (a pointer unknown to CUDA leaves an error to clear)
    if (direct) {
      if (c->stable) launch_order_cells(c->start, c->NC, c->perm, c->stream);
      StepArgs a = make_step_args(c, c->cur);
      c->K->moments(a, P.cell_off, P.cell_off + nc, direct, c->stream);
      CK(cudaStreamSynchronize(c->stream));
      return check_errors(c);
    }
    if (nc > c->mom_cells) {  // one device buffer, grown on demand
      CK(cudaStreamSynchronize(c->stream));
      if (c->mom) CK(cudaFree(c->mom));
      c->mom = nullptr;
      c->mom_cells = 0;
      CK(dalloc(&c->mom, 8 * SP_NFIELDS * nc));
      c->mom_cells = nc;
    }
    double* d = c->mom;
    // reproducible runs: each cell summed in source order (the scatter's
    // order inside a cell is arbitrary; the collision step restores the
    // same order, so this changes no later result)
    if (c->stable) launch_order_cells(c->start, c->NC, c->perm, c->stream);
    StepArgs a = make_step_args(c, c->cur);
    c->K->moments(a, P.cell_off, P.cell_off + nc, d, c->stream);
    CK(cudaMemcpyAsync(out, d, 8 * nf * nc, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  } else {
    std::vector<double> S(8 * nc), vol(nc);
    for (int f = 0; f < 8; ++f)
      CK(cudaMemcpyAsync(S.data() + f * nc, c->samp + f * c->NC + P.cell_off, 8 * nc, cudaMemcpyDeviceToHost,
                         c->stream));
    CK(cudaMemcpyAsync(vol.data(), c->vol + P.cell_off, 8 * nc, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const int64_t nsamp = std::max<int64_t>(0, c->step_host - (int64_t)P.n_steady);
    for (int64_t k = 0; k < nc; ++k) {
      double f[SP_NFIELDS] = {0};
      const double sN = S[k];
      if (nsamp > 0) {
        f[SP_F_N] = sN / (double)nsamp;
        f[SP_F_n] = vol[k] > 0 ? f[SP_F_N] * P.Fn / vol[k] : 0.0;
        f[SP_F_ratio] = S[7 * nc + k] / (double)nsamp;
      }
      if (sN > 0) {
        double U[3], e = 0;
        for (int d = 0; d < 3; ++d) {
          U[d] = S[(1 + d) * nc + k] / sN;
          e += S[(4 + d) * nc + k] / sN - U[d] * U[d];
        }
        f[SP_F_ux] = U[0];
        f[SP_F_uy] = U[1];
        f[SP_F_uz] = U[2];
        f[SP_F_T] = e / (3.0 * P.R);
      }
      for (int i = 0; i < nf; ++i) out[(int64_t)i * nc + k] = f[i];
    }
  }
  return check_errors(c);
}

sp_status sp_get_particles(sp_ctx* c, int inst, double* pos, double* vel, uint32_t* cell, int64_t* n) {
  if (!c || inst < 0 || inst >= c->n_inst) return SP_ERR_ARG;
  sp_status s = ensure_ready(c);
  if (s != SP_OK) return s;
  std::vector<uint32_t> st;
  s = host_starts(c, inst, st);
  if (s != SP_OK) return s;
  const int64_t M = (int64_t)st.back() - st[0];
  if (n) *n = M;
  if (!pos && !vel && !cell) return SP_OK;
  if (cell)
    for (size_t k = 0; k + 1 < st.size(); ++k)
      for (uint32_t i = st[k]; i < st[k + 1]; ++i) cell[i - st[0]] = (uint32_t)k;
  if (!pos && !vel) return SP_OK;
  std::vector<uint32_t> pm;
  s = host_perm_sorted(c, st, pm);
  if (s != SP_OK) return s;
  uint32_t* dperm = nullptr;
  double *dpos = nullptr, *dvel = nullptr;
  CK(dalloc(&dperm, 4 * std::max<int64_t>(M, 1)));
  CK(dalloc(&dpos, 8 * 3 * std::max<int64_t>(M, 1)));
  CK(dalloc(&dvel, 8 * 3 * std::max<int64_t>(M, 1)));
  if (M > 0) CK(cudaMemcpyAsync(dperm, pm.data(), 4 * M, cudaMemcpyHostToDevice, c->stream));
  const void* Ap[3] = {c->pos[c->cur][0], c->pos[c->cur][1], c->pos[c->cur][2]};
  const void* Av[3] = {c->vel[c->cur][0], c->vel[c->cur][1], c->vel[c->cur][2]};
  c->K->gather(c->dim, Ap, Av, dperm, 0, M, dpos, dvel, c->stream);
  if (pos && M > 0) CK(cudaMemcpyAsync(pos, dpos, 8 * c->dim * M, cudaMemcpyDeviceToHost, c->stream));
  if (vel && M > 0) CK(cudaMemcpyAsync(vel, dvel, 8 * 3 * M, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  cudaFree(dperm);
  cudaFree(dpos);
  cudaFree(dvel);
  return check_errors(c);
}

sp_status sp_get_step_record(sp_ctx* c, int inst, int64_t* cell4, uint8_t* resampled, uint32_t* perm,
                             int64_t* n_old) {
  if (!c || inst < 0 || inst >= c->n_inst || !c->record || !c->rec) return SP_ERR_STATE;
  CK(cudaStreamSynchronize(c->stream));
  const InstParams& P = c->hP[inst];
  const int64_t nc = P.ncells;
  if (cell4) {
    std::vector<int32_t> r(4 * nc);
    for (int f = 0; f < 4; ++f)
      CK(cudaMemcpy(r.data() + f * nc, c->rec + f * c->NC + P.cell_off, 4 * nc, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < 4 * nc; ++i) cell4[i] = r[i];
  }
  const int64_t o0 = c->prev_start.empty() ? 0 : c->prev_start[P.cell_off];
  const int64_t o1 = c->prev_start.empty() ? 0 : c->prev_start[P.cell_off + nc];
  if (n_old) *n_old = o1 - o0;
  if (resampled && o1 > o0) CK(cudaMemcpy(resampled, c->resamp + o0, o1 - o0, cudaMemcpyDeviceToHost));
  if (perm) {
    std::vector<uint32_t> st, pm;
    sp_status s = host_starts(c, inst, st);
    if (s != SP_OK) return s;
    s = host_perm_sorted(c, st, pm);
    if (s != SP_OK) return s;
    std::copy(pm.begin(), pm.end(), perm);
  }
  return SP_OK;
}

sp_status sp_get_conservation(sp_ctx* c, int inst, double* out) {
  if (!c || inst < 0 || inst >= c->n_inst || !out) return SP_ERR_ARG;
  if (!c->record || !c->cons) return SP_ERR_STATE;
  const InstParams& P = c->hP[inst];
  const int64_t nc = P.ncells;
  for (int f = 0; f < 6; ++f)
    CK(cudaMemcpyAsync(out + f * nc, c->cons + f * c->NC + P.cell_off, 8 * nc, cudaMemcpyDeviceToHost,
                       c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return SP_OK;
}

sp_status sp_get_cell_start(sp_ctx* c, int inst, uint32_t* start) {
  if (!c || inst < 0 || inst >= c->n_inst || !start) return SP_ERR_ARG;
  sp_status s = ensure_ready(c);
  if (s != SP_OK) return s;
  std::vector<uint32_t> st;
  s = host_starts(c, inst, st);
  if (s != SP_OK) return s;
  for (size_t i = 0; i < st.size(); ++i) start[i] = st[i] - st[0];
  return SP_OK;
}

sp_status sp_get_sigc_max(sp_ctx* c, int inst, double* out) {
  if (!c || inst < 0 || inst >= c->n_inst || !out) return SP_ERR_ARG;
  const InstParams& P = c->hP[inst];
  CK(cudaMemcpyAsync(out, c->smax + P.cell_off, 8 * P.ncells, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return SP_OK;
}

sp_status sp_get_dt(sp_ctx* c, int inst, double* dt, int64_t* step) {
  if (!c || inst < 0 || inst >= c->n_inst) return SP_ERR_ARG;
  sp_status s = ensure_ready(c);
  if (s != SP_OK) return s;
  if (dt) {
    CK(cudaMemcpyAsync(dt, c->dt_cur + inst, 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  if (step) *step = c->step_host;
  return SP_OK;
}

sp_status sp_get_surface(sp_ctx* c, int inst, double* out, double* time) {
  if (!c || inst < 0 || inst >= c->n_inst) return SP_ERR_ARG;
  const InstParams& P = c->hP[inst];
  if (out && P.n_surf > 0) {
    std::vector<double> h(kSurfFields * (size_t)P.n_surf);
    CK(cudaMemcpyAsync(h.data(), c->surf + kSurfFields * P.surf_off, 8 * h.size(), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int b = 0; b < P.n_surf; ++b)
      for (int f = 0; f < kSurfFields; ++f) out[(size_t)f * P.n_surf + b] = h[kSurfFields * (size_t)b + f];
  }
  if (time) {
    CK(cudaMemcpyAsync(time, c->surf_time + inst, 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  return SP_OK;
}

sp_status sp_surface_coefficients(const sp_config* cfg, const double* tal, double time, double rho_inf,
                                  double u_inf, double p_inf, double* elem, double* body) {
  if (!cfg || !tal || !elem || !body) return SP_ERR_ARG;
  const int ns = cfg->n_surf;
  const double qinf = 0.5 * rho_inf * u_inf * u_inf;
  const bool circle = cfg->body == SP_BODY_CIRCLE, sphere = cfg->body == SP_BODY_SPHERE;
  if ((!circle && !sphere) || ns < 1 || !(time > 0) || !(qinf > 0) || !(cfg->body_r > 0))
    return SP_ERR_ARG;
  const double r = cfg->body_r, kPi = 3.14159265358979323846;
  const double depth = circle ? cfg->hi[2] - cfg->lo[2] : 1.0;
  auto inside = [&](const double* x) {
    for (int d = 0; d < cfg->dim; ++d)
      if (x[d] < cfg->lo[d] || x[d] > cfg->hi[d]) return false;
    return true;
  };
  double Aref2 = 0, F[2] = {0, 0}, E = 0, Atot = 0;
  for (int b = 0; b < ns; ++b) {
    // area of the element inside the box, and its |n_x|-weighted area, by
    // midpoint sub-sampling of the element
    double A = 0, Ax = 0;
    if (circle) {
      const int K = 2048;
      const double th0 = -kPi + 2.0 * kPi * b / ns, dth = 2.0 * kPi / ns / K;
      for (int k = 0; k < K; ++k) {
        const double th = th0 + (k + 0.5) * dth;
        const double x[3] = {cfg->body_c[0] + r * cos(th), cfg->body_c[1] + r * sin(th), 0.0};
        if (!inside(x)) continue;
        A += r * dth * depth;
        Ax += fabs(cos(th)) * r * dth * depth;
      }
    } else {
      const int KT = 64, KP = 512;
      const double th0 = kPi * b / ns, dth = kPi / ns / KT, dph = 2.0 * kPi / KP;
      for (int i = 0; i < KT; ++i) {
        const double th = th0 + (i + 0.5) * dth;
        for (int j = 0; j < KP; ++j) {
          const double ph = (j + 0.5) * dph;
          const double x[3] = {cfg->body_c[0] + r * cos(th), cfg->body_c[1] + r * sin(th) * cos(ph),
                               cfg->body_c[2] + r * sin(th) * sin(ph)};
          if (!inside(x)) continue;
          const double dA = r * r * sin(th) * dth * dph;
          A += dA;
          Ax += fabs(cos(th)) * dA;
        }
      }
    }
    elem[0 * (size_t)ns + b] = A;
    if (A > 0) {
      const double at = A * time;
      elem[1 * (size_t)ns + b] = (tal[5 * (size_t)ns + b] / at - p_inf) / qinf;
      elem[2 * (size_t)ns + b] = tal[6 * (size_t)ns + b] / at / qinf;
      elem[3 * (size_t)ns + b] = tal[4 * (size_t)ns + b] / at / (qinf * u_inf);
    } else {
      elem[1 * (size_t)ns + b] = elem[2 * (size_t)ns + b] = elem[3 * (size_t)ns + b] = 0.0;
    }
    Aref2 += Ax;
    Atot += A;
    F[0] += tal[1 * (size_t)ns + b];
    F[1] += tal[2 * (size_t)ns + b];
    E += tal[4 * (size_t)ns + b];
  }
  const double Aref = 0.5 * Aref2;
  if (!(Aref > 0)) return SP_ERR_ARG;
  body[0] = F[0] / time / (qinf * Aref);
  body[1] = F[1] / time / (qinf * Aref);
  body[2] = E / time / (qinf * u_inf * Atot);
  body[3] = Aref;
  return SP_OK;
}

sp_status sp_errors(sp_ctx* c, int64_t* out5) {
  if (!c || !out5) return SP_ERR_ARG;
  unsigned long long h[kNumErr];
  CK(cudaMemcpyAsync(h, c->err, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (int i = 0; i < kNumErr; ++i) out5[i] = (int64_t)h[i];
  return SP_OK;
}

sp_status sp_free(sp_ctx* c) {
  if (!c) return SP_ERR_ARG;
  cudaStreamSynchronize(c->stream);
  destroy_graphs(c);
  if (c->side) {
    cudaStreamDestroy(c->side);
    cudaEventDestroy(c->fork_ev);
    cudaEventDestroy(c->join_ev);
    cudaStreamDestroy(c->side2);
    cudaEventDestroy(c->fork2_ev);
    cudaEventDestroy(c->join2_ev);
    cudaStreamDestroy(c->side3);
    cudaEventDestroy(c->fork3_ev);
    cudaEventDestroy(c->join3_ev);
    for (int k = 0; k < 5; ++k) cudaEventDestroy(c->pev[k]);
  }
  for (int b = 0; b < 2; ++b)
    for (int d = 0; d < 3; ++d) {
      cudaFree(c->pos[b][d]);
      cudaFree(c->vel[b][d]);
    }
  for (double* p : c->dstage) cudaFree(p);
  void* ptrs[] = {c->Lc, c->iLc, c->mrad, c->mface, c->mnode, c->ivol, c->rcp, c->cons, c->mom, c->msum, c->cost, c->cyc, c->surf, c->surf_time, c->batches, c->nbatch, c->ticket, c->part_inst, c->key, c->perm, c->count, c->start, c->cell_inst, c->scan_part, c->big_list,
                  c->big_count, c->vol, c->smax, c->rem, c->samp, c->rec, c->resamp, c->dP, c->dt_cur, c->dt_min,
                  c->step_d, c->Mcur, c->Mtot, c->err, c->ghosts, c->gcount, c->goff, c->gscan_part};
  for (void* p : ptrs) cudaFree(p);
  delete c;
  return SP_OK;
}

}  // extern "C"
