// sp_internal.h -- data structures shared by the host driver and the kernels
// of libsp (not part of the public ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace sp {

constexpr uint32_t kSentinel = 0xFFFFFFFFu;  // key of a removed particle
constexpr int kMaxBounce = 16;               // wall events per particle per step
constexpr int kMaxCross = 4096;              // face crossings per particle per step (O-grid)
// Per-cell sums in the collision kernel: a cell of at most kLaneSumMax
// particles is summed by lanes of its batch's warp, above it by the whole
// warp.  With an FP32 state in 2-D such a cell takes ceil(N / kSplitLanes) lanes
// (at most kMaxParts), each summing a contiguous part; the batch plan keeps
// the lanes of a batch within 32.  FP64 mode: one lane per cell (the
// oracle's summation order).  (Developed cylinder, 864 x 2: split 32 +2.5 %
// over no split; 16 / 24 / 48 / 64 and 8 parts were slower than 32 -- more
// lanes per cell leave fewer cells per batch.)
constexpr int kLaneSumMax = 256;
constexpr int kSplitLanes = 32;
constexpr int kMaxParts = 4;
__host__ __device__ constexpr int cell_lanes(int n, int split) {
  return (split > 0 && n <= kLaneSumMax) ? (n <= split ? 1 : (n + split - 1) / split > kMaxParts ? kMaxParts : (n + split - 1) / split) : 1;
}
constexpr int kSurfFields = 7;  // wall tallies per surface element
constexpr int64_t kNcolCap = int64_t(1) << 24;
constexpr int kBatchClasses = 9;             // batch lists by predicted cost (most expensive first)
constexpr int kMaxWarpsPerBlock = 8;         // collide kernel block size limit
constexpr int kCapSmall = 512;               // default per-warp staging capacity (particles)
constexpr int kWarpsDefault = 4;             // default warps per block
constexpr int kMaxDynSmem = 232448;          // 227 KB per block (opt-in maximum)
// Cells above kHugeCell particles are collided by one block each (the
// huge-cell launch); the other launches stage at most kHugeCell particles
// per warp, so which code collides a cell depends on the cell alone.
constexpr int kHugeCell = 1024;
constexpr int kMaxSub = 8;                   // sub-cells per cell

// Philox stream purposes (high byte of counter word 3).
constexpr uint32_t kPurpNtc = 1, kPurpShk = 2, kPurpWall = 3, kPurpInj = 4, kPurpInjWall = 5;

// Error counters (device, sticky).
enum { kErrCapacity = 0, kErrCellCap = 1, kErrBounce = 2, kErrAr = 3, kErrNcol = 4, kNumErr = 5 };

// Geometry and wall constants of an instance in the particle precision T
// (so per-particle code never converts).
template <class T>
struct Geo {
  T lo[3], hi[3], inv_d[3];
  T eps[3];      // inside-box margin of the free-flight fast path
  T body_c[3], body_r;
  T face_RT[6];  // R * T_face
  T body_RT;     // R * T_wall of the body
  T sigc_coef, sigc_exp;
  T win_lo[6][2], win_hi[6][2];  // open windows of outflow / inflow faces
};

// Per-instance constants, precomputed on the host.
struct InstParams {
  int dim;
  int n[3];
  double lo[3], hi[3], inv_d[3], dl[3], Lmin;
  double m, R, gamma, Pr, omega, T_ref, mu_ref, Fn, cfl, dt_fixed;
  double sigc_coef, sigc_exp;  // sigma_T c_r = coef * c_r^exp
  int face_bc[6];
  int face_win;      // bit f: face f is open only on its window
  double face_T[6];
  int body;
  double body_c[3], body_r, body_Tw;
  int n_steady;
  uint32_t key0, key1;
  int mode;
  int ar_max;
  int ntc_carry;     // carried NTC remainder instead of stochastic rounding
  int subcells;      // sub-cells per axis (1: off)
  int nsub;          // sub-cells per cell (subcells^dim, at most kMaxSub)
  int64_t cell_off;  // first global cell of the instance
  int64_t ncells;
  int n_surf;        // surface elements of the body (0: no tallies)
  int64_t surf_off;  // first element in the context's tally array
  double FnM;        // F_N m: weight of one hit in the tallies
  // constants of the FP64 per-cell arithmetic of the FP32 modes
  double inv3R;      // 1 / (3 R)
  double sqrt_gamma; // sqrt(gamma)
  double tau_k;      // tau = tau_k T^(omega - 1) / n, tau_k = mu_ref T_ref^-omega / (m R)
  double inv_tau_k;  // 1 / tau_k
  double inv_Lmin;   // 1 / L_min
  double inv_Fn;     // 1 / F_N
  float omf;         // 1 - omega in FP32 (the bound that certifies a pure DSMC split)
  // body-fitted O-grid (mesh = 1): n[0] radial layers x n[1] sectors, mnl
  // reservoir rings; its nodes start at mnode_off (node (i, j) at
  // mnode_off + i n[1] + j) and its radii at mrad_off
  int mesh;
  int mnl;
  int64_t mnode_off, mrad_off;
  Geo<double> g64;
  Geo<float> g32;
};

// One reservoir (ghost) cell outside an inflow face.
struct GhostCell {
  int inst;
  int face;
  uint32_t gc;       // index within the face's reservoir (Philox counter)
  int pad;
  double blo[3], bhi[3];
  // O-grid reservoir quadrilateral: ring mlay beyond the outer polygon,
  // sector msec; a1, a2 the areas of its triangles (A B C), (A C D)
  int mlay, msec;
  double a1, a2;
  double lam;        // expected particles = n_face * V / Fn
  double s2RT;       // sqrt(2 R T_face)
  double u[3];       // reservoir drift
};

struct StepArgs {
  // particle buffers: A = current (read through perm), B = output
  const void* Apos[3];
  const void* Avel[3];
  void* Bpos[3];
  void* Bvel[3];
  uint32_t* key;        // [cap]   key of each B slot
  uint32_t* perm;       // [cap]   slot -> source index in A (FP32: sorted in place per cell)
  const uint32_t* start;// [NC+1]  cell offsets of the current state
  uint32_t* count;      // [NC]    next-state histogram (atomics)
  const uint32_t* cell_inst;  // [NC]
  const double* vol;    // [NC]
  const double* ivol;   // [NC] 1 / vol
  const double* rcp;    // [kHugeCell + 1] rcp[k] = 1 / k (rcp[0] = 0)
  double* smax;         // [NC]
  double* rem;          // [NC] carried NTC remainder
  double* samp;         // [8][NC]
  int32_t* rec;         // [4][NC] or null
  double* cons;         // [6][NC] rescale conservation record (record mode) or null
  uint8_t* resamp;      // [cap] or null
  const InstParams* P;  // [n_inst]
  const double* dt_cur; // [n_inst]
  unsigned long long* dt_min;  // [n_inst] (double bits, atomicMin)
  const uint32_t* step; // global step index
  uint32_t* big_list;   // cells above kCapSmall
  uint32_t* big_count;
  uint32_t* ticket;     // work-stealing counter over the batch list
  const uint2* batches; // [kBatchClasses][NC] (first cell, cell count) of each batch, per class
  const uint32_t* nbatch;  // [kBatchClasses] batches per class (taken in class order)
  uint8_t* cost;        // [NC] cost byte: last step's cycles per particle of the cell's batch / cyc[2]
  unsigned long long* cyc;  // [3] batch cycles and particles this step (sums), cost unit (cycles per particle)
  unsigned long long* err;  // [kNumErr]
  int64_t NC;
  int64_t cap;
  int big_cap;          // staging capacity of the big-cell launch
  int cap_small;        // staging capacity per warp of the main launch
  int stable;           // restore source order within cells (reproducible runs)
  double* surf;         // [elements][kSurfFields] wall tallies
  int one;              // a single instance: P0 is its parameter set
  // body-fitted O-grid instances (mesh = 1; all instances of a context
  // share the mesh kind): per-cell size L of Delta t_c and 1/L, faces
  // (state type, [NC][4][3]: outward unit normal, offset), nodes (state
  // type, [.][2]) and node radii of all instances; null without a mesh
  int mesh;
  const double* Lc;
  const double* iLc;
  const void* mface;
  const void* mnode;
  const double* mrad;
  double* msum;         // [7][NC] scratch of the moments kernels
  InstParams P0;        // instance 0, by value (kernel parameter space)
};

struct InjectArgs {
  const GhostCell* ghosts;
  int64_t n_ghost;
  uint32_t* gcount;     // [n_ghost] survivors (pass 0)
  const uint32_t* goff; // [n_ghost] exclusive offsets (pass 1)
  void* Bpos[3];
  void* Bvel[3];
  uint32_t* key;
  uint32_t* count;
  const InstParams* P;
  const double* dt_cur;
  const uint32_t* step;
  const uint32_t* Mcur; // particles of the current state (base of appends)
  unsigned long long* err;
  int64_t cap;
  double* surf;
  const void* mface;    // O-grid faces and nodes (as in StepArgs) or null
  const void* mnode;
};

// Launch wrappers of one precision mode (sp_kern.cu, compiled once per mode:
// f64 = FP64 state and arithmetic; f32 = FP32 state, FP64 per-cell sums and
// arithmetic; f32c = FP32 state and FP32 per-cell sums and arithmetic).
struct KernelSet {
  void (*collide)(int dim, const StepArgs& a, bool big, int grid, int warps, cudaStream_t s);
  void (*collide_huge)(int dim, const StepArgs& a, int grid, cudaStream_t s);
  size_t (*collide_smem)(int warps, int cap);
  int (*collide_blocks_per_sm)(int dim, int warps, int cap, bool one, bool mesh);
  cudaError_t (*configure)();
  void (*inject)(int dim, const InjectArgs& a, int pass, cudaStream_t s);
  void (*moments)(const StepArgs& a, int64_t c0, int64_t c1, double* out, cudaStream_t s);
  void (*keys)(int dim, const void* const pos[3], int64_t M, const uint32_t* part_inst, const InstParams* P,
               uint32_t* key, uint32_t* count, cudaStream_t s);
  void (*keys_mesh)(const void* const pos[3], int64_t M, const uint32_t* part_inst, const InstParams* P,
                    const void* mface, const void* mnode, const double* mrad, uint32_t* key,
                    uint32_t* count, cudaStream_t s);
  void (*gather)(int dim, const void* const Apos[3], const void* const Avel[3], const uint32_t* perm,
                 int64_t s0, int64_t n, double* out_pos, double* out_vel, cudaStream_t s);
  void (*stage_in)(int dim, const double* pos, const double* vel, int64_t n, void* const dpos[3],
                   void* const dvel[3], int64_t off, uint32_t* part_inst, uint32_t inst, cudaStream_t s);
  void (*stage_in32)(int dim, const float* pos, const float* vel, int64_t n, void* const dpos[3],
                     void* const dvel[3], int64_t off, uint32_t* part_inst, uint32_t inst, cudaStream_t s);
};
const KernelSet& kernels_f64();
const KernelSet& kernels_f32();
const KernelSet& kernels_f32c();

// Precision-independent kernels (sp_common.cu).
void launch_scan(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* partial, cudaStream_t s);
void launch_plan(const uint32_t* start, const uint8_t* cost, int64_t NC, int cap, int split, uint2* batches, uint32_t* nbatch,
                 uint32_t* big_list, uint32_t* big_count, cudaStream_t s);
void launch_scatter(const uint32_t* key, const uint32_t* start, uint32_t* count, uint32_t* perm,
                    const uint32_t* Mtot, int64_t cap, cudaStream_t s);
void launch_step_finalize(const InstParams* P, int n_inst, double* dt_cur,
                          unsigned long long* dt_min, uint32_t* step, uint32_t* Mcur,
                          uint32_t* Mtot, const uint32_t* start_new, int64_t NC,
                          const uint32_t* goff, const uint32_t* gcount, int64_t n_ghost,
                          uint32_t* big_count, uint32_t* ticket, uint32_t* nbatch,
                          double* surf_time, unsigned long long* cyc, cudaStream_t s);
int64_t scan_partial_size(int64_t n);

}  // namespace sp
