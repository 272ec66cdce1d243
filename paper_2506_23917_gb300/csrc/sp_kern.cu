// sp_kern.cu -- instantiations and launch wrappers of the libsp kernels for
// one precision mode, compiled once per mode (see build.py):
//   SP_KT  particle state and per-particle arithmetic (float or double),
//   SP_KA  per-cell sums and per-cell arithmetic (float or double),
//   SP_TAG suffix of the exported kernel table (f64, f32, f32c).
#include "sp_device.cuh"

#if !defined(SP_KT) || !defined(SP_KA) || !defined(SP_TAG)
#error "compile with -DSP_KT=<type> -DSP_KA=<type> -DSP_TAG=<suffix>"
#endif
#define SP_CAT2(a, b) a##_##b
#define SP_CAT(a, b) SP_CAT2(a, b)

namespace sp {

namespace {
using T = SP_KT;
using A = SP_KA;

template <int DIM, bool ONE, bool MESH>
void collide_dim1(const StepArgs& a, bool big, int grid, int warps, cudaStream_t s) {
  if (!big) {
    const size_t smem = (size_t)warps * warp_stage_bytes<T, A>(a.cap_small);
    k_collide<T, A, DIM, ONE, MESH><<<grid, 32 * warps, smem, s>>>(a, 0);
  } else {
    const size_t smem = warp_stage_bytes<T, A>(a.big_cap);
    k_collide<T, A, DIM, ONE, MESH><<<grid, 32, smem, s>>>(a, 1);
  }
}

template <int DIM, bool MESH = false>
void collide_dim(const StepArgs& a, bool big, int grid, int warps, cudaStream_t s) {
  if (a.one) collide_dim1<DIM, true, MESH>(a, big, grid, warps, s);
  else collide_dim1<DIM, false, MESH>(a, big, grid, warps, s);
}

// (O-grid instances are 2-D: their kernels take the face-crossing flight)
void collide(int dim, const StepArgs& a, bool big, int grid, int warps, cudaStream_t s) {
  if (dim == 1) collide_dim<1>(a, big, grid, warps, s);
  else if (dim == 2 && a.mesh) collide_dim<2, true>(a, big, grid, warps, s);
  else if (dim == 2) collide_dim<2>(a, big, grid, warps, s);
  else collide_dim<3>(a, big, grid, warps, s);
}

size_t collide_smem(int warps, int cap) { return (size_t)warps * warp_stage_bytes<T, A>(cap); }

template <int DIM, bool MESH = false>
void collide_huge_dim(const StepArgs& a, int grid, cudaStream_t s) {
  const size_t smem = huge_smem_bytes<T, A>();
  if (a.one) k_collide_huge<T, A, DIM, true, MESH><<<grid, kHugeThreads, smem, s>>>(a);
  else k_collide_huge<T, A, DIM, false, MESH><<<grid, kHugeThreads, smem, s>>>(a);
}

void collide_huge(int dim, const StepArgs& a, int grid, cudaStream_t s) {
  if (dim == 1) collide_huge_dim<1>(a, grid, s);
  else if (dim == 2 && a.mesh) collide_huge_dim<2, true>(a, grid, s);
  else if (dim == 2) collide_huge_dim<2>(a, grid, s);
  else collide_huge_dim<3>(a, grid, s);
}

template <int DIM>
void inject_dim(const InjectArgs& a, int pass, cudaStream_t s) {
  const int64_t g = (a.n_ghost + 3) / 4;  // one warp per reservoir cell
  k_inject<T, DIM><<<(unsigned)g, 128, 0, s>>>(a, pass);
}

void inject(int dim, const InjectArgs& a, int pass, cudaStream_t s) {
  if (a.n_ghost == 0) return;
  if (a.mface) {  // O-grid reservoir rings
    k_inject_mesh<T><<<(unsigned)((a.n_ghost + 3) / 4), 128, 0, s>>>(a, pass);
    return;
  }
  if (dim == 1) inject_dim<1>(a, pass, s);
  else if (dim == 2) inject_dim<2>(a, pass, s);
  else inject_dim<3>(a, pass, s);
}

void moments(const StepArgs& a, int64_t c0, int64_t c1, double* out, cudaStream_t s) {
  const int64_t nc = c1 - c0;
  if (nc <= 0) return;
  int64_t g = (nc + 15) / 16;  // a half-warp per cell, 16 cells per block, grid-stride
  if (g > 65535) g = 65535;
  if (out) k_moment_sums<T, A, true><<<(unsigned)g, 256, 0, s>>>(a, c0, c1, a.msum);
  else k_moment_sums<T, A, false><<<(unsigned)g, 256, 0, s>>>(a, c0, c1, a.msum);
  k_moment_cells<sizeof(T) == 4><<<(unsigned)((nc + 255) / 256), 256, 0, s>>>(a, c0, c1, a.msum, out);
}

template <int DIM>
void keys_dim(const void* const pos[3], int64_t M, const uint32_t* part_inst, const InstParams* P,
              uint32_t* key, uint32_t* count, cudaStream_t s) {
  const int64_t g = (M + 255) / 256;
  k_keys<T, DIM><<<(unsigned)g, 256, 0, s>>>((const T*)pos[0], (const T*)pos[1], (const T*)pos[2], M,
                                             part_inst, P, key, count);
}

void keys_mesh(const void* const pos[3], int64_t M, const uint32_t* part_inst, const InstParams* P,
               const void* mface, const void* mnode, const double* mrad, uint32_t* key, uint32_t* count,
               cudaStream_t s) {
  if (M == 0) return;
  const int64_t g = (M + 255) / 256;
  k_keys_mesh<T><<<(unsigned)g, 256, 0, s>>>((const T*)pos[0], (const T*)pos[1], M, part_inst, P,
                                             (const T*)mface, (const T*)mnode, mrad, key, count);
}

void keys(int dim, const void* const pos[3], int64_t M, const uint32_t* part_inst, const InstParams* P,
          uint32_t* key, uint32_t* count, cudaStream_t s) {
  if (M == 0) return;
  if (dim == 1) keys_dim<1>(pos, M, part_inst, P, key, count, s);
  else if (dim == 2) keys_dim<2>(pos, M, part_inst, P, key, count, s);
  else keys_dim<3>(pos, M, part_inst, P, key, count, s);
}

void gather(int dim, const void* const Apos[3], const void* const Avel[3], const uint32_t* perm, int64_t s0,
            int64_t n, double* out_pos, double* out_vel, cudaStream_t s) {
  if (n == 0) return;
  const int64_t g = (n + 255) / 256;
  k_gather<T><<<(unsigned)g, 256, 0, s>>>((const T*)Apos[0], (const T*)Apos[1], (const T*)Apos[2],
                                          (const T*)Avel[0], (const T*)Avel[1], (const T*)Avel[2],
                                          dim, perm, s0, n, out_pos, out_vel);
}

template <class S>
void stage_in(int dim, const S* pos, const S* vel, int64_t n, void* const dpos[3], void* const dvel[3],
              int64_t off, uint32_t* part_inst, uint32_t inst, cudaStream_t s) {
  if (n == 0) return;
  const int64_t g = (n + 255) / 256;
  k_stage_in<T><<<(unsigned)g, 256, 0, s>>>(pos, vel, dim, n, (T*)dpos[0], (T*)dpos[1], (T*)dpos[2],
                                            (T*)dvel[0], (T*)dvel[1], (T*)dvel[2], off, part_inst, inst);
}

template <int DIM, bool ONE, bool MESH>
cudaError_t configure_dim1() {
  cudaError_t e = cudaFuncSetAttribute(k_collide<T, A, DIM, ONE, MESH>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
  if (e == cudaSuccess)  // staging lives in shared memory: prefer the largest carveout
    e = cudaFuncSetAttribute(k_collide<T, A, DIM, ONE, MESH>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             100);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_collide_huge<T, A, DIM, ONE, MESH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)huge_smem_bytes<T, A>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_collide_huge<T, A, DIM, ONE, MESH>,
                             cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  return e;
}

template <int DIM, bool MESH = false>
cudaError_t configure_dim() {
  cudaError_t e = configure_dim1<DIM, true, MESH>();
  if (e == cudaSuccess) e = configure_dim1<DIM, false, MESH>();
  return e;
}

cudaError_t configure() {
  cudaError_t e = configure_dim<1>();
  if (e == cudaSuccess) e = configure_dim<2>();
  if (e == cudaSuccess) e = configure_dim<2, true>();
  if (e == cudaSuccess) e = configure_dim<3>();
  return e;
}

template <int DIM, bool MESH = false>
int blocks_per_sm_dim(int warps, size_t smem, bool one) {
  int n = 0;
  if (one)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_collide<T, A, DIM, true, MESH>, 32 * warps, smem);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_collide<T, A, DIM, false, MESH>, 32 * warps, smem);
  return n;
}

int blocks_per_sm(int dim, int warps, int cap, bool one, bool mesh) {
  const size_t smem = (size_t)warps * warp_stage_bytes<T, A>(cap);
  if (dim == 1) return blocks_per_sm_dim<1>(warps, smem, one);
  if (dim == 2 && mesh) return blocks_per_sm_dim<2, true>(warps, smem, one);
  if (dim == 2) return blocks_per_sm_dim<2>(warps, smem, one);
  return blocks_per_sm_dim<3>(warps, smem, one);
}
}  // namespace

const KernelSet& SP_CAT(kernels, SP_TAG)() {
  static const KernelSet k = {collide,  collide_huge, collide_smem,     blocks_per_sm,   configure,
                              inject,   moments,      keys,             keys_mesh,       gather,
                              stage_in<double>,       stage_in<float>};
  return k;
}

}  // namespace sp
