// sp_kern_f32.cu -- FP32-mode instantiations of the libsp kernels.
#include "sp_device.cuh"

namespace sp {

namespace {
using T = float;

template <int DIM, bool ONE>
void collide_dim1(const StepArgs& a, bool big, int grid, int warps, cudaStream_t s) {
  if (!big) {
    const size_t smem = (size_t)warps * warp_stage_bytes<T>(a.cap_small);
    k_collide<T, DIM, ONE><<<grid, 32 * warps, smem, s>>>(a, 0);
  } else {
    const size_t smem = warp_stage_bytes<T>(a.big_cap);
    k_collide<T, DIM, ONE><<<grid, 32, smem, s>>>(a, 1);
  }
}

template <int DIM>
void collide_dim(const StepArgs& a, bool big, int grid, int warps, cudaStream_t s) {
  if (a.one) collide_dim1<DIM, true>(a, big, grid, warps, s);
  else collide_dim1<DIM, false>(a, big, grid, warps, s);
}

template <int DIM>
void inject_dim(const InjectArgs& a, int pass, cudaStream_t s) {
  const int64_t g = (a.n_ghost + 3) / 4;  // one warp per reservoir cell
  k_inject<T, DIM><<<(unsigned)g, 128, 0, s>>>(a, pass);
}

template <int DIM>
void keys_dim(const void* const pos[3], int64_t M, const uint32_t* part_inst, const InstParams* P,
              uint32_t* key, uint32_t* count, cudaStream_t s) {
  const int64_t g = (M + 255) / 256;
  k_keys<T, DIM><<<(unsigned)g, 256, 0, s>>>((const T*)pos[0], (const T*)pos[1], (const T*)pos[2], M,
                                             part_inst, P, key, count);
}

template <int DIM, bool ONE>
cudaError_t configure_dim1() {
  cudaError_t e = cudaFuncSetAttribute(k_collide<T, DIM, ONE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kMaxDynSmem);
  if (e == cudaSuccess)  // staging lives in shared memory: prefer the largest carveout
    e = cudaFuncSetAttribute(k_collide<T, DIM, ONE>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  return e;
}

template <int DIM>
cudaError_t configure_dim(int) {
  cudaError_t e = configure_dim1<DIM, true>();
  if (e == cudaSuccess) e = configure_dim1<DIM, false>();
  return e;
}

template <int DIM>
int blocks_per_sm(int warps, size_t smem, bool one) {
  int n = 0;
  if (one) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_collide<T, DIM, true>, 32 * warps, smem);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_collide<T, DIM, false>, 32 * warps, smem);
  return n;
}
}  // namespace

void launch_collide_f32(int dim, const StepArgs& a, bool big, int grid, int warps, cudaStream_t s) {
  if (dim == 1) collide_dim<1>(a, big, grid, warps, s);
  else if (dim == 2) collide_dim<2>(a, big, grid, warps, s);
  else collide_dim<3>(a, big, grid, warps, s);
}

size_t collide_smem_f32(int warps, int cap) { return (size_t)warps * warp_stage_bytes<T>(cap); }

void launch_inject_f32(int dim, const InjectArgs& a, int pass, cudaStream_t s) {
  if (a.n_ghost == 0) return;
  if (dim == 1) inject_dim<1>(a, pass, s);
  else if (dim == 2) inject_dim<2>(a, pass, s);
  else inject_dim<3>(a, pass, s);
}

void launch_moments_f32(const StepArgs& a, int64_t c0, int64_t c1, double* out, cudaStream_t s) {
  const int64_t nc = c1 - c0;
  int64_t g = (nc + 255) / 256;  // a warp per 32 cells, 8 warps per block
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  k_moments<T><<<(unsigned)g, 256, 0, s>>>(a, c0, c1, out);
}

void launch_keys_f32(int dim, const void* const pos[3], int64_t M, const uint32_t* part_inst,
                       const InstParams* P, uint32_t* key, uint32_t* count, cudaStream_t s) {
  if (M == 0) return;
  if (dim == 1) keys_dim<1>(pos, M, part_inst, P, key, count, s);
  else if (dim == 2) keys_dim<2>(pos, M, part_inst, P, key, count, s);
  else keys_dim<3>(pos, M, part_inst, P, key, count, s);
}

void launch_gather_f32(int dim, const void* const Apos[3], const void* const Avel[3],
                         const uint32_t* perm, int64_t s0, int64_t n, double* out_pos,
                         double* out_vel, cudaStream_t s) {
  if (n == 0) return;
  const int64_t g = (n + 255) / 256;
  k_gather<T><<<(unsigned)g, 256, 0, s>>>((const T*)Apos[0], (const T*)Apos[1], (const T*)Apos[2],
                                          (const T*)Avel[0], (const T*)Avel[1], (const T*)Avel[2],
                                          dim, perm, s0, n, out_pos, out_vel);
}

void launch_stage_in_f32(int dim, const double* pos, const double* vel, int64_t n, void* const dpos[3],
                          void* const dvel[3], int64_t off, uint32_t* part_inst, uint32_t inst,
                          cudaStream_t s) {
  if (n == 0) return;
  const int64_t g = (n + 255) / 256;
  k_stage_in<T><<<(unsigned)g, 256, 0, s>>>(pos, vel, dim, n, (T*)dpos[0], (T*)dpos[1], (T*)dpos[2],
                                            (T*)dvel[0], (T*)dvel[1], (T*)dvel[2], off, part_inst, inst);
}

void launch_stage_in32_f32(int dim, const float* pos, const float* vel, int64_t n, void* const dpos[3],
                          void* const dvel[3], int64_t off, uint32_t* part_inst, uint32_t inst,
                          cudaStream_t s) {
  if (n == 0) return;
  const int64_t g = (n + 255) / 256;
  k_stage_in<T><<<(unsigned)g, 256, 0, s>>>(pos, vel, dim, n, (T*)dpos[0], (T*)dpos[1], (T*)dpos[2],
                                            (T*)dvel[0], (T*)dvel[1], (T*)dvel[2], off, part_inst, inst);
}

int collide_blocks_per_sm_f32(int dim, int warps, int cap, bool one) {
  const size_t smem = (size_t)warps * warp_stage_bytes<T>(cap);
  if (dim == 1) return blocks_per_sm<1>(warps, smem, one);
  if (dim == 2) return blocks_per_sm<2>(warps, smem, one);
  return blocks_per_sm<3>(warps, smem, one);
}

cudaError_t configure_f32(int big_cap) {
  cudaError_t e = configure_dim<1>(big_cap);
  if (e == cudaSuccess) e = configure_dim<2>(big_cap);
  if (e == cudaSuccess) e = configure_dim<3>(big_cap);
  return e;
}

}  // namespace sp
