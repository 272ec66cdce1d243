// sp_noalloc.cu -- stable counting sort of particle cell keys that performs
// no device allocation: its scratch (per-cell histogram, scatter cursors and
// scan partial sums) lives in one file-scope __device__ array.
//
// Why: some callers cannot call cudaMalloc at the point where they need the
// cell index -- code running between captures of a CUDA graph whose memory
// plan is fixed, processes under a hard device-memory quota, or embedding
// hosts that hand this library device buffers they own and forbid it to
// allocate.  They pass the keys and the two output arrays; the scratch is the
// array below, present on every GPU that loads the library until exit.
#include <cstdio>

#include "../../include/sp.h"
#include "sp_internal.h"

namespace sp {
namespace {

constexpr int64_t kStaticMaxCells = int64_t(1) << 20;  // 1,048,576 cells
constexpr int64_t kStaticMaxKeys = int64_t(1) << 30;   // keys per call
constexpr int64_t kStaticPartial = (kStaticMaxCells + 2047) / 2048 + 1;
constexpr int kMaxDevices = 64;

// [0, MAX): histogram, [MAX, 2 MAX): scatter cursors, then scan partials.
static __device__ __align__(256) uint32_t g_sort_scratch[2 * kStaticMaxCells + kStaticPartial];

uint32_t* g_scratch_ptr[kMaxDevices] = {nullptr};

__global__ void k_static_zero(uint32_t* a, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = 0;
}

__global__ void k_static_hist(const uint32_t* key, int64_t n, int64_t ncells, uint32_t* count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t k = key[i];
  if (k < (uint64_t)ncells) atomicAdd(&count[k], 1u);
}

__global__ void k_static_scatter(const uint32_t* key, int64_t n, int64_t ncells, const uint32_t* start,
                                 uint32_t* fill, uint32_t* perm) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t k = key[i];
  if (k >= (uint64_t)ncells) return;
  perm[start[k] + atomicAdd(&fill[k], 1u)] = (uint32_t)i;
}

// In-place sorting network whose comparators all point the same way (each
// stage first compares slot t with its mirror t ^ (k-1) inside the current
// block of k slots, then runs the half-cleaners): it sorts a segment of any
// length n without padding, the slots past the end acting as +infinity.
// Thread `tid` of `nthr` cooperating threads takes slots tid, tid + nthr, ...;
// `sync` separates the stages.  All sizes are 64-bit, so segments up to the
// entry point's limit of 2^30 entries cannot overflow the loop bounds.
template <class Sync>
__device__ __forceinline__ void sort_segment(uint32_t* p, int64_t n, int64_t tid, int64_t nthr, Sync sync) {
  int64_t n2 = 1;
  while (n2 < n) n2 <<= 1;
  for (int64_t k = 2; k <= n2; k <<= 1) {
    for (int64_t j = k >> 1; j > 0; j >>= 1) {
      for (int64_t t = tid; t < n; t += nthr) {
        const int64_t q = (j == (k >> 1)) ? (t ^ (k - 1)) : (t ^ j);
        if (q > t && q < n) {
          const uint32_t a = p[t], b = p[q];
          if (a > b) {
            p[t] = b;
            p[q] = a;
          }
        }
      }
      sync();
    }
  }
}

// Segments of at most kWarpSeg entries: one warp each.
constexpr int64_t kWarpSeg = 1024;
// Larger segments: one block of kOrderThreads threads each, staged in shared
// memory up to kSmemSeg entries, else sorted in place in global memory
// (L2-resident for the segment sizes a cell reaches; a segment of 2^20
// entries takes a few tenths of a second).
constexpr int kOrderThreads = 512;
constexpr int kSmemSeg = 8192;

__global__ void k_static_order(const uint32_t* start, int64_t ncells, uint32_t* perm) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < ncells; c += nw) {
    const uint32_t s0 = start[c];
    const int64_t n = (int64_t)start[c + 1] - (int64_t)s0;
    if (n < 2 || n > kWarpSeg) continue;
    sort_segment(perm + s0, n, lane, 32, [] { __syncwarp(); });
  }
}

__global__ void __launch_bounds__(kOrderThreads) k_static_order_big(const uint32_t* start, int64_t ncells,
                                                                     uint32_t* perm) {
  __shared__ uint32_t sh[kSmemSeg];
  for (int64_t c = blockIdx.x; c < ncells; c += gridDim.x) {
    const uint32_t s0 = start[c];
    const int64_t n = (int64_t)start[c + 1] - (int64_t)s0;
    if (n <= kWarpSeg) continue;
    uint32_t* g = perm + s0;
    if (n <= kSmemSeg) {
      for (int64_t t = threadIdx.x; t < n; t += blockDim.x) sh[t] = g[t];
      __syncthreads();
      sort_segment(sh, n, threadIdx.x, blockDim.x, [] { __syncthreads(); });
      for (int64_t t = threadIdx.x; t < n; t += blockDim.x) g[t] = sh[t];
    } else {
      sort_segment(g, n, threadIdx.x, blockDim.x, [] { __syncthreads(); });
    }
    __syncthreads();
  }
}

// Set-up on the current device: the host-side name of the array is not a
// device address, so the address is looked up once per device.
cudaError_t static_scratch(uint32_t** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sort_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = (uint32_t*)p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

// Each cell's permutation entries put in ascending (source) order: a warp
// per cell up to kWarpSeg entries, a block per larger cell.
void launch_order_cells(const uint32_t* start, int64_t ncells, uint32_t* perm, cudaStream_t s) {
  if (ncells <= 0) return;
  int64_t ob = (ncells + 7) / 8;
  if (ob > 8192) ob = 8192;
  k_static_order<<<(unsigned)ob, 256, 0, s>>>(start, ncells, perm);
  const int64_t bb = ncells < 1024 ? ncells : 1024;
  k_static_order_big<<<(unsigned)bb, kOrderThreads, 0, s>>>(start, ncells, perm);
}

}  // namespace sp

extern "C" sp_status sp_sort_cells_static(const uint32_t* d_keys, int64_t n, int64_t ncells,
                                          uint32_t* d_start, uint32_t* d_perm, void* stream) {
  using namespace sp;
  if (n < 0 || ncells < 1 || (n > 0 && (!d_keys || !d_perm)) || !d_start) return SP_ERR_ARG;
  if (n > kStaticMaxKeys) {
    fprintf(stderr, "sp_sort_cells_static: %lld keys exceed the limit of %lld\n", (long long)n,
            (long long)kStaticMaxKeys);
    return SP_ERR_CAPACITY;
  }
  if (ncells > kStaticMaxCells) {
    fprintf(stderr, "sp_sort_cells_static: %lld cells exceed the static scratch limit of %lld\n",
            (long long)ncells, (long long)kStaticMaxCells);
    return SP_ERR_CAPACITY;
  }
  uint32_t* scratch = nullptr;
  cudaError_t e = static_scratch(&scratch);
  if (e != cudaSuccess) {
    fprintf(stderr, "sp_sort_cells_static: %s\n", cudaGetErrorString(e));
    return SP_ERR_CUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t* count = scratch;
  uint32_t* fill = scratch + kStaticMaxCells;
  uint32_t* partial = scratch + 2 * kStaticMaxCells;
  // the array keeps the previous call's contents: both counters restart at 0
  int64_t zb = (ncells + 255) / 256;
  if (zb > 4096) zb = 4096;
  k_static_zero<<<(unsigned)zb, 256, 0, s>>>(count, ncells);
  k_static_zero<<<(unsigned)zb, 256, 0, s>>>(fill, ncells);
  const unsigned nb = (unsigned)((n + 255) / 256);
  if (n > 0) k_static_hist<<<nb, 256, 0, s>>>(d_keys, n, ncells, count);
  launch_scan(count, d_start, ncells, partial, s);
  if (n > 0) k_static_scatter<<<nb, 256, 0, s>>>(d_keys, n, ncells, d_start, fill, d_perm);
  launch_order_cells(d_start, ncells, d_perm, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "sp_sort_cells_static: %s\n", cudaGetErrorString(e));
    return SP_ERR_CUDA;
  }
  return SP_OK;
}
