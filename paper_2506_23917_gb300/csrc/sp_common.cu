// sp_common.cu -- precision-independent kernels of libsp: the exclusive
// scan of the cell histogram (counting sort by cell), the scatter that
// writes the slot -> source permutation, and the end-of-step bookkeeping.
#include <cstdint>

#include "sp_internal.h"

namespace sp {

namespace {
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t wsum[kScanThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t s = lane < kScanThreads / 32 ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kScanThreads / 32) wsum[lane] = s;
  }
  __syncthreads();
  const uint32_t before = w > 0 ? wsum[w - 1] : 0;
  *total = wsum[kScanThreads / 32 - 1];
  __syncthreads();
  return before + x - v;
}

__global__ void k_scan_reduce(const uint32_t* in, int64_t n, uint32_t* partial) {
  const int64_t base = (int64_t)blockIdx.x * kTile;
  uint32_t s = 0;
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t j = base + (int64_t)i * kScanThreads + threadIdx.x;
    if (j < n) s += in[j];
  }
  uint32_t tot;
  block_excl_scan(s, &tot);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// out[j] = sum of in[0..j), out[n] = total.  Each thread owns kScanItems
// consecutive elements of the block's tile.
__global__ void k_scan_down(const uint32_t* in, uint32_t* out, int64_t n, const uint32_t* partial,
                            int64_t nb) {
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t j = base + i;
    v[i] = j < n ? in[j] : 0;
    s += v[i];
  }
  // the block's offset: the sum of the earlier blocks' totals (read here
  // rather than scanned by a separate launch)
  uint32_t pre = 0;
  for (int64_t b = threadIdx.x; b < (int64_t)blockIdx.x; b += kScanThreads) pre += partial[b];
  uint32_t off;
  block_excl_scan(pre, &off);
  uint32_t tot;
  uint32_t run = off + block_excl_scan(s, &tot);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t j = base + i;
    if (j < n) out[j] = run;
    run += v[i];
  }
  if (blockIdx.x == nb - 1 && threadIdx.x == 0) out[n] = off + tot;
}

// perm[start[key] + rank] = source index.  The histogram itself is the
// cursor: warp-aggregated atomic decrements hand out each cell's positions
// from its end, and leave the histogram at zero for the next step's counts.
// The order inside a cell is arbitrary here and restored to source order by
// the collision kernel when the run is reproducible.
constexpr int kScatterPer = 4;  // elements per thread, strided by the block size
__global__ void k_scatter(const uint32_t* key, const uint32_t* start, uint32_t* count, uint32_t* perm,
                          const uint32_t* Mtot, int64_t cap) {
  // each thread's kScatterPer elements are requested together, so that their
  // load -> match -> atomic -> store chains overlap
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x * kScatterPer + threadIdx.x;
  const int64_t M = (int64_t)*Mtot;
  const int lane = threadIdx.x & 31;
  uint32_t k[kScatterPer], base[kScatterPer], sk[kScatterPer];
  unsigned peers[kScatterPer];
#pragma unroll
  for (int j = 0; j < kScatterPer; ++j) {
    const int64_t i = i0 + (int64_t)j * blockDim.x;
    k[j] = (i < M && i < cap) ? key[i] : kSentinel;
  }
#pragma unroll
  for (int j = 0; j < kScatterPer; ++j) {
    peers[j] = __match_any_sync(0xFFFFFFFFu, k[j]);
    sk[j] = k[j] != kSentinel ? __ldg(&start[k[j]]) : 0u;
    base[j] = 0;
    if (k[j] != kSentinel && lane == __ffs(peers[j]) - 1)
      base[j] = atomicSub(&count[k[j]], (uint32_t)__popc(peers[j])) - (uint32_t)__popc(peers[j]);
  }
#pragma unroll
  for (int j = 0; j < kScatterPer; ++j) {
    const uint32_t b = __shfl_sync(0xFFFFFFFFu, base[j], __ffs(peers[j]) - 1);
    if (k[j] != kSentinel) {
      const uint32_t rank = __popc(peers[j] & ((1u << lane) - 1u));
      perm[sk[j] + b + rank] = (uint32_t)(i0 + (int64_t)j * blockDim.x);
    }
  }
}

__global__ void k_step_finalize(const InstParams* P, int n_inst, double* dt_cur,
                                unsigned long long* dt_min, uint32_t* step, uint32_t* Mcur,
                                uint32_t* Mtot, const uint32_t* start_new, int64_t NC,
                                const uint32_t* goff, const uint32_t* gcount, int64_t n_ghost,
                                uint32_t* big_count, uint32_t* ticket, uint32_t* nbatch,
                                double* surf_time, unsigned long long* cyc) {
  const uint32_t st = *step;  // index of the step that just ran (read by all first)
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t inj = n_ghost > 0 ? goff[n_ghost - 1] + gcount[n_ghost - 1] : 0u;
    const uint32_t old = *Mcur;
    *Mtot = old + inj;
    *Mcur = start_new[NC];
    *step = *step + 1u;
    *big_count = 0u;
    *ticket = 0u;
    for (int k = 0; k < kBatchClasses; ++k) nbatch[k] = 0u;
    // unit of the cost bytes: 1/16 of this step's mean cycles per particle
    // over all batches (at least 1)
    const unsigned long long u = cyc[1] > 0 ? cyc[0] / (16ull * cyc[1]) : ~0ull;
    cyc[2] = u > 0 ? u : 1ull;
    cyc[0] = 0ull;
    cyc[1] = 0ull;
  }
  for (int i = threadIdx.x; i < n_inst; i += blockDim.x) {
    const unsigned long long inf = 0x7FF0000000000000ull;
    if ((int64_t)st >= (int64_t)P[i].n_steady) surf_time[i] += dt_cur[i];
    if (P[i].dt_fixed > 0) {
      dt_cur[i] = P[i].dt_fixed;
    } else if (dt_min[i] != inf) {
      dt_cur[i] = P[i].cfl * __longlong_as_double((long long)dt_min[i]);
    }
    dt_min[i] = inf;
  }
}
// Work plan of a step: consecutive cells are grouped into batches whose
// particles fit a warp's staging area (at most 32 cells each); cells above
// it go to the big-cell list.  One warp per 32-cell chunk.  Each batch is
// classed by its predicted cost, sum over its cells of N_c w_c, where w_c is
// the cell's cost byte from the last step (its batch's cycles per particle
// in units of 1/16 of the step's mean; 16 before any measurement): in units
// of a full batch at the mean cost (16 cap), classes >= 4, [2, 4),
// [1.5, 2), [1, 1.5), [3/4, 1), [1/2, 3/4), [1/4, 1/2), [1/8, 1/4) and
// below, most expensive first.  The collision kernel hands out the classes
// in that order (longest processing time first), so that the batches still
// running when the list runs out are short ones and the SMs finish the
// launch together: cells where most particles are resampled with many
// rejections, or with many collision candidates, cost several times the
// mean per particle, and a warp takes only a few batches per launch.
// Class k's list is batches[k NC ...].  Batches are independent: their
// order changes no result.
__global__ void k_plan(const uint32_t* start, const uint8_t* cost, int64_t NC, int cap, int split, uint2* batches,
                       uint32_t* nbatch, uint32_t* big_list, uint32_t* big_count) {
  // per block: the batches of each class (shared atomics), then one global
  // atomic per class for the block's place in the class list
  __shared__ uint32_t cnt[kBatchClasses], base[kBatchClasses];
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  const int64_t nw = (int64_t)gridDim.x * wpb;
  const int64_t nchunks = (NC + 31) / 32;
  const int64_t iters = (nchunks + nw - 1) / nw;  // the same for every warp of the block
  for (int64_t it = 0; it < iters; ++it) {
    const int64_t chunk = it * nw + (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5);
    if (threadIdx.x < kBatchClasses) cnt[threadIdx.x] = 0;
    __syncthreads();
    int nb = 0;
    uint2 mine = make_uint2(0, 0);
    int mine_cls = 0;
    uint32_t mine_at = 0;
    if (chunk < nchunks) {
      const int64_t c0 = chunk * 32;
      const int nc = (int)((NC - c0) < 32 ? (NC - c0) : 32);
      // inclusive prefix sums of the particle counts and the predicted costs
      const int64_t nl = lane < nc ? (int64_t)(start[c0 + lane + 1] - start[c0 + lane]) : 0;
      const int64_t wl = lane < nc ? (cost[c0 + lane] ? (int64_t)cost[c0 + lane] : 16) : 0;
      // lanes of the per-cell sums (split cells; at most 32 per batch)
      int lcum = lane < nc ? cell_lanes((int)(nl < 0x7FFFFFFF ? nl : 0x7FFFFFFF), split) : 0;
      int64_t cum = nl, ccum = nl * wl;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xFFFFFFFFu, cum, o);
        const int64_t z = __shfl_up_sync(0xFFFFFFFFu, ccum, o);
        const int w = __shfl_up_sync(0xFFFFFFFFu, lcum, o);
        if (lane >= o) {
          cum += y;
          ccum += z;
          lcum += w;
        }
      }
      int kk = 0;
      while (kk < nc) {
        const int64_t before = kk > 0 ? __shfl_sync(0xFFFFFFFFu, cum, kk - 1) : 0;
        const int lbefore = kk > 0 ? __shfl_sync(0xFFFFFFFFu, lcum, kk - 1) : 0;
        const unsigned fit = __ballot_sync(0xFFFFFFFFu, lane >= kk && lane < nc && cum - before <= cap &&
                                                          lcum - lbefore <= 32);
        const int G = __popc(fit);
        if (G == 0) {  // the cell alone exceeds the staging area: big-cell list
          if (lane == 0) {
            const uint32_t i = atomicAdd(big_count, 1u);
            big_list[i] = (uint32_t)(c0 + kk);
          }
          kk += 1;
          continue;
        }
        const int64_t cb = kk > 0 ? __shfl_sync(0xFFFFFFFFu, ccum, kk - 1) : 0;
        const int64_t cst = __shfl_sync(0xFFFFFFFFu, ccum, kk + G - 1) - cb;
        if (lane == nb) {
          mine = make_uint2((uint32_t)(c0 + kk), (uint32_t)G);
          const int64_t u = 16 * (int64_t)cap;  // a full batch at the mean cost
          int cls;
          if (cst >= 4 * u) cls = 0;
          else if (cst >= 2 * u) cls = 1;
          else if (2 * cst >= 3 * u) cls = 2;
          else if (cst >= u) cls = 3;
          else if (4 * cst >= 3 * u) cls = 4;
          else if (2 * cst >= u) cls = 5;
          else if (4 * cst >= u) cls = 6;
          else if (8 * cst >= u) cls = 7;
          else cls = 8;
          mine_cls = cls;
        }
        ++nb;
        kk += G;
      }
      if (lane < nb) mine_at = atomicAdd(&cnt[mine_cls], 1u);
    }
    __syncthreads();
    if (threadIdx.x < kBatchClasses)
      base[threadIdx.x] = cnt[threadIdx.x] ? atomicAdd(&nbatch[threadIdx.x], cnt[threadIdx.x]) : 0u;
    __syncthreads();
    if (lane < nb) batches[(int64_t)mine_cls * NC + base[mine_cls] + mine_at] = mine;
    __syncthreads();
  }
}

}  // namespace

void launch_plan(const uint32_t* start, const uint8_t* cost, int64_t NC, int cap, int split, uint2* batches,
                 uint32_t* nbatch, uint32_t* big_list, uint32_t* big_count, cudaStream_t s) {
  const int64_t chunks = (NC + 31) / 32;
  int64_t g = (chunks + 7) / 8;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  k_plan<<<(unsigned)g, 256, 0, s>>>(start, cost, NC, cap, split, batches, nbatch, big_list, big_count);
}

int64_t scan_partial_size(int64_t n) { return (n + kTile - 1) / kTile + 1; }

void launch_scan(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* partial, cudaStream_t s) {
  const int64_t nb = (n + kTile - 1) / kTile;
  if (nb == 0) {
    cudaMemsetAsync(out, 0, sizeof(uint32_t), s);
    return;
  }
  k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, partial);
  k_scan_down<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, partial, nb);
}

void launch_scatter(const uint32_t* key, const uint32_t* start, uint32_t* count, uint32_t* perm,
                    const uint32_t* Mtot, int64_t cap, cudaStream_t s) {
  const int64_t g = (cap + 256 * kScatterPer - 1) / (256 * kScatterPer);
  k_scatter<<<(unsigned)(g > 0 ? g : 1), 256, 0, s>>>(key, start, count, perm, Mtot, cap);
}

void launch_step_finalize(const InstParams* P, int n_inst, double* dt_cur,
                          unsigned long long* dt_min, uint32_t* step, uint32_t* Mcur,
                          uint32_t* Mtot, const uint32_t* start_new, int64_t NC,
                          const uint32_t* goff, const uint32_t* gcount, int64_t n_ghost,
                          uint32_t* big_count, uint32_t* ticket, uint32_t* nbatch,
                          double* surf_time, unsigned long long* cyc, cudaStream_t s) {
  k_step_finalize<<<1, 256, 0, s>>>(P, n_inst, dt_cur, dt_min, step, Mcur, Mtot, start_new, NC,
                                    goff, gcount, n_ghost, big_count, ticket, nbatch, surf_time, cyc);
}

}  // namespace sp
