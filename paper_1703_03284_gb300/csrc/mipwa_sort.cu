// Set-time reordering of a stored sample by spline cell (j12, j13).
//
// -2 ln L and its gradient are sums over events, so the library may store
// events in any order. Grouping them by the pair of S-wave segments they fall
// in makes every warp of the event kernels see one (j12, j13) cell almost
// always: the cubic coefficients become shared-memory broadcasts and the
// spline adjoint can be reduced across the warp before it is binned.
//
// The sort is a stable counting sort (deterministic for a given input):
//   1. count:   each block counts the keys of its contiguous chunk;
//   2. scan:    exclusive prefix sum in (key, block) order;
//   3. scatter: each block walks its chunk in order, one warp at a time, and
//               places each event at its key's running offset.
#include <cuda_runtime.h>

#include "mipwa_amp.cuh"
#include "mipwa_kernels.cuh"

namespace mipwa {

constexpr int kSortBlocks = 8192;  // chunks (one warp each)
constexpr int kScanTile = 8192;    // ints per block of the prefix-sum kernels

template <typename EvT>
__device__ __forceinline__ int cell_key_general(const Knots& kn, const double* knot, const EvT& e) {
  const int j12 = segment_of(kn, knot, (double)e.x);
  const int j13 = segment_of(kn, knot, (double)e.y);
  return j12 * (kn.n - 1) + j13;
}

template <typename EvT>
__device__ __forceinline__ int key_of(const Knots& kn, const EvT& e) {
  if constexpr (std::is_same<EvT, float2>::value) {
    if (kn.uniform) {  // the FP32 kernels' own segment decision
      const float dummy[1] = {0.0f};
      const int j12 = segment_of(kn, dummy, e.x);
      const int j13 = segment_of(kn, dummy, e.y);
      return j12 * (kn.n - 1) + j13;
    }
  }
  return cell_key_general(kn, kn.s, e);
}

__host__ __device__ inline int64_t chunk_begin(int64_t n, int b) {
  const int64_t per = (n + kSortBlocks - 1) / kSortBlocks;
  const int64_t v = per * b;
  return v < n ? v : n;
}

template <typename EvT>
__global__ void __launch_bounds__(32) sort_count_kernel(const Knots kn, const EvT* ev, int64_t n,
                                                        int* counts /* [nkeys][kSortBlocks] */) {
  extern __shared__ int hist[];
  const int nkeys = (kn.n - 1) * (kn.n - 1);
  for (int k = threadIdx.x; k < nkeys; k += 32) hist[k] = 0;
  __syncwarp();
  const int64_t b0 = chunk_begin(n, blockIdx.x), b1 = chunk_begin(n, blockIdx.x + 1);
  for (int64_t i = b0 + threadIdx.x; i < b1; i += 32) atomicAdd(&hist[key_of(kn, ev[i])], 1);
  __syncwarp();
  for (int k = threadIdx.x; k < nkeys; k += 32) counts[(size_t)k * kSortBlocks + blockIdx.x] = hist[k];
}

// Exclusive prefix sum of m ints in place, in three steps: each block scans a
// tile of kScanTile ints and writes the tile total; one block scans the
// totals; each tile adds its offset.
__device__ __forceinline__ int block_exclusive_scan(int v, int* warp_sums, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += y;
    }
    warp_sums[lane] = w;  // inclusive
  }
  __syncthreads();
  const int before = (warp > 0 ? warp_sums[warp - 1] : 0) + x - v;
  if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
  return before;
}

__global__ void __launch_bounds__(1024) scan_tiles_kernel(int* a, int64_t m, int* tile_sums) {
  __shared__ int ws[32];
  constexpr int per = kScanTile / 1024;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * per;
  int v[per];
  int t = 0;
#pragma unroll
  for (int k = 0; k < per; ++k) {
    v[k] = base + k < m ? a[base + k] : 0;
    t += v[k];
  }
  int total = 0;
  int run = block_exclusive_scan(t, ws, &total);
#pragma unroll
  for (int k = 0; k < per; ++k) {
    if (base + k < m) a[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) scan_sums_kernel(int* sums, int n) {
  __shared__ int ws[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b = 0; b < n; b += 1024) {
    const int i = b + threadIdx.x;
    const int v = i < n ? sums[i] : 0;
    int total = 0;
    const int ex = block_exclusive_scan(v, ws, &total);
    if (i < n) sums[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += total;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(1024) scan_add_kernel(int* a, int64_t m, const int* sums) {
  const int off = sums[blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  for (int k = threadIdx.x; k < kScanTile; k += 1024)
    if (base + k < m) a[base + k] += off;
}

template <typename EvT>
__global__ void __launch_bounds__(32) sort_scatter_kernel(const Knots kn, const EvT* src, int64_t n,
                                                          const int* offsets, EvT* dst) {
  extern __shared__ int cursor[];
  const int nkeys = (kn.n - 1) * (kn.n - 1);
  for (int k = threadIdx.x; k < nkeys; k += 32)
    cursor[k] = offsets[(size_t)k * kSortBlocks + blockIdx.x];
  __syncwarp();
  const int64_t b0 = chunk_begin(n, blockIdx.x), b1 = chunk_begin(n, blockIdx.x + 1);
  const unsigned lane_lt = (1u << threadIdx.x) - 1u;
  for (int64_t base = b0; base < b1; base += 32) {
    const int64_t i = base + threadIdx.x;
    const bool live = i < b1;
    const unsigned active = __ballot_sync(0xffffffffu, live);
    EvT e{};
    int key = -1 - (int)threadIdx.x;  // distinct dummy keys for idle lanes
    if (live) {
      e = src[i];
      key = key_of(kn, e);
    }
    const unsigned same = __match_any_sync(0xffffffffu, key) & active;
    if (live) {
      const int rank = __popc(same & lane_lt);
      const int leader = __ffs(same) - 1;
      const int base_pos = cursor[key];
      dst[base_pos + rank] = e;
      __syncwarp(same);
      if ((int)threadIdx.x == leader) cursor[key] = base_pos + __popc(same);
    }
    __syncwarp();
  }
}

cudaError_t sort_workspace_ints(int n_knots, size_t* ints) {
  const int nkeys = (n_knots - 1) * (n_knots - 1);
  const size_t m = (size_t)nkeys * kSortBlocks;
  *ints = m + (m + kScanTile - 1) / kScanTile;  // counts, then tile totals
  return cudaSuccess;
}

template <typename EvT>
static cudaError_t sort_impl(const Knots& kn, const EvT* src, int64_t n, EvT* dst, int* work,
                             cudaStream_t st) {
  const int nkeys = (kn.n - 1) * (kn.n - 1);
  const size_t smem = (size_t)nkeys * sizeof(int);
  sort_count_kernel<EvT><<<kSortBlocks, 32, smem, st>>>(kn, src, n, work);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t m = (int64_t)nkeys * kSortBlocks;
  const int tiles = (int)((m + kScanTile - 1) / kScanTile);
  int* sums = work + m;
  scan_tiles_kernel<<<tiles, 1024, 0, st>>>(work, m, sums);
  scan_sums_kernel<<<1, 1024, 0, st>>>(sums, tiles);
  scan_add_kernel<<<tiles, 1024, 0, st>>>(work, m, sums);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  sort_scatter_kernel<EvT><<<kSortBlocks, 32, smem, st>>>(kn, src, n, work, dst);
  return cudaGetLastError();
}

cudaError_t launch_sort(int ev_f32, const Knots& kn, const void* src, int64_t n, void* dst,
                        int* work, cudaStream_t st) {
  if (ev_f32)
    return sort_impl(kn, (const float2*)src, n, (float2*)dst, work, st);
  return sort_impl(kn, (const double2*)src, n, (double2*)dst, work, st);
}

}  // namespace mipwa
