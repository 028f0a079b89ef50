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

constexpr int kSortBlocks = 1024;  // chunks (one warp each)

template <typename EvT>
__device__ __forceinline__ int cell_key_general(const Knots& kn, const double* knot, const EvT& e) {
  const int j12 = segment_of(kn, knot, (double)e.x);
  const int j13 = segment_of(kn, knot, (double)e.y);
  return j12 * (kn.n - 1) + j13;
}

template <typename EvT>
__device__ __forceinline__ int key_of(const Knots& kn, const EvT& e) {
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

// Exclusive scan of m ints in place, one block of 1024 threads: each thread
// scans a contiguous slice, then the slice totals are scanned.
__global__ void __launch_bounds__(1024) sort_scan_kernel(int* a, int64_t m) {
  __shared__ int tot[1024];
  const int64_t per = (m + 1023) / 1024;
  const int64_t s0 = per * threadIdx.x, s1 = (s0 + per < m) ? s0 + per : m;
  int t = 0;
  for (int64_t i = s0; i < s1; ++i) t += a[i];
  tot[threadIdx.x] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int k = 0; k < 1024; ++k) {
      const int v = tot[k];
      tot[k] = run;
      run += v;
    }
  }
  __syncthreads();
  int run = tot[threadIdx.x];
  for (int64_t i = s0; i < s1; ++i) {
    const int v = a[i];
    a[i] = run;
    run += v;
  }
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
  *ints = (size_t)nkeys * kSortBlocks;
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
  sort_scan_kernel<<<1, 1024, 0, st>>>(work, (int64_t)nkeys * kSortBlocks);
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
