// Set-time reordering of a stored sample by spline cell (j12, j13).
//
// -2 ln L and its gradient are sums over events, so the library may store
// events in any order. Grouping them by the pair of S-wave segments they fall
// in makes every warp of the event kernels see one (j12, j13) cell almost
// always: the cubic coefficients become shared-memory broadcasts and the spline
// adjoint can be reduced across the warp before it is binned.
//
// Two passes of a stable counting sort (deterministic for a given input): by
// j12 alone, then by the cell key j12 (N-1) + j13. The result is the single
// sort by cell key (both passes are stable), but every write goes to a long
// run: in the first pass a chunk of events spreads over N-1 keys only, and in
// the second a chunk lies almost entirely in one j12 bucket, so it again
// meets about N-1 keys (a single pass spreads each chunk over (N-1)^2 keys and
// writes runs of a few events). Each pass:
//   1. count:   each warp counts the keys of its contiguous chunk into its
//               own row of a [chunk][key] table (the first pass of a new
//               sample also counts the events outside the Dalitz plot);
//   2. offsets: the table becomes, in place, each (block, key)'s first output
//               position: all events of lower keys, plus the events of the
//               same key in earlier blocks (column sums over groups of
//               blocks, one scan over keys, then the running sums per group);
//   3. scatter: each warp walks its chunk in order, 32 events at a time, and
//               places each event at its key's running offset.
// kSortWarps chunks share a thread block, each warp with its own
// shared-memory table (measured on GB300: one warp per block is fastest; eight
// made the first scatter 15 % slower).
#include <cuda_runtime.h>

#include "mipwa_amp.cuh"
#include "mipwa_kernels.cuh"

namespace mipwa {

constexpr int kSortBlocks = 8192;  // chunks (one warp each); a multiple of kGroup
constexpr int kSortWarps = 1;      // chunks per thread block (one warp each)

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

// Sort key of a pass: the cell key (FULL) or its j12 part.
template <typename EvT, bool FULL>
__device__ __forceinline__ int pass_key(const Knots& kn, const EvT& e) {
  const int k = key_of(kn, e);
  return FULL ? k : k / (kn.n - 1);
}

template <bool FULL>
__host__ __device__ inline int pass_keys(int n_knots) {
  return FULL ? (n_knots - 1) * (n_knots - 1) : n_knots - 1;
}

__host__ __device__ inline int64_t chunk_begin(int64_t n, int b) {
  const int64_t per = (n + kSortBlocks - 1) / kSortBlocks;
  const int64_t v = per * b;
  return v < n ? v : n;
}

// CHECK: also count the events outside the Dalitz plot into *outside (their
// keys are clamped segments, so the histogram stays in range).
template <typename EvT, bool FULL, bool CHECK>
__global__ void __launch_bounds__(32 * kSortWarps)
    sort_count_kernel(const Model m, const EvT* ev, int64_t n, int chunk0,
                      int* counts /* [kSortBlocks][nkeys] */, unsigned long long* outside) {
  extern __shared__ int hist_all[];
  const Knots& kn = m.kn;
  const int nkeys = pass_keys<FULL>(kn.n);
  const int lane = threadIdx.x & 31;
  const int chunk = chunk0 + blockIdx.x * kSortWarps + (threadIdx.x >> 5);
  int* hist = hist_all + (threadIdx.x >> 5) * nkeys;
  for (int k = lane; k < nkeys; k += 32) hist[k] = 0;
  __syncwarp();
  const int64_t b0 = chunk_begin(n, chunk), b1 = chunk_begin(n, chunk + 1);
  unsigned int out = 0;
  for (int64_t i = b0 + lane; i < b1; i += 32) {
    const EvT e = ev[i];
    atomicAdd(&hist[pass_key<EvT, FULL>(kn, e)], 1);
    if constexpr (CHECK) {
      bool in;
      if constexpr (std::is_same<EvT, float2>::value) in = inside_plot_fast(m, e.x, e.y);
      else in = inside_plot(m, e.x, e.y);
      out += in ? 0u : 1u;
    }
  }
  __syncwarp();
  for (int k = lane; k < nkeys; k += 32) counts[(size_t)chunk * nkeys + k] = hist[k];
  if constexpr (CHECK) {
    for (int off = 16; off > 0; off >>= 1) out += __shfl_down_sync(0xffffffffu, out, off);
    if (lane == 0 && out) atomicAdd(outside, (unsigned long long)out);
  }
}

constexpr int kGroup = 64;                        // blocks per column-sum group
constexpr int kGroups = kSortBlocks / kGroup;     // 128

// group_sum[g][k] = sum of counts[b][k] over the blocks b of group g.
__global__ void __launch_bounds__(256) sort_group_sums(const int* counts, int nkeys, int* group_sum) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int g = blockIdx.y;
  if (k >= nkeys) return;
  int t = 0;
  for (int b = g * kGroup; b < (g + 1) * kGroup; ++b) t += counts[(size_t)b * nkeys + k];
  group_sum[(size_t)g * nkeys + k] = t;
}

// One block: per key, the exclusive scan of its group sums (in place) and its
// total; then the exclusive scan of the totals over keys -> key_start.
__global__ void __launch_bounds__(1024) sort_key_starts(int* group_sum, int nkeys, int* key_start) {
  __shared__ int ws[32];
  __shared__ int carry;
  for (int k = threadIdx.x; k < nkeys; k += blockDim.x) {
    int run = 0;
    for (int g = 0; g < kGroups; ++g) {
      const int v = group_sum[(size_t)g * nkeys + k];
      group_sum[(size_t)g * nkeys + k] = run;
      run += v;
    }
    key_start[k] = run;  // total for now
  }
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b = 0; b < nkeys; b += 1024) {
    const int i = b + threadIdx.x;
    const int v = i < nkeys ? key_start[i] : 0;
    // block-wide exclusive scan
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, off);
      if (lane >= off) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int w = ws[lane];
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, w, off);
        if (lane >= off) w += y;
      }
      ws[lane] = w;
    }
    __syncthreads();
    const int ex = (warp > 0 ? ws[warp - 1] : 0) + x - v;
    const int total = ws[31];
    __syncthreads();
    if (i < nkeys) key_start[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += total;
    __syncthreads();
  }
}

// counts[b][k] -> key_start[k] + group prefix + running sum within the group.
__global__ void __launch_bounds__(256) sort_offsets(int* counts, int nkeys, const int* group_sum,
                                                    const int* key_start) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int g = blockIdx.y;
  if (k >= nkeys) return;
  int run = key_start[k] + group_sum[(size_t)g * nkeys + k];
  for (int b = g * kGroup; b < (g + 1) * kGroup; ++b) {
    const int v = counts[(size_t)b * nkeys + k];
    counts[(size_t)b * nkeys + k] = run;
    run += v;
  }
}

template <typename EvT, bool FULL>
__global__ void __launch_bounds__(32 * kSortWarps)
    sort_scatter_kernel(const Knots kn, const EvT* src, int64_t n, const int* offsets, EvT* dst) {
  extern __shared__ int cursor_all[];
  const int nkeys = pass_keys<FULL>(kn.n);
  const int lane = threadIdx.x & 31, chunk = blockIdx.x * kSortWarps + (threadIdx.x >> 5);
  int* cursor = cursor_all + (threadIdx.x >> 5) * nkeys;
  for (int k = lane; k < nkeys; k += 32) cursor[k] = offsets[(size_t)chunk * nkeys + k];
  __syncwarp();
  const int64_t b0 = chunk_begin(n, chunk), b1 = chunk_begin(n, chunk + 1);
  const unsigned lane_lt = (1u << lane) - 1u;
  for (int64_t base = b0; base < b1; base += 32) {
    const int64_t i = base + lane;
    const bool live = i < b1;
    const unsigned active = __ballot_sync(0xffffffffu, live);
    EvT e{};
    int key = -1 - lane;  // distinct dummy keys for idle lanes
    if (live) {
      e = src[i];
      key = pass_key<EvT, FULL>(kn, e);
    }
    const unsigned same = __match_any_sync(0xffffffffu, key) & active;
    if (live) {
      const int rank = __popc(same & lane_lt);
      const int leader = __ffs(same) - 1;
      const int base_pos = cursor[key];
      dst[base_pos + rank] = e;
      __syncwarp(same);
      if (lane == leader) cursor[key] = base_pos + __popc(same);
    }
    __syncwarp();
  }
}

// first[k], last[k] = the index range of key k in a sample grouped by key
// (both zeroed beforehand: an empty key keeps 0, 0).
template <typename EvT>
__global__ void __launch_bounds__(256) cell_bounds_kernel(const Knots kn, const EvT* ev, int64_t n,
                                                          int* first, int* last) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int k = key_of(kn, ev[i]);
    if (i == 0 || key_of(kn, ev[i - 1]) != k) first[k] = (int)i;
    if (i == n - 1 || key_of(kn, ev[i + 1]) != k) last[k] = (int)(i + 1);
  }
}

cudaError_t launch_cell_bounds(int ev_f32, const Knots& kn, const void* ev, int64_t n, int* first,
                               int* last, int grid, cudaStream_t st) {
  const int nkeys = (kn.n - 1) * (kn.n - 1);
  cudaError_t e = cudaMemsetAsync(first, 0, nkeys * sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(last, 0, nkeys * sizeof(int), st);
  if (e != cudaSuccess || n == 0) return e;
  if (ev_f32)
    cell_bounds_kernel<float2><<<grid, 256, 0, st>>>(kn, (const float2*)ev, n, first, last);
  else
    cell_bounds_kernel<double2><<<grid, 256, 0, st>>>(kn, (const double2*)ev, n, first, last);
  return cudaGetLastError();
}

cudaError_t sort_workspace_ints(int n_knots, size_t* ints) {
  const int nkeys = (n_knots - 1) * (n_knots - 1);
  // counts [kSortBlocks][nkeys], group sums [kGroups][nkeys], key starts [nkeys]
  *ints = (size_t)nkeys * (kSortBlocks + kGroups + 1);
  return cudaSuccess;
}

// Count the chunks [c0, c1) (multiples of kSortWarps).
template <typename EvT, bool FULL, bool CHECK>
static cudaError_t count_pass(const Model& m, const EvT* src, int64_t n, int* work,
                              unsigned long long* outside, cudaStream_t st, int c0 = 0,
                              int c1 = kSortBlocks) {
  const size_t smem = (size_t)kSortWarps * pass_keys<FULL>(m.kn.n) * sizeof(int);
  auto kern = sort_count_kernel<EvT, FULL, CHECK>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(c1 - c0) / kSortWarps, 32 * kSortWarps, smem, st>>>(m, src, n, c0, work, outside);
  return cudaGetLastError();
}

// Offsets and scatter of one pass whose counts are in `work`.
template <typename EvT, bool FULL>
static cudaError_t finish_pass(const Knots& kn, const EvT* src, int64_t n, EvT* dst, int* work,
                               cudaStream_t st) {
  const int nkeys = pass_keys<FULL>(kn.n);
  const size_t smem = (size_t)kSortWarps * nkeys * sizeof(int);
  int* group_sum = work + (size_t)nkeys * kSortBlocks;
  int* key_start = group_sum + (size_t)nkeys * kGroups;
  const dim3 cgrid((nkeys + 255) / 256, kGroups);
  sort_group_sums<<<cgrid, 256, 0, st>>>(work, nkeys, group_sum);
  sort_key_starts<<<1, 1024, 0, st>>>(group_sum, nkeys, key_start);
  sort_offsets<<<cgrid, 256, 0, st>>>(work, nkeys, group_sum, key_start);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  auto kern = sort_scatter_kernel<EvT, FULL>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<kSortBlocks / kSortWarps, 32 * kSortWarps, smem, st>>>(kn, src, n, work, dst);
  return cudaGetLastError();
}

// Both passes after the first count: src -> tmp by j12, tmp -> dst by cell.
template <typename EvT>
static cudaError_t sort_rest(const Model& m, const EvT* src, int64_t n, EvT* tmp, EvT* dst,
                             int* work, cudaStream_t st) {
  cudaError_t e = finish_pass<EvT, false>(m.kn, src, n, tmp, work, st);
  if (e == cudaSuccess) e = count_pass<EvT, true, false>(m, tmp, n, work, nullptr, st);
  if (e == cudaSuccess) e = finish_pass<EvT, true>(m.kn, tmp, n, dst, work, st);
  return e;
}

cudaError_t launch_sort_count_checked(int ev_f32, const Model& m, const void* src, int64_t n,
                                      int* work, unsigned long long* outside, cudaStream_t st,
                                      int piece, int n_pieces) {
  const int c0 = kSortBlocks / n_pieces * piece, c1 = kSortBlocks / n_pieces * (piece + 1);
  if (ev_f32)
    return count_pass<float2, false, true>(m, (const float2*)src, n, work, outside, st, c0, c1);
  return count_pass<double2, false, true>(m, (const double2*)src, n, work, outside, st, c0, c1);
}

int64_t sort_piece_begin(int64_t n, int piece, int n_pieces) {
  return chunk_begin(n, kSortBlocks / n_pieces * piece);
}

cudaError_t launch_sort_rest(int ev_f32, const Model& m, const void* src, int64_t n, void* tmp,
                             void* dst, int* work, cudaStream_t st) {
  if (ev_f32)
    return sort_rest(m, (const float2*)src, n, (float2*)tmp, (float2*)dst, work, st);
  return sort_rest(m, (const double2*)src, n, (double2*)tmp, (double2*)dst, work, st);
}

cudaError_t launch_sort(int ev_f32, const Model& m, const void* src, int64_t n, void* tmp,
                        void* dst, int* work, cudaStream_t st) {
  cudaError_t e;
  if (ev_f32) e = count_pass<float2, false, false>(m, (const float2*)src, n, work, nullptr, st);
  else e = count_pass<double2, false, false>(m, (const double2*)src, n, work, nullptr, st);
  if (e != cudaSuccess) return e;
  return launch_sort_rest(ev_f32, m, src, n, tmp, dst, work, st);
}

}  // namespace mipwa
