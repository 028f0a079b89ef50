// Set-time reordering of a stored sample by spline cell (j12, j13).
//
// -2 ln L and its gradient are sums over events, so the library may store
// events in any order. Grouping them by the pair of S-wave segments they fall
// in makes every warp of the event kernels see one (j12, j13) cell almost
// always: the cubic coefficients become shared-memory broadcasts and the spline
// adjoint can be reduced across the warp before it is binned.
//
// A least-significant-digit sort with the segment indices as digits: a stable
// counting pass by j13, then a stable counting pass by j12, which leaves the
// events in the order of the cell key j12 (N-1) + j13, events with equal keys
// in the order they had before (deterministic for a given input). Each pass
// has N-1 <= 63 keys:
//   1. count:   a thread block counts the keys of one contiguous chunk into
//               the chunk's row of a [chunk][key] table (the first pass of a
//               new sample also counts the events outside the Dalitz plot);
//   2. offsets: the table becomes, in place, each (chunk, key)'s first output
//               position: all events of lower keys, plus the events of the
//               same key in earlier chunks (column sums over groups of
//               chunks, one scan over keys, then the running sums per group);
//   3. scatter: a thread block walks its chunk in tiles of consecutive
//               events, orders each tile by key in shared memory (stably:
//               warp by warp, row by row, lane by lane) and writes each key's
//               run of the tile to that key's running output position, so that
//               neighbouring threads store neighbouring events.
#include <cuda_runtime.h>

#include "mipwa_amp.cuh"
#include "mipwa_kernels.cuh"

namespace mipwa {

constexpr int kSortBlocks = 152 * 32;  // chunks; a multiple of kGroup and of 2^7
constexpr int kMaxKeys = 64;           // keys of one pass: N-1 segments
static_assert(kMaxKnots - 1 <= kMaxKeys, "a pass key must fit the tables");

// events per thread loaded together (64 B of them in flight per thread)
template <typename EvT>
constexpr int kBatch = 64 / (int)sizeof(EvT);

// The S-wave segment of one invariant as the event kernels decide it: FP32
// arithmetic for float events on evenly spaced knots, FP64 otherwise.
__device__ __forceinline__ int seg_of(const Knots& kn, float v) {
  if (kn.uniform) {
    const float dummy[1] = {0.0f};
    return segment_of(kn, dummy, v);
  }
  return segment_of(kn, kn.s, (double)v);
}

__device__ __forceinline__ int seg_of(const Knots& kn, double v) {
  return segment_of(kn, kn.s, v);
}

template <typename EvT>
__device__ __forceinline__ int key_of(const Knots& kn, const EvT& e) {
  return seg_of(kn, e.x) * (kn.n - 1) + seg_of(kn, e.y);
}

// Key of a pass: the segment of s12 (DIGIT 0) or of s13 (DIGIT 1).
template <typename EvT, int DIGIT>
__device__ __forceinline__ int digit_of(const Knots& kn, const EvT& e) {
  return DIGIT == 0 ? seg_of(kn, e.x) : seg_of(kn, e.y);
}

__host__ __device__ inline int64_t chunk_begin(int64_t n, int b) {
  const int64_t per = (n + kSortBlocks - 1) / kSortBlocks;
  const int64_t v = per * b;
  return v < n ? v : n;
}

// One thread block per chunk (kCountThreads threads sharing its histogram):
// the count is order-free, so a chunk may be counted by many warps, which
// keeps the SMs full when only a quarter of the chunks (one piece of a sample
// still arriving) is counted. CHECK: also count the events outside the Dalitz
// plot into *outside (their keys are clamped segments, so the histogram stays
// in range).
constexpr int kCountThreads = 256;

template <typename EvT, int DIGIT, bool CHECK>
__global__ void __launch_bounds__(kCountThreads, 4)
    sort_count_kernel(const Model m, const EvT* __restrict__ ev, int64_t n, int chunk0,
                      int* counts /* [kSortBlocks][N-1] */, unsigned long long* outside) {
  __shared__ int hist[kMaxKeys];
  constexpr int B = kBatch<EvT>;
  const Knots& kn = m.kn;
  const int nkeys = kn.n - 1;
  const int chunk = chunk0 + blockIdx.x;
  if (threadIdx.x < kMaxKeys) hist[threadIdx.x] = 0;
  __syncthreads();
  const int64_t b0 = chunk_begin(n, chunk), b1 = chunk_begin(n, chunk + 1);
  unsigned int out = 0;
  for (int64_t base = b0 + threadIdx.x; base < b1; base += kCountThreads * B) {
    EvT e[B];
#pragma unroll
    for (int u = 0; u < B; ++u)
      if (base + kCountThreads * u < b1) e[u] = ev[base + kCountThreads * u];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      if (base + kCountThreads * u < b1) {
        atomicAdd(&hist[digit_of<EvT, DIGIT>(kn, e[u])], 1);
        if constexpr (CHECK) {
          bool in;
          if constexpr (std::is_same<EvT, float2>::value) in = inside_plot_fast(m, e[u].x, e[u].y);
          else in = inside_plot(m, e[u].x, e[u].y);
          out += in ? 0u : 1u;
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < nkeys) counts[(size_t)chunk * nkeys + threadIdx.x] = hist[threadIdx.x];
  if constexpr (CHECK) {
    for (int off = 16; off > 0; off >>= 1) out += __shfl_down_sync(0xffffffffu, out, off);
    if ((threadIdx.x & 31) == 0 && out) atomicAdd(outside, (unsigned long long)out);
  }
}

constexpr int kGroup = 64;                        // blocks per column-sum group
constexpr int kGroups = kSortBlocks / kGroup;     // 76
static_assert(kSortBlocks % kGroup == 0, "kGroup must divide kSortBlocks");

// group_sum[g][k] = sum of counts[b][k] over the blocks b of group g.
__global__ void __launch_bounds__(256) sort_group_sums(const int* counts, int nkeys, int* group_sum) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int g = blockIdx.y;
  if (k >= nkeys) return;
  int t = 0;
  for (int b = g * kGroup; b < (g + 1) * kGroup; ++b) t += counts[(size_t)b * nkeys + k];
  group_sum[(size_t)g * nkeys + k] = t;
}

// group sums read together before any is overwritten
constexpr int kScanChunk = 19;
static_assert(kGroups % kScanChunk == 0, "kScanChunk must divide kGroups");

// One block: per key, the exclusive scan of its group sums (in place) and its
// total; then the exclusive scan of the totals over keys -> key_start.
__global__ void __launch_bounds__(1024) sort_key_starts(int* group_sum, int nkeys, int* key_start) {
  __shared__ int ws[32];
  __shared__ int carry;
  for (int k = threadIdx.x; k < nkeys; k += blockDim.x) {
    int run = 0;
    for (int g0 = 0; g0 < kGroups; g0 += kScanChunk) {
      int v[kScanChunk];
#pragma unroll
      for (int g = 0; g < kScanChunk; ++g) v[g] = group_sum[(size_t)(g0 + g) * nkeys + k];
#pragma unroll
      for (int g = 0; g < kScanChunk; ++g) {
        group_sum[(size_t)(g0 + g) * nkeys + k] = run;
        run += v[g];
      }
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
  int v[kGroup];  // read the group's column before overwriting it
#pragma unroll
  for (int b = 0; b < kGroup; ++b) v[b] = counts[(size_t)(g * kGroup + b) * nkeys + k];
  int run = key_start[k] + group_sum[(size_t)g * nkeys + k];
#pragma unroll
  for (int b = 0; b < kGroup; ++b) {
    counts[(size_t)(g * kGroup + b) * nkeys + k] = run;
    run += v[b];
  }
}

// Scatter of one pass: one thread block per chunk, tiles of kTileRows rows of
// 32 consecutive events per warp (a warp's rows are consecutive, warp w after
// warp w-1), so the order (warp, row, lane) is the event order.
constexpr int kScatterThreads = 256;
constexpr int kScatterWarps = kScatterThreads / 32;
template <typename EvT>
constexpr int kTileRows = kBatch<EvT>;
template <typename EvT>
constexpr int kTile = kScatterThreads * kTileRows<EvT>;

// A weight per event (PAY) travels with it: the events' scalar type.
template <typename EvT>
using Scalar = decltype(EvT::x);

template <typename EvT, bool PAY>
struct ScatterSmem {
  EvT stage[kTile<EvT>];                // the tile in key order
  Scalar<EvT> wstage[PAY ? kTile<EvT> : 1];  // and the weight of each (PAY)
  unsigned char skey[kTile<EvT>];       // and the key of each
  int whist[kScatterWarps][kMaxKeys];   // per warp: count, then its first tile position
  int delta[kMaxKeys];                  // output position - tile position, per key
  int cursor[kMaxKeys];                 // next output position of each key
};

// One tile of tn events starting at src (FULL: tn = kTile, no bounds checks);
// PAY: their weights from wsrc go to wdst alongside.
template <typename EvT, int DIGIT, bool FULL, bool PAY>
__device__ __forceinline__ void scatter_tile(ScatterSmem<EvT, PAY>& sm, const Knots& kn, int nkeys,
                                             const EvT* __restrict__ src,
                                             const Scalar<EvT>* __restrict__ wsrc, int tn,
                                             EvT* __restrict__ dst, Scalar<EvT>* __restrict__ wdst) {
  constexpr int R = kTileRows<EvT>;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lane_lt = (1u << lane) - 1u;
  // the previous tile's last reads of this warp's row are done (barrier 3)
  sm.whist[warp][lane] = 0;
  sm.whist[warp][lane + 32] = 0;
  __syncwarp();
  const int wbase = warp * 32 * R + lane;
  EvT e[R];
  Scalar<EvT> w[PAY ? R : 1];
  int kr[R];  // the key (bits 0-7), then also the rank (bits 8 and up)
#pragma unroll
  for (int u = 0; u < R; ++u) {
    if (FULL || wbase + 32 * u < tn) {
      e[u] = __ldcs(src + wbase + 32 * u);
      if constexpr (PAY) w[u] = __ldcs(wsrc + wbase + 32 * u);
    }
  }
#pragma unroll
  for (int u = 0; u < R; ++u)
    kr[u] = (FULL || wbase + 32 * u < tn) ? digit_of<EvT, DIGIT>(kn, e[u]) : 0;
  // rank of each event among the earlier events of its key in this warp's
  // rows: the live lanes of a row with the same key, from six ballots
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const bool live = FULL || wbase + 32 * u < tn;
    const int key = kr[u];
    unsigned peers = FULL ? 0xffffffffu : __ballot_sync(0xffffffffu, live);
#pragma unroll
    for (int b = 0; b < 6; ++b) {
      const bool bit = (key >> b) & 1;
      const unsigned vb = __ballot_sync(0xffffffffu, bit);
      peers &= bit ? vb : ~vb;
    }
    const int before = sm.whist[warp][key];
    __syncwarp();
    kr[u] = key | ((before + __popc(peers & lane_lt)) << 8);
    if (live && lane == 31 - __clz(peers)) sm.whist[warp][key] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();  // barrier 1: every warp's counts are in
  // warp 0, two keys per lane: each warp's first tile position per key (the
  // tile's exclusive scan over keys plus the events of earlier warps), the
  // offset from tile to output position, and the cursor moved past the tile
  if (warp == 0) {
    int c[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      int run = 0;
#pragma unroll
      for (int w = 0; w < kScatterWarps; ++w) run += sm.whist[w][lane + 32 * h];
      c[h] = run;
    }
    int s0 = c[0], s1 = c[1];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y0 = __shfl_up_sync(0xffffffffu, s0, off);
      const int y1 = __shfl_up_sync(0xffffffffu, s1, off);
      if (lane >= off) {
        s0 += y0;
        s1 += y1;
      }
    }
    s1 += __shfl_sync(0xffffffffu, s0, 31);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = lane + 32 * h;
      int run = h == 0 ? s0 - c[0] : s1 - c[1];  // the tile's first position of key k
      if (k < nkeys) {
        sm.delta[k] = sm.cursor[k] - run;
        sm.cursor[k] += c[h];
      }
#pragma unroll
      for (int w = 0; w < kScatterWarps; ++w) {
        const int v = sm.whist[w][k];
        sm.whist[w][k] = run;
        run += v;
      }
    }
  }
  __syncthreads();  // barrier 2: positions known
#pragma unroll
  for (int u = 0; u < R; ++u) {
    if (FULL || wbase + 32 * u < tn) {
      const int key = kr[u] & 0xff;
      const int p = sm.whist[warp][key] + (kr[u] >> 8);
      sm.stage[p] = e[u];
      if constexpr (PAY) sm.wstage[p] = w[u];
      sm.skey[p] = (unsigned char)key;
    }
  }
  __syncthreads();  // barrier 3: the tile is in key order
  for (int j = threadIdx.x; j < (FULL ? kTile<EvT> : tn); j += kScatterThreads) {
    const int pos = sm.delta[sm.skey[j]] + j;
    dst[pos] = sm.stage[j];
    if constexpr (PAY) wdst[pos] = sm.wstage[j];
  }
}

template <typename EvT, int DIGIT, bool PAY>
__global__ void __launch_bounds__(kScatterThreads, 3)
    sort_scatter_kernel(const Knots kn, const EvT* __restrict__ src,
                        const Scalar<EvT>* __restrict__ wsrc, int64_t n,
                        const int* __restrict__ offsets, EvT* __restrict__ dst,
                        Scalar<EvT>* __restrict__ wdst) {
  constexpr int T = kTile<EvT>;
  __shared__ ScatterSmem<EvT, PAY> sm;
  const int nkeys = kn.n - 1;
  if (threadIdx.x < nkeys)
    sm.cursor[threadIdx.x] = offsets[(size_t)blockIdx.x * nkeys + threadIdx.x];
  __syncthreads();
  const int64_t b0 = chunk_begin(n, blockIdx.x), b1 = chunk_begin(n, blockIdx.x + 1);
  const int len = (int)(b1 - b0);
  src += b0;
  if constexpr (PAY) wsrc += b0;
  int t0 = 0;
  for (; t0 + T <= len; t0 += T)
    scatter_tile<EvT, DIGIT, true, PAY>(sm, kn, nkeys, src + t0, PAY ? wsrc + t0 : nullptr, T, dst,
                                        wdst);
  if (t0 < len)
    scatter_tile<EvT, DIGIT, false, PAY>(sm, kn, nkeys, src + t0, PAY ? wsrc + t0 : nullptr,
                                         len - t0, dst, wdst);
}

// ------------------------------------------------------------ sample weights
// The sum of a sample's weights in FP64, in an order fixed by n alone (so it is
// the same on every call), and the number of weights that are not finite.
constexpr int kWsumBlocks = 256;

template <typename W>
__global__ void __launch_bounds__(256)
    weight_partial_kernel(const W* __restrict__ w, int64_t n, double* part,
                          unsigned long long* bad) {
  __shared__ double red[256];
  const int64_t per = (n + kWsumBlocks - 1) / kWsumBlocks;
  const int64_t b0 = per * blockIdx.x < n ? per * blockIdx.x : n;
  const int64_t b1 = b0 + per < n ? b0 + per : n;
  double s = 0.0;
  unsigned int nb = 0;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += 256) {
    const double x = (double)w[i];
    if (isfinite(x)) s += x;
    else ++nb;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
  for (int off = 16; off > 0; off >>= 1) nb += __shfl_down_sync(0xffffffffu, nb, off);
  if ((threadIdx.x & 31) == 0 && nb) atomicAdd(bad, (unsigned long long)nb);
}

__global__ void __launch_bounds__(256) weight_final_kernel(const double* part, double* out) {
  __shared__ double red[256];
  red[threadIdx.x] = part[threadIdx.x];
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

cudaError_t launch_weight_sum(int f32, const void* w, int64_t n, double* work, cudaStream_t st) {
  unsigned long long* bad = (unsigned long long*)(work + kWsumBlocks + 1);
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  if (f32)
    weight_partial_kernel<float><<<kWsumBlocks, 256, 0, st>>>((const float*)w, n, work, bad);
  else
    weight_partial_kernel<double><<<kWsumBlocks, 256, 0, st>>>((const double*)w, n, work, bad);
  weight_final_kernel<<<1, 256, 0, st>>>(work, work + kWsumBlocks);
  return cudaGetLastError();
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
  const int nkeys = n_knots - 1;
  // counts [kSortBlocks][nkeys], group sums [kGroups][nkeys], key starts [nkeys]
  *ints = (size_t)nkeys * (kSortBlocks + kGroups + 1);
  return cudaSuccess;
}

// The first pass sorts by j13, the second by j12.
constexpr int kFirstDigit = 1, kSecondDigit = 0;

// Count the chunks [c0, c1).
template <typename EvT, int DIGIT, bool CHECK>
static cudaError_t count_pass(const Model& m, const EvT* src, int64_t n, int* work,
                              unsigned long long* outside, cudaStream_t st, int c0 = 0,
                              int c1 = kSortBlocks) {
  sort_count_kernel<EvT, DIGIT, CHECK><<<c1 - c0, kCountThreads, 0, st>>>(m, src, n, c0, work,
                                                                         outside);
  return cudaGetLastError();
}

// Offsets and scatter of one pass whose counts are in `work` (with the
// events' weights from wsrc to wdst when wsrc is not null).
template <typename EvT, int DIGIT>
static cudaError_t finish_pass(const Knots& kn, const EvT* src, int64_t n, EvT* dst, int* work,
                               cudaStream_t st, const Scalar<EvT>* wsrc, Scalar<EvT>* wdst) {
  const int nkeys = kn.n - 1;
  int* group_sum = work + (size_t)nkeys * kSortBlocks;
  int* key_start = group_sum + (size_t)nkeys * kGroups;
  const dim3 cgrid((nkeys + 255) / 256, kGroups);
  sort_group_sums<<<cgrid, 256, 0, st>>>(work, nkeys, group_sum);
  sort_key_starts<<<1, 1024, 0, st>>>(group_sum, nkeys, key_start);
  sort_offsets<<<cgrid, 256, 0, st>>>(work, nkeys, group_sum, key_start);
  if (wsrc)
    sort_scatter_kernel<EvT, DIGIT, true>
        <<<kSortBlocks, kScatterThreads, 0, st>>>(kn, src, wsrc, n, work, dst, wdst);
  else
    sort_scatter_kernel<EvT, DIGIT, false>
        <<<kSortBlocks, kScatterThreads, 0, st>>>(kn, src, nullptr, n, work, dst, nullptr);
  return cudaGetLastError();
}

// Both passes after the first count: src -> tmp by j13, tmp -> dst by j12.
template <typename EvT>
static cudaError_t sort_rest(const Model& m, const EvT* src, int64_t n, EvT* tmp, EvT* dst,
                             int* work, cudaStream_t st, const void* wsrc, void* wtmp,
                             void* wdst) {
  using W = Scalar<EvT>;
  cudaError_t e = finish_pass<EvT, kFirstDigit>(m.kn, src, n, tmp, work, st, (const W*)wsrc,
                                                (W*)wtmp);
  if (e == cudaSuccess) e = count_pass<EvT, kSecondDigit, false>(m, tmp, n, work, nullptr, st);
  if (e == cudaSuccess)
    e = finish_pass<EvT, kSecondDigit>(m.kn, tmp, n, dst, work, st,
                                       wsrc ? (const W*)wtmp : nullptr, (W*)wdst);
  return e;
}

// First chunk of piece p of n_pieces (p = n_pieces: the end): halving pieces,
// 1/2, 1/4, ... of the chunks, the last two equal, so that the piece whose
// count waits for the whole copy is the smallest.
static int piece_chunk(int p, int n_pieces) {
  if (p <= 0) return 0;
  if (p >= n_pieces) return kSortBlocks;
  return kSortBlocks - (kSortBlocks >> p);
}

cudaError_t launch_sort_count_checked(int ev_f32, const Model& m, const void* src, int64_t n,
                                      int* work, unsigned long long* outside, cudaStream_t st,
                                      int piece, int n_pieces) {
  const int c0 = piece_chunk(piece, n_pieces), c1 = piece_chunk(piece + 1, n_pieces);
  if (ev_f32)
    return count_pass<float2, kFirstDigit, true>(m, (const float2*)src, n, work, outside, st, c0,
                                                 c1);
  return count_pass<double2, kFirstDigit, true>(m, (const double2*)src, n, work, outside, st, c0,
                                                c1);
}

int64_t sort_piece_begin(int64_t n, int piece, int n_pieces) {
  return chunk_begin(n, piece_chunk(piece, n_pieces));
}

cudaError_t launch_sort_rest(int ev_f32, const Model& m, const void* src, int64_t n, void* tmp,
                             void* dst, int* work, cudaStream_t st, const void* wsrc, void* wtmp,
                             void* wdst) {
  if (ev_f32)
    return sort_rest(m, (const float2*)src, n, (float2*)tmp, (float2*)dst, work, st, wsrc, wtmp,
                     wdst);
  return sort_rest(m, (const double2*)src, n, (double2*)tmp, (double2*)dst, work, st, wsrc, wtmp,
                   wdst);
}

cudaError_t launch_sort(int ev_f32, const Model& m, const void* src, int64_t n, void* tmp,
                        void* dst, int* work, cudaStream_t st, const void* wsrc, void* wtmp,
                        void* wdst) {
  cudaError_t e;
  if (ev_f32)
    e = count_pass<float2, kFirstDigit, false>(m, (const float2*)src, n, work, nullptr, st);
  else
    e = count_pass<double2, kFirstDigit, false>(m, (const double2*)src, n, work, nullptr, st);
  if (e != cudaSuccess) return e;
  return launch_sort_rest(ev_f32, m, src, n, tmp, dst, work, st, wsrc, wtmp, wdst);
}

}  // namespace mipwa
