// Normalisation integrals of many toys on the tensor cores (sm_103a tcgen05).
//
// The batched fit of arXiv:1703.03284, Sec. 4 (many toy samples fitted, one
// shared normalisation sample) needs, per toy t and normalisation event e,
// the S-wave spline values of Sec. 2 at both Bose channels. With the natural
// cubic spline these are linear in the knot values:
//   a_t(s) = sum_k W_k(s) a_tk,   phi_t(s) = sum_k W_k(s) phi_tk,
// W_k the cardinal spline functions of the knots (on segment j:
// W_k = [k=j] A/h + [k=j+1] B/h + (dM_j/dy_k) (A^3/h - hA)/6
//       + (dM_{j+1}/dy_k) (B^3/h - hB)/6, A = s_{j+1} - s, B = s - s_j).
// So the (toys x knots) block of knot values times the (knots x events)
// cached basis W is a dense contraction. Here it runs as tcgen05.mma (bf16
// operands, FP32 accumulators in tensor memory) with every operand split into
// three bf16 parts, x = x0 + x1 + x2 (exact to 2^-24 of x), keeping the six
// products x_i y_j with i + j <= 2. A persistent kernel takes tiles of 64
// events: the tile's basis parts (stored once per sample in the MMA's
// shared-memory layout) are copied in with cp.async while the previous
// tile's products are read back. Each warp reads one quarter of the
// accumulator lanes (32 toys) and a quarter of the tile's events (16
// columns); each thread (one toy) forms A = sum_r c_r B_r + a12 e^{i phi12}
// + a13 e^{i phi13}, |A|^2, and its toy's running sum over its events; the
// four sums of a toy are added in a fixed order at the end.
//
// Operand layout (no swizzle, K-major): an R x 32 bf16 matrix is stored as
// 8 x 16-byte core matrices, element (r, k) at byte
//   (r / 8) * 512 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2,
// so adjacent core matrices along K are 128 bytes apart (the descriptor's
// leading byte offset) and along rows 512 bytes apart (stride byte offset);
// the second K step of 16 starts 256 bytes in.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mipwa_amp.cuh"
#include "mipwa_kernels.cuh"

namespace mipwa {

namespace {

constexpr int kTcEvents = 64;                    // events per tile (MMA N)
constexpr int kTcToys = 128;                     // toys per group (MMA M)
constexpr int kTcK = 32;                         // knots per operand row (MMA K, two steps)
constexpr int kTcThreads = 512;                  // 16 warps: four per accumulator lane quarter
constexpr int kTcSlices = kTcThreads / 128;      // warps sharing a lane quarter split the events
constexpr int kTcSliceEvents = kTcEvents / kTcSlices;  // 16 events per thread and tile
constexpr int kWMatBytes = kTcEvents * kTcK * 2;         // 4096: one 64 x 32 bf16 matrix
constexpr int kTileBytes = 6 * kWMatBytes;               // channels x parts
constexpr int kThMatBytes = kTcToys * kTcK * 2;          // 8192: one 128 x 32 bf16 matrix
constexpr int kThetaBytes = 6 * kThMatBytes;             // (a, phi) x parts
constexpr int kTmemCols = 512;                   // two buffers of 4 x 64 FP32 columns
constexpr long long kWaitCycles = 1LL << 31;     // ~1 s at 2 GHz: an mbarrier wait gives up
// dynamic shared memory: theta | two W buffers | two B stages | mbarriers;
// more than half of an SM's shared memory, so one block per SM (the block
// allocates all of its tensor memory)
constexpr int kOffTheta = 0;
constexpr int kOffW = kOffTheta + kThetaBytes;
constexpr int kOffB = kOffW + 2 * kTileBytes;
constexpr int kBStageBytes = kTcEvents * kMaxRes * 8;
constexpr int kOffBar = kOffB + 2 * kBStageBytes;
constexpr int kTcSmem = 120 * 1024;
static_assert(kOffBar + 64 <= kTcSmem, "shared memory layout");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: no swizzle, K-major, leading byte offset
// 128 (next core matrix along K), stride byte offset 512 (next 8 rows),
// descriptor version 1 (bits 46-47).
__device__ __forceinline__ uint64_t mat_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((128 >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((512 >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1),
// A and B bf16 (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17,
// M >> 4 at bit 24.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) |
                            ((uint32_t)(kTcEvents >> 3) << 17) | ((uint32_t)(kTcToys >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      :
      : "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :
               : "r"(bar)
               : "memory");
}

// Wait for phase `parity` of an mbarrier for at most kWaitCycles SM cycles;
// false if it did not complete.
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" : : "r"(dst), "l"(src) : "memory");
}

// Byte offset of element (row, k) in an operand matrix of this layout.
__host__ __device__ constexpr int op_offset(int row, int k) {
  return (row / 8) * 512 + (k / 8) * 128 + (row % 8) * 16 + (k % 8) * 2;
}

// x = x0 + x1 + x2 in bf16 (round to nearest), the residuals formed in FP64.
__device__ __forceinline__ void split3(double x, __nv_bfloat16* p) {
  const __nv_bfloat16 b0 = __float2bfloat16_rn((float)x);
  const double r1 = x - (double)__bfloat162float(b0);
  const __nv_bfloat16 b1 = __float2bfloat16_rn((float)r1);
  const double r2 = r1 - (double)__bfloat162float(b1);
  p[0] = b0;
  p[1] = b1;
  p[2] = __float2bfloat16_rn((float)r2);
}

// Cached cardinal basis of one event and channel, its three bf16 parts
// written into the tile's operand matrices (channel ch: matrices 3 ch + part).
__global__ void __launch_bounds__(256) tc_basis_kernel(const Knots kn, const double* dmdy,
                                                       const float2* ev, int64_t n,
                                                       uint8_t* tiles) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 2 * n) return;
  const int64_t e = idx >> 1;
  const int ch = (int)(idx & 1);
  const double s = ch == 0 ? (double)ev[e].x : (double)ev[e].y;
  const int N = kn.n;
  int j = 0;  // segment (clamped to the end segments, as the spline's continuation)
  while (j < N - 2 && s >= kn.s[j + 1]) ++j;
  const double h = kn.s[j + 1] - kn.s[j];
  const double A = kn.s[j + 1] - s, B = s - kn.s[j];
  const double f0 = A / h, f1 = B / h;
  const double f2 = (A * A * A / h - h * A) / 6.0, f3 = (B * B * B / h - h * B) / 6.0;
  uint8_t* tile = tiles + (e / kTcEvents) * (int64_t)kTileBytes;
  const int row = (int)(e % kTcEvents);
  for (int k = 0; k < kTcK; ++k) {
    double w = 0.0;
    if (k < N) {
      w = dmdy[k * N + j] * f2 + dmdy[k * N + j + 1] * f3;
      if (k == j) w += f0;
      if (k == j + 1) w += f1;
    }
    __nv_bfloat16 p[3];
    split3(w, p);
    for (int part = 0; part < 3; ++part)
      *reinterpret_cast<__nv_bfloat16*>(tile + (3 * ch + part) * kWMatBytes + op_offset(row, k)) =
          p[part];
  }
}

// One batched forward evaluation of the normalisation integrals. MODE 0: the
// per-toy sums of |A|^2; MODE 1: also the four products (a12, phi12, a13,
// phi13) of the first tile of the first group into `dump` ([4][128][64]).
template <int MODE>
__global__ void __launch_bounds__(kTcThreads, 1) tc_norm_kernel(const TcArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint32_t tmem_base_sh;
  __shared__ double slice_sum[kTcSlices][kTcToys];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quarter = warp & 3, slice = warp >> 2;  // accumulator lanes, event columns
  const int row = quarter * 32 + lane;               // this thread's toy within the group
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar0 = sbase + kOffBar, bar1 = bar0 + 8;
  float2* bstage = reinterpret_cast<float2*>(smem + kOffB);
  bool ok = true;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :
                 : "r"(smem_u32(&tmem_base_sh)), "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" : : "r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" : : "r"(bar1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;
  uint32_t phase[2] = {0u, 0u};
  const int R = a.n_res;
  const int n_tiles = a.n_tiles;
  for (int g = 0; g < a.n_groups && ok; ++g) {
    // this group's knot values (A operands) and the thread's toy constants
    {
      const uint4* src = a.theta + (size_t)g * (kThetaBytes / 16);
      uint4* dst = reinterpret_cast<uint4*>(smem + kOffTheta);
      for (int i = tid; i < kThetaBytes / 16; i += kTcThreads) dst[i] = src[i];
    }
    const int toy = g * kTcToys + row;
    float cre[kMaxRes], crl[kMaxRes], cim[kMaxRes], cil[kMaxRes];
#pragma unroll
    for (int r = 0; r < kMaxRes; ++r) {
      const bool on = r < R && toy < a.n_toys;
      cre[r] = on ? a.cr[(size_t)toy * 4 * kMaxRes + 4 * r + 0] : 0.0f;
      crl[r] = on ? a.cr[(size_t)toy * 4 * kMaxRes + 4 * r + 1] : 0.0f;
      cim[r] = on ? a.cr[(size_t)toy * 4 * kMaxRes + 4 * r + 2] : 0.0f;
      cil[r] = on ? a.cr[(size_t)toy * 4 * kMaxRes + 4 * r + 3] : 0.0f;
    }
    float sum = 0.0f, comp = 0.0f;  // Kahan sum of the toy's |A|^2
    const int first = blockIdx.x, stride = gridDim.x;
    // prologue: W of the first two tiles in flight, the first MMA issued
    auto load_w = [&](int tile, int buf) {
      const uint8_t* src = a.wtiles + (size_t)tile * kTileBytes;  // 16-byte aligned (cudaMalloc)
      const uint32_t dst = sbase + kOffW + buf * kTileBytes;
      for (int i = tid; i < kTileBytes / 16; i += kTcThreads) cp_async16(dst + 16 * i, src + 16 * i);
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
    auto issue = [&](int buf) {
      // products of the two K steps, small parts first: (2,0) (1,1) (0,2) (1,0) (0,1) (0,0)
      const uint32_t wb = sbase + kOffW + buf * kTileBytes;
      const uint32_t th = sbase + kOffTheta;
#pragma unroll
      for (int q = 0; q < 4; ++q) {           // a12, phi12, a13, phi13
        const int which = q & 1, ch = q >> 1;  // theta: a or phi; W: channel
        const uint32_t d = tmem + (uint32_t)(buf * 256 + q * kTcEvents);
#pragma unroll
        for (int p = 0; p < 6; ++p) {
          const int pa = p == 0 ? 2 : (p == 1 ? 1 : (p == 2 ? 0 : (p == 3 ? 1 : 0)));
          const int pb = p == 0 ? 0 : (p == 1 ? 1 : (p == 2 ? 2 : (p == 3 ? 0 : (p == 4 ? 1 : 0))));
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const uint32_t aaddr = th + (3 * which + pa) * kThMatBytes + ks * 256;
            const uint32_t baddr = wb + (3 * ch + pb) * kWMatBytes + ks * 256;
            mma_bf16(d, mat_desc(aaddr), mat_desc(baddr), (p == 0 && ks == 0) ? 0u : 1u);
          }
        }
      }
      mma_commit(buf == 0 ? bar0 : bar1);
    };
    int tile = first;
    if (tile < n_tiles) load_w(tile, 0);
    if (tile + stride < n_tiles) load_w(tile + stride, 1);
    if (tile < n_tiles) {
      if (tile + stride < n_tiles) asm volatile("cp.async.wait_group 1;" ::: "memory");
      else asm volatile("cp.async.wait_group 0;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        issue(0);
      }
    }
    for (int k = 0; tile < n_tiles; ++k, tile += stride) {
      const int buf = k & 1;
      // the tile's Breit-Wigner terms (c_r B_r is formed per toy below)
      for (int i = tid; i < kTcEvents * R; i += kTcThreads) {
        const int r = i / kTcEvents, el = i % kTcEvents;
        const int64_t e = (int64_t)tile * kTcEvents + el;
        bstage[buf * kTcEvents * kMaxRes + r * kTcEvents + el] =
            e < a.n ? a.basis[(size_t)r * a.n + e] : make_float2(0.0f, 0.0f);
      }
      // the next tile's products start while this one is read back
      const int next = tile + stride;
      if (next < n_tiles) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      }
      __syncthreads();
      if (next < n_tiles && tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        issue(buf ^ 1);
      }
      // every thread waits; the block goes on only if all saw the phase complete
      if (!__syncthreads_and(bar_wait(buf == 0 ? bar0 : bar1, phase[buf]) ? 1 : 0)) {
        ok = false;
        if (tid == 0) atomicOr(a.flags, kFlagTcTimeout);
        break;
      }
      phase[buf] ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const float2* bs = bstage + buf * kTcEvents * kMaxRes;
      const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * 256);
      {
        const int c0 = slice * kTcSliceEvents;
        float va12[16], vp12[16], va13[16], vp13[16];
        tmem_ld16(lane_base + 0 * kTcEvents + c0, va12);
        tmem_ld16(lane_base + 1 * kTcEvents + c0, vp12);
        tmem_ld16(lane_base + 2 * kTcEvents + c0, va13);
        tmem_ld16(lane_base + 3 * kTcEvents + c0, vp13);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (MODE == 1 && g == 0 && tile == 0) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            a.dump[(0 * kTcToys + row) * kTcEvents + c0 + i] = va12[i];
            a.dump[(1 * kTcToys + row) * kTcEvents + c0 + i] = vp12[i];
            a.dump[(2 * kTcToys + row) * kTcEvents + c0 + i] = va13[i];
            a.dump[(3 * kTcToys + row) * kTcEvents + c0 + i] = vp13[i];
          }
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          float re = 0.0f, im = 0.0f;
#pragma unroll
          for (int r = 0; r < kMaxRes; ++r) {
            if (r < R) {
              const float2 b = bs[r * kTcEvents + c0 + i];
              re += mul_hl(cre[r], crl[r], b.x) - mul_hl(cim[r], cil[r], b.y);
              im += mul_hl(cre[r], crl[r], b.y) + mul_hl(cim[r], cil[r], b.x);
            }
          }
          float s1, c1, s2, c2;
          sincos_cw(vp12[i], 0.0f, &s1, &c1);
          sincos_cw(vp13[i], 0.0f, &s2, &c2);
          re += va12[i] * c1 + va13[i] * c2;
          im += va12[i] * s1 + va13[i] * s2;
          const float y = fmaf(re, re, im * im) - comp;
          const float t = sum + y;
          comp = (t - sum) - y;
          sum = t;
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();  // this buffer's products are read: free for the tile after next
      const int after = next + stride;
      if (after < n_tiles) load_w(after, buf);
    }
    slice_sum[slice][row] = (double)sum - (double)comp;
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    if (slice == 0 && toy < a.n_toys) {
      double v = 0.0;
      for (int sl = 0; sl < kTcSlices; ++sl) v += slice_sum[sl][row];
      a.partial[(size_t)blockIdx.x * a.n_groups * kTcToys + toy] = v;
    }
    __syncthreads();
  }
  if (!ok) {
    // a wait gave up: wait (bounded) for the products still in flight before
    // the tensor memory goes
    bar_wait(bar0, phase[0]);
    bar_wait(bar1, phase[1]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 :
                 : "r"(tmem), "r"(kTmemCols)
                 : "memory");
  }
}

}  // namespace

int tc_tile_bytes() { return kTileBytes; }
int tc_theta_bytes() { return kThetaBytes; }
int tc_events_per_tile() { return kTcEvents; }
int tc_toys_per_group() { return kTcToys; }
int tc_max_knots() { return kTcK; }

int tc_theta_offset(int row, int k) { return op_offset(row, k); }

cudaError_t launch_tc_basis(const Knots& kn, const double* dmdy, const float2* ev, int64_t n,
                            uint8_t* tiles, cudaStream_t st) {
  const int64_t n_tiles = (n + kTcEvents - 1) / kTcEvents;
  cudaError_t e = cudaMemsetAsync(tiles, 0, (size_t)n_tiles * kTileBytes, st);
  if (e != cudaSuccess || n == 0) return e;
  const int64_t threads = 2 * n;
  tc_basis_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(kn, dmdy, ev, n, tiles);
  return cudaGetLastError();
}

cudaError_t launch_tc_norm(const TcArgs& a, int grid, int mode, cudaStream_t st) {
  cudaError_t e;
  if (mode == 1) {
    e = cudaFuncSetAttribute(tc_norm_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kTcSmem);
    if (e == cudaSuccess) tc_norm_kernel<1><<<grid, kTcThreads, kTcSmem, st>>>(a);
  } else {
    e = cudaFuncSetAttribute(tc_norm_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kTcSmem);
    if (e == cudaSuccess) tc_norm_kernel<0><<<grid, kTcThreads, kTcSmem, st>>>(a);
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace mipwa
