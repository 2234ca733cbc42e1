// Learned warm start of the mechanical CG: a three-layer message-passing network over the mesh
// (hidden width 64) that predicts the displacement correction on top of linear extrapolation.
//
// Forward layers run on the Blackwell tensor cores (tcgen05.mma kind::f16, BF16 operands, FP32
// accumulator in tensor memory) with the element-message aggregation z_i = sum_j A_ij h_j fused
// into the tile load: a block owns 128 rows, gathers [h_i, z_i] into shared memory as BF16 and
// multiplies by the layer's weights held in shared memory.  Training (backward and Adam) runs in FP32 on CUDA cores with
// deterministic block partials.  The network definition (features, aggregation, loss) is the
// one documented in include/gspm.h (gspm_mpnn_*).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.cuh"
#include "mpnn.cuh"

namespace gspm {

namespace {

constexpr int kRows = 128;      // rows per tile (8 warps x 16)
constexpr int kThreads = 256;
constexpr int kGather = 8;      // neighbour feature loads in flight per lane in k_tc_layer

__device__ __forceinline__ int64_t tid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t tstride() { return (int64_t)gridDim.x * blockDim.x; }

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// ---------------------------------------------------------------------------------------------
// Blackwell tensor cores: tcgen05.mma with the FP32 accumulator in tensor memory (TMEM)
// ---------------------------------------------------------------------------------------------
// A layer's GEMM is one 128 x 64 tile per block and K step: A = the block's 128 rows of [h, z]
// (or of the 16 input features), B = W^T (64 x K), both K-major in shared memory with the
// 128-byte swizzle (rows of 64 bf16, eight-row groups 1024 bytes apart, 16-byte chunk c of row r
// stored at chunk c ^ (r mod 8)).  One thread issues the K / 16 MMAs and commits them to an
// mbarrier; the accumulator (row i in TMEM lane i, column j in TMEM column j) is read back with
// tcgen05.ld by all eight warps (warp w: lanes 32 (w mod 4) .., columns 32 (w / 4) ..).
constexpr int kTileA = kRows * 128;   // bytes of one 64-wide K-block of A
constexpr int kTileB = kHid * 128;    // bytes of one 64-wide K-block of B
constexpr int kTmemCols = 64;         // TMEM columns of the 128 x 64 FP32 accumulator
constexpr size_t kTcSmem = 2 * kTileA + 2 * kTileB + kHid * 4 + 16 + 1024;  // + alignment slack
// spin limit of the accumulator wait (each try_wait may also suspend for a while): far beyond the
// microsecond an MMA group takes, so reaching it means the tensor-core work never completed
constexpr uint32_t kSpinLimit = 1u << 22;
// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and B bf16 (bits 7-9,
// 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) |
                            ((uint32_t)(kHid >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// byte offset of 16-byte chunk c (0..7) of row r in a 128-byte-swizzled K-block
__device__ __forceinline__ uint32_t sw128(int r, int c) {
  return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4));
}
// shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading byte offset >> 4
// (bits 16-29; not used by a swizzled K-major operand), stride byte offset >> 4 = 1024 >> 4
// between eight-row groups (bits 32-45), the fixed 0b001 at bits 46-48, 128-byte swizzle (2 at
// bits 61-63).  The K-block starts on a 1024-byte boundary, so the base offset is 0 and a K step
// inside the block advances the start address by 32 bytes.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   mbar)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void async_proxy_fence() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// true once the mbarrier phase of parity `phase` has completed; false after kSpinLimit polls
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}
// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
        "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
        "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---------------------------------------------------------------------------------------------
// features: m (3), E0(m) Voigt / lambda_s (6), u_prev / u_s (3), (u_prev - u_prev2) / u_s (3), 1
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_features(int64_t n, const T* __restrict__ m, int64_t ld,
                           const uint8_t* __restrict__ mag, const T* __restrict__ up,
                           const T* __restrict__ up2, double l100, double l111,
                           double inv_ls, double inv_us, __nv_bfloat16* __restrict__ F) {
  for (int64_t i = tid(); i < n; i += tstride()) {
    float f[kFeat];
    const double m0 = m[i], m1 = m[ld + i], m2 = m[2 * ld + i];
    f[0] = (float)m0;
    f[1] = (float)m1;
    f[2] = (float)m2;
    if (mag[i]) {
      const double a = 1.5 * l100 * inv_ls, b = 1.5 * l111 * inv_ls;
      f[3] = (float)(a * (m0 * m0 - 1.0 / 3.0));
      f[4] = (float)(a * (m1 * m1 - 1.0 / 3.0));
      f[5] = (float)(a * (m2 * m2 - 1.0 / 3.0));
      f[6] = (float)(b * m1 * m2);
      f[7] = (float)(b * m0 * m2);
      f[8] = (float)(b * m0 * m1);
    } else {
      for (int c = 3; c < 9; ++c) f[c] = 0.f;
    }
    for (int c = 0; c < 3; ++c) {
      const double p = up ? (double)up[3 * i + c] : 0.0, q = up2 ? (double)up2[3 * i + c] : 0.0;
      f[9 + c] = (float)(p * inv_us);
      f[12 + c] = (float)((p - q) * inv_us);
    }
    f[15] = 1.f;
    uint32_t* o = reinterpret_cast<uint32_t*>(F + i * kFeat);
    for (int c = 0; c < kFeat / 2; ++c)
      o[c] = pack2(__float2bfloat16_rn(f[2 * c]), __float2bfloat16_rn(f[2 * c + 1]));
  }
}

// One forward layer on the tensor cores.  MODE 0: h0 = relu(F W_in + b_in) (K = 16, the node
// features); MODE 1: h_out = relu([h, A h] W + b) (K = 128) with the element-message aggregation
// z = A h gathered into the A tile (z optionally saved for the backward pass).  A block owns
// 128 rows per round; TMEM holds its 128 x 64 accumulator.  err (device int) is set when the
// accumulator wait gives up; the block then waits once more (bounded) for its MMAs, frees its
// TMEM and returns.
template <int MODE>
__global__ void __launch_bounds__(kThreads) k_tc_layer(int64_t n, DSell S,
                                                       const float* __restrict__ Aw,
                                                       const __nv_bfloat16* __restrict__ Hin,
                                                       const __nv_bfloat16* __restrict__ WT,
                                                       const float* __restrict__ bias,
                                                       __nv_bfloat16* __restrict__ Hout,
                                                       __nv_bfloat16* __restrict__ Zout,
                                                       int* __restrict__ err) {
  constexpr int K = MODE == 0 ? kFeat : 2 * kHid;
  constexpr int KC = K / 8;  // 16-byte chunks per row
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_addr(smem_raw);
  unsigned char* sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  unsigned char* As = sm;                  // K-blocks 0 (h or F) and 1 (z)
  unsigned char* Bs = sm + 2 * kTileA;     // W^T, K-blocks 0 and 1
  float* bs = reinterpret_cast<float*>(Bs + 2 * kTileB);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(bs + kHid);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  __shared__ int s_fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int t = threadIdx.x; t < kHid * KC; t += blockDim.x) {
    const int o = t / KC, cc = t % KC;
    const uint4 v = *reinterpret_cast<const uint4*>(WT + (int64_t)o * K + cc * 8);
    *reinterpret_cast<uint4*>(Bs + (cc >> 3) * kTileB + sw128(o, cc & 7)) = v;
  }
  for (int k = threadIdx.x; k < kHid; k += blockDim.x) bs[k] = bias[k];
  if (threadIdx.x == 0) {
    s_fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tslot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  async_proxy_fence();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t bar = smem_addr(mbar);
  uint32_t phase = 0;
  int inflight = 0;
  for (int64_t base = (int64_t)blockIdx.x * kRows; base < n; base += (int64_t)gridDim.x * kRows) {
    if (MODE == 0) {
      // 128 rows x 2 chunks of the features, one 16-byte load per thread
      for (int t = threadIdx.x; t < kRows * KC; t += blockDim.x) {
        const int r = t / KC, c = t % KC;
        const int64_t i = base + r;
        const uint4 v = i < n ? *reinterpret_cast<const uint4*>(Hin + i * kFeat + c * 8)
                              : make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(As + sw128(r, c)) = v;
      }
    } else {
      // each warp fills its 16 rows (half a SELL slice) four at a time: lane group g = lane / 8
      // takes row 4 rr + g, lane q = lane % 8 its features 8 q .. 8 q + 7 (one 16-byte chunk);
      // the neighbours go in batches of kGather, all their column loads before their feature
      // loads, so a lane has kGather gathers in flight.  z sums the neighbours in column order.
      const int grp = lane >> 3, q = lane & 7;
      const int64_t s0 = (base + 16 * warp) >> 5;
      const int64_t sb = s0 < S.nslices ? S.sptr[s0] : 0;
      const int len = s0 < S.nslices ? S.slen[s0] : 0;
      for (int rr = 0; rr < 4; ++rr) {
        const int r = 16 * warp + 4 * rr + grp;
        const int64_t i = base + r;
        float z[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) z[c] = 0.f;
        uint4 hi = make_uint4(0u, 0u, 0u, 0u);
        if (i < n) {
          hi = *reinterpret_cast<const uint4*>(Hin + i * kHid + 8 * q);
          const int64_t li = i & 31;
          for (int k0 = 0; k0 < len; k0 += kGather) {
            int64_t j[kGather];
            float a[kGather];
#pragma unroll
            for (int u = 0; u < kGather; ++u) {
              // past the row's end: entry k0 (k0 < len) again, weight 0; no load leaves the slice
              const bool ok = k0 + u < len;
              const int64_t e = sb + (int64_t)(ok ? k0 + u : k0) * 32 + li;
              j[u] = (int64_t)S.col[e];
              const float av = Aw[e];
              a[u] = ok ? av : 0.f;
            }
            uint4 hj[kGather];
#pragma unroll
            for (int u = 0; u < kGather; ++u)
              hj[u] = *reinterpret_cast<const uint4*>(Hin + j[u] * kHid + 8 * q);
#pragma unroll
            for (int u = 0; u < kGather; ++u) {
              const uint32_t w[4] = {hj[u].x, hj[u].y, hj[u].z, hj[u].w};
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                z[2 * c] += a[u] * __bfloat162float(__ushort_as_bfloat16((unsigned short)(w[c] & 0xffffu)));
                z[2 * c + 1] += a[u] * __bfloat162float(__ushort_as_bfloat16((unsigned short)(w[c] >> 16)));
              }
            }
          }
        }
        uint4 zp;
        zp.x = pack2(__float2bfloat16_rn(z[0]), __float2bfloat16_rn(z[1]));
        zp.y = pack2(__float2bfloat16_rn(z[2]), __float2bfloat16_rn(z[3]));
        zp.z = pack2(__float2bfloat16_rn(z[4]), __float2bfloat16_rn(z[5]));
        zp.w = pack2(__float2bfloat16_rn(z[6]), __float2bfloat16_rn(z[7]));
        *reinterpret_cast<uint4*>(As + sw128(r, q)) = hi;
        *reinterpret_cast<uint4*>(As + kTileA + sw128(r, q)) = zp;
        if (Zout && i < n) *reinterpret_cast<uint4*>(Zout + i * kHid + 8 * q) = zp;
      }
    }
    // the A tile written by every thread becomes visible to the tensor cores; one thread issues
    // the K / 16 MMAs of the tile and commits them to the mbarrier
    async_proxy_fence();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_addr(As), b0 = smem_addr(Bs);
#pragma unroll
      for (int ks = 0; ks < K / 16; ++ks) {
        const uint32_t koff = (uint32_t)((ks & 3) * 32);
        tc_mma(tmem, sw128_desc(a0 + (ks >> 2) * kTileA + koff),
               sw128_desc(b0 + (ks >> 2) * kTileB + koff), ks > 0 ? 1u : 0u);
      }
      tc_commit(bar);
    }
    inflight = 1;
    if (!mbar_wait(bar, phase)) s_fail = 1;
    __syncthreads();
    if (s_fail) break;
    inflight = 0;
    phase ^= 1u;
    tc_fence_after();
    // epilogue: warp w reads lanes 32 (w mod 4) .. + 31 (its rows), columns 32 (w / 4) .. + 31
    const int lg = warp & 3, ch = warp >> 2;
    uint32_t v[32];
    tmem_ld32(tmem + ((uint32_t)(32 * lg) << 16) + (uint32_t)(32 * ch), v);
    const int64_t row = base + 32 * lg + lane;
    if (row < n) {
      uint32_t pk[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int col = 32 * ch + 2 * c;
        pk[c] = pack2(__float2bfloat16_rn(fmaxf(__uint_as_float(v[2 * c]) + bs[col], 0.f)),
                      __float2bfloat16_rn(fmaxf(__uint_as_float(v[2 * c + 1]) + bs[col + 1], 0.f)));
      }
      uint4* dst = reinterpret_cast<uint4*>(Hout + row * kHid + 32 * ch);
#pragma unroll
      for (int c = 0; c < 4; ++c) dst[c] = make_uint4(pk[4 * c], pk[4 * c + 1], pk[4 * c + 2], pk[4 * c + 3]);
    }
    // the accumulator and the A tile are consumed before the next round overwrites them
    tc_fence_before();
    __syncthreads();
  }
  if (s_fail) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    if (inflight) mbar_wait(bar, phase);  // bounded: give the MMAs a last chance to finish
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
  }
}

// y = h3 W_out + b_out; mode 0: Y = y (float [n][3]); mode 1: x0 = 2 u_prev - u_prev2 + u_s y
template <typename T>
__global__ void k_output(int64_t n, const __nv_bfloat16* __restrict__ H,
                         const float* __restrict__ Wout, const float* __restrict__ bout, int mode,
                         float* __restrict__ Y, const T* __restrict__ up,
                         const T* __restrict__ up2, double us, T* __restrict__ x0) {
  __shared__ float w[kHid * 3 + 3];
  for (int k = threadIdx.x; k < kHid * 3; k += blockDim.x) w[k] = Wout[k];
  if (threadIdx.x < 3) w[kHid * 3 + threadIdx.x] = bout[threadIdx.x];
  __syncthreads();
  for (int64_t i = tid(); i < n; i += tstride()) {
    float y0 = w[kHid * 3], y1 = w[kHid * 3 + 1], y2 = w[kHid * 3 + 2];
    const uint32_t* hp = reinterpret_cast<const uint32_t*>(H + i * kHid);
    for (int c = 0; c < kHid / 2; ++c) {
      const uint32_t v = hp[c];
      const float a = __bfloat162float(__ushort_as_bfloat16((unsigned short)(v & 0xffffu)));
      const float b = __bfloat162float(__ushort_as_bfloat16((unsigned short)(v >> 16)));
      y0 += a * w[3 * (2 * c)] + b * w[3 * (2 * c + 1)];
      y1 += a * w[3 * (2 * c) + 1] + b * w[3 * (2 * c + 1) + 1];
      y2 += a * w[3 * (2 * c) + 2] + b * w[3 * (2 * c + 1) + 2];
    }
    if (mode == 0) {
      Y[3 * i] = y0;
      Y[3 * i + 1] = y1;
      Y[3 * i + 2] = y2;
    } else {
      const float y[3] = {y0, y1, y2};
      for (int c = 0; c < 3; ++c) {
        const double p = up ? (double)up[3 * i + c] : 0.0, q = up2 ? (double)up2[3 * i + c] : 0.0;
        x0[3 * i + c] = (T)(2.0 * p - q + us * (double)y[c]);
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// training (FP32)
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ float bf(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// dY = 2 (Y - T) / (3n); dH3 = dY W_out^T; block partials of dW_out (h3^T dY), db_out, loss
__global__ void __launch_bounds__(kThreads) k_out_bwd(int64_t n, const float* __restrict__ Y,
                                                      const float* __restrict__ T,
                                                      const __nv_bfloat16* __restrict__ H,
                                                      const float* __restrict__ Wout,
                                                      float* __restrict__ dH,
                                                      float* __restrict__ part) {
  // part per block: [kHid*3 dW_out][3 db_out][1 loss]
  __shared__ float acc[kHid * 3 + 4];
  __shared__ float w[kHid * 3];
  for (int k = threadIdx.x; k < kHid * 3 + 4; k += blockDim.x) acc[k] = 0.f;
  for (int k = threadIdx.x; k < kHid * 3; k += blockDim.x) w[k] = Wout[k];
  __syncthreads();
  const float scale = 2.f / (3.f * (float)n);
  // one warp per row: lanes own features 2*lane, 2*lane+1
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float pw[2][3] = {{0, 0, 0}, {0, 0, 0}}, pb[3] = {0, 0, 0}, pl = 0.f;
  const int64_t nwarps = tstride() >> 5;
  for (int64_t i = tid() >> 5; i < n; i += nwarps) {
    float dy[3];
    for (int c = 0; c < 3; ++c) {
      const float d = Y[3 * i + c] - T[3 * i + c];
      dy[c] = scale * d;
      if (lane == 0) {
        pb[c] += dy[c];
        pl += d * d;
      }
    }
    const float h0 = bf(H + i * kHid + 2 * lane), h1 = bf(H + i * kHid + 2 * lane + 1);
    for (int c = 0; c < 3; ++c) {
      pw[0][c] += h0 * dy[c];
      pw[1][c] += h1 * dy[c];
    }
    dH[i * kHid + 2 * lane] = dy[0] * w[3 * (2 * lane)] + dy[1] * w[3 * (2 * lane) + 1] +
                             dy[2] * w[3 * (2 * lane) + 2];
    dH[i * kHid + 2 * lane + 1] = dy[0] * w[3 * (2 * lane + 1)] +
                                 dy[1] * w[3 * (2 * lane + 1) + 1] +
                                 dy[2] * w[3 * (2 * lane + 1) + 2];
  }
  // fixed-order block accumulation: warps in turn
  for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) {
    if (warp == wv) {
      for (int c = 0; c < 3; ++c) {
        acc[3 * (2 * lane) + c] += pw[0][c];
        acc[3 * (2 * lane + 1) + c] += pw[1][c];
      }
      if (lane == 0) {
        for (int c = 0; c < 3; ++c) acc[kHid * 3 + c] += pb[c];
        acc[kHid * 3 + 3] += pl;
      }
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < kHid * 3 + 4; k += blockDim.x)
    part[(int64_t)blockIdx.x * (kHid * 3 + 4) + k] = acc[k];
}

// For one layer: dA = dH (.) [h > 0]; block partials of dW (X^T dA, X = [h_prev, z]) and db;
// dXself = dA W^T[:, :64] -> dHprev, dZ = dA W^T[:, 64:]
__global__ void __launch_bounds__(kThreads) k_layer_bwd(int64_t n, const float* __restrict__ dH,
                                                        const __nv_bfloat16* __restrict__ Hcur,
                                                        const __nv_bfloat16* __restrict__ Hprev,
                                                        const __nv_bfloat16* __restrict__ Z,
                                                        const float* __restrict__ W,  // [128][64]
                                                        float* __restrict__ dHprev,
                                                        float* __restrict__ dZ,
                                                        float* __restrict__ part) {
  // part per block: [128*64 dW][64 db]
  extern __shared__ __align__(16) unsigned char smem[];
  float* WsT = reinterpret_cast<float*>(smem);          // [64][128]: WsT[c][f] = W[f][c]
  float* Xr = WsT + 2 * kHid * kHid;                    // [8 warps][128]
  float* Dr = Xr + 8 * 2 * kHid;                        // [8 warps][64]
  for (int k = threadIdx.x; k < 2 * kHid * kHid; k += blockDim.x)
    WsT[(k % kHid) * 2 * kHid + k / kHid] = W[k];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // each thread owns dW entries (f, c) for f in {lane + 32 q}, c in {2 warp .. } ... use a
  // simple ownership: thread k owns 32 consecutive entries of the flattened [128][64] block
  float pw[32];
  for (int q = 0; q < 32; ++q) pw[q] = 0.f;
  float pb[2] = {0.f, 0.f};
  const int64_t nwarps = tstride() >> 5;
  // rows are processed warp-synchronously in rounds so that every warp's row is staged before
  // the block-wide dW accumulation of that round
  const int64_t rounds = (n + nwarps - 1) / nwarps;
  for (int64_t rd = 0; rd < rounds; ++rd) {
    const int64_t i = rd * nwarps + (tid() >> 5);
    float* xr = Xr + warp * 2 * kHid;
    float* dr = Dr + warp * kHid;
    if (i < n) {
      for (int c = lane; c < kHid; c += 32) {
        const float hc = bf(Hcur + i * kHid + c);
        const float d = hc > 0.f ? dH[i * kHid + c] : 0.f;
        dr[c] = d;
        xr[c] = bf(Hprev + i * kHid + c);
        xr[kHid + c] = bf(Z + i * kHid + c);
      }
    } else {
      for (int c = lane; c < kHid; c += 32) {
        dr[c] = 0.f;
        xr[c] = 0.f;
        xr[kHid + c] = 0.f;
      }
    }
    __syncwarp();
    if (i < n) {
      // dX[f] = sum_c dA[c] W[f][c], f = lane + 32 q
      for (int q = 0; q < 4; ++q) {
        const int f = lane + 32 * q;
        float s = 0.f;
        for (int c = 0; c < kHid; ++c) s += dr[c] * WsT[c * 2 * kHid + f];
        if (f < kHid)
          dHprev[i * kHid + f] = s;
        else
          dZ[i * kHid + f - kHid] = s;
      }
      pb[0] += dr[lane];
      pb[1] += dr[lane + 32];
    }
    __syncthreads();
    // dW[f][c] += sum over the round's rows of X[f] dA[c]; thread t owns entries 32t .. 32t+31
    for (int w8 = 0; w8 < 8; ++w8) {
      const float* xw = Xr + w8 * 2 * kHid;
      const float* dw = Dr + w8 * kHid;
      for (int q = 0; q < 32; ++q) {
        const int k = 32 * threadIdx.x + q;
        pw[q] += xw[k / kHid] * dw[k % kHid];
      }
    }
    __syncthreads();
  }
  float* pp = part + (int64_t)blockIdx.x * (2 * kHid * kHid + kHid);
  for (int q = 0; q < 32; ++q) pp[32 * threadIdx.x + q] = pw[q];
  // db: lanes of each warp hold two columns; sum warps in fixed order through shared memory
  __syncthreads();
  for (int wv = 0; wv < 8; ++wv) {
    if (warp == wv) {
      if (wv == 0) {
        Dr[lane] = pb[0];
        Dr[lane + 32] = pb[1];
      } else {
        Dr[lane] += pb[0];
        Dr[lane + 32] += pb[1];
      }
    }
    __syncthreads();
  }
  for (int c = threadIdx.x; c < kHid; c += blockDim.x) pp[2 * kHid * kHid + c] = Dr[c];
}

// dH_prev += A^T dZ (SELL with transposed weights), 64-wide, warp per row
__global__ void k_agg_t(int64_t n, DSell S, const float* __restrict__ At, const float* __restrict__ dZ,
                        float* __restrict__ dH) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = tstride() >> 5;
  for (int64_t i = tid() >> 5; i < n; i += nwarps) {
    const int64_t s = i >> 5, li = i & 31;
    const int64_t sb = S.sptr[s];
    const int len = S.slen[s];
    float a0 = 0.f, a1 = 0.f;
    for (int k = 0; k < len; ++k) {
      const int64_t e = sb + (int64_t)k * 32 + li;
      const int64_t j = S.col[e];
      const float a = At[e];
      a0 += a * dZ[j * kHid + lane];
      a1 += a * dZ[j * kHid + lane + 32];
    }
    dH[i * kHid + lane] += a0;
    dH[i * kHid + lane + 32] += a1;
  }
}

// input layer backward: block partials of dW_in (F^T dA0) and db_in
__global__ void __launch_bounds__(kThreads) k_in_bwd(int64_t n, const float* __restrict__ dH,
                                                     const __nv_bfloat16* __restrict__ H0,
                                                     const __nv_bfloat16* __restrict__ F,
                                                     float* __restrict__ part) {
  // part per block: [16*64 dW_in][64 db_in]; thread t owns dW entries 4t .. 4t+3
  float pw[4] = {0, 0, 0, 0};
  float pb = 0.f;
  const int t = threadIdx.x;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    for (int q = 0; q < 4; ++q) {
      const int k = 4 * t + q;
      const int f = k / kHid, c = k % kHid;
      const float d = bf(H0 + i * kHid + c) > 0.f ? dH[i * kHid + c] : 0.f;
      pw[q] += bf(F + i * kFeat + f) * d;
    }
    if (t < kHid) pb += bf(H0 + i * kHid + t) > 0.f ? dH[i * kHid + t] : 0.f;
  }
  float* pp = part + (int64_t)blockIdx.x * (kFeat * kHid + kHid);
  for (int q = 0; q < 4; ++q) pp[4 * t + q] = pw[q];
  if (t < kHid) pp[kFeat * kHid + t] = pb;
}

// grad[k] = sum over blocks of part[b][k] (fixed block order)
__global__ void k_reduce_parts(int nblocks, int count, int stride, const float* __restrict__ part,
                               float* __restrict__ grad) {
  for (int64_t k = tid(); k < count; k += tstride()) {
    float s = 0.f;
    for (int b = 0; b < nblocks; ++b) s += part[(int64_t)b * stride + k];
    grad[k] = s;
  }
}

__global__ void k_adam(int64_t count, float* __restrict__ w, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  for (int64_t k = tid(); k < count; k += tstride()) {
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.f - b1) * gk;
    const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    w[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
  }
}

// bf16 transposed weight copies for the tensor-core layers: dst[o][i] = src[i][o]
__global__ void k_transpose_bf16(int rows, int cols, const float* __restrict__ src,
                                 __nv_bfloat16* __restrict__ dst) {
  for (int64_t k = tid(); k < (int64_t)rows * cols; k += tstride()) {
    const int i = (int)(k / cols), o = (int)(k % cols);
    dst[(int64_t)o * rows + i] = __float2bfloat16_rn(src[k]);
  }
}

__global__ void k_loss_sum(int nblocks, const float* __restrict__ part, int width,
                           float* __restrict__ out) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    float s = 0.f;
    for (int b = 0; b < nblocks; ++b) s += part[(int64_t)b * width + width - 1];
    *out = s;
  }
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------------------------
static inline int grid_rows(const Launch& L, int64_t n) {
  int64_t b = (n + kRows - 1) / kRows;
  const int64_t cap = (int64_t)L.max_blocks;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

size_t mpnn_layer_smem() { return kTcSmem; }
size_t mpnn_layer_bwd_smem() { return (size_t)(2 * kHid * kHid + 8 * 2 * kHid + 8 * kHid) * 4; }

template <typename T>
cudaError_t mpnn_features(const Launch& L, int64_t n, const T* m, int64_t ld, const uint8_t* mag,
                          const T* up, const T* up2, double l100, double l111,
                          double ls, double us, __nv_bfloat16* F) {
  (*L.counter) += 1;
  k_features<T><<<L.blocks_for(n), kBlock, 0, L.stream>>>(n, m, ld, mag, up, up2, l100, l111,
                                                          1.0 / ls, 1.0 / us, F);
  return cudaGetLastError();
}
template cudaError_t mpnn_features<double>(const Launch&, int64_t, const double*, int64_t,
                                           const uint8_t*, const double*, const double*, double,
                                           double, double, double, __nv_bfloat16*);
template cudaError_t mpnn_features<float>(const Launch&, int64_t, const float*, int64_t,
                                          const uint8_t*, const float*, const float*, double,
                                          double, double, double, __nv_bfloat16*);

cudaError_t mpnn_forward(const Launch& L, int64_t n, const DSell& S, const MpnnDev& W,
                         const __nv_bfloat16* F, __nv_bfloat16* const H[4],
                         __nv_bfloat16* const Z[3]) {
  const int g = grid_rows(L, n);
  const size_t sm = mpnn_layer_smem();
  (*L.counter) += 1;
  k_tc_layer<0><<<g, kThreads, sm, L.stream>>>(n, S, W.A, F, W.WinT, W.b_in, H[0], nullptr,
                                               W.err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int l = 0; l < kLayers; ++l) {
    (*L.counter) += 1;
    k_tc_layer<1><<<g, kThreads, sm, L.stream>>>(n, S, W.A, H[l], W.WT[l], W.b[l], H[l + 1],
                                                 Z ? Z[l] : nullptr, W.err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t mpnn_output(const Launch& L, int64_t n, const MpnnDev& W, const __nv_bfloat16* H3,
                        int mode, float* Y, const T* up, const T* up2, double us, T* x0) {
  (*L.counter) += 1;
  k_output<T><<<L.blocks_for(n), kBlock, 0, L.stream>>>(n, H3, W.Wout, W.bout, mode, Y, up, up2,
                                                      us, x0);
  return cudaGetLastError();
}

template cudaError_t mpnn_output<double>(const Launch&, int64_t, const MpnnDev&,
                                         const __nv_bfloat16*, int, float*, const double*,
                                         const double*, double, double*);
template cudaError_t mpnn_output<float>(const Launch&, int64_t, const MpnnDev&,
                                        const __nv_bfloat16*, int, float*, const float*,
                                        const float*, double, float*);

cudaError_t mpnn_backward(const Launch& L, int64_t n, const DSell& S, const MpnnDev& W,
                          const __nv_bfloat16* F, __nv_bfloat16* const H[4],
                          __nv_bfloat16* const Z[3], const float* Y, const float* T, float* dHa,
                          float* dHb, float* dZ, float* part, float* grad, float* loss) {
  // grad layout = parameter layout: W_in, b_in, {W_l, b_l} x 3, W_out, b_out
  const int gb = grid_rows(L, n);
  cudaError_t e;
  const int wout = kHid * 3 + 4;
  (*L.counter) += 2;
  k_out_bwd<<<gb, kThreads, 0, L.stream>>>(n, Y, T, H[kLayers], W.Wout, dHa, part);
  float* g_out = grad + kOffWout;
  k_reduce_parts<<<1, 256, 0, L.stream>>>(gb, wout - 1, wout, part, g_out);  // W_out, b_out
  (*L.counter) += 1;
  k_loss_sum<<<1, 32, 0, L.stream>>>(gb, part, wout, loss);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  float* dH = dHa;
  float* dHp = dHb;
  const int wl = 2 * kHid * kHid + kHid;
  const size_t sm = mpnn_layer_bwd_smem();
  for (int l = kLayers - 1; l >= 0; --l) {
    (*L.counter) += 3;
    k_layer_bwd<<<gb, kThreads, sm, L.stream>>>(n, dH, H[l + 1], H[l], Z[l], W.Wf[l], dHp, dZ,
                                                part);
    k_reduce_parts<<<(wl + 255) / 256, 256, 0, L.stream>>>(gb, wl, wl, part, grad + kOffW[l]);
    k_agg_t<<<L.blocks_for(n * 32), kBlock, 0, L.stream>>>(n, S, W.At, dZ, dHp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    float* t = dH;
    dH = dHp;
    dHp = t;
  }
  const int wi = kFeat * kHid + kHid;
  (*L.counter) += 2;
  k_in_bwd<<<gb, kThreads, 0, L.stream>>>(n, dH, H[0], F, part);
  k_reduce_parts<<<(wi + 255) / 256, 256, 0, L.stream>>>(gb, wi, wi, part, grad);
  return cudaGetLastError();
}

cudaError_t mpnn_adam(const Launch& L, float* w, const float* g, float* m, float* v, float lr,
                      int t) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  (*L.counter) += 1;
  k_adam<<<L.blocks_for(kParams), kBlock, 0, L.stream>>>(kParams, w, g, m, v, lr, b1, b2, 1e-8f,
                                                         c1, c2);
  return cudaGetLastError();
}

cudaError_t mpnn_refresh_bf16(const Launch& L, __nv_bfloat16* WinT, __nv_bfloat16* const WT[3],
                              const float* params) {
  (*L.counter) += 1 + kLayers;
  k_transpose_bf16<<<8, 256, 0, L.stream>>>(kFeat, kHid, params + kOffWin, WinT);
  for (int l = 0; l < kLayers; ++l)
    k_transpose_bf16<<<32, 256, 0, L.stream>>>(2 * kHid, kHid, params + kOffW[l], WT[l]);
  return cudaGetLastError();
}

cudaError_t mpnn_setup_smem() {
  cudaError_t e = cudaFuncSetAttribute(k_tc_layer<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)mpnn_layer_smem());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_tc_layer<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)mpnn_layer_smem());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_layer_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)mpnn_layer_bwd_smem());
}

}  // namespace gspm
