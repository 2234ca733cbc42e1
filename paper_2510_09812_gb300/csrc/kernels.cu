// GSPM kernels for sm_103a.  The path is HBM-bound: sparse row gathers over a SELL-32 node graph
// (one thread per node row, one warp per 32-row slice, every (k, b) value run of a slice one
// coalesced 128/256-byte load), FP64 reductions with a fixed summation order, and fused
// pointwise updates.  Matrix values and column indices are streamed with evict-first loads so
// that the gathered vectors stay resident in L2.
//
// A context holds one or more meshes ("segments", a batch), concatenated slice-aligned in one
// SELL structure.  Everything that reduces (CG inner products, volume averages, the projection's
// <|dm|>) runs over a static list of work items (segment, slice range): each item leaves one
// partial per component and the last item of a segment to arrive sums that segment's partials in
// item order, so results are per mesh and bitwise reproducible.  CG scalars, pins, applied
// fields and volume averages are per segment; a segment whose CG converged skips its items.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <type_traits>
#include <unordered_map>

#include "kernels.cuh"

namespace gspm {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(kFull, x, o);
  return x;
}

// Compensated summation (Kahan): s + c carries the running sum with the low-order part lost by
// each add kept in c (subtracted at the end: total = s - c)
template <typename T>
__device__ __forceinline__ void kahan_add(T& s, T& c, T x) {
  const T y = x - c;
  const T t = s + y;
  c = (t - s) - y;
  s = t;
}

__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

// Programmatic dependent launch (the CG loop kernels): a kernel launched with
// launch_pdl first waits until the previous kernel of the stream has completed and its memory
// is visible, then lets the next kernel be scheduled (its blocks wait the same way), so
// launch latency overlaps the running kernel.  Outside such a launch both are no-ops.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// The last item of `seg` to arrive (its block partials already in red.partial[item]) sums the
// segment's item partials in item order and returns true (totals in res[0..NC), valid in every
// thread of that block).
template <int NC>
__device__ __forceinline__ bool seg_arrive(int item, int seg, const DSeg& G, const ItemList& IL,
                                           const Red& red, double* res) {
  __shared__ double sm[NC][32];
  __shared__ int am_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(G.counter + seg, 1u);
    am_last = (t == (unsigned)IL.seg_nitems[seg] - 1u);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  const int i0 = IL.seg_item0[seg], ni = IL.seg_nitems[seg];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < ni; b += blockDim.x)
      acc += __ldcg(red.partial + (int64_t)(i0 + b) * kRedComp + c);
    acc = warp_sum(acc);
    if (lane == 0) sm[c][warp] = acc;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const double x = warp_sum(lane < nw ? sm[c][lane] : 0.0);
      if (lane == 0) res[c] = x;
    }
  }
  if (threadIdx.x == 0) G.counter[seg] = 0u;
  __syncthreads();
  return true;
}

// Block reduction of NC values into partial[item] (FP64 tree), then seg_arrive.
template <int NC>
__device__ __forceinline__ bool seg_reduce(double (&v)[NC], int item, int seg, const DSeg& G,
                                           const ItemList& IL, const Red& red, double* res) {
  __shared__ double sm[NC][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const double x = warp_sum(v[c]);
    if (lane == 0) sm[c][warp] = x;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const double x = warp_sum(lane < nw ? sm[c][lane] : 0.0);
      if (lane == 0) red.partial[(int64_t)item * kRedComp + c] = x;
    }
  }
  return seg_arrive<NC>(item, seg, G, IL, red, res);
}

// Double-float addition (h, l) += (bh, bl): Knuth's TwoSum of the high parts, the low parts
// added to its error term, renormalised (the _rn intrinsics keep the compiler from contracting
// or reassociating the steps)
__device__ __forceinline__ void df_add(float& h, float& l, float bh, float bl) {
  const float s = __fadd_rn(h, bh);
  const float z = __fsub_rn(s, h);
  float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, z)), __fsub_rn(bh, z));
  e = __fadd_rn(e, __fadd_rn(l, bl));
  h = __fadd_rn(s, e);
  l = __fsub_rn(e, __fsub_rn(h, s));
}

// seg_reduce of per-thread values given as unevaluated sums hi + lo in T.  T = float: the warp
// and block trees run in double-float arithmetic (FP32 operations, about 44 significant bits;
// an FP64 instruction costs ~64 FP32 ones on this part and the FP64 trees dominated the short
// CG vector kernels), one FP64 conversion per block and value.  T = double: seg_reduce.
template <typename T, int NC>
__device__ __forceinline__ bool seg_reduce_hl(const T (&hi)[NC], const T (&lo)[NC], int item,
                                              int seg, const DSeg& G, const ItemList& IL,
                                              const Red& red, double* res) {
  if constexpr (std::is_same<T, double>::value) {
    double v[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) v[c] = hi[c] + lo[c];
    return seg_reduce<NC>(v, item, seg, G, IL, red, res);
  } else {
    __shared__ float smh[NC][32], sml[NC][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      float h = hi[c], l = lo[c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float bh = __shfl_down_sync(kFull, h, o), bl = __shfl_down_sync(kFull, l, o);
        df_add(h, l, bh, bl);
      }
      if (lane == 0) {
        smh[c][warp] = h;
        sml[c][warp] = l;
      }
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        float h = lane < nw ? smh[c][lane] : 0.f, l = lane < nw ? sml[c][lane] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float bh = __shfl_down_sync(kFull, h, o), bl = __shfl_down_sync(kFull, l, o);
          df_add(h, l, bh, bl);
        }
        if (lane == 0) red.partial[(int64_t)item * kRedComp + c] = (double)h + (double)l;
      }
    }
    return seg_arrive<NC>(item, seg, G, IL, red, res);
  }
}

// The difference forms sum_j A_ij (x_j - x_i) of the zero-row-sum operators (K^ms, K^mech, F^ms,
// G) are used in FP32, where they keep smooth fields from cancelling; in FP64 the plain products
// are accurate enough and each extra subtraction costs FP64 issue slots.
template <typename T>
constexpr int kDiff = std::is_same<T, float>::value ? 1 : 0;

__device__ __forceinline__ bool row_valid(const DSeg& G, int seg, int64_t row) {
  return row - G.seg_row0[seg] < G.seg_nrow[seg];
}

// y_r(row) = sum_k A(row, k) x_r(col(row, k)) for one row of a scalar SELL matrix, neighbours
// k = k0, k0 + kstep, ...  diff != 0 (an operator whose rows sum to zero: K^ms, K^mech): formed as
// sum_k A(row, k) (x_r(col) - x_r(row)), equal in exact arithmetic; a smooth x then does not
// cancel in the sum, and the FP32 rounding of the values cannot make the operator act on the
// constants (its rows' rounded sums no longer enter).
template <typename V, typename X, typename Acc, int NR, int VAR = 0>
__device__ __forceinline__ void sell_scalar_row(const DSell& A, const V* __restrict__ val,
                                                int64_t s, int lane, const X* __restrict__ x,
                                                int64_t ld, const int (&skip)[NR],
                                                Acc (&acc)[NR], int k0 = 0, int kstep = 1,
                                                int diff = 0) {
  const int64_t base = A.sptr[s];
  const int len = A.slen[s];
  const int32_t* cp = A.col + base + lane;
  const V* vp = val + base + lane;
  const int64_t row = s * 32 + lane;
  X xi[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    acc[r] = Acc(0);
    xi[r] = diff && row < A.n ? x[r * ld + row] : X(0);
  }
  if (VAR == 1 || VAR == 3) {
    // eight neighbours per round: their columns and values first, then the gathers, then the
    // FMAs (more loads in flight per thread).  Past the row's end the round re-reads entry kb
    // (kb < len), so every load is unconditional and inside the slice, with weight 0.
    for (int kb = k0; kb < len; kb += 8 * kstep) {
      int j[8];
      V w[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int k = kb + u * kstep;
        const int kc = k < len ? k : kb;
        j[u] = __ldcs(cp + (int64_t)kc * 32);
        const V wv = __ldcs(vp + (int64_t)kc * 32);
        w[u] = k < len ? wv : V(0);
      }
#pragma unroll
      for (int r = 0; r < NR; ++r)
        if (!skip[r]) {
          X g[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) g[u] = __ldg(x + r * ld + j[u]) - xi[r];
#pragma unroll
          for (int u = 0; u < 8; ++u) acc[r] += (Acc)w[u] * (Acc)g[u];
        }
    }
    return;
  }
#pragma unroll 4
  for (int k = k0; k < len; k += kstep) {
    const int j = __ldcs(cp + (int64_t)k * 32);
    const Acc a = (Acc)__ldcs(vp + (int64_t)k * 32);
#pragma unroll
    for (int r = 0; r < NR; ++r)
      if (!skip[r]) acc[r] += a * (Acc)(__ldg(x + r * ld + j) - xi[r]);
  }
}

// 3x3-block row: y(row, a) = sum_k sum_b A(row, k)_ab x(col, b); x, y arrays of [n][3].
// diff != 0: sum_k A(row, k) (x(col) - x(row)), as in sell_scalar_row.
template <typename V, typename X, typename Acc, int VAR>
__device__ __forceinline__ void sell_block_row(const DSell& A, const V* __restrict__ val,
                                               int64_t s, int lane, const X* __restrict__ x,
                                               Acc (&acc)[3], int k0 = 0, int kstep = 1,
                                               int diff = 0) {
  const int64_t base = A.sptr[s];
  const int len = A.slen[s];
  const int32_t* cp = A.col + base + lane;
  const V* vp = val + base * 9 + lane;
  const int64_t row = s * 32 + lane;
  const bool own = diff && row < A.n;
  const X xi0 = own ? x[3 * row] : X(0), xi1 = own ? x[3 * row + 1] : X(0),
          xi2 = own ? x[3 * row + 2] : X(0);
  acc[0] = acc[1] = acc[2] = Acc(0);
  if (VAR == 1 || VAR == 3) {
    // five neighbours per round: all loads first, then the FMAs; past the row's end entry kb
    // is re-read with weight 0 (unconditional loads, all inside the slice)
    for (int kb = k0; kb < len; kb += 5 * kstep) {
      int j[5];  // 32-bit: five fewer registers than 64-bit indices in this unrolled round
      V w[5][9];
#pragma unroll
      for (int u = 0; u < 5; ++u) {
        const int k = kb + u * kstep;
        const bool ok = k < len;
        const int kc = ok ? k : kb;
        j[u] = __ldcs(cp + (int64_t)kc * 32);
        const V* bp = vp + (int64_t)kc * 288;
#pragma unroll
        for (int e = 0; e < 9; ++e) {
          const V wv = __ldcs(bp + e * 32);
          w[u][e] = ok ? wv : V(0);
        }
      }
#pragma unroll
      for (int u = 0; u < 5; ++u) {
        const X* xj = x + 3 * (int64_t)j[u];
        const Acc x0 = (Acc)(__ldg(xj) - xi0), x1 = (Acc)(__ldg(xj + 1) - xi1),
                  x2 = (Acc)(__ldg(xj + 2) - xi2);
#pragma unroll
        for (int a = 0; a < 3; ++a)
          acc[a] += (Acc)w[u][3 * a] * x0 + (Acc)w[u][3 * a + 1] * x1 + (Acc)w[u][3 * a + 2] * x2;
      }
    }
  } else {
#pragma unroll 2
    for (int k = k0; k < len; k += kstep) {
      const int64_t j = __ldcs(cp + (int64_t)k * 32);
      const V* bp = vp + (int64_t)k * 288;
      const Acc x0 = (Acc)(__ldg(x + 3 * j) - xi0), x1 = (Acc)(__ldg(x + 3 * j + 1) - xi1),
                x2 = (Acc)(__ldg(x + 3 * j + 2) - xi2);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        acc[a] += (Acc)__ldcs(bp + (3 * a + 0) * 32) * x0;
        acc[a] += (Acc)__ldcs(bp + (3 * a + 1) * 32) * x1;
        acc[a] += (Acc)__ldcs(bp + (3 * a + 2) * 32) * x2;
      }
    }
  }
}

// Compensated dot product in FP32 (Ogita, Rump and Oishi, "Accurate sum and dot product", SIAM
// J. Sci. Comput. 26 (2005), Algorithm Dot2): each product is split exactly into p + e with an
// FMA, the running sum kept exactly as s plus the accumulated errors c by Knuth's TwoSum, so
// s + c is as accurate as the dot product computed in twice the working precision.  The CG
// initial residuals b - A x (which cancel heavily with a warm start) use it instead of FP64
// arithmetic, whose rate on this part is 1/64 of FP32's.
struct Dot2 {
  float s = 0.f, c = 0.f;
  // the _rn intrinsics keep the compiler from contracting or reassociating these steps
  __device__ __forceinline__ void add(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = fmaf(a, b, -p);
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float d = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    c = __fadd_rn(c, __fadd_rn(d, e));
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// sell_scalar_row / sell_block_row with Dot2 accumulators (FP32 operands)
template <int NR>
__device__ __forceinline__ void sell_scalar_row_dot2(const DSell& A, const float* __restrict__ val,
                                                     int64_t s, int lane,
                                                     const float* __restrict__ x, int64_t ld,
                                                     Dot2 (&acc)[NR], int diff = 0) {
  const int64_t base = A.sptr[s];
  const int len = A.slen[s];
  const int32_t* cp = A.col + base + lane;
  const float* vp = val + base + lane;
  const int64_t row = s * 32 + lane;
  float xi[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) xi[r] = diff && row < A.n ? x[r * ld + row] : 0.f;
#pragma unroll 4
  for (int k = 0; k < len; ++k) {
    const int j = __ldcs(cp + (int64_t)k * 32);
    const float a = __ldcs(vp + (int64_t)k * 32);
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r].add(a, __fsub_rn(__ldg(x + r * ld + j), xi[r]));
  }
}
__device__ __forceinline__ void sell_block_row_dot2(const DSell& A, const float* __restrict__ val,
                                                    int64_t s, int lane,
                                                    const float* __restrict__ x,
                                                    Dot2 (&acc)[3], int diff = 0) {
  const int64_t base = A.sptr[s];
  const int len = A.slen[s];
  const int32_t* cp = A.col + base + lane;
  const float* vp = val + base * 9 + lane;
  const int64_t row = s * 32 + lane;
  const bool own = diff && row < A.n;
  const float xi0 = own ? x[3 * row] : 0.f, xi1 = own ? x[3 * row + 1] : 0.f,
              xi2 = own ? x[3 * row + 2] : 0.f;
#pragma unroll 2
  for (int k = 0; k < len; ++k) {
    const int64_t j = __ldcs(cp + (int64_t)k * 32);
    const float* bp = vp + (int64_t)k * 288;
    const float x0 = __fsub_rn(__ldg(x + 3 * j), xi0), x1 = __fsub_rn(__ldg(x + 3 * j + 1), xi1),
                x2 = __fsub_rn(__ldg(x + 3 * j + 2), xi2);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      acc[a].add(__ldcs(bp + (3 * a + 0) * 32), x0);
      acc[a].add(__ldcs(bp + (3 * a + 1) * 32), x1);
      acc[a].add(__ldcs(bp + (3 * a + 2) * 32), x2);
    }
  }
}

// Work unit of the SELL kernels for schedule VAR: one slice per warp (VAR 0, 1), or half a slice
// per warp with two lanes per row (VAR 2).  unit_row() gives, for this lane, the slice, the SELL
// lane of its row, and the first neighbour and stride it handles.
template <int VAR>
__device__ __forceinline__ void unit_row(int64_t u, int lane, int64_t& s, int& sl, int& k0,
                                         int& kstep) {
  if (VAR == 2) {
    s = u >> 1;
    sl = (int)(u & 1) * 16 + (lane & 15);
    k0 = lane >> 4;
    kstep = 2;
  } else {
    s = u;
    sl = lane;
    k0 = 0;
    kstep = 1;
  }
}
// minimum resident blocks per SM a schedule is compiled for (register cap)
template <int VAR>
constexpr int min_blocks() {
  return VAR == 3 ? 3 : 1;
}
template <int VAR>
__device__ __forceinline__ int units_per_slice() {
  return VAR == 2 ? 2 : 1;
}
// combine the two partial row results of VAR 2 (lanes l and l+16); true on the lane that owns
// the row's result
template <int VAR, typename Acc, int N>
__device__ __forceinline__ bool unit_combine(Acc (&acc)[N], int lane) {
  if (VAR != 2) return true;
#pragma unroll
  for (int a = 0; a < N; ++a) acc[a] += __shfl_xor_sync(kFull, acc[a], 16);
  return lane < 16;
}

// ------------------------------------------------------------------------------------------
// volume average per segment: out[seg*nc + c] = sum_i w_i f(i, c) (+ add[c]); Sec. 2.4 with
// nodal weights M_L,i / V(segment)
// ------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kBlock) k_wsum(DSeg G, ItemList IL, int nc, const T* __restrict__ f,
                                                 int64_t cs, int64_t ns,
                                                 const int64_t* __restrict__ perm,
                                                 const double* __restrict__ w, double* out,
                                                 const double* add, Red red) {
  for (int item = blockIdx.x; item < IL.nitems; item += gridDim.x) {
    const int seg = IL.seg[item];
    double v[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) v[c] = 0.0;
    const int64_t r0 = (int64_t)IL.sl0[item] * 32, r1 = (int64_t)IL.sl1[item] * 32;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      if (!row_valid(G, seg, i)) continue;
      const double wi = w[i];
      const int64_t src = perm ? perm[i] : i;
#pragma unroll
      for (int c = 0; c < 9; ++c)
        if (c < nc) v[c] += wi * (double)f[src * ns + c * cs];
    }
    __shared__ double res[9];
    if (seg_reduce<9>(v, item, seg, G, IL, red, res) && threadIdx.x == 0)
      for (int c = 0; c < nc; ++c) out[seg * nc + c] = res[c] + (add ? add[c] : 0.0);
  }
}

// ------------------------------------------------------------------------------------------
// plain SpMV (operator access, autotuning)
// ------------------------------------------------------------------------------------------
template <typename T, int VAR>
__global__ void __launch_bounds__(kBlock, min_blocks<VAR>()) k_spmv1(DSell A, const T* __restrict__ val,
                                                  const T* __restrict__ x, T* __restrict__ y,
                                                  int diff) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = gstride() >> 5;
  const int skip[1] = {0};
  for (int64_t u = gtid() >> 5; u < A.nslices * units_per_slice<VAR>(); u += nw) {
    int64_t s;
    int sl, k0, ks;
    unit_row<VAR>(u, lane, s, sl, k0, ks);
    T acc[1];
    sell_scalar_row<T, T, T, 1, VAR>(A, val, s, sl, x, 0, skip, acc, k0, ks, diff);
    const int64_t row = s * 32 + sl;
    if (unit_combine<VAR>(acc, lane) && row < A.n) y[row] = acc[0];
  }
}

template <typename T, int VAR>
__global__ void __launch_bounds__(kBlock, min_blocks<VAR>()) k_spmv9(DSell A, const T* __restrict__ val,
                                                  const T* __restrict__ x, T* __restrict__ y,
                                                  int diff) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = gstride() >> 5;
  for (int64_t u = gtid() >> 5; u < A.nslices * units_per_slice<VAR>(); u += nw) {
    int64_t s;
    int sl, k0, ks;
    unit_row<VAR>(u, lane, s, sl, k0, ks);
    T acc[3];
    sell_block_row<T, T, T, VAR>(A, val, s, sl, x, acc, k0, ks, diff);
    const int64_t row = s * 32 + sl;
    if (unit_combine<VAR>(acc, lane) && row < A.n) {
      y[3 * row] = acc[0];
      y[3 * row + 1] = acc[1];
      y[3 * row + 2] = acc[2];
    }
  }
}

// ------------------------------------------------------------------------------------------
// conjugate gradients (Sec. 2.5, unpreconditioned), all scalars on the device, per segment
// ------------------------------------------------------------------------------------------
// pc: 0 plain CG, 1 two-level preconditioner (beta from k_pcg_z), 2 Jacobi preconditioner
// fused into the update (rz given here)
__device__ __forceinline__ void cg_start(CGState* st, int* nactive, int nr, const double* bb,
                                         const double* rr, double rtol, int max_iter,
                                         int allow_zero_x, int pc = 0,
                                         const double* rz = nullptr) {
  int any = 0, zero = 0;
  for (int k = 0; k < 3; ++k) {
    CGRhs& q = st->r[k];
    if (k < nr) {
      q.bb = bb[k];
      q.rr = rr[k];
      q.tol2 = rtol * rtol * bb[k];
      q.iters = 0;
      q.alpha = q.beta = q.pq = 0.0;
      q.rz = rz ? rz[k] : 0.0;
      q.done = (bb[k] == 0.0 || rr[k] < q.tol2) ? 1 : 0;
      if (bb[k] == 0.0) zero = 1;
      any |= !q.done;
    } else {
      q = CGRhs{0, 0, 0, 0, 0, 0, 0, 0, 1};
    }
  }
  st->nr = nr;
  st->active = any;
  st->max_iter = max_iter;
  st->noconv = 0;
  st->zero_x = allow_zero_x ? zero : 0;
  st->pc = pc;
  st->proj = 0;
  for (int a = 0; a < 3; ++a) st->sr[a] = st->sub[a] = 0.0;
  if (any) atomicAdd(nactive, 1);
}

// r = b' - A x, p = r (scalar B = 1 or 3x3 block B = 9), one right-hand side, where
//   bmean != NULL: b' = b - bmean[seg] per component (the consistent singular system's
//                  right-hand side: b projected off the constants),
//   pinned:        b' = b with r = 0 at the segment's pinned row (the pinned system; x and b
//                  are 0 there).
template <typename T, int B>
__global__ void __launch_bounds__(kBlock) k_cg_init(DSell A, DSeg G, ItemList IL, const T* __restrict__ val,
                                                    const T* __restrict__ b,
                                                    const T* __restrict__ x,
                                                    T* __restrict__ r, T* __restrict__ p,
                                                    CGState* st, int* nactive, double rtol,
                                                    int max_iter, Red red,
                                                    const double* __restrict__ bmean,
                                                    int pinned, int pc) {
  constexpr int NC = B == 9 ? 3 : 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int item = blockIdx.x; item < IL.nitems; item += gridDim.x) {
    const int seg = IL.seg[item];
    const int64_t pin = pinned ? G.seg_pin[seg] : -1;
    double bm[NC];
#pragma unroll
    for (int a = 0; a < NC; ++a) bm[a] = bmean ? bmean[NC * seg + a] : 0.0;
    double v[2 + NC];  // rr, bb, per-component sums of r
#pragma unroll
    for (int a = 0; a < 2 + NC; ++a) v[a] = 0.0;
    for (int64_t s = IL.sl0[item] + warp; s < IL.sl1[item]; s += kBlock / 32) {
      const int64_t row = s * 32 + lane;
      const bool ok = row_valid(G, seg, row);
      // A x to twice the working precision (FP64, or compensated FP32): with a good initial
      // guess b - A x cancels heavily
      if (B == 1) {
        double acc[1];
        if constexpr (std::is_same<T, float>::value) {
          Dot2 d[1];
          sell_scalar_row_dot2<1>(A, val, s, lane, x, 0, d, 1);
          acc[0] = d[0].value();
        } else {
          const int skip[1] = {0};
          sell_scalar_row<T, T, double, 1>(A, val, s, lane, x, 0, skip, acc, 0, 1, kDiff<T>);
        }
        if (ok) {
          const double bv = (double)b[row] - bm[0];
          const T rv = row == pin ? T(0) : (T)(bv - acc[0]);
          r[row] = rv;
          p[row] = rv;
          v[0] += (double)rv * (double)rv;
          v[1] += bv * bv;
          v[2] += (double)rv;
        }
      } else {
        double acc[3];
        if constexpr (std::is_same<T, float>::value) {
          Dot2 d[3];
          sell_block_row_dot2(A, val, s, lane, x, d, 1);
          for (int a = 0; a < 3; ++a) acc[a] = d[a].value();
        } else {
          sell_block_row<T, T, double, 0>(A, val, s, lane, x, acc, 0, 1, kDiff<T>);
        }
        if (ok) {
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const double bv = (double)b[3 * row + a] - bm[a];
            const T rv = row == pin ? T(0) : (T)(bv - acc[a]);
            r[3 * row + a] = rv;
            p[3 * row + a] = rv;
            v[0] += (double)rv * (double)rv;
            v[1] += bv * bv;
            v[2 + a] += (double)rv;
          }
        }
      }
    }
    __shared__ double res[2 + NC];
    if (seg_reduce<2 + NC>(v, item, seg, G, IL, red, res) && threadIdx.x == 0) {
      // projected form: r.r without the constant part of r, p0 = r0 minus its mean
      const double inv_n = 1.0 / (double)G.seg_nrow[seg];
      double s2 = 0.0;
      for (int a = 0; a < NC; ++a) s2 += res[2 + a] * res[2 + a];
      const double rrp = res[0] - s2 * inv_n;
      const double bb[1] = {res[1]}, rr[1] = {bmean ? (rrp > 0.0 ? rrp : 0.0) : res[0]};
      CGState* sg = st + seg;
      cg_start(sg, nactive, 1, bb, rr, rtol, max_iter, 1, pc);
      if (bmean) {
        sg->proj = 1;
        for (int a = 0; a < NC; ++a) {
          sg->sr[a] = res[2 + a];
          sg->sub[a] = res[2 + a] * inv_n;
        }
      }
    }
  }
}

// GSPM systems (M + c eps K) g = M f with x0 = f already in x: b = M x, r = b - A x, p = r
template <typename T, int NR>
__global__ void __launch_bounds__(kBlock) k_cg_init_gs(DSell A, DSeg G, ItemList IL,
                                                       const T* __restrict__ aval,
                                                       const T* __restrict__ mval, int64_t ld,
                                                       const T* __restrict__ x,
                                                       T* __restrict__ r, T* __restrict__ p,
                                                       CGState* st, int* nactive, double rtol,
                                                       int max_iter, Red red,
                                                       const T* __restrict__ dinv) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int skip[NR] = {};
  for (int item = blockIdx.x; item < IL.nitems; item += gridDim.x) {
    const int seg = IL.seg[item];
    double v[3 * NR];  // rr, bb, rz per right-hand side
#pragma unroll
    for (int k = 0; k < 3 * NR; ++k) v[k] = 0.0;
    for (int64_t s = IL.sl0[item] + warp; s < IL.sl1[item]; s += kBlock / 32) {
      // M x and A x to twice the working precision (FP64, or compensated FP32): their
      // difference (-c eps K x) is small against either
      double ax[NR], mx[NR];
      if constexpr (std::is_same<T, float>::value) {
        Dot2 da[NR], dm[NR];
        sell_scalar_row_dot2<NR>(A, aval, s, lane, x, ld, da);
        sell_scalar_row_dot2<NR>(A, mval, s, lane, x, ld, dm);
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          ax[k] = da[k].value();
          mx[k] = dm[k].value();
        }
      } else {
        sell_scalar_row<T, T, double, NR>(A, aval, s, lane, x, ld, skip, ax);
        sell_scalar_row<T, T, double, NR>(A, mval, s, lane, x, ld, skip, mx);
      }
      const int64_t row = s * 32 + lane;
      if (row_valid(G, seg, row)) {
        const T d = dinv ? dinv[row] : T(1);
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          const T rv = (T)(mx[k] - ax[k]);
          const T zv = d * rv;
          r[k * ld + row] = rv;
          p[k * ld + row] = zv;
          v[3 * k] += (double)rv * (double)rv;
          v[3 * k + 1] += mx[k] * mx[k];
          v[3 * k + 2] += (double)rv * (double)zv;
        }
      }
    }
    __shared__ double res[3 * NR];
    if (seg_reduce<3 * NR>(v, item, seg, G, IL, red, res) && threadIdx.x == 0) {
      double bb[NR], rr[NR], rz[NR];
      for (int k = 0; k < NR; ++k) {
        rr[k] = res[3 * k];
        bb[k] = res[3 * k + 1];
        rz[k] = res[3 * k + 2];
      }
      cg_start(st + seg, nactive, NR, bb, rr, rtol, max_iter, 0, dinv ? 2 : 0, rz);
    }
  }
}

// True residual of a finished K^ms (B = 1) or K^mech (B = 9) solve, independent of the CG
// recursion: per segment, over every row but the pinned one, sum (b - A x)^2 and b^2 into
// out[2 seg] and out[2 seg + 1].  A x is accumulated in FP64 (a product of two FP32 values is
// exact in FP64), so the result measures the solution against the operator as stored.  x is
// zero at the pinned row, so on the other rows A x is the pinned operator's product too.
template <typename T, int B>
__global__ void __launch_bounds__(kBlock) k_true_res(DSell A, DSeg G, ItemList IL,
                                                     const T* __restrict__ val,
                                                     const T* __restrict__ b,
                                                     const T* __restrict__ x,
                                                     const T* __restrict__ xlo, Red red,
                                                     double* out) {
  constexpr int NC = B == 9 ? 3 : 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int item = blockIdx.x; item < IL.nitems; item += gridDim.x) {
    const int seg = IL.seg[item];
    const int64_t pin = G.seg_pin[seg];
    double v[2] = {0.0, 0.0};
    for (int64_t s = IL.sl0[item] + warp; s < IL.sl1[item]; s += kBlock / 32) {
      const int64_t row = s * 32 + lane;
      double acc[3] = {0.0, 0.0, 0.0};
      if (B == 1) {
        const int skip[1] = {0};
        double a1[1];
        sell_scalar_row<T, T, double, 1>(A, val, s, lane, x, 0, skip, a1, 0, 1, kDiff<T>);
        acc[0] = a1[0];
        if (xlo) {
          sell_scalar_row<T, T, double, 1>(A, val, s, lane, xlo, 0, skip, a1, 0, 1, kDiff<T>);
          acc[0] += a1[0];
        }
      } else {
        sell_block_row<T, T, double, 0>(A, val, s, lane, x, acc, 0, 1, kDiff<T>);
        if (xlo) {
          double a3[3];
          sell_block_row<T, T, double, 0>(A, val, s, lane, xlo, a3, 0, 1, kDiff<T>);
          for (int a = 0; a < 3; ++a) acc[a] += a3[a];
        }
      }
      if (row_valid(G, seg, row) && row != pin) {
#pragma unroll
        for (int a = 0; a < NC; ++a) {
          const double bv = (double)b[NC * row + a], rv = bv - acc[a];
          v[0] += rv * rv;
          v[1] += bv * bv;
        }
      }
    }
    __shared__ double res[2];
    if (seg_reduce<2>(v, item, seg, G, IL, red, res) && threadIdx.x == 0) {
      out[2 * seg] = res[0];
      out[2 * seg + 1] = res[1];
    }
  }
}

// q = A p with the p.q dot fused; the segment's last item forms alpha = rr / p.q.
// pinned: q = 0 at the segment's pinned row (the pinned operator; p is 0 there).
// DIFF: the operator's rows sum to zero (K^ms, K^mech), products in difference form
template <typename T, int B, int NR, int VAR, int DIFF>
__global__ void __launch_bounds__(kBlock, min_blocks<VAR>()) k_cg_spmv(DSell A, DSeg G, ItemList IL, const T* __restrict__ val,
                                                    int64_t ld, const T* __restrict__ p,
                                                    T* __restrict__ q, CGState* st, Red red,
                                                    int pinned) {
  pdl_enter();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int item = blockIdx.x; item < IL.nitems; item += gridDim.x) {
    const int seg = IL.seg[item];
    CGState* sg = st + seg;
    if (!sg->active) continue;
    const int64_t pin = pinned ? G.seg_pin[seg] : -1;
    int skip[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) skip[k] = sg->r[k].done;
    // p.q per thread in T with a compensated (Kahan) sum, across threads and items in FP64:
    // the terms p_i (A p)_i cancel heavily for smooth p
    T tv[NR], tc[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) tv[k] = tc[k] = T(0);
    const int64_t u0 = (int64_t)IL.sl0[item] * units_per_slice<VAR>();
    const int64_t u1 = (int64_t)IL.sl1[item] * units_per_slice<VAR>();
    for (int64_t u = u0 + warp; u < u1; u += kBlock / 32) {
      int64_t s;
      int sl, k0, ks;
      unit_row<VAR>(u, lane, s, sl, k0, ks);
      const int64_t row = s * 32 + sl;
      if (B == 1) {
        T acc[NR];
        sell_scalar_row<T, T, T, NR, VAR>(A, val, s, sl, p, ld, skip, acc, k0, ks, DIFF);
        if (row == pin) {
#pragma unroll
          for (int k = 0; k < NR; ++k) acc[k] = T(0);
        }
        if (unit_combine<VAR>(acc, lane) && row_valid(G, seg, row)) {
#pragma unroll
          for (int k = 0; k < NR; ++k)
            if (!skip[k]) {
              q[k * ld + row] = acc[k];
              kahan_add(tv[k], tc[k], p[k * ld + row] * acc[k]);
            }
        }
      } else {
        T acc[3];
        sell_block_row<T, T, T, VAR>(A, val, s, sl, p, acc, k0, ks, DIFF);
        if (row == pin) acc[0] = acc[1] = acc[2] = T(0);
        if (unit_combine<VAR>(acc, lane) && row_valid(G, seg, row)) {
          T pq = T(0);
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            q[3 * row + a] = acc[a];
            pq += p[3 * row + a] * acc[a];
          }
          kahan_add(tv[0], tc[0], pq);
        }
      }
    }
    T lo[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) lo[k] = -tc[k];
    __shared__ double res[NR];
    if (seg_reduce_hl<T, NR>(tv, lo, item, seg, G, IL, red, res) && threadIdx.x == 0) {
      for (int k = 0; k < NR; ++k) {
        CGRhs& c = sg->r[k];
        if (c.done) continue;
        c.pq = res[k];
        if (res[k] > 0.0) {
          c.alpha = (sg->pc ? c.rz : c.rr) / res[k];
        } else {  // p = 0: nothing left to reduce
          c.alpha = 0.0;
          c.done = 1;
        }
      }
    }
  }
}

// 16-byte packs of vector elements for the CG vector kernels
template <typename T> struct Pack16;
template <> struct Pack16<float> { using V = float4; static constexpr int W = 4; };
template <> struct Pack16<double> { using V = double2; static constexpr int W = 2; };

template <typename T>
__device__ __forceinline__ void ld16(const T* p, T (&v)[Pack16<T>::W]) {
  *reinterpret_cast<typename Pack16<T>::V*>(v) = *reinterpret_cast<const typename Pack16<T>::V*>(p);
}
template <typename T>
__device__ __forceinline__ void st16(T* p, const T (&v)[Pack16<T>::W]) {
  *reinterpret_cast<typename Pack16<T>::V*>(p) = *reinterpret_cast<const typename Pack16<T>::V*>(v);
}

// Element range [e0, e1) of an item in a vector of epr elements per row, clipped to the
// segment's rows.  e0 is a multiple of 32 * epr, so 16-byte aligned when the vector is.
__device__ __forceinline__ void item_elems(const DSeg& G, const ItemList& IL, int item, int seg,
                                           int epr, int64_t& e0, int64_t& e1) {
  e0 = (int64_t)IL.sl0[item] * 32 * epr;
  const int64_t rend = G.seg_row0[seg] + G.seg_nrow[seg];
  const int64_t rhi = (int64_t)IL.sl1[item] * 32;
  e1 = (rhi < rend ? rhi : rend) * epr;
}

// x += alpha p, r -= alpha q, r.r fused; the segment's last item forms beta and decides
// convergence.  Vectors hold epr elements per row (1: scalar SoA with stride ld; 3: [n][3]).
// VEC: all vectors 16-byte aligned (and ld a multiple of the pack width), so the item's range
// moves in 16-byte packs with a scalar tail.
// dinv != NULL (scalar rows, Jacobi preconditioner fused): also r.D^-1 r per right-hand side,
// and the segment's last item forms beta = r.z / rz_old.
template <typename T, int NR, bool VEC>
__global__ void __launch_bounds__(kBlock) k_cg_update(DSeg G, ItemList IL, int epr, int64_t ld,
                                                      T* __restrict__ x, T* __restrict__ r,
                                                      const T* __restrict__ p,
                                                      const T* __restrict__ q, CGState* st,
                                                      int* nactive, Red red,
                                                      const T* __restrict__ dinv) {
  pdl_enter();
  constexpr int W = Pack16<T>::W;
  for (int item = blockIdx.x; item < IL.nitems; item += gridDim.x) {
    const int seg = IL.seg[item];
    CGState* sg = st + seg;
    if (!sg->active) continue;
    int skip[NR];
    T al[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      skip[k] = sg->r[k].done;
      al[k] = (T)sg->r[k].alpha;
    }
    const bool proj = NR == 1 && sg->proj;
    // r.r, then r.D^-1 r: each thread sums its elements (a few hundred at most) in T, the
    // block and the items in FP64; projected form: also the sums of r per component (element
    // e of the item has component e mod epr: item ranges start at whole rows)
    T tv[2 * NR + 3];
#pragma unroll
    for (int k = 0; k < 2 * NR + 3; ++k) tv[k] = T(0);
    int64_t e0, e1;
    item_elems(G, IL, item, seg, epr, e0, e1);
    int64_t etail = e0;
    if (VEC) {
      const int64_t np = (e1 - e0) / W;
      for (int64_t t = threadIdx.x; t < np; t += blockDim.x) {
        T dv[W];
        if (dinv) ld16(dinv + e0 + t * W, dv);
        const int cb = epr == 3 ? (int)((t * W) % 3) : 0;
#pragma unroll
        for (int k = 0; k < NR; ++k)
          if (!skip[k]) {
            const int64_t o = k * ld + e0 + t * W;
            T xv[W], rv[W], pv[W], qv[W];
            ld16(x + o, xv);
            ld16(r + o, rv);
            ld16(p + o, pv);
            ld16(q + o, qv);
#pragma unroll
            for (int c = 0; c < W; ++c) {
              xv[c] += al[k] * pv[c];
              rv[c] -= al[k] * qv[c];
              tv[k] += rv[c] * rv[c];
              if (dinv) tv[NR + k] += rv[c] * dv[c] * rv[c];
              if (proj) {
                const int cc = epr == 3 ? (cb + c >= 3 ? cb + c - 3 : cb + c) : 0;
                tv[2 * NR] += cc == 0 ? rv[c] : T(0);
                tv[2 * NR + 1] += cc == 1 ? rv[c] : T(0);
                tv[2 * NR + 2] += cc == 2 ? rv[c] : T(0);
              }
            }
            st16(x + o, xv);
            st16(r + o, rv);
          }
      }
      etail = e0 + np * W;
    }
    for (int64_t i = etail + threadIdx.x; i < e1; i += blockDim.x) {
      const T d = dinv ? dinv[i] : T(0);
#pragma unroll
      for (int k = 0; k < NR; ++k)
        if (!skip[k]) {
          const int64_t o = k * ld + i;
          x[o] += al[k] * p[o];
          const T rv = r[o] - al[k] * q[o];
          r[o] = rv;
          tv[k] += rv * rv;
          tv[NR + k] += rv * d * rv;
          if (proj) {
            const int cc = (int)(i % epr);
            tv[2 * NR] += cc == 0 ? rv : T(0);
            tv[2 * NR + 1] += cc == 1 ? rv : T(0);
            tv[2 * NR + 2] += cc == 2 ? rv : T(0);
          }
        }
    }
    T lo[2 * NR + 3];
#pragma unroll
    for (int k = 0; k < 2 * NR + 3; ++k) lo[k] = T(0);
    __shared__ double res[2 * NR + 3];
    if (seg_reduce_hl<T, 2 * NR + 3>(tv, lo, item, seg, G, IL, red, res) && threadIdx.x == 0) {
      int any = 0;
      for (int k = 0; k < NR; ++k) {
        CGRhs& c = sg->r[k];
        if (c.done) continue;
        c.iters += 1;
        double rrk = res[k];
        if (proj) {
          // r.r without r's constant part; plain CG subtracts r's mean in the p-update
          const double inv_n = 1.0 / (double)G.seg_nrow[seg];
          double s2 = 0.0;
          for (int a = 0; a < 3; ++a) {
            sg->sr[a] = res[2 * NR + a];
            s2 += res[2 * NR + a] * res[2 * NR + a];
            if (sg->pc == 0) sg->sub[a] = res[2 * NR + a] * inv_n;
          }
          rrk -= s2 * inv_n;
          rrk = rrk > 0.0 ? rrk : 0.0;
        }
        if (sg->pc == 0) {
          c.beta = rrk / c.rr;
        } else if (sg->pc == 2) {
          c.beta = c.rz != 0.0 ? res[NR + k] / c.rz : 0.0;
          c.rz = res[NR + k];
        }  // pc 1: beta from r.z in k_pcg_z
        c.rr = rrk;
        if (rrk < c.tol2) {
          c.done = 1;
        } else if (c.iters >= sg->max_iter) {
          c.done = 1;
          sg->noconv += 1;
        }
        any |= !c.done;
      }
      sg->active = any;
      if (!any) atomicSub(nactive, 1);
    }
  }
}

// p = r + beta p
// In a graph loop, block 0 also decides whether the loop runs again (nactive is final: the
// update kernel before this one has finished).
// dinv != NULL: p = D^-1 r + beta p (Jacobi preconditioner, scalar rows)
template <typename T, int NR, bool VEC>
__global__ void __launch_bounds__(kBlock) k_cg_pupdate(DSeg G, ItemList IL, int epr, int64_t ld,
                                                       const T* __restrict__ r,
                                                       T* __restrict__ p, const CGState* st,
                                                       LoopCtl lc, const T* __restrict__ dinv) {
  pdl_enter();
  constexpr int W = Pack16<T>::W;
  if (lc.count && blockIdx.x == 0 && threadIdx.x == 0) {
    const int c = *lc.count + 1;
    *lc.count = c;
    *lc.total += (unsigned long long)lc.body;
    cudaGraphSetConditional(lc.handle, (__ldcg(lc.nactive) > 0 && c < lc.limit) ? 1u : 0u);
  }
  for (int item = blockIdx.x; item < IL.nitems; item += gridDim.x) {
    const int seg = IL.seg[item];
    const CGState* sg = st + seg;
    if (!sg->active) continue;
    int skip[NR];
    T be[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      skip[k] = sg->r[k].done;
      be[k] = (T)sg->r[k].beta;
    }
    // projected form: the input's mean per component comes off (element e of the item has
    // component e mod epr)
    T sb[3] = {T(0), T(0), T(0)};
    if (NR == 1 && sg->proj)
      for (int a = 0; a < 3; ++a) sb[a] = (T)sg->sub[a];
    int64_t e0, e1;
    item_elems(G, IL, item, seg, epr, e0, e1);
    int64_t etail = e0;
    if (VEC) {
      const int64_t np = (e1 - e0) / W;
      for (int64_t t = threadIdx.x; t < np; t += blockDim.x) {
        T dv[W];
        if (dinv) ld16(dinv + e0 + t * W, dv);
        const int cb = epr == 3 ? (int)((t * W) % 3) : 0;
#pragma unroll
        for (int k = 0; k < NR; ++k)
          if (!skip[k]) {
            const int64_t o = k * ld + e0 + t * W;
            T rv[W], pv[W];
            ld16(r + o, rv);
            ld16(p + o, pv);
#pragma unroll
            for (int c = 0; c < W; ++c) {
              const int cc = epr == 3 ? (cb + c >= 3 ? cb + c - 3 : cb + c) : 0;
              const T sub = cc == 0 ? sb[0] : (cc == 1 ? sb[1] : sb[2]);
              pv[c] = ((dinv ? dv[c] * rv[c] : rv[c]) - sub) + be[k] * pv[c];
            }
            st16(p + o, pv);
          }
      }
      etail = e0 + np * W;
    }
    for (int64_t i = etail + threadIdx.x; i < e1; i += blockDim.x) {
      const T d = dinv ? dinv[i] : T(1);
      const int cc = (int)(i % epr);
      const T sub = cc == 0 ? sb[0] : (cc == 1 ? sb[1] : sb[2]);
#pragma unroll
      for (int k = 0; k < NR; ++k)
        if (!skip[k]) {
          const int64_t o = k * ld + i;
          p[o] = (d * r[o] - sub) + be[k] * p[o];
        }
    }
  }
}

// x(i, c) -= x(pin, c) over each segment's rows (element (i, c) at x[i * epr + c]): the
// singular system's solution moved to the pinned system's (zero at the pinned node).  xp holds
// the segment's pinned values, read by k_pin_gather first.
template <typename T>
__global__ void k_pin_gather(DSeg G, int epr, const T* __restrict__ x, double* __restrict__ xp) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G.nseg * epr;
       i += gridDim.x * blockDim.x) {
    const int seg = i / epr, c = i % epr;
    xp[i] = (double)x[G.seg_pin[seg] * epr + c];
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_pin_shift(DSell A, DSeg G, int epr, T* __restrict__ x,
                                                      const double* __restrict__ xp) {
  const int64_t len = (int64_t)A.nslices * 32 * epr;
  for (int64_t e = gtid(); e < len; e += gstride()) {
    const int64_t row = e / epr;
    const int seg = G.seg_of_slice[row >> 5];
    if (!row_valid(G, seg, row)) continue;
    x[e] = (T)((double)x[e] - xp[seg * epr + (int)(e - row * epr)]);
  }
}

// p(i, c) -= st[seg].sub[c] on the active segments of the projected CG (p0 = z0 minus its mean)
template <typename T>
__global__ void __launch_bounds__(kBlock) k_cg_psub(DSell A, DSeg G, int epr, T* __restrict__ p,
                                                    const CGState* __restrict__ st) {
  const int64_t len = (int64_t)A.nslices * 32 * epr;
  for (int64_t e = gtid(); e < len; e += gstride()) {
    const int64_t row = e / epr;
    const int seg = G.seg_of_slice[row >> 5];
    const CGState& sg = st[seg];
    if (!row_valid(G, seg, row) || !sg.active || !sg.proj) continue;
    p[e] -= (T)sg.sub[e - row * epr];
  }
}

// rc(I, a) = sum over the rows i of aggregate I of r(i, a): one block per aggregate, threads
// stride over its rows, block tree in a fixed order, all in T (rc only applies the
// preconditioner; FP64 adds cost ~16x FP32 ones on this part and dominated this kernel).
// With contiguous aggregates the rows are read in order (no row list).
template <typename T, int EPR>
__global__ void __launch_bounds__(kBlock) k_restrict(DCoarse C, const T* __restrict__ r,
                                                     const int64_t* __restrict__ rc_off,
                                                     T* __restrict__ rc) {
  pdl_enter();
  __shared__ T sm[EPR][kBlock / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t I = blockIdx.x; I < C.nagg; I += gridDim.x) {
    T acc[EPR];
#pragma unroll
    for (int a = 0; a < EPR; ++a) acc[a] = T(0);
    // four rows per thread and round: their indices, then their values, then the sums
    const int q0 = C.agg_ptr[I], q1 = C.agg_ptr[I + 1];
    const int64_t first = C.contig && q1 > q0 ? (int64_t)C.agg_rows[q0] - q0 : -1;
    for (int q = q0 + threadIdx.x; q < q1; q += 4 * blockDim.x) {
      int64_t row[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int qq = q + u * blockDim.x;
        row[u] = qq < q1 ? (first >= 0 ? first + qq : (int64_t)C.agg_rows[qq]) : -1;
      }
      T v[4][EPR];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int a = 0; a < EPR; ++a) v[u][a] = row[u] >= 0 ? r[row[u] * EPR + a] : T(0);
#pragma unroll
      for (int a = 0; a < EPR; ++a) acc[a] += (v[0][a] + v[1][a]) + (v[2][a] + v[3][a]);
    }
#pragma unroll
    for (int a = 0; a < EPR; ++a) {
      T v = acc[a];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
      if (lane == 0) sm[a][warp] = v;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int a = 0; a < EPR; ++a) {
        T v = lane < kBlock / 32 ? sm[a][lane] : T(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
        if (lane == 0) {
          const int sg = C.agg_seg[I];
          rc[rc_off[sg] + (I - C.seg_agg0[sg]) * EPR + a] = (T)v;
        }
      }
    }
    __syncthreads();
  }
}


// The same for contiguous aggregates (GSPM_ORDER_AGGREGATE) of scalar rows: one warp per
// aggregate, no barrier.  The aggregate's elements [e0, e1) of r are read as 16-byte packs, kRestrictPacks per
// lane in flight, with the unaligned head and tail (fewer than one pack each) taken by single
// lanes; element e has component e mod EPR.  Each lane sums its packs in order, the warp tree is
// fixed, so the result does not depend on the grid.
constexpr int kRestrictPacks = 8;
template <typename T, int EPR>
__global__ void __launch_bounds__(kBlock) k_restrict_contig(DCoarse C, const T* __restrict__ r,
                                                            const int64_t* __restrict__ rc_off,
                                                            T* __restrict__ rc) {
  pdl_enter();
  constexpr int W = Pack16<T>::W, U = kRestrictPacks;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t I = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; I < C.nagg;
       I += nwarps) {
    const int q0 = C.agg_ptr[I], q1 = C.agg_ptr[I + 1];
    T acc[EPR];
#pragma unroll
    for (int a = 0; a < EPR; ++a) acc[a] = T(0);
    if (q1 > q0) {
      const int64_t e0 = (int64_t)C.agg_rows[q0] * EPR, e1 = e0 + (int64_t)(q1 - q0) * EPR;
      int64_t a0 = (e0 + W - 1) / W * W;
      if (a0 > e1) a0 = e1;
      int64_t a1 = e1 / W * W;
      if (a1 < a0) a1 = a0;
      const int nh = (int)(a0 - e0), nt = (int)(e1 - a1);
      if (lane < nh + nt) {
        const int64_t e = lane < nh ? e0 + lane : a1 + (lane - nh);
        acc[EPR == 1 ? 0 : (int)(e % EPR)] += r[e];
      }
      const int64_t np = (a1 - a0) / W;
      const int cb0 = EPR == 1 ? 0 : (int)(a0 % EPR);
      for (int64_t t0 = 0; t0 < np; t0 += 32 * U) {
        T v[U][W];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t t = t0 + 32 * u + lane;
          if (t < np) {
            ld16(r + a0 + t * W, v[u]);
          } else {
#pragma unroll
            for (int c = 0; c < W; ++c) v[u][c] = T(0);
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t t = t0 + 32 * u + lane;
          // component of the pack's first element: (a0 + t W) mod EPR
          const int cb = EPR == 1 ? 0 : (int)((cb0 + (t % EPR) * (W % EPR)) % EPR);
#pragma unroll
          for (int c = 0; c < W; ++c) {
            if (EPR == 1) {
              acc[0] += v[u][c];
            } else {
              const int cc = (cb + c) % EPR;
#pragma unroll
              for (int a = 0; a < EPR; ++a) acc[a] += cc == a ? v[u][c] : T(0);
            }
          }
        }
      }
    }
#pragma unroll
    for (int a = 0; a < EPR; ++a) {
      T v = acc[a];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
      if (lane == 0) {
        const int sg = C.agg_seg[I];
        rc[rc_off[sg] + (I - C.seg_agg0[sg]) * EPR + a] = v;
      }
    }
  }
}

// N contiguous values through 16-byte packs (N * sizeof(T) a multiple of 16, p aligned)
template <typename T, int N>
__device__ __forceinline__ void ldn(const T* p, T (&v)[N]) {
  constexpr int W = Pack16<T>::W;
#pragma unroll
  for (int k = 0; k < N / W; ++k)
    *reinterpret_cast<typename Pack16<T>::V*>(v + k * W) =
        *reinterpret_cast<const typename Pack16<T>::V*>(p + k * W);
}
template <typename T, int N>
__device__ __forceinline__ void stn(T* p, const T (&v)[N]) {
  constexpr int W = Pack16<T>::W;
#pragma unroll
  for (int k = 0; k < N / W; ++k)
    *reinterpret_cast<typename Pack16<T>::V*>(p + k * W) =
        *reinterpret_cast<const typename Pack16<T>::V*>(v + k * W);
}

// ec = A_c^-1 rc from the stored upper triangle (see launch_coarse_symv), loads of 16-byte packs
// (eight bfloat16 or two doubles), accumulated in T: it only applies the preconditioner, and
// FP64 instructions cost ~16x FP32 ones per warp on this part.
template <typename S>
struct CoarsePack;
template <>
struct CoarsePack<uint16_t> {
  static constexpr int W = 8;
  using Raw = uint4;
  __device__ __forceinline__ static Raw load(const uint16_t* p) {
    return __ldcs(reinterpret_cast<const uint4*>(p));
  }
  __device__ __forceinline__ static Raw zero() { return make_uint4(0u, 0u, 0u, 0u); }
  __device__ __forceinline__ static void cvt(const Raw& u, float (&v)[8]) {
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[2 * k] = __uint_as_float(w[k] << 16);  // bfloat16 -> float is exact
      v[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
    }
  }
};
template <>
struct CoarsePack<double> {
  static constexpr int W = 2;
  using Raw = double2;
  __device__ __forceinline__ static Raw load(const double* p) {
    return __ldcs(reinterpret_cast<const double2*>(p));
  }
  __device__ __forceinline__ static Raw zero() { return make_double2(0.0, 0.0); }
  __device__ __forceinline__ static void cvt(const Raw& u, double (&v)[2]) {
    v[0] = u.x;
    v[1] = u.y;
  }
};

// Tile (I, J) of the stored upper triangle: A_IJ rc_J -> prow[t], and off the diagonal
// A_IJ^T rc_I -> pcol[t].  A warp row-load covers RPW tile rows (LPR lanes per row, W values
// per lane); the row sums reduce over a row's lanes, the column sums over the lanes that hold
// the same columns and then over the warps in a fixed order.
template <typename T, typename S>
__global__ void __launch_bounds__(kBlock) k_coarse_symv_tiles(DSymTiles TL,
                                                              const S* __restrict__ inv,
                                                              const int64_t* __restrict__ rc_off,
                                                              const T* __restrict__ rc,
                                                              T* __restrict__ Q) {
  pdl_enter();
  constexpr int kCoarseTile = coarse_tile<T>();
  constexpr int W = CoarsePack<S>::W, LPR = kCoarseTile / W, RPW = 32 / LPR;
  constexpr int NW = kBlock / 32, RPP = NW * RPW, NP = kCoarseTile / RPP;
  static_assert(LPR <= 32 && NP >= 1, "tile layout");
  __shared__ T srow[kCoarseTile];
  __shared__ T scol[NW][kCoarseTile];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int cp = lane % LPR, rg = lane / LPR;
  for (int64_t t = blockIdx.x; t < TL.ntiles; t += gridDim.x) {
    const int seg = TL.tseg[t], I = TL.tI[t], J = TL.tJ[t];
    const S* tile = inv + t * (int64_t)(kCoarseTile * kCoarseTile);
    const T* xs = rc + rc_off[seg];
    typename CoarsePack<S>::Raw a[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p)
      a[p] = CoarsePack<S>::load(tile + (p * RPP + warp * RPW + rg) * kCoarseTile + cp * W);
    T xj[W];
    ldn<T, W>(xs + (int64_t)J * kCoarseTile + cp * W, xj);
    T cs[W];
#pragma unroll
    for (int c = 0; c < W; ++c) cs[c] = T(0);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const int row = p * RPP + warp * RPW + rg;
      T w[W];
      CoarsePack<S>::cvt(a[p], w);
      T rs = T(0);
#pragma unroll
      for (int c = 0; c < W; ++c) rs += w[c] * xj[c];
#pragma unroll
      for (int o = 1; o < LPR; o <<= 1) rs += __shfl_xor_sync(kFull, rs, o);
      if (cp == 0) srow[row] = rs;
      const T xi = xs[(int64_t)I * kCoarseTile + row];
#pragma unroll
      for (int c = 0; c < W; ++c) cs[c] += w[c] * xi;
    }
#pragma unroll
    for (int o = LPR; o < 32; o <<= 1)
#pragma unroll
      for (int c = 0; c < W; ++c) cs[c] += __shfl_xor_sync(kFull, cs[c], o);
    if (rg == 0)
#pragma unroll
      for (int c = 0; c < W; ++c) scol[warp][cp * W + c] = cs[c];
    __syncthreads();
    if (threadIdx.x < kCoarseTile) {
      const int64_t Tn = TL.seg_T[seg];
      T* q = Q + TL.seg_q0[seg];
      q[((int64_t)I * kCoarseTile + threadIdx.x) * Tn + J] = srow[threadIdx.x];
      if (I != J) {
        T v = T(0);
#pragma unroll
        for (int w = 0; w < NW; ++w) v += scol[w][threadIdx.x];
        q[((int64_t)J * kCoarseTile + threadIdx.x) * Tn + I] = v;
      }
    }
    __syncthreads();
  }
}

// ec(g) = the sum of row g of Q (one warp per coarse row, lanes over the columns, fixed order)
template <typename T>
__global__ void __launch_bounds__(kBlock) k_coarse_symv_sum(DCoarse C, DSymTiles TL, int epr,
                                                            const T* __restrict__ Q,
                                                            T* __restrict__ ec) {
  pdl_enter();
  const int lane = threadIdx.x & 31;
  const int64_t ncoarse = C.nagg * epr;
  for (int64_t g = gtid() >> 5; g < ncoarse; g += gstride() >> 5) {
    const int seg = C.agg_seg[g / epr];
    const int64_t loc = g - (int64_t)C.seg_agg0[seg] * epr;
    const int64_t Tn = TL.seg_T[seg];
    const T* q = Q + TL.seg_q0[seg] + loc * Tn;
    T acc = T(0);
    for (int64_t j = lane; j < Tn; j += 32) acc += q[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(kFull, acc, o);
    if (lane == 0) ec[g] = acc;
  }
}

// z = D^-1 r + P ec, r.z; init: z is the first search direction p.  Four rows per thread and
// round (their 4 * EPR values are whole 16-byte packs: item ranges start at multiples of 32
// rows), the round's r.z summed in T, one FP64 add per round; scalar tail rows.
template <typename T, int EPR>
__global__ void __launch_bounds__(kBlock) k_pcg_z(DSeg G, ItemList IL, DCoarse C,
                                                  const T* __restrict__ r,
                                                  const T* __restrict__ dinv,
                                                  const T* __restrict__ ec,
                                                  T* __restrict__ z, CGState* st, int init,
                                                  Red red) {
  pdl_enter();
  constexpr int N = 4 * EPR;
  for (int item = blockIdx.x; item < IL.nitems; item += gridDim.x) {
    const int seg = IL.seg[item];
    CGState* sg = st + seg;
    if (!sg->active) continue;
    const bool proj = sg->proj;
    const int64_t r0 = (int64_t)IL.sl0[item] * 32;
    const int64_t rend = G.seg_row0[seg] + G.seg_nrow[seg];
    const int64_t rhi = (int64_t)IL.sl1[item] * 32;
    const int64_t r1 = rhi < rend ? rhi : rend;
    const int64_t ng = (r1 - r0) / 4;
    // per thread in T (r.z Kahan-compensated, the sums of z plain: they only give the mean that
    // the projection removes), across threads in double-float
    T rzs = T(0), rzc = T(0), zs[EPR];
#pragma unroll
    for (int a = 0; a < EPR; ++a) zs[a] = T(0);
    for (int64_t g = threadIdx.x; g < ng; g += blockDim.x) {
      const int64_t row = r0 + 4 * g;
      T rv[N], dv[N], zv[N];
      ldn<T, N>(r + row * EPR, rv);
      ldn<T, N>(dinv + row * EPR, dv);
      const int4 ag = *reinterpret_cast<const int4*>(C.agg_of_row + row);
      const int agv[4] = {ag.x, ag.y, ag.z, ag.w};
      T rz = T(0);
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int a = 0; a < EPR; ++a) {
          const int e = u * EPR + a;
          zv[e] = dv[e] * rv[e] + ec[(int64_t)agv[u] * EPR + a];
          rz += rv[e] * zv[e];
          zs[a] += zv[e];
        }
      stn<T, N>(z + row * EPR, zv);
      kahan_add(rzs, rzc, rz);
    }
    for (int64_t row = r0 + 4 * ng + threadIdx.x; row < r1; row += blockDim.x) {
      const int64_t I = C.agg_of_row[row];
#pragma unroll
      for (int a = 0; a < EPR; ++a) {
        const int64_t e = row * EPR + a;
        const T rv = r[e];
        const T zv = dinv[e] * rv + ec[I * EPR + a];
        z[e] = zv;
        kahan_add(rzs, rzc, rv * zv);
        zs[a] += zv;
      }
    }
    T hi[1 + EPR], lo[1 + EPR];
    hi[0] = rzs;
    lo[0] = -rzc;
#pragma unroll
    for (int a = 0; a < EPR; ++a) {
      hi[1 + a] = proj ? zs[a] : T(0);
      lo[1 + a] = T(0);
    }
    __shared__ double res[1 + EPR];
    if (seg_reduce_hl<T, 1 + EPR>(hi, lo, item, seg, G, IL, red, res) && threadIdx.x == 0) {
      CGRhs& c = sg->r[0];
      double rz = res[0];
      if (proj) {
        // z projected off the constants (the p-update subtracts its mean): r.(z - zbar 1)
        const double inv_n = 1.0 / (double)G.seg_nrow[seg];
        for (int a = 0; a < EPR; ++a) {
          const double zbar = res[1 + a] * inv_n;
          rz -= zbar * sg->sr[a];
          sg->sub[a] = zbar;
        }
      }
      if (init) {
        c.rz = rz;
      } else if (!c.done) {
        c.beta = c.rz != 0.0 ? rz / c.rz : 0.0;
        c.rz = rz;
      }
    }
  }
}


__global__ void k_loop_start(LoopCtl lc) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *lc.count = 0;
    cudaGraphSetConditional(lc.handle, __ldcg(lc.nactive) > 0 ? 1u : 0u);
  }
}

__global__ void k_solve_stats(const CGState* st, int nseg, int kind, long long* acc) {
  for (int sg = blockIdx.x * blockDim.x + threadIdx.x; sg < nseg; sg += gridDim.x * blockDim.x) {
    const CGState& c = st[sg];
    int it = 0;
    for (int k = 0; k < c.nr; ++k)
      it = kind == 2 ? it + c.r[k].iters : (c.r[k].iters > it ? c.r[k].iters : it);
    acc[4 * sg + kind] += it;
    acc[4 * sg + 3] += c.noconv;
  }
}

// x = 0 for segments whose right-hand side vanished
template <typename T>
__global__ void k_cg_zero(DSeg G, ItemList IL, int epr, T* x, const CGState* st) {
  for (int item = blockIdx.x; item < IL.nitems; item += gridDim.x) {
    const int seg = IL.seg[item];
    if (!st[seg].zero_x) continue;
    int64_t e0, e1;
    item_elems(G, IL, item, seg, epr, e0, e1);
    for (int64_t i = e0 + threadIdx.x; i < e1; i += blockDim.x) x[i] = T(0);
  }
}

// One round of a row kernel over the F^ms / G values (three per entry): kRowRound neighbours'
// columns and values loaded before any gather, so each lane has that many independent loads in
// flight.  Entries past the row's length give column 0 and value 0 without a load, and their
// addresses are those of entry kb (kb < len), so no address leaves the slice either way.
constexpr int kRowRound = 5;
template <typename T>
__device__ __forceinline__ void row_round(const int32_t* cp, const T* vp, int kb, int len,
                                          int (&j)[kRowRound], T (&f)[kRowRound][3]) {
#pragma unroll
  for (int u = 0; u < kRowRound; ++u) {
    const int k = kb + u;
    const bool ok = k < len;
    const int kc = ok ? k : kb;
    j[u] = ok ? __ldcs(cp + (int64_t)kc * 32) : 0;
    const T* fp = vp + (int64_t)kc * 96;
#pragma unroll
    for (int a = 0; a < 3; ++a) f[u][a] = ok ? __ldcs(fp + 32 * a) : T(0);
  }
}

// ------------------------------------------------------------------------------------------
// F^ms / G operators (Sec. 2.3): right-hand sides and derivatives as row gathers
// ------------------------------------------------------------------------------------------
// Every row of F^ms and of G sums to zero (sum_j d_a phi_j = 0; the integral of d_a phi_i over
// its patch vanishes), so in FP32 each product is formed as sum_j F_ij (x_j - x_i): the same
// value in exact arithmetic, but a smooth or nearly uniform x (m, sigma0, U, u) no longer
// cancels in the sum, and the rounding of F and G to FP32 does not turn a uniform x into a
// spurious result (kDiff).
//
// b_i = sum_j F_{ij,a} m_{j,a}  (Eq. RHS_b divided by m_s); pin_zero: the segment's pinned
// entry is 0 (right-hand side of the pinned system)
template <typename T>
__global__ void __launch_bounds__(kBlock) k_fdiv(DSell A, DSeg G, const T* __restrict__ Fv,
                                                 const T* __restrict__ m, int64_t ld,
                                                 T* __restrict__ b, int pin_zero) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = gstride() >> 5;
  for (int64_t s = gtid() >> 5; s < A.nslices; s += nw) {
    const int64_t base = A.sptr[s];
    const int len = A.slen[s];
    const int32_t* cp = A.col + base + lane;
    const T* vp = Fv + base * 3 + lane;
    const int64_t row = s * 32 + lane;
    const bool in = row < A.n;
    const bool own = in && kDiff<T>;
    const T m0 = own ? m[row] : T(0), m1 = own ? m[ld + row] : T(0),
            m2 = own ? m[2 * ld + row] : T(0);
    T acc = T(0);
    for (int kb = 0; kb < len; kb += kRowRound) {
      int j[kRowRound];
      T f[kRowRound][3];
      row_round(cp, vp, kb, len, j, f);
#pragma unroll
      for (int u = 0; u < kRowRound; ++u)
        acc += f[u][0] * (__ldg(m + j[u]) - m0) + f[u][1] * (__ldg(m + ld + j[u]) - m1) +
               f[u][2] * (__ldg(m + 2 * ld + j[u]) - m2);
    }
    if (in) b[row] = pin_zero && row == G.seg_pin[G.seg_of_slice[s]] ? T(0) : acc;
  }
}

// h~_d,a = (F_a U)_i / M_L,i  (= -grad U, Sec. 2.3 with the lumped-mass normalisation)
template <typename T>
__global__ void __launch_bounds__(kBlock) k_fgrad(DSell A, const T* __restrict__ Fv,
                                                  const T* __restrict__ U,
                                                  const T* __restrict__ Ulo,
                                                  const double* __restrict__ invML,
                                                  T* __restrict__ hd, int64_t ld) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = gstride() >> 5;
  for (int64_t s = gtid() >> 5; s < A.nslices; s += nw) {
    const int64_t base = A.sptr[s];
    const int len = A.slen[s];
    const int32_t* cp = A.col + base + lane;
    const T* vp = Fv + base * 3 + lane;
    const int64_t row = s * 32 + lane;
    const T ui = kDiff<T> && row < A.n ? U[row] : T(0);
    const T uil = Ulo && row < A.n ? Ulo[row] : T(0);
    T a0 = T(0), a1 = T(0), a2 = T(0);
    for (int kb = 0; kb < len; kb += kRowRound) {
      int j[kRowRound];
      T f[kRowRound][3];
      row_round(cp, vp, kb, len, j, f);
#pragma unroll
      for (int u = 0; u < kRowRound; ++u) {
        const T du = ((T)__ldg(U + j[u]) - ui) + (Ulo ? __ldg(Ulo + j[u]) - uil : T(0));
        a0 += f[u][0] * du;
        a1 += f[u][1] * du;
        a2 += f[u][2] * du;
      }
    }
    if (row < A.n) {
      const T im = (T)invML[row];
      hd[row] = a0 * im;
      hd[ld + row] = a1 * im;
      hd[2 * ld + row] = a2 * im;
    }
  }
}

// E = E_bar(segment) + sym grad u with grad_a u_b = -(F_a u_b)_i / M_L,i; E stored SoA Voigt
// (11, 22, 33, 23, 13, 12) with tensor shear components
template <typename T>
__global__ void __launch_bounds__(kBlock) k_fstrain(DSell A, DSeg G, const T* __restrict__ Fv,
                                                    const T* __restrict__ u,
                                                    const T* __restrict__ ulo,
                                                    const double* __restrict__ invML,
                                                    const double* __restrict__ Ebar,
                                                    T* __restrict__ E, int64_t ld) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = gstride() >> 5;
  for (int64_t s = gtid() >> 5; s < A.nslices; s += nw) {
    const int64_t base = A.sptr[s];
    const int len = A.slen[s];
    const int32_t* cp = A.col + base + lane;
    const T* vp = Fv + base * 3 + lane;
    const int64_t row = s * 32 + lane;
    const bool in = row < A.n;
    const bool own = in && kDiff<T>;
    const T ui[3] = {own ? u[3 * row] : T(0), own ? u[3 * row + 1] : T(0),
                     own ? u[3 * row + 2] : T(0)};
    const bool lo = ulo && in;
    const T uil[3] = {lo ? ulo[3 * row] : T(0), lo ? ulo[3 * row + 1] : T(0),
                      lo ? ulo[3 * row + 2] : T(0)};
    T g[3][3] = {};
    for (int kb = 0; kb < len; kb += kRowRound) {
      int j[kRowRound];
      T f[kRowRound][3];
      row_round(cp, vp, kb, len, j, f);
#pragma unroll
      for (int q = 0; q < kRowRound; ++q) {
        const T* uq = u + 3 * (int64_t)j[q];
        T uj[3] = {uq[0] - ui[0], uq[1] - ui[1], uq[2] - ui[2]};
        if (ulo) {
          const T* lq = ulo + 3 * (int64_t)j[q];
#pragma unroll
          for (int b = 0; b < 3; ++b) uj[b] += lq[b] - uil[b];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) g[a][b] += f[q][a] * uj[b];
      }
    }
    if (in) {
      const double* eb = Ebar + 6 * G.seg_of_slice[s];
      const T im = -(T)invML[row];  // g[a][b] * im = d_a u_b
      E[row] = (T)eb[0] + g[0][0] * im;
      E[ld + row] = (T)eb[1] + g[1][1] * im;
      E[2 * ld + row] = (T)eb[2] + g[2][2] * im;
      E[3 * ld + row] = (T)eb[3] + T(0.5) * (g[1][2] + g[2][1]) * im;
      E[4 * ld + row] = (T)eb[4] + T(0.5) * (g[0][2] + g[2][0]) * im;
      E[5 * ld + row] = (T)eb[5] + T(0.5) * (g[0][1] + g[1][0]) * im;
    }
  }
}

// b^mech_(i,a) = sum_j sum_c G_{ij,c} sigma0_{j,ac}, sigma0 = C E0 (nodal, [n][6] Voigt)
// (= F^mech E0 of Eq. RHS_b for a uniform C); pin_zero: the segment's pinned node's entries are 0
template <typename T>
__global__ void __launch_bounds__(kBlock) k_gdiv(DSell A, DSeg G, const T* __restrict__ Gv,
                                                 const T* __restrict__ sig0,
                                                 T* __restrict__ b, int pin_zero) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = gstride() >> 5;
  for (int64_t s = gtid() >> 5; s < A.nslices; s += nw) {
    const int64_t base = A.sptr[s];
    const int len = A.slen[s];
    const int32_t* cp = A.col + base + lane;
    const T* vp = Gv + base * 3 + lane;
    const int64_t row = s * 32 + lane;
    const bool in = row < A.n;
    T si[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) si[c] = in && kDiff<T> ? sig0[6 * row + c] : T(0);
    T b0 = T(0), b1 = T(0), b2 = T(0);
    for (int kb = 0; kb < len; kb += kRowRound) {
      int j[kRowRound];
      T gv[kRowRound][3];
      row_round(cp, vp, kb, len, j, gv);
#pragma unroll
      for (int q = 0; q < kRowRound; ++q) {
        const T* sj = sig0 + 6 * (int64_t)j[q];
        const T g0 = gv[q][0], g1 = gv[q][1], g2 = gv[q][2];
        const T s11 = __ldg(sj) - si[0], s22 = __ldg(sj + 1) - si[1],
                s33 = __ldg(sj + 2) - si[2], s23 = __ldg(sj + 3) - si[3],
                s13 = __ldg(sj + 4) - si[4], s12 = __ldg(sj + 5) - si[5];
        b0 += g0 * s11 + g1 * s12 + g2 * s13;
        b1 += g0 * s12 + g1 * s22 + g2 * s23;
        b2 += g0 * s13 + g1 * s23 + g2 * s33;
      }
    }
    if (in) {
      const bool pz = pin_zero && row == G.seg_pin[G.seg_of_slice[s]];
      b[3 * row] = pz ? T(0) : b0;
      b[3 * row + 1] = pz ? T(0) : b1;
      b[3 * row + 2] = pz ? T(0) : b2;
    }
  }
}

// ------------------------------------------------------------------------------------------
// pointwise material laws
// ------------------------------------------------------------------------------------------
// Table A.1: E0 = 3/2 [lambda100 (m_i^2 - 1/3); lambda111 m_i m_j], Voigt 11,22,33,23,13,12
template <typename T>
__device__ __forceinline__ void e0_of(T m0, T m1, T m2, const DevParams& P, T (&e)[6]) {
  const T a = T(1.5) * (T)P.l100, b = T(1.5) * (T)P.l111, third = T(1.0 / 3.0);
  e[0] = a * (m0 * m0 - third);
  e[1] = a * (m1 * m1 - third);
  e[2] = a * (m2 * m2 - third);
  e[3] = b * m1 * m2;
  e[4] = b * m0 * m2;
  e[5] = b * m0 * m1;
}

// sigma = C E for the cubic stiffness (tensor shear: sigma_ij = 2 C44 E_ij)
template <typename T>
__device__ __forceinline__ void stress_of(const T (&e)[6], const DevParams& P, T (&s)[6]) {
  const T C11 = (T)P.C11, C12 = (T)P.C12, C44 = (T)P.C44;
  s[0] = C11 * e[0] + C12 * (e[1] + e[2]);
  s[1] = C11 * e[1] + C12 * (e[0] + e[2]);
  s[2] = C11 * e[2] + C12 * (e[0] + e[1]);
  s[3] = T(2) * C44 * e[3];
  s[4] = T(2) * C44 * e[4];
  s[5] = T(2) * C44 * e[5];
}

// App. D rotations: v_mesh = R v_crystal; symmetric tensors in Voigt order (tensor shear)
// A_mesh = R A_crystal R^T.  to_mesh = 0 applies the inverse (R^T v, R^T A R).
template <typename T>
__device__ __forceinline__ void rot_vec(const DevParams& P, bool to_mesh, const T (&v)[3],
                                        T (&o)[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T acc = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) acc += (T)(to_mesh ? P.R[3 * i + k] : P.R[3 * k + i]) * v[k];
    o[i] = acc;
  }
}

template <typename T>
__device__ __forceinline__ void rot_sym(const DevParams& P, bool to_mesh, const T (&v)[6],
                                        T (&o)[6]) {
  const T A[3][3] = {{v[0], v[5], v[4]}, {v[5], v[1], v[3]}, {v[4], v[3], v[2]}};
  T Q[3][3], B[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) Q[i][k] = (T)(to_mesh ? P.R[3 * i + k] : P.R[3 * k + i]);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      T acc = T(0);
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) acc += Q[i][a] * A[a][b] * Q[j][b];
      B[i][j] = acc;
    }
  o[0] = B[0][0];
  o[1] = B[1][1];
  o[2] = B[2][2];
  o[3] = B[1][2];
  o[4] = B[0][2];
  o[5] = B[0][1];
}

// E0(m) and sigma0 = C E0 in the mesh axes; rotated crystal (Algorithm D.1 step 1): both
// evaluated in the crystal axes at R^T m and rotated to the mesh axes
template <typename T>
__global__ void __launch_bounds__(kBlock) k_e0(int64_t n, const T* __restrict__ m, int64_t ld,
                                               const uint8_t* __restrict__ mag, DevParams P,
                                               T* __restrict__ E0, T* __restrict__ sig0) {
  for (int64_t i = gtid(); i < n; i += gstride()) {
    T e[6] = {}, s[6] = {};
    if (mag[i]) {
      if (P.rotated) {
        const T mm[3] = {m[i], m[ld + i], m[2 * ld + i]};
        T mc[3], ec[6], sc[6];
        rot_vec<T>(P, false, mm, mc);
        e0_of<T>(mc[0], mc[1], mc[2], P, ec);
        stress_of<T>(ec, P, sc);
        rot_sym<T>(P, true, ec, e);
        rot_sym<T>(P, true, sc, s);
      } else {
        e0_of<T>(m[i], m[ld + i], m[2 * ld + i], P, e);
        stress_of<T>(e, P, s);
      }
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      E0[c * ld + i] = e[c];
      sig0[6 * i + c] = s[c];
    }
  }
}

// h = -kappa m_a (|m|^2 - m_a^2) + H/m_s + (3/(mu0 ms^2)) [l100 m_a s_aa + l111 (m_b s_ab +
// m_c s_ac)] + h~_d - N_d m_bar, with s = C (E - E0(m)), H and m_bar of the node's segment;
// zero off Omega_m
template <typename T>
__global__ void __launch_bounds__(kBlock) k_hfield(int64_t n, DSeg G, const T* __restrict__ m,
                                                   const T* __restrict__ hd,
                                                   const T* __restrict__ E, int64_t ld,
                                                   const double* __restrict__ mbar,
                                                   const double* __restrict__ hz,
                                                   const uint8_t* __restrict__ mag, DevParams P,
                                                   int mode, double coef, T* __restrict__ h,
                                                   T* __restrict__ x) {
  const T kap = (T)P.kappa, mec = (T)P.me_coef, l100 = (T)P.l100, l111 = (T)P.l111;
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const T mv[3] = {m[i], m[ld + i], m[2 * ld + i]};
    T hv[3] = {T(0), T(0), T(0)};
    if (mag[i]) {
      const int seg = G.seg_of_slice[i >> 5];
      const double* mb = mbar + 3 * seg;
      const double* hs = hz + 3 * seg;
      // crystal terms (anisotropy, magnetoelastic) in the crystal axes: m_c = R^T m and
      // E_c = R^T E R when rotated (Algorithm D.1 step 4), rotated back with R at the end
      T mc[3], Ec[6];
      if (P.rotated) {
        const T Em[6] = {E[i], E[ld + i], E[2 * ld + i], E[3 * ld + i], E[4 * ld + i],
                         E[5 * ld + i]};
        rot_vec<T>(P, false, mv, mc);
        rot_sym<T>(P, false, Em, Ec);
      } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) mc[a] = mv[a];
#pragma unroll
        for (int c = 0; c < 6; ++c) Ec[c] = E[c * ld + i];
      }
      T e0[6], d[6], s[6];
      e0_of<T>(mc[0], mc[1], mc[2], P, e0);
#pragma unroll
      for (int c = 0; c < 6; ++c) d[c] = Ec[c] - e0[c];
      stress_of<T>(d, P, s);
      // full symmetric stress lookup: (0,0)->0 (1,1)->1 (2,2)->2 (1,2)->3 (0,2)->4 (0,1)->5
      const T S[3][3] = {{s[0], s[5], s[4]}, {s[5], s[1], s[3]}, {s[4], s[3], s[2]}};
      const T m2sum = mc[0] * mc[0] + mc[1] * mc[1] + mc[2] * mc[2];
      T hc[3], hm[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int b = (a + 1) % 3, c = (a + 2) % 3;
        const T an = -kap * mc[a] * (m2sum - mc[a] * mc[a]);
        const T me = mec * (l100 * mc[a] * S[a][a] + l111 * (mc[b] * S[a][b] + mc[c] * S[a][c]));
        hc[a] = an + me;
      }
      if (P.rotated) {
        rot_vec<T>(P, true, hc, hm);
      } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) hm[a] = hc[a];
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const T far = (T)(hs[a] - (P.Nd[3 * a] * mb[0] + P.Nd[3 * a + 1] * mb[1] +
                                   P.Nd[3 * a + 2] * mb[2]));
        hv[a] = hm[a] + far + hd[a * ld + i];
      }
    }
    if (mode == 0) {
#pragma unroll
      for (int a = 0; a < 3; ++a) h[a * ld + i] = hv[a];
    } else {
#pragma unroll
      for (int a = 0; a < 3; ++a) x[a * ld + i] = (T)((double)mv[a] + coef * (double)hv[a]);
    }
  }
}

// x_k = m_{c0+k} + dtau h_{c0+k}, k < nc  (GSPM right-hand-side fields f, Algorithm B.1)
template <typename T>
__global__ void __launch_bounds__(kBlock) k_gs_prep(int64_t n, int64_t ld, const T* __restrict__ m,
                                                    const T* __restrict__ h, double dtau, int c0,
                                                    int nc, T* __restrict__ x) {
  for (int64_t i = gtid(); i < n; i += gstride())
    for (int k = 0; k < nc; ++k) {
      const int c = c0 + k;
      x[k * ld + i] = (T)((double)m[c * ld + i] + dtau * (double)h[c * ld + i]);
    }
}

// Gauss-Seidel stages of Algorithm B.1 step 2 (slot layout of x in the driver):
//  Gauss-Seidel sweep (printed = 0):
//   stage 1: x0 = g2, x1 = g3        -> m*1 = m1 + g2 m3 - g3 m2;         x2 = m*1 + dtau h1
//   stage 2: x2 = g*1                -> m*2 = m2 + g3 m*1 - g*1 m3;       x0 = m*2 + dtau h2
//   stage 3: x0 = g*2                -> m*3 = m3 + g*1 m*2 - g*2 m*1
//  literal print (printed = 1):
//   stage 1: x0..2 = g1, g2, g3      -> m*1 = m1 + g2 m3 - g3 m2, m*2 = m2 + g3 m1 - g1 m3;
//                                       x0 = m*1 + dtau h1, x1 = m*2 + dtau h2
//   stage 3: x0 = g*1, x1 = g*2      -> m*3 = m3 + g*1 m*2 - g*2 m*1
template <typename T>
__global__ void __launch_bounds__(kBlock) k_gs_stage(int64_t n, int64_t ld, int stage, int printed,
                                                     const T* __restrict__ m,
                                                     const T* __restrict__ h, double dtau,
                                                     T* __restrict__ x, T* __restrict__ ms) {
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const double m1 = m[i], m2 = m[ld + i], m3 = m[2 * ld + i];
    if (!printed) {
      if (stage == 1) {
        const double s1 = m1 + ((double)x[i] * m3 - (double)x[ld + i] * m2);
        ms[i] = (T)s1;
        x[2 * ld + i] = (T)((double)(T)s1 + dtau * (double)h[i]);
      } else if (stage == 2) {
        const double s1 = ms[i];
        const double s2 = m2 + ((double)x[ld + i] * s1 - (double)x[2 * ld + i] * m3);
        ms[ld + i] = (T)s2;
        x[i] = (T)((double)(T)s2 + dtau * (double)h[ld + i]);
      } else {
        const double s1 = ms[i], s2 = ms[ld + i];
        ms[2 * ld + i] = (T)(m3 + ((double)x[2 * ld + i] * s2 - (double)x[i] * s1));
      }
    } else {
      if (stage == 1) {
        const double g1 = x[i], g2 = x[ld + i], g3 = x[2 * ld + i];
        const double s1 = m1 + (g2 * m3 - g3 * m2);
        const double s2 = m2 + (g3 * m1 - g1 * m3);
        ms[i] = (T)s1;
        ms[ld + i] = (T)s2;
        x[i] = (T)((double)(T)s1 + dtau * (double)h[i]);
        x[ld + i] = (T)((double)(T)s2 + dtau * (double)h[ld + i]);
      } else {
        const double s1 = ms[i], s2 = ms[ld + i];
        ms[2 * ld + i] = (T)(m3 + ((double)x[i] * s2 - (double)x[ld + i] * s1));
      }
    }
  }
}

// Algorithm B.1 step 4: m = m** / |m**| on Omega_m; <|m_new - m_old|> over each segment's
// magnetic nodes
template <typename T>
// (bad[seg] counts the segment's magnetic nodes whose m** is not finite or is zero: the step's
// state is then not valid)
__global__ void __launch_bounds__(kBlock) k_project(DSeg G, ItemList IL, int64_t ld, const T* __restrict__ x,
                                                    const uint8_t* __restrict__ mag,
                                                    T* __restrict__ m, double* dm_out,
                                                    const double* __restrict__ inv_nmag,
                                                    Red red, int* bad) {
  for (int item = blockIdx.x; item < IL.nitems; item += gridDim.x) {
    const int seg = IL.seg[item];
    double v[1] = {0.0};
    const int64_t r0 = (int64_t)IL.sl0[item] * 32, r1 = (int64_t)IL.sl1[item] * 32;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      if (!row_valid(G, seg, i) || !mag[i]) continue;
      const T a = x[i], b = x[ld + i], c = x[2 * ld + i];
      const T n2 = a * a + b * b + c * c;
      if (!(n2 > T(0)) || !isfinite(n2)) atomicAdd(bad + seg, 1);
      const T inv = T(1) / sqrt(n2);
      const T na = a * inv, nb = b * inv, nc = c * inv;
      const T da = na - m[i], db = nb - m[ld + i], dc = nc - m[2 * ld + i];
      v[0] += (double)sqrt(da * da + db * db + dc * dc);
      m[i] = na;
      m[ld + i] = nb;
      m[2 * ld + i] = nc;
    }
    __shared__ double res[1];
    if (seg_reduce<1>(v, item, seg, G, IL, red, res) && threadIdx.x == 0)
      dm_out[seg] = res[0] * inv_nmag[seg];
  }
}

// ------------------------------------------------------------------------------------------
// layout changes between the ABI ([n][nc] float64, unique-node order) and internal arrays;
// perm[i] < 0 marks a padding row (no node)
// ------------------------------------------------------------------------------------------
// lo != NULL: the field is kept as an unevaluated sum dst + lo (the refined solutions of the
// mixed path): dst = v rounded to T, lo = the rest
template <typename T>
__global__ void k_import(int64_t n, int nc, const double* __restrict__ src,
                         const int64_t* __restrict__ perm, T* __restrict__ dst, int64_t cs,
                         int64_t ns, const uint8_t* __restrict__ mask, T* __restrict__ lo) {
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const int64_t o = perm[i];
    const bool z = o < 0 || (mask && !mask[i]);
    for (int c = 0; c < nc; ++c) {
      const double v = z ? 0.0 : src[o * nc + c];
      const T h = (T)v;
      dst[i * ns + c * cs] = h;
      if (lo) lo[i * ns + c * cs] = (T)(v - (double)h);
    }
  }
}

template <typename T>
__global__ void k_export(int64_t n, int nc, const T* __restrict__ src, int64_t cs, int64_t ns,
                         const int64_t* __restrict__ perm, double* __restrict__ dst,
                         const T* __restrict__ lo) {
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const int64_t o = perm[i];
    if (o < 0) continue;
    for (int c = 0; c < nc; ++c)
      dst[o * nc + c] = (double)src[i * ns + c * cs] + (lo ? (double)lo[i * ns + c * cs] : 0.0);
  }
}

template <typename S, typename D>
__global__ void k_convert(int64_t len, const S* __restrict__ s, D* __restrict__ d) {
  for (int64_t i = gtid(); i < len; i += gstride()) d[i] = (D)s[i];
}

// linear extrapolation of the previous two solutions: u <- 2 u - u2, u2 <- old u
template <typename T>
__global__ void k_extrapolate(int64_t len, T* __restrict__ u, T* __restrict__ u2) {
  for (int64_t i = gtid(); i < len; i += gstride()) {
    const T a = u[i], b = u2[i];
    u2[i] = a;
    u[i] = T(2) * a - b;
  }
}

// t = (a - (2 b - c)) * scale
template <typename T>
__global__ void k_scaled_diff(int64_t len, const T* __restrict__ a, const T* __restrict__ b,
                              const T* __restrict__ c, double scale, float* __restrict__ t) {
  for (int64_t i = gtid(); i < len; i += gstride())
    t[i] = (float)(((double)a[i] - (2.0 * (double)b[i] - (double)c[i])) * scale);
}

}  // namespace

// ------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------
int resident_per_sm(const void* kernel) {
  static std::mutex mu;
  static std::unordered_map<const void*, int> occ;
  std::lock_guard<std::mutex> lock(mu);
  auto it = occ.find(kernel);
  if (it == occ.end()) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, kBlock, 0) != cudaSuccess ||
        nb < 1)
      nb = 1;
    it = occ.emplace(kernel, nb).first;
  }
  return it->second;
}

int grid_for(const Launch& L, int64_t threads, const void* kernel) {
  const int per_sm = resident_per_sm(kernel);
  int64_t b = (threads + kBlock - 1) / kBlock;
  const int64_t cap = std::min<int64_t>((int64_t)per_sm * L.sms, L.max_blocks);
  if (b > cap) b = cap;
  return b < 1 ? 1 : (int)b;
}

// Grid and item list of a reducing kernel: the list made for the kernel's residency, one block
// per item (capped at the resident capacity and the launch limit).
struct ItemGrid {
  int grid;
  ItemList list;
};
static ItemGrid item_grid(const Launch& L, const DSeg& G, const void* kernel) {
  const int per_sm = resident_per_sm(kernel);
  const ItemList& il = G.list[(per_sm < kItemLists ? per_sm : kItemLists) - 1];
  return ItemGrid{grid_for(L, (int64_t)il.nitems * kBlock, kernel), il};
}

#define ST_CUDA(...)                      \
  do {                                    \
    const cudaError_t e_ = (__VA_ARGS__); \
    if (e_ != cudaSuccess) return e_;     \
  } while (0)

// Launch of a CG loop kernel with programmatic stream serialisation (see pdl_enter)
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*k)(KArgs...), int grid, cudaStream_t stream, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kBlock);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

#define GSPM_GRID(L, threads, kern) grid_for((L), (threads), reinterpret_cast<const void*>(kern))
#define GSPM_IGRID(L, G, kern) item_grid((L), (G), reinterpret_cast<const void*>(kern))

template <typename T>
cudaError_t launch_wsum(const Launch& L, const DSeg& G, int nc, const T* f, int64_t cs,
                        int64_t ns, const int64_t* perm, const double* w, double* out,
                        const double* add, Red red) {
  (*L.counter) += 1;
  auto k = k_wsum<T>;
  const ItemGrid ig = GSPM_IGRID(L, G, k);
  k<<<ig.grid, kBlock, 0, L.stream>>>(G, ig.list, nc, f, cs, ns, perm, w, out, add, red);
  return cudaGetLastError();
}

template <typename T, int VAR>
static void spmv_variant(const Launch& L, const DSell& A, const T* val, int B, const T* x, T* y,
                         int diff) {
  const int64_t threads = (VAR == 2 ? 64 : 32) * A.nslices;
  if (B == 1) {
    auto k = k_spmv1<T, VAR>;
    k<<<GSPM_GRID(L, threads, k), kBlock, 0, L.stream>>>(A, val, x, y, diff);
  } else {
    auto k = k_spmv9<T, VAR>;
    k<<<GSPM_GRID(L, threads, k), kBlock, 0, L.stream>>>(A, val, x, y, diff);
  }
}

template <typename T>
cudaError_t launch_spmv(const Launch& L, const DSell& A, const T* val, int B, const T* x, T* y,
                        int variant, int diff) {
  (*L.counter) += 1;
  diff = diff && kDiff<T>;
  switch (variant) {
    case 1: spmv_variant<T, 1>(L, A, val, B, x, y, diff); break;
    case 2: spmv_variant<T, 2>(L, A, val, B, x, y, diff); break;
    case 3: spmv_variant<T, 3>(L, A, val, B, x, y, diff); break;
    default: spmv_variant<T, 0>(L, A, val, B, x, y, diff); break;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_init(const Launch& L, const DSell& A, const DSeg& G, const T* val, int B,
                           const T* b, const T* x, T* r, T* p, CGState* st, int* nactive, double rtol,
                           int max_iter, Red red, const double* bmean, int pinned, int pc) {
  (*L.counter) += 1;
  if (B == 1) {
    auto k = k_cg_init<T, 1>;
    const ItemGrid ig = GSPM_IGRID(L, G, k);
    k<<<ig.grid, kBlock, 0, L.stream>>>(A, G, ig.list, val, b, x, r, p, st, nactive, rtol,
                                        max_iter, red, bmean, pinned, pc);
  } else {
    auto k = k_cg_init<T, 9>;
    const ItemGrid ig = GSPM_IGRID(L, G, k);
    k<<<ig.grid, kBlock, 0, L.stream>>>(A, G, ig.list, val, b, x, r, p, st, nactive, rtol,
                                        max_iter, red, bmean, pinned, pc);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_true_res(const Launch& L, const DSell& A, const DSeg& G, const T* val, int B,
                            const T* b, const T* x, const T* xlo, Red red, double* out) {
  (*L.counter) += 1;
  if (B == 1) {
    auto k = k_true_res<T, 1>;
    const ItemGrid ig = GSPM_IGRID(L, G, k);
    k<<<ig.grid, kBlock, 0, L.stream>>>(A, G, ig.list, val, b, x, xlo, red, out);
  } else {
    auto k = k_true_res<T, 9>;
    const ItemGrid ig = GSPM_IGRID(L, G, k);
    k<<<ig.grid, kBlock, 0, L.stream>>>(A, G, ig.list, val, b, x, xlo, red, out);
  }
  return cudaGetLastError();
}

// (hi, lo) <- hi + dx as an unevaluated sum: Knuth's TwoSum of hi and dx, so that hi + lo keeps
// the correction below the last bit of hi (lo is zero on entry)
template <typename T>
__global__ void k_refine_add(int64_t len, T* __restrict__ hi, T* __restrict__ lo,
                             const T* __restrict__ dx) {
  for (int64_t i = gtid(); i < len; i += gstride()) {
    const T a = hi[i], b = dx[i];
    T s, e;
    if constexpr (std::is_same<T, float>::value) {
      s = __fadd_rn(a, b);
      const T bp = __fsub_rn(s, a), ap = __fsub_rn(s, bp);
      e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
    } else {
      s = __dadd_rn(a, b);
      const T bp = __dsub_rn(s, a), ap = __dsub_rn(s, bp);
      e = __dadd_rn(__dsub_rn(a, ap), __dsub_rn(b, bp));
    }
    hi[i] = s;
    lo[i] = e;
  }
}

template <typename T>
cudaError_t launch_refine_add(const Launch& L, int64_t len, T* hi, T* lo, const T* dx) {
  (*L.counter) += 1;
  auto k = k_refine_add<T>;
  k<<<GSPM_GRID(L, len, k), kBlock, 0, L.stream>>>(len, hi, lo, dx);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_init_gs(const Launch& L, const DSell& A, const DSeg& G, const T* aval,
                              const T* mval, int nr, int64_t ld, T* x, T* r, T* p, CGState* st,
                              int* nactive, double rtol, int max_iter, Red red, const T* dinv) {
  (*L.counter) += 1;
  switch (nr) {
    case 1: {
      auto k = k_cg_init_gs<T, 1>;
      const ItemGrid ig = GSPM_IGRID(L, G, k);
      k<<<ig.grid, kBlock, 0, L.stream>>>(A, G, ig.list, aval, mval, ld, x, r, p, st, nactive,
                                                      rtol, max_iter, red, dinv);
      break;
    }
    case 2: {
      auto k = k_cg_init_gs<T, 2>;
      const ItemGrid ig = GSPM_IGRID(L, G, k);
      k<<<ig.grid, kBlock, 0, L.stream>>>(A, G, ig.list, aval, mval, ld, x, r, p, st, nactive,
                                                      rtol, max_iter, red, dinv);
      break;
    }
    case 3: {
      auto k = k_cg_init_gs<T, 3>;
      const ItemGrid ig = GSPM_IGRID(L, G, k);
      k<<<ig.grid, kBlock, 0, L.stream>>>(A, G, ig.list, aval, mval, ld, x, r, p, st, nactive,
                                                      rtol, max_iter, red, dinv);
      break;
    }
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T, int VAR>
static cudaError_t cg_spmv_variant(const Launch& L, const DSell& A, const DSeg& G, const T* val,
                                   int B, int nr, int64_t ld, const T* p, T* q, CGState* st,
                                   Red red, int pinned, int diff) {
  if (B == 9) {
    auto k = k_cg_spmv<T, 9, 1, VAR, kDiff<T>>;
    const ItemGrid ig = GSPM_IGRID(L, G, k);
    return launch_pdl(k, ig.grid, L.stream, A, G, ig.list, val, ld, p, q, st, red, pinned);
  } else if (nr == 1 && diff && kDiff<T>) {
    auto k = k_cg_spmv<T, 1, 1, VAR, 1>;
    const ItemGrid ig = GSPM_IGRID(L, G, k);
    return launch_pdl(k, ig.grid, L.stream, A, G, ig.list, val, ld, p, q, st, red, pinned);
  } else if (nr == 1) {
    auto k = k_cg_spmv<T, 1, 1, VAR, 0>;
    const ItemGrid ig = GSPM_IGRID(L, G, k);
    return launch_pdl(k, ig.grid, L.stream, A, G, ig.list, val, ld, p, q, st, red, pinned);
  } else if (nr == 2) {
    auto k = k_cg_spmv<T, 1, 2, VAR, 0>;
    const ItemGrid ig = GSPM_IGRID(L, G, k);
    return launch_pdl(k, ig.grid, L.stream, A, G, ig.list, val, ld, p, q, st, red, pinned);
  } else if (nr == 3) {
    auto k = k_cg_spmv<T, 1, 3, VAR, 0>;
    const ItemGrid ig = GSPM_IGRID(L, G, k);
    return launch_pdl(k, ig.grid, L.stream, A, G, ig.list, val, ld, p, q, st, red, pinned);
  } else {
    return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_cg_spmv(const Launch& L, const DSell& A, const DSeg& G, const T* val, int B,
                           int nr, int64_t ld, const T* p, T* q, CGState* st, Red red,
                           int variant, int pinned, int diff) {
  (*L.counter) += 1;
  switch (variant) {
    case 1: return cg_spmv_variant<T, 1>(L, A, G, val, B, nr, ld, p, q, st, red, pinned, diff);
    case 2: return cg_spmv_variant<T, 2>(L, A, G, val, B, nr, ld, p, q, st, red, pinned, diff);
    case 3: return cg_spmv_variant<T, 3>(L, A, G, val, B, nr, ld, p, q, st, red, pinned, diff);
    default: return cg_spmv_variant<T, 0>(L, A, G, val, B, nr, ld, p, q, st, red, pinned, diff);
  }
}

static bool aligned16(const void* ptr) { return ((uintptr_t)ptr & 15u) == 0; }

template <typename T, int NR, bool VEC>
static cudaError_t cg_update_nr(const Launch& L, const DSeg& G, int epr, int64_t ld, T* x, T* r,
                         const T* p, const T* q, CGState* st, int* nactive, Red red,
                         const T* dinv) {
  auto k = k_cg_update<T, NR, VEC>;
  const ItemGrid ig = GSPM_IGRID(L, G, k);
  return launch_pdl(k, ig.grid, L.stream, G, ig.list, epr, ld, x, r, p, q, st, nactive, red, dinv);
}

template <typename T, bool VEC>
static cudaError_t cg_update_vec(const Launch& L, const DSeg& G, int epr, int nr, int64_t ld,
                                 T* x, T* r, const T* p, const T* q, CGState* st, int* nactive,
                                 Red red, const T* dinv) {
  switch (nr) {
    case 1: ST_CUDA(cg_update_nr<T, 1, VEC>(L, G, epr, ld, x, r, p, q, st, nactive, red, dinv)); break;
    case 2: ST_CUDA(cg_update_nr<T, 2, VEC>(L, G, epr, ld, x, r, p, q, st, nactive, red, dinv)); break;
    case 3: ST_CUDA(cg_update_nr<T, 3, VEC>(L, G, epr, ld, x, r, p, q, st, nactive, red, dinv)); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_update(const Launch& L, const DSeg& G, int epr, int nr, int64_t ld, T* x,
                             T* r, const T* p, const T* q, CGState* st, int* nactive, Red red,
                             const T* dinv) {
  (*L.counter) += 1;
  if (dinv && epr != 1) return cudaErrorInvalidValue;
  const bool vec = aligned16(x) && aligned16(r) && aligned16(p) && aligned16(q) &&
                   (!dinv || aligned16(dinv)) && (nr == 1 || ld % Pack16<T>::W == 0);
  return vec ? cg_update_vec<T, true>(L, G, epr, nr, ld, x, r, p, q, st, nactive, red, dinv)
             : cg_update_vec<T, false>(L, G, epr, nr, ld, x, r, p, q, st, nactive, red, dinv);
}

template <typename T, int NR, bool VEC>
static cudaError_t cg_pupdate_nr(const Launch& L, const DSeg& G, int epr, int64_t ld, const T* r, T* p,
                          const CGState* st, const LoopCtl& lc, const T* dinv) {
  auto k = k_cg_pupdate<T, NR, VEC>;
  const ItemGrid ig = GSPM_IGRID(L, G, k);
  return launch_pdl(k, ig.grid, L.stream, G, ig.list, epr, ld, r, p, st, lc, dinv);
}

template <typename T, bool VEC>
static cudaError_t cg_pupdate_vec(const Launch& L, const DSeg& G, int epr, int nr, int64_t ld,
                                  const T* r, T* p, const CGState* st, const LoopCtl& lc,
                                  const T* dinv) {
  switch (nr) {
    case 1: ST_CUDA(cg_pupdate_nr<T, 1, VEC>(L, G, epr, ld, r, p, st, lc, dinv)); break;
    case 2: ST_CUDA(cg_pupdate_nr<T, 2, VEC>(L, G, epr, ld, r, p, st, lc, dinv)); break;
    case 3: ST_CUDA(cg_pupdate_nr<T, 3, VEC>(L, G, epr, ld, r, p, st, lc, dinv)); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_pupdate(const Launch& L, const DSeg& G, int epr, int nr, int64_t ld,
                              const T* r, T* p, const CGState* st, const LoopCtl& lc,
                              const T* dinv) {
  (*L.counter) += 1;
  if (dinv && epr != 1) return cudaErrorInvalidValue;
  const bool vec = aligned16(r) && aligned16(p) && (!dinv || aligned16(dinv)) &&
                   (nr == 1 || ld % Pack16<T>::W == 0);
  return vec ? cg_pupdate_vec<T, true>(L, G, epr, nr, ld, r, p, st, lc, dinv)
             : cg_pupdate_vec<T, false>(L, G, epr, nr, ld, r, p, st, lc, dinv);
}

template <typename T>
cudaError_t launch_restrict(const Launch& L, const DCoarse& C, int epr, const T* r,
                            const int64_t* rc_off, T* rc) {
  (*L.counter) += 1;
  // scalar rows: a warp per contiguous aggregate (6.4 against 13 us per launch at 3M nodes,
  // cold); three components: a block per aggregate (15.9 us against 23 us for a warp)
  if (epr == 1 && C.contig && aligned16(r)) {
    auto k = k_restrict_contig<T, 1>;
    ST_CUDA(launch_pdl(k, GSPM_GRID(L, C.nagg * 32, k), L.stream, C, r, rc_off, rc));
  } else if (epr == 3) {
    auto k = k_restrict<T, 3>;
    ST_CUDA(launch_pdl(k, GSPM_GRID(L, C.nagg * kBlock, k), L.stream, C, r, rc_off, rc));
  } else if (epr == 1) {
    auto k = k_restrict<T, 1>;
    ST_CUDA(launch_pdl(k, GSPM_GRID(L, C.nagg * kBlock, k), L.stream, C, r, rc_off, rc));
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarse_symv(const Launch& L, const DCoarse& C, const DSymTiles& TL, int epr,
                               const typename CoarseStore<T>::type* inv, const int64_t* rc_off,
                               const T* rc, T* Q, T* ec) {
  (*L.counter) += 2;
  if (!aligned16(inv) || !aligned16(rc)) return cudaErrorInvalidValue;
  auto k1 = k_coarse_symv_tiles<T, typename CoarseStore<T>::type>;
  ST_CUDA(launch_pdl(k1, GSPM_GRID(L, TL.ntiles * kBlock, k1), L.stream, TL, inv, rc_off, rc, Q));
  auto k2 = k_coarse_symv_sum<T>;
  ST_CUDA(launch_pdl(k2, GSPM_GRID(L, C.nagg * epr * 32, k2), L.stream, C, TL, epr, Q, ec));
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_pcg_z(const Launch& L, const DSeg& G, const DCoarse& C, int epr, const T* r,
                         const T* dinv, const T* ec, T* z, CGState* st, int init, Red red) {
  (*L.counter) += 1;
  if (epr == 3) {
    auto k = k_pcg_z<T, 3>;
    const ItemGrid ig = GSPM_IGRID(L, G, k);
    ST_CUDA(launch_pdl(k, ig.grid, L.stream, G, ig.list, C, r, dinv, ec, z, st, init, red));
  } else if (epr == 1) {
    auto k = k_pcg_z<T, 1>;
    const ItemGrid ig = GSPM_IGRID(L, G, k);
    ST_CUDA(launch_pdl(k, ig.grid, L.stream, G, ig.list, C, r, dinv, ec, z, st, init, red));
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_loop_start(const Launch& L, const LoopCtl& lc) {
  (*L.counter) += 1;
  k_loop_start<<<1, 32, 0, L.stream>>>(lc);
  return cudaGetLastError();
}

cudaError_t launch_solve_stats(const Launch& L, const CGState* st, int nseg, int kind,
                               long long* acc) {
  (*L.counter) += 1;
  k_solve_stats<<<(nseg + 127) / 128, 128, 0, L.stream>>>(st, nseg, kind, acc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pin_shift(const Launch& L, const DSell& A, const DSeg& G, int epr, T* x,
                             double* xp) {
  (*L.counter) += 2;
  k_pin_gather<T><<<(G.nseg * epr + 127) / 128, 128, 0, L.stream>>>(G, epr, x, xp);
  auto k = k_pin_shift<T>;
  k<<<GSPM_GRID(L, A.nslices * 32 * epr, k), kBlock, 0, L.stream>>>(A, G, epr, x, xp);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_seg_shift(const Launch& L, const DSell& A, const DSeg& G, int epr, T* x,
                             const double* xs) {
  (*L.counter) += 1;
  auto k = k_pin_shift<T>;
  k<<<GSPM_GRID(L, A.nslices * 32 * epr, k), kBlock, 0, L.stream>>>(A, G, epr, x, xs);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_psub(const Launch& L, const DSell& A, const DSeg& G, int epr, T* p,
                           const CGState* st) {
  (*L.counter) += 1;
  auto k = k_cg_psub<T>;
  k<<<GSPM_GRID(L, A.nslices * 32 * epr, k), kBlock, 0, L.stream>>>(A, G, epr, p, st);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_zero(const Launch& L, const DSeg& G, int epr, T* x, const CGState* st) {
  (*L.counter) += 1;
  auto k = k_cg_zero<T>;
  const ItemGrid ig = GSPM_IGRID(L, G, k);
  k<<<ig.grid, kBlock, 0, L.stream>>>(G, ig.list, epr, x, st);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fdiv(const Launch& L, const DSell& A, const DSeg& G, const T* Fv, const T* m,
                        int64_t ld, T* b, int pin_zero) {
  (*L.counter) += 1;
  auto k = k_fdiv<T>;
  k<<<GSPM_GRID(L, A.nslices * 32, k), kBlock, 0, L.stream>>>(A, G, Fv, m, ld, b, pin_zero);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fgrad(const Launch& L, const DSell& A, const T* Fv, const T* U, const T* Ulo,
                         const double* invML, T* hd, int64_t ld) {
  (*L.counter) += 1;
  auto k = k_fgrad<T>;
  k<<<GSPM_GRID(L, A.nslices * 32, k), kBlock, 0, L.stream>>>(A, Fv, U, Ulo, invML, hd, ld);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fstrain(const Launch& L, const DSell& A, const DSeg& G, const T* Fv,
                           const T* u, const T* ulo, const double* invML, const double* Ebar,
                           T* E, int64_t ld) {
  (*L.counter) += 1;
  auto k = k_fstrain<T>;
  k<<<GSPM_GRID(L, A.nslices * 32, k), kBlock, 0, L.stream>>>(A, G, Fv, u, ulo, invML, Ebar, E,
                                                               ld);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gdiv(const Launch& L, const DSell& A, const DSeg& G, const T* Gv,
                        const T* sig0, T* b, int pin_zero) {
  (*L.counter) += 1;
  auto k = k_gdiv<T>;
  k<<<GSPM_GRID(L, A.nslices * 32, k), kBlock, 0, L.stream>>>(A, G, Gv, sig0, b, pin_zero);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_e0(const Launch& L, int64_t n, const T* m, int64_t ld, const uint8_t* mag,
                      const DevParams& P, T* E0, T* sig0) {
  (*L.counter) += 1;
  auto k = k_e0<T>;
  k<<<GSPM_GRID(L, n, k), kBlock, 0, L.stream>>>(n, m, ld, mag, P, E0, sig0);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_hfield(const Launch& L, int64_t n, const DSeg& G, const T* m, const T* hd,
                          const T* E, int64_t ld, const double* mbar, const double* hz,
                          const uint8_t* mag, const DevParams& P, int mode, double coef, T* h,
                          T* x) {
  (*L.counter) += 1;
  auto k = k_hfield<T>;
  k<<<GSPM_GRID(L, n, k), kBlock, 0, L.stream>>>(n, G, m, hd, E, ld, mbar, hz, mag, P, mode,
                                                  coef, h, x);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gs_prep(const Launch& L, int64_t n, int64_t ld, const T* m, const T* h,
                           double dtau, int c0, int nc, T* x) {
  (*L.counter) += 1;
  auto k = k_gs_prep<T>;
  k<<<GSPM_GRID(L, n, k), kBlock, 0, L.stream>>>(n, ld, m, h, dtau, c0, nc, x);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gs_stage(const Launch& L, int64_t n, int64_t ld, int stage, int printed,
                            const T* m, const T* h, double dtau, T* x, T* ms) {
  (*L.counter) += 1;
  auto k = k_gs_stage<T>;
  k<<<GSPM_GRID(L, n, k), kBlock, 0, L.stream>>>(n, ld, stage, printed, m, h, dtau, x, ms);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_project(const Launch& L, const DSeg& G, int64_t ld, const T* x,
                           const uint8_t* mag, T* m, double* dm_out, const double* inv_nmag,
                           Red red, int* bad) {
  (*L.counter) += 1;
  auto k = k_project<T>;
  const ItemGrid ig = GSPM_IGRID(L, G, k);
  k<<<ig.grid, kBlock, 0, L.stream>>>(G, ig.list, ld, x, mag, m, dm_out, inv_nmag, red, bad);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_import(const Launch& L, int64_t n, int nc, const double* src,
                          const int64_t* perm, T* dst, int64_t cs, int64_t ns,
                          const uint8_t* mask, T* lo) {
  (*L.counter) += 1;
  auto k = k_import<T>;
  k<<<GSPM_GRID(L, n, k), kBlock, 0, L.stream>>>(n, nc, src, perm, dst, cs, ns, mask, lo);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_export(const Launch& L, int64_t n, int nc, const T* src, int64_t cs,
                          int64_t ns, const int64_t* perm, double* dst, const T* lo) {
  (*L.counter) += 1;
  auto k = k_export<T>;
  k<<<GSPM_GRID(L, n, k), kBlock, 0, L.stream>>>(n, nc, src, cs, ns, perm, dst, lo);
  return cudaGetLastError();
}

template <typename S, typename D>
cudaError_t launch_convert(const Launch& L, int64_t len, const S* src, D* dst) {
  (*L.counter) += 1;
  auto k = k_convert<S, D>;
  k<<<GSPM_GRID(L, len, k), kBlock, 0, L.stream>>>(len, src, dst);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_extrapolate(const Launch& L, int64_t len, T* u, T* u2) {
  (*L.counter) += 1;
  auto k = k_extrapolate<T>;
  k<<<GSPM_GRID(L, len, k), kBlock, 0, L.stream>>>(len, u, u2);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scaled_diff(const Launch& L, int64_t len, const T* a, const T* b, const T* c,
                               double scale, float* t) {
  (*L.counter) += 1;
  auto k = k_scaled_diff<T>;
  k<<<GSPM_GRID(L, len, k), kBlock, 0, L.stream>>>(len, a, b, c, scale, t);
  return cudaGetLastError();
}

#define GSPM_INSTANTIATE(T)                                                                       \
  template cudaError_t launch_wsum<T>(const Launch&, const DSeg&, int, const T*, int64_t,        \
                                      int64_t, const int64_t*, const double*, double*,            \
                                      const double*, Red);                                        \
  template cudaError_t launch_spmv<T>(const Launch&, const DSell&, const T*, int, const T*, T*,   \
                                      int, int);                                                  \
  template cudaError_t launch_cg_init<T>(const Launch&, const DSell&, const DSeg&, const T*, int, \
                                         const T*, const T*, T*, T*, CGState*, int*, double, int, Red,  \
                                         const double*, int, int);                                \
  template cudaError_t launch_true_res<T>(const Launch&, const DSell&, const DSeg&, const T*, int,  \
                                          const T*, const T*, const T*, Red, double*);            \
  template cudaError_t launch_refine_add<T>(const Launch&, int64_t, T*, T*, const T*);            \
  template cudaError_t launch_restrict<T>(const Launch&, const DCoarse&, int, const T*,           \
                                          const int64_t*, T*);                                    \
  template cudaError_t launch_coarse_symv<T>(const Launch&, const DCoarse&, const DSymTiles&, int, \
                                             const typename CoarseStore<T>::type*, const int64_t*, \
                                             const T*, T*, T*);                                   \
  template cudaError_t launch_pcg_z<T>(const Launch&, const DSeg&, const DCoarse&, int, const T*, \
                                       const T*, const T*, T*, CGState*, int, Red);              \
  template cudaError_t launch_cg_init_gs<T>(const Launch&, const DSell&, const DSeg&, const T*,   \
                                            const T*, int, int64_t, T*, T*, T*, CGState*, int*,   \
                                            double, int, Red, const T*);                          \
  template cudaError_t launch_cg_spmv<T>(const Launch&, const DSell&, const DSeg&, const T*, int, \
                                         int, int64_t, const T*, T*, CGState*, Red, int, int, int); \
  template cudaError_t launch_cg_update<T>(const Launch&, const DSeg&, int, int, int64_t, T*, T*, \
                                           const T*, const T*, CGState*, int*, Red, const T*);    \
  template cudaError_t launch_cg_pupdate<T>(const Launch&, const DSeg&, int, int, int64_t,        \
                                            const T*, T*, const CGState*, const LoopCtl&,         \
                                            const T*);                                            \
  template cudaError_t launch_cg_zero<T>(const Launch&, const DSeg&, int, T*, const CGState*);    \
  template cudaError_t launch_fdiv<T>(const Launch&, const DSell&, const DSeg&, const T*,         \
                                      const T*, int64_t, T*, int);                                \
  template cudaError_t launch_fgrad<T>(const Launch&, const DSell&, const T*, const T*, const T*, \
                                       const double*, T*, int64_t);                               \
  template cudaError_t launch_fstrain<T>(const Launch&, const DSell&, const DSeg&, const T*,      \
                                         const T*, const T*, const double*, const double*, T*,    \
                                         int64_t);                                                \
  template cudaError_t launch_gdiv<T>(const Launch&, const DSell&, const DSeg&, const T*,         \
                                      const T*, T*, int);                                         \
  template cudaError_t launch_pin_shift<T>(const Launch&, const DSell&, const DSeg&, int, T*,     \
                                           double*);                                              \
  template cudaError_t launch_seg_shift<T>(const Launch&, const DSell&, const DSeg&, int, T*,     \
                                           const double*);                                        \
  template cudaError_t launch_cg_psub<T>(const Launch&, const DSell&, const DSeg&, int, T*,       \
                                         const CGState*);                                         \
  template cudaError_t launch_e0<T>(const Launch&, int64_t, const T*, int64_t, const uint8_t*,    \
                                    const DevParams&, T*, T*);                                    \
  template cudaError_t launch_hfield<T>(const Launch&, int64_t, const DSeg&, const T*, const T*,  \
                                        const T*, int64_t, const double*, const double*,          \
                                        const uint8_t*, const DevParams&, int, double, T*, T*);   \
  template cudaError_t launch_gs_prep<T>(const Launch&, int64_t, int64_t, const T*, const T*,     \
                                         double, int, int, T*);                                   \
  template cudaError_t launch_gs_stage<T>(const Launch&, int64_t, int64_t, int, int, const T*,    \
                                          const T*, double, T*, T*);                              \
  template cudaError_t launch_project<T>(const Launch&, const DSeg&, int64_t, const T*,           \
                                         const uint8_t*, T*, double*, const double*, Red, int*);  \
  template cudaError_t launch_import<T>(const Launch&, int64_t, int, const double*,               \
                                        const int64_t*, T*, int64_t, int64_t, const uint8_t*, T*); \
  template cudaError_t launch_export<T>(const Launch&, int64_t, int, const T*, int64_t, int64_t,  \
                                        const int64_t*, double*, const T*);                       \
  template cudaError_t launch_extrapolate<T>(const Launch&, int64_t, T*, T*);                     \
  template cudaError_t launch_scaled_diff<T>(const Launch&, int64_t, const T*, const T*,          \
                                             const T*, double, float*);

GSPM_INSTANTIATE(double)
GSPM_INSTANTIATE(float)
template cudaError_t launch_convert<double, float>(const Launch&, int64_t, const double*, float*);
template cudaError_t launch_convert<float, double>(const Launch&, int64_t, const float*, double*);
template cudaError_t launch_convert<double, double>(const Launch&, int64_t, const double*, double*);
template cudaError_t launch_convert<float, float>(const Launch&, int64_t, const float*, float*);

}  // namespace gspm
