// GSPM kernels for sm_103a.  The path is HBM-bound: sparse row gathers over a SELL-32 node graph
// (one thread per node row, one warp per 32-row slice, every (k, b) value run of a slice one
// coalesced 128/256-byte load), FP64 grid reductions with a fixed summation order, and fused
// pointwise updates.  Matrix values and column indices are streamed with evict-first loads so
// that the gathered vectors stay resident in L2.
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace gspm {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(kFull, x, o);
  return x;
}

// Deterministic grid reduction (last-block pattern).  Every block reduces its NC values with a
// fixed warp/block tree, writes one partial per component, and the last block to arrive sums
// the partials in block order with the same tree.  Returns true in the last block, whose
// threads then find the totals in res[0..NC).
template <int NC>
__device__ __forceinline__ bool grid_reduce(double (&v)[NC], const Red& red, double* res) {
  __shared__ double sm[NC][32];
  __shared__ int am_last;
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
      if (lane == 0) red.partial[(int64_t)blockIdx.x * kRedComp + c] = x;
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(red.counter, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      acc += __ldcg(red.partial + (int64_t)b * kRedComp + c);
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
  if (threadIdx.x == 0) *red.counter = 0u;
  __syncthreads();
  return true;
}

__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

// y_r(row) = sum_k A(row, k) x_r(col(row, k)) for one row of a scalar SELL matrix.
template <typename V, typename X, typename Acc, int NR>
__device__ __forceinline__ void sell_scalar_row(const DSell& A, const V* __restrict__ val,
                                                int64_t s, int lane, const X* __restrict__ x,
                                                int64_t ld, const int (&skip)[NR],
                                                Acc (&acc)[NR]) {
  const int64_t base = A.sptr[s];
  const int len = A.slen[s];
  const int32_t* cp = A.col + base + lane;
  const V* vp = val + base + lane;
#pragma unroll
  for (int r = 0; r < NR; ++r) acc[r] = Acc(0);
#pragma unroll 4
  for (int k = 0; k < len; ++k) {
    const int j = __ldcs(cp + (int64_t)k * 32);
    const Acc a = (Acc)__ldcs(vp + (int64_t)k * 32);
#pragma unroll
    for (int r = 0; r < NR; ++r)
      if (!skip[r]) acc[r] += a * (Acc)__ldg(x + r * ld + j);
  }
}

// 3x3-block row: y(row, a) = sum_k sum_b A(row, k)_ab x(col, b); x, y arrays of [n][3].
template <typename V, typename X, typename Acc>
__device__ __forceinline__ void sell_block_row(const DSell& A, const V* __restrict__ val,
                                               int64_t s, int lane, const X* __restrict__ x,
                                               Acc (&acc)[3]) {
  const int64_t base = A.sptr[s];
  const int len = A.slen[s];
  const int32_t* cp = A.col + base + lane;
  const V* vp = val + base * 9 + lane;
  acc[0] = acc[1] = acc[2] = Acc(0);
#pragma unroll 2
  for (int k = 0; k < len; ++k) {
    const int64_t j = __ldcs(cp + (int64_t)k * 32);
    const V* bp = vp + (int64_t)k * 288;
    const Acc x0 = (Acc)__ldg(x + 3 * j), x1 = (Acc)__ldg(x + 3 * j + 1),
              x2 = (Acc)__ldg(x + 3 * j + 2);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      acc[a] += (Acc)__ldcs(bp + (3 * a + 0) * 32) * x0;
      acc[a] += (Acc)__ldcs(bp + (3 * a + 1) * 32) * x1;
      acc[a] += (Acc)__ldcs(bp + (3 * a + 2) * 32) * x2;
    }
  }
}

// ------------------------------------------------------------------------------------------
// volume average: out[c] = sum_i w_i f(i, c) (+ add[c]); Sec. 2.4 with nodal weights M_L,i / V
// ------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kBlock) k_wsum(int64_t n, int nc, const T* __restrict__ f,
                                                 int64_t cs, int64_t ns,
                                                 const int64_t* __restrict__ perm,
                                                 const double* __restrict__ w, double* out,
                                                 const double* add, Red red) {
  double v[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) v[c] = 0.0;
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const double wi = w[i];
    const int64_t src = perm ? perm[i] : i;
#pragma unroll
    for (int c = 0; c < 9; ++c)
      if (c < nc) v[c] += wi * (double)f[src * ns + c * cs];
  }
  __shared__ double res[9];
  if (grid_reduce<9>(v, red, res) && threadIdx.x == 0)
    for (int c = 0; c < nc; ++c) out[c] = res[c] + (add ? add[c] : 0.0);
}

// ------------------------------------------------------------------------------------------
// plain SpMV (operator access)
// ------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kBlock) k_spmv1(DSell A, const T* __restrict__ val,
                                                  const T* __restrict__ x, T* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = gstride() >> 5;
  const int skip[1] = {0};
  for (int64_t s = gtid() >> 5; s < A.nslices; s += nw) {
    T acc[1];
    sell_scalar_row<T, T, T, 1>(A, val, s, lane, x, 0, skip, acc);
    const int64_t row = s * 32 + lane;
    if (row < A.n) y[row] = acc[0];
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_spmv9(DSell A, const T* __restrict__ val,
                                                  const T* __restrict__ x, T* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = gstride() >> 5;
  for (int64_t s = gtid() >> 5; s < A.nslices; s += nw) {
    T acc[3];
    sell_block_row<T, T, T>(A, val, s, lane, x, acc);
    const int64_t row = s * 32 + lane;
    if (row < A.n) {
      y[3 * row] = acc[0];
      y[3 * row + 1] = acc[1];
      y[3 * row + 2] = acc[2];
    }
  }
}

// ------------------------------------------------------------------------------------------
// conjugate gradients (Sec. 2.5, unpreconditioned), all scalars on the device
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void cg_start(CGState* st, int nr, const double* bb, const double* rr,
                                         double rtol, int max_iter, int allow_zero_x) {
  int any = 0, zero = 0;
  for (int k = 0; k < 3; ++k) {
    CGRhs& q = st->r[k];
    if (k < nr) {
      q.bb = bb[k];
      q.rr = rr[k];
      q.tol2 = rtol * rtol * bb[k];
      q.iters = 0;
      q.alpha = q.beta = q.pq = 0.0;
      q.done = (bb[k] == 0.0 || rr[k] < q.tol2) ? 1 : 0;
      if (bb[k] == 0.0) zero = 1;
      any |= !q.done;
    } else {
      q = CGRhs{0, 0, 0, 0, 0, 0, 0, 1};
    }
  }
  st->nr = nr;
  st->active = any;
  st->max_iter = max_iter;
  st->noconv = 0;
  st->zero_x = allow_zero_x ? zero : 0;
}

// r = b - A x, p = r (scalar B = 1 or 3x3 block B = 9), one right-hand side
template <typename T, int B>
__global__ void __launch_bounds__(kBlock) k_cg_init(DSell A, const T* __restrict__ val,
                                                    const double* __restrict__ b,
                                                    const double* __restrict__ x,
                                                    double* __restrict__ r, T* __restrict__ p,
                                                    CGState* st, double rtol, int max_iter,
                                                    Red red) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = gstride() >> 5;
  double v[2] = {0.0, 0.0};  // rr, bb
  for (int64_t s = gtid() >> 5; s < A.nslices; s += nw) {
    const int64_t row = s * 32 + lane;
    if (B == 1) {
      double acc[1];
      const int skip[1] = {0};
      sell_scalar_row<T, double, double, 1>(A, val, s, lane, x, 0, skip, acc);
      if (row < A.n) {
        const double rv = b[row] - acc[0];
        r[row] = rv;
        p[row] = (T)rv;
        v[0] += rv * rv;
        v[1] += b[row] * b[row];
      }
    } else {
      double acc[3];
      sell_block_row<T, double, double>(A, val, s, lane, x, acc);
      if (row < A.n) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const double rv = b[3 * row + a] - acc[a];
          r[3 * row + a] = rv;
          p[3 * row + a] = (T)rv;
          v[0] += rv * rv;
          v[1] += b[3 * row + a] * b[3 * row + a];
        }
      }
    }
  }
  __shared__ double res[2];
  if (grid_reduce<2>(v, red, res) && threadIdx.x == 0) {
    const double bb[1] = {res[1]}, rr[1] = {res[0]};
    cg_start(st, 1, bb, rr, rtol, max_iter, 1);
  }
}

// GSPM systems (M + c eps K) g = M f with x0 = f already in x: b = M x, r = b - A x, p = r
template <typename T, int NR>
__global__ void __launch_bounds__(kBlock) k_cg_init_gs(DSell A, const T* __restrict__ aval,
                                                       const T* __restrict__ mval, int64_t ld,
                                                       const double* __restrict__ x,
                                                       double* __restrict__ r,
                                                       T* __restrict__ p, CGState* st,
                                                       double rtol, int max_iter, Red red) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = gstride() >> 5;
  const int skip[NR] = {};
  double v[2 * NR];
#pragma unroll
  for (int k = 0; k < 2 * NR; ++k) v[k] = 0.0;
  for (int64_t s = gtid() >> 5; s < A.nslices; s += nw) {
    double ax[NR], mx[NR];
    sell_scalar_row<T, double, double, NR>(A, aval, s, lane, x, ld, skip, ax);
    sell_scalar_row<T, double, double, NR>(A, mval, s, lane, x, ld, skip, mx);
    const int64_t row = s * 32 + lane;
    if (row < A.n) {
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        const double rv = mx[k] - ax[k];
        r[k * ld + row] = rv;
        p[k * ld + row] = (T)rv;
        v[2 * k] += rv * rv;
        v[2 * k + 1] += mx[k] * mx[k];
      }
    }
  }
  __shared__ double res[2 * NR];
  if (grid_reduce<2 * NR>(v, red, res) && threadIdx.x == 0) {
    double bb[NR], rr[NR];
    for (int k = 0; k < NR; ++k) {
      rr[k] = res[2 * k];
      bb[k] = res[2 * k + 1];
    }
    cg_start(st, NR, bb, rr, rtol, max_iter, 0);
  }
}

// q = A p with the p.q dot fused; last block forms alpha = rr / p.q
template <typename T, int B, int NR>
__global__ void __launch_bounds__(kBlock) k_cg_spmv(DSell A, const T* __restrict__ val, int64_t ld,
                                                    const T* __restrict__ p, T* __restrict__ q,
                                                    CGState* st, Red red) {
  if (!st->active) return;
  int skip[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) skip[k] = st->r[k].done;
  const int lane = threadIdx.x & 31;
  const int64_t nw = gstride() >> 5;
  double v[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) v[k] = 0.0;
  for (int64_t s = gtid() >> 5; s < A.nslices; s += nw) {
    const int64_t row = s * 32 + lane;
    if (B == 1) {
      T acc[NR];
      sell_scalar_row<T, T, T, NR>(A, val, s, lane, p, ld, skip, acc);
      if (row < A.n) {
#pragma unroll
        for (int k = 0; k < NR; ++k)
          if (!skip[k]) {
            q[k * ld + row] = acc[k];
            v[k] += (double)p[k * ld + row] * (double)acc[k];
          }
      }
    } else {
      T acc[3];
      sell_block_row<T, T, T>(A, val, s, lane, p, acc);
      if (row < A.n) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          q[3 * row + a] = acc[a];
          v[0] += (double)p[3 * row + a] * (double)acc[a];
        }
      }
    }
  }
  __shared__ double res[NR];
  if (grid_reduce<NR>(v, red, res) && threadIdx.x == 0) {
    for (int k = 0; k < NR; ++k) {
      CGRhs& c = st->r[k];
      if (c.done) continue;
      c.pq = res[k];
      if (res[k] > 0.0) {
        c.alpha = c.rr / res[k];
      } else {  // p = 0: nothing left to reduce
        c.alpha = 0.0;
        c.done = 1;
      }
    }
  }
}

// x += alpha p, r -= alpha q, r.r fused; last block forms beta and the stopping decision
template <typename T, int NR>
__global__ void __launch_bounds__(kBlock) k_cg_update(int64_t len, int64_t ld, double* __restrict__ x,
                                                      double* __restrict__ r,
                                                      const T* __restrict__ p,
                                                      const T* __restrict__ q, CGState* st,
                                                      Red red) {
  if (!st->active) return;
  int skip[NR];
  double al[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    skip[k] = st->r[k].done;
    al[k] = st->r[k].alpha;
  }
  double v[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) v[k] = 0.0;
  for (int64_t i = gtid(); i < len; i += gstride()) {
#pragma unroll
    for (int k = 0; k < NR; ++k)
      if (!skip[k]) {
        const int64_t o = k * ld + i;
        x[o] += al[k] * (double)p[o];
        const double rv = r[o] - al[k] * (double)q[o];
        r[o] = rv;
        v[k] += rv * rv;
      }
  }
  __shared__ double res[NR];
  if (grid_reduce<NR>(v, red, res) && threadIdx.x == 0) {
    int any = 0;
    for (int k = 0; k < NR; ++k) {
      CGRhs& c = st->r[k];
      if (c.done) continue;
      c.iters += 1;
      c.beta = res[k] / c.rr;
      c.rr = res[k];
      if (res[k] < c.tol2) {
        c.done = 1;
      } else if (c.iters >= st->max_iter) {
        c.done = 1;
        st->noconv += 1;
      }
      any |= !c.done;
    }
    st->active = any;
  }
}

template <typename T, int NR>
__global__ void __launch_bounds__(kBlock) k_cg_pupdate(int64_t len, int64_t ld,
                                                       const double* __restrict__ r,
                                                       T* __restrict__ p, const CGState* st) {
  if (!st->active) return;
  int skip[NR];
  double be[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    skip[k] = st->r[k].done;
    be[k] = st->r[k].beta;
  }
  for (int64_t i = gtid(); i < len; i += gstride()) {
#pragma unroll
    for (int k = 0; k < NR; ++k)
      if (!skip[k]) {
        const int64_t o = k * ld + i;
        p[o] = (T)(r[o] + be[k] * (double)p[o]);
      }
  }
}

__global__ void k_cg_zero(int64_t len, double* x, const CGState* st) {
  if (!st->zero_x) return;
  for (int64_t i = gtid(); i < len; i += gstride()) x[i] = 0.0;
}

// ------------------------------------------------------------------------------------------
// F^ms / G operators (Sec. 2.3): right-hand sides and derivatives as row gathers
// ------------------------------------------------------------------------------------------
// b_i = sum_j F_{ij,a} m_{j,a}  (Eq. RHS_b divided by m_s); pinned entry 0
template <typename T>
__global__ void __launch_bounds__(kBlock) k_fdiv(DSell A, const T* __restrict__ Fv,
                                                 const T* __restrict__ m, int64_t ld,
                                                 double* __restrict__ b, int64_t pin) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = gstride() >> 5;
  for (int64_t s = gtid() >> 5; s < A.nslices; s += nw) {
    const int64_t base = A.sptr[s];
    const int len = A.slen[s];
    const int32_t* cp = A.col + base + lane;
    const T* vp = Fv + base * 3 + lane;
    T acc = T(0);
#pragma unroll 4
    for (int k = 0; k < len; ++k) {
      const int64_t j = __ldcs(cp + (int64_t)k * 32);
      const T* fp = vp + (int64_t)k * 96;
      acc += __ldcs(fp) * __ldg(m + j) + __ldcs(fp + 32) * __ldg(m + ld + j) +
             __ldcs(fp + 64) * __ldg(m + 2 * ld + j);
    }
    const int64_t row = s * 32 + lane;
    if (row < A.n) b[row] = row == pin ? 0.0 : (double)acc;
  }
}

// h~_d,a = (F_a U)_i / M_L,i  (= -grad U, Sec. 2.3 with the lumped-mass normalisation)
template <typename T>
__global__ void __launch_bounds__(kBlock) k_fgrad(DSell A, const T* __restrict__ Fv,
                                                  const double* __restrict__ U,
                                                  const double* __restrict__ invML,
                                                  T* __restrict__ hd, int64_t ld) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = gstride() >> 5;
  for (int64_t s = gtid() >> 5; s < A.nslices; s += nw) {
    const int64_t base = A.sptr[s];
    const int len = A.slen[s];
    const int32_t* cp = A.col + base + lane;
    const T* vp = Fv + base * 3 + lane;
    T a0 = T(0), a1 = T(0), a2 = T(0);
#pragma unroll 4
    for (int k = 0; k < len; ++k) {
      const int64_t j = __ldcs(cp + (int64_t)k * 32);
      const T* fp = vp + (int64_t)k * 96;
      const T u = (T)__ldg(U + j);
      a0 += __ldcs(fp) * u;
      a1 += __ldcs(fp + 32) * u;
      a2 += __ldcs(fp + 64) * u;
    }
    const int64_t row = s * 32 + lane;
    if (row < A.n) {
      const T im = (T)invML[row];
      hd[row] = a0 * im;
      hd[ld + row] = a1 * im;
      hd[2 * ld + row] = a2 * im;
    }
  }
}

// E = E_bar + sym grad u with grad_a u_b = -(F_a u_b)_i / M_L,i; E stored SoA Voigt
// (11, 22, 33, 23, 13, 12) with tensor shear components
template <typename T>
__global__ void __launch_bounds__(kBlock) k_fstrain(DSell A, const T* __restrict__ Fv,
                                                    const double* __restrict__ u,
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
    T g[3][3] = {};
#pragma unroll 2
    for (int k = 0; k < len; ++k) {
      const int64_t j = __ldcs(cp + (int64_t)k * 32);
      const T* fp = vp + (int64_t)k * 96;
      const T f[3] = {__ldcs(fp), __ldcs(fp + 32), __ldcs(fp + 64)};
      const T uj[3] = {(T)__ldg(u + 3 * j), (T)__ldg(u + 3 * j + 1), (T)__ldg(u + 3 * j + 2)};
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) g[a][b] += f[a] * uj[b];
    }
    const int64_t row = s * 32 + lane;
    if (row < A.n) {
      const T im = -(T)invML[row];  // g[a][b] * im = d_a u_b
      E[row] = (T)Ebar[0] + g[0][0] * im;
      E[ld + row] = (T)Ebar[1] + g[1][1] * im;
      E[2 * ld + row] = (T)Ebar[2] + g[2][2] * im;
      E[3 * ld + row] = (T)Ebar[3] + T(0.5) * (g[1][2] + g[2][1]) * im;
      E[4 * ld + row] = (T)Ebar[4] + T(0.5) * (g[0][2] + g[2][0]) * im;
      E[5 * ld + row] = (T)Ebar[5] + T(0.5) * (g[0][1] + g[1][0]) * im;
    }
  }
}

// b^mech_(i,a) = sum_j sum_c G_{ij,c} sigma0_{j,ac}, sigma0 = C E0 (nodal, [n][6] Voigt);
// pinned node's entries 0  (= F^mech E0 of Eq. RHS_b for a spatially uniform C)
template <typename T>
__global__ void __launch_bounds__(kBlock) k_gdiv(DSell A, const T* __restrict__ Gv,
                                                 const T* __restrict__ sig0,
                                                 double* __restrict__ b, int64_t pin) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = gstride() >> 5;
  for (int64_t s = gtid() >> 5; s < A.nslices; s += nw) {
    const int64_t base = A.sptr[s];
    const int len = A.slen[s];
    const int32_t* cp = A.col + base + lane;
    const T* vp = Gv + base * 3 + lane;
    T b0 = T(0), b1 = T(0), b2 = T(0);
#pragma unroll 2
    for (int k = 0; k < len; ++k) {
      const int64_t j = __ldcs(cp + (int64_t)k * 32);
      const T* gp = vp + (int64_t)k * 96;
      const T g0 = __ldcs(gp), g1 = __ldcs(gp + 32), g2 = __ldcs(gp + 64);
      const T* sj = sig0 + 6 * j;
      const T s11 = __ldg(sj), s22 = __ldg(sj + 1), s33 = __ldg(sj + 2), s23 = __ldg(sj + 3),
              s13 = __ldg(sj + 4), s12 = __ldg(sj + 5);
      b0 += g0 * s11 + g1 * s12 + g2 * s13;
      b1 += g0 * s12 + g1 * s22 + g2 * s23;
      b2 += g0 * s13 + g1 * s23 + g2 * s33;
    }
    const int64_t row = s * 32 + lane;
    if (row < A.n) {
      const bool pz = row == pin;
      b[3 * row] = pz ? 0.0 : (double)b0;
      b[3 * row + 1] = pz ? 0.0 : (double)b1;
      b[3 * row + 2] = pz ? 0.0 : (double)b2;
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

template <typename T>
__global__ void __launch_bounds__(kBlock) k_e0(int64_t n, const T* __restrict__ m, int64_t ld,
                                               const uint8_t* __restrict__ mag, DevParams P,
                                               T* __restrict__ E0, T* __restrict__ sig0) {
  for (int64_t i = gtid(); i < n; i += gstride()) {
    T e[6] = {}, s[6] = {};
    if (mag[i]) {
      e0_of<T>(m[i], m[ld + i], m[2 * ld + i], P, e);
      stress_of<T>(e, P, s);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      E0[c * ld + i] = e[c];
      sig0[6 * i + c] = s[c];
    }
  }
}

// h = -kappa m_a (|m|^2 - m_a^2) + H/m_s + (3/(mu0 ms^2)) [l100 m_a s_aa + l111 (m_b s_ab +
// m_c s_ac)] + h~_d - N_d m_bar, with s = C (E - E0(m)); zero off Omega_m
template <typename T>
__global__ void __launch_bounds__(kBlock) k_hfield(int64_t n, const T* __restrict__ m,
                                                   const T* __restrict__ hd,
                                                   const T* __restrict__ E, int64_t ld,
                                                   const double* __restrict__ mbar,
                                                   const uint8_t* __restrict__ mag, DevParams P,
                                                   int mode, double coef, T* __restrict__ h,
                                                   double* __restrict__ x) {
  T far[3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
    far[a] = (T)(P.hz[a] - (P.Nd[3 * a] * mbar[0] + P.Nd[3 * a + 1] * mbar[1] +
                            P.Nd[3 * a + 2] * mbar[2]));
  const T kap = (T)P.kappa, mec = (T)P.me_coef, l100 = (T)P.l100, l111 = (T)P.l111;
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const T mv[3] = {m[i], m[ld + i], m[2 * ld + i]};
    T hv[3] = {T(0), T(0), T(0)};
    if (mag[i]) {
      T e0[6], d[6], s[6];
      e0_of<T>(mv[0], mv[1], mv[2], P, e0);
#pragma unroll
      for (int c = 0; c < 6; ++c) d[c] = E[c * ld + i] - e0[c];
      stress_of<T>(d, P, s);
      // full symmetric stress lookup: (0,0)->0 (1,1)->1 (2,2)->2 (1,2)->3 (0,2)->4 (0,1)->5
      const T S[3][3] = {{s[0], s[5], s[4]}, {s[5], s[1], s[3]}, {s[4], s[3], s[2]}};
      const T m2sum = mv[0] * mv[0] + mv[1] * mv[1] + mv[2] * mv[2];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int b = (a + 1) % 3, c = (a + 2) % 3;
        const T an = -kap * mv[a] * (m2sum - mv[a] * mv[a]);
        const T me = mec * (l100 * mv[a] * S[a][a] + l111 * (mv[b] * S[a][b] + mv[c] * S[a][c]));
        hv[a] = an + far[a] + me + hd[a * ld + i];
      }
    }
    if (mode == 0) {
#pragma unroll
      for (int a = 0; a < 3; ++a) h[a * ld + i] = hv[a];
    } else {
#pragma unroll
      for (int a = 0; a < 3; ++a) x[a * ld + i] = (double)mv[a] + coef * (double)hv[a];
    }
  }
}

// x_k = m_{c0+k} + dtau h_{c0+k}, k < nc  (GSPM right-hand-side fields f, Algorithm B.1)
template <typename T>
__global__ void __launch_bounds__(kBlock) k_gs_prep(int64_t n, int64_t ld, const T* __restrict__ m,
                                                    const T* __restrict__ h, double dtau, int c0,
                                                    int nc, double* __restrict__ x) {
  for (int64_t i = gtid(); i < n; i += gstride())
    for (int k = 0; k < nc; ++k) {
      const int c = c0 + k;
      x[k * ld + i] = (double)m[c * ld + i] + dtau * (double)h[c * ld + i];
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
                                                     double* __restrict__ x,
                                                     T* __restrict__ ms) {
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const double m1 = m[i], m2 = m[ld + i], m3 = m[2 * ld + i];
    if (!printed) {
      if (stage == 1) {
        const double s1 = m1 + (x[i] * m3 - x[ld + i] * m2);
        ms[i] = (T)s1;
        x[2 * ld + i] = (double)(T)s1 + dtau * (double)h[i];
      } else if (stage == 2) {
        const double s1 = ms[i];
        const double s2 = m2 + (x[ld + i] * s1 - x[2 * ld + i] * m3);
        ms[ld + i] = (T)s2;
        x[i] = (double)(T)s2 + dtau * (double)h[ld + i];
      } else {
        const double s1 = ms[i], s2 = ms[ld + i];
        ms[2 * ld + i] = (T)(m3 + (x[2 * ld + i] * s2 - x[i] * s1));
      }
    } else {
      if (stage == 1) {
        const double g1 = x[i], g2 = x[ld + i], g3 = x[2 * ld + i];
        const double s1 = m1 + (g2 * m3 - g3 * m2);
        const double s2 = m2 + (g3 * m1 - g1 * m3);
        ms[i] = (T)s1;
        ms[ld + i] = (T)s2;
        x[i] = (double)(T)s1 + dtau * (double)h[i];
        x[ld + i] = (double)(T)s2 + dtau * (double)h[ld + i];
      } else {
        const double s1 = ms[i], s2 = ms[ld + i];
        ms[2 * ld + i] = (T)(m3 + (x[i] * s2 - x[ld + i] * s1));
      }
    }
  }
}

// Algorithm B.1 step 4: m = m** / |m**| on Omega_m; <|m_new - m_old|> over magnetic nodes
template <typename T>
__global__ void __launch_bounds__(kBlock) k_project(int64_t n, int64_t ld,
                                                    const double* __restrict__ x,
                                                    const uint8_t* __restrict__ mag,
                                                    T* __restrict__ m, double* dm_out,
                                                    double inv_nmag, Red red) {
  double v[1] = {0.0};
  for (int64_t i = gtid(); i < n; i += gstride()) {
    if (!mag[i]) continue;
    const T a = (T)x[i], b = (T)x[ld + i], c = (T)x[2 * ld + i];
    const T inv = T(1) / sqrt(a * a + b * b + c * c);
    const T na = a * inv, nb = b * inv, nc = c * inv;
    const T da = na - m[i], db = nb - m[ld + i], dc = nc - m[2 * ld + i];
    v[0] += (double)sqrt(da * da + db * db + dc * dc);
    m[i] = na;
    m[ld + i] = nb;
    m[2 * ld + i] = nc;
  }
  __shared__ double res[1];
  if (grid_reduce<1>(v, red, res) && threadIdx.x == 0) *dm_out = res[0] * inv_nmag;
}

// ------------------------------------------------------------------------------------------
// layout changes between the ABI ([n][nc] float64, unique-node order) and internal arrays
// ------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_import(int64_t n, int nc, const double* __restrict__ src,
                         const int64_t* __restrict__ perm, T* __restrict__ dst, int64_t cs,
                         int64_t ns, const uint8_t* __restrict__ mask) {
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const int64_t o = perm[i];
    const bool z = mask && !mask[i];
    for (int c = 0; c < nc; ++c) dst[i * ns + c * cs] = z ? T(0) : (T)src[o * nc + c];
  }
}

template <typename T>
__global__ void k_export(int64_t n, int nc, const T* __restrict__ src, int64_t cs, int64_t ns,
                         const int64_t* __restrict__ perm, double* __restrict__ dst) {
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const int64_t o = perm[i];
    for (int c = 0; c < nc; ++c) dst[o * nc + c] = (double)src[i * ns + c * cs];
  }
}

template <typename S, typename D>
__global__ void k_convert(int64_t len, const S* __restrict__ s, D* __restrict__ d) {
  for (int64_t i = gtid(); i < len; i += gstride()) d[i] = (D)s[i];
}

}  // namespace

// ------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------
#define GSPM_LAUNCH(L, threads) \
  (*(L).counter) += 1;          \
  const int nb = (L).blocks_for(threads)

template <typename T>
cudaError_t launch_wsum(const Launch& L, int64_t n, int nc, const T* f, int64_t cs, int64_t ns,
                        const int64_t* perm, const double* w, double* out, const double* add,
                        Red red) {
  GSPM_LAUNCH(L, n);
  k_wsum<T><<<nb, kBlock, 0, L.stream>>>(n, nc, f, cs, ns, perm, w, out, add, red);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spmv(const Launch& L, const DSell& A, const T* val, int B, const T* x, T* y) {
  GSPM_LAUNCH(L, A.nslices * 32);
  if (B == 1)
    k_spmv1<T><<<nb, kBlock, 0, L.stream>>>(A, val, x, y);
  else
    k_spmv9<T><<<nb, kBlock, 0, L.stream>>>(A, val, x, y);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_init(const Launch& L, const DSell& A, const T* val, int B, const double* b,
                           double* x, double* r, T* p, CGState* st, double rtol, int max_iter,
                           Red red) {
  GSPM_LAUNCH(L, A.nslices * 32);
  if (B == 1)
    k_cg_init<T, 1><<<nb, kBlock, 0, L.stream>>>(A, val, b, x, r, p, st, rtol, max_iter, red);
  else
    k_cg_init<T, 9><<<nb, kBlock, 0, L.stream>>>(A, val, b, x, r, p, st, rtol, max_iter, red);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_init_gs(const Launch& L, const DSell& A, const T* aval, const T* mval,
                              int nr, int64_t ld, double* x, double* r, T* p, CGState* st,
                              double rtol, int max_iter, Red red) {
  GSPM_LAUNCH(L, A.nslices * 32);
  switch (nr) {
    case 1: k_cg_init_gs<T, 1><<<nb, kBlock, 0, L.stream>>>(A, aval, mval, ld, x, r, p, st, rtol, max_iter, red); break;
    case 2: k_cg_init_gs<T, 2><<<nb, kBlock, 0, L.stream>>>(A, aval, mval, ld, x, r, p, st, rtol, max_iter, red); break;
    case 3: k_cg_init_gs<T, 3><<<nb, kBlock, 0, L.stream>>>(A, aval, mval, ld, x, r, p, st, rtol, max_iter, red); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_spmv(const Launch& L, const DSell& A, const T* val, int B, int nr,
                           int64_t ld, const T* p, T* q, CGState* st, Red red) {
  GSPM_LAUNCH(L, A.nslices * 32);
  if (B == 9) {
    k_cg_spmv<T, 9, 1><<<nb, kBlock, 0, L.stream>>>(A, val, ld, p, q, st, red);
  } else {
    switch (nr) {
      case 1: k_cg_spmv<T, 1, 1><<<nb, kBlock, 0, L.stream>>>(A, val, ld, p, q, st, red); break;
      case 2: k_cg_spmv<T, 1, 2><<<nb, kBlock, 0, L.stream>>>(A, val, ld, p, q, st, red); break;
      case 3: k_cg_spmv<T, 1, 3><<<nb, kBlock, 0, L.stream>>>(A, val, ld, p, q, st, red); break;
      default: return cudaErrorInvalidValue;
    }
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_update(const Launch& L, int64_t len, int nr, int64_t ld, double* x,
                             double* r, const T* p, const T* q, CGState* st, Red red) {
  GSPM_LAUNCH(L, len);
  switch (nr) {
    case 1: k_cg_update<T, 1><<<nb, kBlock, 0, L.stream>>>(len, ld, x, r, p, q, st, red); break;
    case 2: k_cg_update<T, 2><<<nb, kBlock, 0, L.stream>>>(len, ld, x, r, p, q, st, red); break;
    case 3: k_cg_update<T, 3><<<nb, kBlock, 0, L.stream>>>(len, ld, x, r, p, q, st, red); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_pupdate(const Launch& L, int64_t len, int nr, int64_t ld, const double* r,
                              T* p, const CGState* st) {
  GSPM_LAUNCH(L, len);
  switch (nr) {
    case 1: k_cg_pupdate<T, 1><<<nb, kBlock, 0, L.stream>>>(len, ld, r, p, st); break;
    case 2: k_cg_pupdate<T, 2><<<nb, kBlock, 0, L.stream>>>(len, ld, r, p, st); break;
    case 3: k_cg_pupdate<T, 3><<<nb, kBlock, 0, L.stream>>>(len, ld, r, p, st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_cg_zero(const Launch& L, int64_t len, double* x, const CGState* st) {
  GSPM_LAUNCH(L, len);
  k_cg_zero<<<nb, kBlock, 0, L.stream>>>(len, x, st);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fdiv(const Launch& L, const DSell& A, const T* Fv, const T* m, int64_t ld,
                        double* b, int64_t pin) {
  GSPM_LAUNCH(L, A.nslices * 32);
  k_fdiv<T><<<nb, kBlock, 0, L.stream>>>(A, Fv, m, ld, b, pin);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fgrad(const Launch& L, const DSell& A, const T* Fv, const double* U,
                         const double* invML, T* hd, int64_t ld) {
  GSPM_LAUNCH(L, A.nslices * 32);
  k_fgrad<T><<<nb, kBlock, 0, L.stream>>>(A, Fv, U, invML, hd, ld);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fstrain(const Launch& L, const DSell& A, const T* Fv, const double* u,
                           const double* invML, const double* Ebar, T* E, int64_t ld) {
  GSPM_LAUNCH(L, A.nslices * 32);
  k_fstrain<T><<<nb, kBlock, 0, L.stream>>>(A, Fv, u, invML, Ebar, E, ld);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gdiv(const Launch& L, const DSell& A, const T* Gv, const T* sig0, double* b,
                        int64_t pin) {
  GSPM_LAUNCH(L, A.nslices * 32);
  k_gdiv<T><<<nb, kBlock, 0, L.stream>>>(A, Gv, sig0, b, pin);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_e0(const Launch& L, int64_t n, const T* m, int64_t ld, const uint8_t* mag,
                      const DevParams& P, T* E0, T* sig0) {
  GSPM_LAUNCH(L, n);
  k_e0<T><<<nb, kBlock, 0, L.stream>>>(n, m, ld, mag, P, E0, sig0);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_hfield(const Launch& L, int64_t n, const T* m, const T* hd, const T* E,
                          int64_t ld, const double* mbar, const uint8_t* mag, const DevParams& P,
                          int mode, double coef, T* h, double* x) {
  GSPM_LAUNCH(L, n);
  k_hfield<T><<<nb, kBlock, 0, L.stream>>>(n, m, hd, E, ld, mbar, mag, P, mode, coef, h, x);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gs_prep(const Launch& L, int64_t n, int64_t ld, const T* m, const T* h,
                           double dtau, int c0, int nc, double* x) {
  GSPM_LAUNCH(L, n);
  k_gs_prep<T><<<nb, kBlock, 0, L.stream>>>(n, ld, m, h, dtau, c0, nc, x);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gs_stage(const Launch& L, int64_t n, int64_t ld, int stage, int printed,
                            const T* m, const T* h, double dtau, double* x, T* ms) {
  GSPM_LAUNCH(L, n);
  k_gs_stage<T><<<nb, kBlock, 0, L.stream>>>(n, ld, stage, printed, m, h, dtau, x, ms);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_project(const Launch& L, int64_t n, int64_t ld, const double* x,
                           const uint8_t* mag, T* m, double* dm_out, double inv_nmag, Red red) {
  GSPM_LAUNCH(L, n);
  k_project<T><<<nb, kBlock, 0, L.stream>>>(n, ld, x, mag, m, dm_out, inv_nmag, red);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_import(const Launch& L, int64_t n, int nc, const double* src,
                          const int64_t* perm, T* dst, int64_t cs, int64_t ns,
                          const uint8_t* mask) {
  GSPM_LAUNCH(L, n);
  k_import<T><<<nb, kBlock, 0, L.stream>>>(n, nc, src, perm, dst, cs, ns, mask);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_export(const Launch& L, int64_t n, int nc, const T* src, int64_t cs,
                          int64_t ns, const int64_t* perm, double* dst) {
  GSPM_LAUNCH(L, n);
  k_export<T><<<nb, kBlock, 0, L.stream>>>(n, nc, src, cs, ns, perm, dst);
  return cudaGetLastError();
}

template <typename S, typename D>
cudaError_t launch_convert(const Launch& L, int64_t len, const S* src, D* dst) {
  GSPM_LAUNCH(L, len);
  k_convert<S, D><<<nb, kBlock, 0, L.stream>>>(len, src, dst);
  return cudaGetLastError();
}

#define GSPM_INSTANTIATE(T)                                                                      \
  template cudaError_t launch_wsum<T>(const Launch&, int64_t, int, const T*, int64_t, int64_t,   \
                                      const int64_t*, const double*, double*, const double*, Red); \
  template cudaError_t launch_spmv<T>(const Launch&, const DSell&, const T*, int, const T*, T*); \
  template cudaError_t launch_cg_init<T>(const Launch&, const DSell&, const T*, int,             \
                                         const double*, double*, double*, T*, CGState*, double,  \
                                         int, Red);                                               \
  template cudaError_t launch_cg_init_gs<T>(const Launch&, const DSell&, const T*, const T*, int, \
                                            int64_t, double*, double*, T*, CGState*, double,     \
                                            int, Red);                                            \
  template cudaError_t launch_cg_spmv<T>(const Launch&, const DSell&, const T*, int, int,        \
                                         int64_t, const T*, T*, CGState*, Red);                  \
  template cudaError_t launch_cg_update<T>(const Launch&, int64_t, int, int64_t, double*,        \
                                           double*, const T*, const T*, CGState*, Red);          \
  template cudaError_t launch_cg_pupdate<T>(const Launch&, int64_t, int, int64_t, const double*, \
                                            T*, const CGState*);                                  \
  template cudaError_t launch_fdiv<T>(const Launch&, const DSell&, const T*, const T*, int64_t,  \
                                      double*, int64_t);                                          \
  template cudaError_t launch_fgrad<T>(const Launch&, const DSell&, const T*, const double*,     \
                                       const double*, T*, int64_t);                               \
  template cudaError_t launch_fstrain<T>(const Launch&, const DSell&, const T*, const double*,   \
                                         const double*, const double*, T*, int64_t);              \
  template cudaError_t launch_gdiv<T>(const Launch&, const DSell&, const T*, const T*, double*,  \
                                      int64_t);                                                   \
  template cudaError_t launch_e0<T>(const Launch&, int64_t, const T*, int64_t, const uint8_t*,   \
                                    const DevParams&, T*, T*);                                    \
  template cudaError_t launch_hfield<T>(const Launch&, int64_t, const T*, const T*, const T*,    \
                                        int64_t, const double*, const uint8_t*,                  \
                                        const DevParams&, int, double, T*, double*);              \
  template cudaError_t launch_gs_prep<T>(const Launch&, int64_t, int64_t, const T*, const T*,    \
                                         double, int, int, double*);                              \
  template cudaError_t launch_gs_stage<T>(const Launch&, int64_t, int64_t, int, int, const T*,   \
                                          const T*, double, double*, T*);                         \
  template cudaError_t launch_project<T>(const Launch&, int64_t, int64_t, const double*,         \
                                         const uint8_t*, T*, double*, double, Red);               \
  template cudaError_t launch_import<T>(const Launch&, int64_t, int, const double*,              \
                                        const int64_t*, T*, int64_t, int64_t, const uint8_t*);    \
  template cudaError_t launch_export<T>(const Launch&, int64_t, int, const T*, int64_t, int64_t, \
                                        const int64_t*, double*);

GSPM_INSTANTIATE(double)
GSPM_INSTANTIATE(float)
template cudaError_t launch_convert<double, float>(const Launch&, int64_t, const double*, float*);
template cudaError_t launch_convert<float, double>(const Launch&, int64_t, const float*, double*);
template cudaError_t launch_convert<double, double>(const Launch&, int64_t, const double*, double*);

}  // namespace gspm
