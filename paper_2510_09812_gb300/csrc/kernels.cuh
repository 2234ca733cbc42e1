// Device-side types and launcher declarations of the GSPM kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace gspm {

// SELL-32 node graph on the device (see HostSell).
struct DSell {
  const int64_t* sptr;
  const int32_t* slen;
  const int32_t* col;
  int64_t nslices;
  int64_t n;
};

// Scratch for deterministic reductions: one partial per work item and component.
struct Red {
  double* partial;     // [max items of any list * kRedComp]
};

// Work items of the reducing kernels: item i covers the slices [sl0[i], sl1[i]) of segment
// seg[i]; items are grouped by segment (segment s owns items seg_item0[s] .. + seg_nitems[s]).
struct ItemList {
  int nitems;
  const int32_t* seg;        // [nitems]
  const int32_t* sl0;        // [nitems]
  const int32_t* sl1;        // [nitems]
  const int32_t* seg_item0;  // [nseg]
  const int32_t* seg_nitems; // [nseg]
};
constexpr int kItemLists = 8;  // one list per residency 1..8 blocks per SM

// Segments (meshes of a batch).  Segment s owns the rows [seg_row0[s], seg_row0[s] +
// seg_nrow[s]) (its last slice may end in padding rows).  A reducing kernel that keeps k blocks
// resident per SM uses list[k - 1], which holds about k x SMs items (at least one per segment,
// otherwise proportional to the segment's slices), so every block of its single wave reduces
// one item.  counter[s] is the arrival counter of segment s, 0 between kernels.
struct DSeg {
  int nseg;
  const int32_t* seg_of_slice;  // [nslices]
  const int64_t* seg_row0;      // [nseg]
  const int64_t* seg_nrow;      // [nseg]
  const int64_t* seg_pin;       // [nseg] pinned row (global internal index)
  unsigned* counter;            // [nseg]
  ItemList list[kItemLists];
};
constexpr int kRedComp = 16;
constexpr int kBlock = 256;

// Per-solve CG scalars, device resident.  One entry per right-hand side (up to 3).
struct CGRhs {
  double bb, rr, pq, alpha, beta, tol2, rz;  // rz = r.z of the preconditioned CG
  int iters, done;
};
struct CGState {
  CGRhs r[3];
  int nr, active, max_iter, noconv, zero_x, pc;  // pc: preconditioned (one RHS)
  // proj: CG on the singular system projected off the constants (one right-hand side):
  // sr = per-component sums of r, sub = the per-component mean that the p-update subtracts
  // from its input (z, or r without preconditioner)
  int proj, pad;
  double sr[3], sub[3];
};

// Aggregates of the two-level preconditioner, all segments: rows of aggregate I are
// agg_rows[agg_ptr[I] .. agg_ptr[I+1]) (ascending); segment s owns aggregates
// seg_agg0[s] .. seg_agg0[s+1]-1.  With e components per row, coarse index = I * e + a and the
// segment's dense inverse block of side nc = (its aggregates) * e starts at inv_off[s].
struct DCoarse {
  int64_t nagg;
  const int32_t* agg_of_row;  // [n rows] aggregate of each row, -1 on padding rows
  const int32_t* agg_ptr;     // [nagg + 1]
  const int32_t* agg_rows;    // [rows in aggregates]
  const int32_t* agg_seg;     // [nagg]
  const int32_t* seg_agg0;    // [nseg + 1]
  int contig;                 // every aggregate's rows are consecutive (GSPM_ORDER_AGGREGATE)
};

// Material constants needed on the device (reduced units of App. B).  The applied field
// H_ext / m_s is per segment (device array hz[3 * seg + a]).
struct DevParams {
  double kappa, me_coef, l100, l111, C11, C12, C44;
  double Nd[9];
  double dtau, alpha;
  double R[9];   // App. D: v_mesh = R v_crystal (C11, C12, C44, lambda, K1 in crystal axes)
  int rotated;   // R is not the identity
};

// Device-side loop control of a CG loop replayed as a CUDA-graph WHILE node.  After each
// iteration one thread sets the node's condition to (active segments > 0 and iterations < limit),
// so the loop ends when every segment has converged (or stopped at max_iter) and never runs more
// than `limit` times.  count == NULL: not in a graph (launched directly).
struct LoopCtl {
  cudaGraphConditionalHandle handle;
  const int* nactive;
  int* count;                 // iterations of the current loop
  int limit;
  int body;                   // kernels per iteration of the loop body
  unsigned long long* total;  // kernels executed by all loop bodies (launch accounting)
};

struct Launch {
  cudaStream_t stream;
  int max_blocks;        // upper bound of any grid (sizes the reduction scratch): 8 x SMs
  int sms;               // multiprocessors of the device
  int64_t* counter;      // kernel launches issued
  int blocks_for(int64_t threads) const {
    int64_t b = (threads + kBlock - 1) / kBlock;
    if (b > max_blocks) b = max_blocks;
    return b < 1 ? 1 : (int)b;
  }
};

// Grid for a grid-stride kernel: enough blocks for `threads`, capped at the number of blocks the
// kernel can keep resident (occupancy x SMs, looked up once per kernel) and at max_blocks, so
// that every block runs in the first wave.
int grid_for(const Launch& L, int64_t threads, const void* kernel);

// SpMV schedules chosen by the autotuner: 0 = one thread per row, 1 = one thread per row with
// the next neighbours' loads issued ahead of their FMAs, 2 = two threads per row (alternate
// neighbours, combined with a shuffle), 3 = schedule 1 compiled for three resident blocks per
// SM (fewer registers, more warps in flight).
constexpr int kSpmvVariants = 4;

// ---- launchers ----------------------------------------------------------------------------
// T = double: plain FP64 path.  T = float: mixed path (FP32 matrices, fields and CG vectors;
// every inner product, norm and volume average accumulated in FP64).
template <typename T>
cudaError_t launch_wsum(const Launch& L, const DSeg& G, int nc, const T* f, int64_t cs,
                        int64_t ns, const int64_t* perm, const double* w, double* out,
                        const double* add, Red red);  // out[seg * nc + c]
template <typename T>
cudaError_t launch_spmv(const Launch& L, const DSell& A, const T* val, int B, const T* x,
                        T* y, int variant = 0, int diff = 0);  // B = 1 scalar, B = 9 block
// (x, y AoS 3); diff != 0: the operator's rows sum to zero (K^ms, K^mech) and each row is
// formed as sum_j A_ij (x_j - x_i)
// CG pieces.  st and the arrival counters are per segment; nactive counts active segments.
// epr = elements per row of the vectors (1: scalar, SoA with stride ld; 3: [n][3]).
// bmean != NULL: solve the consistent singular system with b projected off the constants
// (bmean = per-segment mean of each component) by CG projected off the constants: r.r is taken
// without r's constant part, and every search direction has its mean removed (the p-update
// subtracts st.sub; after init, launch_cg_psub does it for p0).  In exact arithmetic these
// means are zero (K 1 = 0); with K rounded to FP32 K 1 is not, and without the projection the
// iteration would chase the constants, along which K has no curvature.
// pinned: the pinned system (Sec. 2.5).
template <typename T>
cudaError_t launch_cg_init(const Launch& L, const DSell& A, const DSeg& G, const T* val, int B,
                           const T* b, const T* x, T* r, T* p, CGState* st, int* nactive, double rtol,
                           int max_iter, Red red, const double* bmean, int pinned, int pc);
// dinv != NULL: Jacobi-preconditioned CG (p = z = D^-1 r, fused into update and p-update)
// ||b - A x||^2 and ||b||^2 per segment over the rows but the pinned one, A x accumulated in
// FP64 (B = 1: K^ms, x and b [n]; B = 9: K^mech, [n][3]): out[2 seg], out[2 seg + 1]
template <typename T>
cudaError_t launch_true_res(const Launch& L, const DSell& A, const DSeg& G, const T* val, int B,
                            const T* b, const T* x, const T* xlo, Red red, double* out);
// (hi, lo) <- hi + dx (TwoSum, lo zero on entry), len elements: the refined solutions of the
// mixed path are unevaluated sums hi + lo
template <typename T>
cudaError_t launch_refine_add(const Launch& L, int64_t len, T* hi, T* lo, const T* dx);
template <typename T>
cudaError_t launch_cg_init_gs(const Launch& L, const DSell& A, const DSeg& G, const T* aval,
                              const T* mval, int nr, int64_t ld, T* x, T* r, T* p, CGState* st,
                              int* nactive, double rtol, int max_iter, Red red, const T* dinv);
template <typename T>
cudaError_t launch_cg_spmv(const Launch& L, const DSell& A, const DSeg& G, const T* val, int B,
                           int nr, int64_t ld, const T* p, T* q, CGState* st, Red red,
                           int variant, int pinned, int diff);
// x(i, c) -= x(pin of i's segment, c) for x[i * epr + c]; xp: nseg * epr doubles of scratch
template <typename T>
cudaError_t launch_pin_shift(const Launch& L, const DSell& A, const DSeg& G, int epr, T* x,
                             double* xp);
// x(i, c) -= xs[seg * epr + c] over each segment's rows
template <typename T>
cudaError_t launch_seg_shift(const Launch& L, const DSell& A, const DSeg& G, int epr, T* x,
                             const double* xs);
// p(i, c) -= st[seg].sub[c] for the active segments that run the projected CG
template <typename T>
cudaError_t launch_cg_psub(const Launch& L, const DSell& A, const DSeg& G, int epr, T* p,
                           const CGState* st);
template <typename T>
cudaError_t launch_cg_update(const Launch& L, const DSeg& G, int epr, int nr, int64_t ld, T* x,
                             T* r, const T* p, const T* q, CGState* st, int* nactive, Red red,
                             const T* dinv = nullptr);
template <typename T>
cudaError_t launch_cg_pupdate(const Launch& L, const DSeg& G, int epr, int nr, int64_t ld,
                              const T* r, T* p, const CGState* st, const LoopCtl& lc,
                              const T* dinv = nullptr);
// Two-level preconditioner z = D^-1 r + P A_c^-1 P^T r (one right-hand side, epr components):
// rc = P^T r (per aggregate sums), ec = A_c^-1 rc (per segment dense block), then z and r.z;
// the segment's last item stores rz (init) or beta = r.z / rz_old and rz.
// rc layout: segment s's block starts at rc_off[s] and is zero-padded to coarse_ld(nc) values
// (whole tiles); ec is indexed by the global coarse index.
template <typename T>
cudaError_t launch_restrict(const Launch& L, const DCoarse& C, int epr, const T* r,
                            const int64_t* rc_off, T* rc);
// Storage of the dense coarse inverse: bfloat16 bits (uint16_t) under FP32 arithmetic, the
// arithmetic type otherwise.  The inverse only applies the preconditioner: any fixed symmetric
// positive definite rounding of it leaves the CG's solution unchanged.  It is symmetric, so
// only its upper triangle is stored, as square tiles (I <= J) of each segment's block
// (zero-padded to whole tiles), row-major within a tile, tile rows one after another: tile
// (I, J) of a segment with T tile rows is its tile number I T - I (I - 1) / 2 + (J - I).  The
// tile side (coarse_tile: 128 for BF16, 64 for FP64) makes a row of a tile 16 or 32 lanes of
// 16-byte packs.
template <typename T> struct CoarseStore { using type = T; };
template <> struct CoarseStore<float> { using type = uint16_t; };
template <typename T>
__host__ __device__ constexpr int coarse_tile() {
  return sizeof(typename CoarseStore<T>::type) == 2 ? 128 : 64;
}
template <typename T>
inline int64_t coarse_ld(int64_t nc) {
  return (nc + coarse_tile<T>() - 1) / coarse_tile<T>() * coarse_tile<T>();
}
// The stored tiles of all segments: tile t of the global list belongs to segment tseg[t], tile
// row tI[t], column tJ[t]; segment s's tiles start at seg_tile0[s] and it has seg_T[s] tile rows.
// The partials of segment s sit in Q at seg_q0[s], one row of seg_T[s] values per (padded)
// coarse row of the segment.
struct DSymTiles {
  int64_t ntiles;
  const int32_t* tseg;
  const int32_t* tI;
  const int32_t* tJ;
  const int64_t* seg_tile0;
  const int32_t* seg_T;
  const int64_t* seg_q0;
};
// ec = A_c^-1 rc with the stored upper triangle, in two kernels: each tile (I, J) writes the
// partial products A_IJ rc_J to Q(row I tile + r, J) and, off the diagonal, A_IJ^T rc_I to
// Q(row J tile + c, I) (every stored value read once); then each coarse row sums its row of Q
// in column order.  Q: scratch of sum over segments of T^2 tile values.
template <typename T>
cudaError_t launch_coarse_symv(const Launch& L, const DCoarse& C, const DSymTiles& TL, int epr,
                               const typename CoarseStore<T>::type* inv, const int64_t* rc_off,
                               const T* rc, T* Q, T* ec);
template <typename T>
cudaError_t launch_pcg_z(const Launch& L, const DSeg& G, const DCoarse& C, int epr, const T* r,
                         const T* dinv, const T* ec, T* z, CGState* st, int init, Red red);
// Graph loops: reset the iteration count and set the WHILE condition to (nactive > 0).
cudaError_t launch_loop_start(const Launch& L, const LoopCtl& lc);
// Add one solve's iterations (kind 0 K^ms, 1 K^mech: the largest over right-hand sides;
// 2 GS: their sum) and non-converged count to acc[4 * seg + kind] and acc[4 * seg + 3].
cudaError_t launch_solve_stats(const Launch& L, const CGState* st, int nseg, int kind,
                               long long* acc);
template <typename T>
cudaError_t launch_cg_zero(const Launch& L, const DSeg& G, int epr, T* x, const CGState* st);

template <typename T>
cudaError_t launch_fdiv(const Launch& L, const DSell& A, const DSeg& G, const T* Fv, const T* m,
                        int64_t ld, T* b, int pin_zero);
template <typename T>
cudaError_t launch_fgrad(const Launch& L, const DSell& A, const T* Fv, const T* U, const T* Ulo,
                         const double* invML, T* hd, int64_t ld);
template <typename T>
cudaError_t launch_fstrain(const Launch& L, const DSell& A, const DSeg& G, const T* Fv,
                           const T* u, const T* ulo, const double* invML, const double* Ebar,
                           T* E, int64_t ld);
template <typename T>
cudaError_t launch_gdiv(const Launch& L, const DSell& A, const DSeg& G, const T* Gv,
                        const T* sig0, T* b, int pin_zero);
template <typename T>
cudaError_t launch_e0(const Launch& L, int64_t n, const T* m, int64_t ld, const uint8_t* mag,
                      const DevParams& P, T* E0, T* sig0);
// h(m) = h_anis + H/ms + h_me(m, C(E - E0(m))) + hd - Nd mbar at magnetic nodes, 0 elsewhere
// (mbar, hz per segment).  mode 0: write h (SoA 3).  mode 1: write x_c = m_c + coef * h_c.
template <typename T>
cudaError_t launch_hfield(const Launch& L, int64_t n, const DSeg& G, const T* m, const T* hd,
                          const T* E, int64_t ld, const double* mbar, const double* hz,
                          const uint8_t* mag, const DevParams& P, int mode, double coef, T* h,
                          T* x);
// GSPM Gauss-Seidel pieces (Algorithm B.1 step 2); see the driver for the stage layout.
template <typename T>
cudaError_t launch_gs_prep(const Launch& L, int64_t n, int64_t ld, const T* m, const T* h,
                           double dtau, int c0, int nc, T* x);
template <typename T>
cudaError_t launch_gs_stage(const Launch& L, int64_t n, int64_t ld, int stage, int printed,
                            const T* m, const T* h, double dtau, T* x, T* ms);
template <typename T>
cudaError_t launch_project(const Launch& L, const DSeg& G, int64_t ld, const T* x,
                           const uint8_t* mag, T* m, double* dm_out, const double* inv_nmag,
                           Red red, int* bad);  // dm_out[seg]; bad[seg] += non-finite or zero m**

template <typename T>
cudaError_t launch_import(const Launch& L, int64_t n, int nc, const double* src,
                          const int64_t* perm, T* dst, int64_t cs, int64_t ns,
                          const uint8_t* mask, T* lo = nullptr);
template <typename T>
cudaError_t launch_export(const Launch& L, int64_t n, int nc, const T* src, int64_t cs,
                          int64_t ns, const int64_t* perm, double* dst, const T* lo = nullptr);
template <typename S, typename D>
cudaError_t launch_convert(const Launch& L, int64_t len, const S* src, D* dst);
template <typename T>
cudaError_t launch_extrapolate(const Launch& L, int64_t len, T* u, T* u2);
template <typename T>
cudaError_t launch_scaled_diff(const Launch& L, int64_t len, const T* a, const T* b, const T* c,
                               double scale, float* t);

}  // namespace gspm
