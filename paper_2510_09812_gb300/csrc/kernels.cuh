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

// Scratch for deterministic grid reductions: one partial per block and component, plus the
// arrival counter of the last-block pattern (reset to 0 by the last block).
struct Red {
  double* partial;     // [max_blocks * kRedComp]
  unsigned* counter;
};
constexpr int kRedComp = 16;
constexpr int kBlock = 256;

// Per-solve CG scalars, device resident.  One entry per right-hand side (up to 3).
struct CGRhs {
  double bb, rr, pq, alpha, beta, tol2;
  int iters, done;
};
struct CGState {
  CGRhs r[3];
  int nr, active, max_iter, noconv, zero_x, pad[3];
};

// Material constants needed on the device (reduced units of App. B).
struct DevParams {
  double kappa, me_coef, l100, l111, C11, C12, C44;
  double hz[3];   // H_ext / m_s
  double Nd[9];
  double dtau, alpha;
};

struct Launch {
  cudaStream_t stream;
  int max_blocks;        // resident-block cap used for grid-stride kernels
  int64_t* counter;      // kernel launches issued
  int blocks_for(int64_t threads) const {
    int64_t b = (threads + kBlock - 1) / kBlock;
    if (b > max_blocks) b = max_blocks;
    return b < 1 ? 1 : (int)b;
  }
};

// ---- launchers (T = double: plain FP64 path; T = float: mixed path) --------------------------
template <typename T> struct Types {
  using V = T;       // matrix values
  using F = T;       // nodal fields m, h, h_d, E, E0, sigma0
  using XP = T;      // CG search direction p and q = A p
  using XR = double; // CG iterate x, residual r
};

template <typename T>
cudaError_t launch_wsum(const Launch& L, int64_t n, int nc, const T* f, int64_t cs, int64_t ns,
                        const int64_t* perm, const double* w, double* out, const double* add,
                        Red red);
template <typename T>
cudaError_t launch_spmv(const Launch& L, const DSell& A, const T* val, int B, const T* x,
                        T* y);  // B = 1 scalar, B = 9 block (x, y AoS 3)
template <typename T>
cudaError_t launch_cg_init(const Launch& L, const DSell& A, const T* val, int B, const double* b,
                           double* x, double* r, T* p, CGState* st, double rtol, int max_iter,
                           Red red);
template <typename T>
cudaError_t launch_cg_init_gs(const Launch& L, const DSell& A, const T* aval, const T* mval,
                              int nr, int64_t ld, double* x, double* r, T* p, CGState* st,
                              double rtol, int max_iter, Red red);
template <typename T>
cudaError_t launch_cg_spmv(const Launch& L, const DSell& A, const T* val, int B, int nr,
                           int64_t ld, const T* p, T* q, CGState* st, Red red);
template <typename T>
cudaError_t launch_cg_update(const Launch& L, int64_t len, int nr, int64_t ld, double* x,
                             double* r, const T* p, const T* q, CGState* st, Red red);
template <typename T>
cudaError_t launch_cg_pupdate(const Launch& L, int64_t len, int nr, int64_t ld, const double* r,
                              T* p, const CGState* st);
cudaError_t launch_cg_zero(const Launch& L, int64_t len, double* x, const CGState* st);

template <typename T>
cudaError_t launch_fdiv(const Launch& L, const DSell& A, const T* Fv, const T* m, int64_t ld,
                        double* b, int64_t pin);
template <typename T>
cudaError_t launch_fgrad(const Launch& L, const DSell& A, const T* Fv, const double* U,
                         const double* invML, T* hd, int64_t ld);
template <typename T>
cudaError_t launch_fstrain(const Launch& L, const DSell& A, const T* Fv, const double* u,
                           const double* invML, const double* Ebar, T* E, int64_t ld);
template <typename T>
cudaError_t launch_gdiv(const Launch& L, const DSell& A, const T* Gv, const T* sig0, double* b,
                        int64_t pin);
template <typename T>
cudaError_t launch_e0(const Launch& L, int64_t n, const T* m, int64_t ld, const uint8_t* mag,
                      const DevParams& P, T* E0, T* sig0);
// h(m) = h_anis + H/ms + h_me(m, C(E - E0(m))) + hd - Nd mbar at magnetic nodes, 0 elsewhere.
// mode 0: write h (SoA 3).  mode 1: write x_c = m_c + coef * h_c (double SoA 3).
template <typename T>
cudaError_t launch_hfield(const Launch& L, int64_t n, const T* m, const T* hd, const T* E,
                          int64_t ld, const double* mbar, const uint8_t* mag, const DevParams& P,
                          int mode, double coef, T* h, double* x);
// GSPM Gauss-Seidel pieces (Algorithm B.1 step 2); see the driver for the stage layout.
template <typename T>
cudaError_t launch_gs_prep(const Launch& L, int64_t n, int64_t ld, const T* m, const T* h,
                           double dtau, int c0, int nc, double* x);
template <typename T>
cudaError_t launch_gs_stage(const Launch& L, int64_t n, int64_t ld, int stage, int printed,
                            const T* m, const T* h, double dtau, double* x, T* ms);
template <typename T>
cudaError_t launch_project(const Launch& L, int64_t n, int64_t ld, const double* x,
                           const uint8_t* mag, T* m, double* dm_out, double inv_nmag, Red red);

template <typename T>
cudaError_t launch_import(const Launch& L, int64_t n, int nc, const double* src,
                          const int64_t* perm, T* dst, int64_t cs, int64_t ns,
                          const uint8_t* mask);
template <typename T>
cudaError_t launch_export(const Launch& L, int64_t n, int nc, const T* src, int64_t cs,
                          int64_t ns, const int64_t* perm, double* dst);
template <typename S, typename D>
cudaError_t launch_convert(const Launch& L, int64_t len, const S* src, D* dst);

}  // namespace gspm
