// C ABI and step driver of the GSPM library.  The host only sequences kernels on the context's
// stream; every arithmetic step of the method runs on the device.  CG loops keep their scalars on
// the device and the host reads one small status block per check (after the number of
// iterations the previous solve of the same kind needed), so no per-iteration round trip.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <type_traits>
#include <string>
#include <vector>

#include "internal.h"
#include "kernels.cuh"

namespace gspm {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

#define CK(call)                                                                  \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
      return GSPM_ECUDA;                                                          \
    }                                                                             \
  } while (0)

#define ST(call)                 \
  do {                           \
    int s_ = (call);             \
    if (s_ != GSPM_OK) return s_; \
  } while (0)

// launch with optional event timing of its kernel class
#define TK(cls, call) ST(timed((cls), [&]() -> int { CK(call); return GSPM_OK; }))

// device allocation with accounting
struct DevMem {
  std::vector<void*> ptrs;
  int64_t bytes = 0;
  ~DevMem() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename X>
  int alloc(X** out, int64_t count) {
    void* p = nullptr;
    const size_t sz = (size_t)std::max<int64_t>(count, 1) * sizeof(X);
    cudaError_t e = cudaMalloc(&p, sz);
    if (e != cudaSuccess) {
      set_error("cudaMalloc(%zu bytes): %s", sz, cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? GSPM_ENOMEM : GSPM_ECUDA;
    }
    ptrs.push_back(p);
    bytes += (int64_t)sz;
    *out = (X*)p;
    return GSPM_OK;
  }
};

struct SolveInfo {
  int iters = 0;
  double relres = 0.0;
  int noconv = 0;
};

class EngineBase {
 public:
  virtual ~EngineBase() = default;
  virtual int step(int n_steps, const double H[3], gspm_step_stats* st) = 0;
  virtual int solve_elastic(const double* m, double* u, int where, int x0_mode, const double* x0,
                            double rtol, int* iters, double* relres) = 0;
  virtual int volume_avg(const double* f, int where, int nc, double* out) = 0;
  virtual int apply(int op, const double* x, double* y, int where) = 0;
  virtual int set_field(int field, const double* data, int where) = 0;
  virtual int get_field(int field, double* data, int where) = 0;
  virtual int64_t device_bytes() const = 0;
  virtual int profile_enable(unsigned mask) = 0;
  virtual int profile_read(int cls, double* ms, int64_t* launches) = 0;
};

template <typename T>
class Engine final : public EngineBase {
 public:
  Engine(const HostMesh& hm, const HostSell& hs, const HostOps& ops, const Params& P,
         const gspm_options& opt, cudaStream_t stream, int64_t* counter)
      : hm_(hm), P_(P), opt_(opt) {
    n_ = hm.n;
    ld_ = (n_ + 31) / 32 * 32;
    nslices_ = hs.nslices;
    entries_ = hs.entries;
    pin_ = ops.pin;
    nmag_ = hm.n_mag_nodes;
    L_.stream = stream;
    L_.counter = counter;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    L_.max_blocks = std::max(1, sms) * 8;
  }
  ~Engine() override {
    if (host_state_) cudaFreeHost(host_state_);
    for (cudaEvent_t e : prof_ev_) cudaEventDestroy(e);
  }

  int init(const HostSell& hs, const HostOps& ops) {
    const int64_t n = n_, ld = ld_, E = entries_;
    ST(mem_.alloc(&sptr_, nslices_ + 1));
    ST(mem_.alloc(&slen_, nslices_));
    ST(mem_.alloc(&col_, E));
    CK(cudaMemcpy(sptr_, hs.sptr.data(), (nslices_ + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(slen_, hs.slen.data(), nslices_ * sizeof(int32_t), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(col_, hs.col.data(), E * sizeof(int32_t), cudaMemcpyHostToDevice));
    A_ = DSell{sptr_, slen_, col_, nslices_, n};
    ST(upload(&Kms_, ops.Kms));
    ST(upload(&Aeps_, ops.Aeps));
    ST(upload(&Aaeps_, ops.Aaeps));
    ST(upload(&M_, ops.M));
    ST(upload(&F_, ops.F));
    ST(upload(&G_, ops.G));
    ST(upload(&Kmech_, ops.Kmech));
    ST(mem_.alloc(&invML_, n));
    ST(mem_.alloc(&w_, n));
    ST(mem_.alloc(&mag_, n));
    ST(mem_.alloc(&perm_, n));
    CK(cudaMemcpy(invML_, ops.invML.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(w_, ops.w.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(mag_, ops.mag.data(), n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(perm_, hm_.perm.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice));
    ST(mem_.alloc(&m_, 3 * ld));
    ST(mem_.alloc(&ms_, 3 * ld));
    ST(mem_.alloc(&h_, 3 * ld));
    ST(mem_.alloc(&hd_, 3 * ld));
    ST(mem_.alloc(&E_, 6 * ld));
    ST(mem_.alloc(&E0_, 6 * ld));
    ST(mem_.alloc(&sig0_, 6 * n));
    ST(mem_.alloc(&U_, ld));
    ST(mem_.alloc(&u_, 3 * n));
    ST(mem_.alloc(&b_, 3 * ld));
    ST(mem_.alloc(&r_, 3 * ld));
    ST(mem_.alloc(&x_, 3 * ld));
    ST(mem_.alloc(&p_, 3 * ld));
    ST(mem_.alloc(&q_, 3 * ld));
    ST(mem_.alloc(&stage_, 9 * n));
    ST(mem_.alloc(&tin_, 3 * ld));
    ST(mem_.alloc(&tout_, 3 * ld));
    ST(mem_.alloc(&cg_, kSolveSlots));
    ST(mem_.alloc(&scal_, 32));
    ST(mem_.alloc(&red_.partial, (int64_t)L_.max_blocks * kRedComp));
    ST(mem_.alloc(&red_.counter, 1));
    CK(cudaMemset(red_.counter, 0, sizeof(unsigned)));
    CK(cudaMemset(scal_, 0, 32 * sizeof(double)));
    CK(cudaMemset(m_, 0, 3 * ld * sizeof(T)));
    CK(cudaMemset(ms_, 0, 3 * ld * sizeof(T)));
    CK(cudaMemset(h_, 0, 3 * ld * sizeof(T)));
    CK(cudaMemset(hd_, 0, 3 * ld * sizeof(T)));
    CK(cudaMemset(E_, 0, 6 * ld * sizeof(T)));
    CK(cudaMemset(U_, 0, ld * sizeof(double)));
    CK(cudaMemset(u_, 0, 3 * n * sizeof(double)));
    CK(cudaMemset(x_, 0, 3 * ld * sizeof(double)));
    CK(cudaMemset(p_, 0, 3 * ld * sizeof(T)));
    CK(cudaMemset(q_, 0, 3 * ld * sizeof(T)));
    CK(cudaMemset(cg_, 0, kSolveSlots * sizeof(CGState)));
    // E_ext (added to <E0> when forming E_bar)
    CK(cudaMemcpy(scal_ + kEext, P_.E_ext, 6 * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMallocHost(&host_state_, sizeof(CGState)));
    for (int k = 0; k < kSolveSlots; ++k) pred_[k] = 8;
    CK(cudaDeviceSynchronize());
    return GSPM_OK;
  }

  int64_t device_bytes() const override { return mem_.bytes; }

  int profile_enable(unsigned mask) override {
    CK(cudaStreamSynchronize(L_.stream));
    prof_mask_ = mask;
    prof_used_ = 0;
    return GSPM_OK;
  }

  int profile_read(int cls, double* ms, int64_t* launches) override {
    if (cls < 0 || cls >= GSPM_KCLASS_COUNT) {
      set_error("profile_read: bad class %d", cls);
      return GSPM_EINVAL;
    }
    CK(cudaStreamSynchronize(L_.stream));
    double tot = 0.0;
    int64_t cnt = 0;
    for (size_t k = 0; k < prof_used_; ++k) {
      if (prof_cls_[k] != cls) continue;
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, prof_ev_[2 * k], prof_ev_[2 * k + 1]));
      tot += t;
      ++cnt;
    }
    if (ms) *ms = tot;
    if (launches) *launches = cnt;
    return GSPM_OK;
  }

  // ---------------------------------------------------------------- one GSPM step
  int step(int n_steps, const double H[3], gspm_step_stats* st) override {
    DevParams D = dev_params(H);
    gspm_step_stats acc;
    memset(&acc, 0, sizeof(acc));
    const int64_t n = n_, ld = ld_;
    double* mbar = scal_ + kMbar;
    double* mbar_s = scal_ + kMbarS;
    double* Ebar = scal_ + kEbar;
    double* dm = scal_ + kDm;
    const int printed = (opt_.flags & GSPM_FLAG_ROW2_PRINTED) ? 1 : 0;
    for (int s = 0; s < n_steps; ++s) {
      // a1 volume average of m (Sec. 2.4)
      TK(GSPM_KCLASS_POINTWISE, launch_wsum<T>(L_, n, 3, m_, ld, 1, nullptr, w_, mbar, nullptr, red_));
      // a2 b^ms / m_s = F^ms m (Eq. RHS_b), a3 CG on pinned K^ms, x0 = previous U
      TK(GSPM_KCLASS_ROWOPS, launch_fdiv<T>(L_, A_, F_, m_, ld, b_, pin_));
      SolveInfo ims;
      ST(solve_general(kSlotMs, Kms_, 1, b_, U_, n, opt_.rtol_ms, &ims));
      // a4 local demagnetising field h~_d = -grad U
      TK(GSPM_KCLASS_ROWOPS, launch_fgrad<T>(L_, A_, F_, U_, invML_, hd_, ld));
      // a5 E0(m), sigma0 = C E0, E_bar = <E0> + C^-1 sigma_ext
      TK(GSPM_KCLASS_POINTWISE, launch_e0<T>(L_, n, m_, ld, mag_, D, E0_, sig0_));
      TK(GSPM_KCLASS_POINTWISE, launch_wsum<T>(L_, n, 6, E0_, ld, 1, nullptr, w_, Ebar, scal_ + kEext, red_));
      // a6 b^mech = F^mech E0, a7 CG on pinned K^mech, x0 = previous u
      TK(GSPM_KCLASS_ROWOPS, launch_gdiv<T>(L_, A_, G_, sig0_, b_, pin_));
      SolveInfo imech;
      ST(solve_general(kSlotMech, Kmech_, 9, b_, u_, 3 * n, opt_.rtol_mech, &imech));
      // a8 strain E = E_bar + sym grad u
      TK(GSPM_KCLASS_ROWOPS, launch_fstrain<T>(L_, A_, F_, u_, invML_, Ebar, E_, ld));
      // a9 h(m^n)
      TK(GSPM_KCLASS_POINTWISE, launch_hfield<T>(L_, n, m_, hd_, E_, ld, mbar, mag_, D, 0, 0.0, h_, nullptr));
      // a10 Gauss-Seidel stages (Algorithm B.1 steps 1-2), (M + eps K) g = M f, x0 = f
      SolveInfo ig[8];
      int ngs = 0;
      if (!printed) {
        TK(GSPM_KCLASS_POINTWISE, launch_gs_prep<T>(L_, n, ld, m_, h_, P_.dtau, 1, 2, x_));
        ST(solve_gs(kSlotGs0, Aeps_, 0, 2, &ig[0]));
        TK(GSPM_KCLASS_POINTWISE, launch_gs_stage<T>(L_, n, ld, 1, 0, m_, h_, P_.dtau, x_, ms_));
        ST(solve_gs(kSlotGs1, Aeps_, 2, 1, &ig[2]));
        TK(GSPM_KCLASS_POINTWISE, launch_gs_stage<T>(L_, n, ld, 2, 0, m_, h_, P_.dtau, x_, ms_));
        ST(solve_gs(kSlotGs2, Aeps_, 0, 1, &ig[3]));
        TK(GSPM_KCLASS_POINTWISE, launch_gs_stage<T>(L_, n, ld, 3, 0, m_, h_, P_.dtau, x_, ms_));
        ngs = 4;
      } else {
        TK(GSPM_KCLASS_POINTWISE, launch_gs_prep<T>(L_, n, ld, m_, h_, P_.dtau, 0, 3, x_));
        ST(solve_gs(kSlotGs0, Aeps_, 0, 3, &ig[0]));
        TK(GSPM_KCLASS_POINTWISE, launch_gs_stage<T>(L_, n, ld, 1, 1, m_, h_, P_.dtau, x_, ms_));
        ST(solve_gs(kSlotGs1, Aeps_, 0, 2, &ig[3]));
        TK(GSPM_KCLASS_POINTWISE, launch_gs_stage<T>(L_, n, ld, 3, 1, m_, h_, P_.dtau, x_, ms_));
        ngs = 5;
      }
      // a11 h(m*) with h~_d and E held, far field from m_bar*; f = m* + alpha dtau h*
      TK(GSPM_KCLASS_POINTWISE, launch_wsum<T>(L_, n, 3, ms_, ld, 1, nullptr, w_, mbar_s, nullptr, red_));
      TK(GSPM_KCLASS_POINTWISE, launch_hfield<T>(L_, n, ms_, hd_, E_, ld, mbar_s, mag_, D, 1, P_.alpha * P_.dtau,
                          nullptr, x_));
      // a12 (M + alpha eps K) m** = M f, three right-hand sides
      ST(solve_gs(kSlotGsD, Aaeps_, 0, 3, &ig[ngs]));
      ngs += 3;
      // a13 projection and <|dm|>
      TK(GSPM_KCLASS_POINTWISE, launch_project<T>(L_, n, ld, x_, mag_, m_, dm,
                           nmag_ > 0 ? 1.0 / (double)nmag_ : 0.0, red_));
      acc.steps += 1;
      acc.it_ms += ims.iters;
      acc.it_mech += imech.iters;
      acc.it_ms_last = ims.iters;
      acc.it_mech_last = imech.iters;
      acc.res_ms_last = ims.relres;
      acc.res_mech_last = imech.relres;
      acc.noconv += ims.noconv + imech.noconv;
      for (int k = 0; k < 8; ++k) {
        acc.it_gs_last[k] = k < ngs ? ig[k].iters : 0;
        if (k < ngs) {
          acc.it_gs += ig[k].iters;
          acc.noconv += ig[k].noconv;
        }
      }
    }
    if (st) {
      double hs[4];
      CK(cudaMemcpyAsync(hs, scal_ + kMbar, 3 * sizeof(double), cudaMemcpyDeviceToHost, L_.stream));
      CK(cudaMemcpyAsync(hs + 3, dm, sizeof(double), cudaMemcpyDeviceToHost, L_.stream));
      CK(cudaStreamSynchronize(L_.stream));
      acc.m_bar[0] = hs[0];
      acc.m_bar[1] = hs[1];
      acc.m_bar[2] = hs[2];
      acc.dm_last = hs[3];
      *st = acc;
    }
    CK(cudaGetLastError());
    return acc.noconv ? GSPM_ENOCONV : GSPM_OK;
  }

  int solve_elastic(const double* m, double* u, int where, int x0_mode, const double* x0,
                    double rtol, int* iters, double* relres) override {
    const int64_t n = n_, ld = ld_;
    if (!m) {
      set_error("solve_elastic: m is NULL");
      return GSPM_EINVAL;
    }
    DevParams D = dev_params(nullptr);
    // magnetisation into the m* buffer (the context's m is left alone)
    ST(import_field(m, where, 3, ms_, ld, 1, mag_));
    if (x0_mode == 0) {
      CK(cudaMemsetAsync(u_, 0, 3 * n * sizeof(double), L_.stream));
    } else if (x0_mode == 2) {
      if (!x0) {
        set_error("solve_elastic: x0_mode 2 needs x0");
        return GSPM_EINVAL;
      }
      ST(import_field(x0, where, 3, u_, 1, 3, nullptr));
    } else if (x0_mode != 1) {
      set_error("solve_elastic: bad x0_mode %d", x0_mode);
      return GSPM_EINVAL;
    }
    TK(GSPM_KCLASS_POINTWISE, launch_e0<T>(L_, n, ms_, ld, mag_, D, E0_, sig0_));
    TK(GSPM_KCLASS_POINTWISE, launch_wsum<T>(L_, n, 6, E0_, ld, 1, nullptr, w_, scal_ + kEbar, scal_ + kEext, red_));
    TK(GSPM_KCLASS_ROWOPS, launch_gdiv<T>(L_, A_, G_, sig0_, b_, pin_));
    SolveInfo info;
    ST(solve_general(kSlotMech, Kmech_, 9, b_, u_, 3 * n,
                     rtol > 0 ? rtol : opt_.rtol_mech, &info));
    TK(GSPM_KCLASS_ROWOPS, launch_fstrain<T>(L_, A_, F_, u_, invML_, scal_ + kEbar, E_, ld));
    if (u) ST(export_field(u_, 1, 3, 3, u, where));
    CK(cudaStreamSynchronize(L_.stream));
    if (iters) *iters = info.iters;
    if (relres) *relres = info.relres;
    return info.noconv ? GSPM_ENOCONV : GSPM_OK;
  }

  int volume_avg(const double* f, int where, int nc, double* out) override {
    if (nc < 1 || nc > 9 || !f || !out) {
      set_error("volume_avg: need 1 <= ncomp <= 9 and non-null pointers");
      return GSPM_EINVAL;
    }
    const double* src = f;
    if (where == GSPM_HOST) {
      CK(cudaMemcpyAsync(stage_, f, n_ * nc * sizeof(double), cudaMemcpyHostToDevice, L_.stream));
      src = stage_;
    }
    CK(launch_wsum<double>(L_, n_, nc, src, 1, nc, perm_, w_, scal_ + kAvg, nullptr, red_));
    CK(cudaMemcpyAsync(out, scal_ + kAvg, nc * sizeof(double), cudaMemcpyDeviceToHost, L_.stream));
    CK(cudaStreamSynchronize(L_.stream));
    return GSPM_OK;
  }

  int apply(int op, const double* x, double* y, int where) override {
    const int64_t ld = ld_;
    if (!x || !y) {
      set_error("apply: null pointer");
      return GSPM_EINVAL;
    }
    switch (op) {
      case GSPM_OP_K_MS: case GSPM_OP_A_EPS: case GSPM_OP_A_AEPS: case GSPM_OP_M: {
        const T* val = op == GSPM_OP_K_MS ? Kms_ : op == GSPM_OP_A_EPS ? Aeps_
                     : op == GSPM_OP_A_AEPS ? Aaeps_ : M_;
        ST(import_field(x, where, 1, tin_, 1, 1, nullptr));
        CK(launch_spmv<T>(L_, A_, val, 1, tin_, tout_));
        ST(export_field(tout_, 1, 1, 1, y, where));
        break;
      }
      case GSPM_OP_K_MECH:
        ST(import_field(x, where, 3, tin_, 1, 3, nullptr));
        CK(launch_spmv<T>(L_, A_, Kmech_, 9, tin_, tout_));
        ST(export_field(tout_, 1, 3, 3, y, where));
        break;
      case GSPM_OP_DIV:
        ST(import_field(x, where, 3, tin_, ld, 1, nullptr));
        CK(launch_fdiv<T>(L_, A_, F_, tin_, ld, b_, pin_));
        ST(export_field(b_, 1, 1, 1, y, where));
        break;
      case GSPM_OP_GRAD:
        ST(import_field(x, where, 1, r_, 1, 1, nullptr));
        CK(launch_fgrad<T>(L_, A_, F_, r_, invML_, tout_, ld));
        ST(export_field(tout_, ld, 1, 3, y, where));
        break;
      default:
        set_error("apply: unknown operator %d", op);
        return GSPM_EINVAL;
    }
    if (where == GSPM_HOST) CK(cudaStreamSynchronize(L_.stream));
    return GSPM_OK;
  }

  int set_field(int field, const double* data, int where) override {
    const int64_t ld = ld_;
    if (!data) {
      set_error("set_field: null pointer");
      return GSPM_EINVAL;
    }
    switch (field) {
      case GSPM_FIELD_M: ST(import_field(data, where, 3, m_, ld, 1, mag_)); break;
      case GSPM_FIELD_U:
        ST(import_field(data, where, 1, U_, 1, 1, nullptr));
        CK(cudaMemsetAsync(U_ + pin_, 0, sizeof(double), L_.stream));
        break;
      case GSPM_FIELD_DISP:
        ST(import_field(data, where, 3, u_, 1, 3, nullptr));
        CK(cudaMemsetAsync(u_ + 3 * pin_, 0, 3 * sizeof(double), L_.stream));
        break;
      default:
        set_error("set_field: field %d is not writable", field);
        return GSPM_EINVAL;
    }
    if (where == GSPM_HOST) CK(cudaStreamSynchronize(L_.stream));
    return GSPM_OK;
  }

  int get_field(int field, double* data, int where) override {
    const int64_t ld = ld_;
    if (!data) {
      set_error("get_field: null pointer");
      return GSPM_EINVAL;
    }
    switch (field) {
      case GSPM_FIELD_M: ST(export_field(m_, ld, 1, 3, data, where)); break;
      case GSPM_FIELD_U: ST(export_field(U_, 1, 1, 1, data, where)); break;
      case GSPM_FIELD_DISP: ST(export_field(u_, 1, 3, 3, data, where)); break;
      case GSPM_FIELD_HD: ST(export_field(hd_, ld, 1, 3, data, where)); break;
      case GSPM_FIELD_STRAIN: ST(export_field(E_, ld, 1, 6, data, where)); break;
      case GSPM_FIELD_H: ST(export_field(h_, ld, 1, 3, data, where)); break;
      default:
        set_error("get_field: unknown field %d", field);
        return GSPM_EINVAL;
    }
    if (where == GSPM_HOST) CK(cudaStreamSynchronize(L_.stream));
    return GSPM_OK;
  }

 private:
  static constexpr int kSlotMs = 0, kSlotMech = 1, kSlotGs0 = 2, kSlotGs1 = 3, kSlotGs2 = 4,
                       kSlotGsD = 5, kSolveSlots = 6;
  static constexpr int kMbar = 0, kMbarS = 3, kEbar = 6, kEext = 12, kDm = 18, kAvg = 20;

  template <typename X>
  int upload(T** dst, const std::vector<X>& src) {
    ST(mem_.alloc(dst, (int64_t)src.size()));
    if (std::is_same<T, X>::value) {
      CK(cudaMemcpy(*dst, src.data(), src.size() * sizeof(X), cudaMemcpyHostToDevice));
    } else {
      std::vector<T> tmp(src.begin(), src.end());
      CK(cudaMemcpy(*dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice));
    }
    return GSPM_OK;
  }

  DevParams dev_params(const double* H) const {
    DevParams D;
    D.kappa = P_.kappa;
    D.me_coef = P_.me_coef;
    D.l100 = P_.l100;
    D.l111 = P_.l111;
    D.C11 = P_.C11;
    D.C12 = P_.C12;
    D.C44 = P_.C44;
    for (int a = 0; a < 3; ++a) D.hz[a] = H ? H[a] / P_.Ms : 0.0;
    for (int k = 0; k < 9; ++k) D.Nd[k] = P_.Nd[k];
    D.dtau = P_.dtau;
    D.alpha = P_.alpha;
    return D;
  }

  // host/device [n][nc] float64 (unique order) -> internal array dst(i, c) = dst[i*ns + c*cs]
  template <typename X>
  int import_field(const double* src, int where, int nc, X* dst, int64_t cs, int64_t ns,
                   const uint8_t* mask) {
    const double* s = src;
    if (where == GSPM_HOST) {
      CK(cudaMemcpyAsync(stage_, src, n_ * nc * sizeof(double), cudaMemcpyHostToDevice, L_.stream));
      s = stage_;
    } else if (where != GSPM_DEVICE) {
      set_error("bad `where` %d", where);
      return GSPM_EINVAL;
    }
    CK(launch_import<X>(L_, n_, nc, s, perm_, dst, cs, ns, mask));
    return GSPM_OK;
  }

  template <typename X>
  int export_field(const X* src, int64_t cs, int64_t ns, int nc, double* dst, int where) {
    if (where == GSPM_DEVICE) {
      CK(launch_export<X>(L_, n_, nc, src, cs, ns, perm_, dst));
    } else if (where == GSPM_HOST) {
      CK(launch_export<X>(L_, n_, nc, src, cs, ns, perm_, stage_));
      CK(cudaMemcpyAsync(dst, stage_, n_ * nc * sizeof(double), cudaMemcpyDeviceToHost, L_.stream));
    } else {
      set_error("bad `where` %d", where);
      return GSPM_EINVAL;
    }
    return GSPM_OK;
  }

  // Launch CG iterations in chunks; after each chunk read the device status block once.
  template <class Iter>
  int cg_loop(int slot, Iter iter, SolveInfo* info) {
    CGState* st = cg_ + slot;
    int chunk = std::max(1, pred_[slot]);
    int launched = 0;
    for (;;) {
      for (int c = 0; c < chunk; ++c) ST(iter());
      launched += chunk;
      CK(cudaMemcpyAsync(host_state_, st, sizeof(CGState), cudaMemcpyDeviceToHost, L_.stream));
      CK(cudaStreamSynchronize(L_.stream));
      if (!host_state_->active || launched > opt_.max_iter + 1) break;
      // first solve of a kind: grow geometrically; afterwards small top-up chunks
      chunk = seen_[slot] ? 3 : std::max(2, std::min(32, launched / 4));
    }
    int it = 0;
    double rel = 0.0;
    for (int k = 0; k < host_state_->nr; ++k) {
      it = std::max(it, host_state_->r[k].iters);
      const double bb = host_state_->r[k].bb;
      rel = std::max(rel, bb > 0 ? std::sqrt(host_state_->r[k].rr / bb) : 0.0);
    }
    pred_[slot] = std::max(1, it);
    seen_[slot] = 1;
    info->iters = it;
    info->relres = rel;
    info->noconv = host_state_->noconv;
    return GSPM_OK;
  }

  // K x = b for the pinned Omega_c systems (B = 1 scalar K^ms, B = 9 block K^mech)
  int solve_general(int slot, const T* val, int B, const double* b, double* x, int64_t len,
                    double rtol, SolveInfo* info) {
    CGState* st = cg_ + slot;
    TK(GSPM_KCLASS_CG_INIT, launch_cg_init<T>(L_, A_, val, B, b, x, r_, p_, st, rtol, opt_.max_iter, red_));
    auto iter = [&]() -> int {
      TK(B == 9 ? GSPM_KCLASS_SPMV_MECH : GSPM_KCLASS_SPMV_MS, launch_cg_spmv<T>(L_, A_, val, B, 1, len, p_, q_, st, red_));
      TK(GSPM_KCLASS_CG_VEC, launch_cg_update<T>(L_, len, 1, len, x, r_, p_, q_, st, red_));
      TK(GSPM_KCLASS_CG_VEC, launch_cg_pupdate<T>(L_, len, 1, len, r_, p_, st));
      return GSPM_OK;
    };
    ST(cg_loop(slot, iter, info));
    TK(GSPM_KCLASS_CG_INIT, launch_cg_zero(L_, len, x, st));
    return GSPM_OK;
  }

  // (M + c eps K) g = M f for nr right-hand sides held in x slots [slot0, slot0 + nr)
  int solve_gs(int slot, const T* aval, int slot0, int nr, SolveInfo* info) {
    CGState* st = cg_ + slot;
    double* x = x_ + slot0 * ld_;
    TK(GSPM_KCLASS_CG_INIT, launch_cg_init_gs<T>(L_, A_, aval, M_, nr, ld_, x, r_, p_, st, opt_.rtol_gs, opt_.max_iter,
                            red_));
    auto iter = [&]() -> int {
      TK(GSPM_KCLASS_SPMV_GS, launch_cg_spmv<T>(L_, A_, aval, 1, nr, ld_, p_, q_, st, red_));
      TK(GSPM_KCLASS_CG_VEC, launch_cg_update<T>(L_, n_, nr, ld_, x, r_, p_, q_, st, red_));
      TK(GSPM_KCLASS_CG_VEC, launch_cg_pupdate<T>(L_, n_, nr, ld_, r_, p_, st));
      return GSPM_OK;
    };
    SolveInfo tot;
    ST(cg_loop(slot, iter, &tot));
    for (int k = 0; k < nr; ++k) {
      info[k].iters = host_state_->r[k].iters;
      const double bb = host_state_->r[k].bb;
      info[k].relres = bb > 0 ? std::sqrt(host_state_->r[k].rr / bb) : 0.0;
      info[k].noconv = 0;
    }
    info[0].noconv = tot.noconv;
    return GSPM_OK;
  }

  // launch f() bracketed by CUDA events when class cls is being profiled
  template <class Fn>
  int timed(int cls, Fn f) {
    if (!(prof_mask_ & (1u << cls))) return f();
    if (prof_used_ == prof_cls_.size()) {
      cudaEvent_t a, b;
      CK(cudaEventCreate(&a));
      CK(cudaEventCreate(&b));
      prof_ev_.push_back(a);
      prof_ev_.push_back(b);
      prof_cls_.push_back(cls);
    }
    prof_cls_[prof_used_] = cls;
    CK(cudaEventRecord(prof_ev_[2 * prof_used_], L_.stream));
    ST(f());
    CK(cudaEventRecord(prof_ev_[2 * prof_used_ + 1], L_.stream));
    ++prof_used_;
    return GSPM_OK;
  }

  unsigned prof_mask_ = 0;
  size_t prof_used_ = 0;
  std::vector<int> prof_cls_;
  std::vector<cudaEvent_t> prof_ev_;
  const HostMesh& hm_;
  Params P_;
  gspm_options opt_;
  Launch L_;
  DevMem mem_;
  int64_t n_ = 0, ld_ = 0, nslices_ = 0, entries_ = 0, pin_ = 0, nmag_ = 0;
  DSell A_{};
  int64_t* sptr_ = nullptr;
  int32_t* slen_ = nullptr;
  int32_t* col_ = nullptr;
  T *Kms_ = nullptr, *Aeps_ = nullptr, *Aaeps_ = nullptr, *M_ = nullptr, *F_ = nullptr,
    *G_ = nullptr, *Kmech_ = nullptr;
  double *invML_ = nullptr, *w_ = nullptr;
  uint8_t* mag_ = nullptr;
  int64_t* perm_ = nullptr;
  T *m_ = nullptr, *ms_ = nullptr, *h_ = nullptr, *hd_ = nullptr, *E_ = nullptr, *E0_ = nullptr,
    *sig0_ = nullptr, *p_ = nullptr, *q_ = nullptr, *tin_ = nullptr, *tout_ = nullptr;
  double *U_ = nullptr, *u_ = nullptr, *b_ = nullptr, *r_ = nullptr, *x_ = nullptr,
         *stage_ = nullptr, *scal_ = nullptr;
  CGState* cg_ = nullptr;
  CGState* host_state_ = nullptr;
  Red red_{};
  int pred_[kSolveSlots];
  int seen_[kSolveSlots] = {};
};

}  // namespace gspm

using namespace gspm;

struct gspm_ctx {
  HostMesh hm;
  HostSell hs;
  Params P;
  gspm_options opt;
  bool host_only = false;
  int64_t launches = 0;
  std::unique_ptr<EngineBase> eng;
};

extern "C" {

const char* gspm_last_error(void) { return g_err.c_str(); }

int gspm_mesh_load(const gspm_mesh_desc* mesh, const gspm_material* mat,
                   const gspm_options* opt, gspm_ctx** out) {
  if (!mesh || !mat || !opt || !out) {
    set_error("mesh_load: null argument");
    return GSPM_EINVAL;
  }
  *out = nullptr;
  if (opt->precision != GSPM_PREC_F64 && opt->precision != GSPM_PREC_MIXED) {
    set_error("mesh_load: unknown precision %d", opt->precision);
    return GSPM_EINVAL;
  }
  if (opt->max_iter <= 0 || !(opt->rtol_gs > 0) || !(opt->rtol_ms > 0) || !(opt->rtol_mech > 0)) {
    set_error("mesh_load: need max_iter > 0 and positive tolerances");
    return GSPM_EINVAL;
  }
  std::unique_ptr<gspm_ctx> c(new gspm_ctx());
  c->opt = *opt;
  c->host_only = (opt->flags & GSPM_FLAG_HOST_ONLY) != 0;
  ST(make_params(mat, opt, &c->P));
  ST(host_mesh_build(mesh, opt->ordering, &c->hm));
  host_sell_build(c->hm, &c->hs);
  if (!c->host_only) {
    HostOps ops;
    host_assemble(c->hm, c->hs, c->P, &ops);
    cudaStream_t s = (cudaStream_t)opt->stream;
    if (opt->precision == GSPM_PREC_F64) {
      auto e = std::make_unique<Engine<double>>(c->hm, c->hs, ops, c->P, c->opt, s, &c->launches);
      ST(e->init(c->hs, ops));
      c->eng = std::move(e);
    } else {
      auto e = std::make_unique<Engine<float>>(c->hm, c->hs, ops, c->P, c->opt, s, &c->launches);
      ST(e->init(c->hs, ops));
      c->eng = std::move(e);
    }
  }
  *out = c.release();
  return GSPM_OK;
}

void gspm_destroy(gspm_ctx* ctx) {
  if (!ctx) return;
  if (ctx->eng && ctx->opt.stream) cudaStreamSynchronize((cudaStream_t)ctx->opt.stream);
  delete ctx;
}

int gspm_mesh_info_get(const gspm_ctx* ctx, gspm_mesh_info* out) {
  if (!ctx || !out) {
    set_error("mesh_info: null argument");
    return GSPM_EINVAL;
  }
  out->n_stored = ctx->hm.n_stored;
  out->n_unique = ctx->hm.n;
  out->n_tets = ctx->hm.n_tets;
  out->n_magnetic_nodes = ctx->hm.n_mag_nodes;
  out->n_magnetic_tets = ctx->hm.n_mag_tets;
  out->nnz = ctx->hm.rowptr.empty() ? 0 : ctx->hm.rowptr.back();
  out->sell_entries = ctx->hs.entries;
  out->volume = ctx->hm.volume;
  out->volume_magnetic = ctx->hm.volume_mag;
  out->eps = ctx->P.eps;
  out->dtau = ctx->P.dtau;
  out->device_bytes = ctx->eng ? ctx->eng->device_bytes() : 0;
  return GSPM_OK;
}

int gspm_mesh_export(const gspm_ctx* ctx, int what, void* out, int64_t count) {
  if (!ctx || !out) {
    set_error("mesh_export: null argument");
    return GSPM_EINVAL;
  }
  const HostMesh& hm = ctx->hm;
  auto put = [&](const void* src, int64_t len, size_t elem) -> int {
    if (count != len) {
      set_error("mesh_export: count %lld, structure has %lld", (long long)count, (long long)len);
      return GSPM_EINVAL;
    }
    memcpy(out, src, (size_t)len * elem);
    return GSPM_OK;
  };
  switch (what) {
    case GSPM_EXPORT_UNIQUE_OF_STORED: return put(hm.unique_of_stored.data(), hm.n_stored, 8);
    case GSPM_EXPORT_ROWPTR: return put(hm.rowptr.data(), hm.n + 1, 8);
    case GSPM_EXPORT_COLS: return put(hm.cols.data(), (int64_t)hm.cols.size(), 8);
    case GSPM_EXPORT_PERM: return put(hm.perm.data(), hm.n, 8);
    case GSPM_EXPORT_NODE_MAGNETIC: return put(hm.node_mag.data(), hm.n, 1);
    case GSPM_EXPORT_LUMPED_MASS: return put(hm.ML.data(), hm.n, 8);
    default:
      set_error("mesh_export: unknown selector %d", what);
      return GSPM_EINVAL;
  }
}

#define NEED_ENGINE(ctx)                                           \
  do {                                                             \
    if (!(ctx)) {                                                  \
      set_error("null context");                                   \
      return GSPM_EINVAL;                                          \
    }                                                              \
    if (!(ctx)->eng) {                                             \
      set_error("context was created host-only (no device state)"); \
      return GSPM_ESTATE;                                          \
    }                                                              \
  } while (0)

int gspm_set_field(gspm_ctx* ctx, int field, const double* data, int where) {
  NEED_ENGINE(ctx);
  return ctx->eng->set_field(field, data, where);
}

int gspm_get_field(gspm_ctx* ctx, int field, double* data, int where) {
  NEED_ENGINE(ctx);
  return ctx->eng->get_field(field, data, where);
}

int gspm_step(gspm_ctx* ctx, int n_steps, const double H_ext[3], gspm_step_stats* stats) {
  NEED_ENGINE(ctx);
  if (n_steps < 0 || !H_ext) {
    set_error("step: need n_steps >= 0 and H_ext");
    return GSPM_EINVAL;
  }
  return ctx->eng->step(n_steps, H_ext, stats);
}

int gspm_solve_elastic(gspm_ctx* ctx, const double* m, double* u, int where, int x0_mode,
                       const double* x0, double rtol, int* iters, double* relres) {
  NEED_ENGINE(ctx);
  return ctx->eng->solve_elastic(m, u, where, x0_mode, x0, rtol, iters, relres);
}

int gspm_volume_avg(gspm_ctx* ctx, const double* field, int where, int ncomp, double* out_host) {
  NEED_ENGINE(ctx);
  return ctx->eng->volume_avg(field, where, ncomp, out_host);
}

int gspm_apply(gspm_ctx* ctx, int op, const double* x, double* y, int where) {
  NEED_ENGINE(ctx);
  return ctx->eng->apply(op, x, y, where);
}

int64_t gspm_launch_count(const gspm_ctx* ctx) { return ctx ? ctx->launches : 0; }

int gspm_profile_enable(gspm_ctx* ctx, unsigned class_mask) {
  NEED_ENGINE(ctx);
  return ctx->eng->profile_enable(class_mask);
}

int gspm_profile_read(gspm_ctx* ctx, int kclass, double* total_ms, int64_t* launches) {
  NEED_ENGINE(ctx);
  return ctx->eng->profile_read(kclass, total_ms, launches);
}

}  // extern "C"
