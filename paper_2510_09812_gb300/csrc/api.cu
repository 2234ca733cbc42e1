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

#include <nvtx3/nvToolsExt.h>

#include "internal.h"
#include "kernels.cuh"
#include "mpnn.cuh"

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

// NVTX range for tools (Nsight); a no-op when no tool is attached
struct Trace {
  explicit Trace(const char* name) { nvtxRangePushA(name); }
  ~Trace() { nvtxRangePop(); }
  Trace(const Trace&) = delete;
  Trace& operator=(const Trace&) = delete;
};

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

// Rounding of the coarse inverse to its storage type: doubles as they are; bfloat16 (its bits in
// a uint16_t) by round-to-nearest-even of the float value (finite values)
template <typename S>
S to_store(double v);
template <>
inline double to_store<double>(double v) {
  return v;
}
template <>
inline uint16_t to_store<uint16_t>(double v) {
  const float f = (float)v;
  uint32_t u;
  std::memcpy(&u, &f, sizeof(u));
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

class EngineBase {
 public:
  virtual ~EngineBase() = default;
  virtual int step(int n_steps, const double* H, bool per_segment, gspm_step_stats* st) = 0;
  virtual int solve_elastic(const double* m, double* u, int where, int x0_mode, const double* x0,
                            double rtol, int* iters, double* relres) = 0;
  virtual int volume_avg(const double* f, int where, int nc, double* out) = 0;
  virtual int apply(int op, const double* x, double* y, int where) = 0;
  virtual int set_field(int field, const double* data, int where) = 0;
  virtual int get_field(int field, double* data, int where) = 0;
  virtual int64_t device_bytes() const = 0;
  virtual void tune_info(int* vb, int* vs, int* vg, float* tb, float* ts, float* tg,
                         int* item_slices) const = 0;
  virtual int profile_enable(unsigned mask) = 0;
  virtual int profile_read(int cls, double* ms, int64_t* launches) = 0;
  virtual int set_x0_mode(int mode) = 0;
  virtual int set_graph(int on) = 0;
  virtual int set_true_residual(int on) = 0;
  virtual int set_rtol(double gs, double ms, double mech) = 0;
  virtual int mpnn_params(float* out, const float* in, int64_t count) = 0;
  virtual int mpnn_predict(const double* m, const double* up, const double* up2, double* out,
                           int what, int where) = 0;
  virtual int mpnn_dataset_reserve(int capacity) = 0;
  virtual int mpnn_dataset_add(const double* m, const double* up, const double* up2,
                               const double* ustar, int where, int* index) = 0;
  virtual int mpnn_loss_grad(int pair, double* loss, float* grad) = 0;
  virtual int mpnn_train(int iters, double lr, uint64_t seed, double* l0, double* l1) = 0;
};

template <typename T>
class Engine final : public EngineBase {
 public:
  Engine(const HostBatch& hb, const Params& P, const gspm_options& opt, cudaStream_t stream,
         int64_t* counter)
      : hb_(hb), P_(P), opt_(opt) {
    n_ = hb.sell.n;
    ld_ = (n_ + 31) / 32 * 32;
    nslices_ = hb.sell.nslices;
    entries_ = hb.sell.entries;
    nseg_ = (int)hb.seg_row0.size();
    nmag_ = hb.n_mag_nodes;
    nodes_ = hb.n_nodes;
    L_.stream = stream;
    L_.counter = counter;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    L_.max_blocks = std::max(1, sms) * 8;
    L_.sms = std::max(1, sms);
  }
  ~Engine() override {
    if (gexec_) cudaGraphExecDestroy(gexec_);
    if (cap_stream_) cudaStreamDestroy(cap_stream_);
    if (body_stream_) cudaStreamDestroy(body_stream_);
    if (host_graph_) cudaFreeHost(host_graph_);
    if (host_state_) cudaFreeHost(host_state_);
    if (host_bad_) cudaFreeHost(host_bad_);
    if (host_active_) cudaFreeHost(host_active_);
    if (host_scal_) cudaFreeHost(host_scal_);
    for (cudaEvent_t e : prof_ev_) cudaEventDestroy(e);
  }

  int init() {
    const HostSell& hs = hb_.sell;
    const HostOps& ops = hb_.ops;
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
    // inverse diagonals of M + eps K and M + alpha eps K (Jacobi preconditioner of the GSPM
    // solves): a row's diagonal is the sum of its entries in its own column (SELL padding
    // entries point at the row itself and hold 0)
    if (!(opt_.flags & (GSPM_FLAG_PLAIN_CG | GSPM_FLAG_PINNED_CG))) {
      std::vector<double> de(n, 0.0), da(n, 0.0);
      for (int64_t sl = 0; sl < nslices_; ++sl)
        for (int k = 0; k < hs.slen[sl]; ++k)
          for (int lane = 0; lane < 32; ++lane) {
            const int64_t row = sl * 32 + lane, ent = hs.sptr[sl] + (int64_t)k * 32 + lane;
            if (row < n && hs.col[ent] == row) {
              de[row] += ops.Aeps[ent];
              da[row] += ops.Aaeps[ent];
            }
          }
      for (int64_t i = 0; i < n; ++i) {
        de[i] = de[i] > 0.0 ? 1.0 / de[i] : 1.0;
        da[i] = da[i] > 0.0 ? 1.0 / da[i] : 1.0;
      }
      ST(upload(&dgs_eps_, de));
      ST(upload(&dgs_aeps_, da));
    }
    // per-row arrays are padded to whole slices (ld rows; zero, or -1 for perm, on the padding)
    // so that every kernel may address the rows of its last slice
    ST(mem_.alloc(&invML_, ld));
    ST(mem_.alloc(&w_, ld));
    ST(mem_.alloc(&mag_, ld));
    ST(mem_.alloc(&perm_, ld));
    CK(cudaMemset(invML_, 0, ld * sizeof(double)));
    CK(cudaMemset(w_, 0, ld * sizeof(double)));
    CK(cudaMemset(mag_, 0, ld));
    CK(cudaMemset(perm_, 0xff, ld * sizeof(int64_t)));
    CK(cudaMemcpy(invML_, ops.invML.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(w_, ops.w.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(mag_, ops.mag.data(), n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(perm_, hb_.perm.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice));
    ST(init_segments());
    ST(mem_.alloc(&m_, 3 * ld));
    ST(mem_.alloc(&ms_, 3 * ld));
    ST(mem_.alloc(&h_, 3 * ld));
    ST(mem_.alloc(&hd_, 3 * ld));
    ST(mem_.alloc(&E_, 6 * ld));
    ST(mem_.alloc(&E0_, 6 * ld));
    ST(mem_.alloc(&sig0_, 6 * ld));
    ST(mem_.alloc(&U_, ld));
    ST(mem_.alloc(&u_, 3 * ld));
    ST(mem_.alloc(&u2_, 3 * ld));
    if (std::is_same<T, float>::value) {
      // low parts of the refined K^ms / K^mech solutions and the correction solves' iterate
      ST(mem_.alloc(&Ulo_, ld));
      ST(mem_.alloc(&ulo_, 3 * ld));
      ST(mem_.alloc(&dx_, 3 * ld));
      CK(cudaMemset(Ulo_, 0, ld * sizeof(T)));
      CK(cudaMemset(ulo_, 0, 3 * ld * sizeof(T)));
    }
    ST(mem_.alloc(&utmp_, 3 * ld));
    ST(mem_.alloc(&uin_, 3 * ld));
    ST(mem_.alloc(&uin2_, 3 * ld));
    CK(cudaMemset(sig0_, 0, 6 * ld * sizeof(T)));
    CK(cudaMemset(utmp_, 0, 3 * ld * sizeof(T)));
    CK(cudaMemset(uin_, 0, 3 * ld * sizeof(T)));
    CK(cudaMemset(uin2_, 0, 3 * ld * sizeof(T)));
    {
      std::vector<float> a(ops.Agg.begin(), ops.Agg.end()), at(ops.AggT.begin(), ops.AggT.end());
      ST(mem_.alloc(&agg_, (int64_t)a.size()));
      ST(mem_.alloc(&aggT_, (int64_t)at.size()));
      CK(cudaMemcpy(agg_, a.data(), a.size() * sizeof(float), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(aggT_, at.data(), at.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    h_scale_ = hb_.seg_h[0];
    ST(mem_.alloc(&b_, 3 * ld));
    ST(mem_.alloc(&r_, 3 * ld));
    ST(mem_.alloc(&x_, 3 * ld));
    ST(mem_.alloc(&p_, 3 * ld));
    ST(mem_.alloc(&q_, 3 * ld));
    ST(mem_.alloc(&stage_, 9 * n));
    ST(mem_.alloc(&tin_, 3 * ld));
    ST(mem_.alloc(&tout_, 3 * ld));
    ST(mem_.alloc(&cg_, (int64_t)kSolveSlots * nseg_));
    ST(mem_.alloc(&proj_, 6 * (int64_t)nseg_));
    ST(mem_.alloc(&tres_, 4 * (int64_t)nseg_));
    CK(cudaMemset(tres_, 0, 4 * nseg_ * sizeof(double)));
    ST(mem_.alloc(&bad_, (int64_t)nseg_));
    CK(cudaMemset(bad_, 0, nseg_ * sizeof(int)));
    CK(cudaMallocHost(&host_bad_, nseg_ * sizeof(int)));
    ST(mem_.alloc(&pinsave_, 3 * (int64_t)nseg_));
    ST(mem_.alloc(&wmean_, n));
    {
      std::vector<double> wm(n, 0.0);
      for (int sg = 0; sg < nseg_; ++sg)
        for (int64_t i = 0; i < hb_.seg_nrow[sg]; ++i)
          wm[hb_.seg_row0[sg] + i] = 1.0 / (double)hb_.seg_nrow[sg];
      CK(cudaMemcpy(wmean_, wm.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    }
    ST(mem_.alloc(&nactive_, kSolveSlots));
    ST(mem_.alloc(&scal_, (int64_t)kScalPerSeg * nseg_ + 8));
    CK(cudaMemset(scal_, 0, ((int64_t)kScalPerSeg * nseg_ + 8) * sizeof(double)));
    CK(cudaMemset(nactive_, 0, kSolveSlots * sizeof(int)));
    CK(cudaMemset(m_, 0, 3 * ld * sizeof(T)));
    CK(cudaMemset(ms_, 0, 3 * ld * sizeof(T)));
    CK(cudaMemset(h_, 0, 3 * ld * sizeof(T)));
    CK(cudaMemset(hd_, 0, 3 * ld * sizeof(T)));
    CK(cudaMemset(E_, 0, 6 * ld * sizeof(T)));
    CK(cudaMemset(U_, 0, ld * sizeof(T)));
    CK(cudaMemset(u_, 0, 3 * ld * sizeof(T)));
    CK(cudaMemset(u2_, 0, 3 * ld * sizeof(T)));
    CK(cudaMemset(x_, 0, 3 * ld * sizeof(T)));
    CK(cudaMemset(r_, 0, 3 * ld * sizeof(T)));
    CK(cudaMemset(b_, 0, 3 * ld * sizeof(T)));
    CK(cudaMemset(p_, 0, 3 * ld * sizeof(T)));
    CK(cudaMemset(q_, 0, 3 * ld * sizeof(T)));
    CK(cudaMemset(cg_, 0, (int64_t)kSolveSlots * nseg_ * sizeof(CGState)));
    // E_ext (added to <E0> when forming E_bar) and 1 / (magnetic nodes) per segment
    CK(cudaMemcpy(eext(), P_.E_ext, 6 * sizeof(double), cudaMemcpyHostToDevice));
    {
      std::vector<double> inv(nseg_);
      for (int s = 0; s < nseg_; ++s)
        inv[s] = hb_.seg_nmag[s] > 0 ? 1.0 / (double)hb_.seg_nmag[s] : 0.0;
      CK(cudaMemcpy(inv_nmag(), inv.data(), nseg_ * sizeof(double), cudaMemcpyHostToDevice));
    }
    CK(cudaMallocHost(&host_state_, (int64_t)nseg_ * sizeof(CGState)));
    CK(cudaMallocHost(&host_active_, sizeof(int)));
    CK(cudaMallocHost(&host_scal_, ((int64_t)kScalPerSeg * nseg_ + 8) * sizeof(double)));
    for (int k = 0; k < kSolveSlots; ++k) pred_[k] = 8;
    CK(cudaDeviceSynchronize());
    if (!(opt_.flags & GSPM_FLAG_NO_AUTOTUNE)) ST(autotune());
    graph_on_ = (opt_.flags & GSPM_FLAG_GRAPH) != 0;
    if (!hb_.coarse.empty()) ST(init_coarse());
    pinned_ = (opt_.flags & GSPM_FLAG_PINNED_CG) ? 1 : 0;
    resolve_ = (opt_.flags & GSPM_FLAG_RESOLVE_AT_MSTAR) != 0;
    return GSPM_OK;
  }

  // Project autotuner: time every SpMV schedule as the CG loops run it (the product fused with
  // p.q and alpha, k_cg_spmv) on this mesh's own operators: K^mech for the 3x3-block solves,
  // K^ms for the scalar ones, M + eps K with one, two and three right-hand sides for the GSPM
  // solves (their summed time decides).  A scratch CG state with every segment active and a
  // non-constant search direction (so that p.Ap > 0) is reset before each schedule; one warm-up
  // and five timed launches with CUDA events on the context's stream; the fastest is kept.
  int autotune() {
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CGState* st = nullptr;
    ST(mem_.alloc(&st, (int64_t)nseg_));
    std::vector<CGState> hs(nseg_);
    for (auto& c : hs) {
      memset(&c, 0, sizeof(c));
      c.nr = 3;
      c.active = 1;
      c.max_iter = 1 << 30;
      for (int k = 0; k < 3; ++k) c.r[k].bb = c.r[k].rr = c.r[k].rz = 1.0;
    }
    {
      std::vector<T> pv((size_t)3 * ld_);
      for (size_t i = 0; i < pv.size(); ++i) pv[i] = (T)(1.0 + 0.5 * std::sin(0.37 * (double)i));
      CK(cudaMemcpy(tin_, pv.data(), pv.size() * sizeof(T), cudaMemcpyHostToDevice));
    }
    const int pinned = (opt_.flags & GSPM_FLAG_PINNED_CG) ? 1 : 0;
    auto time_variant = [&](const T* val, int B, int nr, int diff, int pin, int var,
                            float* ms) -> int {
      CK(cudaMemcpyAsync(st, hs.data(), nseg_ * sizeof(CGState), cudaMemcpyHostToDevice,
                         L_.stream));
      const int64_t ld = B == 9 ? 3 * n_ : (nr == 1 ? n_ : ld_);
      CK(launch_cg_spmv<T>(L_, A_, SG_, val, B, nr, ld, tin_, tout_, st, red_, var, pin, diff));
      CK(cudaEventRecord(e0, L_.stream));
      for (int k = 0; k < 5; ++k)
        CK(launch_cg_spmv<T>(L_, A_, SG_, val, B, nr, ld, tin_, tout_, st, red_, var, pin, diff));
      CK(cudaEventRecord(e1, L_.stream));
      CK(cudaEventSynchronize(e1));
      CK(cudaEventElapsedTime(ms, e0, e1));
      *ms /= 5.f;
      return GSPM_OK;
    };
    float best_b = 1e30f, best_s = 1e30f, best_g = 1e30f;
    for (int v = 0; v < kSpmvVariants; ++v) {
      float t = 0.f;
      ST(time_variant(Kmech_, 9, 1, 1, pinned, v, &t));
      tune_ms_block_[v] = t;
      if (t < best_b) { best_b = t; var_block_ = v; }
      ST(time_variant(Kms_, 1, 1, 1, pinned, v, &t));
      tune_ms_scalar_[v] = t;
      if (t < best_s) { best_s = t; var_scalar_ = v; }
      // the GSPM operators are not in difference form: their own schedule
      float tg = 0.f;
      for (int nr = 1; nr <= 3; ++nr) {
        ST(time_variant(Aeps_, 1, nr, 0, 0, v, &t));
        tg += t;
      }
      tune_ms_gs_[v] = tg;
      if (tg < best_g) { best_g = tg; var_gs_ = v; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return GSPM_OK;
  }

 public:
  void tune_info(int* vb, int* vs, int* vg, float* tb, float* ts, float* tg,
                 int* item_slices) const override {
    *vb = var_block_;
    *vs = var_scalar_;
    *vg = var_gs_;
    *item_slices = item_slices_;
    for (int v = 0; v < kSpmvVariants; ++v) {
      tb[v] = tune_ms_block_[v];
      ts[v] = tune_ms_scalar_[v];
      tg[v] = tune_ms_gs_[v];
    }
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
  // Per-step solve records of the direct (non-graph) path: per segment, for K^ms, K^mech and
  // each Gauss-Seidel right-hand side in sweep order.
  struct StepInfo {
    std::vector<SolveInfo> ims, imech, ig[8];
    std::vector<SolveInfo> ims2, imech2;  // the solves at m* (GSPM_FLAG_RESOLVE_AT_MSTAR)
    int ngs = 0;
  };

  // H: applied field (A/m), three values per segment when per_segment, else one for all.
  // st: per-segment statistics (nseg entries) or NULL.
  int step(int n_steps, const double* H, bool per_segment, gspm_step_stats* st) override {
    DevParams D = dev_params();
    const int printed = (opt_.flags & GSPM_FLAG_ROW2_PRINTED) ? 1 : 0;
    for (int s = 0; s < nseg_; ++s)
      for (int a = 0; a < 3; ++a)
        host_scal_[3 * s + a] = (per_segment ? H[3 * s + a] : H[a]) / P_.Ms;
    CK(cudaMemcpyAsync(hz(), host_scal_, 3 * nseg_ * sizeof(double), cudaMemcpyHostToDevice,
                       L_.stream));
    CK(cudaMemsetAsync(bad_, 0, nseg_ * sizeof(int), L_.stream));
    if (graph_on_ && prof_mask_ == 0) {
      const int rc = step_graph(n_steps, D, printed, st);
      if (rc != GSPM_OK && rc != GSPM_ENOCONV) return rc;
      ST(check_finite());
      return rc;
    }
    std::vector<gspm_step_stats> acc(nseg_);
    for (auto& a : acc) memset(&a, 0, sizeof(a));
    StepInfo si;
    for (int stp = 0; stp < n_steps; ++stp) {
      ST(step_once(D, printed, &si));
      for (int sg = 0; sg < nseg_; ++sg) {
        gspm_step_stats& a = acc[sg];
        a.steps += 1;
        a.it_ms += si.ims[sg].iters;
        a.it_mech += si.imech[sg].iters;
        a.noconv += si.ims[sg].noconv + si.imech[sg].noconv;
        const SolveInfo& lms = resolve_ ? si.ims2[sg] : si.ims[sg];
        const SolveInfo& lme = resolve_ ? si.imech2[sg] : si.imech[sg];
        if (resolve_) {
          a.it_ms += lms.iters;
          a.it_mech += lme.iters;
          a.noconv += lms.noconv + lme.noconv;
        }
        a.it_ms_last = lms.iters;
        a.it_mech_last = lme.iters;
        a.res_ms_last = lms.relres;
        a.res_mech_last = lme.relres;
        for (int k = 0; k < 8; ++k) {
          a.it_gs_last[k] = k < si.ngs ? si.ig[k][sg].iters : 0;
          if (k < si.ngs) {
            a.it_gs += si.ig[k][sg].iters;
            a.noconv += si.ig[k][sg].noconv;
          }
        }
      }
    }
    int noconv = 0;
    for (auto& a : acc) noconv += a.noconv;
    if (st) {
      CK(cudaMemcpyAsync(host_scal_, scal_, 13 * nseg_ * sizeof(double), cudaMemcpyDeviceToHost,
                         L_.stream));
      ST(read_true_res());
      CK(cudaStreamSynchronize(L_.stream));
      for (int sg = 0; sg < nseg_; ++sg) {
        for (int a = 0; a < 3; ++a) acc[sg].m_bar[a] = host_scal_[3 * sg + a];
        acc[sg].dm_last = host_scal_[12 * nseg_ + sg];
        true_res_of(sg, &acc[sg]);
        st[sg] = acc[sg];
      }
    }
    CK(cudaGetLastError());
    ST(check_finite());
    return noconv ? GSPM_ENOCONV : GSPM_OK;
  }

  // GSPM_ENUMERIC if a projection of this call met a non-finite or zero m** (synchronises)
  // the learned guess's tensor-core layers report a wait that gave up through mpnn_err_
  int check_net() {
    if (!mpnn_err_) return GSPM_OK;
    int e = 0;
    CK(cudaMemcpyAsync(&e, mpnn_err_, sizeof(int), cudaMemcpyDeviceToHost, L_.stream));
    CK(cudaStreamSynchronize(L_.stream));
    if (e) {
      set_error("learned initial guess: a tensor-core layer did not complete within its wait limit");
      return GSPM_ETIMEOUT;
    }
    return GSPM_OK;
  }

  int check_finite() {
    ST(check_net());
    CK(cudaMemcpyAsync(host_bad_, bad_, nseg_ * sizeof(int), cudaMemcpyDeviceToHost, L_.stream));
    CK(cudaStreamSynchronize(L_.stream));
    for (int sg = 0; sg < nseg_; ++sg)
      if (host_bad_[sg] > 0) {
        set_error("step: m** not finite or zero at %d magnetic nodes of mesh %d", host_bad_[sg],
                  sg);
        return GSPM_ENUMERIC;
      }
    return GSPM_OK;
  }

  // The kernel sequence of one GSPM step (Algorithm B.1 with the field and equilibrium solves
  // of Sec. 2).  While a graph is being captured the CG loops become WHILE nodes and `si` is
  // left alone.
  int step_once(const DevParams& D, int printed, StepInfo* si) {
    Trace trace_step("gspm_step");
    const int64_t n = n_, ld = ld_;
    // a1 volume average of m (Sec. 2.4)
    TK(GSPM_KCLASS_POINTWISE, launch_wsum<T>(L_, SG_, 3, m_, ld, 1, nullptr, w_, mbar(), nullptr, red_));
    // a2 b^ms / m_s = F^ms m (Eq. RHS_b), a3 CG on pinned K^ms, x0 = previous U
    TK(GSPM_KCLASS_RHS_MS, launch_fdiv<T>(L_, A_, SG_, F_, m_, ld, b_, pinned_));
    ST(solve_system(kSlotMs, Kms_, 1, b_, U_, Ulo_, opt_.rtol_ms, &si->ims));
    // a4 local demagnetising field h~_d = -grad U
    TK(GSPM_KCLASS_GRAD_MS, launch_fgrad<T>(L_, A_, F_, U_, Ulo_, invML_, hd_, ld));
    // a5 E0(m), sigma0 = C E0, E_bar = <E0> + C^-1 sigma_ext
    TK(GSPM_KCLASS_POINTWISE, launch_e0<T>(L_, n, m_, ld, mag_, D, E0_, sig0_));
    TK(GSPM_KCLASS_POINTWISE, launch_wsum<T>(L_, SG_, 6, E0_, ld, 1, nullptr, w_, ebar(), eext(), red_));
    // a6 b^mech = F^mech E0, a7 CG on pinned K^mech, x0 per the initial-guess mode
    TK(GSPM_KCLASS_RHS_MECH, launch_gdiv<T>(L_, A_, SG_, G_, sig0_, b_, pinned_));
    ST(mech_initial_guess(m_, x0_mode_));
    ST(solve_system(kSlotMech, Kmech_, 9, b_, u_, ulo_, opt_.rtol_mech, &si->imech));
    // a8 strain E = E_bar + sym grad u
    TK(GSPM_KCLASS_STRAIN, launch_fstrain<T>(L_, A_, SG_, F_, u_, ulo_, invML_, ebar(), E_, ld));
    // a9 h(m^n)
    TK(GSPM_KCLASS_POINTWISE, launch_hfield<T>(L_, n, SG_, m_, hd_, E_, ld, mbar(), hz(), mag_, D, 0, 0.0, h_, nullptr));
    // a10 Gauss-Seidel stages (Algorithm B.1 steps 1-2), (M + eps K) g = M f, x0 = f
    std::vector<SolveInfo>* ig = si->ig;
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
    TK(GSPM_KCLASS_POINTWISE, launch_wsum<T>(L_, SG_, 3, ms_, ld, 1, nullptr, w_, mbar_s(), nullptr, red_));
    if (resolve_) {
      // variant: the magnetostatic and mechanical equilibria solved again at m* (x0 = the
      // step-n solutions), so h[m*] is the whole effective field of m*
      TK(GSPM_KCLASS_RHS_MS, launch_fdiv<T>(L_, A_, SG_, F_, ms_, ld, b_, pinned_));
      ST(solve_system(kSlotMs, Kms_, 1, b_, U_, Ulo_, opt_.rtol_ms, &si->ims2));
      TK(GSPM_KCLASS_GRAD_MS, launch_fgrad<T>(L_, A_, F_, U_, Ulo_, invML_, hd_, ld));
      TK(GSPM_KCLASS_POINTWISE, launch_e0<T>(L_, n, ms_, ld, mag_, D, E0_, sig0_));
      TK(GSPM_KCLASS_POINTWISE, launch_wsum<T>(L_, SG_, 6, E0_, ld, 1, nullptr, w_, ebar(), eext(), red_));
      TK(GSPM_KCLASS_RHS_MECH, launch_gdiv<T>(L_, A_, SG_, G_, sig0_, b_, pinned_));
      ST(solve_system(kSlotMech, Kmech_, 9, b_, u_, ulo_, opt_.rtol_mech, &si->imech2));
      TK(GSPM_KCLASS_STRAIN, launch_fstrain<T>(L_, A_, SG_, F_, u_, ulo_, invML_, ebar(), E_, ld));
    }
    TK(GSPM_KCLASS_POINTWISE, launch_hfield<T>(L_, n, SG_, ms_, hd_, E_, ld, mbar_s(), hz(), mag_, D, 1, P_.alpha * P_.dtau, nullptr, x_));
    // a12 (M + alpha eps K) m** = M f, three right-hand sides
    ST(solve_gs(kSlotGsD, Aaeps_, 0, 3, &ig[ngs]));
    ngs += 3;
    // a13 projection and <|dm|>
    TK(GSPM_KCLASS_POINTWISE, launch_project<T>(L_, SG_, ld, x_, mag_, m_, dmv(), inv_nmag(), red_, bad_));
    si->ngs = ngs;
    return GSPM_OK;
  }

  // ---------------------------------------------------------------- CUDA-graph replay
  // One step is captured once (per initial-guess mode) into a graph whose CG loops are WHILE
  // nodes: the body (SpMV, update, p-update) repeats until the device-side count of active
  // segments reaches zero, with the iteration limit max_iter + 2 as a backstop.  A call of
  // n steps is n graph launches and one synchronisation at the end; statistics come from device
  // accumulators and the CG status blocks.
  int set_graph(int on) override {
    graph_on_ = on != 0;
    return GSPM_OK;
  }

  int set_true_residual(int on) override {
    tres_on_ = on != 0;
    return GSPM_OK;
  }

  // new stopping tolerances (<= 0 keeps one); a captured graph is captured again
  int set_rtol(double gs, double ms, double mech) override {
    if (!(gs < 1.0) || !(ms < 1.0) || !(mech < 1.0)) {
      set_error("set_rtol: tolerances must be below 1");
      return GSPM_EINVAL;
    }
    if (gs > 0) opt_.rtol_gs = gs;
    if (ms > 0) opt_.rtol_ms = ms;
    if (mech > 0) opt_.rtol_mech = mech;
    ++cfg_gen_;
    return GSPM_OK;
  }

  // the true residuals of the last K^ms and K^mech solves into host_scal_[13 nseg ..) (async)
  int read_true_res() {
    if (tres_on_)
      CK(cudaMemcpyAsync(host_scal_ + 13 * nseg_, tres_, 4 * nseg_ * sizeof(double),
                         cudaMemcpyDeviceToHost, L_.stream));
    return GSPM_OK;
  }
  void true_res_of(int sg, gspm_step_stats* a) const {
    a->true_res_ms_last = a->true_res_mech_last = -1.0;
    if (!tres_on_) return;
    const double* t = host_scal_ + 13 * nseg_;
    a->true_res_ms_last = t[2 * sg + 1] > 0 ? std::sqrt(t[2 * sg] / t[2 * sg + 1]) : 0.0;
    a->true_res_mech_last =
        t[2 * nseg_ + 2 * sg + 1] > 0 ? std::sqrt(t[2 * nseg_ + 2 * sg] / t[2 * nseg_ + 2 * sg + 1]) : 0.0;
  }

  int graph_alloc() {
    if (loop_cnt_) return GSPM_OK;
    ST(mem_.alloc(&loop_cnt_, kSolveSlots));
    ST(mem_.alloc(&loop_total_, 1));
    ST(mem_.alloc(&gstats_, 4 * (int64_t)nseg_));
    CK(cudaMemset(loop_cnt_, 0, kSolveSlots * sizeof(int)));
    CK(cudaMemset(loop_total_, 0, sizeof(unsigned long long)));
    const size_t hb = 4 * (size_t)nseg_ * sizeof(long long) + sizeof(unsigned long long) +
                      (size_t)kSolveSlots * nseg_ * sizeof(CGState);
    CK(cudaMallocHost(&host_graph_, hb));
    CK(cudaStreamCreateWithFlags(&cap_stream_, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&body_stream_, cudaStreamNonBlocking));
    return GSPM_OK;
  }

  int build_graph(const DevParams& D, int printed) {
    Trace trace("gspm_graph_capture");
    ST(graph_alloc());
    if (gexec_) {
      CK(cudaGraphExecDestroy(gexec_));
      gexec_ = nullptr;
    }
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    const cudaStream_t outer = L_.stream;
    const int64_t c0 = *L_.counter;
    cudaError_t e = cudaStreamBeginCaptureToGraph(cap_stream_, g, nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeRelaxed);
    int rc = GSPM_OK;
    if (e == cudaSuccess) {
      L_.stream = cap_stream_;
      capturing_ = true;
      graph_body_ = 0;
      StepInfo si;
      rc = step_once(D, printed, &si);
      capturing_ = false;
      L_.stream = outer;
      cudaGraph_t out = nullptr;
      e = cudaStreamEndCapture(cap_stream_, &out);
    }
    const int64_t captured = *L_.counter - c0;
    *L_.counter = c0;  // nothing has run yet
    if (rc == GSPM_OK && e == cudaSuccess) e = cudaGraphInstantiate(&gexec_, g, 0);
    cudaGraphDestroy(g);
    ST(rc);
    if (e != cudaSuccess) {
      gexec_ = nullptr;
      set_error("graph capture of the step failed: %s", cudaGetErrorString(e));
      return GSPM_ECUDA;
    }
    graph_static_ = captured - graph_body_;
    gexec_x0_ = x0_mode_;
    gexec_tres_ = tres_on_;
    gexec_gen_ = cfg_gen_;
    return GSPM_OK;
  }

  // A CG loop as a WHILE node of the graph being captured on L_.stream.
  template <class Iter>
  int cg_graph_loop(int slot, Iter iter, int kind, int body_kernels) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    CK(cudaStreamGetCaptureInfo(L_.stream, &cs, nullptr, &g, nullptr, nullptr, nullptr));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
    const LoopCtl lc{h, nactive_ + slot, loop_cnt_ + slot, opt_.max_iter + 2, body_kernels,
                     loop_total_};
    CK(launch_loop_start(L_, lc));
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(L_.stream, &cs, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    CK(cudaStreamUpdateCaptureDependencies(L_.stream, &node, nullptr, 1,
                                           cudaStreamSetCaptureDependencies));
    const cudaStream_t outer = L_.stream;
    CK(cudaStreamBeginCaptureToGraph(body_stream_, body, nullptr, nullptr, 0,
                                     cudaStreamCaptureModeRelaxed));
    L_.stream = body_stream_;
    loop_ = lc;
    const int64_t c0 = *L_.counter;
    const int rc = iter();
    graph_body_ += *L_.counter - c0;
    loop_ = LoopCtl{};
    L_.stream = outer;
    cudaGraph_t done = nullptr;
    const cudaError_t e = cudaStreamEndCapture(body_stream_, &done);
    ST(rc);
    CK(e);
    CK(launch_solve_stats(L_, cg_ + (int64_t)slot * nseg_, nseg_, kind, gstats_));
    return GSPM_OK;
  }

  static SolveInfo info_of(const CGState& c, int k) {
    SolveInfo s;
    for (int j = 0; j < c.nr; ++j) {
      if (k >= 0 && j != k) continue;
      s.iters = std::max(s.iters, c.r[j].iters);
      const double bb = c.r[j].bb;
      s.relres = std::max(s.relres, bb > 0 ? std::sqrt(c.r[j].rr / bb) : 0.0);
    }
    s.noconv = c.noconv;
    return s;
  }

  int step_graph(int n_steps, const DevParams& D, int printed, gspm_step_stats* st) {
    if (!gexec_ || gexec_x0_ != x0_mode_ || gexec_tres_ != tres_on_ || gexec_gen_ != cfg_gen_)
      ST(build_graph(D, printed));
    CK(cudaMemsetAsync(gstats_, 0, 4 * (size_t)nseg_ * sizeof(long long), L_.stream));
    for (int s = 0; s < n_steps; ++s) CK(cudaGraphLaunch(gexec_, L_.stream));
    *L_.counter += graph_static_ * n_steps;
    long long* hst = reinterpret_cast<long long*>(host_graph_);
    unsigned long long* hloops = reinterpret_cast<unsigned long long*>(hst + 4 * nseg_);
    CGState* hcg = reinterpret_cast<CGState*>(hloops + 1);
    CK(cudaMemcpyAsync(hst, gstats_, 4 * (size_t)nseg_ * sizeof(long long),
                       cudaMemcpyDeviceToHost, L_.stream));
    CK(cudaMemcpyAsync(hloops, loop_total_, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                       L_.stream));
    CK(cudaMemcpyAsync(hcg, cg_, (size_t)kSolveSlots * nseg_ * sizeof(CGState),
                       cudaMemcpyDeviceToHost, L_.stream));
    CK(cudaMemcpyAsync(host_scal_, scal_, 13 * nseg_ * sizeof(double), cudaMemcpyDeviceToHost,
                       L_.stream));
    ST(read_true_res());
    CK(cudaStreamSynchronize(L_.stream));
    // kernels the loop bodies ran
    *L_.counter += (int64_t)(*hloops - loops_seen_);
    loops_seen_ = *hloops;
    // Gauss-Seidel solves in sweep order: (slot, right-hand side)
    static const int kGsOrder[2][8][2] = {
        {{kSlotGs0, 0}, {kSlotGs0, 1}, {kSlotGs1, 0}, {kSlotGs2, 0}, {kSlotGsD, 0},
         {kSlotGsD, 1}, {kSlotGsD, 2}, {-1, 0}},
        {{kSlotGs0, 0}, {kSlotGs0, 1}, {kSlotGs0, 2}, {kSlotGs1, 0}, {kSlotGs1, 1},
         {kSlotGsD, 0}, {kSlotGsD, 1}, {kSlotGsD, 2}}};
    int noconv = 0;
    for (int sg = 0; sg < nseg_; ++sg) {
      noconv += (int)hst[4 * sg + 3];
      if (!st) continue;
      gspm_step_stats a;
      memset(&a, 0, sizeof(a));
      a.steps = n_steps;
      a.it_ms = hst[4 * sg + 0];
      a.it_mech = hst[4 * sg + 1];
      a.it_gs = hst[4 * sg + 2];
      a.noconv = (int)hst[4 * sg + 3];
      SolveInfo ms = info_of(hcg[kSlotMs * nseg_ + sg], -1);
      SolveInfo me = info_of(hcg[kSlotMech * nseg_ + sg], -1);
      if (Ulo_) {  // refined solves: both CG loops, the residual of the correction solve
        const SolveInfo ms2 = info_of(hcg[kSlotMs2 * nseg_ + sg], -1);
        const SolveInfo me2 = info_of(hcg[kSlotMech2 * nseg_ + sg], -1);
        ms.iters += ms2.iters;
        ms.relres = ms2.relres;
        me.iters += me2.iters;
        me.relres = me2.relres;
      }
      a.it_ms_last = ms.iters;
      a.it_mech_last = me.iters;
      a.res_ms_last = ms.relres;
      a.res_mech_last = me.relres;
      for (int k = 0; k < 8; ++k) {
        const int slot = kGsOrder[printed][k][0];
        a.it_gs_last[k] =
            slot < 0 ? 0 : info_of(hcg[slot * nseg_ + sg], kGsOrder[printed][k][1]).iters;
      }
      for (int c = 0; c < 3; ++c) a.m_bar[c] = host_scal_[3 * sg + c];
      a.dm_last = host_scal_[12 * nseg_ + sg];
      true_res_of(sg, &a);
      st[sg] = a;
    }
    CK(cudaGetLastError());
    return noconv ? GSPM_ENOCONV : GSPM_OK;
  }

  int solve_elastic(const double* m, double* u, int where, int x0_mode, const double* x0,
                    double rtol, int* iters, double* relres) override {
    const int64_t n = n_, ld = ld_;
    if (!m) {
      set_error("solve_elastic: m is NULL");
      return GSPM_EINVAL;
    }
    DevParams D = dev_params();
    // magnetisation into the m* buffer (the context's m is left alone)
    ST(import_field(m, where, 3, ms_, ld, 1, mag_));
    if (x0_mode == 2) {
      if (!x0) {
        set_error("solve_elastic: x0_mode 2 needs x0");
        return GSPM_EINVAL;
      }
      ST(import_field(x0, where, 3, utmp_, 1, 3, nullptr));
      CK(cudaMemcpyAsync(u2_, u_, 3 * n * sizeof(T), cudaMemcpyDeviceToDevice, L_.stream));
      CK(cudaMemcpyAsync(u_, utmp_, 3 * n * sizeof(T), cudaMemcpyDeviceToDevice, L_.stream));
    } else {
      static const int map[5] = {GSPM_X0_ZERO, GSPM_X0_PREV, -1, GSPM_X0_EXTRAPOLATE,
                                 GSPM_X0_LEARNED};
      if (x0_mode < 0 || x0_mode > 4) {
        set_error("solve_elastic: bad x0_mode %d", x0_mode);
        return GSPM_EINVAL;
      }
      ST(mech_initial_guess(ms_, map[x0_mode]));
    }
    TK(GSPM_KCLASS_POINTWISE, launch_e0<T>(L_, n, ms_, ld, mag_, D, E0_, sig0_));
    TK(GSPM_KCLASS_POINTWISE, launch_wsum<T>(L_, SG_, 6, E0_, ld, 1, nullptr, w_, ebar(), eext(), red_));
    TK(GSPM_KCLASS_RHS_MECH, launch_gdiv<T>(L_, A_, SG_, G_, sig0_, b_, pinned_));
    std::vector<SolveInfo> info;
    ST(solve_system(kSlotMech, Kmech_, 9, b_, u_, ulo_, rtol > 0 ? rtol : opt_.rtol_mech, &info));
    TK(GSPM_KCLASS_STRAIN, launch_fstrain<T>(L_, A_, SG_, F_, u_, ulo_, invML_, ebar(), E_, ld));
    if (u) ST(export_field(u_, 1, 3, 3, u, where, ulo_));
    CK(cudaStreamSynchronize(L_.stream));
    int it = 0, nc = 0;
    double rel = 0.0;
    for (auto& i : info) {
      it = std::max(it, i.iters);
      rel = std::max(rel, i.relres);
      nc += i.noconv;
    }
    if (iters) *iters = it;
    if (relres) *relres = rel;
    return nc ? GSPM_ENOCONV : GSPM_OK;
  }

  int volume_avg(const double* f, int where, int nc, double* out) override {
    if (nc < 1 || nc > 9 || !f || !out) {
      set_error("volume_avg: need 1 <= ncomp <= 9 and non-null pointers");
      return GSPM_EINVAL;
    }
    const double* src = f;
    if (where == GSPM_HOST) {
      CK(cudaMemcpyAsync(stage_, f, nodes_ * nc * sizeof(double), cudaMemcpyHostToDevice,
                         L_.stream));
      src = stage_;
    }
    CK(launch_wsum<double>(L_, SG_, nc, src, 1, nc, perm_, w_, avg(), nullptr, red_));
    CK(cudaMemcpyAsync(out, avg(), nseg_ * nc * sizeof(double), cudaMemcpyDeviceToHost, L_.stream));
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
        if (op == GSPM_OP_K_MS) ST(pin_hide(1));
        CK(launch_spmv<T>(L_, A_, val, 1, tin_, tout_, var_scalar_, op == GSPM_OP_K_MS ? 1 : 0));
        if (op == GSPM_OP_K_MS) ST(pin_restore(1));
        ST(export_field(tout_, 1, 1, 1, y, where));
        break;
      }
      case GSPM_OP_K_MECH:
        ST(import_field(x, where, 3, tin_, 1, 3, nullptr));
        ST(pin_hide(3));
        CK(launch_spmv<T>(L_, A_, Kmech_, 9, tin_, tout_, var_block_, 1));
        ST(pin_restore(3));
        ST(export_field(tout_, 1, 3, 3, y, where));
        break;
      case GSPM_OP_DIV:
        ST(import_field(x, where, 3, tin_, ld, 1, nullptr));
        CK(launch_fdiv<T>(L_, A_, SG_, F_, tin_, ld, b_, 1));
        ST(export_field(b_, 1, 1, 1, y, where));
        break;
      case GSPM_OP_GRAD:
        ST(import_field(x, where, 1, r_, 1, 1, nullptr));
        CK(launch_fgrad<T>(L_, A_, F_, r_, nullptr, invML_, tout_, ld));
        ST(export_field(tout_, ld, 1, 3, y, where));
        break;
      default:
        set_error("apply: unknown operator %d", op);
        return GSPM_EINVAL;
    }
    if (where == GSPM_HOST) CK(cudaStreamSynchronize(L_.stream));
    return GSPM_OK;
  }

  // The stored K^ms and K^mech are the unpinned periodic operators.  The pinned operator of
  // Sec. 2.5 (pinned rows and columns replaced by the identity) is y = K (x with x_pin = 0),
  // then y_pin = x_pin: pin_hide keeps each segment's x_pin aside in tin_ and zeroes it,
  // pin_restore writes it into tout_.
  int pin_hide(int epr) {
    for (int sg = 0; sg < nseg_; ++sg) {
      T* xp = tin_ + epr * hb_.seg_pin[sg];
      CK(cudaMemcpyAsync(pinsave_ + 3 * sg, xp, epr * sizeof(T), cudaMemcpyDeviceToDevice,
                         L_.stream));
      CK(cudaMemsetAsync(xp, 0, epr * sizeof(T), L_.stream));
    }
    return GSPM_OK;
  }
  int pin_restore(int epr) {
    for (int sg = 0; sg < nseg_; ++sg)
      CK(cudaMemcpyAsync(tout_ + epr * hb_.seg_pin[sg], pinsave_ + 3 * sg, epr * sizeof(T),
                         cudaMemcpyDeviceToDevice, L_.stream));
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
        ST(import_field(data, where, 1, U_, 1, 1, nullptr, Ulo_));
        for (int sg = 0; sg < nseg_; ++sg) {
          CK(cudaMemsetAsync(U_ + hb_.seg_pin[sg], 0, sizeof(T), L_.stream));
          if (Ulo_) CK(cudaMemsetAsync(Ulo_ + hb_.seg_pin[sg], 0, sizeof(T), L_.stream));
        }
        break;
      case GSPM_FIELD_DISP:
        ST(import_field(data, where, 3, u_, 1, 3, nullptr, ulo_));
        for (int sg = 0; sg < nseg_; ++sg) {
          CK(cudaMemsetAsync(u_ + 3 * hb_.seg_pin[sg], 0, 3 * sizeof(T), L_.stream));
          if (ulo_) CK(cudaMemsetAsync(ulo_ + 3 * hb_.seg_pin[sg], 0, 3 * sizeof(T), L_.stream));
        }
        break;
      case GSPM_FIELD_DISP_PREV:
        ST(import_field(data, where, 3, u2_, 1, 3, nullptr));
        for (int sg = 0; sg < nseg_; ++sg)
          CK(cudaMemsetAsync(u2_ + 3 * hb_.seg_pin[sg], 0, 3 * sizeof(T), L_.stream));
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
      case GSPM_FIELD_U: ST(export_field(U_, 1, 1, 1, data, where, Ulo_)); break;
      case GSPM_FIELD_DISP: ST(export_field(u_, 1, 3, 3, data, where, ulo_)); break;
      case GSPM_FIELD_DISP_PREV: ST(export_field(u2_, 1, 3, 3, data, where)); break;
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


  int set_x0_mode(int mode) override {
    if (mode < GSPM_X0_PREV || mode > GSPM_X0_LEARNED) {
      set_error("set_x0_mode: bad mode %d", mode);
      return GSPM_EINVAL;
    }
    if (mode == GSPM_X0_LEARNED && nseg_ != 1) {
      set_error("set_x0_mode: the learned initial guess is single-mesh only");
      return GSPM_ESTATE;
    }
    if (mode == GSPM_X0_LEARNED && !net_ready_) {
      set_error("set_x0_mode: the learned warm start needs parameters (gspm_mpnn_set_params)");
      return GSPM_ESTATE;
    }
    x0_mode_ = mode;
    return GSPM_OK;
  }

  // out != NULL: read parameters; in != NULL: write them (and refresh the BF16 copies)
  int mpnn_params(float* out, const float* in, int64_t count) override {
    if (count != kParams) {
      set_error("mpnn params: count %lld, the network has %d", (long long)count, kParams);
      return GSPM_EINVAL;
    }
    ST(net_alloc());
    if (in) {
      CK(cudaMemcpyAsync(params_, in, kParams * sizeof(float), cudaMemcpyHostToDevice, L_.stream));
      CK(cudaMemsetAsync(adam_m_, 0, kParams * sizeof(float), L_.stream));
      CK(cudaMemsetAsync(adam_v_, 0, kParams * sizeof(float), L_.stream));
      adam_t_ = 0;
      CK(mpnn_refresh_bf16(L_, WinT_, WT_, params_));
      CK(cudaStreamSynchronize(L_.stream));
      net_ready_ = true;
    }
    if (out) {
      CK(cudaMemcpyAsync(out, params_, kParams * sizeof(float), cudaMemcpyDeviceToHost, L_.stream));
      CK(cudaStreamSynchronize(L_.stream));
    }
    return GSPM_OK;
  }

  int mpnn_predict(const double* m, const double* up, const double* up2, double* out, int what,
                   int where) override {
    if (!net_ready_) {
      set_error("mpnn_predict: no parameters set");
      return GSPM_ESTATE;
    }
    if (!m || !out || (what != 0 && what != 1)) {
      set_error("mpnn_predict: need m, out and what in {0, 1}");
      return GSPM_EINVAL;
    }
    ST(import_field(m, where, 3, ms_, ld_, 1, mag_));
    if (up) ST(import_field(up, where, 3, uin_, 1, 3, nullptr));
    else CK(cudaMemsetAsync(uin_, 0, 3 * n_ * sizeof(T), L_.stream));
    if (up2) ST(import_field(up2, where, 3, uin2_, 1, 3, nullptr));
    else CK(cudaMemsetAsync(uin2_, 0, 3 * n_ * sizeof(T), L_.stream));
    ST(net_forward(ms_, uin_, uin2_, nullptr));
    if (what == 0) {
      CK(mpnn_output<T>(L_, n_, net_, H_[kLayers], 0, Y_, nullptr, nullptr, 0.0, nullptr));
      CK((launch_convert<float, T>(L_, 3 * n_, Y_, utmp_)));
    } else {
      CK(mpnn_output(L_, n_, net_, H_[kLayers], 1, nullptr, uin_, uin2_, u_scale(), utmp_));
    }
    ST(export_field(utmp_, 1, 3, 3, out, where));
    CK(cudaStreamSynchronize(L_.stream));
    return check_net();
  }

  int mpnn_dataset_reserve(int capacity) override {
    if (capacity < 1) {
      set_error("mpnn_dataset_reserve: capacity must be positive");
      return GSPM_EINVAL;
    }
    ST(net_alloc());
    if (ds_F_) {
      set_error("mpnn_dataset_reserve: dataset already reserved");
      return GSPM_ESTATE;
    }
    ST(mem_.alloc(&ds_F_, (int64_t)capacity * n_ * kFeat));
    ST(mem_.alloc(&ds_T_, (int64_t)capacity * n_ * 3));
    ds_cap_ = capacity;
    ds_n_ = 0;
    return GSPM_OK;
  }

  // one (m, u_prev, u_prev2) -> u* pair: stores the features and the target
  // t = (u* - (2 u_prev - u_prev2)) / u_s
  int mpnn_dataset_add(const double* m, const double* up, const double* up2, const double* ustar,
                       int where, int* index) override {
    if (!ds_F_ || ds_n_ >= ds_cap_) {
      set_error("mpnn_dataset_add: dataset not reserved or full");
      return GSPM_ESTATE;
    }
    if (!m || !ustar) {
      set_error("mpnn_dataset_add: need m and u*");
      return GSPM_EINVAL;
    }
    ST(import_field(m, where, 3, ms_, ld_, 1, mag_));
    if (up) ST(import_field(up, where, 3, uin_, 1, 3, nullptr));
    else CK(cudaMemsetAsync(uin_, 0, 3 * n_ * sizeof(T), L_.stream));
    if (up2) ST(import_field(up2, where, 3, uin2_, 1, 3, nullptr));
    else CK(cudaMemsetAsync(uin2_, 0, 3 * n_ * sizeof(T), L_.stream));
    ST(import_field(ustar, where, 3, utmp_, 1, 3, nullptr));
    __nv_bfloat16* F = ds_F_ + (int64_t)ds_n_ * n_ * kFeat;
    CK(mpnn_features<T>(L_, n_, ms_, ld_, mag_, uin_, uin2_, P_.l100, P_.l111, l_scale(),
                        u_scale(), F));
    CK(launch_target(ds_T_ + (int64_t)ds_n_ * n_ * 3));
    if (index) *index = ds_n_;
    ++ds_n_;
    if (where == GSPM_HOST) CK(cudaStreamSynchronize(L_.stream));
    return GSPM_OK;
  }

  int mpnn_loss_grad(int pair, double* loss, float* grad) override {
    if (!net_ready_ || pair < 0 || pair >= ds_n_) {
      set_error("mpnn_loss_grad: need parameters and a stored pair");
      return GSPM_EINVAL;
    }
    ST(net_step(pair, /*update=*/false, 0.0));
    float l = 0.f;
    CK(cudaMemcpyAsync(&l, loss_, sizeof(float), cudaMemcpyDeviceToHost, L_.stream));
    if (grad) CK(cudaMemcpyAsync(grad, grad_, kParams * sizeof(float), cudaMemcpyDeviceToHost, L_.stream));
    CK(cudaStreamSynchronize(L_.stream));
    ST(check_net());
    if (loss) *loss = (double)l / (3.0 * (double)n_);
    return GSPM_OK;
  }

  // iterations of Adam, each on one stored pair drawn with a splitmix64 stream of `seed`
  int mpnn_train(int iters, double lr, uint64_t seed, double* l0, double* l1) override {
    if (!net_ready_ || ds_n_ < 1 || iters < 1) {
      set_error("mpnn_train: need parameters, a non-empty dataset and iterations >= 1");
      return GSPM_EINVAL;
    }
    float lf = 0.f, ll = 0.f;
    for (int it = 0; it < iters; ++it) {
      uint64_t z = seed + (uint64_t)(it + 1) * 0x9E3779B97F4A7C15ull;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      const int pair = (int)(z % (uint64_t)ds_n_);
      ST(net_step(pair, /*update=*/true, lr));
      if (it == 0) CK(cudaMemcpyAsync(&lf, loss_, sizeof(float), cudaMemcpyDeviceToHost, L_.stream));
    }
    CK(cudaMemcpyAsync(&ll, loss_, sizeof(float), cudaMemcpyDeviceToHost, L_.stream));
    CK(cudaStreamSynchronize(L_.stream));
    ST(check_net());
    if (l0) *l0 = (double)lf / (3.0 * (double)n_);
    if (l1) *l1 = (double)ll / (3.0 * (double)n_);
    return GSPM_OK;
  }

 private:
  // kSlotMs2 / kSlotMech2: the correction solves of the refinement (mixed precision)
  static constexpr int kSlotMs = 0, kSlotMech = 1, kSlotGs0 = 2, kSlotGs1 = 3, kSlotGs2 = 4,
                       kSlotGsD = 5, kSlotMs2 = 6, kSlotMech2 = 7, kSolveSlots = 8;
  // stopping tolerance of the first FP32 solve of a refined K^ms / K^mech solve (the correction
  // solve then reaches the requested one); above the recursive-vs-true residual gap of FP32 CG
  // on these operators (5e-5 of ||b|| at 3M nodes)
  static constexpr double kRtolInner = 1e-4;

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

  DevParams dev_params() const {
    DevParams D;
    D.kappa = P_.kappa;
    D.me_coef = P_.me_coef;
    D.l100 = P_.l100;
    D.l111 = P_.l111;
    D.C11 = P_.C11;
    D.C12 = P_.C12;
    D.C44 = P_.C44;
    for (int k = 0; k < 9; ++k) D.Nd[k] = P_.Nd[k];
    D.dtau = P_.dtau;
    D.alpha = P_.alpha;
    for (int k = 0; k < 9; ++k) D.R[k] = P_.R[k];
    D.rotated = P_.rotated;
    return D;
  }

  // host/device [n][nc] float64 (unique order) -> internal array dst(i, c) = dst[i*ns + c*cs]
  template <typename X>
  int import_field(const double* src, int where, int nc, X* dst, int64_t cs, int64_t ns,
                   const uint8_t* mask, X* lo = nullptr) {
    const double* s = src;
    if (where == GSPM_HOST) {
      CK(cudaMemcpyAsync(stage_, src, nodes_ * nc * sizeof(double), cudaMemcpyHostToDevice,
                         L_.stream));
      s = stage_;
    } else if (where != GSPM_DEVICE) {
      set_error("bad `where` %d", where);
      return GSPM_EINVAL;
    }
    CK(launch_import<X>(L_, n_, nc, s, perm_, dst, cs, ns, mask, lo));
    return GSPM_OK;
  }

  template <typename X>
  int export_field(const X* src, int64_t cs, int64_t ns, int nc, double* dst, int where,
                   const X* lo = nullptr) {
    if (where == GSPM_DEVICE) {
      CK(launch_export<X>(L_, n_, nc, src, cs, ns, perm_, dst, lo));
    } else if (where == GSPM_HOST) {
      CK(launch_export<X>(L_, n_, nc, src, cs, ns, perm_, stage_, lo));
      CK(cudaMemcpyAsync(dst, stage_, nodes_ * nc * sizeof(double), cudaMemcpyDeviceToHost,
                         L_.stream));
    } else {
      set_error("bad `where` %d", where);
      return GSPM_EINVAL;
    }
    return GSPM_OK;
  }

  // Launch CG iterations in chunks; after each chunk read the number of still-active
  // segments (one int), then the per-segment status blocks once at the end.
  template <class Iter>
  int cg_loop(int slot, Iter iter, std::vector<SolveInfo>* info) {
    CGState* st = cg_ + (int64_t)slot * nseg_;
    int chunk = std::max(1, pred_[slot]);
    int launched = 0;
    for (;;) {
      for (int c = 0; c < chunk; ++c) ST(iter());
      launched += chunk;
      CK(cudaMemcpyAsync(host_active_, nactive_ + slot, sizeof(int), cudaMemcpyDeviceToHost,
                         L_.stream));
      CK(cudaStreamSynchronize(L_.stream));
      if (*host_active_ <= 0 || launched > opt_.max_iter + 1) break;
      // first solve of a kind: grow geometrically; afterwards small top-up chunks
      chunk = seen_[slot] ? 3 : std::max(2, std::min(32, launched / 4));
    }
    CK(cudaMemcpyAsync(host_state_, st, nseg_ * sizeof(CGState), cudaMemcpyDeviceToHost,
                       L_.stream));
    CK(cudaStreamSynchronize(L_.stream));
    info->assign(nseg_, SolveInfo());
    int itmax = 0;
    for (int sg = 0; sg < nseg_; ++sg) {
      const CGState& c = host_state_[sg];
      int it = 0;
      double rel = 0.0;
      for (int k = 0; k < c.nr; ++k) {
        it = std::max(it, c.r[k].iters);
        const double bb = c.r[k].bb;
        rel = std::max(rel, bb > 0 ? std::sqrt(c.r[k].rr / bb) : 0.0);
      }
      (*info)[sg].iters = it;
      (*info)[sg].relres = rel;
      (*info)[sg].noconv = c.noconv;
      itmax = std::max(itmax, it);
    }
    pred_[slot] = std::max(1, itmax);
    seen_[slot] = 1;
    return GSPM_OK;
  }

  // K x = b for one K^ms (B = 1) or K^mech (B = 9) solve.  Mixed precision: iterative
  // refinement (Wilkinson's scheme with the working-precision solver run in FP32): a first FP32
  // CG solve to kRtolInner leaves x; a second CG restarts from x, its initial residual b - K x
  // formed to twice the working precision (k_cg_init), and accumulates the correction in the
  // separate array dx_ from zero until ||r|| < rtol ||b||; then (x, xlo) = x + dx as an
  // unevaluated FP32 sum, so the solution keeps the digits that FP32 rounding of x would lose.
  // The recursive residual of a single FP32 solve drifts from b - K x by about
  // eps_32 ||K|| ||x|| (5e-5 of ||b|| at 3M nodes); the correction solve's drift is that of the
  // much smaller dx.  FP64 (xlo == NULL): one solve.
  int solve_system(int slot, const T* val, int B, const T* b, T* x, T* xlo, double rtol,
                   std::vector<SolveInfo>* info) {
    const int epr = B == 9 ? 3 : 1;
    const int slot2 = slot == kSlotMs ? kSlotMs2 : kSlotMech2;
    if (!xlo) {
      ST(solve_general(slot, val, B, b, x, x, rtol, info));
    } else {
      const int64_t len = epr * n_;
      std::vector<SolveInfo> i1, i2;
      CK(cudaMemsetAsync(xlo, 0, len * sizeof(T), L_.stream));
      ST(solve_general(slot, val, B, b, x, x, std::max(rtol, kRtolInner), &i1));
      CK(cudaMemsetAsync(dx_, 0, len * sizeof(T), L_.stream));
      ST(solve_general(slot2, val, B, b, x, dx_, rtol, &i2));
      TK(GSPM_KCLASS_CG_INIT, launch_refine_add<T>(L_, len, x, xlo, dx_));
      if (!capturing_) {
        info->assign(nseg_, SolveInfo());
        for (int sg = 0; sg < nseg_; ++sg) {
          (*info)[sg].iters = i1[sg].iters + i2[sg].iters;
          (*info)[sg].relres = i2[sg].relres;
          (*info)[sg].noconv = i1[sg].noconv + i2[sg].noconv;
        }
      }
    }
    if (tres_on_)
      TK(GSPM_KCLASS_CG_INIT, launch_true_res<T>(L_, A_, SG_, val, B, b, x, xlo, red_, tres_ + (B == 9 ? 2 * nseg_ : 0)));
    return GSPM_OK;
  }

  // CG for K x = b (B = 1 scalar K^ms, B = 9 block K^mech), pinned or singular form, started from
  // x0 (read only) with the iterates accumulated into x: x == x0 is the plain solve; x != x0
  // (zero on entry) is the correction solve of solve_system, whose solution is x0 + x
  int solve_general(int slot, const T* val, int B, const T* b, const T* x0, T* x, double rtol,
                    std::vector<SolveInfo>* info) {
    Trace trace(B == 9 ? "cg_mech" : "cg_ms");
    CGState* st = cg_ + (int64_t)slot * nseg_;
    int* na = nactive_ + slot;
    const int epr = B == 9 ? 3 : 1;
    const int64_t len = epr * n_;
    double* bmean = proj_;
    double* xpin = proj_ + 3 * nseg_;
    CK(cudaMemsetAsync(na, 0, sizeof(int), L_.stream));
    const bool restart = x != x0;
    if (pinned_) {
      // the pinned system (Sec. 2.5): x0 moved to zero at the pinned node
      if (!restart) TK(GSPM_KCLASS_CG_INIT, launch_pin_shift<T>(L_, A_, SG_, epr, x, xpin));
    } else {
      // the consistent singular system: x0 minus its per-segment mean of each component, and b
      // minus its mean
      if (!restart) {
        TK(GSPM_KCLASS_CG_INIT, launch_wsum<T>(L_, SG_, epr, x, 1, epr, nullptr, wmean_, xpin, nullptr, red_));
        TK(GSPM_KCLASS_CG_INIT, launch_seg_shift<T>(L_, A_, SG_, epr, x, xpin));
      }
      TK(GSPM_KCLASS_CG_INIT, launch_wsum<T>(L_, SG_, epr, b, 1, epr, nullptr, wmean_, bmean, nullptr, red_));
    }
    // two-level preconditioned CG on the singular systems (the pinned form stays plain)
    const bool pc = pc_ && !pinned_;
    const typename CoarseStore<T>::type* cinv = epr == 3 ? cinv3_ : cinv1_;
    const DSymTiles& TL = epr == 3 ? TL3_ : TL1_;
    const int64_t* rco = epr == 3 ? rc_off3_ : rc_off1_;
    const T* dinv = epr == 3 ? dinv3_ : dinv1_;
    auto precondition = [&](T* z, int init) -> int {
      TK(GSPM_KCLASS_CG_VEC, launch_restrict<T>(L_, CC_, epr, r_, rco, rc_));
      TK(GSPM_KCLASS_CG_VEC, launch_coarse_symv<T>(L_, CC_, TL, epr, cinv, rco, rc_, qsym_, ec_));
      TK(GSPM_KCLASS_CG_VEC, launch_pcg_z<T>(L_, SG_, CC_, epr, r_, dinv, ec_, z, st, init, red_));
      return GSPM_OK;
    };
    TK(GSPM_KCLASS_CG_INIT, launch_cg_init<T>(L_, A_, SG_, val, B, b, x0, r_, p_, st, na, rtol, opt_.max_iter, red_, pinned_ ? nullptr : bmean, pinned_, pc ? 1 : 0));
    if (pc) ST(precondition(p_, 1));
    // singular system: p0 projected off the constants
    if (!pinned_) TK(GSPM_KCLASS_CG_INIT, launch_cg_psub<T>(L_, A_, SG_, epr, p_, st));
    auto iter = [&]() -> int {
      TK(B == 9 ? GSPM_KCLASS_SPMV_MECH : GSPM_KCLASS_SPMV_MS, launch_cg_spmv<T>(L_, A_, SG_, val, B, 1, len, p_, q_, st, red_, B == 9 ? var_block_ : var_scalar_, pinned_, 1));
      TK(GSPM_KCLASS_CG_VEC, launch_cg_update<T>(L_, SG_, epr, 1, len, x, r_, p_, q_, st, na, red_));
      if (pc) {
        // z into q (free after the update), then p = z + beta p
        ST(precondition(q_, 0));
        TK(GSPM_KCLASS_CG_VEC, launch_cg_pupdate<T>(L_, SG_, epr, 1, len, q_, p_, st, loop_));
      } else {
        TK(GSPM_KCLASS_CG_VEC, launch_cg_pupdate<T>(L_, SG_, epr, 1, len, r_, p_, st, loop_));
      }
      return GSPM_OK;
    };
    if (capturing_)
      ST(cg_graph_loop(slot, iter, B == 9 ? 1 : 0, pc ? 7 : 3));
    else
      ST(cg_loop(slot, iter, info));
    // singular system: move the solution to the pinned one (zero at the pinned node)
    if (!pinned_) TK(GSPM_KCLASS_CG_INIT, launch_pin_shift<T>(L_, A_, SG_, epr, x, xpin));
    TK(GSPM_KCLASS_CG_INIT, launch_cg_zero<T>(L_, SG_, epr, x, st));
    return GSPM_OK;
  }

  // (M + c eps K) g = M f for nr right-hand sides held in x slots [slot0, slot0 + nr); info[k]
  // receives, per segment, the solve of right-hand side k
  int solve_gs(int slot, const T* aval, int slot0, int nr, std::vector<SolveInfo>* info) {
    Trace trace(aval == Aeps_ ? "cg_gs_eps" : "cg_gs_alpha_eps");
    CGState* st = cg_ + (int64_t)slot * nseg_;
    int* na = nactive_ + slot;
    T* x = x_ + slot0 * ld_;
    CK(cudaMemsetAsync(na, 0, sizeof(int), L_.stream));
    const T* dinv = aval == Aeps_ ? dgs_eps_ : dgs_aeps_;  // NULL: plain CG
    TK(GSPM_KCLASS_CG_INIT, launch_cg_init_gs<T>(L_, A_, SG_, aval, M_, nr, ld_, x, r_, p_, st, na, opt_.rtol_gs, opt_.max_iter, red_, dinv));
    auto iter = [&]() -> int {
      TK(GSPM_KCLASS_SPMV_GS, launch_cg_spmv<T>(L_, A_, SG_, aval, 1, nr, ld_, p_, q_, st, red_, var_gs_, 0, 0));
      TK(GSPM_KCLASS_CG_VEC, launch_cg_update<T>(L_, SG_, 1, nr, ld_, x, r_, p_, q_, st, na, red_, dinv));
      TK(GSPM_KCLASS_CG_VEC, launch_cg_pupdate<T>(L_, SG_, 1, nr, ld_, r_, p_, st, loop_, dinv));
      return GSPM_OK;
    };
    if (capturing_) return cg_graph_loop(slot, iter, 2, 3);
    std::vector<SolveInfo> tot;
    ST(cg_loop(slot, iter, &tot));
    for (int k = 0; k < nr; ++k) {
      info[k].assign(nseg_, SolveInfo());
      for (int sg = 0; sg < nseg_; ++sg) {
        const CGRhs& c = host_state_[sg].r[k];
        info[k][sg].iters = c.iters;
        info[k][sg].relres = c.bb > 0 ? std::sqrt(c.rr / c.bb) : 0.0;
        info[k][sg].noconv = k == 0 ? tot[sg].noconv : 0;
      }
    }
    return GSPM_OK;
  }

  // Device copy of the two-level preconditioner: aggregates in batch numbering (segment s's
  // aggregates follow those of the segments before it), per-segment dense inverse blocks for
  // the scalar (K^ms) and 3-component (K^mech) coarse operators, inverse diagonals.
  int init_coarse() {
    const int S = nseg_;
    std::vector<int32_t> agg0(S + 1, 0);
    for (int sg = 0; sg < S; ++sg) agg0[sg + 1] = agg0[sg] + (int32_t)hb_.coarse[sg].n_agg;
    const int64_t na = agg0[S];
    std::vector<int32_t> aor(n_, -1), aseg(na);
    std::vector<int64_t> cnt(na + 1, 0);
    for (int sg = 0; sg < S; ++sg) {
      const HostCoarse& hc = hb_.coarse[sg];
      for (int64_t i = 0; i < hb_.seg_nrow[sg]; ++i) {
        const int32_t I = agg0[sg] + hc.agg[i];
        aor[hb_.seg_row0[sg] + i] = I;
        ++cnt[I + 1];
      }
      for (int64_t I = agg0[sg]; I < agg0[sg + 1]; ++I) aseg[I] = sg;
    }
    for (int64_t I = 0; I < na; ++I) cnt[I + 1] += cnt[I];
    std::vector<int32_t> aptr(cnt.begin(), cnt.end()), arows(cnt[na]);
    {
      std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
      for (int64_t row = 0; row < n_; ++row)
        if (aor[row] >= 0) arows[fill[aor[row]]++] = (int32_t)row;
    }
    // the inverses' stored upper-triangle tiles (see launch_coarse_symv): the symmetric part of
    // the FP64 inverse rounded once to the storage type, checked positive definite after the
    // rounding (coarse_round_spd)
    using S16 = typename CoarseStore<T>::type;
    constexpr int64_t TS = coarse_tile<T>();
    struct Tiles {
      std::vector<S16> data;
      std::vector<int32_t> tseg, tI, tJ, Tn;
      std::vector<int64_t> t0, q0;
      int64_t qn = 0;
    } tl[2];  // [0]: 3 components (K^mech), [1]: 1 (K^ms)
    for (int q = 0; q < 2; ++q) {
      const int e = q == 0 ? 3 : 1;
      Tiles& X = tl[q];
      X.t0.resize(S);
      X.Tn.resize(S);
      X.q0.resize(S);
      for (int sg = 0; sg < S; ++sg) {
        const HostCoarse& hc = hb_.coarse[sg];
        const std::vector<double>& inv = e == 3 ? hc.store_mech : hc.store_ms;
        const int64_t nc = e * hc.n_agg, Tn = (nc + TS - 1) / TS;
        X.t0[sg] = (int64_t)X.tseg.size();
        X.Tn[sg] = (int32_t)Tn;
        X.q0[sg] = X.qn;
        X.qn += Tn * TS * Tn;
        for (int64_t I = 0; I < Tn; ++I)
          for (int64_t J = I; J < Tn; ++J) {
            X.tseg.push_back(sg);
            X.tI.push_back((int32_t)I);
            X.tJ.push_back((int32_t)J);
            const size_t base = X.data.size();
            X.data.resize(base + TS * TS, S16(0));
            for (int64_t r = 0; r < TS && I * TS + r < nc; ++r)
              for (int64_t c = 0; c < TS && J * TS + c < nc; ++c) {
                const int64_t gi = I * TS + r, gj = J * TS + c;
                X.data[base + r * TS + c] = to_store<S16>(inv[gi * nc + gj]);
              }
          }
      }
    }
    std::vector<T> d3(3 * n_, T(0)), d1(n_, T(0));
    for (int sg = 0; sg < S; ++sg) {
      const HostCoarse& hc = hb_.coarse[sg];
      const int64_t r0 = hb_.seg_row0[sg];
      for (int64_t i = 0; i < hb_.seg_nrow[sg]; ++i) {
        d1[r0 + i] = (T)hc.dinv_ms[i];
        for (int a = 0; a < 3; ++a) d3[3 * (r0 + i) + a] = (T)hc.dinv_mech[3 * i + a];
      }
    }
    int64_t max_q = 0;
    for (int q = 0; q < 2; ++q) {
      Tiles& X = tl[q];
      const int64_t nt = (int64_t)X.tseg.size();
      max_q = std::max(max_q, X.qn);
      S16* d_data;
      int32_t *d_tseg, *d_tI, *d_tJ, *d_Tn;
      int64_t *d_t0, *d_q0;
      ST(mem_.alloc(&d_data, nt * TS * TS));
      ST(mem_.alloc(&d_tseg, nt));
      ST(mem_.alloc(&d_tI, nt));
      ST(mem_.alloc(&d_tJ, nt));
      ST(mem_.alloc(&d_t0, S));
      ST(mem_.alloc(&d_Tn, S));
      ST(mem_.alloc(&d_q0, S));
      CK(cudaMemcpy(d_data, X.data.data(), X.data.size() * sizeof(S16), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(d_tseg, X.tseg.data(), nt * 4, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(d_tI, X.tI.data(), nt * 4, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(d_tJ, X.tJ.data(), nt * 4, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(d_t0, X.t0.data(), S * 8, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(d_Tn, X.Tn.data(), S * 4, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(d_q0, X.q0.data(), S * 8, cudaMemcpyHostToDevice));
      (q == 0 ? cinv3_ : cinv1_) = d_data;
      (q == 0 ? TL3_ : TL1_) = DSymTiles{nt, d_tseg, d_tI, d_tJ, d_t0, d_Tn, d_q0};
    }
    ST(mem_.alloc(&qsym_, max_q));
    int32_t *d_aor, *d_aptr, *d_arows, *d_aseg, *d_agg0;
    ST(mem_.alloc(&d_aor, n_));
    ST(mem_.alloc(&d_aptr, na + 1));
    ST(mem_.alloc(&d_arows, (int64_t)arows.size()));
    ST(mem_.alloc(&d_aseg, na));
    ST(mem_.alloc(&d_agg0, S + 1));
    ST(mem_.alloc(&dinv3_, 3 * n_));
    ST(mem_.alloc(&dinv1_, n_));
    // rc: per segment a block zero-padded to whole tiles
    std::vector<int64_t> rco3(S), rco1(S);
    int64_t r3 = 0, r1 = 0;
    for (int sg = 0; sg < S; ++sg) {
      const int64_t a = hb_.coarse[sg].n_agg;
      rco3[sg] = r3;
      rco1[sg] = r1;
      r3 += coarse_ld<T>(3 * a);
      r1 += coarse_ld<T>(a);
    }
    ST(mem_.alloc(&rc_, std::max(r3, r1)));
    CK(cudaMemset(rc_, 0, std::max(r3, r1) * sizeof(T)));
    ST(mem_.alloc(&rc_off3_, S));
    ST(mem_.alloc(&rc_off1_, S));
    CK(cudaMemcpy(rc_off3_, rco3.data(), S * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(rc_off1_, rco1.data(), S * 8, cudaMemcpyHostToDevice));
    ST(mem_.alloc(&ec_, 3 * na));
    CK(cudaMemcpy(d_aor, aor.data(), n_ * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_aptr, aptr.data(), (na + 1) * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_arows, arows.data(), arows.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_aseg, aseg.data(), na * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_agg0, agg0.data(), (S + 1) * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dinv3_, d3.data(), 3 * n_ * sizeof(T), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dinv1_, d1.data(), n_ * sizeof(T), cudaMemcpyHostToDevice));
    int contig = 1;
    for (int64_t I = 0; I < na && contig; ++I)
      for (int32_t q = aptr[I]; q < aptr[I + 1]; ++q)
        if (arows[q] != arows[aptr[I]] + (q - aptr[I])) {
          contig = 0;
          break;
        }
    CC_ = DCoarse{na, d_aor, d_aptr, d_arows, d_aseg, d_agg0, contig};
    pc_ = true;
    return GSPM_OK;
  }

  // per-segment device scalars: m_bar [3S], m_bar* [3S], E_bar [6S], <|dm|> [S], H/m_s [3S],
  // 1/(magnetic nodes) [S], volume averages [9S]; then C^-1 sigma_ext [6]
  static constexpr int kScalPerSeg = 26;
  double* mbar() const { return scal_; }
  double* mbar_s() const { return scal_ + 3 * nseg_; }
  double* ebar() const { return scal_ + 6 * nseg_; }
  double* dmv() const { return scal_ + 12 * nseg_; }
  double* hz() const { return scal_ + 13 * nseg_; }
  double* inv_nmag() const { return scal_ + 16 * nseg_; }
  double* avg() const { return scal_ + 17 * nseg_; }
  double* eext() const { return scal_ + 26 * nseg_; }

  // Segment tables and the work items of the reducing kernels.  List k - 1 serves kernels that
  // keep k blocks resident per SM: about k x SMs items, each segment getting a share
  // proportional to its slices (at least one item, at most one per slice), its slices split
  // evenly, so every block of the single resident wave reduces one item.
  // Work-item lists over per-segment runs of units (slices, aggregates or coarse rows): unit
  // u0[s] + i, i < nu[s], of segment s.  List k - 1 serves kernels that keep k blocks resident
  // per SM: about k x SMs items, each segment getting a share proportional to its units (at
  // least one item, at most one per unit), its units split evenly.
  int make_item_lists(const std::vector<int64_t>& u0, const std::vector<int64_t>& nu,
                      ItemList* lists, int* max_items) {
    const int S = (int)nu.size();
    int64_t total = 0;
    for (int64_t v : nu) total += v;
    for (int k = 1; k <= kItemLists; ++k) {
      const double target = (double)k * L_.sms;
      std::vector<int32_t> iseg, isl0, isl1, sitem0(S), snit(S);
      for (int sg = 0; sg < S; ++sg) {
        const int64_t a = u0[sg], n = nu[sg];
        int64_t ni = std::llround(target * (double)n / (double)std::max<int64_t>(1, total));
        ni = std::max<int64_t>(1, std::min<int64_t>(std::max<int64_t>(1, n), ni));
        sitem0[sg] = (int32_t)iseg.size();
        for (int64_t i = 0; i < ni; ++i) {
          iseg.push_back(sg);
          isl0.push_back((int32_t)(a + i * n / ni));
          isl1.push_back((int32_t)(a + (i + 1) * n / ni));
        }
        snit[sg] = (int32_t)ni;
      }
      const int ni = (int)iseg.size();
      int32_t *d_iseg, *d_isl0, *d_isl1, *d_si0, *d_sni;
      ST(mem_.alloc(&d_iseg, ni));
      ST(mem_.alloc(&d_isl0, ni));
      ST(mem_.alloc(&d_isl1, ni));
      ST(mem_.alloc(&d_si0, S));
      ST(mem_.alloc(&d_sni, S));
      CK(cudaMemcpy(d_iseg, iseg.data(), ni * 4, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(d_isl0, isl0.data(), ni * 4, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(d_isl1, isl1.data(), ni * 4, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(d_si0, sitem0.data(), S * 4, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(d_sni, snit.data(), S * 4, cudaMemcpyHostToDevice));
      lists[k - 1] = ItemList{ni, d_iseg, d_isl0, d_isl1, d_si0, d_sni};
      *max_items = std::max(*max_items, ni);
    }
    return GSPM_OK;
  }

  int init_segments() {
    const int S = nseg_;
    int32_t* d_sos;
    int64_t *d_r0, *d_nr, *d_pin;
    unsigned* d_cnt;
    ST(mem_.alloc(&d_sos, nslices_));
    ST(mem_.alloc(&d_r0, S));
    ST(mem_.alloc(&d_nr, S));
    ST(mem_.alloc(&d_pin, S));
    ST(mem_.alloc(&d_cnt, S));
    CK(cudaMemcpy(d_sos, hb_.seg_of_slice.data(), nslices_ * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_r0, hb_.seg_row0.data(), S * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_nr, hb_.seg_nrow.data(), S * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_pin, hb_.seg_pin.data(), S * 8, cudaMemcpyHostToDevice));
    CK(cudaMemset(d_cnt, 0, S * sizeof(unsigned)));
    DSeg g{};
    g.nseg = S;
    g.seg_of_slice = d_sos;
    g.seg_row0 = d_r0;
    g.seg_nrow = d_nr;
    g.seg_pin = d_pin;
    g.counter = d_cnt;
    std::vector<int64_t> u0(S), nu(S);
    for (int sg = 0; sg < S; ++sg) {
      u0[sg] = hb_.seg_sl0[sg];
      nu[sg] = hb_.seg_nsl[sg];
    }
    int max_items = 0;
    ST(make_item_lists(u0, nu, g.list, &max_items));
    item_slices_ = (int)((nslices_ + g.list[0].nitems - 1) / g.list[0].nitems);
    SG_ = g;
    nitems_ = max_items;
    ST(mem_.alloc(&red_.partial, (int64_t)max_items * kRedComp));
    return GSPM_OK;
  }

  double l_scale() const { return std::max(std::fabs(P_.l100), std::fabs(P_.l111)) > 0
                                      ? std::max(std::fabs(P_.l100), std::fabs(P_.l111)) : 1.0; }
  double u_scale() const { return l_scale() * h_scale_; }

  int net_alloc() {
    if (params_) return GSPM_OK;
    if (nseg_ != 1) {
      set_error("the learned initial guess is single-mesh only");
      return GSPM_ESTATE;
    }
    CK(mpnn_setup_smem());
    ST(mem_.alloc(&params_, kParams));
    ST(mem_.alloc(&grad_, kParams));
    ST(mem_.alloc(&adam_m_, kParams));
    ST(mem_.alloc(&adam_v_, kParams));
    ST(mem_.alloc(&loss_, 4));
    ST(mem_.alloc(&WinT_, kHid * kFeat));
    for (int l = 0; l < kLayers; ++l) ST(mem_.alloc(&WT_[l], kHid * 2 * kHid));
    ST(mem_.alloc(&F_in_, n_ * kFeat));
    for (int l = 0; l <= kLayers; ++l) ST(mem_.alloc(&H_[l], n_ * kHid));
    ST(mem_.alloc(&Y_, 3 * n_));
    net_.WinT = WinT_;
    net_.b_in = params_ + kOffBin;
    for (int l = 0; l < kLayers; ++l) {
      net_.WT[l] = WT_[l];
      net_.Wf[l] = params_ + kOffW[l];
      net_.b[l] = params_ + kOffW[l] + 2 * kHid * kHid;
    }
    net_.Wout = params_ + kOffWout;
    net_.bout = params_ + kOffBout;
    net_.A = agg_;
    net_.At = aggT_;
    ST(mem_.alloc(&mpnn_err_, 1));
    CK(cudaMemset(mpnn_err_, 0, sizeof(int)));
    net_.err = mpnn_err_;
    return GSPM_OK;
  }

  int net_train_alloc() {
    if (dHa_) return GSPM_OK;
    for (int l = 0; l < kLayers; ++l) ST(mem_.alloc(&Z_[l], n_ * kHid));
    ST(mem_.alloc(&dHa_, n_ * kHid));
    ST(mem_.alloc(&dHb_, n_ * kHid));
    ST(mem_.alloc(&dZ_, n_ * kHid));
    ST(mem_.alloc(&part_, (int64_t)L_.max_blocks * (2 * kHid * kHid + kHid)));
    return GSPM_OK;
  }

  // features of (m, up, up2) into F_in_, then the forward pass (Z saved when training)
  int net_forward(const T* m, const T* up, const T* up2, __nv_bfloat16* const* Z) {
    CK(mpnn_features<T>(L_, n_, m, ld_, mag_, up, up2, P_.l100, P_.l111, l_scale(), u_scale(),
                        F_in_));
    CK(mpnn_forward(L_, n_, A_, net_, F_in_, H_, Z));
    return GSPM_OK;
  }

  int net_step(int pair, bool update, double lr) {
    ST(net_train_alloc());
    const __nv_bfloat16* F = ds_F_ + (int64_t)pair * n_ * kFeat;
    CK(mpnn_forward(L_, n_, A_, net_, F, H_, Z_));
    CK(mpnn_output<T>(L_, n_, net_, H_[kLayers], 0, Y_, nullptr, nullptr, 0.0, nullptr));
    CK(mpnn_backward(L_, n_, A_, net_, F, H_, Z_, Y_, ds_T_ + (int64_t)pair * n_ * 3, dHa_, dHb_,
                     dZ_, part_, grad_, loss_));
    if (update) {
      ++adam_t_;
      CK(mpnn_adam(L_, params_, grad_, adam_m_, adam_v_, (float)lr, adam_t_));
      CK(mpnn_refresh_bf16(L_, WinT_, WT_, params_));
    }
    return GSPM_OK;
  }

  // t = (u* - (2 up - up2)) / u_s from utmp_ (u*), uin_, uin2_
  cudaError_t launch_target(float* t) {
    return launch_scaled_diff<T>(L_, 3 * n_, utmp_, uin_, uin2_, 1.0 / u_scale(), t);
  }

  // x0 of the mechanical CG, leaving u_prev2 <- u_prev and u <- x0 (u_prev = u on entry)
  int mech_initial_guess(const T* m, int mode) {
    const int64_t len = 3 * n_;
    switch (mode) {
      case GSPM_X0_PREV:
        CK(cudaMemcpyAsync(u2_, u_, len * sizeof(T), cudaMemcpyDeviceToDevice, L_.stream));
        break;
      case GSPM_X0_ZERO:
        CK(cudaMemcpyAsync(u2_, u_, len * sizeof(T), cudaMemcpyDeviceToDevice, L_.stream));
        CK(cudaMemsetAsync(u_, 0, len * sizeof(T), L_.stream));
        break;
      case GSPM_X0_EXTRAPOLATE:
        TK(GSPM_KCLASS_POINTWISE, launch_extrapolate<T>(L_, len, u_, u2_));
        break;
      case GSPM_X0_LEARNED:
        if (!net_ready_) {
          set_error("learned warm start requested without parameters");
          return GSPM_ESTATE;
        }
        ST(timed(GSPM_KCLASS_LEARNED, [&]() -> int {
          ST(net_forward(m, u_, u2_, nullptr));
          CK(mpnn_output(L_, n_, net_, H_[kLayers], 1, nullptr, u_, u2_, u_scale(), utmp_));
          return GSPM_OK;
        }));
        CK(cudaMemcpyAsync(u2_, u_, len * sizeof(T), cudaMemcpyDeviceToDevice, L_.stream));
        CK(cudaMemcpyAsync(u_, utmp_, len * sizeof(T), cudaMemcpyDeviceToDevice, L_.stream));
        CK(cudaMemsetAsync(u_ + 3 * hb_.seg_pin[0], 0, 3 * sizeof(T), L_.stream));
        break;
      default:
        set_error("bad x0 mode %d", mode);
        return GSPM_EINVAL;
    }
    return GSPM_OK;
  }

  // learned warm start state
  int x0_mode_ = GSPM_X0_PREV;
  bool net_ready_ = false;
  double h_scale_ = 1.0;
  float *params_ = nullptr, *grad_ = nullptr, *adam_m_ = nullptr, *adam_v_ = nullptr,
        *loss_ = nullptr, *Y_ = nullptr, *agg_ = nullptr, *aggT_ = nullptr, *dHa_ = nullptr,
        *dHb_ = nullptr, *dZ_ = nullptr, *part_ = nullptr, *ds_T_ = nullptr;
  __nv_bfloat16 *WinT_ = nullptr, *F_in_ = nullptr, *ds_F_ = nullptr;
  __nv_bfloat16* WT_[3] = {};
  __nv_bfloat16* H_[4] = {};
  __nv_bfloat16* Z_[3] = {};
  int adam_t_ = 0, ds_cap_ = 0, ds_n_ = 0;
  MpnnDev net_{};
  int* mpnn_err_ = nullptr;
  T *u2_ = nullptr, *utmp_ = nullptr, *uin_ = nullptr, *uin2_ = nullptr;

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
  const HostBatch& hb_;
  Params P_;
  gspm_options opt_;
  Launch L_;
  DevMem mem_;
  int64_t n_ = 0, ld_ = 0, nslices_ = 0, entries_ = 0, nmag_ = 0, nodes_ = 0;
  int nseg_ = 1, nitems_ = 0, item_slices_ = 1;
  DSeg SG_{};
  int* nactive_ = nullptr;
  int* host_active_ = nullptr;
  double* host_scal_ = nullptr;
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
  T *U_ = nullptr, *u_ = nullptr, *b_ = nullptr, *r_ = nullptr, *x_ = nullptr;
  T *Ulo_ = nullptr, *ulo_ = nullptr, *dx_ = nullptr;  // refinement (mixed precision only)
  double *stage_ = nullptr, *scal_ = nullptr;
  CGState* cg_ = nullptr;
  CGState* host_state_ = nullptr;
  Red red_{};
  int pred_[kSolveSlots];
  int var_block_ = 0, var_scalar_ = 0, var_gs_ = 0;
  float tune_ms_block_[kSpmvVariants] = {}, tune_ms_scalar_[kSpmvVariants] = {},
        tune_ms_gs_[kSpmvVariants] = {};
  int seen_[kSolveSlots] = {};
  // K^ms / K^mech solves: pinned system (flag) or the consistent singular one (default)
  int pinned_ = 0;
  bool resolve_ = false;     // equilibria solved again at m* (Algorithm B.1 step 3 variant)
  double* wmean_ = nullptr;  // [n] 1 / (rows of the row's segment), 0 on padding rows
  double* proj_ = nullptr;   // [6 nseg] per-segment means of b, then pinned values of x
  double* tres_ = nullptr;   // [4 nseg] ||b - K x||^2, ||b||^2 of the last K^ms, K^mech solves
  bool tres_on_ = false;     // compute them after every K^ms / K^mech solve
  T* pinsave_ = nullptr;     // [3 nseg]
  int* bad_ = nullptr;       // [nseg] non-finite or zero m** met by the projection
  int* host_bad_ = nullptr;  // pinned copy
  // two-level preconditioner
  bool pc_ = false;
  DCoarse CC_{};
  typename CoarseStore<T>::type *cinv3_ = nullptr, *cinv1_ = nullptr;  // stored tiles
  DSymTiles TL3_{}, TL1_{};
  T* qsym_ = nullptr;  // partial products of the tiled coarse product
  int64_t *rc_off3_ = nullptr, *rc_off1_ = nullptr;
  T *dinv3_ = nullptr, *dinv1_ = nullptr;
  T *dgs_eps_ = nullptr, *dgs_aeps_ = nullptr;  // Jacobi of the GSPM solves (NULL: plain)
  T *rc_ = nullptr, *ec_ = nullptr;
  // CUDA-graph replay state
  bool graph_on_ = false, capturing_ = false;
  cudaStream_t cap_stream_ = nullptr, body_stream_ = nullptr;
  cudaGraphExec_t gexec_ = nullptr;
  int gexec_x0_ = -1;
  bool gexec_tres_ = false;
  int gexec_gen_ = -1, cfg_gen_ = 0;  // option generation the graph was captured with
  int64_t graph_static_ = 0;  // launches per replay outside the loop bodies
  int64_t graph_body_ = 0;    // launches captured inside loop bodies (once each)
  LoopCtl loop_{};            // loop control of the body being captured (zero otherwise)
  int* loop_cnt_ = nullptr;
  unsigned long long* loop_total_ = nullptr;
  unsigned long long loops_seen_ = 0;
  long long* gstats_ = nullptr;  // [nseg][4]: it_ms, it_mech, it_gs, noconv
  void* host_graph_ = nullptr;   // pinned: gstats, loop total, CG status blocks
};

}  // namespace gspm

using namespace gspm;

struct gspm_ctx {
  std::vector<HostMesh> hm;   // per segment (host structures, exports)
  HostBatch hb;               // concatenated batch (device layout)
  Params P;
  gspm_options opt;
  bool host_only = false;
  int64_t launches = 0;
  std::unique_ptr<EngineBase> eng;
};

static int load_batch(const gspm_mesh_desc* meshes, int nmesh, const gspm_material* mat,
                      const gspm_options* opt, gspm_ctx** out) {
  if (!meshes || nmesh < 1 || !mat || !opt || !out) {
    set_error("mesh_load: null argument or no mesh");
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
  c->hm.resize(nmesh);
  std::vector<HostSell> hs(nmesh);
  std::vector<HostOps> ops(nmesh);
  for (int k = 0; k < nmesh; ++k) {
    const int st = host_mesh_build(meshes + k, opt->ordering, opt->coarse_nodes, &c->hm[k]);
    if (st != GSPM_OK) {
      if (nmesh > 1) {
        std::string msg = g_err;
        set_error("mesh %d: %s", k, msg.c_str());
      }
      return st;
    }
  }
  // two-level preconditioner of the K^ms / K^mech solves (singular form only): aggregates of
  // coarse_nodes_of(coarse_nodes, n) nodes; host-only contexts build it too (for export)
  std::vector<HostCoarse> coarse;
  const bool two_level = !(opt->flags & (GSPM_FLAG_PINNED_CG | GSPM_FLAG_PLAIN_CG));
  for (int k = 0; k < nmesh; ++k) {
    host_sell_build(c->hm[k], &hs[k]);
    if (!c->host_only || two_level) host_assemble(c->hm[k], hs[k], c->P, &ops[k]);
  }
  if (two_level) {
    coarse.resize(nmesh);
    for (int k = 0; k < nmesh; ++k) {
      const int64_t npa = coarse_nodes_of(opt->coarse_nodes, c->hm[k].n);
      const int st = host_coarse_build(c->hm[k], hs[k], ops[k], npa,
                                       opt->precision == GSPM_PREC_MIXED ? 1 : 0, &coarse[k]);
      if (st != GSPM_OK) return st;
    }
  }
  if (c->host_only) {
    c->hb.sell = std::move(hs[0]);
    c->hb.n_nodes = 0;
    for (auto& h : c->hm) c->hb.n_nodes += h.n;
    c->hb.coarse = std::move(coarse);
  } else {
    host_batch_build(c->hm, hs, ops, &c->hb);
    c->hb.coarse = std::move(coarse);
    cudaStream_t s = (cudaStream_t)opt->stream;
    if (opt->precision == GSPM_PREC_F64) {
      auto e = std::make_unique<Engine<double>>(c->hb, c->P, c->opt, s, &c->launches);
      ST(e->init());
      c->eng = std::move(e);
    } else {
      auto e = std::make_unique<Engine<float>>(c->hb, c->P, c->opt, s, &c->launches);
      ST(e->init());
      c->eng = std::move(e);
    }
    // operator values now live on the device (the coarse operators stay for export)
    for (auto& hc : c->hb.coarse) {
      hc.inv_mech = std::vector<double>();
      hc.inv_ms = std::vector<double>();
      hc.store_mech = std::vector<double>();
      hc.store_ms = std::vector<double>();
      hc.dinv_mech = std::vector<double>();
      hc.dinv_ms = std::vector<double>();
    }
    c->hb.ops = HostOps();
    c->hb.sell.col.clear();
    c->hb.sell.col.shrink_to_fit();
  }
  *out = c.release();
  return GSPM_OK;
}

extern "C" {

const char* gspm_last_error(void) { return g_err.c_str(); }

int gspm_mesh_load(const gspm_mesh_desc* mesh, const gspm_material* mat,
                   const gspm_options* opt, gspm_ctx** out) {
  return load_batch(mesh, 1, mat, opt, out);
}

int gspm_batch_load(const gspm_mesh_desc* meshes, int n_meshes, const gspm_material* mat,
                    const gspm_options* opt, gspm_ctx** out) {
  return load_batch(meshes, n_meshes, mat, opt, out);
}

int gspm_batch_segment(const gspm_ctx* ctx, int seg, int64_t* node_offset, int64_t* n_nodes) {
  if (!ctx || seg < 0 || seg >= (int)ctx->hm.size()) {
    set_error("batch_segment: bad context or segment %d", seg);
    return GSPM_EINVAL;
  }
  int64_t off = 0;
  for (int k = 0; k < seg; ++k) off += ctx->hm[k].n;
  if (node_offset) *node_offset = off;
  if (n_nodes) *n_nodes = ctx->hm[seg].n;
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
  memset(out, 0, sizeof(*out));
  for (const HostMesh& h : ctx->hm) {
    out->n_stored += h.n_stored;
    out->n_unique += h.n;
    out->n_tets += h.n_tets;
    out->n_magnetic_nodes += h.n_mag_nodes;
    out->n_magnetic_tets += h.n_mag_tets;
    out->nnz += h.rowptr.empty() ? 0 : h.rowptr.back();
    out->volume += h.volume;
    out->volume_magnetic += h.volume_mag;
  }
  out->sell_entries = ctx->hb.sell.entries;
  out->n_segments = (int)ctx->hm.size();
  out->eps = ctx->P.eps;
  out->dtau = ctx->P.dtau;
  out->device_bytes = ctx->eng ? ctx->eng->device_bytes() : 0;
  out->n_aggregates = 0;
  for (const auto& hc : ctx->hb.coarse) {
    out->n_aggregates += hc.n_agg;
    out->coarse_shift_ms = std::max(out->coarse_shift_ms, hc.shift_ms);
    out->coarse_shift_mech = std::max(out->coarse_shift_mech, hc.shift_mech);
  }
  if (ctx->eng) {
    float tb[kSpmvVariants], ts[kSpmvVariants], tg[kSpmvVariants];
    int vb = 0, vs = 0, vg = 0, is = 0;
    ctx->eng->tune_info(&vb, &vs, &vg, tb, ts, tg, &is);
    out->spmv_schedule_block = vb;
    out->spmv_schedule_scalar = vs;
    out->spmv_schedule_gs = vg;
    out->item_slices = is;
    for (int v = 0; v < kSpmvVariants && v < GSPM_SPMV_SCHEDULES; ++v) {
      out->spmv_ms_block[v] = tb[v];
      out->spmv_ms_scalar[v] = ts[v];
      out->spmv_ms_gs[v] = tg[v];
    }
  }
  return GSPM_OK;
}

int gspm_mesh_export(const gspm_ctx* ctx, int what, void* out, int64_t count) {
  if (!ctx || !out) {
    set_error("mesh_export: null argument");
    return GSPM_EINVAL;
  }
  if (ctx->hm.size() != 1) {
    set_error("mesh_export: only for single-mesh contexts");
    return GSPM_ESTATE;
  }
  const HostMesh& hm = ctx->hm[0];
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
    case GSPM_EXPORT_AGGREGATES:
    case GSPM_EXPORT_COARSE_K_MS:
    case GSPM_EXPORT_COARSE_K_MECH:
    case GSPM_EXPORT_COARSE_INV_MS:
    case GSPM_EXPORT_COARSE_INV_MECH:
    case GSPM_EXPORT_COARSE_STORED_MS:
    case GSPM_EXPORT_COARSE_STORED_MECH: {
      if (ctx->hb.coarse.empty()) {
        set_error("mesh_export: the context has no two-level preconditioner");
        return GSPM_ESTATE;
      }
      const HostCoarse& hc = ctx->hb.coarse[0];
      if (what == GSPM_EXPORT_COARSE_K_MS) return put(hc.Kc_ms.data(), (int64_t)hc.Kc_ms.size(), 8);
      if (what == GSPM_EXPORT_COARSE_K_MECH)
        return put(hc.Kc_mech.data(), (int64_t)hc.Kc_mech.size(), 8);
      if (what == GSPM_EXPORT_COARSE_INV_MS || what == GSPM_EXPORT_COARSE_INV_MECH) {
        const std::vector<double>& v = what == GSPM_EXPORT_COARSE_INV_MS ? hc.inv_ms : hc.inv_mech;
        if (v.empty()) {
          set_error("mesh_export: coarse inverses are kept by host-only contexts only");
          return GSPM_ESTATE;
        }
        return put(v.data(), (int64_t)v.size(), 8);
      }
      if (what == GSPM_EXPORT_COARSE_STORED_MS || what == GSPM_EXPORT_COARSE_STORED_MECH) {
        const std::vector<double>& v =
            what == GSPM_EXPORT_COARSE_STORED_MS ? hc.store_ms : hc.store_mech;
        if (v.empty()) {
          set_error("mesh_export: stored coarse inverses are kept by host-only contexts only");
          return GSPM_ESTATE;
        }
        return put(v.data(), (int64_t)v.size(), 8);
      }
      std::vector<int32_t> a(hm.n);
      for (int64_t i = 0; i < hm.n; ++i) a[hm.perm[i]] = hc.agg[i];
      return put(a.data(), hm.n, 4);
    }
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

int gspm_coarse_round(const double* A, int64_t n, int bf16, double* out, double* shift) {
  if (!A || !out || n < 1 || (bf16 != 0 && bf16 != 1)) {
    set_error("coarse_round: need A, out, n >= 1 and bf16 in {0, 1}");
    return GSPM_EINVAL;
  }
  std::vector<double> st;
  double sh = 0.0;
  const int rc = coarse_round_spd(A, n, bf16, &st, &sh);
  if (rc != GSPM_OK) return rc;
  memcpy(out, st.data(), (size_t)(n * n) * sizeof(double));
  if (shift) *shift = sh;
  return GSPM_OK;
}

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
  return ctx->eng->step(n_steps, H_ext, false, stats);
}

int gspm_batch_step(gspm_ctx* ctx, int n_steps, const double* H_ext, gspm_step_stats* stats) {
  NEED_ENGINE(ctx);
  if (n_steps < 0 || !H_ext) {
    set_error("batch_step: need n_steps >= 0 and H_ext");
    return GSPM_EINVAL;
  }
  return ctx->eng->step(n_steps, H_ext, true, stats);
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

int gspm_set_graph(gspm_ctx* ctx, int on) {
  NEED_ENGINE(ctx);
  return ctx->eng->set_graph(on);
}

int gspm_set_true_residual(gspm_ctx* ctx, int on) {
  NEED_ENGINE(ctx);
  return ctx->eng->set_true_residual(on);
}

int gspm_set_rtol(gspm_ctx* ctx, double rtol_gs, double rtol_ms, double rtol_mech) {
  NEED_ENGINE(ctx);
  const int rc = ctx->eng->set_rtol(rtol_gs, rtol_ms, rtol_mech);
  if (rc == GSPM_OK) {
    if (rtol_gs > 0) ctx->opt.rtol_gs = rtol_gs;
    if (rtol_ms > 0) ctx->opt.rtol_ms = rtol_ms;
    if (rtol_mech > 0) ctx->opt.rtol_mech = rtol_mech;
  }
  return rc;
}

int gspm_set_x0_mode(gspm_ctx* ctx, int mode) {
  NEED_ENGINE(ctx);
  return ctx->eng->set_x0_mode(mode);
}

int gspm_mpnn_set_params(gspm_ctx* ctx, const float* params, int64_t count) {
  NEED_ENGINE(ctx);
  if (!params) {
    set_error("mpnn_set_params: null pointer");
    return GSPM_EINVAL;
  }
  return ctx->eng->mpnn_params(nullptr, params, count);
}

int gspm_mpnn_get_params(gspm_ctx* ctx, float* params, int64_t count) {
  NEED_ENGINE(ctx);
  if (!params) {
    set_error("mpnn_get_params: null pointer");
    return GSPM_EINVAL;
  }
  return ctx->eng->mpnn_params(params, nullptr, count);
}

int gspm_mpnn_predict(gspm_ctx* ctx, const double* m, const double* u_prev, const double* u_prev2,
                      double* out, int what, int where) {
  NEED_ENGINE(ctx);
  return ctx->eng->mpnn_predict(m, u_prev, u_prev2, out, what, where);
}

int gspm_mpnn_dataset_reserve(gspm_ctx* ctx, int capacity) {
  NEED_ENGINE(ctx);
  return ctx->eng->mpnn_dataset_reserve(capacity);
}

int gspm_mpnn_dataset_add(gspm_ctx* ctx, const double* m, const double* u_prev,
                          const double* u_prev2, const double* u_star, int where, int* index) {
  NEED_ENGINE(ctx);
  return ctx->eng->mpnn_dataset_add(m, u_prev, u_prev2, u_star, where, index);
}

int gspm_mpnn_loss_grad(gspm_ctx* ctx, int pair, double* loss, float* grad) {
  NEED_ENGINE(ctx);
  return ctx->eng->mpnn_loss_grad(pair, loss, grad);
}

int gspm_mpnn_train(gspm_ctx* ctx, int iterations, double lr, uint64_t seed, double* loss_first,
                    double* loss_last) {
  NEED_ENGINE(ctx);
  return ctx->eng->mpnn_train(iterations, lr, seed, loss_first, loss_last);
}

int gspm_profile_enable(gspm_ctx* ctx, unsigned class_mask) {
  NEED_ENGINE(ctx);
  return ctx->eng->profile_enable(class_mask);
}

int gspm_profile_read(gspm_ctx* ctx, int kclass, double* total_ms, int64_t* launches) {
  NEED_ENGINE(ctx);
  return ctx->eng->profile_read(kclass, total_ms, launches);
}

}  // extern "C"
