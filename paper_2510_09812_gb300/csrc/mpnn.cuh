// Learned warm start: sizes, parameter layout and launchers (see mpnn.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.cuh"

namespace gspm {

constexpr int kHid = 64;     // hidden width
constexpr int kFeat = 16;    // node features
constexpr int kLayers = 3;   // message-passing layers
// flat FP32 parameter layout: W_in [16][64], b_in [64], {W_l [128][64], b_l [64]} x 3,
// W_out [64][3], b_out [3]
constexpr int kOffWin = 0;
constexpr int kOffBin = kFeat * kHid;
constexpr int kLayerSize = 2 * kHid * kHid + kHid;
constexpr int kOffW[3] = {kOffBin + kHid, kOffBin + kHid + kLayerSize,
                          kOffBin + kHid + 2 * kLayerSize};
constexpr int kOffWout = kOffBin + kHid + 3 * kLayerSize;
constexpr int kOffBout = kOffWout + kHid * 3;
constexpr int kParams = kOffBout + 3;

// device views of the network
struct MpnnDev {
  const __nv_bfloat16* WinT;   // [64][16]  (W_in transposed, bf16)
  const float* b_in;
  const __nv_bfloat16* WT[3];  // [64][128] (W_l transposed, bf16)
  const float* b[3];
  const float* Wf[3];          // [128][64] fp32 master copies (backward)
  const float* Wout;           // [64][3]
  const float* bout;
  const float* A;              // SELL weights of the element-message averaging
  const float* At;             // SELL weights of its transpose
  int* err;                    // set by a forward layer whose tensor-core wait gave up
};

size_t mpnn_layer_smem();
size_t mpnn_layer_bwd_smem();
cudaError_t mpnn_setup_smem();
template <typename T>
cudaError_t mpnn_features(const Launch& L, int64_t n, const T* m, int64_t ld, const uint8_t* mag,
                          const T* up, const T* up2, double l100, double l111, double ls,
                          double us, __nv_bfloat16* F);
cudaError_t mpnn_forward(const Launch& L, int64_t n, const DSell& S, const MpnnDev& W,
                         const __nv_bfloat16* F, __nv_bfloat16* const H[4],
                         __nv_bfloat16* const Z[3]);
template <typename T>
cudaError_t mpnn_output(const Launch& L, int64_t n, const MpnnDev& W, const __nv_bfloat16* H3,
                        int mode, float* Y, const T* up, const T* up2, double us, T* x0);
cudaError_t mpnn_backward(const Launch& L, int64_t n, const DSell& S, const MpnnDev& W,
                          const __nv_bfloat16* F, __nv_bfloat16* const H[4],
                          __nv_bfloat16* const Z[3], const float* Y, const float* T, float* dHa,
                          float* dHb, float* dZ, float* part, float* grad, float* loss);
cudaError_t mpnn_adam(const Launch& L, float* w, const float* g, float* m, float* v, float lr,
                      int t);
cudaError_t mpnn_refresh_bf16(const Launch& L, __nv_bfloat16* WinT, __nv_bfloat16* const WT[3],
                              const float* params);

}  // namespace gspm
