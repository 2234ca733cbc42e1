// Allocation-free volume average.
//
// Some callers cannot allocate device memory: code that runs inside another framework's fixed
// memory pool (where a cudaMalloc outside the pool would break its budget or fragment it),
// real-time loops and host callbacks where cudaMalloc's implicit device synchronisation is not
// acceptable, and plug-ins that only receive pointers.  gspm_volume_avg_noalloc serves them: the
// caller passes the field, the quadrature weights and the output on the device; the reduction's
// scratch (one partial per block plus an arrival counter) lives in a file-scope __device__ array
// of fixed size that every GPU loading this library holds until the process exits.
//
// The host never dereferences the array's name (in host code it is only a stand-in symbol); the
// device address is looked up once per device with cudaGetSymbolAddress, with that device
// current, on the first call made on that device.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "gspm.h"

namespace gspm {
void set_error(const char* fmt, ...);
}

namespace {

constexpr int kThreads = 256;
constexpr int kComp = 16;                        // partial slots per block (ncomp <= 9 used)
constexpr int kMaxBlocks = GSPM_NOALLOC_MAX_BLOCKS;
constexpr int kScratch = kMaxBlocks * kComp + 32;  // partials, then the counter slot

// Reduction scratch shared by every call on this device: kMaxBlocks x 16 doubles of block
// partials followed by the arrival counter (first 4 bytes of the next 256-byte run).
static __device__ __align__(256) double g_noalloc_scratch[kScratch];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

__device__ __forceinline__ double wsum_warp(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

// out[c] = sum_i w_i f[i*nc + c]: fixed-order per-thread sums, warp and block trees, one partial
// per block, and the last block to arrive (ticket on the counter) adds the partials in block
// order and resets the counter.
__global__ void __launch_bounds__(kThreads)
k_wsum_noalloc(int64_t n, int nc, const double* __restrict__ f, const double* __restrict__ w,
               double* __restrict__ out, double* scratch) {
  double v[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) v[c] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double wi = w[i];
#pragma unroll
    for (int c = 0; c < 9; ++c)
      if (c < nc) v[c] += wi * f[i * nc + c];
  }
  __shared__ double sm[9][32];
  __shared__ int last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    const double x = wsum_warp(v[c]);
    if (lane == 0) sm[c][warp] = x;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      const double x = wsum_warp(lane < nw ? sm[c][lane] : 0.0);
      if (lane == 0) scratch[(int64_t)blockIdx.x * kComp + c] = x;
    }
  }
  unsigned* counter = reinterpret_cast<unsigned*>(scratch + (int64_t)kMaxBlocks * kComp);
  if (threadIdx.x == 0) {
    __threadfence();
    last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      acc += __ldcg(scratch + (int64_t)b * kComp + c);
    acc = wsum_warp(acc);
    if (lane == 0) sm[c][warp] = acc;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      const double x = wsum_warp(lane < nw ? sm[c][lane] : 0.0);
      if (lane == 0 && c < nc) out[c] = x;
    }
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// Device address of the scratch for the current device, looked up once per device.
int scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    gspm::set_error("volume_avg_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    return GSPM_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    gspm::set_error("volume_avg_noalloc: device ordinal %d above %d", dev, kMaxDevices - 1);
    return GSPM_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      gspm::set_error("volume_avg_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      return GSPM_ECUDA;
    }
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return GSPM_OK;
}

}  // namespace

extern "C" int gspm_volume_avg_noalloc(const double* field, const double* weights, int64_t n,
                                       int ncomp, double* out, void* stream) {
  if (!field || !weights || !out) {
    gspm::set_error("volume_avg_noalloc: null pointer");
    return GSPM_EINVAL;
  }
  if (n <= 0) {
    gspm::set_error("volume_avg_noalloc: n must be positive (got %lld)", (long long)n);
    return GSPM_EINVAL;
  }
  if (ncomp < 1 || ncomp > GSPM_NOALLOC_MAX_COMP) {
    gspm::set_error("volume_avg_noalloc: ncomp %d outside 1..%d (the fixed scratch holds at most "
                    "%d components per block)", ncomp, GSPM_NOALLOC_MAX_COMP,
                    GSPM_NOALLOC_MAX_COMP);
    return GSPM_EINVAL;
  }
  double* scratch = nullptr;
  int st = scratch_address(&scratch);
  if (st != GSPM_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the arrival counter must start at zero (a previous call resets it; clear it regardless)
  cudaError_t e = cudaMemsetAsync(scratch + (int64_t)kMaxBlocks * kComp, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) {
    gspm::set_error("volume_avg_noalloc: cudaMemsetAsync: %s", cudaGetErrorString(e));
    return GSPM_ECUDA;
  }
  int64_t blocks = (n + kThreads - 1) / kThreads;
  if (blocks > kMaxBlocks) blocks = kMaxBlocks;
  k_wsum_noalloc<<<(int)blocks, kThreads, 0, s>>>(n, ncomp, field, weights, out, scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    gspm::set_error("volume_avg_noalloc: launch: %s", cudaGetErrorString(e));
    return GSPM_ECUDA;
  }
  return GSPM_OK;
}
