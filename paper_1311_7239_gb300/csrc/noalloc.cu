// lbm_residual_noalloc: the FP64 steady-state residual reduction for callers that must not
// allocate device memory.
//
// Some callers cannot let a library call cudaMalloc: services that pre-size one device memory
// pool at start-up and must not grow it later, hosts whose framework owns every device byte
// through its own allocator, and real-time loops where cudaMalloc/cudaFree would synchronise the
// device and stall unrelated streams at unpredictable moments.  This entry point gives them the
// residual r = ||u - u_prev||_2 / ||u||_2 of two velocity fields they already hold, without
// creating a context and without any allocation: the per-block partial sums live in the fixed
// array below, which every GPU that loads liblbm.so holds until the process exits.
#include <cuda_runtime.h>
#include <math.h>
#include <mutex>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kCellsPerThread = 64;
constexpr int kMaxBlocks = 4096;
// Largest field this entry point accepts: kMaxBlocks * kThreads * kCellsPerThread = 2^26 cells.
constexpr long long kMaxCells = (long long)kMaxBlocks * kThreads * kCellsPerThread;

// Scratch: two partial sums per block, then the two totals.  Every call overwrites the slots
// it uses before reading them, so nothing has to start at zero; concurrent calls share it.
static __device__ __align__(256) double g_residual_scratch[2 * kMaxBlocks + 2];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[kThreads / 32], sb[kThreads / 32];
  a = warp_sum(a);
  b = warp_sum(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  if (w == 0) {
    a = l < kThreads / 32 ? sa[l] : 0.0;
    b = l < kThreads / 32 ? sb[l] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
  }
}

// Pass 1: block b sums |u - u_prev|^2 and |u|^2 over its cells into scratch[2b], scratch[2b+1].
__global__ void __launch_bounds__(kThreads) k_partials(const float* __restrict__ ux, const float* __restrict__ uy,
                                                       const float* __restrict__ px, const float* __restrict__ py,
                                                       long long n, double* __restrict__ scratch) {
  double num = 0.0, den = 0.0;
  const long long stride = (long long)gridDim.x * kThreads;
  for (long long k = (long long)blockIdx.x * kThreads + threadIdx.x; k < n; k += stride) {
    const double a = ux[k], b = uy[k];
    const double dx = a - (double)px[k], dy = b - (double)py[k];
    num += dx * dx + dy * dy;
    den += a * a + b * b;
  }
  block_sum2(num, den);
  if (threadIdx.x == 0) {
    scratch[2 * blockIdx.x] = num;
    scratch[2 * blockIdx.x + 1] = den;
  }
}

// Pass 2: one block adds the partials in a fixed order; the totals go to the last two slots and
// r to *r_dev (a device address, or nullptr).
__global__ void __launch_bounds__(kThreads) k_finish(double* __restrict__ scratch, int nblocks, double* __restrict__ r_dev) {
  double num = 0.0, den = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += kThreads) {
    num += scratch[2 * i];
    den += scratch[2 * i + 1];
  }
  block_sum2(num, den);
  if (threadIdx.x == 0) {
    scratch[2 * kMaxBlocks] = num;
    scratch[2 * kMaxBlocks + 1] = den;
    const double r = den > 0.0 ? sqrt(num / den) : 0.0;
    if (r_dev) *r_dev = r;
  }
}

// Device address of the scratch array on the current device, looked up once per device.
cudaError_t scratch_address(int device, double** out) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_residual_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[device];
  return cudaSuccess;
}

}  // namespace

extern "C" int lbm_residual_noalloc(const float* ux, const float* uy, const float* ux_prev, const float* uy_prev,
                                    int64_t n, double* r, void* stream) {
  if (!ux || !uy || !ux_prev || !uy_prev || !r) return lbm::record_error(LBM_EINVAL, "lbm_residual_noalloc: null argument");
  if (n <= 0 || n > kMaxCells)
    return lbm::record_error(LBM_EINVAL, "lbm_residual_noalloc: n must be in [1, 67108864] (its fixed scratch holds 4096 blocks)");
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices)
    return lbm::record_error(LBM_ECUDA, "lbm_residual_noalloc: no usable current device");
  double* scratch = nullptr;
  if (scratch_address(device, &scratch) != cudaSuccess)
    return lbm::record_error(LBM_ECUDA, "lbm_residual_noalloc: cudaGetSymbolAddress of the scratch array failed");
  cudaPointerAttributes a;
  bool r_on_device = false;
  if (cudaPointerGetAttributes(&a, r) == cudaSuccess)
    r_on_device = a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
  else
    cudaGetLastError();
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long per_block = (long long)kThreads * kCellsPerThread;
  const int nblocks = (int)((n + per_block - 1) / per_block);
  k_partials<<<nblocks, kThreads, 0, s>>>(ux, uy, ux_prev, uy_prev, (long long)n, scratch);
  k_finish<<<1, kThreads, 0, s>>>(scratch, nblocks, r_on_device ? r : nullptr);
  if (cudaGetLastError() != cudaSuccess) return lbm::record_error(LBM_ECUDA, "lbm_residual_noalloc: kernel launch failed");
  if (!r_on_device) {
    double tot[2];
    if (cudaMemcpyAsync(tot, scratch + 2 * kMaxBlocks, sizeof(tot), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return lbm::record_error(LBM_ECUDA, "lbm_residual_noalloc: copy of the result failed");
    *r = tot[1] > 0.0 ? sqrt(tot[0] / tot[1]) : 0.0;
  }
  return LBM_OK;
}
