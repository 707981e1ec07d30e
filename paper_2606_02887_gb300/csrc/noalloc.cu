// Dense A*X product for callers that cannot allocate device memory.
//
// Same kernels as the handle's product (k_gemm_dense + k_ax_finish), but the split-K
// slices and the FP64 partial sums live in one file-scope __device__ array of fixed
// size instead of memory obtained from cudaMalloc.  Nothing here allocates: no
// cudaMalloc / cudaFree, no host heap.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/snmf.h"
#include "common.cuh"

namespace {

constexpr size_t kScratchBytes = SNMF_NOALLOC_SCRATCH_BYTES;
constexpr size_t kPartialBytes = 1u << 20;  // FP64 partial sums + the reduced scalar
constexpr int kMaxDevices = 64;

// Shared by every call on a device; keeps the last call's contents.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device (the host-side symbol is only a stand-in).
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Sum part[slot][0][q] over slots in a fixed order (one block).
__global__ void k_sum_slots(const double* __restrict__ part, int nslots, int q, double* __restrict__ out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int t = threadIdx.x; t < nslots; t += blockDim.x) s += part[(int64_t)t * snmf::kNQ + q];
  s = snmf::block_sum(s, sh);
  if (threadIdx.x == 0) *out = s;
}

}  // namespace

extern "C" snmf_status snmf_apply_dense_noalloc(const void* A, int dtype, int64_t n, int64_t lda,
                                                const void* X, void* Y, int cols, double* xax,
                                                void* stream) {
  if (!A || !X || !Y || n < 1 || cols < 1 || lda < n || (dtype != SNMF_F64 && dtype != SNMF_F32))
    return SNMF_ERR_ARG;
  const size_t esz = dtype == SNMF_F64 ? 8 : 4;
  const int64_t nslots = (n + snmf::kRowTile - 1) / snmf::kRowTile;
  const size_t slice = (size_t)n * (size_t)cols * esz;
  // two split-K slices must fit beside the partial sums
  if (2 * slice > kScratchBytes - kPartialBytes ||
      (size_t)nslots * snmf::kNQ * sizeof(double) + 256 > kPartialBytes)
    return SNMF_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SNMF_ERR_CUDA;
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      // first call on this device (current): resolve the array's device address
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return SNMF_ERR_CUDA;
      g_scratch_addr[dev] = p;
    }
    base = g_scratch_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* scratch = static_cast<unsigned char*>(base);
  double* part = reinterpret_cast<double*>(scratch);                 // partial sums
  double* total = part + (kPartialBytes / sizeof(double)) - 8;       // reduced <X, A X>
  void* ws = scratch + kPartialBytes;                                // split-K slices
  const size_t ws_elems = (kScratchBytes - kPartialBytes) / esz;

  snmf::AxArgs a{};
  a.kind = snmf::AX_DENSE;
  a.A = A;
  a.lda = lda;
  a.a_dtype = dtype == SNMF_F64 ? 0 : 1;
  const int td = dtype == SNMF_F64 ? 0 : 1;
  snmf::Dims d;
  d.n = n; d.r = cols; d.b = 1; d.N = cols; d.ld = cols;
  const int splits = snmf::launch_ax(a, td, n, cols, cols, X, Y, ws, ws_elems, nullptr, s);
  const int ns = snmf::launch_ax_finish_impl(td, d, Y, ws, splits, 0.0, nullptr, X, nullptr, part, 0,
                                             nullptr, s);
  k_sum_slots<<<1, 256, 0, s>>>(part, ns, 0, total);
  if (cudaGetLastError() != cudaSuccess) return SNMF_ERR_CUDA;
  if (xax) {
    if (cudaMemcpyAsync(xax, total, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return SNMF_ERR_CUDA;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return SNMF_ERR_CUDA;
  return SNMF_OK;
}
