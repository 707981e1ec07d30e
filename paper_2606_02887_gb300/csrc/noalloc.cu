// Dense A*X product for callers that cannot allocate device memory.
//
// Same kernels as the handle's product (k_gemm_dense + k_ax_finish), but the split-K
// slices and the FP64 partial sums live in one file-scope __device__ array of fixed
// size instead of memory obtained from cudaMalloc.  Nothing here allocates: no
// cudaMalloc / cudaFree, no host heap.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/snmf.h"
#include "common.cuh"

namespace {

constexpr size_t kScratchBytes = SNMF_NOALLOC_SCRATCH_BYTES;
constexpr size_t kPartialBytes = SNMF_NOALLOC_PARTIAL_BYTES;  // FP64 partial sums + the reduced scalar
constexpr int kMaxDevices = 64;
constexpr int64_t kRecordBytes = (int64_t)snmf::kNQ * sizeof(double);  // one partial record per row slice
static_assert(kRecordBytes == 256, "SNMF_NOALLOC_MAX_ROWS assumes 256-byte partial records");
static_assert(SNMF_NOALLOC_MAX_ROWS == (int64_t)snmf::kRowTile * (int64_t)((kPartialBytes - 256) / kRecordBytes),
              "SNMF_NOALLOC_MAX_ROWS must follow from the partial-sum region");

// Shared by every call on a device; keeps the last call's contents.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device, valid for the context it was resolved in (the
// host-side symbol is only a stand-in).  A new context (after a device reset, or a caller's
// own driver-API context) resolves it again.
struct ScratchAddr {
  void* ptr = nullptr;
  CUcontext ctx = nullptr;
};
ScratchAddr g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

using CtxGetCurrentFn = CUresult (*)(CUcontext*);

// cuCtxGetCurrent through the runtime's driver entry point (no link against libcuda).
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(p);
  });
  return fn;
}

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
  const size_t slice = (size_t)n * (size_t)cols * esz;
  // two split-K slices must fit beside the partial sums, one partial record per 64 rows
  if (n > SNMF_NOALLOC_MAX_ROWS || 2 * slice > SNMF_NOALLOC_MAX_SLICE_PAIR_BYTES) return SNMF_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SNMF_ERR_CUDA;
  // the current context (NULL before the first runtime call of the thread initialises one)
  CUcontext ctx = nullptr;
  const CtxGetCurrentFn get_ctx = ctx_get_current();
  if (!get_ctx || get_ctx(&ctx) != CUDA_SUCCESS) ctx = nullptr;
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    ScratchAddr& slot = g_scratch_addr[dev];
    if (!slot.ptr || !ctx || slot.ctx != ctx) {
      // first call in this context (or the context cannot be identified): resolve the
      // array's device address here
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return SNMF_ERR_CUDA;
      slot.ptr = p;
      slot.ctx = ctx;
    }
    base = slot.ptr;
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
