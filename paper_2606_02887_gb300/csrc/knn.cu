// Graph pre-processing for Graph-SNMPBB and clustering scores on the GPU.
//
//   snmf_knn_graph      k nearest neighbours of every point (brute force, squared Euclidean
//                       distance, ties: lower index first), self-tuning scale s_i = distance to
//                       the sigma_rank-th neighbour, S_ij = exp(-d_ij^2 / (s_i s_j)) on the kNN
//                       pairs, symmetrised as max(S, S^T), degrees d_i = sum_j S_ij and the CSR
//                       matrix A^ = D^-1/2 S D^-1/2 (columns ascending per row).
//   snmf_cluster_assign label_i = argmax_c of the restart's H factor row (ties: lowest c).
//   snmf_cluster_scores contingency table of two labelings on the device; the adjusted Rand
//                       index and the accuracy of the best one-to-one label matching from it
//                       on the host (Hungarian method on the small table).
// Every reduction is in a fixed order: the outputs do not depend on thread scheduling.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <limits>
#include <vector>

#include "../../include/snmf.h"
#include "common.cuh"

namespace snmf {
namespace {

constexpr int QB = 64;  // queries per CTA (one per thread)
constexpr int CB = 64;  // candidates staged per round
constexpr int KMAX = 32;

// Top-K (K = compile-time bound, k <= K at run time) by squared distance, candidates in
// increasing index order; a candidate replaces an entry only when strictly closer (or the entry
// is still empty), so equal distances keep the lower index first and every slot ends up holding
// a valid index (k < n).  A non-finite distance counts as +inf and raises *bad.
template <int K>
__global__ void __launch_bounds__(QB) k_knn(const float* __restrict__ X, int64_t n, int d, int k,
                                            int32_t* __restrict__ nbr, float* __restrict__ nd2,
                                            int* __restrict__ bad) {
  extern __shared__ float ksm[];
  const int ds = d + 1;  // odd row stride: conflict-free per-thread rows
  float* Qs = ksm;
  float* Cs = ksm + QB * ds;
  const int64_t q = (int64_t)blockIdx.x * QB + threadIdx.x;
  for (int e = threadIdx.x; e < QB * d; e += QB) {
    const int r = e / d, t = e % d;
    const int64_t i = (int64_t)blockIdx.x * QB + r;
    Qs[r * ds + t] = i < n ? X[i * d + t] : 0.f;
  }
  float kd[K];
  int32_t ki[K];
#pragma unroll
  for (int t = 0; t < K; ++t) {
    kd[t] = INFINITY;
    ki[t] = INT_MAX;
  }
  for (int64_t c0 = 0; c0 < n; c0 += CB) {
    __syncthreads();
    for (int e = threadIdx.x; e < CB * d; e += QB) {
      const int r = e / d, t = e % d;
      const int64_t j = c0 + r;
      Cs[r * ds + t] = j < n ? X[j * d + t] : 0.f;
    }
    __syncthreads();
    if (q < n) {
      const int cn = (int)(n - c0 < CB ? n - c0 : CB);
      const float* qr = Qs + threadIdx.x * ds;
      for (int c = 0; c < cn; ++c) {
        const int64_t j = c0 + c;
        if (j == q) continue;
        const float* cr = Cs + c * ds;
        float acc = 0.f;
        for (int t = 0; t < d; ++t) {
          const float df = qr[t] - cr[t];
          acc = fmaf(df, df, acc);
        }
        float v = acc;
        if (!isfinite(v)) {
          v = INFINITY;
          atomicOr(bad, 1);
        }
        int32_t vi = (int32_t)j;
#pragma unroll
        for (int t = 0; t < K; ++t) {
          if (t < k && (v < kd[t] || (v == kd[t] && vi < ki[t]))) {
            const float tv = kd[t];
            const int32_t ti = ki[t];
            kd[t] = v;
            ki[t] = vi;
            v = tv;
            vi = ti;
          }
        }
      }
    }
  }
  if (q < n) {
#pragma unroll
    for (int t = 0; t < K; ++t)
      if (t < k) {
        nbr[q * k + t] = ki[t];
        nd2[q * k + t] = kd[t];
      }
  }
}

// scale s_i, directed similarities, in-degree counts
__global__ void k_knn_sim(const int32_t* __restrict__ nbr, const float* __restrict__ nd2, int64_t n, int k,
                          int sigma_rank, float* __restrict__ sval, int32_t* __restrict__ cnt,
                          int* __restrict__ bad) {
  const int64_t total = n * k;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / k;
    const int32_t j = nbr[e];
    const float si = sqrtf(nd2[i * k + sigma_rank - 1]);
    const float sj = sqrtf(nd2[(int64_t)j * k + sigma_rank - 1]);
    const float v = expf(-nd2[e] / (si * sj));
    if (!(si * sj > 0.f) || !isfinite(v)) atomicOr(bad, 1);  // zero scale: duplicate points
    sval[e] = v;
    atomicAdd(&cnt[j], 1);  // the reverse entry (j, i)
  }
}

// exclusive scan of v[0..n) (+ k per element) into out[0..n], one block, fixed order
__global__ void __launch_bounds__(1024) k_scan(const int32_t* __restrict__ v, int64_t n, int add,
                                               int32_t* __restrict__ out) {
  __shared__ int64_t part[1024];
  const int64_t per = (n + blockDim.x - 1) / blockDim.x;
  const int64_t b = threadIdx.x * per, e = b + per < n ? b + per : n;
  int64_t s = 0;
  for (int64_t i = b; i < e; ++i) s += v[i] + add;
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t run = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      const int64_t x = part[t];
      part[t] = run;
      run += x;
    }
    out[n] = (int32_t)run;
  }
  __syncthreads();
  int64_t run = part[threadIdx.x];
  for (int64_t i = b; i < e; ++i) {
    out[i] = (int32_t)run;
    run += v[i] + add;
  }
}

// both directions of every kNN pair into the rows' slots (order within a row arbitrary)
__global__ void k_knn_fill(const int32_t* __restrict__ nbr, const float* __restrict__ sval, int64_t n, int k,
                           const int32_t* __restrict__ off, int32_t* __restrict__ fill, int32_t* __restrict__ ecol,
                           float* __restrict__ eval) {
  const int64_t total = n * k;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = (int32_t)(e / k), j = nbr[e];
    const float s = sval[e];
    const int32_t a = off[i] + atomicAdd(&fill[i], 1);
    ecol[a] = j;
    eval[a] = s;
    const int32_t bslot = off[j] + atomicAdd(&fill[j], 1);
    ecol[bslot] = i;
    eval[bslot] = s;
  }
}

// One warp per row.  A row holds each column at most twice (the forward kNN entry and the
// reverse one).  pass 0: element x represents its column when no other element of the column
// has a larger value (or the same value at a lower position); flags and counts.  pass 1: the
// representative's rank among the row's representatives by column is its CSR position.
__global__ void k_knn_dedupe(const int32_t* __restrict__ off, const int32_t* __restrict__ ecol,
                             const float* __restrict__ eval, int64_t n, int pass, uint8_t* __restrict__ erep,
                             int32_t* __restrict__ cntu, const int32_t* __restrict__ rowptr,
                             int32_t* __restrict__ colidx, float* __restrict__ sout) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n) return;
  const int32_t b = off[i], L = off[i + 1] - off[i];
  int reps = 0;
  for (int x = lane; x < L; x += 32) {
    const int32_t cx = ecol[b + x];
    const float vx = eval[b + x];
    if (pass == 0) {
      bool rep = true;
      for (int y = 0; y < L; ++y) {
        const int32_t cy = ecol[b + y];
        const float vy = eval[b + y];
        if (cy == cx && y != x && (vy > vx || (vy == vx && y < x))) rep = false;
      }
      erep[b + x] = rep ? 1 : 0;
      reps += rep ? 1 : 0;
    } else if (erep[b + x]) {
      int rank = 0;
      for (int y = 0; y < L; ++y) rank += (erep[b + y] && ecol[b + y] < cx) ? 1 : 0;
      colidx[rowptr[i] + rank] = cx;
      sout[rowptr[i] + rank] = vx;
    }
  }
  if (pass == 0) {
    for (int o = 16; o > 0; o >>= 1) reps += __shfl_xor_sync(0xffffffffu, reps, o);
    if (lane == 0) cntu[i] = reps;
  }
}

// degrees (fixed order: column order, lane-strided then a fixed butterfly)
__global__ void k_knn_degree(const int32_t* __restrict__ rowptr, const float* __restrict__ sv, int64_t n,
                             float* __restrict__ deg) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n) return;
  double s = 0.0;
  for (int32_t e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) s += (double)sv[e];
  s = warp_sum(s);
  if (lane == 0) deg[i] = (float)s;
}

__global__ void k_knn_normalize(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                const float* __restrict__ sv, const float* __restrict__ deg, int64_t n,
                                float* __restrict__ ahat) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n) return;
  for (int32_t e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32)
    ahat[e] = (float)((double)sv[e] / sqrt((double)deg[i] * (double)deg[colidx[e]]));
}

__global__ void k_contingency(const int32_t* __restrict__ truth, const int32_t* __restrict__ pred, int64_t n, int k1,
                              int k2, unsigned long long* __restrict__ table, int* __restrict__ bad) {
  extern __shared__ unsigned int hist[];
  for (int e = threadIdx.x; e < k1 * k2; e += blockDim.x) hist[e] = 0u;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int a = truth[i], b = pred[i];
    if (a < 0 || a >= k1 || b < 0 || b >= k2) { atomicOr(bad, 1); continue; }
    atomicAdd(&hist[a * k2 + b], 1u);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < k1 * k2; e += blockDim.x)
    if (hist[e]) atomicAdd(&table[e], (unsigned long long)hist[e]);
}

template <typename T>
__global__ void k_assign(const T* __restrict__ F, int64_t n, int64_t ld, int64_t col0, int r, int32_t* __restrict__ lab) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T* row = F + i * ld + col0;
    int best = 0;
    T bv = row[0];
    for (int c = 1; c < r; ++c)
      if (row[c] > bv) { bv = row[c]; best = c; }
    lab[i] = best;
  }
}

template <int K>
void launch_knn(const float* X, int64_t n, int d, int k, int32_t* nbr, float* nd2, int* bad, cudaStream_t s) {
  const size_t smem = (size_t)(QB + CB) * (d + 1) * sizeof(float);
  cudaFuncSetAttribute(k_knn<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_knn<K><<<(unsigned)((n + QB - 1) / QB), QB, smem, s>>>(X, n, d, k, nbr, nd2, bad);
}

// Best one-to-one matching maximising the matched count: the Hungarian method with potentials
// on the square cost matrix -T (padded with zeros), shortest augmenting paths one row at a
// time.  Returns the matched total.
long long max_matching(const std::vector<long long>& T, int rows, int cols) {
  const int m = std::max(rows, cols);
  auto cost = [&](int a, int b) -> long long { return (a < rows && b < cols) ? -T[(size_t)a * cols + b] : 0; };
  const long long INF = std::numeric_limits<long long>::max() / 4;
  std::vector<long long> u(m + 1, 0), v(m + 1, 0);
  std::vector<int> match(m + 1, 0), way(m + 1, 0);  // match[col] = row (1-based; 0 = free)
  for (int a = 1; a <= m; ++a) {
    match[0] = a;
    int j0 = 0;
    std::vector<long long> minv(m + 1, INF);
    std::vector<char> used(m + 1, 0);
    do {
      used[j0] = 1;
      const int a0 = match[j0];
      long long delta = INF;
      int j1 = 0;
      for (int j = 1; j <= m; ++j) {
        if (used[j]) continue;
        const long long cur = cost(a0 - 1, j - 1) - u[a0] - v[j];
        if (cur < minv[j]) { minv[j] = cur; way[j] = j0; }
        if (minv[j] < delta) { delta = minv[j]; j1 = j; }
      }
      for (int j = 0; j <= m; ++j) {
        if (used[j]) { u[match[j]] += delta; v[j] -= delta; }
        else minv[j] -= delta;
      }
      j0 = j1;
    } while (match[j0] != 0);
    do {
      const int j1 = way[j0];
      match[j0] = match[j1];
      j0 = j1;
    } while (j0);
  }
  long long total = 0;
  for (int j = 1; j <= m; ++j)
    if (match[j] >= 1 && match[j] <= rows && j <= cols) total += T[(size_t)(match[j] - 1) * cols + (j - 1)];
  return total;
}

}  // namespace
}  // namespace snmf

using namespace snmf;

extern "C" snmf_status snmf_knn_graph(const float* X, int64_t n, int d, int k, int sigma_rank, int32_t* rowptr,
                                      int32_t* colidx, float* a_hat, float* s_values, float* degree,
                                      int64_t capacity, int64_t* nnz, void* stream) {
  if (!X || !rowptr || !colidx || !a_hat || !nnz || n < 2 || d < 1 || d > 1024 || k < 1 || k > KMAX || k >= n ||
      sigma_rank < 1 || sigma_rank > k || 2 * n * (int64_t)k > INT_MAX)
    return SNMF_ERR_ARG;
  if ((size_t)(QB + CB) * (d + 1) * sizeof(float) > 200 * 1024) return SNMF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t nk = n * k;
  int32_t *nbr = nullptr, *cnt = nullptr, *off = nullptr, *fill = nullptr, *ecol = nullptr, *cntu = nullptr;
  float *nd2 = nullptr, *sval = nullptr, *eval = nullptr, *sv = nullptr, *dg = nullptr;
  uint8_t* erep = nullptr;
  int* bad = nullptr;
  auto cleanup = [&] {
    cudaFree(bad);
    cudaFree(nbr); cudaFree(cnt); cudaFree(off); cudaFree(fill); cudaFree(ecol); cudaFree(cntu); cudaFree(erep);
    cudaFree(nd2); cudaFree(sval); cudaFree(eval); cudaFree(sv); cudaFree(dg);
  };
  snmf_status st = SNMF_OK;
#define KCK(call)                                                                                        \
  do {                                                                                                   \
    const cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) { st = e_ == cudaErrorMemoryAllocation ? SNMF_ERR_OOM : SNMF_ERR_CUDA; cleanup(); return st; } \
  } while (0)
  KCK(cudaMalloc(&nbr, nk * sizeof(int32_t)));
  KCK(cudaMalloc(&nd2, nk * sizeof(float)));
  KCK(cudaMalloc(&sval, nk * sizeof(float)));
  KCK(cudaMalloc(&cnt, n * sizeof(int32_t)));
  KCK(cudaMalloc(&fill, n * sizeof(int32_t)));
  KCK(cudaMalloc(&off, (n + 1) * sizeof(int32_t)));
  KCK(cudaMalloc(&cntu, n * sizeof(int32_t)));
  KCK(cudaMalloc(&ecol, 2 * nk * sizeof(int32_t)));
  KCK(cudaMalloc(&eval, 2 * nk * sizeof(float)));
  KCK(cudaMalloc(&sv, 2 * nk * sizeof(float)));
  KCK(cudaMalloc(&dg, n * sizeof(float)));
  KCK(cudaMalloc(&erep, 2 * nk));
  KCK(cudaMalloc(&bad, sizeof(int)));
  KCK(cudaMemsetAsync(bad, 0, sizeof(int), s));
  KCK(cudaMemsetAsync(cnt, 0, n * sizeof(int32_t), s));
  KCK(cudaMemsetAsync(fill, 0, n * sizeof(int32_t), s));
  if (k <= 16) launch_knn<16>(X, n, d, k, nbr, nd2, bad, s);
  else launch_knn<32>(X, n, d, k, nbr, nd2, bad, s);
  const int g = (int)std::min<int64_t>((nk + 255) / 256, 152 * 16);
  k_knn_sim<<<g, 256, 0, s>>>(nbr, nd2, n, k, sigma_rank, sval, cnt, bad);
  k_scan<<<1, 1024, 0, s>>>(cnt, n, k, off);  // row slots: k own + in-degree
  k_knn_fill<<<g, 256, 0, s>>>(nbr, sval, n, k, off, fill, ecol, eval);
  const int rb = (int)((n + 7) / 8);
  k_knn_dedupe<<<rb, 256, 0, s>>>(off, ecol, eval, n, 0, erep, cntu, nullptr, nullptr, nullptr);
  k_scan<<<1, 1024, 0, s>>>(cntu, n, 0, rowptr);
  int32_t total = 0;
  int hbad = 0;
  KCK(cudaMemcpyAsync(&total, rowptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  KCK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  KCK(cudaStreamSynchronize(s));
  *nnz = total;
  if (hbad) { cleanup(); return SNMF_ERR_NUMERIC; }
  if (total > capacity) { cleanup(); return SNMF_ERR_ARG; }
  k_knn_dedupe<<<rb, 256, 0, s>>>(off, ecol, eval, n, 1, erep, cntu, rowptr, colidx, sv);
  k_knn_degree<<<rb, 256, 0, s>>>(rowptr, sv, n, dg);
  k_knn_normalize<<<rb, 256, 0, s>>>(rowptr, colidx, sv, dg, n, a_hat);
  if (s_values) KCK(cudaMemcpyAsync(s_values, sv, (size_t)total * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (degree) KCK(cudaMemcpyAsync(degree, dg, (size_t)n * sizeof(float), cudaMemcpyDeviceToDevice, s));
  KCK(cudaGetLastError());
  KCK(cudaStreamSynchronize(s));
#undef KCK
  cleanup();
  return SNMF_OK;
}

extern "C" snmf_status snmf_cluster_scores(const int32_t* truth, const int32_t* pred, int64_t n, int k_true,
                                           int k_pred, int64_t* table, double* ari, double* accuracy, void* stream) {
  if (!truth || !pred || n < 2 || k_true < 1 || k_pred < 1 || k_true > 512 || k_pred > 512 ||
      (int64_t)k_true * k_pred > 4096)
    return SNMF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* dt = nullptr;
  int* bad = nullptr;
  const size_t tb = (size_t)k_true * k_pred * sizeof(unsigned long long);
  if (cudaMalloc(&dt, tb) != cudaSuccess) return SNMF_ERR_OOM;
  if (cudaMalloc(&bad, sizeof(int)) != cudaSuccess) { cudaFree(dt); return SNMF_ERR_OOM; }
  std::vector<unsigned long long> ht((size_t)k_true * k_pred);
  int hbad = 0;
  cudaError_t e = cudaMemsetAsync(dt, 0, tb, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 4);
    k_contingency<<<blocks, 256, (size_t)k_true * k_pred * sizeof(unsigned), s>>>(truth, pred, n, k_true, k_pred, dt, bad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(ht.data(), dt, tb, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(dt);
  cudaFree(bad);
  if (e != cudaSuccess) return SNMF_ERR_CUDA;
  if (hbad) return SNMF_ERR_ARG;
  std::vector<long long> T(ht.begin(), ht.end());
  if (table) for (size_t x = 0; x < T.size(); ++x) table[x] = T[x];
  // adjusted Rand index (Hubert and Arabie) in FP64 from the table
  auto comb = [](double x) { return x * (x - 1.0) / 2.0; };
  double idx = 0.0, sa = 0.0, sb = 0.0, tot = 0.0;
  std::vector<double> rs(k_true, 0.0), cs(k_pred, 0.0);
  for (int a = 0; a < k_true; ++a)
    for (int b = 0; b < k_pred; ++b) {
      const double v = (double)T[(size_t)a * k_pred + b];
      idx += comb(v);
      rs[a] += v;
      cs[b] += v;
      tot += v;
    }
  for (double v : rs) sa += comb(v);
  for (double v : cs) sb += comb(v);
  const double expv = sa * sb / comb(tot), mx = 0.5 * (sa + sb);
  if (ari) *ari = (mx != expv) ? (idx - expv) / (mx - expv) : 1.0;
  if (accuracy) *accuracy = (double)max_matching(T, k_true, k_pred) / tot;
  return SNMF_OK;
}

// exported for capi.cu (the handle's factor buffers live there)
namespace snmf {
void launch_assign(int tdtype, const void* F, int64_t n, int64_t ld, int64_t col0, int r, int32_t* lab, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
  if (tdtype == 0) k_assign<double><<<blocks, 256, 0, s>>>((const double*)F, n, ld, col0, r, lab);
  else k_assign<float><<<blocks, 256, 0, s>>>((const float*)F, n, ld, col0, r, lab);
}
}  // namespace snmf
