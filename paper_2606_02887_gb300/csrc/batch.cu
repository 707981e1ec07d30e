// Uneven batch: many independent SNMPBB problems (penalty form, Sec. 2.1 / Algorithm 1)
// of different sizes n_p and ranks r_p, solved together on one GPU.
//
// Every step of Algorithm 1 is ONE grouped launch over a work list of (problem, tile)
// items that covers all problems; items are ordered by problem size, largest first, so
// the long items start early.  Each item's CTA runs the same device bodies as the
// single-problem kernels with that problem's sizes and offsets.  A per-problem arrival
// counter lets the last CTA of a problem run the problem's FP64 control step (line
// search, BB step, convergence test) inside the producing launch, so no CTA ever waits
// for another and the launch boundaries are the only synchronisation.  One outer
// iteration of all problems is captured once into a CUDA graph and replayed; a problem
// that has converged drops out through its active flag (its items return at once).
//
// Layout in HBM:
//   A_all  rows of all problems packed (problem p at rows arow_p .. arow_p + n_p), one
//          common pitch lda = n_max rounded up to 64, zero beyond column n_p; FP64, FP32
//          or BF16 (the stored operator; ||A_p||^2 is taken from the stored values)
//   factors (W, Ht, B, gradients, Z, D, ...): problem p is an n_p x r_p row-major block at
//          element offset xoff_p, blocks packed in problem order
//   r x r matrices (G, FP64 Grams) and partial-sum slots: per-problem regions, offsets in
//          the BProb table.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <numeric>
#include <string>
#include <vector>

#include "ax_tc.cuh"
#include "batch.cuh"
#include "common.cuh"
#include "rowops.cuh"
#include "rowops_dev.cuh"

namespace snmf {

namespace {

constexpr int kPBM = 64;      // product rows per work item
constexpr int kGChunk = 256;  // Gram rows per work item

// Per-problem sizes and offsets (device-resident table).
struct BProb {
  int64_t n;
  int r;
  int nrt;      // row-kernel items (row tiles of the row GEMM)
  int npt;      // product items
  int gch;      // Gram items (row chunks)
  int slot0;    // first partial slot of the row kernels (= index of its first row item)
  int pslot0;   // first partial slot of the product (= index of its first product item)
  int ntt;      // tensor-core product items (128-row tiles; BF16 A)
  int tslot0;   // first partial slot of the tensor-core product
  int64_t arow; // first row in A_all
  int64_t xoff; // element offset of the problem's factor blocks
  int64_t goff; // offset of its r x r factor-type matrix
  int64_t g3off;// offset of its three FP64 r x r Grams
  int64_t gpoff;// offset (doubles) of its Gram chunk partials
  double lam;   // penalty weight lambda_p
  double normA2;// ||A_p||_F^2 of the stored values
};

__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ double to_f(double v) { return v; }

template <typename TD>
__device__ __forceinline__ TD from_d(double v) { return (TD)v; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_d<__nv_bfloat16>(double v) { return __float2bfloat16_rn((float)v); }

// A_p (n x n, ld n, source type) -> rows of A_all (pitch lda, zero beyond column n)
template <typename TS, typename TD>
__global__ void k_bconvert(const TS* __restrict__ src, int64_t n, TD* __restrict__ dst, int64_t lda) {
  const int64_t total = n * lda;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / lda, k = e % lda;
    dst[e] = from_d<TD>(k < n ? (double)src[i * n + k] : 0.0);
  }
}

// sum of squares and sum of the stored A_p, FP64 partial per product item
template <typename TA>
__global__ void __launch_bounds__(256)
k_bsums(const TA* __restrict__ A, int64_t lda, const BProb* __restrict__ probs, const int2* __restrict__ items,
        double* __restrict__ part) {
  __shared__ double sh[32];
  const int2 it = items[blockIdx.x];
  const BProb& pb = probs[it.x];
  const int64_t n = pb.n;
  const int64_t r0 = (int64_t)it.y * kPBM;
  const int64_t rows = min((int64_t)kPBM, n - r0);
  double s2 = 0.0, s1 = 0.0;
  for (int64_t e = threadIdx.x; e < rows * n; e += blockDim.x) {
    const int64_t i = r0 + e / n, k = e % n;
    const double v = (double)to_f(A[(pb.arow + i) * lda + k]);
    s2 += v * v;
    s1 += v;
  }
  s2 = block_sum(s2, sh);
  s1 = block_sum(s1, sh);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s2;
    part[2 * blockIdx.x + 1] = s1;
  }
}

// per-problem fixed-order sum of the item partials: out[2p] = ||A_p||^2, out[2p+1] = sum
__global__ void k_bsums_reduce(const BProb* __restrict__ probs, const double* __restrict__ part,
                               double* __restrict__ out) {
  const BProb& pb = probs[blockIdx.x];
  double s2 = 0.0, s1 = 0.0;
  for (int t = threadIdx.x; t < pb.npt; t += 32) {
    s2 += part[2 * (pb.pslot0 + t)];
    s1 += part[2 * (pb.pslot0 + t) + 1];
  }
  s2 = warp_sum(s2);
  s1 = warp_sum(s1);
  if (threadIdx.x == 0) {
    out[2 * blockIdx.x] = s2;
    out[2 * blockIdx.x + 1] = s1;
  }
}

// Grouped product (CUDA cores): item (p, t) computes rows t*64 .. of Y_p = A_p X_p over the
// full K = n_p (A_p rows streamed once, X_p from L2), epilogue Y += lambda_p X and, when
// P1 is given, the per-item partial <P1, A_p X_p> in the item's partial slot.  CTAs beyond
// the *cnt items of the (compacted) list return at once.
template <typename T, typename TA>
__global__ void __launch_bounds__(256)
k_bgemm(const TA* __restrict__ A, int64_t lda, const BProb* __restrict__ probs, const int2* __restrict__ items,
        const int* __restrict__ cnt, const T* __restrict__ X, T* __restrict__ Y, int add_lam,
        const T* __restrict__ P1, double* __restrict__ part, const Ctl* __restrict__ ctl, const int* __restrict__ run) {
  constexpr int BK = sizeof(T) == 8 ? 16 : 32;
  if ((int)blockIdx.x >= *cnt) return;
  constexpr int NA = kPBM * BK / 256;
  constexpr int NX = BK * 64 / 256;
  __shared__ T As[2][BK][kPBM + 4];
  __shared__ T Xs[2][BK][64 + 4];
  __shared__ T sh[32];
  const int2 it = items[blockIdx.x];
  const int p = it.x;
  const BProb& pb = probs[p];
  const int64_t n = pb.n;
  const int r = pb.r;
  const int64_t row0 = (int64_t)it.y * kPBM;
  const T* Xp = X + pb.xoff;
  const TA* Ap = A + (pb.arow + row0) * lda;
  const bool live = !(run && *run == 0) && !(ctl && !ctl[p].active);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T d1 = T(0);
  if (live) {
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    T ra[NA], rx[NX];
    auto load = [&](int64_t k0) {
#pragma unroll
      for (int m = 0; m < NA; ++m) {
        const int e = threadIdx.x + 256 * m;
        const int rr = e / BK, kk = e % BK;
        ra[m] = (row0 + rr < n && k0 + kk < n) ? (T)to_f(Ap[(int64_t)rr * lda + k0 + kk]) : T(0);
      }
#pragma unroll
      for (int m = 0; m < NX; ++m) {
        const int e = threadIdx.x + 256 * m;
        const int kr = e >> 6, c = e & 63;
        rx[m] = (k0 + kr < n && c < r) ? Xp[(k0 + kr) * r + c] : T(0);
      }
    };
    auto store = [&](int buf) {
#pragma unroll
      for (int m = 0; m < NA; ++m) {
        const int e = threadIdx.x + 256 * m;
        As[buf][e % BK][e / BK] = ra[m];
      }
#pragma unroll
      for (int m = 0; m < NX; ++m) {
        const int e = threadIdx.x + 256 * m;
        Xs[buf][e >> 6][e & 63] = rx[m];
      }
    };
    int buf = 0;
    load(0);
    store(0);
    __syncthreads();
    for (int64_t k0 = 0; k0 < n; k0 += BK) {
      const bool more = k0 + BK < n;
      if (more) load(k0 + BK);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T a[4], x[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) x[j] = Xs[buf][kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], x[j], acc[i][j]);
      }
      if (more) store(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
    const T lam = (T)pb.lam;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t row = row0 + ty + 16 * i;
      if (row >= n) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = tx + 16 * j;
        if (c >= r) continue;
        const int64_t idx = pb.xoff + row * r + c;
        T y = acc[i][j];
        if (P1) d1 += P1[idx] * y;
        if (add_lam) y += lam * X[idx];
        Y[idx] = y;
      }
    }
  }
  if (part) {
    d1 = block_sum_t(d1, sh);
    if (threadIdx.x == 0) part[(int64_t)(pb.pslot0 + it.y) * kNQ] = (double)d1;
  }
}

// Grouped Gram X_p^T Y_p (pair `pair` of `npairs`), chunk items; lambda_p on the diagonal
// of the factor-type copy when use_lam; rho_p fused in the last CTA (FP32 working type).
template <typename T>
__global__ void __launch_bounds__(256)
k_bgram(const BProb* __restrict__ probs, const int2* __restrict__ items, const int* __restrict__ cnt,
        const T* __restrict__ X, const T* __restrict__ Y, double* __restrict__ gpart, int pair, int npairs,
        const Ctl* __restrict__ ctl, const int* run, double* __restrict__ G64, T* __restrict__ GT, int tpair,
        int use_lam, unsigned* __restrict__ counters, Ctl* __restrict__ rho_ctl, int rho_iters) {
  if ((int)blockIdx.x >= *cnt) return;  // beyond the (compacted) list
  const int2 it = items[blockIdx.x];
  const BProb& pb = probs[it.x];
  gram_body<T>(X + pb.xoff, Y + pb.xoff, pb.n, pb.r, 1, pb.r, kGChunk, 1, gpart + pb.gpoff, pair, npairs,
               ctl ? ctl + it.x : nullptr, run, G64 + pb.g3off, GT ? GT + pb.goff : nullptr, tpair,
               use_lam ? pb.lam : 0.0, counters + 3 * it.x, rho_ctl ? rho_ctl + it.x : nullptr, rho_iters,
               1.0, 0.0, it.y, pb.gch, 0);
}

// rho_p = ||G_p||_2 (FP64 working type), one block per problem
template <typename PT>
__global__ void __launch_bounds__(256)
k_brho(const BProb* __restrict__ probs, const double* __restrict__ G64, int iters, Ctl* __restrict__ ctl) {
  __shared__ double sh[32];
  __shared__ PT v[64], w[64];
  __shared__ PT Gs[64 * 64];
  const BProb& pb = probs[blockIdx.x];
  Ctl& c = ctl[blockIdx.x];
  if (!c.active) return;
  rho_body<PT>(G64 + pb.g3off, pb.r, iters, 1.0, 0.0, c, v, w, Gs, sh);
}

// Grouped row GEMM with the fused Algorithm-1 epilogues and the per-problem control step.
template <typename T, int OP, int EPI, int BM, int NC>
__global__ void __launch_bounds__(256, 2)
k_brow(RowArgs base, const BProb* __restrict__ probs, const int2* __restrict__ items, const int* __restrict__ cnt) {
  if ((int)blockIdx.x >= *cnt) return;  // beyond the (compacted) list
  const int2 it = items[blockIdx.x];
  const BProb& pb = probs[it.x];
  RowArgs a = base;
  const size_t o = (size_t)pb.xoff * sizeof(T);
  auto cs = [&](const void* q) -> const void* { return q ? (const void*)((const char*)q + o) : nullptr; };
  auto ms = [&](void* q) -> void* { return q ? (void*)((char*)q + o) : nullptr; };
  a.n = pb.n;
  a.r = pb.r;
  a.b = 1;
  a.ld = pb.r;
  a.G = (const T*)base.G + pb.goff;
  a.X = cs(base.X); a.g_in = cs(base.g_in); a.Zin = cs(base.Zin); a.Din = cs(base.Din);
  a.B = cs(base.B); a.LX = nullptr;
  a.Xout = ms(base.Xout); a.gout = ms(base.gout); a.Dout = ms(base.Dout); a.D2out = ms(base.D2out);
  a.Din2 = cs(base.Din2); a.gZout = ms(base.gZout);
  a.Xold = cs(base.Xold); a.gold = cs(base.gold); a.Zold = cs(base.Zold); a.gZold = cs(base.gZold);
  a.Wcur = cs(base.Wcur); a.gWcur = cs(base.gWcur);
  a.ctl = base.ctl + it.x;
  a.part = base.part + (int64_t)pb.slot0 * kNQ;
  a.counters = base.counters + it.x;
  a.G64fix = base.G64fix ? base.G64fix + pb.g3off : nullptr;
  a.P.nr = pb.n * (int64_t)pb.r;
  rowgemm_body<T, OP, EPI, BM, NC>(a, 0, it.y, 0, 1, (unsigned)pb.nrt);
}

// The same for problems with r <= 32 through the shared-memory tile body (TileCfg rows per
// item); dynamic shared memory of rowtile_smem bytes.
template <typename T, int OP, int EPI, int NC>
__global__ void __launch_bounds__(256, EPI == EPI_GRAD ? 2 : 3)
k_browt(RowArgs base, const BProb* __restrict__ probs, const int2* __restrict__ items, const int* __restrict__ cnt) {
  extern __shared__ __align__(16) unsigned char tsm[];
  if ((int)blockIdx.x >= *cnt) return;  // beyond the (compacted) list
  const int2 it = items[blockIdx.x];
  const BProb& pb = probs[it.x];
  RowArgs a = base;
  const size_t o = (size_t)pb.xoff * sizeof(T);
  auto cs = [&](const void* q) -> const void* { return q ? (const void*)((const char*)q + o) : nullptr; };
  auto ms = [&](void* q) -> void* { return q ? (void*)((char*)q + o) : nullptr; };
  a.n = pb.n;
  a.r = pb.r;
  a.b = 1;
  a.ld = pb.r;
  a.G = (const T*)base.G + pb.goff;
  a.X = cs(base.X); a.g_in = cs(base.g_in); a.Zin = cs(base.Zin); a.Din = cs(base.Din);
  a.B = cs(base.B); a.LX = nullptr;
  a.Xout = ms(base.Xout); a.gout = ms(base.gout); a.Dout = ms(base.Dout); a.D2out = ms(base.D2out);
  a.Din2 = cs(base.Din2); a.gZout = ms(base.gZout);
  a.Xold = cs(base.Xold); a.gold = cs(base.gold); a.Zold = cs(base.Zold); a.gZold = cs(base.gZold);
  a.Wcur = cs(base.Wcur); a.gWcur = cs(base.gWcur);
  a.ctl = base.ctl + it.x;
  a.part = base.part + (int64_t)pb.slot0 * kNQ;
  a.counters = base.counters + it.x;
  a.G64fix = base.G64fix ? base.G64fix + pb.g3off : nullptr;
  a.P.nr = pb.n * (int64_t)pb.r;
  rowtile_body<T, OP, EPI, NC>(a, 0, it.y, (unsigned)pb.nrt, reinterpret_cast<T*>(tsm));
}

// Work-list compaction: the items of the problems that are still active, in the original
// order, for the five lists (row items of the tile body, row items of the generic body,
// Gram chunks, CUDA-core product tiles, tensor-core product tiles); counts to cnt[0..4];
// *run = any problem active.  One block; problems in list order `order`.
struct CompactArgs {
  const int* order;
  int nprob;
  const Ctl* ctl;
  const int2* full[4];
  int2* comp[4];
  const TcItem* tfull;
  TcItem* tcomp;
  const int* pst;   // [5][nprob]: first item of problem p in each full list
  const int* psz;   // [5][nprob]: items of problem p in each list
  int* cnt;
  int* run;
};

__global__ void __launch_bounds__(1024) k_bcompact(CompactArgs ca) {
  __shared__ int sc[5][1024];
  const int tid = threadIdx.x;
  const int per = (ca.nprob + 1023) / 1024;
  const int i0 = min(ca.nprob, tid * per), i1 = min(ca.nprob, i0 + per);
  int loc[5] = {0, 0, 0, 0, 0};
  int any = 0;
  for (int i = i0; i < i1; ++i) {
    const int p = ca.order[i];
    if (!ca.ctl[p].active) continue;
    any = 1;
    for (int L = 0; L < 5; ++L) loc[L] += ca.psz[L * ca.nprob + p];
  }
  for (int L = 0; L < 5; ++L) sc[L][tid] = loc[L];
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {  // inclusive scan
    int v[5];
    for (int L = 0; L < 5; ++L) v[L] = tid >= off ? sc[L][tid - off] : 0;
    __syncthreads();
    for (int L = 0; L < 5; ++L) sc[L][tid] += v[L];
    __syncthreads();
  }
  int pos[5];
  for (int L = 0; L < 5; ++L) pos[L] = sc[L][tid] - loc[L];
  for (int i = i0; i < i1; ++i) {
    const int p = ca.order[i];
    if (!ca.ctl[p].active) continue;
    for (int L = 0; L < 5; ++L) {
      const int st = ca.pst[L * ca.nprob + p], sz = ca.psz[L * ca.nprob + p];
      for (int t = 0; t < sz; ++t) {
        if (L < 4) ca.comp[L][pos[L] + t] = ca.full[L][st + t];
        else ca.tcomp[pos[L] + t] = ca.tfull[st + t];
      }
      pos[L] += sz;
    }
  }
  any = __syncthreads_or(any);
  if (tid == 1023)
    for (int L = 0; L < 5; ++L) ca.cnt[L] = sc[L][1023];
  if (tid == 0) *ca.run = any;
}


// final per-problem statistics (one warp per problem); tc: the product partials are per
// tensor-core item
__global__ void k_bfinal(Ctl* __restrict__ ctl, const double* __restrict__ pax, const double* __restrict__ prow,
                         const double* __restrict__ G64p, const BProb* __restrict__ probs, int tc) {
  __shared__ double sh[32];
  const BProb& pb = probs[blockIdx.x];
  const int64_t rr = (int64_t)pb.r * pb.r;
  const double* G = G64p + pb.g3off;
  const int ps = tc ? pb.tslot0 : pb.pslot0, np_ = tc ? pb.ntt : pb.npt;
  final_pen_body(ctl[blockIdx.x], pax + (int64_t)ps * kNQ, np_, prow + (int64_t)pb.slot0 * kNQ,
                 pb.nrt, G, G + rr, G + 2 * rr, 1, 0, pb.r, pb.normA2, sh);
}

enum { XB_W = 0, XB_HT, XB_B, XB_G, XB_Z, XB_D, XB_GZ, XB_D2, XB_N };

}  // namespace

struct BatchCtx {
  int nprob = 0;
  snmf_options opt{};
  int prec = SNMF_F32, tdtype = 1, a_dtype = 1;  // a_dtype: 0 f64, 1 f32, 2 bf16
  size_t esz = 4;
  std::vector<BProb> hp;
  BProb* dp = nullptr;
  std::vector<int2> h_row, h_rowg, h_prod, h_gram;  // row items: tile body (r <= 32) / generic
  int2* it_rowg = nullptr;
  int nslot = 0;
  std::vector<TcItem> h_tc;        // BF16: tensor-core product items
  TcItem* it_tc = nullptr;
  void *xh = nullptr, *xl = nullptr;  // BF16 hi / lo parts of the product operand (transposed)
  int64_t xt_rows = 0;
  int* dev_err = nullptr;
  long long budget = 2000000000LL;
  int tc_fail = 0;
  int2 *it_row = nullptr, *it_prod = nullptr, *it_gram = nullptr;
  // compacted lists of the active problems (rebuilt by k_bcompact), per-problem ranges in the
  // full lists, counts (cnt_full: constant full sizes; cnt_act: compacted)
  int2 *c_row = nullptr, *c_rowg = nullptr, *c_gram = nullptr, *c_prod = nullptr;
  TcItem* c_tc = nullptr;
  int *pst = nullptr, *psz = nullptr, *d_order = nullptr, *cnt_full = nullptr, *cnt_act = nullptr;
  std::vector<int> order;
  bool use_full = false;  // launches being recorded cover every problem (final evaluation)
  bool accurate = false;  // BF16: FP32 CUDA-core product instead of tcgen05 (final evaluation)
  int64_t lda = 0, rows_total = 0, xtot = 0;
  void* A = nullptr;
  void* buf[XB_N] = {};
  double *prow = nullptr, *pax = nullptr, *gpart = nullptr, *G64fix = nullptr, *G64p = nullptr, *dsc = nullptr;
  void* GT = nullptr;
  Ctl* ctl = nullptr;
  int* run = nullptr;
  unsigned* counters = nullptr;
  __nv_bfloat16* mlp_w = nullptr;
  float *rec_feat = nullptr, *rec_targ = nullptr;
  int* rec_count = nullptr;
  int rec_cap = 0;
  int* h_flag = nullptr;
  cudaStream_t user = nullptr, s = nullptr;
  cudaStream_t s2 = nullptr;  // side branch: grouped Gram beside the grouped product
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, evsync = nullptr, evfork = nullptr, evjoin = nullptr;
  cudaGraphExec_t exec[3] = {nullptr, nullptr, nullptr};
  int nodes[3] = {0, 0, 0};
  std::vector<Ctl> h_ctl;
  std::vector<double> sumA;
  bool have_result = false;
};

namespace {

#define BCK(call)                                                                    \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      *err = std::string(#call) + ": " + cudaGetErrorString(e_);                     \
      return e_ == cudaErrorMemoryAllocation ? SNMF_ERR_OOM : SNMF_ERR_CUDA;         \
    }                                                                                \
  } while (0)

Params bparams(const BatchCtx* b) {
  Params P{};
  const snmf_options& o = b->opt;
  P.formulation = 0;
  P.memory = o.nonmonotone_M;
  P.bb = o.bb_variant;
  P.max_ls = o.max_ls;
  P.max_iter = o.max_iter;
  P.power_iters = o.power_iters;
  P.controller = o.step_controller;
  P.theta = o.theta;
  P.phi = o.phi;
  P.eta = o.eta;
  P.alpha_min = o.alpha_min;
  P.alpha_max = o.alpha_max;
  P.beta_shrink = o.beta_shrink;
  P.tol = o.tol;
  P.rho_factor = 1.0;
  P.gamma = 0.0;
  P.mlp_w = b->mlp_w;
  P.rec_feat = o.step_controller == 2 ? b->rec_feat : nullptr;
  P.rec_targ = b->rec_targ;
  P.rec_count = b->rec_count;
  P.rec_cap = b->rec_cap;
  return P;
}

int row_bm(const BatchCtx* b) { return b->tdtype == 0 ? 32 : 64; }

// ---- grouped launches -------------------------------------------------------------------
// list L (0 row tile body, 1 row generic body, 2 Gram, 3 CUDA-core product, 4 tensor-core
// product) and its device count for the launches being recorded
const int* bcnt(const BatchCtx* b, int L) { return (b->use_full ? b->cnt_full : b->cnt_act) + L; }
const int2* blist(const BatchCtx* b, int L) {
  if (L == 0) return b->use_full ? b->it_row : b->c_row;
  if (L == 1) return b->use_full ? b->it_rowg : b->c_rowg;
  if (L == 2) return b->use_full ? b->it_gram : b->c_gram;
  return b->use_full ? b->it_prod : b->c_prod;
}

void bprod(BatchCtx* b, const void* X, void* Y, const void* P1, double* part, const Ctl* ctl, const int* run) {
  const unsigned g = (unsigned)b->h_prod.size();
  if (b->a_dtype == 2 && !b->accurate) {
    // tcgen05: X_p split into BF16 hi / lo parts (transposed), then one CTA per 128-row tile
    const int nt = (int)b->h_tc.size();
    const TcItem* tl = b->use_full ? b->it_tc : b->c_tc;
    launch_bsplit_x(tl, nt, bcnt(b, 4), (const float*)X, b->xh, b->xl, b->lda, ctl, sizeof(Ctl),
                    offsetof(Ctl, active), run, b->s);
    if (launch_bgemm_tc(b->A, b->lda, b->rows_total, b->xh, b->xl, b->xt_rows, tl, nt, bcnt(b, 4), (const float*)X,
                        (float*)Y, 1, (const float*)P1, part, kNQ, ctl, sizeof(Ctl), offsetof(Ctl, active), run,
                        b->dev_err, b->budget, b->s) < 0)
      b->tc_fail = tc_last_status() ? tc_last_status() : -1;
    return;
  }
  const int2* il = blist(b, 3);
  const int* c = bcnt(b, 3);
  if (b->tdtype == 0)
    k_bgemm<double, double><<<g, 256, 0, b->s>>>((const double*)b->A, b->lda, b->dp, il, c, (const double*)X,
                                                 (double*)Y, 1, (const double*)P1, part, ctl, run);
  else if (b->a_dtype == 2)
    k_bgemm<float, __nv_bfloat16><<<g, 256, 0, b->s>>>((const __nv_bfloat16*)b->A, b->lda, b->dp, il, c,
                                                       (const float*)X, (float*)Y, 1, (const float*)P1, part,
                                                       ctl, run);
  else
    k_bgemm<float, float><<<g, 256, 0, b->s>>>((const float*)b->A, b->lda, b->dp, il, c, (const float*)X,
                                               (float*)Y, 1, (const float*)P1, part, ctl, run);
}

void bgram(BatchCtx* b, const void* X, const void* Y, int pair, int npairs, const Ctl* ctl, const int* run,
           double* G64, void* GT, int tpair, int use_lam, Ctl* rho_ctl, cudaStream_t st = nullptr) {
  const unsigned g = (unsigned)b->h_gram.size();
  const int it = b->opt.power_iters;
  if (!st) st = b->s;
  if (b->tdtype == 0)
    k_bgram<double><<<g, 256, 0, st>>>(b->dp, blist(b, 2), bcnt(b, 2), (const double*)X, (const double*)Y,
                                       b->gpart, pair, npairs, ctl, run, G64, (double*)GT, tpair, use_lam,
                                       b->counters, nullptr, it);
  else
    k_bgram<float><<<g, 256, 0, st>>>(b->dp, blist(b, 2), bcnt(b, 2), (const float*)X, (const float*)Y,
                                      b->gpart, pair, npairs, ctl, run, G64, (float*)GT, tpair, use_lam,
                                      b->counters, rho_ctl, it);
  if (b->tdtype == 0 && rho_ctl)
    k_brho<double><<<b->nprob, 256, 0, st>>>(b->dp, G64, it, rho_ctl);
}

RowArgs brow_base(BatchCtx* b, const Params& P) {
  RowArgs a{};
  a.G = b->GT;
  a.ctl = b->ctl;
  a.run = b->run;
  a.part = b->prow;
  a.counters = b->counters + 3 * b->nprob;
  a.G64fix = b->G64fix;
  a.P = P;
  return a;
}

template <typename T, int OP, int EPI, int NC>
void launch_browt(BatchCtx* b, const RowArgs& a) {
  static bool attr = false;
  const size_t smem = rowtile_smem<T>(EPI == EPI_DIR ? 2 + NC : 2);
  if (!attr) {
    cudaFuncSetAttribute(k_browt<T, OP, EPI, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  k_browt<T, OP, EPI, NC><<<(unsigned)b->h_row.size(), 256, smem, b->s>>>(a, b->dp, blist(b, 0), bcnt(b, 0));
}

void brow(BatchCtx* b, int op, int epi, const RowArgs& a, int nc = 1) {
  if (!b->h_row.empty()) {
#define BT(T)                                                                    \
    if (epi == EPI_GRAD) {                                                       \
      if (op == OP_LOAD) launch_browt<T, OP_LOAD, EPI_GRAD, 1>(b, a);            \
      else launch_browt<T, OP_UPD, EPI_GRAD, 1>(b, a);                           \
    } else if (nc == 1) launch_browt<T, OP_ZSTEP, EPI_DIR, 1>(b, a);             \
    else launch_browt<T, OP_ZSTEP, EPI_DIR, 2>(b, a);
    if (b->tdtype == 0) { BT(double) } else { BT(float) }
#undef BT
  }
  if (b->h_rowg.empty()) return;
  const unsigned g = (unsigned)b->h_rowg.size();
#define BR(T, O, E, M, C) k_brow<T, O, E, M, C><<<g, 256, 0, b->s>>>(a, b->dp, blist(b, 1), bcnt(b, 1))
#define BR_T(T, M)                                                       \
  if (epi == EPI_GRAD) {                                                 \
    if (op == OP_LOAD) BR(T, OP_LOAD, EPI_GRAD, M, 1);                   \
    else BR(T, OP_UPD, EPI_GRAD, M, 1);                                  \
  } else if (nc == 1) BR(T, OP_ZSTEP, EPI_DIR, M, 1);                    \
  else BR(T, OP_ZSTEP, EPI_DIR, M, 2);  /* record mode is not offered on batch handles */
  if (b->tdtype == 0) { BR_T(double, 32) } else { BR_T(float, 64) }
#undef BR_T
#undef BR
}

// run flag and the compacted work lists of the problems still active
void bany(BatchCtx* b) {
  CompactArgs ca;
  ca.order = b->d_order;
  ca.nprob = b->nprob;
  ca.ctl = b->ctl;
  ca.full[0] = b->it_row; ca.full[1] = b->it_rowg; ca.full[2] = b->it_gram; ca.full[3] = b->it_prod;
  ca.comp[0] = b->c_row; ca.comp[1] = b->c_rowg; ca.comp[2] = b->c_gram; ca.comp[3] = b->c_prod;
  ca.tfull = b->it_tc;
  ca.tcomp = b->c_tc;
  ca.pst = b->pst;
  ca.psz = b->psz;
  ca.cnt = b->cnt_act;
  ca.run = b->run;
  k_bcompact<<<1, 1024, 0, b->s>>>(ca);
}

// one block of Algorithm 1 for all problems (penalty form; mirrors the single-problem path)
void bpen_block(BatchCtx* b, int xv, int xf, bool is_w, const Params& P) {
  void* X = b->buf[xv];
  void* Xf = b->buf[xf];
  // G = Xf^T Xf (+lam I) and rho depend on Xf alone: they run on the side stream beside the
  // product (a fork and a join of the captured graph) and share no buffer with it
  cudaEventRecord(b->evfork, b->s);
  cudaStreamWaitEvent(b->s2, b->evfork, 0);
  bgram(b, Xf, Xf, 0, 1, b->ctl, b->run, b->G64fix, b->GT, 0, 1, b->ctl, b->s2);
  cudaEventRecord(b->evjoin, b->s2);
  bprod(b, Xf, b->buf[XB_B], nullptr, nullptr, b->ctl, b->run);             // B = A Xf + lam Xf
  cudaStreamWaitEvent(b->s, b->evjoin, 0);
  {
    RowArgs a = brow_base(b, P);
    a.X = X; a.B = b->buf[XB_B]; a.gout = b->buf[XB_G];
    a.ctl_mode = is_w ? CTL_START_W : CTL_START_H;
    brow(b, OP_LOAD, EPI_GRAD, a);
  }
  bany(b);
  const int K = b->opt.inner_iters;
  const int nc = b->opt.step_controller == 1 ? 2 : (b->opt.step_controller == 2 ? kNCand : 1);
  for (int k = 0; k < K; ++k) {
    {
      RowArgs a = brow_base(b, P);
      a.B = b->buf[XB_B];
      a.Dout = b->buf[XB_D]; a.gZout = b->buf[XB_GZ];
      a.Wcur = X; a.gWcur = b->buf[XB_G];
      a.X = X; a.g_in = b->buf[XB_G]; a.Xout = b->buf[XB_Z];
      a.want_q = 1;
      a.ctl_mode = CTL_LS;
      a.dstore = nc == kNCand ? 4 : 0;
      a.D2out = b->buf[XB_D2];
      brow(b, OP_ZSTEP, EPI_DIR, a, nc);
    }
    {
      RowArgs a = brow_base(b, P);
      a.B = b->buf[XB_B];
      a.gout = b->buf[XB_G];
      a.Xold = X; a.gold = b->buf[XB_G];
      a.Zold = b->buf[XB_Z]; a.gZold = b->buf[XB_GZ];
      a.Xout = X;
      a.ctl_mode = is_w ? CTL_UPD_W : (k == K - 1 ? CTL_UPD_H_LAST : CTL_UPD_H);
      a.Zin = b->buf[XB_Z]; a.Din = b->buf[XB_D]; a.Din2 = b->buf[XB_D2];
      brow(b, OP_UPD, EPI_GRAD, a);
    }
  }
}

void bpen_init(BatchCtx* b, const Params& P) {
  bany(b);
  bprod(b, b->buf[XB_W], b->buf[XB_B], nullptr, nullptr, b->ctl, b->run);
  bgram(b, b->buf[XB_W], b->buf[XB_W], 0, 1, b->ctl, b->run, b->G64fix, b->GT, 0, 1, nullptr);
  RowArgs a = brow_base(b, P);
  a.X = b->buf[XB_HT]; a.B = b->buf[XB_B]; a.gout = b->buf[XB_G];
  a.ctl_mode = CTL_START_INIT;
  brow(b, OP_LOAD, EPI_GRAD, a);
}

void bpen_iteration(BatchCtx* b, const Params& P) {
  bpen_block(b, XB_W, XB_HT, true, P);
  bpen_block(b, XB_HT, XB_W, false, P);
  bany(b);
}

void bpen_final(BatchCtx* b, const Params& P) {
  // every problem contributes: full work lists, no run flag, no active test.  <W, A Ht> of
  // the closed-form residual comes from an FP32 CUDA-core product (the tensor-core
  // accumulation bias would be amplified by the cancellation in the residual).
  b->use_full = true;
  b->accurate = true;
  bprod(b, b->buf[XB_HT], b->buf[XB_B], b->buf[XB_W], b->pax, nullptr, nullptr);
  bgram(b, b->buf[XB_W], b->buf[XB_W], 0, 3, nullptr, nullptr, b->G64p, b->GT, 1, 1, nullptr);
  bgram(b, b->buf[XB_HT], b->buf[XB_HT], 1, 3, nullptr, nullptr, b->G64p, b->GT, 1, 1, nullptr);
  bgram(b, b->buf[XB_W], b->buf[XB_HT], 2, 3, nullptr, nullptr, b->G64p, b->GT, 1, 1, nullptr);
  RowArgs a = brow_base(b, P);
  a.X = b->buf[XB_W]; a.B = b->buf[XB_B]; a.gout = b->buf[XB_G];
  a.run = nullptr;
  a.ctl = b->ctl + b->nprob;  // second Ctl array: all live
  a.ctl_mode = CTL_NONE;
  brow(b, OP_LOAD, EPI_GRAD, a);
  k_bfinal<<<b->nprob, 32, 0, b->s>>>(b->ctl, b->pax, b->prow, b->G64p, b->dp, 0);
  b->use_full = false;
  b->accurate = false;
}

snmf_status sync_user_b(BatchCtx* b, std::string* err) {
  if (!b->user) return SNMF_OK;
  BCK(cudaEventRecord(b->evsync, b->user));
  BCK(cudaStreamWaitEvent(b->s, b->evsync, 0));
  return SNMF_OK;
}

}  // namespace

int batch_nprob(const BatchCtx* b) { return b ? b->nprob : 0; }

void batch_set_budget(BatchCtx* b, long long cycles) {
  if (!b) return;
  b->budget = cycles;
  // the captured solve graphs hold the old budget in their kernel parameters
  for (auto& e : b->exec) {
    if (e) cudaGraphExecDestroy(e);
    e = nullptr;
  }
}

snmf_status batch_validate(const snmf_matrix* Am, const snmf_options& o, std::string* err) {
  const int np = Am->nprob;
  if (np < 1 || !Am->batch_desc || !Am->values) { *err = "dense batch: nprob >= 1, batch_desc and values required"; return SNMF_ERR_ARG; }
  if (o.formulation != SNMF_PENALTY) { *err = "dense batch: penalty form only"; return SNMF_ERR_ARG; }
  if (o.batch != 1) { *err = "dense batch: batch (restarts) must be 1"; return SNMF_ERR_ARG; }
  if (o.precision == SNMF_FP8) { *err = "dense batch: FP8 not available"; return SNMF_ERR_ARG; }
  if (o.step_controller == 2 || o.step_controller == 4) {
    *err = "dense batch: record and rollout modes need a single-problem handle";
    return SNMF_ERR_ARG;
  }
  if (o.precision == SNMF_F64 && Am->dtype != SNMF_F64) { *err = "dense batch: F64 precision needs F64 values"; return SNMF_ERR_ARG; }
  if (Am->dtype != SNMF_F64 && Am->dtype != SNMF_F32) { *err = "dense batch: values must be F64 or F32"; return SNMF_ERR_ARG; }
  if (Am->location != SNMF_ON_DEVICE && Am->location != SNMF_ON_HOST) { *err = "bad location"; return SNMF_ERR_ARG; }
  std::vector<int64_t> ns(np), rs(np), ao(np);
  for (int p = 0; p < np; ++p) {
    ns[p] = Am->batch_desc[3 * p];
    rs[p] = Am->batch_desc[3 * p + 1];
    ao[p] = Am->batch_desc[3 * p + 2];
    if (ns[p] < 1 || rs[p] < 1 || rs[p] > 64 || rs[p] > ns[p] || ao[p] < 0) {
      *err = "dense batch: problem " + std::to_string(p) + " needs n >= 1, 1 <= r <= min(n, 64), offset >= 0";
      return SNMF_ERR_ARG;
    }
  }
  return SNMF_OK;
}

snmf_status batch_create(BatchCtx** out, const snmf_matrix* Am, const snmf_options& o, cudaStream_t stream,
                         std::string* err) {
  *out = nullptr;
  const snmf_status vs = batch_validate(Am, o, err);
  if (vs != SNMF_OK) return vs;
  const int np = Am->nprob;
  std::vector<int64_t> ns(np), rs(np), ao(np);
  int64_t nmax = 0, aext = 0;
  for (int p = 0; p < np; ++p) {
    ns[p] = Am->batch_desc[3 * p];
    rs[p] = Am->batch_desc[3 * p + 1];
    ao[p] = Am->batch_desc[3 * p + 2];
    nmax = std::max(nmax, ns[p]);
    aext = std::max(aext, ao[p] + ns[p] * ns[p]);
  }
  BatchCtx* b = new BatchCtx();
  auto bail = [&](snmf_status st) { batch_destroy(b); return st; };
#define CKB(call)                                                                    \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      *err = std::string(#call) + ": " + cudaGetErrorString(e_);                     \
      return bail(e_ == cudaErrorMemoryAllocation ? SNMF_ERR_OOM : SNMF_ERR_CUDA);   \
    }                                                                                \
  } while (0)
  b->nprob = np;
  b->opt = o;
  b->prec = o.precision;
  b->tdtype = o.precision == SNMF_F64 ? 0 : 1;
  b->esz = b->tdtype == 0 ? 8 : 4;
  b->a_dtype = o.precision == SNMF_F64 ? 0 : (o.precision == SNMF_BF16 ? 2 : 1);
  b->user = stream;
  CKB(cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking));
  CKB(cudaStreamCreateWithFlags(&b->s2, cudaStreamNonBlocking));
  CKB(cudaEventCreateWithFlags(&b->evfork, cudaEventDisableTiming));
  CKB(cudaEventCreateWithFlags(&b->evjoin, cudaEventDisableTiming));
  CKB(cudaEventCreate(&b->ev0));
  CKB(cudaEventCreate(&b->ev1));
  CKB(cudaEventCreateWithFlags(&b->evsync, cudaEventDisableTiming));
  if (sync_user_b(b, err) != SNMF_OK) return bail(SNMF_ERR_CUDA);
  // ---- layout and work lists (items of the largest problems first) ----
  b->lda = (nmax + 63) / 64 * 64;
  b->hp.resize(np);
  int64_t arow = 0, xoff = 0, goff = 0, g3off = 0, gpoff = 0;
  const int bm = row_bm(b);
  for (int p = 0; p < np; ++p) {
    BProb& q = b->hp[p];
    q.n = ns[p];
    q.r = (int)rs[p];
    const int rows = rs[p] <= 32 ? (b->tdtype == 0 ? TileCfg<double>::TR : TileCfg<float>::TR) : bm;
    q.nrt = (int)((ns[p] + rows - 1) / rows);
    q.npt = (int)((ns[p] + kPBM - 1) / kPBM);
    q.gch = (int)((ns[p] + kGChunk - 1) / kGChunk);
    q.arow = arow;
    q.xoff = xoff;
    q.goff = goff;
    q.g3off = g3off;
    q.gpoff = gpoff;
    arow += ns[p];
    xoff += ns[p] * rs[p];
    goff += rs[p] * rs[p];
    g3off += 3 * rs[p] * rs[p];
    gpoff += (int64_t)q.gch * 3 * rs[p] * rs[p];
  }
  b->rows_total = arow;
  b->xtot = xoff;
  std::vector<int> order(np);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return ns[x] > ns[y]; });
  int nslot = 0;
  for (int p : order) {
    BProb& q = b->hp[p];
    q.slot0 = nslot;
    nslot += q.nrt;
    std::vector<int2>& lst = q.r <= 32 ? b->h_row : b->h_rowg;
    for (int t = 0; t < q.nrt; ++t) lst.push_back(make_int2(p, t));
    q.pslot0 = (int)b->h_prod.size();
    for (int t = 0; t < q.npt; ++t) b->h_prod.push_back(make_int2(p, t));
    for (int c = 0; c < q.gch; ++c) b->h_gram.push_back(make_int2(p, c));
  }
  // ---- A_all in the stored precision ----
  const int src_dt = Am->dtype == SNMF_F64 ? 0 : 1;
  const size_t ssz = src_dt == 0 ? 8 : 4;
  const size_t asz = b->a_dtype == 0 ? 8 : (b->a_dtype == 2 ? 2 : 4);
  CKB(cudaMalloc(&b->A, (size_t)b->rows_total * b->lda * asz));
  const void* src = Am->values;
  void* staging = nullptr;
  if (Am->location == SNMF_ON_HOST) {
    CKB(cudaMalloc(&staging, (size_t)aext * ssz));
    CKB(cudaMemcpyAsync(staging, src, (size_t)aext * ssz, cudaMemcpyHostToDevice, b->s));
    src = staging;
  }
  for (int p = 0; p < np; ++p) {
    const BProb& q = b->hp[p];
    const int64_t tot = q.n * b->lda;
    const int blocks = (int)std::min<int64_t>((tot + 255) / 256, 152 * 8);
    const char* sp = (const char*)src + (size_t)ao[p] * ssz;
    char* dp = (char*)b->A + (size_t)q.arow * b->lda * asz;
#define CONV(TS, TD) k_bconvert<TS, TD><<<blocks, 256, 0, b->s>>>((const TS*)sp, q.n, (TD*)dp, b->lda)
    if (src_dt == 0) {
      if (b->a_dtype == 0) CONV(double, double);
      else if (b->a_dtype == 1) CONV(double, float);
      else CONV(double, __nv_bfloat16);
    } else {
      if (b->a_dtype == 1) CONV(float, float);
      else CONV(float, __nv_bfloat16);
    }
#undef CONV
  }
  CKB(cudaGetLastError());
  // ---- device tables and workspaces ----
  CKB(cudaMalloc(&b->dp, np * sizeof(BProb)));
  b->nslot = nslot;
  CKB(cudaMalloc(&b->it_row, std::max<size_t>(b->h_row.size(), 1) * sizeof(int2)));
  CKB(cudaMalloc(&b->it_rowg, std::max<size_t>(b->h_rowg.size(), 1) * sizeof(int2)));
  if (!b->h_rowg.empty())
    CKB(cudaMemcpyAsync(b->it_rowg, b->h_rowg.data(), b->h_rowg.size() * sizeof(int2), cudaMemcpyHostToDevice, b->s));
  CKB(cudaMalloc(&b->it_prod, b->h_prod.size() * sizeof(int2)));
  CKB(cudaMalloc(&b->it_gram, b->h_gram.size() * sizeof(int2)));
  if (!b->h_row.empty())
    CKB(cudaMemcpyAsync(b->it_row, b->h_row.data(), b->h_row.size() * sizeof(int2), cudaMemcpyHostToDevice, b->s));
  CKB(cudaMemcpyAsync(b->it_prod, b->h_prod.data(), b->h_prod.size() * sizeof(int2), cudaMemcpyHostToDevice, b->s));
  CKB(cudaMemcpyAsync(b->it_gram, b->h_gram.data(), b->h_gram.size() * sizeof(int2), cudaMemcpyHostToDevice, b->s));
  CKB(cudaMemcpyAsync(b->dp, b->hp.data(), np * sizeof(BProb), cudaMemcpyHostToDevice, b->s));
  for (int x = 0; x < XB_N; ++x) {
    CKB(cudaMalloc(&b->buf[x], (size_t)b->xtot * b->esz));
    CKB(cudaMemsetAsync(b->buf[x], 0, (size_t)b->xtot * b->esz, b->s));
  }
  CKB(cudaMalloc(&b->prow, (size_t)b->nslot * kNQ * sizeof(double)));
  CKB(cudaMalloc(&b->pax, b->h_prod.size() * kNQ * sizeof(double)));  // >= tensor-core items
  CKB(cudaMalloc(&b->dev_err, sizeof(int)));
  CKB(cudaMemsetAsync(b->dev_err, 0, sizeof(int), b->s));
  if (o.timeout_cycles > 0) b->budget = o.timeout_cycles;
  CKB(cudaMalloc(&b->gpart, std::max<int64_t>(gpoff, 1) * sizeof(double)));
  CKB(cudaMalloc(&b->G64fix, g3off * sizeof(double)));
  CKB(cudaMalloc(&b->G64p, g3off * sizeof(double)));
  CKB(cudaMalloc(&b->GT, goff * b->esz));
  CKB(cudaMalloc(&b->ctl, 2 * np * sizeof(Ctl)));
  CKB(cudaMalloc(&b->run, sizeof(int)));
  CKB(cudaMalloc(&b->counters, 4 * np * sizeof(unsigned)));
  CKB(cudaMemsetAsync(b->counters, 0, 4 * np * sizeof(unsigned), b->s));
  CKB(cudaMalloc(&b->dsc, (2 * b->h_prod.size() + 2 * np) * sizeof(double)));
  CKB(cudaMallocHost(&b->h_flag, sizeof(int)));
  if (o.step_controller == 1 || o.step_controller == 3) {
    std::vector<__nv_bfloat16> wb(kMlpParams);
    for (int i = 0; i < kMlpParams; ++i) wb[i] = __float2bfloat16_rn(o.mlp_weights[i]);
    CKB(cudaMalloc(&b->mlp_w, kMlpParams * sizeof(__nv_bfloat16)));
    CKB(cudaMemcpyAsync(b->mlp_w, wb.data(), kMlpParams * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice, b->s));
    CKB(cudaStreamSynchronize(b->s));
  }
  if (o.step_controller == 2) {
    b->rec_cap = 1 << 20;
    CKB(cudaMalloc(&b->rec_feat, (size_t)b->rec_cap * kMlpIn * sizeof(float)));
    CKB(cudaMalloc(&b->rec_targ, (size_t)b->rec_cap * sizeof(float)));
    CKB(cudaMalloc(&b->rec_count, sizeof(int)));
    CKB(cudaMemsetAsync(b->rec_count, 0, sizeof(int), b->s));
  }
  // ---- ||A_p||^2 and sum(A_p) of the stored values; lambda_p ----
  {
    const unsigned g = (unsigned)b->h_prod.size();
    if (b->a_dtype == 0) k_bsums<double><<<g, 256, 0, b->s>>>((const double*)b->A, b->lda, b->dp, b->it_prod, b->dsc);
    else if (b->a_dtype == 1) k_bsums<float><<<g, 256, 0, b->s>>>((const float*)b->A, b->lda, b->dp, b->it_prod, b->dsc);
    else k_bsums<__nv_bfloat16><<<g, 256, 0, b->s>>>((const __nv_bfloat16*)b->A, b->lda, b->dp, b->it_prod, b->dsc);
    double* outp = b->dsc + 2 * b->h_prod.size();
    k_bsums_reduce<<<np, 32, 0, b->s>>>(b->dp, b->dsc, outp);
    std::vector<double> sums(2 * np);
    CKB(cudaMemcpyAsync(sums.data(), outp, 2 * np * sizeof(double), cudaMemcpyDeviceToHost, b->s));
    CKB(cudaStreamSynchronize(b->s));
    if (staging) cudaFree(staging);
    staging = nullptr;
    b->sumA.resize(np);
    for (int p = 0; p < np; ++p) {
      if (!std::isfinite(sums[2 * p])) { *err = "A_" + std::to_string(p) + " has NaN/Inf entries"; return bail(SNMF_ERR_NUMERIC); }
      b->hp[p].normA2 = sums[2 * p];
      b->hp[p].lam = o.lambda_sym >= 0.0 ? o.lambda_sym : 0.01 * std::sqrt(sums[2 * p]);
      b->sumA[p] = sums[2 * p + 1];
    }
    if (b->a_dtype == 2) {
      // tensor-core items (largest problems first) and the transposed BF16 operand parts:
      // problem p owns rows xrow_p .. xrow_p + r_p rounded up to 16 (zero beyond r_p / n_p)
      std::vector<int64_t> xr(np);
      int64_t xrow = 0;
      for (int p = 0; p < np; ++p) {
        xr[p] = xrow;
        xrow += (b->hp[p].r + 15) / 16 * 16;
      }
      b->xt_rows = xrow;
      for (int p : order) {
        BProb& q = b->hp[p];
        q.ntt = (int)((q.n + 127) / 128);
        q.tslot0 = (int)b->h_tc.size();
        for (int t = 0; t < q.ntt; ++t) {
          TcItem ti{};
          ti.arow = q.arow + 128 * t;
          ti.xoff = q.xoff;
          ti.m0 = 128 * t;
          ti.n = (int)q.n;
          ti.r = q.r;
          ti.bn = (q.r + 15) / 16 * 16;
          ti.xrow = (int)xr[p];
          ti.kt = (int)((q.n + 63) / 64);
          ti.prob = p;
          ti.slot = (int)b->h_tc.size();
          ti.lam = (float)q.lam;
          b->h_tc.push_back(ti);
        }
      }
      CKB(cudaMalloc(&b->it_tc, b->h_tc.size() * sizeof(TcItem)));
      CKB(cudaMemcpyAsync(b->it_tc, b->h_tc.data(), b->h_tc.size() * sizeof(TcItem), cudaMemcpyHostToDevice, b->s));
      const size_t xb = (size_t)b->xt_rows * b->lda * 2;
      CKB(cudaMalloc(&b->xh, xb));
      CKB(cudaMalloc(&b->xl, xb));
      CKB(cudaMemsetAsync(b->xh, 0, xb, b->s));
      CKB(cudaMemsetAsync(b->xl, 0, xb, b->s));
    }
    CKB(cudaMemcpyAsync(b->dp, b->hp.data(), np * sizeof(BProb), cudaMemcpyHostToDevice, b->s));
    CKB(cudaStreamSynchronize(b->s));
  }
  // per-problem item ranges of every list (each list holds the problems in `order`),
  // full counts, and the compacted copies (start as the full lists)
  {
    b->order = order;
    std::vector<int> pst(5 * np, 0), psz(5 * np, 0);
    auto fill = [&](int L, int i, int p) {
      if (psz[L * np + p] == 0) pst[L * np + p] = i;
      psz[L * np + p]++;
    };
    for (size_t i = 0; i < b->h_row.size(); ++i) fill(0, (int)i, b->h_row[i].x);
    for (size_t i = 0; i < b->h_rowg.size(); ++i) fill(1, (int)i, b->h_rowg[i].x);
    for (size_t i = 0; i < b->h_gram.size(); ++i) fill(2, (int)i, b->h_gram[i].x);
    for (size_t i = 0; i < b->h_prod.size(); ++i) fill(3, (int)i, b->h_prod[i].x);
    for (size_t i = 0; i < b->h_tc.size(); ++i) fill(4, (int)i, b->h_tc[i].prob);
    const int cf[5] = {(int)b->h_row.size(), (int)b->h_rowg.size(), (int)b->h_gram.size(), (int)b->h_prod.size(),
                       (int)b->h_tc.size()};
    CKB(cudaMalloc(&b->pst, 5 * np * sizeof(int)));
    CKB(cudaMalloc(&b->psz, 5 * np * sizeof(int)));
    CKB(cudaMalloc(&b->d_order, np * sizeof(int)));
    CKB(cudaMalloc(&b->cnt_full, 5 * sizeof(int)));
    CKB(cudaMalloc(&b->cnt_act, 5 * sizeof(int)));
    CKB(cudaMemcpyAsync(b->pst, pst.data(), 5 * np * sizeof(int), cudaMemcpyHostToDevice, b->s));
    CKB(cudaMemcpyAsync(b->psz, psz.data(), 5 * np * sizeof(int), cudaMemcpyHostToDevice, b->s));
    CKB(cudaMemcpyAsync(b->d_order, order.data(), np * sizeof(int), cudaMemcpyHostToDevice, b->s));
    CKB(cudaMemcpyAsync(b->cnt_full, cf, 5 * sizeof(int), cudaMemcpyHostToDevice, b->s));
    CKB(cudaMemcpyAsync(b->cnt_act, cf, 5 * sizeof(int), cudaMemcpyHostToDevice, b->s));
    int2** comp[4] = {&b->c_row, &b->c_rowg, &b->c_gram, &b->c_prod};
    const int2* full[4] = {b->it_row, b->it_rowg, b->it_gram, b->it_prod};
    for (int L = 0; L < 4; ++L) {
      CKB(cudaMalloc(comp[L], std::max(cf[L], 1) * sizeof(int2)));
      if (cf[L]) CKB(cudaMemcpyAsync(*comp[L], full[L], cf[L] * sizeof(int2), cudaMemcpyDeviceToDevice, b->s));
    }
    CKB(cudaMalloc(&b->c_tc, std::max(cf[4], 1) * sizeof(TcItem)));
    if (cf[4]) CKB(cudaMemcpyAsync(b->c_tc, b->it_tc, cf[4] * sizeof(TcItem), cudaMemcpyDeviceToDevice, b->s));
    CKB(cudaStreamSynchronize(b->s));
  }
#undef CKB
  *out = b;
  return SNMF_OK;
}

snmf_status batch_solve(BatchCtx* b, bool host, void* W, void* Ht, snmf_stats* out, std::string* err) {
  const size_t fbytes = (size_t)b->xtot * b->esz;
  const cudaMemcpyKind kin = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const cudaMemcpyKind kout = host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (sync_user_b(b, err) != SNMF_OK) return SNMF_ERR_CUDA;
  BCK(cudaEventRecord(b->ev0, b->s));
  int64_t launches = 0;
  if (W) {
    BCK(cudaMemcpyAsync(b->buf[XB_W], W, fbytes, kin, b->s));
  } else {
    for (int p = 0; p < b->nprob; ++p) {
      const BProb& q = b->hp[p];
      const double mean = b->sumA[p] / ((double)q.n * (double)q.n);
      const double upper = b->opt.init_scale * std::sqrt(std::max(mean, 0.0) / q.r);
      launch_philox_uniform(b->tdtype, (char*)b->buf[XB_W] + (size_t)q.xoff * b->esz, q.n, q.r, q.r,
                            b->opt.seed + (uint64_t)p, upper, b->s);
    }
    launches += b->nprob;
  }
  if (Ht) BCK(cudaMemcpyAsync(b->buf[XB_HT], Ht, fbytes, kin, b->s));
  else BCK(cudaMemcpyAsync(b->buf[XB_HT], b->buf[XB_W], fbytes, cudaMemcpyDeviceToDevice, b->s));
  const int np = b->nprob;
  b->h_ctl.assign(2 * np, Ctl{});
  for (int j = 0; j < 2 * np; ++j) {
    b->h_ctl[j].active = 1;
    b->h_ctl[j].lam = b->hp[j % np].lam;
    b->h_ctl[j].rho = 1.0;
    b->h_ctl[j].mlp_mult = 1.0;
  }
  BCK(cudaMemcpyAsync(b->ctl, b->h_ctl.data(), 2 * np * sizeof(Ctl), cudaMemcpyHostToDevice, b->s));
  static const int one = 1;
  BCK(cudaMemcpyAsync(b->run, &one, sizeof(int), cudaMemcpyHostToDevice, b->s));
  const Params P = bparams(b);
  if (!b->exec[0]) {
    for (int g = 0; g < 3; ++g) {
      cudaGraph_t gr;
      BCK(cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal));
      if (g == 0) bpen_init(b, P);
      else if (g == 1) bpen_iteration(b, P);
      else bpen_final(b, P);
      BCK(cudaStreamEndCapture(b->s, &gr));
      size_t nn = 0;
      BCK(cudaGraphGetNodes(gr, nullptr, &nn));
      b->nodes[g] = (int)nn;
      BCK(cudaGraphInstantiate(&b->exec[g], gr, 0));
      cudaGraphDestroy(gr);
    }
  }
  BCK(cudaGraphLaunch(b->exec[0], b->s));
  launches += b->nodes[0];
  int launched = 0, chunk = 1;
  const int maxit = b->opt.max_iter;
  while (launched < maxit) {
    const int m = std::min(chunk, maxit - launched);
    for (int t = 0; t < m; ++t) BCK(cudaGraphLaunch(b->exec[1], b->s));
    launched += m;
    BCK(cudaMemcpyAsync(b->h_flag, b->run, sizeof(int), cudaMemcpyDeviceToHost, b->s));
    BCK(cudaStreamSynchronize(b->s));
    if (*b->h_flag == 0) break;
    chunk = std::min(chunk * 2, 8);
  }
  launches += (int64_t)b->nodes[1] * launched;
  BCK(cudaGraphLaunch(b->exec[2], b->s));
  launches += b->nodes[2];
  if (W) BCK(cudaMemcpyAsync(W, b->buf[XB_W], fbytes, kout, b->s));
  if (Ht) BCK(cudaMemcpyAsync(Ht, b->buf[XB_HT], fbytes, kout, b->s));
  BCK(cudaEventRecord(b->ev1, b->s));
  BCK(cudaMemcpyAsync(b->h_ctl.data(), b->ctl, np * sizeof(Ctl), cudaMemcpyDeviceToHost, b->s));
  BCK(cudaStreamSynchronize(b->s));
  if (b->user) {
    BCK(cudaEventRecord(b->evsync, b->s));
    BCK(cudaStreamWaitEvent(b->user, b->evsync, 0));
  }
  if (b->tc_fail) {
    const int tf = b->tc_fail;
    b->tc_fail = 0;
    cudaGetLastError();
    *err = "tensor-core product not launched (status " + std::to_string(tf) + ")";
    return SNMF_ERR_CUDA;
  }
  BCK(cudaGetLastError());
  int derr = 0;
  BCK(cudaMemcpy(&derr, b->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (derr) {
    BCK(cudaMemset(b->dev_err, 0, sizeof(int)));
    *err = "a bounded device wait of the tensor-core product ran out (code " + std::to_string(derr) + ")";
    return SNMF_ERR_TIMEOUT;
  }
  float ms = 0.f;
  cudaEventElapsedTime(&ms, b->ev0, b->ev1);
  b->have_result = true;
  int conv = 1, lsf = 0, iters = 0, nan = 0, tried = 0, acc = 0;
  double fsum = 0.0, resmax = 0.0, pgmax = 0.0;
  for (int p = 0; p < np; ++p) {
    const Ctl& c = b->h_ctl[p];
    conv &= (c.pg0 == 0.0 || c.pg <= b->opt.tol * c.pg0) ? 1 : 0;
    lsf += c.ls_fail;
    iters = std::max(iters, c.iters);
    nan |= c.nan_seen;
    tried += c.mlp_tried;
    acc += c.mlp_accept;
    fsum += c.fin_f;
    resmax = std::max(resmax, c.fin_res);
    pgmax = std::max(pgmax, c.fin_pg);
  }
  if (out) {
    out->iters = iters;
    out->converged = conv;
    out->ls_fail = lsf;
    out->clipped_steps = 0;
    out->best_restart = 0;
    out->ax_products = 1 + 2 * launched + 1;  // grouped products (each covers every problem)
    out->kernel_launches = launches;
    out->graph_replays = launched;
    out->ctl_proposals = tried;
    out->ctl_accepted = acc;
    out->f = fsum;
    out->residual = resmax;
    out->pg_rel = pgmax;
    out->seconds = ms * 1e-3;
  }
  if (nan) { *err = "NaN/Inf in the scalar state"; return SNMF_ERR_NUMERIC; }
  return conv ? SNMF_OK : SNMF_NOT_CONVERGED;
}

snmf_status batch_problem_stats(BatchCtx* b, double* f, double* residual, double* pg_rel, int32_t* iters,
                                std::string* err) {
  if (!b->have_result) { *err = "no solve has run"; return SNMF_ERR_STATE; }
  for (int p = 0; p < b->nprob; ++p) {
    const Ctl& c = b->h_ctl[p];
    if (f) f[p] = c.fin_f;
    if (residual) residual[p] = c.fin_res;
    if (pg_rel) pg_rel[p] = c.fin_pg;
    if (iters) iters[p] = c.iters;
  }
  return SNMF_OK;
}

snmf_status batch_profile_ax(BatchCtx* b, int iters, double* ms, std::string* err) {
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  b->use_full = true;  // every problem
  bprod(b, b->buf[XB_W], b->buf[XB_Z], nullptr, nullptr, nullptr, nullptr);  // warm-up
  BCK(cudaEventRecord(e0, b->s));
  for (int t = 0; t < iters; ++t) bprod(b, b->buf[XB_W], b->buf[XB_Z], nullptr, nullptr, nullptr, nullptr);
  BCK(cudaEventRecord(e1, b->s));
  b->use_full = false;
  BCK(cudaStreamSynchronize(b->s));
  BCK(cudaGetLastError());
  float m = 0.f;
  cudaEventElapsedTime(&m, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = m / iters;
  return SNMF_OK;
}

snmf_status batch_get_factors(BatchCtx* b, void* W, void* Ht, std::string* err) {
  if (!b->have_result) { *err = "no solve has run"; return SNMF_ERR_STATE; }
  const size_t fbytes = (size_t)b->xtot * b->esz;
  if (W) BCK(cudaMemcpyAsync(W, b->buf[XB_W], fbytes, cudaMemcpyDeviceToDevice, b->s));
  if (Ht) BCK(cudaMemcpyAsync(Ht, b->buf[XB_HT], fbytes, cudaMemcpyDeviceToDevice, b->s));
  BCK(cudaStreamSynchronize(b->s));
  return SNMF_OK;
}

void batch_destroy(BatchCtx* b) {
  if (!b) return;
  if (b->s) cudaStreamSynchronize(b->s);
  if (b->s2) cudaStreamSynchronize(b->s2);
  for (auto& e : b->exec)
    if (e) cudaGraphExecDestroy(e);
  cudaFree(b->A);
  cudaFree(b->dp);
  cudaFree(b->it_row);
  cudaFree(b->it_prod);
  cudaFree(b->it_gram);
  cudaFree(b->it_rowg);
  for (void* q : {(void*)b->c_row, (void*)b->c_rowg, (void*)b->c_gram, (void*)b->c_prod, (void*)b->c_tc,
                  (void*)b->pst, (void*)b->psz, (void*)b->d_order, (void*)b->cnt_full, (void*)b->cnt_act})
    cudaFree(q);
  cudaFree(b->it_tc);
  cudaFree(b->xh);
  cudaFree(b->xl);
  cudaFree(b->dev_err);
  for (void* p : b->buf) cudaFree(p);
  double* d[] = {b->prow, b->pax, b->gpart, b->G64fix, b->G64p, b->dsc};
  for (double* p : d) cudaFree(p);
  cudaFree(b->GT);
  cudaFree(b->ctl);
  cudaFree(b->run);
  cudaFree(b->counters);
  cudaFree(b->mlp_w);
  cudaFree(b->rec_feat);
  cudaFree(b->rec_targ);
  cudaFree(b->rec_count);
  if (b->h_flag) cudaFreeHost(b->h_flag);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  if (b->evsync) cudaEventDestroy(b->evsync);
  if (b->evfork) cudaEventDestroy(b->evfork);
  if (b->evjoin) cudaEventDestroy(b->evjoin);
  if (b->s2) cudaStreamDestroy(b->s2);
  if (b->s) cudaStreamDestroy(b->s);
  delete b;
}

}  // namespace snmf
