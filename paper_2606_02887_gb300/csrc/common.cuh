// Shared definitions of the SNMPBB CUDA path (sm_103a).
//
// Data layout in HBM (all row-major):
//   factors X (W, Ht, Z, D, gradients, products): n x N with N = r * b; restart j owns
//   columns [j r, (j+1) r).  Element type T = double (FP64 precision) or float.
//   partial sums: part[slot][restart][NQ] (double), one slot per CTA of a row kernel,
//   reduced in a fixed order by the control kernels (deterministic, no atomics).
//   Gram partials: gpart[chunk][pair][restart][r*r] (double), reduced in fixed order.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tune.cuh"

namespace snmf {

constexpr int kNQ = 32;         // dot slots per partial record
constexpr int kNCand = 9;       // candidate steps evaluated in the controller's record mode
constexpr int kMlpIn = 5, kMlpHidden = 64;
constexpr int kMlpParams = kMlpIn * kMlpHidden + 2 * kMlpHidden + 1;
constexpr int kMaxHist = 64;    // max nonmonotone memory M
constexpr int kRowTile = 64;    // rows per CTA of the row kernels
constexpr int kMaxR = 256;      // max rank per restart

// Per-restart scalar state of Algorithm 1 (FP64, device resident).
struct Ctl {
  double rho;        // rho_0 of the block (penalty) / rho_k (direct), as used in the Z step
  double alpha;      // BB step for the D direction of the current step
  double beta;       // accepted line-search step (0 after a failed search)
  double phibeta;    // phi * beta used by the relaxed update
  double f;          // f(X_k) minus the block constant (penalty) / f(X_k) (direct)
  double F;          // nonmonotone reference F_k
  double fZ;         // f(Z_k)
  double gd;         // <grad f(Z_k), D_k>
  double q;          // curvature term of the line-search polynomial
  double ss, sy, yy; // <S,S>, <S,Y>, <Y,Y> of the last update
  double pg0;        // joint projected-gradient norm at the start
  double pgH2;       // squared projected gradient of the last H block (penalty)
  double pg;         // last joint projected-gradient norm
  double lam;        // penalty weight lambda
  double xax;        // <X, A X> of the current W (direct)
  double xax_z, zad, dad;   // <Z,AZ>, <Z,AD>, <D,AD> (direct)
  double zlz, dlz, dld;     // <Z,LZ>, <D,LZ>, <D,LD> (direct, graph)
  double fhist[kMaxHist];
  int hlen, hpos;
  int k;             // step index within the block (penalty) or since start (direct)
  int active;        // 1 while iterating
  int iters;         // outer iterations (penalty) / steps (direct)
  int ls_fail;
  int clipped;       // direct: steps with clipped entries
  int clip_now;      // direct: current update clipped
  int nan_seen;
  double fin_f, fin_res, fin_pg;   // final per-restart results
  double gnorm_prev; // ||g_{k-1}|| for the step controller features
  double f_prev, f_prev2;
  double mlp_mult;   // multiplier proposed by the learned controller (1 = plain BB)
  int mlp_tried;     // proposals made by the learned controller
  int commit;       // direct: the update of this step is to be committed
  double cand_alpha[kNCand];  // candidate BB-type steps of the current step (controller modes)
  int dsel;          // direction used by the update: 0 = D, 1 = D2 (plain BB fallback)
  int mlp_accept;    // proposals accepted at beta = 1
  int feat_ok;       // features of the current state are defined (k >= 1 in a block)
  float feat[kMlpIn];
  double pg_prev;    // projected-gradient norm of the previous iterate (features)
  double last_dec;   // previous objective decrease (features)
};

struct Dims {
  int64_t n;    // rows
  int r;        // rank per restart
  int b;        // restarts
  int N;        // r * b
  int64_t ld;   // leading dimension of factor buffers (= N)
};

// Launch-time scalars shared by the orchestration kernels.
struct Params {
  int formulation;   // 0 penalty, 1 direct
  int memory;        // nonmonotone M (0 = eta rule)
  int bb;            // 0 BB1, 1 BB2
  int max_ls;
  int max_iter;
  int power_iters;
  int controller;    // step controller: 0 plain BB, 1/3 learned, 2 record, 4 rollout branch
  double theta, phi, eta, alpha_min, alpha_max, beta_shrink, tol;
  double rho_factor; // direct form rho scaling
  double normA2;     // ||A||_F^2 of the stored operator
  double gamma;      // graph weight (0 = none)
  const __nv_bfloat16* mlp_w;  // learned controller weights: W1[64][5], b1[64], W2[64], b2
  float* rec_feat;   // record mode: features [cap][5]
  float* rec_targ;   // record mode: target log2 multipliers [cap]
  int* rec_count;
  int rec_cap;
  int64_t nr;        // entries per restart (n * r), for the active-set feature
  double* ring;      // per-iteration statistics: ring[j][slot][kRingVals] (NULL: off)
  int ring_cap;      // slots per restart
  int inner;         // inner steps per block (penalty form)
  int branch_step;   // controller 4: inner step, counted over the solve, that takes the 9 multipliers
};

// Values of one statistics record (penalty and naive forms: written at the start of every W block,
// i.e. once per outer iteration, for the state after the previous iteration).
constexpr int kRingVals = 8;  // iteration, pg / pg0, pg, alpha, beta, ls_fail, ctl proposals accepted, active

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Fixed-order block sum in the working type T (result in every thread); `sh` holds >= 32 T.
template <typename T>
__device__ __forceinline__ T block_sum_t(T v, T* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  T t = T(0);
  for (int w = 0; w < nw; ++w) t += sh[w];
  __syncthreads();
  return t;
}

// Fixed-order block sum over blockDim.x threads (multiple of 32, <= 1024).
// Result valid in every thread.  `sh` holds >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  double out = sh[0];
  __syncthreads();
  return out;
}

// ---------------------------------------------------------------------------
// host launchers (defined in the .cu files)
// ---------------------------------------------------------------------------

// Product kinds of the A*X operator
enum AxKind { AX_DENSE = 0, AX_CSR = 1 };

// Symmetric-half storage of a dense BF16 A (Sec. 1.2: A is symmetric): only the 128 x 128
// tiles (a, b) with a <= b of the tile grid (nt = ceil(n / 128) tiles a side) are stored, each
// tile row-major with a pitch of 128 elements and zero beyond n, tile (a, b) at element offset
// sym_tile(a, b, nt) * 128 * 128 (the upper tile rows one after another).  A_ij for a tile
// below the diagonal is the transpose of the stored tile (b, a).
__host__ __device__ inline int64_t sym_tile(int64_t a, int64_t b, int64_t nt) {
  return a * (2 * nt - a + 1) / 2 + (b - a);
}
__host__ __device__ inline int64_t sym_tiles(int64_t n) {
  const int64_t nt = (n + 127) / 128;
  return nt * (nt + 1) / 2;
}

struct AxArgs {
  // dense
  const void* A; int64_t lda; int a_dtype;  // a_dtype: 0 f64, 1 f32, 2 bf16, 3 fp8(e4m3) + scales
  const float* a_scale;                     // fp8: per 128x128 tile scale (power of two)
  // csr
  const int32_t* rowptr; const int32_t* colidx; const void* vals; int v_dtype;
  int kind;
  int accurate;  // BF16 dense: FP32 CUDA-core accumulation instead of the tensor-core product
  int sym;       // BF16 dense: A holds the upper tiles of the symmetric matrix (sym_tile)
};

// Y = A X (raw product, T = double/float), n x cols, ld = leading dimension of X and Y.
// Dense products may split K: the splits write ws[s] (n x ld each) and the finish pass
// sums them.  Returns the number of splits used (1 = result already in Y).
int launch_ax(const AxArgs& a, int tdtype, int64_t n, int cols, int64_t ld,
              const void* X, void* Y, void* ws, size_t ws_elems, const int* run_flag,
              cudaStream_t s, const ProdTune* tune = nullptr);

// Structure check of a device CSR matrix: *bad |= 1 for a bad rowptr (rowptr[0] != 0,
// rowptr[n] != nnz or decreasing), |= 2 for a column index outside [0, n).  *bad must be
// zeroed by the caller.
void launch_csr_check(const int32_t* rowptr, const int32_t* colidx, int64_t n, int64_t nnz, int* bad,
                      cudaStream_t s);

// Epilogue of a product over the restarts of d: Y = sum_s ws[s] (splits > 1),
// per-restart partials <P1, A X> -> part[slot][j][q0], <P2, A X> -> [q0+1], then
// Y += c * X2 (when X2 != NULL); dots_after = 1 takes the partials of the final Y instead.
// Returns the number of partial slots written.
int launch_ax_finish_impl(int tdtype, const Dims& d, void* Y, const void* ws, int splits,
                          double c, const void* X2, const void* P1, const void* P2,
                          double* part, int q0, const int* run_flag, cudaStream_t s, int dots_after = 0);

// label_i = argmax_c F[i, col0 + c], c < r (ties: lowest c) (knn.cu)
void launch_assign(int tdtype, const void* F, int64_t n, int64_t ld, int64_t col0, int r, int32_t* lab, cudaStream_t s);

// The paper's normalized Laplacian L = I - D^-1/2 A D^-1/2 (Sec. 2.2) of a dense (FP64/FP32)
// or CSR A: s[i] = d_i^-1/2 (0 where d_i <= 0, d_i the FP64 row sum) and out = the entries of
// -D^-1/2 A D^-1/2 in the factor type (dense: n x n with leading dimension n; CSR: the values
// on A's pattern), so that L X = X + out X.
void launch_normalized_adjacency(const AxArgs& a, int tdtype, int64_t n, double* s, void* out, cudaStream_t st);

}  // namespace snmf
