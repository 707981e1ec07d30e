// LAI-SNMPBB (Sec. 2.3, Eq. (8)): randomized eigen-sketch A ~ U E U^T and the product
// A X ~ U (E (U^T X)), U^T X formed first.
//
//   k_utx      M = E (U^T X) (k x N): CTA (row chunk, 64x64 output tile), partial per chunk
//              in the working type, last CTA of each tile sums the chunks in order and scales
//              row l by lambda_l.
//   k_rowmul   Out = In M (n x K times K x m), K <= 128: 32-row x 64-column tiles, K staged
//              in chunks of 32.  Serves U M, Y R^-1 (CholeskyQR) and Q P (Ritz vectors).
//   k_chol     Cholesky R^T R = G (+ shift) of an l x l FP64 Gram and R^-1, one block.
//   k_jacobi   parallel cyclic Jacobi eigensolver of a symmetric l x l FP64 matrix, one block,
//              round-robin pairing (l/2 disjoint rotations per round).
//   k_select   indices of the k eigenvalues of largest magnitude, eigenvector block P_k.
#include <math.h>

#include <algorithm>
#include <string>

#include "ax_tc.cuh"
#include "lai.cuh"
#include "rowops.cuh"

namespace snmf {

namespace {

inline int cdivi(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// NT: output columns per tile (32 for N <= 32, else 64); RS rows staged per round with the next
// round's loads in flight.
template <typename T, int NT, int RS>
__global__ void __launch_bounds__(256)
k_utx(const T* __restrict__ U, int k, const T* __restrict__ X, int64_t n, int N, int64_t ldx,
      int64_t chunk, T* __restrict__ part, const double* __restrict__ lam, T* __restrict__ M,
      unsigned* __restrict__ counters, const int* run) {
  constexpr int MC = NT / 16;        // micro tile columns
  constexpr int LU = RS * 64 / 256;  // staged U values per thread
  constexpr int LX = RS * NT / 256;  // staged X values per thread
  const int lt = blockIdx.y, ct = blockIdx.z;  // 64 x NT tile of the k x N output
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t i_begin = (int64_t)blockIdx.x * chunk, i_end = min(n, i_begin + chunk);
  __shared__ T Us[RS][64 + 1];
  __shared__ T Xs[RS][NT + 1];
  __shared__ unsigned ticket;
  T acc[4][MC];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < MC; ++c) acc[a][c] = T(0);
  const bool skip = run && *run == 0;
  const int l0 = lt * 64, c0 = ct * NT;
  if (!skip) {
    T uv[LU], xv[LX];
    auto fetch = [&](int64_t i0) {
#pragma unroll
      for (int m = 0; m < LU; ++m) {
        const int e = threadIdx.x + 256 * m, rr = e >> 6, cc = e & 63;
        const int64_t i = i0 + rr;
        uv[m] = (i < i_end && l0 + cc < k) ? U[i * k + l0 + cc] : T(0);
      }
#pragma unroll
      for (int m = 0; m < LX; ++m) {
        const int e = threadIdx.x + 256 * m, rr = e / NT, cc = e % NT;
        const int64_t i = i0 + rr;
        xv[m] = (i < i_end && c0 + cc < N) ? X[i * ldx + c0 + cc] : T(0);
      }
    };
    if (i_begin < i_end) fetch(i_begin);
    for (int64_t i0 = i_begin; i0 < i_end; i0 += RS) {
#pragma unroll
      for (int m = 0; m < LU; ++m) {
        const int e = threadIdx.x + 256 * m;
        Us[e >> 6][e & 63] = uv[m];
      }
#pragma unroll
      for (int m = 0; m < LX; ++m) {
        const int e = threadIdx.x + 256 * m;
        Xs[e / NT][e % NT] = xv[m];
      }
      __syncthreads();
      if (i0 + RS < i_end) fetch(i0 + RS);  // the next round's loads fly during this one
#pragma unroll 8
      for (int rr = 0; rr < RS; ++rr) {
        T ua[4], xb[MC];
#pragma unroll
        for (int a = 0; a < 4; ++a) ua[a] = Us[rr][ty + 16 * a];
#pragma unroll
        for (int c = 0; c < MC; ++c) xb[c] = Xs[rr][tx + 16 * c];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < MC; ++c) acc[a][c] = fma(ua[a], xb[c], acc[a][c]);
      }
      __syncthreads();
    }
  }
  const int64_t kn = (int64_t)k * N;
  T* out = part + (int64_t)blockIdx.x * kn;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int l = l0 + ty + 16 * a;
    if (l >= k) continue;
#pragma unroll
    for (int c = 0; c < MC; ++c) {
      const int col = c0 + tx + 16 * c;
      if (col < N) out[(int64_t)l * N + col] = acc[a][c];
    }
  }
  __threadfence();
  __syncthreads();
  const int tile_id = lt * gridDim.z + ct;
  if (threadIdx.x == 0) ticket = atomicAdd(&counters[tile_id], 1u);
  __syncthreads();
  if (ticket != gridDim.x - 1) return;
  // last CTA of the tile: each thread sums its NE entries over the chunks in chunk order,
  // several chunks' loads in flight
  constexpr int NE = 64 * NT / 256;
  constexpr int UF = NE >= 16 ? 2 : 4;
  int64_t off[NE];
  bool ok[NE];
  T sacc[NE];
#pragma unroll
  for (int u = 0; u < NE; ++u) {
    const int e = threadIdx.x + 256 * u;
    const int l = l0 + e / NT, col = c0 + e % NT;
    ok[u] = l < k && col < N;
    off[u] = ok[u] ? (int64_t)l * N + col : 0;
    sacc[u] = T(0);
  }
#pragma unroll UF
  for (int c = 0; c < (int)gridDim.x; ++c) {
    T v[NE];
#pragma unroll
    for (int u = 0; u < NE; ++u) v[u] = ok[u] ? __ldcg(part + (int64_t)c * kn + off[u]) : T(0);
#pragma unroll
    for (int u = 0; u < NE; ++u) sacc[u] += v[u];
  }
#pragma unroll
  for (int u = 0; u < NE; ++u)
    if (ok[u]) M[off[u]] = sacc[u] * (T)lam[l0 + (threadIdx.x + 256 * u) / NT];
  if (threadIdx.x == 0) counters[tile_id] = 0u;
}

// BR rows x NC columns per CTA (32 x 64, or 64 x 32 for m <= 32), K staged in chunks of 32.
template <typename T, int BR, int NC>
__global__ void __launch_bounds__(256)
k_rowmul(const T* __restrict__ In, int64_t ldi, int K, const T* __restrict__ Mm, int m, int64_t n,
         T* __restrict__ Out, int64_t ldo, const int* run) {
  constexpr int PR = BR / 16, QC = NC / 16;  // rows and columns per thread
  constexpr int LI = BR * 32 / 256, LM = 32 * NC / 256;
  if (run && *run == 0) return;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t row0 = (int64_t)blockIdx.x * BR;
  const int col0 = blockIdx.y * NC;
  __shared__ T Is[BR][33];
  __shared__ T Ms[32][NC + 1];
  T acc[PR][QC];
#pragma unroll
  for (int p = 0; p < PR; ++p)
#pragma unroll
    for (int q = 0; q < QC; ++q) acc[p][q] = T(0);
  for (int k0 = 0; k0 < K; k0 += 32) {
    T iv[LI], mv[LM];
#pragma unroll
    for (int u = 0; u < LI; ++u) {
      const int e = threadIdx.x + 256 * u, rr = e >> 5, kk = e & 31;
      const int64_t i = row0 + rr;
      iv[u] = (i < n && k0 + kk < K) ? In[i * ldi + k0 + kk] : T(0);
    }
#pragma unroll
    for (int u = 0; u < LM; ++u) {
      const int e = threadIdx.x + 256 * u, kk = e / NC, cc = e % NC;
      mv[u] = (k0 + kk < K && col0 + cc < m) ? Mm[(int64_t)(k0 + kk) * m + col0 + cc] : T(0);
    }
#pragma unroll
    for (int u = 0; u < LI; ++u) {
      const int e = threadIdx.x + 256 * u;
      Is[e >> 5][e & 31] = iv[u];
    }
#pragma unroll
    for (int u = 0; u < LM; ++u) {
      const int e = threadIdx.x + 256 * u;
      Ms[e / NC][e % NC] = mv[u];
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      T a[PR];
#pragma unroll
      for (int p = 0; p < PR; ++p) a[p] = Is[ty + 16 * p][kk];
#pragma unroll
      for (int q = 0; q < QC; ++q) {
        const T mq = Ms[kk][tx + 16 * q];
#pragma unroll
        for (int p = 0; p < PR; ++p) acc[p][q] = fma(a[p], mq, acc[p][q]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < PR; ++p) {
    const int64_t i = row0 + ty + 16 * p;
    if (i >= n) continue;
#pragma unroll
    for (int q = 0; q < QC; ++q) {
      const int c = col0 + tx + 16 * q;
      if (c < m) Out[i * ldo + c] = acc[p][q];
    }
  }
}

// Cholesky of G + shift I (l x l FP64, row-major, overwritten by R, upper) and Rinv (FP64,
// then copied to the working type).  *fail = 1 on a non-positive pivot.
template <typename T>
__global__ void k_chol(double* __restrict__ G, int l, double shift_rel, double* __restrict__ Rinv,
                       T* __restrict__ RinvT, int* __restrict__ fail) {
  __shared__ double piv;
  __shared__ double tr;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < l; ++i) t += G[i * l + i];
    tr = t;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < l; e += blockDim.x) G[e * l + e] += shift_rel * tr;
  __syncthreads();
  for (int j = 0; j < l; ++j) {
    if (threadIdx.x == 0) {
      const double d = G[j * l + j];
      piv = d > 0.0 ? sqrt(d) : -1.0;
      if (!(d > 0.0)) *fail = 1;
    }
    __syncthreads();
    if (piv <= 0.0) return;
    for (int c = j + threadIdx.x; c < l; c += blockDim.x) G[j * l + c] = (c == j) ? piv : G[j * l + c] / piv;
    __syncthreads();
    // trailing update G[a][c] -= R[j][a] R[j][c]  (a, c > j, upper triangle)
    const int m = l - j - 1;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int a = j + 1 + e / m, c = j + 1 + e % m;
      if (c >= a) G[a * l + c] -= G[j * l + a] * G[j * l + c];
    }
    __syncthreads();
  }
  // zero the strict lower triangle (R upper)
  for (int e = threadIdx.x; e < l * l; e += blockDim.x)
    if (e / l > e % l) G[e] = 0.0;
  __syncthreads();
  // Rinv: column c solves R x = e_c (back substitution), one thread per column
  for (int c = threadIdx.x; c < l; c += blockDim.x) {
    for (int i = l - 1; i >= 0; --i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int t = i + 1; t <= c; ++t) s -= G[i * l + t] * Rinv[t * l + c];
      Rinv[i * l + c] = (i <= c) ? s / G[i * l + i] : 0.0;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) RinvT[e] = (T)Rinv[e];
}

// Parallel cyclic Jacobi: A (l x l FP64, symmetric, overwritten) -> eigenvalues on the
// diagonal, V (l x l FP64) eigenvectors in columns.  Round-robin pairing over m = even(l)
// indices (index l is a dummy when l is odd).  Stops when the off-diagonal norm is below
// tol times the Frobenius norm, or after max_sweeps.
__global__ void k_jacobi(double* __restrict__ A, double* __restrict__ V, int l, int max_sweeps, double tol) {
  extern __shared__ double cs[];  // [m/2] c, [m/2] s, [m/2] p, [m/2] q (as doubles)
  __shared__ double red[32];
  const int m = (l + 1) / 2 * 2, h = m / 2;
  double* C = cs;
  double* Sn = cs + h;
  int* Pp = reinterpret_cast<int*>(cs + 2 * h);
  int* Qq = Pp + h;
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) V[e] = (e / l == e % l) ? 1.0 : 0.0;
  __syncthreads();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
      const double v = A[e];
      tot += v * v;
      if (e / l != e % l) off += v * v;
    }
    off = block_sum(off, red);
    tot = block_sum(tot, red);
    if (off <= tol * tol * tot) break;
    for (int round = 0; round < m - 1; ++round) {
      for (int i = threadIdx.x; i < h; i += blockDim.x) {
        auto player = [&](int j) { return j == 0 ? 0 : ((j - 1 + round) % (m - 1)) + 1; };
        int p = player(i), q = player(m - 1 - i);
        if (p > q) { const int t = p; p = q; q = t; }
        double c = 1.0, s = 0.0;
        if (q < l) {
          const double apq = A[p * l + q];
          if (apq != 0.0) {
            const double tau = (A[q * l + q] - A[p * l + p]) / (2.0 * apq);
            const double t = (tau >= 0.0) ? 1.0 / (tau + sqrt(1.0 + tau * tau)) : -1.0 / (-tau + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        }
        C[i] = c; Sn[i] = s; Pp[i] = p; Qq[i] = q;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int e = threadIdx.x; e < h * l; e += blockDim.x) {
        const int i = e / l, row = e % l;
        const int p = Pp[i], q = Qq[i];
        if (q >= l) continue;
        const double c = C[i], s = Sn[i];
        const double ap = A[row * l + p], aq = A[row * l + q];
        A[row * l + p] = c * ap - s * aq;
        A[row * l + q] = s * ap + c * aq;
        const double vp = V[row * l + p], vq = V[row * l + q];
        V[row * l + p] = c * vp - s * vq;
        V[row * l + q] = s * vp + c * vq;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int e = threadIdx.x; e < h * l; e += blockDim.x) {
        const int i = e / l, col = e % l;
        const int p = Pp[i], q = Qq[i];
        if (q >= l) continue;
        const double c = C[i], s = Sn[i];
        const double ap = A[p * l + col], aq = A[q * l + col];
        A[p * l + col] = c * ap - s * aq;
        A[q * l + col] = s * ap + c * aq;
      }
      __syncthreads();
    }
  }
}

// pick the k eigenvalues of largest |value| (ties: lower index first), write lam[k] and the
// l x k eigenvector block P (working type, row-major)
template <typename T>
__global__ void k_select(const double* __restrict__ A, const double* __restrict__ V, int l, int k,
                         double* __restrict__ lam, T* __restrict__ P, double* __restrict__ sumsq) {
  __shared__ int idx[128];
  if (threadIdx.x == 0) {
    bool used[128];
    for (int i = 0; i < l; ++i) used[i] = false;
    double s2 = 0.0;
    for (int t = 0; t < k; ++t) {
      int best = -1;
      double bv = -1.0;
      for (int i = 0; i < l; ++i)
        if (!used[i] && fabs(A[i * l + i]) > bv) { bv = fabs(A[i * l + i]); best = i; }
      used[best] = true;
      idx[t] = best;
      lam[t] = A[best * l + best];
      s2 += lam[t] * lam[t];
    }
    *sumsq = s2;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < l * k; e += blockDim.x) {
    const int row = e / k, t = e % k;
    P[e] = (T)V[row * l + idx[t]];
  }
}

template <typename T>
__global__ void k_sym(double* __restrict__ A, int l) {
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int p = e / l, q = e % l;
    if (p < q) {
      const double v = 0.5 * (A[p * l + q] + A[q * l + p]);
      A[p * l + q] = v;
      A[q * l + p] = v;
    }
  }
}

int ck(cudaError_t e, std::string& msg, const char* what) {
  if (e == cudaSuccess) return 0;
  msg = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? -3 : -2;
}

}  // namespace

void launch_rowmul(int tdtype, const void* In, int64_t ldi, int K, const void* M, int m, int64_t n, void* Out,
                   int64_t ldo, const int* run, cudaStream_t s) {
#define RM_ARGS(T) (const T*)In, ldi, K, (const T*)M, m, n, (T*)Out, ldo, run
  if (m <= 32) {  // narrow output: 64 rows x 32 columns per CTA, no masked half
    dim3 grid(cdivi(n, 64), 1);
    if (tdtype == 0) k_rowmul<double, 64, 32><<<grid, 256, 0, s>>>(RM_ARGS(double));
    else k_rowmul<float, 64, 32><<<grid, 256, 0, s>>>(RM_ARGS(float));
  } else {
    dim3 grid(cdivi(n, 32), cdivi(m, 64));
    if (tdtype == 0) k_rowmul<double, 32, 64><<<grid, 256, 0, s>>>(RM_ARGS(double));
    else k_rowmul<float, 32, 64><<<grid, 256, 0, s>>>(RM_ARGS(float));
  }
#undef RM_ARGS
}

int lai_apply(const LaiOp& op, int tdtype, const Dims& d, const void* X, void* Y, double c, const void* X2,
              const void* P1, const void* P2, double* part, const int* run, cudaStream_t s) {
  const int N = d.N;
  const int64_t chunk = (d.n + op.nchunks - 1) / op.nchunks;
  const bool narrow = N <= 32;
  dim3 g1(op.nchunks, cdivi(op.k, 64), narrow ? 1 : cdivi(N, 64));
#define UTX_ARGS(T) (const T*)op.U, op.k, (const T*)X, d.n, N, d.ld, chunk, (T*)op.xpart, op.lam, (T*)op.M, \
                    op.counters, run
  if (tdtype == 0) {
    if (narrow) k_utx<double, 32, 32><<<g1, 256, 0, s>>>(UTX_ARGS(double));
    else k_utx<double, 64, 32><<<g1, 256, 0, s>>>(UTX_ARGS(double));
  } else {
    if (narrow) k_utx<float, 32, 64><<<g1, 256, 0, s>>>(UTX_ARGS(float));
    else k_utx<float, 64, 32><<<g1, 256, 0, s>>>(UTX_ARGS(float));
  }
#undef UTX_ARGS
  launch_rowmul(tdtype, op.U, op.k, op.k, op.M, N, d.n, Y, d.ld, run, s);
  return launch_ax_finish_impl(tdtype, d, Y, nullptr, 1, c, X2, P1, P2, part, 0, run, s);
}

// product of the input operator with an n x cols block (ld = cols), for the sketch
static int sketch_product(const AxArgs& A, int td, int64_t n, int cols, const void* X, void* Y, void* ws,
                          size_t ws_elems, void* xh, void* xl, int* err, cudaStream_t s) {
  Dims d;
  d.n = n; d.r = cols; d.b = 1; d.N = cols; d.ld = cols;
  int splits;
  if (A.kind == AX_DENSE && A.a_dtype == 2) {
    splits = launch_ax_tc(A.A, n, (const float*)X, cols, cols, xh, xl, (float*)Y, (float*)ws, ws_elems, err,
                          2000000000LL, s, nullptr, 2, A.sym);
    if (splits < 1) return -1;
  } else {
    splits = launch_ax(A, td, n, cols, cols, X, Y, ws, ws_elems, nullptr, s);
  }
  double* dummy = nullptr;
  (void)dummy;
  return splits;
}

int lai_build(LaiOp& op, const AxArgs& A, int td, int64_t n, int k, int ell, int power_iters, uint64_t seed,
              int maxN, cudaStream_t s, std::string& msg) {
  lai_free(op);
  const size_t esz = td == 0 ? 8 : 4;
  const size_t blk = (size_t)n * ell;
  void *Y = nullptr, *Q = nullptr, *ws = nullptr, *xh = nullptr, *xl = nullptr, *RinvT = nullptr, *Pk = nullptr;
  double *G = nullptr, *Rinv = nullptr, *V = nullptr, *gpart = nullptr, *part = nullptr, *sums = nullptr;
  unsigned* counters = nullptr;
  int *fail = nullptr, *err = nullptr;
  int rc = 0;
  auto cleanup = [&]() {
    cudaFree(Y); cudaFree(Q); cudaFree(ws); cudaFree(xh); cudaFree(xl); cudaFree(RinvT); cudaFree(Pk);
    cudaFree(G); cudaFree(Rinv); cudaFree(V); cudaFree(gpart); cudaFree(part); cudaFree(sums);
    cudaFree(counters); cudaFree(fail); cudaFree(err);
  };
#define LCK(call)                                   \
  do {                                              \
    rc = ck((call), msg, #call);                    \
    if (rc) { cleanup(); return rc; }               \
  } while (0)
  const size_t ws_elems = (A.kind == AX_DENSE) ? 4 * blk : 0;
  LCK(cudaMalloc(&Y, blk * esz));
  LCK(cudaMalloc(&Q, blk * esz));
  if (ws_elems) LCK(cudaMalloc(&ws, ws_elems * esz));
  if (A.kind == AX_DENSE && A.a_dtype == 2) {
    LCK(cudaMalloc(&xh, (size_t)ell * tc_ld(n) * 2));
    LCK(cudaMalloc(&xl, (size_t)ell * tc_ld(n) * 2));
  }
  const int nch = (int)std::max<int64_t>(1, std::min<int64_t>(152 / ((ell + 63) / 64 * ((ell + 63) / 64)), n / 512));
  LCK(cudaMalloc(&G, (size_t)ell * ell * sizeof(double)));
  LCK(cudaMalloc(&Rinv, (size_t)ell * ell * sizeof(double)));
  LCK(cudaMalloc(&V, (size_t)ell * ell * sizeof(double)));
  LCK(cudaMalloc(&RinvT, (size_t)ell * ell * esz));
  LCK(cudaMalloc(&Pk, (size_t)ell * k * esz));
  LCK(cudaMalloc(&gpart, (size_t)nch * ell * ell * sizeof(double)));
  LCK(cudaMalloc(&part, (size_t)1024 * sizeof(double)));
  LCK(cudaMalloc(&sums, 4 * sizeof(double)));
  LCK(cudaMalloc(&counters, 64 * sizeof(unsigned)));
  LCK(cudaMemsetAsync(counters, 0, 64 * sizeof(unsigned), s));
  LCK(cudaMalloc(&fail, sizeof(int)));
  LCK(cudaMemsetAsync(fail, 0, sizeof(int), s));
  LCK(cudaMalloc(&err, sizeof(int)));
  LCK(cudaMemsetAsync(err, 0, sizeof(int), s));
  Dims dl;
  dl.n = n; dl.r = ell; dl.b = 1; dl.N = ell; dl.ld = ell;

  // Omega (Gaussian, Philox) -> Q; Y = A Omega
  launch_philox_gaussian(td, Q, n, ell, seed, s);
  auto product = [&](const void* X, void* Out) -> int {
    const int sp = sketch_product(A, td, n, ell, X, Out, ws, ws_elems, xh, xl, err, s);
    if (sp < 0) { msg = "sketch product failed"; return -2; }
    if (sp > 1) launch_ax_finish_impl(td, dl, Out, ws, sp, 0.0, nullptr, nullptr, nullptr, part, 0, nullptr, s);
    return 0;
  };
  // Q <- orth(Y) by CholeskyQR2 (first pass with a tiny diagonal shift)
  auto cholqr = [&](void* Yb, void* Qb) -> int {
    for (int pass = 0; pass < 2; ++pass) {
      const void* src = pass == 0 ? Yb : Qb;
      launch_gram(td, src, src, dl, 0, 1, gpart, nch, nullptr, nullptr, G, nullptr, -1, 0.0, counters, s);
      if (td == 0)
        k_chol<double><<<1, 256, 0, s>>>(G, ell, pass == 0 ? 1e-14 : 0.0, Rinv, (double*)RinvT, fail);
      else
        k_chol<float><<<1, 256, 0, s>>>(G, ell, pass == 0 ? 1e-7 : 0.0, Rinv, (float*)RinvT, fail);
      // Qb = src Rinv (via Yb when reading Qb: multiply into Yb then swap contents)
      void* dst = pass == 0 ? Qb : Yb;
      launch_rowmul(td, src, ell, ell, RinvT, ell, n, dst, ell, nullptr, s);
      if (pass == 1) {
        if (cudaMemcpyAsync(Qb, Yb, blk * esz, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return -2;
      }
    }
    return 0;
  };
  if ((rc = product(Q, Y))) { cleanup(); return rc; }
  if ((rc = cholqr(Y, Q))) { cleanup(); return rc; }
  for (int it = 0; it < power_iters; ++it) {
    if ((rc = product(Q, Y))) { cleanup(); return rc; }
    if ((rc = cholqr(Y, Q))) { cleanup(); return rc; }
  }
  // T = Q^T (A Q), symmetrised; eigendecomposition; U = Q P_k
  if ((rc = product(Q, Y))) { cleanup(); return rc; }
  launch_gram(td, Q, Y, dl, 0, 1, gpart, nch, nullptr, nullptr, G, nullptr, -1, 0.0, counters, s);
  k_sym<double><<<1, 256, 0, s>>>(G, ell);
  const int h = (ell + 1) / 2;
  k_jacobi<<<1, 256, 4 * h * sizeof(double), s>>>(G, V, ell, 40, 1e-13);
  LCK(cudaMalloc(&op.lam, (size_t)k * sizeof(double)));
  LCK(cudaMalloc(&op.U, (size_t)n * k * esz));
  if (td == 0) k_select<double><<<1, 256, 0, s>>>(G, V, ell, k, op.lam, (double*)Pk, sums);
  else k_select<float><<<1, 256, 0, s>>>(G, V, ell, k, op.lam, (float*)Pk, sums);
  launch_rowmul(td, Q, ell, ell, Pk, k, n, op.U, k, nullptr, s);
  double host_sums = 0.0;
  int host_fail = 0, host_err = 0;
  LCK(cudaMemcpyAsync(&host_sums, sums, sizeof(double), cudaMemcpyDeviceToHost, s));
  LCK(cudaMemcpyAsync(&host_fail, fail, sizeof(int), cudaMemcpyDeviceToHost, s));
  LCK(cudaMemcpyAsync(&host_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  LCK(cudaStreamSynchronize(s));
  LCK(cudaGetLastError());
  if (host_fail || host_err) {
    msg = host_fail ? "CholeskyQR: non-positive pivot (sketch rank deficient)" : "sketch product wait timed out";
    cleanup();
    lai_free(op);
    return -2;
  }
  op.k = k;
  op.n = n;
  op.normA2 = host_sums;
  op.maxN = maxN;
  op.nchunks = (int)std::max<int64_t>(1, std::min<int64_t>(152 / ((maxN + 63) / 64), n / 1024));
  LCK(cudaMalloc(&op.xpart, (size_t)op.nchunks * k * maxN * esz));
  LCK(cudaMalloc(&op.M, (size_t)k * maxN * esz));
  LCK(cudaMalloc(&op.counters, 4096 * sizeof(unsigned)));
  LCK(cudaMemsetAsync(op.counters, 0, 4096 * sizeof(unsigned), s));
  LCK(cudaStreamSynchronize(s));
  cleanup();
  return 0;
#undef LCK
}

// SVD start of Sec. 4.1 guideline (4) from the eigen-sketch of a symmetric A (k = r): the
// singular values of A are |lambda| with left vectors U and right vectors U sign(lambda), so
// |U E^1/2| and |E^1/2 P^T|^T are both |U| |lambda|^1/2 (column-wise).  Written to every one of
// the b restart column blocks of W (n x r b, ld r b).
namespace {
template <typename T>
__global__ void k_svd_start(const T* __restrict__ U, const double* __restrict__ lam, int64_t n, int r, int b,
                            T* __restrict__ W) {
  const int64_t total = n * (int64_t)r;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / r;
    const int c = (int)(e % r);
    const T v = (T)(fabs((double)U[e]) * sqrt(fabs(lam[c])));
    for (int j = 0; j < b; ++j) W[i * (int64_t)r * b + (int64_t)j * r + c] = v;
  }
}
}  // namespace

void launch_svd_start(int tdtype, const LaiOp& op, int64_t n, int r, int b, void* W, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>((n * r + 255) / 256, 152 * 8);
  if (tdtype == 0) k_svd_start<double><<<blocks, 256, 0, s>>>((const double*)op.U, op.lam, n, r, b, (double*)W);
  else k_svd_start<float><<<blocks, 256, 0, s>>>((const float*)op.U, op.lam, n, r, b, (float*)W);
}

void lai_free(LaiOp& op) {
  cudaFree(op.U); cudaFree(op.lam); cudaFree(op.xpart); cudaFree(op.M); cudaFree(op.counters);
  op = LaiOp{};
}

}  // namespace snmf
