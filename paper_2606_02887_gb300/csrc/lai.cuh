// LAI-SNMPBB operator (Sec. 2.3, Eq. (8)): A ~ U E U^T from a randomized eigen-sketch;
// A X is applied as U (E (U^T X)) with U^T X formed first.
#pragma once

#include <string>

#include "common.cuh"

namespace snmf {

struct LaiOp {
  void* U = nullptr;        // n x k, factor type, row-major (ld = k)
  double* lam = nullptr;    // k eigenvalues (device FP64)
  double* xpart = nullptr;  // split-K partials of U^T X [chunk][k][N] (FP64)
  void* M = nullptr;        // E U^T X, k x N (factor type)
  unsigned* counters = nullptr;  // arrival counters of the U^T X reduction
  int k = 0;
  int nchunks = 0;
  int maxN = 0;
  int64_t n = 0;
  double normA2 = 0.0;      // sum of kept eigenvalues squared
};

// Y = U (E (U^T X)) (+ c X2) with per-restart dots <P1, AX>, <P2, AX>; returns slots.
int lai_apply(const LaiOp& op, int tdtype, const Dims& d, const void* X, void* Y, double c,
              const void* X2, const void* P1, const void* P2, double* part, const int* run,
              cudaStream_t s);

// Build the sketch: l = k + p Gaussian columns (Philox seed), `power_iters` subspace
// iterations, CholeskyQR2 orthonormalisation, Jacobi eigensolver of Q^T A Q, keep the k
// eigenpairs of largest |eigenvalue|.  Returns 0, -2 (CUDA) or -3 (allocation).
int lai_build(LaiOp& op, const AxArgs& A, int tdtype, int64_t n, int k, int ell, int power_iters,
              uint64_t seed, int maxN, cudaStream_t s, std::string& msg);

void lai_free(LaiOp& op);

// W (n x r b, ld r b) = |U| |lambda|^1/2 of a sketch with k = r, in every restart's columns:
// the SVD start |U E^1/2| of Sec. 4.1 guideline (4) for symmetric A (H_0^T equals it).
void launch_svd_start(int tdtype, const LaiOp& op, int64_t n, int r, int b, void* W, cudaStream_t s);

// Out (n x m, ldo) = In (n x K, ldi) M (K x m row-major), K <= 128 (factor type).
void launch_rowmul(int tdtype, const void* In, int64_t ldi, int K, const void* M, int m, int64_t n, void* Out,
                   int64_t ldo, const int* run, cudaStream_t s);

}  // namespace snmf
