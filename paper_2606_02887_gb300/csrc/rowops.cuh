// Launchers of the O(n r^2) kernels and the control kernels (defined in rowops.cu).
#pragma once

#include "common.cuh"

namespace snmf {

// control step fused into the last CTA of a restart (RowArgs::ctl_mode)
enum { CTL_NONE = 0, CTL_START_W, CTL_START_H, CTL_START_INIT, CTL_LS, CTL_UPD_W, CTL_UPD_H, CTL_UPD_H_LAST,
       CTL_UPD_W_LAST_NAIVE };

// operand of the row GEMM X G: loaded, Z = Proj[X - g/rho], or X' = Proj[Z + phi beta D]
enum { OP_LOAD = 0, OP_ZSTEP = 1, OP_UPD = 2 };
// epilogue: gradient (+ S/Y and increment dots) or the D direction (+ dots)
enum { EPI_GRAD = 0, EPI_DIR = 1 };

// Arguments of k_rowgemm.  Gradient g = op(X) G - B (+ gamma LX), G = per-restart r x r
// matrix in the factor type.  Partial layout (part[slot][j][q], slot = CTA):
//   EPI_GRAD: q0 ||P grad||^2, q1 1/2 <g - B, X>, q2 <S,S>, q3 <S,Y>, q4 <Y,Y>,
//             q5 1/2 <X - Zold, g + gZold>
//   EPI_DIR : q0 <g, D>, q1 <D, D>, q2 1/2 <Z - Wcur, g + gWcur>, q3 <D, LX>, q4 <D G, D>;
//             candidates m >= 1 (controller modes): q(5+3(m-1)) <g, D_m>, +1 <D_m, D_m>, +2 <D_m G, D_m>
//   EPI_GRAD: q6 number of zero entries of X
struct RowArgs {
  int64_t n; int r; int b; int64_t ld;
  const void* G;
  const void* X;       // OP_LOAD / OP_ZSTEP
  const void* g_in;    // OP_ZSTEP
  const void* Zin;     // OP_UPD
  const void* Din;     // OP_UPD
  const void* B;
  const void* LX; double gamma;
  const Ctl* ctl;
  const int* run;
  void* Xout;          // operand value written (Z for OP_ZSTEP, X' for OP_UPD/OP_LOAD copy)
  void* gout;          // EPI_GRAD: gradient
  void* Dout;          // EPI_DIR: direction (candidate `dstore`)
  void* D2out;         // EPI_DIR with two candidates: the plain BB direction
  const void* Din2;    // OP_UPD: second direction, used where ctl[j].dsel == 1
  int dstore;          // EPI_DIR: candidate written to Dout
  void* gZout;         // EPI_DIR: gradient at Z
  const void* Xold; const void* gold;    // EPI_GRAD: S = X - Xold, Y = g - gold
  const void* Zold; const void* gZold;   // EPI_GRAD: increment f(X) - f(Zold)
  const void* Wcur; const void* gWcur;   // EPI_DIR: increment f(Z) - f(Wcur)
  int want_q;          // EPI_DIR, one column tile: also <D G, D> -> q4
  double* part;
  int ctl_mode;        // CTL_*: control step run by the last CTA of each restart
  unsigned* counters;  // per-restart arrival counters (zero between launches)
  const double* G64fix;
  Params P;
  int tile;            // 1: the shared-memory tile body (r <= 32, no graph term, <= 2 candidates)
  int bm;              // general body, FP32: rows per CTA (32 or 64; 0 = built-in choice)
};

// Row kernels of a step for FP32 penalty blocks with r in {16, 32, 64} (rowfuse.cu): the D step
// writes g(Z) only (RowArgs X, g_in, B -> gZout; fused line search, ctl_mode CTL_LS) and the
// update recomputes Z and D from X, g, g(Z) (RowArgs Xout = X and gout = g, updated in place,
// gZold, B; ctl_mode CTL_UPD_*).  bm: rows per CTA (64 or 128; r = 16: 128 or 256).  nc = 2:
// the learned step with fallback (the proposal and the plain BB direction, Ctl::cand_alpha).
bool rowfuse_supported(int tdtype, int r);
int rowfuse_bm(int r, int bm_req);
void launch_rowfuse_dstep(const RowArgs& a, int bm, int nc, cudaStream_t s);
void launch_rowfuse_update(const RowArgs& a, int bm, int nc, cudaStream_t s);
// The same pair with the row products on the tensor cores (rowtc.cu: tcgen05 kind::tf32 with
// hi / lo operand parts; FP32 factors, r = 64, one direction per step).  err: device error
// code, set when a bounded wait for the tensor cores runs out.
bool rowtc_supported(int tdtype, int r, int nc);
void launch_rowtc_dstep(const RowArgs& a, int* err, cudaStream_t s);
void launch_rowtc_update(const RowArgs& a, int* err, cudaStream_t s);
// Block-start gradient of the same FP32, r = 64 blocks (no graph term): g = X G - B into
// RowArgs gout from X, B; the block-start control step (ctl_mode) in the last CTA of each
// restart, over ceil(n / 128) partial slots.
void launch_rowtc_grad(const RowArgs& a, int* err, cudaStream_t s);
// The same pair as persistent warp-specialised kernels (rowtma.cu: one CTA per SM over 128-row
// tiles, inputs streamed by TMA into shared slots, outputs stored by TMA).  ld: the factor
// arrays' row pitch (a multiple of 4).  false when the tensor maps cannot be encoded (nothing
// launched).
bool rowtma_supported(int tdtype, int r, int nc, int64_t ld);
bool launch_rowtma_dstep(const RowArgs& a, int* err, cudaStream_t s);
bool launch_rowtma_update(const RowArgs& a, int* err, cudaStream_t s);

void launch_gram(int tdtype, const void* X, const void* Y, const Dims& d, int pair, int npairs,
                 double* gpart, int nchunks, const Ctl* ctl, const int* run, double* G64, void* GT,
                 int tpair, double lam_shift, unsigned* counters, cudaStream_t s,
                 Ctl* rho_ctl = nullptr, int rho_iters = 0, double rho_scale = 1.0, double rho_shift = 0.0);
// partial slots per restart written by launch_rowgemm (tile: the tile body's row tiles)
int rowgemm_slots(const Dims& d, int tdtype, int tile = 0, int bm = 0);
void launch_rowgemm(int tdtype, int op, int epi, const RowArgs& a, cudaStream_t s, int ncand = 1);
void launch_zstep(int tdtype, const Dims& d, const void* X, const void* g, void* Z, const Ctl* ctl,
                  cudaStream_t s);
int launch_xupd(int tdtype, const Dims& d, const void* Z, const void* D, void* Xn, const void* AZ,
                const void* AD, void* AXn, const Ctl* ctl, double* part, cudaStream_t s);
void launch_copy_live(int tdtype, const Dims& d, const void* src, void* dst, const Ctl* ctl,
                      cudaStream_t s);
// rho = scale ||G||_2 + shift per restart (shift: gamma ||L||_2 of a graph-regularised block)
void launch_rho(int tdtype, const double* G64, const Dims& d, int iters, double scale, Ctl* ctl,
                int set_alpha, cudaStream_t s, double shift = 0.0);
void launch_philox_uniform(int tdtype, void* out, int64_t rows, int cols, int64_t ld, uint64_t seed,
                           double scale, cudaStream_t s);
void launch_philox_gaussian(int tdtype, void* out, int64_t rows, int cols, uint64_t seed,
                            cudaStream_t s);
void launch_matrix_sums(int kind, int vdtype, const void* vals, int64_t n, int64_t lda, int64_t nnz,
                        double* part, double* out, cudaStream_t s);
void launch_convert(int sdtype, int ddtype, const void* src, int64_t rows, int64_t cols, int64_t lds,
                    void* dst, int64_t ldd, cudaStream_t s);

void launch_ctl_pen_ls(Ctl* ctl, const double* prow, int nrow, const double* pax, int nax, int b,
                       int r, const double* G64fix, const double* DtD, const Params& P, int graph,
                       cudaStream_t s);
void launch_ctl_dir_init(Ctl* ctl, const double* pax, int nax, const double* prow, int nrow,
                         const double* plx, int nlx, const double* GW, int b, int r, const Params& P,
                         cudaStream_t s);
void launch_ctl_dir_alpha(Ctl* ctl, int b, const Params& P, cudaStream_t s);
void launch_ctl_dir_ls(Ctl* ctl, const double* pz, int nz, const double* prow, int nrow,
                       const double* pd, int nd, const double* GZ, const double* ZD,
                       const double* DDm, const double* pgl, const double* pgd, int b, int r,
                       const Params& P, cudaStream_t s);
void launch_ctl_dir_clip(Ctl* ctl, const double* pclip, int nslots, int b, int* recompute,
                         cudaStream_t s);
void launch_ctl_dir_upd(Ctl* ctl, const double* prow, int nrow, const double* pax, int nax,
                        const double* plx, int nlx, const double* GW, const int* recompute, int b,
                        int r, const Params& P, cudaStream_t s);
void init_kernel_attributes();
void launch_sum_pairs(const double* part, int m, double* out, cudaStream_t s);
void launch_any_active(const Ctl* ctl, int b, int* flag, int* recompute, cudaStream_t s);
void launch_ctl_final_pen(Ctl* ctl, const double* pax, int nax, const double* prow, int nrow,
                          const double* GW, const double* GH, const double* WH, int b, int r,
                          const Params& P, cudaStream_t s);
void launch_ctl_final_dir(Ctl* ctl, const double* GW, int b, int r, const Params& P, cudaStream_t s);

}  // namespace snmf
