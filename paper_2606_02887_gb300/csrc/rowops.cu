// O(n r^2) kernels of an SNMPBB step and the per-restart FP64 control logic.
//
//   k_gram       r x r Gram X_j^T Y_j of each restart j (Eq. (2.1): H H^T, and the
//                Z^T D, D^T D products of the line-search polynomial); FP64 partials per
//                row chunk, reduced in a fixed order by the last CTA of each tile.
//   k_rowgemm    X G - B (+ gamma L X): the gradients of Eqs. (2.1)-(2.2) with the
//                r x r factor G in shared memory, fused with the elementwise steps of
//                Algorithm 1 (Z step, D direction, relaxed update) and the FP64
//                partial inner products the control kernels need.
//   k_ctl_*      one block per restart: rho (power method, Eq. (2.11)), BB step
//                (Alg. 1 line 3, Eq. (2.10)), reference F_k and the backtracking
//                Armijo search in closed form (Alg. 1 line 4), convergence test.
#include <math.h>

#include "common.cuh"
#include "rowops.cuh"
#include "rowops_dev.cuh"

namespace snmf {

namespace {

template <typename T, int TW, int RS>
__global__ void __launch_bounds__(256)
k_gram(const T* __restrict__ X, const T* __restrict__ Y, int64_t n, int r, int b, int64_t ld,
       int64_t chunk, int ntile, double* __restrict__ gpart, int pair, int npairs,
       const Ctl* __restrict__ ctl, const int* run, double* __restrict__ G64, T* __restrict__ GT,
       int tpair, double lam_shift, unsigned* __restrict__ counters, Ctl* __restrict__ rho_ctl,
       int rho_iters, double rho_scale, double rho_shift) {
  gram_body<T, TW, RS>(X, Y, n, r, b, ld, chunk, ntile, gpart, pair, npairs, ctl, run, G64, GT, tpair,
                       lam_shift, counters, rho_ctl, rho_iters, rho_scale, rho_shift, blockIdx.x, gridDim.x,
                       blockIdx.y);
}

template <typename T, int OP, int EPI, int BM, int NC>
__global__ void __launch_bounds__(256, BM == 32 ? 4 : 3) k_rowgemm(RowArgs a) {
  rowgemm_body<T, OP, EPI, BM, NC>(a, blockIdx.z, blockIdx.x, blockIdx.y, gridDim.y, gridDim.x * gridDim.y);
}

// r <= 32: the shared-memory tile body, CTA = TileCfg<T>::TR rows of restart blockIdx.z
template <typename T, int OP, int EPI, int NC>
__global__ void __launch_bounds__(256, EPI == EPI_GRAD ? 2 : 3) k_rowtile(RowArgs a) {
  extern __shared__ __align__(16) unsigned char tsm[];
  rowtile_body<T, OP, EPI, NC>(a, blockIdx.z, blockIdx.x, gridDim.x, reinterpret_cast<T*>(tsm));
}

template <typename T, int OP, int EPI, int NC>
void launch_rowtile(const RowArgs& a, cudaStream_t s) {
  static bool attr = false;
  const size_t smem = rowtile_smem<T>(EPI == EPI_DIR ? 2 + NC : 2);
  if (!attr) {
    cudaFuncSetAttribute(k_rowtile<T, OP, EPI, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  dim3 grid((unsigned)((a.n + TileCfg<T>::TR - 1) / TileCfg<T>::TR), 1, a.b);
  k_rowtile<T, OP, EPI, NC><<<grid, 256, smem, s>>>(a);
}

// Elementwise: Z = Proj[X - g / rho] (Alg. 1 line 2) for restarts that are live.
template <typename T>
__global__ void k_zstep(int64_t n, int r, int b, int64_t ld, const T* __restrict__ X,
                        const T* __restrict__ g, T* __restrict__ Z, const Ctl* __restrict__ ctl) {
  const int64_t total = n * (int64_t)r * b;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ((int64_t)r * b);
    const int col = (int)(e % ((int64_t)r * b));
    const int j = col / r;
    if (!ctl[j].active) continue;
    const int64_t idx = i * ld + col;
    const T v = X[idx] - g[idx] * (T)(1.0 / ctl[j].rho);
    Z[idx] = v > T(0) ? v : T(0);
  }
}

// Relaxed update W' = Proj[Z + phi beta D] (Alg. 1 line 4), optional linear reuse
// AW' = AZ + phi beta AD (valid when nothing is clipped), clip-count partials.
template <typename T>
__global__ void __launch_bounds__(256)
k_xupd(int64_t n, int r, int b, int64_t ld, const T* __restrict__ Z, const T* __restrict__ D,
       T* __restrict__ Xn, const T* __restrict__ AZ, const T* __restrict__ AD,
       T* __restrict__ AXn, const Ctl* __restrict__ ctl, double* __restrict__ part) {
  __shared__ double sh[32];
  const int j = blockIdx.y;
  const int64_t i0 = (int64_t)blockIdx.x * kRowTile;
  double clip = 0.0;
  if (ctl[j].active) {
    const T pb = (T)ctl[j].phibeta;
    const int tile = kRowTile * r;
    for (int e = threadIdx.x; e < tile; e += blockDim.x) {
      const int64_t i = i0 + e / r;
      if (i >= n) break;
      const int64_t idx = i * ld + (int64_t)j * r + (e % r);
      const T v = Z[idx] + pb * D[idx];
      if (v < T(0)) clip += 1.0;
      Xn[idx] = v > T(0) ? v : T(0);
      if (AXn) AXn[idx] = AZ[idx] + pb * AD[idx];
    }
  }
  clip = block_sum(clip, sh);
  if (threadIdx.x == 0) part[((int64_t)blockIdx.x * b + j) * kNQ + 0] = clip;
}

template <typename T>
__global__ void k_copy_live(int64_t n, int r, int b, int64_t ld, const T* __restrict__ src,
                            T* __restrict__ dst, const Ctl* __restrict__ ctl) {
  const int64_t total = n * (int64_t)r * b;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ((int64_t)r * b);
    const int col = (int)(e % ((int64_t)r * b));
    if (ctl && !ctl[col / r].commit) continue;
    dst[i * ld + col] = src[i * ld + col];
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// rho = ||G||_2 by the power method from the ones vector (fixed count) and the
// Rayleigh quotient; rho_scale multiplies the result (direct form).  PT is the
// arithmetic type (double in FP64 precision, float otherwise).
// ---------------------------------------------------------------------------
template <typename PT>
__global__ void k_rho(const double* __restrict__ G64, int r, int iters, double rho_scale, double rho_shift,
                      Ctl* __restrict__ ctl, int set_alpha) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ double sh[32];
  __shared__ PT v[kMaxR], w[kMaxR];
  const int j = blockIdx.x;
  Ctl& c = ctl[j];
  if (!c.active) return;
  PT* Gs = ((size_t)r * r * sizeof(PT) <= 96 * 1024) ? reinterpret_cast<PT*>(smem_raw) : nullptr;
  rho_body<PT>(G64 + (int64_t)j * r * r, r, iters, rho_scale, rho_shift, c, v, w, Gs, sh);
  (void)set_alpha;
}

// ---------------------------------------------------------------------------
// Penalty form control (Sec. 2.1) as a separate launch: the line search.  The block start and
// the update run fused into the producing row kernels (fused_control).
// prow: row-kernel partials (q layout of EPI_GRAD / EPI_DIR), nrow slots.
// ---------------------------------------------------------------------------
// After DIR (q: 0 gd, 1 dd, 2 f(Z)-f(X_k)) and the Gram of D (pair `dpair`):
// line search on f(Z + beta D) - f(Z) = beta gd + beta^2/2 q with
// q = <D^T D, H H^T> + lambda ||D||^2 + gamma <D, L D>.
__global__ void k_ctl_pen_ls(Ctl* __restrict__ ctl, const double* __restrict__ prow, int nrow,
                             const double* __restrict__ pax, int nax, int b, int r,
                             const double* __restrict__ G64fix, const double* __restrict__ DtD,
                             Params P, int graph) {
  __shared__ double sh[32];
  pen_ls_body(ctl[blockIdx.x], prow, nrow, pax, nax, b, r, blockIdx.x, G64fix, DtD, P, graph, sh);
}

// ---------------------------------------------------------------------------
// Direct form control (Eq. (2) with 1/4 scaling; closed-form objective
// 1/4 (||A||^2 - 2 <X, A X> + ||X^T X||^2) + gamma/2 <X, L X>, FP64 assembly).
// ---------------------------------------------------------------------------
__device__ double direct_f(double normA2, double xax, double gg, double gam, double xlx) {
  return 0.25 * (normA2 - 2.0 * xax + gg) + 0.5 * gam * xlx;
}

// init: pax q0 = <W, AW>; prow (EPI_GRAD) q0 = pg2; GW = W^T W; graph: plx q0 = <W,LW>
__global__ void k_ctl_dir_init(Ctl* __restrict__ ctl, const double* __restrict__ pax, int nax,
                               const double* __restrict__ prow, int nrow,
                               const double* __restrict__ plx, int nlx, const double* __restrict__ GW,
                               int b, int r, Params P) {
  __shared__ double sh[32];
  const int j = blockIdx.x;
  Ctl& c = ctl[j];
  const double xax = reduce_slots(pax, nax, b, j, 0, sh);
  const double pg2 = reduce_slots(prow, nrow, b, j, 0, sh);
  const double gg = dot_rr(GW + (int64_t)j * r * r, GW + (int64_t)j * r * r, r, sh);
  double xlx = 0.0;
  if (plx) xlx = reduce_slots(plx, nlx, b, j, 0, sh);
  if (threadIdx.x != 0) return;
  c.xax = xax;
  c.f = direct_f(P.normA2, xax, gg, P.gamma, xlx);
  c.F = c.f;
  hist_reset(c, c.f);
  c.pg0 = sqrt(pg2);
  c.pg = c.pg0;
  c.k = 0;
  c.iters = 0;
  c.active = (c.pg0 > 0.0 && P.max_iter > 0) ? 1 : 0;
  c.commit = 0;
  c.ss = c.sy = c.yy = 0.0;
}

// after k_rho: alpha for this step (k = 0: 1/rho, else BB with fallback)
__global__ void k_ctl_dir_alpha(Ctl* __restrict__ ctl, Params P) {
  const int j = blockIdx.x;
  Ctl& c = ctl[j];
  if (threadIdx.x != 0) return;
  c.commit = 0;
  if (!c.active) return;
  c.alpha = (c.k == 0) ? 1.0 / c.rho : bb_step(c, P, c.rho);
}

// Quartic line search.  pz: q0 <Z,AZ>; prow (EPI_DIR): q0 gd, q1 dd; pd: q0 <Z,AD>, q1 <D,AD>;
// Grams: P0 = Z^T Z (GZ), M = Z^T D (ZD), P2 = D^T D (DD).  Graph: pgl q0 <Z,LZ>, q1 <D,LZ>
// (from the LZ finish) and pgd q0 <D,LD>.
__global__ void k_ctl_dir_ls(Ctl* __restrict__ ctl, const double* __restrict__ pz, int nz,
                             const double* __restrict__ prow, int nrow,
                             const double* __restrict__ pd, int nd, const double* __restrict__ GZ,
                             const double* __restrict__ ZD, const double* __restrict__ DDm,
                             const double* __restrict__ pgl, const double* __restrict__ pgd,
                             int b, int r, Params P) {
  __shared__ double sh[32];
  const int j = blockIdx.x;
  Ctl& c = ctl[j];
  if (!c.active) return;
  const int64_t o = (int64_t)j * r * r;
  const double xaz = reduce_slots(pz, nz, b, j, 0, sh);
  const double gd = reduce_slots(prow, nrow, b, j, 0, sh);
  const double zad = reduce_slots(pd, nd, b, j, 0, sh);
  const double dad = reduce_slots(pd, nd, b, j, 1, sh);
  const double p00 = dot_rr(GZ + o, GZ + o, r, sh);
  const double p01 = dot_sym2(ZD + o, GZ + o, r, sh);
  const double p02 = dot_rr(GZ + o, DDm + o, r, sh);
  const double p11 = norm_sym2(ZD + o, r, sh);
  const double p12 = dot_sym2(ZD + o, DDm + o, r, sh);
  const double p22 = dot_rr(DDm + o, DDm + o, r, sh);
  double zlz = 0.0, dlz = 0.0, dld = 0.0;
  if (pgl) {
    zlz = reduce_slots(pgl, nz, b, j, 0, sh);
    dlz = reduce_slots(prow, nrow, b, j, 3, sh);
    dld = reduce_slots(pgd, nd, b, j, 0, sh);
  }
  if (threadIdx.x != 0) return;
  c.xax_z = xaz; c.zad = zad; c.dad = dad; c.gd = gd;
  c.zlz = zlz; c.dlz = dlz; c.dld = dld;
  c.q = p22;  // kept for diagnostics
  auto fval = [&](double t) {
    const double xax = xaz + 2.0 * t * zad + t * t * dad;
    const double gg = p00 + 2.0 * t * p01 + t * t * (p11 + 2.0 * p02) + 2.0 * t * t * t * p12 +
                      t * t * t * t * p22;
    const double xlx = zlz + 2.0 * t * dlz + t * t * dld;
    return direct_f(P.normA2, xax, gg, P.gamma, xlx);
  };
  c.fZ = fval(0.0);
  if (c.k > 0) c.F = reference(c, P);
  double beta = 1.0;
  bool ok = false;
  for (int t = 0; t < P.max_ls; ++t) {
    if (fval(beta) <= c.F + P.theta * beta * gd) { ok = true; break; }
    beta *= P.beta_shrink;
  }
  if (!ok) { beta = 0.0; c.ls_fail++; }
  c.beta = beta;
  c.phibeta = P.phi * beta;
  // objective at the unclipped relaxed point (used when the update clips nothing)
  c.xax = xaz + 2.0 * c.phibeta * zad + c.phibeta * c.phibeta * dad;
  if (!isfinite(c.fZ) || !isfinite(gd)) { c.nan_seen = 1; c.active = 0; }
}

// clip counts from k_xupd (q0); sets *recompute when any live restart clipped
__global__ void k_ctl_dir_clip(Ctl* __restrict__ ctl, const double* __restrict__ pclip, int nslots,
                               int b, int* __restrict__ recompute) {
  __shared__ double sh[32];
  const int j = blockIdx.x;
  Ctl& c = ctl[j];
  if (!c.active) return;
  const double cl = reduce_slots(pclip, nslots, b, j, 0, sh);
  if (threadIdx.x != 0) return;
  c.clip_now = cl > 0.0 ? 1 : 0;
  if (c.clip_now) { c.clipped++; atomicExch(recompute, 1); }
}

// after the gradient at W' (prow EPI_GRAD: q0 pg2, q2 ss, q3 sy, q4 yy), Gram GW of W',
// optional recomputed <W', AW'> (pax q0), graph <W', LW'> (plx q0).
__global__ void k_ctl_dir_upd(Ctl* __restrict__ ctl, const double* __restrict__ prow, int nrow,
                              const double* __restrict__ pax, int nax,
                              const double* __restrict__ plx, int nlx,
                              const double* __restrict__ GW, const int* __restrict__ recompute,
                              int b, int r, Params P) {
  __shared__ double sh[32];
  const int j = blockIdx.x;
  Ctl& c = ctl[j];
  if (!c.active) return;
  const double pg2 = reduce_slots(prow, nrow, b, j, 0, sh);
  const double ss = reduce_slots(prow, nrow, b, j, 2, sh);
  const double sy = reduce_slots(prow, nrow, b, j, 3, sh);
  const double yy = reduce_slots(prow, nrow, b, j, 4, sh);
  const double gg = dot_rr(GW + (int64_t)j * r * r, GW + (int64_t)j * r * r, r, sh);
  double xax_re = 0.0, xlx = 0.0;
  if (pax) xax_re = reduce_slots(pax, nax, b, j, 0, sh);
  if (plx) xlx = reduce_slots(plx, nlx, b, j, 0, sh);
  if (threadIdx.x != 0) return;
  if (*recompute) c.xax = xax_re;  // A W' was recomputed for every restart
  c.ss = ss; c.sy = sy; c.yy = yy;
  c.f = direct_f(P.normA2, c.xax, gg, P.gamma, xlx);
  hist_push(c, c.f, P.memory);
  c.k++;
  c.iters++;
  c.pg = sqrt(pg2);
  c.commit = 1;
  if (!isfinite(c.f)) { c.nan_seen = 1; c.active = 0; c.commit = 0; return; }
  if (c.pg <= P.tol * c.pg0 || c.iters >= P.max_iter) c.active = 0;
}

// *flag = OR over restarts of ctl[j].active
__global__ void k_any_active(const Ctl* __restrict__ ctl, int b, int* __restrict__ flag,
                             int* __restrict__ recompute) {
  if (threadIdx.x != 0) return;
  int any = 0;
  for (int j = 0; j < b; ++j) any |= ctl[j].active;
  *flag = any;
  if (recompute) *recompute = 0;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11) for the default initialisation and the LAI
// sketch; stream layout identical to the oracle's description.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int i = 0; i < 10; ++i) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

template <typename T>
__global__ void k_philox_uniform(T* __restrict__ out, int64_t rows, int cols, int64_t ld,
                                 uint64_t seed, double scale) {
  const int64_t total = rows * cols;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    uint32_t c[4] = {(uint32_t)t, (uint32_t)((uint64_t)t >> 32), 1u, 0u};
    philox(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const double u = ((double)c[0] + 0.5) * 2.3283064365386963e-10;
    out[(t / cols) * ld + (t % cols)] = (T)(u * scale);
  }
}

template <typename T>
__global__ void k_philox_gaussian(T* __restrict__ out, int64_t rows, int cols, uint64_t seed) {
  const int64_t total = rows * cols;
  const int64_t npairs = (total + 1) / 2;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npairs;
       p += (int64_t)gridDim.x * blockDim.x) {
    uint32_t c[4] = {(uint32_t)p, (uint32_t)((uint64_t)p >> 32), 0u, 0u};
    philox(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const double u1 = ((double)c[0] + 0.5) * 2.3283064365386963e-10;
    const double u2 = ((double)c[1] + 0.5) * 2.3283064365386963e-10;
    const double rad = sqrt(-2.0 * log(u1));
    const double ang = 6.283185307179586 * u2;
    const int64_t t0 = 2 * p;
    out[t0] = (T)(rad * cos(ang));
    if (t0 + 1 < total) out[t0 + 1] = (T)(rad * sin(ang));
  }
}

// sum of squares / sum of a dense or CSR matrix (FP64 partial per block, fixed order)
template <typename TA>
__global__ void k_sumsq_dense(const TA* __restrict__ A, int64_t n, int64_t lda,
                              double* __restrict__ part) {
  __shared__ double sh[32];
  double s2 = 0.0, s1 = 0.0;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
      const double v = (double)A[i * lda + k];
      s2 += v * v;
      s1 += v;
    }
  }
  s2 = block_sum(s2, sh);
  s1 = block_sum(s1, sh);
  if (threadIdx.x == 0) { part[2 * blockIdx.x] = s2; part[2 * blockIdx.x + 1] = s1; }
}

template <typename TV>
__global__ void k_sumsq_vec(const TV* __restrict__ v, int64_t m, double* __restrict__ part) {
  __shared__ double sh[32];
  double s2 = 0.0, s1 = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double x = (double)v[e];
    s2 += x * x;
    s1 += x;
  }
  s2 = block_sum(s2, sh);
  s1 = block_sum(s1, sh);
  if (threadIdx.x == 0) { part[2 * blockIdx.x] = s2; part[2 * blockIdx.x + 1] = s1; }
}

__global__ void k_sum_pairs(const double* __restrict__ part, int m, double* __restrict__ out) {
  __shared__ double sh[32];
  double a = 0.0, c = 0.0;
  for (int t = threadIdx.x; t < m; t += blockDim.x) { a += part[2 * t]; c += part[2 * t + 1]; }
  a = block_sum(a, sh);
  c = block_sum(c, sh);
  if (threadIdx.x == 0) { out[0] = a; out[1] = c; }
}

template <typename TS, typename TD>
__global__ void k_convert(const TS* __restrict__ src, int64_t rows, int64_t cols, int64_t lds,
                          TD* __restrict__ dst, int64_t ldd) {
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols, k = e % cols;
    dst[i * ldd + k] = (TD)src[i * lds + k];
  }
}

// final per-restart stats (penalty): pax q0 = <W, A Ht>; GW = W^T W, GH = Ht^T Ht,
// WH = W^T Ht; prow q0 = pg2 of the W gradient at the final point.
__global__ void k_ctl_final_pen(Ctl* __restrict__ ctl, const double* __restrict__ pax, int nax,
                                const double* __restrict__ prow, int nrow,
                                const double* __restrict__ GW, const double* __restrict__ GH,
                                const double* __restrict__ WH, int b, int r, Params P) {
  __shared__ double sh[32];
  const int j = blockIdx.x;
  const int64_t o = (int64_t)j * r * r;
  final_pen_body(ctl[j], pax, nax, prow, nrow, GW + o, GH + o, WH + o, b, j, r, P.normA2, sh);
  // A restart still active here stopped on the iteration limit: the control step that would
  // have recorded its last state never ran, so its ring record is written from the final point.
  Ctl& c = ctl[j];
  if (threadIdx.x == 0 && P.ring && P.ring_cap > 0 && c.active && !c.nan_seen) {
    double* rec = P.ring + ((int64_t)j * P.ring_cap + (c.iters % P.ring_cap)) * kRingVals;
    rec[0] = (double)c.iters;
    rec[1] = c.fin_pg;
    rec[2] = c.fin_pg * c.pg0;
    rec[3] = c.alpha;
    rec[4] = c.beta;
    rec[5] = (double)c.ls_fail;
    rec[6] = (double)c.mlp_accept;
    rec[7] = 0.0;
  }
}

// final per-restart stats (direct)
__global__ void k_ctl_final_dir(Ctl* __restrict__ ctl, const double* __restrict__ GW, int b, int r,
                                Params P) {
  __shared__ double sh[32];
  const int j = blockIdx.x;
  Ctl& c = ctl[j];
  const int64_t o = (int64_t)j * r * r;
  const double gg = dot_rr(GW + o, GW + o, r, sh);
  if (threadIdx.x != 0) return;
  const double res2 = P.normA2 - 2.0 * c.xax + gg;
  c.fin_res = sqrt(fmax(res2, 0.0) / P.normA2);
  c.fin_f = c.f;
  c.fin_pg = (c.pg0 > 0.0) ? c.pg / c.pg0 : 0.0;
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
void launch_gram(int tdtype, const void* X, const void* Y, const Dims& d, int pair, int npairs,
                 double* gpart, int nchunks, const Ctl* ctl, const int* run, double* G64, void* GT,
                 int tpair, double lam_shift, unsigned* counters, cudaStream_t s, Ctl* rho_ctl,
                 int rho_iters, double rho_scale, double rho_shift) {
  // r <= 32: one 32 x 32 tile per restart (a 64-wide tile would compute 4x the entries)
  const bool narrow = d.r <= 32;
  const int ntile = narrow ? 1 : (d.r + 63) / 64;
  const int64_t chunk = (d.n + nchunks - 1) / nchunks;
  dim3 grid(nchunks, d.b * ntile * ntile);
#define GRAM_ARGS(T) (const T*)X, (const T*)Y, d.n, d.r, d.b, d.ld, chunk, ntile, gpart, pair, npairs, ctl, run, \
                     G64, (T*)GT, tpair, lam_shift, counters
  if (tdtype == 0) {
    if (narrow) k_gram<double, 32, 32><<<grid, 256, 0, s>>>(GRAM_ARGS(double), nullptr, 0, 1.0, 0.0);
    else k_gram<double, 64, 32><<<grid, 256, 0, s>>>(GRAM_ARGS(double), nullptr, 0, 1.0, 0.0);
  } else {
    if (narrow)
      k_gram<float, 32, 64><<<grid, 256, 0, s>>>(GRAM_ARGS(float), rho_ctl, rho_iters, rho_scale, rho_shift);
    else
      k_gram<float, 64, 32><<<grid, 256, 0, s>>>(GRAM_ARGS(float), rho_ctl, rho_iters, rho_scale, rho_shift);
  }
#undef GRAM_ARGS
}

static int rowgemm_bm(const Dims& d, int tdtype) {
  if (tdtype == 0) return 32;  // FP64: keeps the operand/D tile and the G tile within 48 KB
  return (d.n + 63) / 64 * ((d.r + 63) / 64) * d.b >= 2 * 152 ? 64 : 32;
}

int rowgemm_slots(const Dims& d, int tdtype, int tile, int bm_req) {
  if (tile) return cdiv(d.n, tdtype == 0 ? TileCfg<double>::TR : TileCfg<float>::TR);
  const int bm = (tdtype == 1 && (bm_req == 32 || bm_req == 64)) ? bm_req : rowgemm_bm(d, tdtype);
  return cdiv(d.n, bm) * cdiv(d.r, 64);
}

void launch_rowgemm(int tdtype, int op, int epi, const RowArgs& a, cudaStream_t s, int ncand) {
  if (a.tile && a.r <= 32 && !a.LX && ncand <= 2) {
#define TB(T)                                                                   \
    if (epi == EPI_GRAD) {                                                      \
      if (op == OP_LOAD) launch_rowtile<T, OP_LOAD, EPI_GRAD, 1>(a, s);         \
      else if (op == OP_ZSTEP) launch_rowtile<T, OP_ZSTEP, EPI_GRAD, 1>(a, s);  \
      else launch_rowtile<T, OP_UPD, EPI_GRAD, 1>(a, s);                        \
    } else if (op == OP_LOAD) launch_rowtile<T, OP_LOAD, EPI_DIR, 1>(a, s);     \
    else if (ncand == 1) launch_rowtile<T, OP_ZSTEP, EPI_DIR, 1>(a, s);         \
    else launch_rowtile<T, OP_ZSTEP, EPI_DIR, 2>(a, s);
    if (tdtype == 0) { TB(double) } else { TB(float) }
#undef TB
    return;
  }
  Dims d;
  d.n = a.n; d.r = a.r; d.b = a.b; d.N = a.r * a.b; d.ld = a.ld;
  const int bm = (tdtype == 1 && (a.bm == 32 || a.bm == 64)) ? a.bm : rowgemm_bm(d, tdtype);
  dim3 grid(cdiv(a.n, bm), cdiv(a.r, 64), a.b);
#define RG(T, O, E, M, C) k_rowgemm<T, O, E, M, C><<<grid, 256, 0, s>>>(a)
#define RG_M(T, O, E, C) \
  if (sizeof(T) == 8 || bm == 32) RG(T, O, E, 32, C); else RG(float, O, E, 64, C);
#define RG_T(T)                                                             \
  if (epi == EPI_GRAD) {                                                    \
    if (op == OP_LOAD) { RG_M(T, OP_LOAD, EPI_GRAD, 1) }                    \
    else if (op == OP_ZSTEP) { RG_M(T, OP_ZSTEP, EPI_GRAD, 1) }             \
    else { RG_M(T, OP_UPD, EPI_GRAD, 1) }                                   \
  } else if (ncand == 1) {                                                  \
    if (op == OP_LOAD) { RG_M(T, OP_LOAD, EPI_DIR, 1) }                     \
    else { RG_M(T, OP_ZSTEP, EPI_DIR, 1) }                                  \
  } else if (ncand == 2) {                                                  \
    RG_M(T, OP_ZSTEP, EPI_DIR, 2)                                           \
  } else {                                                                  \
    RG_M(T, OP_ZSTEP, EPI_DIR, kNCand)                                      \
  }
  if (tdtype == 0) { RG_T(double) } else { RG_T(float) }
#undef RG_T
#undef RG_M
#undef RG
}

static int grid1d(int64_t total) { return (int)imin64((total + 255) / 256, 152 * 16); }

void launch_zstep(int tdtype, const Dims& d, const void* X, const void* g, void* Z, const Ctl* ctl,
                  cudaStream_t s) {
  const int blocks = grid1d(d.n * d.N);
  if (tdtype == 0)
    k_zstep<double><<<blocks, 256, 0, s>>>(d.n, d.r, d.b, d.ld, (const double*)X, (const double*)g,
                                           (double*)Z, ctl);
  else
    k_zstep<float><<<blocks, 256, 0, s>>>(d.n, d.r, d.b, d.ld, (const float*)X, (const float*)g,
                                          (float*)Z, ctl);
}

int launch_xupd(int tdtype, const Dims& d, const void* Z, const void* D, void* Xn, const void* AZ,
                const void* AD, void* AXn, const Ctl* ctl, double* part, cudaStream_t s) {
  dim3 grid(cdiv(d.n, kRowTile), d.b);
  if (tdtype == 0)
    k_xupd<double><<<grid, 256, 0, s>>>(d.n, d.r, d.b, d.ld, (const double*)Z, (const double*)D,
                                        (double*)Xn, (const double*)AZ, (const double*)AD,
                                        (double*)AXn, ctl, part);
  else
    k_xupd<float><<<grid, 256, 0, s>>>(d.n, d.r, d.b, d.ld, (const float*)Z, (const float*)D,
                                       (float*)Xn, (const float*)AZ, (const float*)AD, (float*)AXn,
                                       ctl, part);
  return grid.x;
}

void launch_copy_live(int tdtype, const Dims& d, const void* src, void* dst, const Ctl* ctl,
                      cudaStream_t s) {
  const int blocks = grid1d(d.n * d.N);
  if (tdtype == 0)
    k_copy_live<double><<<blocks, 256, 0, s>>>(d.n, d.r, d.b, d.ld, (const double*)src, (double*)dst, ctl);
  else
    k_copy_live<float><<<blocks, 256, 0, s>>>(d.n, d.r, d.b, d.ld, (const float*)src, (float*)dst, ctl);
}

void init_kernel_attributes() {
  static bool done = false;
  if (done) return;
  cudaFuncSetAttribute(k_rho<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  cudaFuncSetAttribute(k_rho<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  done = true;
}

void launch_rho(int tdtype, const double* G64, const Dims& d, int iters, double scale, Ctl* ctl,
                int set_alpha, cudaStream_t s, double shift) {
  if (tdtype == 0) {
    size_t sm = (size_t)d.r * d.r * sizeof(double);
    if (sm > 96 * 1024) sm = 0;
    k_rho<double><<<d.b, 256, sm, s>>>(G64, d.r, iters, scale, shift, ctl, set_alpha);
  } else {
    size_t sm = (size_t)d.r * d.r * sizeof(float);
    if (sm > 96 * 1024) sm = 0;
    k_rho<float><<<d.b, 256, sm, s>>>(G64, d.r, iters, scale, shift, ctl, set_alpha);
  }
}

void launch_philox_uniform(int tdtype, void* out, int64_t rows, int cols, int64_t ld, uint64_t seed,
                           double scale, cudaStream_t s) {
  const int blocks = grid1d(rows * cols);
  if (tdtype == 0) k_philox_uniform<double><<<blocks, 256, 0, s>>>((double*)out, rows, cols, ld, seed, scale);
  else k_philox_uniform<float><<<blocks, 256, 0, s>>>((float*)out, rows, cols, ld, seed, scale);
}

void launch_philox_gaussian(int tdtype, void* out, int64_t rows, int cols, uint64_t seed,
                            cudaStream_t s) {
  const int blocks = grid1d((rows * cols + 1) / 2);
  if (tdtype == 0) k_philox_gaussian<double><<<blocks, 256, 0, s>>>((double*)out, rows, cols, seed);
  else k_philox_gaussian<float><<<blocks, 256, 0, s>>>((float*)out, rows, cols, seed);
}

// ||A||_F^2 and sum(A) -> out[0], out[1] (device doubles); part needs 2*1024 doubles
void launch_matrix_sums(int kind, int vdtype, const void* vals, int64_t n, int64_t lda, int64_t nnz,
                        double* part, double* out, cudaStream_t s) {
  int blocks = 1024;
  if (kind == AX_DENSE) {
    blocks = (int)imin64(n, 1024);
    if (vdtype == 0) k_sumsq_dense<double><<<blocks, 256, 0, s>>>((const double*)vals, n, lda, part);
    else k_sumsq_dense<float><<<blocks, 256, 0, s>>>((const float*)vals, n, lda, part);
  } else {
    blocks = (int)imax64(1, imin64((nnz + 255) / 256, 1024));
    if (vdtype == 0) k_sumsq_vec<double><<<blocks, 256, 0, s>>>((const double*)vals, nnz, part);
    else k_sumsq_vec<float><<<blocks, 256, 0, s>>>((const float*)vals, nnz, part);
  }
  k_sum_pairs<<<1, 256, 0, s>>>(part, blocks, out);
}

void launch_sum_pairs(const double* part, int m, double* out, cudaStream_t s) {
  k_sum_pairs<<<1, 256, 0, s>>>(part, m, out);
}

void launch_convert(int sdtype, int ddtype, const void* src, int64_t rows, int64_t cols, int64_t lds,
                    void* dst, int64_t ldd, cudaStream_t s) {
  const int blocks = grid1d(rows * cols);
  if (sdtype == 0 && ddtype == 0)
    k_convert<double, double><<<blocks, 256, 0, s>>>((const double*)src, rows, cols, lds, (double*)dst, ldd);
  else if (sdtype == 0 && ddtype == 1)
    k_convert<double, float><<<blocks, 256, 0, s>>>((const double*)src, rows, cols, lds, (float*)dst, ldd);
  else if (sdtype == 1 && ddtype == 0)
    k_convert<float, double><<<blocks, 256, 0, s>>>((const float*)src, rows, cols, lds, (double*)dst, ldd);
  else
    k_convert<float, float><<<blocks, 256, 0, s>>>((const float*)src, rows, cols, lds, (float*)dst, ldd);
}

void launch_ctl_pen_ls(Ctl* ctl, const double* prow, int nrow, const double* pax, int nax, int b,
                       int r, const double* G64fix, const double* DtD, const Params& P, int graph,
                       cudaStream_t s) {
  k_ctl_pen_ls<<<b, 32, 0, s>>>(ctl, prow, nrow, pax, nax, b, r, G64fix, DtD, P, graph);
}
void launch_ctl_dir_init(Ctl* ctl, const double* pax, int nax, const double* prow, int nrow,
                         const double* plx, int nlx, const double* GW, int b, int r, const Params& P,
                         cudaStream_t s) {
  k_ctl_dir_init<<<b, 32, 0, s>>>(ctl, pax, nax, prow, nrow, plx, nlx, GW, b, r, P);
}
void launch_ctl_dir_alpha(Ctl* ctl, int b, const Params& P, cudaStream_t s) {
  k_ctl_dir_alpha<<<b, 32, 0, s>>>(ctl, P);
}
void launch_ctl_dir_ls(Ctl* ctl, const double* pz, int nz, const double* prow, int nrow,
                       const double* pd, int nd, const double* GZ, const double* ZD,
                       const double* DDm, const double* pgl, const double* pgd, int b, int r,
                       const Params& P, cudaStream_t s) {
  k_ctl_dir_ls<<<b, 32, 0, s>>>(ctl, pz, nz, prow, nrow, pd, nd, GZ, ZD, DDm, pgl, pgd, b, r, P);
}
void launch_ctl_dir_clip(Ctl* ctl, const double* pclip, int nslots, int b, int* recompute,
                         cudaStream_t s) {
  k_ctl_dir_clip<<<b, 32, 0, s>>>(ctl, pclip, nslots, b, recompute);
}
void launch_ctl_dir_upd(Ctl* ctl, const double* prow, int nrow, const double* pax, int nax,
                        const double* plx, int nlx, const double* GW, const int* recompute, int b,
                        int r, const Params& P, cudaStream_t s) {
  k_ctl_dir_upd<<<b, 32, 0, s>>>(ctl, prow, nrow, pax, nax, plx, nlx, GW, recompute, b, r, P);
}
void launch_any_active(const Ctl* ctl, int b, int* flag, int* recompute, cudaStream_t s) {
  k_any_active<<<1, 32, 0, s>>>(ctl, b, flag, recompute);
}
void launch_ctl_final_pen(Ctl* ctl, const double* pax, int nax, const double* prow, int nrow,
                          const double* GW, const double* GH, const double* WH, int b, int r,
                          const Params& P, cudaStream_t s) {
  k_ctl_final_pen<<<b, 32, 0, s>>>(ctl, pax, nax, prow, nrow, GW, GH, WH, b, r, P);
}
void launch_ctl_final_dir(Ctl* ctl, const double* GW, int b, int r, const Params& P, cudaStream_t s) {
  k_ctl_final_dir<<<b, 32, 0, s>>>(ctl, GW, b, r, P);
}

}  // namespace snmf
