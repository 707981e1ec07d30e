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

namespace snmf {

namespace {

inline int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
inline int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }
inline int64_t imax64(int64_t a, int64_t b) { return a > b ? a : b; }

// ------------------------------------------------------------------------------
// control helpers and bodies (run by one block: a control kernel, or the last CTA of
// a producing kernel for that restart)
// ------------------------------------------------------------------------------
// Warp-level (one warp) fixed-order reductions: lane l sums entries l, l+32, ... in order,
// then a butterfly of fixed shape; every lane gets the same value.
__device__ double reduce_slots(const double* part, int nslots, int b, int j, int q, double* /*sh*/) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  int t = lane;
  for (; t + 96 < nslots; t += 128) {  // four loads in flight, summed in slot order
    const double v0 = __ldcg(part + ((int64_t)t * b + j) * kNQ + q);
    const double v1 = __ldcg(part + ((int64_t)(t + 32) * b + j) * kNQ + q);
    const double v2 = __ldcg(part + ((int64_t)(t + 64) * b + j) * kNQ + q);
    const double v3 = __ldcg(part + ((int64_t)(t + 96) * b + j) * kNQ + q);
    s += v0; s += v1; s += v2; s += v3;
  }
  for (; t < nslots; t += 32) s += __ldcg(part + ((int64_t)t * b + j) * kNQ + q);
  return warp_sum(s);
}

// All kNQ quantities of restart j at once (each slot's record is 64 contiguous bytes);
// out[q] = fixed-order sum over slots, in every lane.
__device__ void reduce_slots_all(const double* part, int nslots, int b, int j, double* out) {
  const int lane = threadIdx.x & 31;
  double acc[kNQ];
#pragma unroll
  for (int q = 0; q < kNQ; ++q) acc[q] = 0.0;
  int t = lane;
  for (; t + 32 < nslots; t += 64) {
    const double2* r0 = reinterpret_cast<const double2*>(part + ((int64_t)t * b + j) * kNQ);
    const double2* r1 = reinterpret_cast<const double2*>(part + ((int64_t)(t + 32) * b + j) * kNQ);
    double2 a[4], c[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) { a[u] = __ldcg(r0 + u); c[u] = __ldcg(r1 + u); }
#pragma unroll
    for (int u = 0; u < 4; ++u) { acc[2 * u] += a[u].x; acc[2 * u + 1] += a[u].y; }
#pragma unroll
    for (int u = 0; u < 4; ++u) { acc[2 * u] += c[u].x; acc[2 * u + 1] += c[u].y; }
  }
  for (; t < nslots; t += 32) {
    const double2* r0 = reinterpret_cast<const double2*>(part + ((int64_t)t * b + j) * kNQ);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const double2 a = __ldcg(r0 + u);
      acc[2 * u] += a.x;
      acc[2 * u + 1] += a.y;
    }
  }
#pragma unroll
  for (int q = 0; q < kNQ; ++q) out[q] = warp_sum(acc[q]);
}

// sum_e A[e] B[e] over r*r entries (fixed order); A/B FP64 matrices.
__device__ double dot_rr(const double* A, const double* B, int r, double* /*sh*/) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int e = lane; e < r * r; e += 32) s += __ldcg(A + e) * __ldcg(B + e);
  return warp_sum(s);
}

// sum_{p,q} (M + M^T)_{pq} X_{pq} for a general r x r M and symmetric X
__device__ double dot_sym2(const double* M, const double* X, int r, double* /*sh*/) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int e = lane; e < r * r; e += 32) {
    const int p = e / r, q = e % r;
    s += (M[e] + M[q * r + p]) * X[e];
  }
  return warp_sum(s);
}

// <M+M^T, M+M^T> for general M
__device__ double norm_sym2(const double* M, int r, double* /*sh*/) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int e = lane; e < r * r; e += 32) {
    const int p = e / r, q = e % r;
    const double v = M[e] + M[q * r + p];
    s += v * v;
  }
  return warp_sum(s);
}

__device__ double bb_step(const Ctl& c, const Params& P, double rho) {
  // Alg. 1 line 3 / Eq. (2.10), with the fallback 1/rho when <S,Y> <= 0
  double a;
  if (!(c.sy > 0.0)) a = 1.0 / rho;
  else a = (P.bb == 0) ? c.ss / c.sy : c.sy / c.yy;
  return fmin(P.alpha_max, fmax(P.alpha_min, a));
}

__device__ void hist_reset(Ctl& c, double f) {
  c.hlen = 1;
  c.hpos = 0;
  c.fhist[0] = f;
}

__device__ void hist_push(Ctl& c, double f, int M) {
  const int cap = M > 0 ? M : 1;
  c.hpos = (c.hpos + 1) % cap;
  c.fhist[c.hpos] = f;
  if (c.hlen < cap) c.hlen++;
}

// F_k of Alg. 1 line 4 (eta averaging) or the max of the last M values; called at k > 0
// after f(X_k) has been pushed.
__device__ double reference(const Ctl& c, const Params& P) {
  if (P.memory > 0) {
    double m = -INFINITY;
    for (int t = 0; t < c.hlen; ++t) m = fmax(m, c.fhist[t]);
    return m;
  }
  return c.f + P.eta * (c.F - c.f);
}

// rho = rho_scale * ||G||_2: power method from the ones vector (fixed count) and the
// Rayleigh quotient (Alg. 1 line 2, Eq. (2.11)), by a whole block of 256 threads: row p of
// G v is summed by tpr threads (adjacent lanes, fixed butterfly), the norm by a fixed-order
// block reduction.  Gs: G in shared memory (PT) or NULL; v, w: shared scratch (r entries);
// sh: shared scratch of 8 doubles.
template <typename PT>
__device__ void rho_body(const double* __restrict__ Gj, int r, int iters, double rho_scale, Ctl& c,
                         PT* __restrict__ v, PT* __restrict__ w, PT* __restrict__ Gs, double* sh) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (Gs)
    for (int e = tid; e < r * r; e += nt) Gs[e] = (PT)__ldcg(Gj + e);
  const PT v0 = (PT)(1.0 / sqrt((double)r));
  for (int p = tid; p < r; p += nt) v[p] = v0;
  __syncthreads();
  auto gval = [&](int q, int p) -> PT { return Gs ? Gs[q * r + p] : (PT)__ldcg(Gj + q * r + p); };
  const int tpr = r <= 64 ? 4 : (r <= 128 ? 2 : 1);  // threads per row (nt = 256)
  const int p = tid / tpr, part_id = tid % tpr;
  const int lane = tid & 31, wid = tid >> 5;
  // G v for row p restricted to the q-range of this thread; tpr partial sums combined in a fixed order
  auto row_dot = [&]() -> PT {
    PT s0 = 0, s1 = 0;
    if (p < r) {
      int q = part_id;
      for (; q + tpr < r; q += 2 * tpr) {
        s0 += gval(q, p) * v[q];
        s1 += gval(q + tpr, p) * v[q + tpr];
      }
      if (q < r) s0 += gval(q, p) * v[q];
    }
    PT s = s0 + s1;
    if (tpr >= 2) s += __shfl_xor_sync(0xffffffffu, s, 1);
    if (tpr >= 4) s += __shfl_xor_sync(0xffffffffu, s, 2);
    return s;
  };
  // arithmetic in PT (FP32 in the reduced-precision modes: FP64 is slow on this part)
  PT* shp = reinterpret_cast<PT*>(sh);
  PT rho = 0;
  bool zero = false;
  for (int it = 0; it < iters; ++it) {
    const PT s = row_dot();
    PT sq = (p < r && part_id == 0) ? s * s : PT(0);
    sq = warp_sum(sq);
    if (lane == 0) shp[wid] = sq;
    __syncthreads();
    PT tot = 0;
    for (int u = 0; u < (nt >> 5); ++u) tot += shp[u];
    if (tot == PT(0)) { zero = true; break; }
    if (p < r && part_id == 0) w[p] = s / sqrt(tot);
    __syncthreads();
    if (p < r && part_id == 0) v[p] = w[p];
    __syncthreads();
  }
  if (!zero) {
    const PT s = row_dot();
    PT pr = (p < r && part_id == 0) ? v[p] * s : PT(0);
    pr = warp_sum(pr);
    __syncthreads();
    if (lane == 0) shp[wid] = pr;
    __syncthreads();
    for (int u = 0; u < (nt >> 5); ++u) rho += shp[u];
  }
  if (tid == 0) {
    double rr = rho_scale * (double)rho;
    if (!(rr > 0.0)) rr = 1.0;  // zero Gram: unit scaling
    c.rho = rr;
  }
  __syncthreads();
}

// Penalty block start: joint projected gradient / convergence (W block), reset of the
// block's reference (Alg. 1 line 4: F_0 = f(X_0)) and alpha_0 = 1/rho.  One warp.
__device__ void pen_start_body(Ctl& c, const double* prow, int nrow, int b, int j, const Params& P,
                               int is_w_block, int first, double* sh) {
  if (!c.active) return;
  const double pg2 = reduce_slots(prow, nrow, b, j, 0, sh);
  if ((threadIdx.x & 31) != 0) return;
  if (is_w_block) {
    const double joint = sqrt(pg2 + c.pgH2);
    c.pg = joint;
    if (c.iters == 0) c.pg0 = joint;
    else if (joint <= P.tol * c.pg0 || c.iters >= P.max_iter) { c.active = 0; return; }
    if (!isfinite(joint)) { c.nan_seen = 1; c.active = 0; return; }
  } else {
    if (first) { c.pgH2 = pg2; return; }  // solve initialisation: H gradient at start
  }
  c.f = 0.0;  // block-relative objective: f(X_0) = 0
  c.F = 0.0;
  hist_reset(c, 0.0);
  c.k = 0;
  c.alpha = 1.0 / c.rho;
}

// Line search after the D direction (q: 0 gd, 1 dd, 2 f(Z)-f(X_k), 4 <D G, D> when fused):
// f(Z + beta D) - f(Z) = beta gd + beta^2/2 q, q = <D (H H^T + lambda I), D> + gamma <D, L D>.
__device__ void pen_ls_body(Ctl& c, const double* prow, int nrow, const double* pax, int nax, int b, int r,
                            int j, const double* G64fix, const double* DtD, const Params& P, int graph,
                            double* sh) {
  if (!c.active) return;
  double qs[kNQ];
  reduce_slots_all(prow, nrow, b, j, qs);
  const double gd = qs[0], dd = qs[1], dzw = qs[2];
  const double qg = DtD ? dot_rr(DtD + (int64_t)j * r * r, G64fix + (int64_t)j * r * r, r, sh) + c.lam * dd
                        : qs[4];
  double dld = 0.0;
  if (graph) dld = reduce_slots(pax, nax, b, j, 0, sh);
  if ((threadIdx.x & 31) != 0) return;
  const double q = qg + P.gamma * dld;
  c.gd = gd;
  c.q = q;
  c.fZ = c.f + dzw;
  if (c.k > 0) c.F = reference(c, P);
  double beta = 1.0;
  bool ok = false;
  for (int t = 0; t < P.max_ls; ++t) {
    const double fz = c.fZ + beta * gd + 0.5 * beta * beta * q;
    if (fz <= c.F + P.theta * beta * gd) { ok = true; break; }
    beta *= P.beta_shrink;
  }
  if (!ok) { beta = 0.0; c.ls_fail++; }
  if (!isfinite(c.fZ) || !isfinite(q) || !isfinite(gd)) { c.nan_seen = 1; c.active = 0; }
  c.beta = beta;
  c.phibeta = P.phi * beta;
}

// After the relaxed update (q: 0 pg2, 2 ss, 3 sy, 4 yy, 5 f(X')-f(Z)).  One warp.
__device__ void pen_upd_body(Ctl& c, const double* prow, int nrow, int b, int j, const Params& P, int is_h_block,
                             int last, double* sh) {
  if (!c.active) return;
  double qs[kNQ];
  reduce_slots_all(prow, nrow, b, j, qs);
  const double pg2 = qs[0], ss = qs[2], sy = qs[3], yy = qs[4], dwz = qs[5];
  if ((threadIdx.x & 31) != 0) return;
  c.ss = ss; c.sy = sy; c.yy = yy;
  c.f = c.fZ + dwz;
  hist_push(c, c.f, P.memory);
  c.k++;
  c.alpha = bb_step(c, P, c.rho);
  if (is_h_block) {
    c.pgH2 = pg2;
    if (last) c.iters++;
  }
  if (!isfinite(c.f)) { c.nan_seen = 1; c.active = 0; }
}

// Fused control after a producing kernel: modes of RowArgs::ctl_mode.
__device__ void fused_control(int mode, Ctl& c, const double* part, int nslots, int b, int r, int j,
                              const Params& P, const double* G64fix, double* sh) {
  switch (mode) {
    case CTL_START_W: pen_start_body(c, part, nslots, b, j, P, 1, 0, sh); break;
    case CTL_START_H: pen_start_body(c, part, nslots, b, j, P, 0, 0, sh); break;
    case CTL_START_INIT: pen_start_body(c, part, nslots, b, j, P, 0, 1, sh); break;
    case CTL_LS: pen_ls_body(c, part, nslots, nullptr, 0, b, r, j, G64fix, nullptr, P, 0, sh); break;
    case CTL_UPD_W: pen_upd_body(c, part, nslots, b, j, P, 0, 0, sh); break;
    case CTL_UPD_H: pen_upd_body(c, part, nslots, b, j, P, 1, 0, sh); break;
    case CTL_UPD_H_LAST: pen_upd_body(c, part, nslots, b, j, P, 1, 1, sh); break;
    default: break;
  }
}


// ------------------------------------------------------------------------------
// Gram X_j^T Y_j per restart j.  CTA (chunk, tile): a 64x64 output tile over a chunk of
// rows (16x16 threads, 4x4 micro tiles), FP64 partial written to gpart.  The last CTA of
// each tile (arrival counter) sums the partials in chunk order and writes G64 (and the
// factor-type copy with lam_shift * I on the diagonal when pair == tpair): a fixed-order,
// deterministic two-stage reduction in one launch.
// ------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_gram(const T* __restrict__ X, const T* __restrict__ Y, int64_t n, int r, int b, int64_t ld,
       int64_t chunk, int ntile, double* __restrict__ gpart, int pair, int npairs,
       const Ctl* __restrict__ ctl, const int* run, double* __restrict__ G64, T* __restrict__ GT,
       int tpair, double lam_shift, unsigned* __restrict__ counters, Ctl* __restrict__ rho_ctl,
       int rho_iters, double rho_scale) {
  const int j = blockIdx.y / (ntile * ntile);
  const int t = blockIdx.y % (ntile * ntile);
  const int ti = t / ntile, tj = t % ntile;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t i_begin = (int64_t)blockIdx.x * chunk;
  const int64_t i_end = min(n, i_begin + chunk);
  constexpr int RS = 32;  // rows staged per round
  __shared__ T Xs[RS][64 + 1];
  __shared__ T Ys[RS][64 + 1];
  __shared__ unsigned ticket;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = T(0);
  const bool skip = (run && *run == 0) || (ctl && !ctl[j].active);
  if (!skip) {
    const int64_t cx = (int64_t)j * r + ti * 64;
    const int64_t cy = (int64_t)j * r + tj * 64;
    const int wx = min(64, r - ti * 64), wy = min(64, r - tj * 64);
    for (int64_t i0 = i_begin; i0 < i_end; i0 += RS) {
      T xv_[RS * 64 / 256], yv_[RS * 64 / 256];
#pragma unroll
      for (int m = 0; m < RS * 64 / 256; ++m) {
        const int e = threadIdx.x + 256 * m;
        const int rr = e >> 6, cc = e & 63;
        const int64_t i = i0 + rr;
        xv_[m] = (i < i_end && cc < wx) ? X[i * ld + cx + cc] : T(0);
        yv_[m] = (i < i_end && cc < wy) ? Y[i * ld + cy + cc] : T(0);
      }
#pragma unroll
      for (int m = 0; m < RS * 64 / 256; ++m) {
        const int e = threadIdx.x + 256 * m;
        Xs[e >> 6][e & 63] = xv_[m];
        Ys[e >> 6][e & 63] = yv_[m];
      }
      __syncthreads();
#pragma unroll 8
      for (int rr = 0; rr < RS; ++rr) {
        T xa[4], yb[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) xa[a] = Xs[rr][ty + 16 * a];
#pragma unroll
        for (int c = 0; c < 4; ++c) yb[c] = Ys[rr][tx + 16 * c];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[a][c] = fma(xa[a], yb[c], acc[a][c]);
      }
      __syncthreads();
    }
  }
  const int64_t rr2 = (int64_t)r * r;
  const int64_t tile_base = ((int64_t)pair * b + j) * rr2;   // offset inside one chunk slab
  const int64_t slab = (int64_t)npairs * b * rr2;
  T* gp = reinterpret_cast<T*>(gpart);  // chunk partials in the working type
  T* out = gp + (int64_t)blockIdx.x * slab + tile_base;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int p = ti * 64 + ty + 16 * a;
    if (p >= r) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int q = tj * 64 + tx + 16 * c;
      if (q < r) out[(int64_t)p * r + q] = acc[a][c];
    }
  }
  __threadfence();
  __syncthreads();
  const int tile_id = ((pair * b + j) * ntile + ti) * ntile + tj;
  if (threadIdx.x == 0) ticket = atomicAdd(&counters[tile_id], 1u);
  __syncthreads();
  if (ticket != gridDim.x - 1) return;
  // last CTA of this tile: fixed-order sum over the chunks
  // each thread owns 16 tile entries and sums them over the chunks in chunk order, with
  // the 16 loads of a chunk (and the next chunk's) in flight together
  const int nch = (int)gridDim.x;
  int64_t off_[16];
  bool ok_[16];
  T sacc[16];
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    const int e = threadIdx.x + 256 * u;
    const int p = ti * 64 + (e >> 6), q = tj * 64 + (e & 63);
    ok_[u] = (p < r && q < r);
    off_[u] = tile_base + (int64_t)(ok_[u] ? p : 0) * r + (ok_[u] ? q : 0);
    sacc[u] = T(0);
  }
#pragma unroll 2
  for (int c = 0; c < nch; ++c) {
    T v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) v[u] = ok_[u] ? __ldcg(gp + (int64_t)c * slab + off_[u]) : T(0);
#pragma unroll
    for (int u = 0; u < 16; ++u) sacc[u] += v[u];
  }
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    if (!ok_[u]) continue;
    const int e = threadIdx.x + 256 * u;
    const int p = ti * 64 + (e >> 6), q = tj * 64 + (e & 63);
    G64[off_[u]] = (double)sacc[u];
    if (GT && pair == tpair) GT[(int64_t)j * rr2 + (int64_t)p * r + q] = sacc[u] + (p == q ? (T)lam_shift : T(0));
  }
  if (threadIdx.x == 0) counters[tile_id] = 0u;  // ready for the next launch
  if (sizeof(T) == 4 && rho_ctl && ntile == 1 && pair == 0 && rho_ctl[j].active) {
    // the restart's Gram is complete: rho = rho_scale ||G||_2 here (saves a launch)
    __shared__ T vv[64], ww[64];
    __shared__ T Gsr[64 * 64];
    __shared__ double shr[8];
    __syncthreads();
    rho_body<T>(G64 + tile_base, r, rho_iters, rho_scale, rho_ctl[j], vv, ww, Gsr, shr);
  }
}

// ------------------------------------------------------------------------------
// Row GEMM with fused Algorithm-1 epilogues.
// ------------------------------------------------------------------------------
template <typename T, int OP, int EPI, int BM>
__global__ void __launch_bounds__(256, 2) k_rowgemm(RowArgs a) {
  constexpr int MR = BM / 16;  // rows per thread
  constexpr int KC = sizeof(T) == 4 ? 64 : 32;  // K columns staged per round
  constexpr int XS_ELEMS = BM * (KC + 1);
  constexpr int DS_ELEMS = (EPI == EPI_DIR) ? BM * 65 : 1;
  constexpr int U_ELEMS = XS_ELEMS > DS_ELEMS ? XS_ELEMS : DS_ELEMS;
  const int j = blockIdx.z;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const int col0 = blockIdx.y * 64;  // within restart
  const int r = a.r;
  const int64_t ld = a.ld;
  const int64_t jc = (int64_t)j * r;
  __shared__ T shq[8][8];
  __shared__ __align__(16) T ubuf[U_ELEMS];   // operand tile, later the D tile
  __shared__ T Gs[KC][64 + 1];
  T (*Xs)[KC + 1] = reinterpret_cast<T (*)[KC + 1]>(ubuf);
  T (*Ds)[65] = reinterpret_cast<T (*)[65]>(ubuf);
  const Ctl& cj = a.ctl[j];
  const bool live = cj.active && !(a.run && *a.run == 0);
  T dq[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // per-CTA partials in the working type
  if (live) {
    const T* G = (const T*)a.G + (int64_t)j * r * r;
    const T inv_rho = (T)(1.0 / cj.rho);
    const T pb = (T)cj.phibeta;
    const T alpha = (T)cj.alpha;
    const T* X = (const T*)a.X;
    const T* gin = (const T*)a.g_in;
    const T* Zin = (const T*)a.Zin;
    const T* Din = (const T*)a.Din;
    auto operand = [&](int64_t i, int64_t col) -> T {
      const int64_t idx = i * ld + col;
      if (OP == OP_LOAD) return X[idx];
      if (OP == OP_ZSTEP) { T v = X[idx] - gin[idx] * inv_rho; return v > T(0) ? v : T(0); }
      T v = Zin[idx] + pb * Din[idx];
      return v > T(0) ? v : T(0);
    };
    T acc[MR][4];
#pragma unroll
    for (int p = 0; p < MR; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[p][q] = T(0);
    for (int k0 = 0; k0 < r; k0 += KC) {
      {
        // all loads of the round in flight before the shared-memory stores
        constexpr int NX = BM * KC / 256, NG = KC * 64 / 256;
        T xv_[NX], gv_[NG];
#pragma unroll
        for (int m = 0; m < NX; ++m) {
          const int e = threadIdx.x + 256 * m;
          const int rr = e / KC, kk = e % KC;
          const int64_t i = row0 + rr;
          xv_[m] = (i < a.n && k0 + kk < r) ? operand(i, jc + k0 + kk) : T(0);
        }
#pragma unroll
        for (int m = 0; m < NG; ++m) {
          const int e = threadIdx.x + 256 * m;
          const int gk = e >> 6, gc = e & 63;
          gv_[m] = (k0 + gk < r && col0 + gc < r) ? G[(int64_t)(k0 + gk) * r + col0 + gc] : T(0);
        }
#pragma unroll
        for (int m = 0; m < NX; ++m) {
          const int e = threadIdx.x + 256 * m;
          Xs[e / KC][e % KC] = xv_[m];
        }
#pragma unroll
        for (int m = 0; m < NG; ++m) {
          const int e = threadIdx.x + 256 * m;
          Gs[e >> 6][e & 63] = gv_[m];
        }
      }
      __syncthreads();
      const int kn = min(KC, r - k0);
#pragma unroll 8
      for (int kk = 0; kk < kn; ++kk) {
        T xa[MR], gb[4];
#pragma unroll
        for (int p = 0; p < MR; ++p) xa[p] = Xs[ty + 16 * p][kk];
#pragma unroll
        for (int q = 0; q < 4; ++q) gb[q] = Gs[kk][tx + 16 * q];
#pragma unroll
        for (int p = 0; p < MR; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[p][q] = fma(xa[p], gb[q], acc[p][q]);
      }
      __syncthreads();
    }
    // epilogue
    T tq[6] = {0, 0, 0, 0, 0, 0};
    const T* B = (const T*)a.B;
    const T* LX = (const T*)a.LX;
    const T gam = (T)a.gamma;
    T dloc[MR][4];
#pragma unroll
    for (int p = 0; p < MR; ++p) {
      const int64_t i = row0 + ty + 16 * p;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        dloc[p][q] = T(0);
        const int c = col0 + tx + 16 * q;
        if (i >= a.n || c >= r) continue;
        const int64_t idx = i * ld + jc + c;
        const T xv = operand(i, jc + c);
        T g = acc[p][q] - B[idx];
        if (LX) g += gam * LX[idx];
        if (EPI == EPI_GRAD) {
          const T pgv = xv > T(0) ? g : (g < T(0) ? g : T(0));
          tq[0] += pgv * pgv;                              // ||P grad||^2
          tq[1] += T(0.5) * (g - B[idx]) * xv;              // f - const (quadratic block)
          if (a.Xold) {
            const T sv = xv - ((const T*)a.Xold)[idx];
            const T yv = g - ((const T*)a.gold)[idx];
            tq[2] += sv * sv;
            tq[3] += sv * yv;
            tq[4] += yv * yv;
          }
          if (a.Zold) {                                     // f(X') - f(Z), trapezoid (exact)
            tq[5] += T(0.5) * (xv - ((const T*)a.Zold)[idx]) * (g + ((const T*)a.gZold)[idx]);
          }
          if (a.gout) ((T*)a.gout)[idx] = g;
          if (a.Xout) ((T*)a.Xout)[idx] = xv;  // after Xold was read (may alias)
        } else {  // EPI_DIR
          if (a.Xout) ((T*)a.Xout)[idx] = xv;
          T d = xv - alpha * g;
          d = (d > T(0) ? d : T(0)) - xv;
          ((T*)a.Dout)[idx] = d;
          dloc[p][q] = d;
          if (a.gZout) ((T*)a.gZout)[idx] = g;
          tq[0] += g * d;                                   // <grad f(Z), D>
          tq[1] += d * d;                                   // ||D||^2
          if (a.Wcur) {                                     // f(Z) - f(W), trapezoid (exact)
            tq[2] += T(0.5) * (xv - ((const T*)a.Wcur)[idx]) * (g + ((const T*)a.gWcur)[idx]);
          }
          if (LX) tq[3] += d * LX[idx];                     // <D, L Z> (direct, graph)
        }
      }
    }
#pragma unroll
    for (int m = 0; m < 6; ++m) dq[m] = tq[m];
    if (EPI == EPI_DIR && a.want_q) {
      // <D G, D> of the line-search quadratic (the whole restart is one column tile)
#pragma unroll
      for (int p = 0; p < MR; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) Ds[ty + 16 * p][tx + 16 * q] = dloc[p][q];
      __syncthreads();
      T acc2[MR][4];
#pragma unroll
      for (int p = 0; p < MR; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc2[p][q] = T(0);
      for (int k0 = 0; k0 < r; k0 += KC) {
        {
          constexpr int NG = KC * 64 / 256;
          T gv_[NG];
#pragma unroll
          for (int m = 0; m < NG; ++m) {
            const int e = threadIdx.x + 256 * m;
            const int gk = e >> 6, gc = e & 63;
            gv_[m] = (k0 + gk < r && gc < r) ? G[(int64_t)(k0 + gk) * r + gc] : T(0);
          }
#pragma unroll
          for (int m = 0; m < NG; ++m) {
            const int e = threadIdx.x + 256 * m;
            Gs[e >> 6][e & 63] = gv_[m];
          }
        }
        __syncthreads();
        const int kn = min(KC, r - k0);
#pragma unroll 8
        for (int kk = 0; kk < kn; ++kk) {
          T gb[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) gb[q] = Gs[kk][tx + 16 * q];
#pragma unroll
          for (int p = 0; p < MR; ++p) {
            const T dv = Ds[ty + 16 * p][k0 + kk];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc2[p][q] = fma(dv, gb[q], acc2[p][q]);
          }
        }
        __syncthreads();
      }
      T qq = T(0);
#pragma unroll
      for (int p = 0; p < MR; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) qq += acc2[p][q] * dloc[p][q];
      dq[4] = qq;
    }
  }
  // one combined fixed-order reduction of the partial dots
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const T v = warp_sum(dq[m]);
    if (lane == 0) shq[m][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    T v = T(0);
#pragma unroll
    for (int w = 0; w < 8; ++w) v += shq[threadIdx.x][w];
    const int slot = blockIdx.x * gridDim.y + blockIdx.y;
    a.part[((int64_t)slot * a.b + j) * kNQ + threadIdx.x] = (double)v;
  }
  if (a.ctl_mode) {
    // the last CTA of restart j runs its control step (all partials of j are written)
    __shared__ unsigned ticket;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) ticket = atomicAdd(&a.counters[j], 1u);
    __syncthreads();
    const unsigned per = gridDim.x * gridDim.y;
    if (ticket == per - 1) {
      if (threadIdx.x == 0) a.counters[j] = 0u;
      if (threadIdx.x < 32)
        fused_control(a.ctl_mode, const_cast<Ctl&>(a.ctl[j]), a.part, (int)per, a.b, a.r, j, a.P, a.G64fix,
                      nullptr);
    }
  }
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
__global__ void k_rho(const double* __restrict__ G64, int r, int iters, double rho_scale,
                      Ctl* __restrict__ ctl, int set_alpha) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ double sh[32];
  __shared__ PT v[kMaxR], w[kMaxR];
  const int j = blockIdx.x;
  Ctl& c = ctl[j];
  if (!c.active) return;
  PT* Gs = ((size_t)r * r * sizeof(PT) <= 96 * 1024) ? reinterpret_cast<PT*>(smem_raw) : nullptr;
  rho_body<PT>(G64 + (int64_t)j * r * r, r, iters, rho_scale, c, v, w, Gs, sh);
  (void)set_alpha;
}

// ---------------------------------------------------------------------------
// Penalty form control (Sec. 2.1): block start / line search / update.
// prow: row-kernel partials (q layout of EPI_GRAD / EPI_DIR), nrow slots.
// ---------------------------------------------------------------------------
__global__ void k_ctl_pen_start(Ctl* __restrict__ ctl, const double* __restrict__ prow, int nrow,
                                int b, Params P, int is_w_block, int first) {
  __shared__ double sh[32];
  pen_start_body(ctl[blockIdx.x], prow, nrow, b, blockIdx.x, P, is_w_block, first, sh);
}

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

// After UPD (q: 0 pg2, 1 f-const, 2 ss, 3 sy, 4 yy, 5 f(X')-f(Z)).
__global__ void k_ctl_pen_upd(Ctl* __restrict__ ctl, const double* __restrict__ prow, int nrow,
                              int b, Params P, int is_h_block, int last) {
  __shared__ double sh[32];
  pen_upd_body(ctl[blockIdx.x], prow, nrow, b, blockIdx.x, P, is_h_block, last, sh);
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
  Ctl& c = ctl[j];
  const int64_t o = (int64_t)j * r * r;
  const double wah = reduce_slots(pax, nax, b, j, 0, sh);
  const double pg2 = reduce_slots(prow, nrow, b, j, 0, sh);
  const double gwgh = dot_rr(GW + o, GH + o, r, sh);
  double trw = 0.0, trh = 0.0, trwh = 0.0;
  for (int p = threadIdx.x; p < r; p += blockDim.x) {
    trw += GW[o + p * r + p];
    trh += GH[o + p * r + p];
    trwh += WH[o + p * r + p];
  }
  trw = block_sum(trw, sh);
  trh = block_sum(trh, sh);
  trwh = block_sum(trwh, sh);
  if (threadIdx.x != 0) return;
  const double res2 = P.normA2 - 2.0 * wah + gwgh;
  c.fin_res = sqrt(fmax(res2, 0.0) / P.normA2);
  c.fin_f = 0.5 * res2 + 0.5 * c.lam * (trw - 2.0 * trwh + trh);
  c.fin_pg = (c.pg0 > 0.0) ? sqrt(pg2 + c.pgH2) / c.pg0 : 0.0;
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
                 int rho_iters, double rho_scale) {
  const int ntile = (d.r + 63) / 64;
  const int64_t chunk = (d.n + nchunks - 1) / nchunks;
  dim3 grid(nchunks, d.b * ntile * ntile);
  if (tdtype == 0)
    k_gram<double><<<grid, 256, 0, s>>>((const double*)X, (const double*)Y, d.n, d.r, d.b, d.ld, chunk,
                                        ntile, gpart, pair, npairs, ctl, run, G64, (double*)GT, tpair,
                                        lam_shift, counters, nullptr, 0, 1.0);
  else
    k_gram<float><<<grid, 256, 0, s>>>((const float*)X, (const float*)Y, d.n, d.r, d.b, d.ld, chunk,
                                       ntile, gpart, pair, npairs, ctl, run, G64, (float*)GT, tpair,
                                       lam_shift, counters, rho_ctl, rho_iters, rho_scale);
}

static int rowgemm_bm(const Dims& d, int tdtype) {
  if (tdtype == 0) return 32;  // FP64: keeps the operand/D tile and the G tile within 48 KB
  return (d.n + 63) / 64 * ((d.r + 63) / 64) * d.b >= 2 * 152 ? 64 : 32;
}

int rowgemm_slots(const Dims& d, int tdtype) {
  const int bm = rowgemm_bm(d, tdtype);
  return cdiv(d.n, bm) * cdiv(d.r, 64);
}

void launch_rowgemm(int tdtype, int op, int epi, const RowArgs& a, cudaStream_t s) {
  Dims d;
  d.n = a.n; d.r = a.r; d.b = a.b; d.N = a.r * a.b; d.ld = a.ld;
  const int bm = rowgemm_bm(d, tdtype);
  dim3 grid(cdiv(a.n, bm), cdiv(a.r, 64), a.b);
#define RG(T, O, E, M) k_rowgemm<T, O, E, M><<<grid, 256, 0, s>>>(a)
#define RG_M(T, O, E) \
  if (sizeof(T) == 8 || bm == 32) RG(T, O, E, 32); else RG(float, O, E, 64);
#define RG_T(T)                                                   \
  if (epi == EPI_GRAD) {                                          \
    if (op == OP_LOAD) { RG_M(T, OP_LOAD, EPI_GRAD) }             \
    else if (op == OP_ZSTEP) { RG_M(T, OP_ZSTEP, EPI_GRAD) }      \
    else { RG_M(T, OP_UPD, EPI_GRAD) }                            \
  } else {                                                        \
    if (op == OP_LOAD) { RG_M(T, OP_LOAD, EPI_DIR) }              \
    else if (op == OP_ZSTEP) { RG_M(T, OP_ZSTEP, EPI_DIR) }       \
    else { RG_M(T, OP_UPD, EPI_DIR) }                             \
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
                int set_alpha, cudaStream_t s) {
  if (tdtype == 0) {
    size_t sm = (size_t)d.r * d.r * sizeof(double);
    if (sm > 96 * 1024) sm = 0;
    k_rho<double><<<d.b, 256, sm, s>>>(G64, d.r, iters, scale, ctl, set_alpha);
  } else {
    size_t sm = (size_t)d.r * d.r * sizeof(float);
    if (sm > 96 * 1024) sm = 0;
    k_rho<float><<<d.b, 256, sm, s>>>(G64, d.r, iters, scale, ctl, set_alpha);
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

void launch_ctl_pen_start(Ctl* ctl, const double* prow, int nrow, int b, const Params& P, int is_w,
                          int first, cudaStream_t s) {
  k_ctl_pen_start<<<b, 32, 0, s>>>(ctl, prow, nrow, b, P, is_w, first);
}
void launch_ctl_pen_ls(Ctl* ctl, const double* prow, int nrow, const double* pax, int nax, int b,
                       int r, const double* G64fix, const double* DtD, const Params& P, int graph,
                       cudaStream_t s) {
  k_ctl_pen_ls<<<b, 32, 0, s>>>(ctl, prow, nrow, pax, nax, b, r, G64fix, DtD, P, graph);
}
void launch_ctl_pen_upd(Ctl* ctl, const double* prow, int nrow, int b, const Params& P, int is_h,
                        int last, cudaStream_t s) {
  k_ctl_pen_upd<<<b, 32, 0, s>>>(ctl, prow, nrow, b, P, is_h, last);
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
