// Device bodies shared by the per-restart kernels (rowops.cu) and the grouped kernels of
// the uneven batch (batch.cu): fixed-order slot reductions, the FP64 control steps of
// Algorithm 1, the Gram and the row GEMM with its fused epilogues.  The bodies take their
// CTA coordinates as arguments, so one CTA of either launcher runs one work item.
#pragma once

#include <math.h>

#include <type_traits>

#include "common.cuh"
#include "mlp_dev.cuh"
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
template <int NV>
__device__ void reduce_slots_all(const double* part, int nslots, int b, int j, double* out) {
  const int lane = threadIdx.x & 31;
  double acc[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) acc[q] = 0.0;
  int t = lane;
  for (; t + 32 < nslots; t += 64) {
    const double2* r0 = reinterpret_cast<const double2*>(part + ((int64_t)t * b + j) * kNQ);
    const double2* r1 = reinterpret_cast<const double2*>(part + ((int64_t)(t + 32) * b + j) * kNQ);
    double2 a[NV / 2], c[NV / 2];
#pragma unroll
    for (int u = 0; u < NV / 2; ++u) { a[u] = __ldcg(r0 + u); c[u] = __ldcg(r1 + u); }
#pragma unroll
    for (int u = 0; u < NV / 2; ++u) { acc[2 * u] += a[u].x; acc[2 * u + 1] += a[u].y; }
#pragma unroll
    for (int u = 0; u < NV / 2; ++u) { acc[2 * u] += c[u].x; acc[2 * u + 1] += c[u].y; }
  }
  for (; t < nslots; t += 32) {
    const double2* r0 = reinterpret_cast<const double2*>(part + ((int64_t)t * b + j) * kNQ);
#pragma unroll
    for (int u = 0; u < NV / 2; ++u) {
      const double2 a = __ldcg(r0 + u);
      acc[2 * u] += a.x;
      acc[2 * u + 1] += a.y;
    }
  }
#pragma unroll
  for (int q = 0; q < NV; ++q) out[q] = warp_sum(acc[q]);
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
__device__ void rho_body(const double* __restrict__ Gj, int r, int iters, double rho_scale, double rho_shift, Ctl& c,
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
    double rr = rho_scale * (double)rho + rho_shift;  // shift: gamma ||L||_2 of a graph block
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
    const bool stop = c.iters > 0 && (joint <= P.tol * c.pg0 || c.iters >= P.max_iter);
    const bool bad = !stop && !isfinite(joint);
    if (P.ring && P.ring_cap > 0) {  // statistics of the state reached by the last outer iteration
      double* rec = P.ring + ((int64_t)j * P.ring_cap + (c.iters % P.ring_cap)) * kRingVals;
      rec[0] = (double)c.iters;
      rec[1] = c.pg0 > 0.0 ? joint / c.pg0 : 0.0;
      rec[2] = joint;
      rec[3] = c.alpha;
      rec[4] = c.beta;
      rec[5] = (double)c.ls_fail;
      rec[6] = (double)c.mlp_accept;
      rec[7] = (stop || bad) ? 0.0 : 1.0;  // 1: the restart goes on
    }
    if (stop) { c.active = 0; return; }
    if (bad) { c.nan_seen = 1; c.active = 0; return; }
  } else {
    if (first) { c.pgH2 = pg2; return; }  // solve initialisation: H gradient at start
  }
  c.f = 0.0;  // block-relative objective: f(X_0) = 0
  c.F = 0.0;
  hist_reset(c, 0.0);
  c.k = 0;
  c.alpha = 1.0 / c.rho;
  for (int m = 0; m < kNCand; ++m) c.cand_alpha[m] = c.alpha;  // k = 0: every candidate is 1/rho
  c.dsel = 0;
  c.feat_ok = 0;
  c.pg_prev = sqrt(pg2);
  c.last_dec = 0.0;
}

// backtracking from beta = 1 on f(Z + beta D) - f(Z) = beta gd + beta^2/2 q against the
// reference (Alg. 1 line 4); returns beta (0 when no trial is accepted)
__device__ double backtrack(double fZ, double F, double gd, double q, const Params& P, bool* ok) {
  double beta = 1.0;
  for (int t = 0; t < P.max_ls; ++t) {
    const double fz = fZ + beta * gd + 0.5 * beta * beta * q;
    if (fz <= F + P.theta * beta * gd) { *ok = true; return beta; }
    beta *= P.beta_shrink;
  }
  *ok = false;
  return 0.0;
}

// Line search after the D direction (q: 0 gd, 1 dd, 2 f(Z)-f(X_k), 4 <D G, D> when fused):
// f(Z + beta D) - f(Z) = beta gd + beta^2/2 q, q = <D (H H^T + lambda I), D> + gamma <D, L D>.
// nc = 2 (learned controller): candidate 0 is the proposal, accepted only at beta = 1, else
// the plain BB direction (candidate 1) with ordinary backtracking.  The lean learned step
// (controller 3) has one candidate, the proposal, with ordinary backtracking.  nc = 9 (record mode):
// every candidate multiplier is line-searched, the best accepted decrease is recorded as
// the training label, and the plain BB candidate (index 4) is followed.
__device__ void pen_ls_body(Ctl& c, const double* prow, int nrow, const double* pax, int nax, int b, int r,
                            int j, const double* G64fix, const double* DtD, const Params& P, int graph,
                            double* sh, int nc = 1) {
  if (!c.active) return;
  double qs[kNQ];
  if (nc > 2) reduce_slots_all<kNQ>(prow, nrow, b, j, qs);
  else reduce_slots_all<8>(prow, nrow, b, j, qs);
  const double gd = qs[0], dd = qs[1], dzw = qs[2];
  const double qg = DtD ? dot_rr(DtD + (int64_t)j * r * r, G64fix + (int64_t)j * r * r, r, sh) + c.lam * dd
                        : qs[4];
  double dld = 0.0;
  if (graph) dld = reduce_slots(pax, nax, b, j, 0, sh);
  if ((threadIdx.x & 31) != 0) return;
  const double q = qg + P.gamma * dld;
  c.fZ = c.f + dzw;
  if (c.k > 0) c.F = reference(c, P);
  double beta = 0.0;
  bool ok = false;
  c.dsel = 0;
  if (nc == 1) {
    c.gd = gd;
    c.q = q;
    beta = backtrack(c.fZ, c.F, gd, q, P, &ok);
    if (P.controller == 3 && c.feat_ok) {  // lean learned step: the proposal, backtracked
      c.mlp_tried++;
      if (ok && beta == 1.0) c.mlp_accept++;
    }
  } else if (nc == 2) {
    // proposal: Armijo test at beta = 1 only
    const double fz1 = c.fZ + gd + 0.5 * q;
    c.mlp_tried++;
    if (fz1 <= c.F + P.theta * gd) {
      beta = 1.0;
      ok = true;
      c.mlp_accept++;
      c.gd = gd;
      c.q = q;
    } else {
      const double gd1 = qs[5], q1 = qs[7];
      c.dsel = 1;
      c.gd = gd1;
      c.q = q1;
      beta = backtrack(c.fZ, c.F, gd1, q1, P, &ok);
    }
  } else {
    // record mode: label = candidate with the best accepted decrease
    int best = 4;
    double best_dec = 0.0;
    double beta4 = 0.0;
    bool ok4 = false;
    for (int m = 0; m < nc; ++m) {
      const double gdm = m == 0 ? gd : qs[5 + 3 * (m - 1)];
      const double qm = m == 0 ? q : qs[5 + 3 * (m - 1) + 2];
      bool okm = false;
      const double bm = backtrack(c.fZ, c.F, gdm, qm, P, &okm);
      const double dec = okm ? bm * gdm + 0.5 * bm * bm * qm : 0.0;
      if (dec < best_dec) { best_dec = dec; best = m; }
      if (m == 4) { beta4 = bm; ok4 = okm; c.gd = gdm; c.q = qm; }
    }
    if (c.feat_ok && P.rec_feat) {
      const int idx = atomicAdd(P.rec_count, 1);
      if (idx < P.rec_cap) {
        for (int u = 0; u < kMlpIn; ++u) P.rec_feat[(int64_t)idx * kMlpIn + u] = c.feat[u];
        P.rec_targ[idx] = 0.5f * (float)(best - 4);  // log2 of the best multiplier
      }
    }
    beta = beta4;
    ok = ok4;
  }
  if (!ok) { beta = 0.0; c.ls_fail++; }
  if (!isfinite(c.fZ) || !isfinite(q) || !isfinite(gd)) { c.nan_seen = 1; c.active = 0; }
  c.beta = beta;
  c.phibeta = P.phi * beta;
}

// After the relaxed update (q: 0 pg2, 2 ss, 3 sy, 4 yy, 5 f(X')-f(Z), 6 zero entries).
// One warp: BB step of the next iteration and, with a controller, its candidates.
// Controller features (scale free): ln(BB1 rho), ln(BB2 rho), ||P grad|| ratio, objective
// decrease ratio, active-set fraction.
__device__ void pen_upd_body(Ctl& c, const double* prow, int nrow, int b, int j, const Params& P, int is_h_block,
                             int last, double* sh, int nc = 1) {
  if (!c.active) return;
  double qs[8];
  reduce_slots_all<8>(prow, nrow, b, j, qs);
  const double pg2 = qs[0], ss = qs[2], sy = qs[3], yy = qs[4], dwz = qs[5], zeros = qs[6];
  const double f_old = c.f;
  const double f_new = c.fZ + dwz;
  double alpha_bb;  // Alg. 1 line 3 / Eq. (2.10) with the 1/rho fallback when <S,Y> <= 0
  if (!(sy > 0.0)) alpha_bb = 1.0 / c.rho;
  else alpha_bb = (P.bb == 0) ? ss / sy : sy / yy;
  alpha_bb = fmin(P.alpha_max, fmax(P.alpha_min, alpha_bb));
  if (nc > 1) {
    // The features feed an FP32 network, so they are formed in FP32 from the FP64 sums (the
    // FP64 units of this GPU are slow, and this runs on one warp at the end of the launch).
    float phi[kMlpIn];
    const float rho = (float)c.rho;
    const float ssf = (float)ss, syf = (float)sy, yyf = (float)yy;
    const float bb1r = syf > 0.f ? ssf * rho / syf : 1.f;  // BB1 rho, BB2 rho (1 without curvature)
    const float bb2r = (syf > 0.f && yyf > 0.f) ? syf * rho / yyf : 1.f;
    const float pgf = sqrtf((float)pg2);
    const double dec = f_old - f_new;
    const float prev = (float)c.pg_prev;
    phi[0] = logf(fminf(fmaxf(bb1r, 1e-6f), 1e6f));
    phi[1] = logf(fminf(fmaxf(bb2r, 1e-6f), 1e6f));
    phi[2] = prev > 0.f ? fminf(pgf / prev, 10.f) : 1.f;
    phi[3] = fminf(fmaxf((float)dec / fmaxf(fabsf((float)c.last_dec), 1e-37f), -10.f), 10.f);
    phi[4] = (float)zeros / (float)P.nr;
    const double pg = (double)pgf;
    float mult = 1.f;
    // rollout branch (controller 4): this step's index counted over the whole solve
    const bool branch = P.controller == 4 &&
                        (int64_t)c.iters * 2 * P.inner + (int64_t)is_h_block * P.inner + c.k == P.branch_step;
    if ((nc == 2 || nc == 3) && P.controller != 4) mult = mlp_multiplier(P.mlp_w, phi);  // all lanes
    if ((threadIdx.x & 31) == 0) {
      for (int u = 0; u < kMlpIn; ++u) c.feat[u] = phi[u];
      c.feat_ok = 1;
      c.pg_prev = pg;
      c.last_dec = dec;
      if (nc == 2) {
        c.mlp_mult = mult;
        c.cand_alpha[0] = fmin(P.alpha_max, fmax(P.alpha_min, (double)mult * alpha_bb));
        c.cand_alpha[1] = alpha_bb;
      } else if (nc == 3 && P.controller == 4) {
        // rollout branch: candidate j % 9 scales the next step by 2^((c - 4) / 2); the group's
        // plain candidate records the features of the branch point, tagged with the group
        if (branch) {
          const int cand = j % kNCand;
          alpha_bb = fmin(P.alpha_max, fmax(P.alpha_min, exp2(0.5 * (cand - 4)) * alpha_bb));
          if (cand == 4 && P.rec_feat) {
            const int idx = atomicAdd(P.rec_count, 1);
            if (idx < P.rec_cap) {
              for (int u = 0; u < kMlpIn; ++u) P.rec_feat[(int64_t)idx * kMlpIn + u] = phi[u];
              P.rec_targ[idx] = (float)(j / kNCand);
            }
          }
        }
      } else if (nc == 3) {  // lean learned step: the next D uses the proposal directly
        c.mlp_mult = mult;
        alpha_bb = fmin(P.alpha_max, fmax(P.alpha_min, (double)mult * alpha_bb));
      } else {
        for (int m = 0; m < kNCand; ++m)
          c.cand_alpha[m] = fmin(P.alpha_max, fmax(P.alpha_min, exp2(0.5 * (m - 4)) * alpha_bb));
      }
    }
  }
  if ((threadIdx.x & 31) != 0) return;
  c.ss = ss; c.sy = sy; c.yy = yy;
  c.f = f_new;
  hist_push(c, c.f, P.memory);
  c.k++;
  c.alpha = alpha_bb;
  if (is_h_block) {
    c.pgH2 = pg2;
    if (last) c.iters++;
  } else if (last) {
    c.iters++;  // naive variant: the W block is the whole outer iteration
  }
  if (!isfinite(c.f)) { c.nan_seen = 1; c.active = 0; }
}

// Final per-restart statistics of the penalty form: pax q0 = <W, A Ht>, prow q0 = ||P grad_W||^2
// at the final point; GW = W^T W, GH = Ht^T Ht, WH = W^T Ht of this restart.
__device__ void final_pen_body(Ctl& c, const double* pax, int nax, const double* prow, int nrow,
                               const double* GW, const double* GH, const double* WH, int b, int j,
                               int r, double normA2, double* sh) {
  const double wah = reduce_slots(pax, nax, b, j, 0, sh);
  const double pg2 = reduce_slots(prow, nrow, b, j, 0, sh);
  const double gwgh = dot_rr(GW, GH, r, sh);
  double trw = 0.0, trh = 0.0, trwh = 0.0;
  for (int p = threadIdx.x; p < r; p += blockDim.x) {
    trw += GW[p * r + p];
    trh += GH[p * r + p];
    trwh += WH[p * r + p];
  }
  trw = block_sum(trw, sh);
  trh = block_sum(trh, sh);
  trwh = block_sum(trwh, sh);
  if (threadIdx.x != 0) return;
  const double res2 = normA2 - 2.0 * wah + gwgh;
  c.fin_res = sqrt(fmax(res2, 0.0) / normA2);
  c.fin_f = 0.5 * res2 + 0.5 * c.lam * (trw - 2.0 * trwh + trh);
  c.fin_pg = (c.pg0 > 0.0) ? sqrt(pg2 + c.pgH2) / c.pg0 : 0.0;
}

// Fused control after a producing kernel: modes of RowArgs::ctl_mode.
__device__ void fused_control(int mode, Ctl& c, const double* part, int nslots, int b, int r, int j,
                              const Params& P, const double* G64fix, double* sh, int nc) {
  // candidates of the solve (3: the lean learned step, one candidate)
  const int pc = P.controller == 1 ? 2 : (P.controller == 2 ? kNCand : (P.controller >= 3 ? 3 : 1));
  switch (mode) {
    case CTL_START_W: pen_start_body(c, part, nslots, b, j, P, 1, 0, sh); break;
    case CTL_START_H: pen_start_body(c, part, nslots, b, j, P, 0, 0, sh); break;
    case CTL_START_INIT: pen_start_body(c, part, nslots, b, j, P, 0, 1, sh); break;
    case CTL_LS: pen_ls_body(c, part, nslots, nullptr, 0, b, r, j, G64fix, nullptr, P, 0, sh, nc); break;
    case CTL_UPD_W: pen_upd_body(c, part, nslots, b, j, P, 0, 0, sh, pc); break;
    case CTL_UPD_H: pen_upd_body(c, part, nslots, b, j, P, 1, 0, sh, pc); break;
    case CTL_UPD_H_LAST: pen_upd_body(c, part, nslots, b, j, P, 1, 1, sh, pc); break;
    case CTL_UPD_W_LAST_NAIVE: pen_upd_body(c, part, nslots, b, j, P, 0, 1, sh, pc); break;
    default: break;
  }
}


// ------------------------------------------------------------------------------
// Gram X_j^T Y_j per restart j.  CTA (chunk, tile): a TW x TW output tile over a chunk of
// rows (16x16 threads, TW/16 x TW/16 micro tiles; TW = 64, or 32 for r <= 32), RS rows staged
// per round with the next round's loads in flight, X staged once when X and Y are the same
// slice; FP64 partial written to gpart.  The last CTA of each tile (arrival counter) sums the
// partials in chunk order and writes G64 (and the factor-type copy with lam_shift * I on the
// diagonal when pair == tpair): a fixed-order, deterministic two-stage reduction in one launch.
// ------------------------------------------------------------------------------
// CTA coordinates are arguments: `cidx` of `nch` row chunks, `jt` = restart * ntile^2 + tile.
template <typename T, int TW = 64, int RS = 32>
__device__ __forceinline__ void
gram_body(const T* __restrict__ X, const T* __restrict__ Y, int64_t n, int r, int b, int64_t ld,
          int64_t chunk, int ntile, double* __restrict__ gpart, int pair, int npairs,
          const Ctl* __restrict__ ctl, const int* run, double* __restrict__ G64, T* __restrict__ GT,
          int tpair, double lam_shift, unsigned* __restrict__ counters, Ctl* __restrict__ rho_ctl,
          int rho_iters, double rho_scale, double rho_shift, int cidx, int nch, int jt) {
  constexpr int MT = TW / 16;             // micro tile
  constexpr int LD = RS * TW / 256;       // staged values per thread and operand
  static_assert(RS * TW % 256 == 0, "staging split over 256 threads");
  const int j = jt / (ntile * ntile);
  const int t = jt % (ntile * ntile);
  const int ti = t / ntile, tj = t % ntile;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t i_begin = (int64_t)cidx * chunk;
  const int64_t i_end = min(n, i_begin + chunk);
  __shared__ T Xs[RS][TW + 1];
  __shared__ T Ys[RS][TW + 1];
  __shared__ unsigned ticket;
  T acc[MT][MT];
#pragma unroll
  for (int a = 0; a < MT; ++a)
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[a][c] = T(0);
  const bool skip = (run && *run == 0) || (ctl && !ctl[j].active);
  if (!skip) {
    const int64_t cx = (int64_t)j * r + ti * TW;
    const int64_t cy = (int64_t)j * r + tj * TW;
    const int wx = min(TW, r - ti * TW), wy = min(TW, r - tj * TW);
    const bool same = (X == Y) && (ti == tj);  // X^T X on a diagonal tile: one operand
    T xv_[LD], yv_[LD];
    auto fetch = [&](int64_t i0) {
#pragma unroll
      for (int m = 0; m < LD; ++m) {
        const int e = threadIdx.x + 256 * m;
        const int rr = e / TW, cc = e % TW;
        const int64_t i = i0 + rr;
        xv_[m] = (i < i_end && cc < wx) ? X[i * ld + cx + cc] : T(0);
        if (!same) yv_[m] = (i < i_end && cc < wy) ? Y[i * ld + cy + cc] : T(0);
      }
    };
    if (i_begin < i_end) fetch(i_begin);
    for (int64_t i0 = i_begin; i0 < i_end; i0 += RS) {
#pragma unroll
      for (int m = 0; m < LD; ++m) {
        const int e = threadIdx.x + 256 * m;
        Xs[e / TW][e % TW] = xv_[m];
        if (!same) Ys[e / TW][e % TW] = yv_[m];
      }
      __syncthreads();
      if (i0 + RS < i_end) fetch(i0 + RS);  // the next round's loads fly during this one
      const T(*Yr)[TW + 1] = same ? Xs : Ys;
#pragma unroll 8
      for (int rr = 0; rr < RS; ++rr) {
        T xa[MT], yb[MT];
#pragma unroll
        for (int a = 0; a < MT; ++a) xa[a] = Xs[rr][ty + 16 * a];
#pragma unroll
        for (int c = 0; c < MT; ++c) yb[c] = Yr[rr][tx + 16 * c];
#pragma unroll
        for (int a = 0; a < MT; ++a)
#pragma unroll
          for (int c = 0; c < MT; ++c) acc[a][c] = fma(xa[a], yb[c], acc[a][c]);
      }
      __syncthreads();
    }
  }
  const int64_t rr2 = (int64_t)r * r;
  const int64_t tile_base = ((int64_t)pair * b + j) * rr2;   // offset inside one chunk slab
  const int64_t slab = (int64_t)npairs * b * rr2;
  T* gp = reinterpret_cast<T*>(gpart);  // chunk partials in the working type
  T* out = gp + (int64_t)cidx * slab + tile_base;
#pragma unroll
  for (int a = 0; a < MT; ++a) {
    const int p = ti * TW + ty + 16 * a;
    if (p >= r) continue;
#pragma unroll
    for (int c = 0; c < MT; ++c) {
      const int q = tj * TW + tx + 16 * c;
      if (q < r) out[(int64_t)p * r + q] = acc[a][c];
    }
  }
  __threadfence();
  __syncthreads();
  const int tile_id = ((pair * b + j) * ntile + ti) * ntile + tj;
  if (threadIdx.x == 0) ticket = atomicAdd(&counters[tile_id], 1u);
  __syncthreads();
  if (ticket == nch - 1) {
    // last CTA of this tile: fixed-order sum over the chunks
    // each thread owns NE tile entries and sums them over the chunks in chunk order, with
    // the loads of several chunks in flight together
    // nch: chunks of this tile
    constexpr int NE = TW * TW / 256;
    constexpr int UF = NE >= 16 ? 2 : 4;  // chunks in flight (registers: NE loads each)
    int64_t off_[NE];
    bool ok_[NE];
    T sacc[NE];
#pragma unroll
    for (int u = 0; u < NE; ++u) {
      const int e = threadIdx.x + 256 * u;
      const int p = ti * TW + e / TW, q = tj * TW + e % TW;
      ok_[u] = (p < r && q < r);
      off_[u] = tile_base + (int64_t)(ok_[u] ? p : 0) * r + (ok_[u] ? q : 0);
      sacc[u] = T(0);
    }
#pragma unroll UF
    for (int c = 0; c < nch; ++c) {
      T v[NE];
#pragma unroll
      for (int u = 0; u < NE; ++u) v[u] = ok_[u] ? __ldcg(gp + (int64_t)c * slab + off_[u]) : T(0);
#pragma unroll
      for (int u = 0; u < NE; ++u) sacc[u] += v[u];
    }
#pragma unroll
    for (int u = 0; u < NE; ++u) {
      if (!ok_[u]) continue;
      const int e = threadIdx.x + 256 * u;
      const int p = ti * TW + e / TW, q = tj * TW + e % TW;
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
      rho_body<T>(G64 + tile_base, r, rho_iters, rho_scale, rho_shift, rho_ctl[j], vv, ww, Gsr, shr);
    }
  }
  __syncthreads();  // no early return: a CTA may run several items
}

// ------------------------------------------------------------------------------
// Row GEMM with fused Algorithm-1 epilogues.
// ------------------------------------------------------------------------------
// CTA coordinates are arguments: restart j, row tile bx, column tile by of gy, `per` CTAs
// per restart (the partial slot of the CTA is bx * gy + by).
template <typename T, int OP, int EPI, int BM, int NC>
__device__ __forceinline__ void rowgemm_body(const RowArgs& a, int j, int bx, int by, int gy, unsigned per) {
  constexpr int MR = BM / 16;  // rows per thread
  constexpr int KC = sizeof(T) == 4 ? 64 : 32;  // K columns staged per round
  constexpr int XS_ELEMS = BM * (KC + 1);
  constexpr int DS_ELEMS = (EPI == EPI_DIR) ? BM * 65 : 1;
  constexpr int U_ELEMS = XS_ELEMS > DS_ELEMS ? XS_ELEMS : DS_ELEMS;
  constexpr int NV = NC > 2 ? 32 : 8;  // partial values written per CTA (NC = 2 uses 8)
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t row0 = (int64_t)bx * BM;
  const int col0 = by * 64;  // within restart
  const int r = a.r;
  const int64_t ld = a.ld;
  const int64_t jc = (int64_t)j * r;
  __shared__ T shq[NV][8];
  __shared__ __align__(16) T ubuf[U_ELEMS];   // operand tile, later the D tile
  __shared__ T Gs[KC][64 + 1];
  T (*Xs)[KC + 1] = reinterpret_cast<T (*)[KC + 1]>(ubuf);
  T (*Ds)[65] = reinterpret_cast<T (*)[65]>(ubuf);
  const Ctl& cj = a.ctl[j];
  const bool live = cj.active && !(a.run && *a.run == 0);
  T dq[NV];
#pragma unroll
  for (int m = 0; m < NV; ++m) dq[m] = T(0);
  if (live) {
    const T* G = (const T*)a.G + (int64_t)j * r * r;
    const T inv_rho = (T)(1.0 / cj.rho);
    const T pb = (T)cj.phibeta;
    const T* X = (const T*)a.X;
    const T* gin = (const T*)a.g_in;
    const T* Zin = (const T*)a.Zin;
    const T* Din = (const T*)((OP == OP_UPD && cj.dsel) ? a.Din2 : a.Din);
    T alph[NC];
#pragma unroll
    for (int m = 0; m < NC; ++m) alph[m] = (T)(NC == 1 ? cj.alpha : cj.cand_alpha[m]);
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
    const T* B = (const T*)a.B;
    const T* LX = (const T*)a.LX;
    const T gam = (T)a.gamma;
    T gl[MR][4], xl[MR][4];  // gradient and operand of the thread's elements
    // With r <= KC the operand tile of this CTA's rows is still in shared memory.
    const bool xs_ok = r <= KC && col0 == 0;
#pragma unroll
    for (int p = 0; p < MR; ++p) {
      const int64_t i = row0 + ty + 16 * p;
      // the row's loads first: the stores below may alias inputs (Xout / Xold), so
      // keeping them apart lets all four elements' loads be in flight together
      bool vq[4];
      int64_t iq[4];
      T xq[4], bq[4], lq[4], o0[4], o1[4], o2[4], o3[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = col0 + tx + 16 * q;
        vq[q] = i < a.n && c < r;
        iq[q] = i * ld + jc + c;
        xq[q] = bq[q] = lq[q] = o0[q] = o1[q] = o2[q] = o3[q] = T(0);
        if (!vq[q]) continue;
        const int64_t idx = iq[q];
        xq[q] = xs_ok ? Xs[ty + 16 * p][c] : operand(i, jc + c);
        bq[q] = B[idx];
        if (LX) lq[q] = LX[idx];
        if (EPI == EPI_GRAD) {
          if (a.Xold) { o0[q] = ((const T*)a.Xold)[idx]; o1[q] = ((const T*)a.gold)[idx]; }
          if (a.Zold) { o2[q] = ((const T*)a.Zold)[idx]; o3[q] = ((const T*)a.gZold)[idx]; }
        } else if (a.Wcur) {
          o0[q] = ((const T*)a.Wcur)[idx];
          o1[q] = ((const T*)a.gWcur)[idx];
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        gl[p][q] = T(0);
        xl[p][q] = T(0);
        if (!vq[q]) continue;
        const int64_t idx = iq[q];
        const T xv = xq[q];
        T g = acc[p][q] - bq[q];
        if (LX) g += gam * lq[q];
        gl[p][q] = g;
        xl[p][q] = xv;
        if (EPI == EPI_GRAD) {
          const T pgv = xv > T(0) ? g : (g < T(0) ? g : T(0));
          dq[0] += pgv * pgv;                              // ||P grad||^2
          dq[1] += T(0.5) * (g - bq[q]) * xv;               // f - const (quadratic block)
          if (a.Xold) {
            const T sv = xv - o0[q];
            const T yv = g - o1[q];
            dq[2] += sv * sv;
            dq[3] += sv * yv;
            dq[4] += yv * yv;
          }
          if (a.Zold) dq[5] += T(0.5) * (xv - o2[q]) * (g + o3[q]);  // f(X') - f(Z), trapezoid (exact)
          if (xv == T(0)) dq[6] += T(1);                    // active (zero) entries
          if (a.gout) ((T*)a.gout)[idx] = g;
          if (a.Xout) ((T*)a.Xout)[idx] = xv;
        } else {  // EPI_DIR
          if (a.Xout) ((T*)a.Xout)[idx] = xv;
          if (a.gZout) ((T*)a.gZout)[idx] = g;
          if (a.Wcur) dq[2] += T(0.5) * (xv - o0[q]) * (g + o1[q]);  // f(Z) - f(W), trapezoid (exact)
#pragma unroll
          for (int m = 0; m < NC; ++m) {
            T d = xv - alph[m] * g;
            d = (d > T(0) ? d : T(0)) - xv;
            if (m == a.dstore) ((T*)a.Dout)[idx] = d;
            if (NC == 2 && m == 1) ((T*)a.D2out)[idx] = d;
            const int base = m == 0 ? 0 : 5 + 3 * (m - 1);
            dq[base] += g * d;                              // <grad f(Z), D_m>
            dq[base + 1] += d * d;                          // ||D_m||^2
            if (m == 0 && LX) dq[3] += d * lq[q];           // <D, L Z> (direct, graph)
          }
        }
      }
    }
    __syncthreads();  // the operand tile (read above) and the D tile below share memory
    if (EPI == EPI_DIR && a.want_q) {
      // <D_m G, D_m> of each candidate's line-search quadratic (restart = one column tile)
#pragma unroll 1
      for (int m = 0; m < NC; ++m) {
#pragma unroll
        for (int p = 0; p < MR; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            T d = xl[p][q] - alph[m] * gl[p][q];
            d = (d > T(0) ? d : T(0)) - xl[p][q];
            const int c = col0 + tx + 16 * q;
            const int64_t i = row0 + ty + 16 * p;
            Ds[ty + 16 * p][tx + 16 * q] = (i < a.n && c < r) ? d : T(0);
          }
        __syncthreads();
        T acc2[MR][4];
#pragma unroll
        for (int p = 0; p < MR; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc2[p][q] = T(0);
        for (int k0 = 0; k0 < r; k0 += KC) {
          if (!xs_ok) {  // else G (r <= KC) is still in shared memory from the first product
            constexpr int NG = KC * 64 / 256;
            T gv_[NG];
#pragma unroll
            for (int u = 0; u < NG; ++u) {
              const int e = threadIdx.x + 256 * u;
              const int gk = e >> 6, gc = e & 63;
              gv_[u] = (k0 + gk < r && gc < r) ? G[(int64_t)(k0 + gk) * r + gc] : T(0);
            }
#pragma unroll
            for (int u = 0; u < NG; ++u) {
              const int e = threadIdx.x + 256 * u;
              Gs[e >> 6][e & 63] = gv_[u];
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
          for (int q = 0; q < 4; ++q) qq += acc2[p][q] * Ds[ty + 16 * p][tx + 16 * q];
        dq[m == 0 ? 4 : 5 + 3 * (m - 1) + 2] += qq;
        __syncthreads();
      }
    }
  }
  // one combined fixed-order reduction of the partial dots
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int m = 0; m < NV; ++m) {
    const T v = warp_sum(dq[m]);
    if (lane == 0) shq[m][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    T v = T(0);
#pragma unroll
    for (int w = 0; w < 8; ++w) v += shq[threadIdx.x][w];
    const int slot = bx * gy + by;
    a.part[((int64_t)slot * a.b + j) * kNQ + threadIdx.x] = (double)v;
  }
  if (a.ctl_mode) {
    // the last CTA of restart j runs its control step (all partials of j are written)
    __shared__ unsigned ticket;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) ticket = atomicAdd(&a.counters[j], 1u);
    __syncthreads();
        if (ticket == per - 1) {
      if (threadIdx.x == 0) a.counters[j] = 0u;
      if (threadIdx.x < 32)
        fused_control(a.ctl_mode, const_cast<Ctl&>(a.ctl[j]), a.part, (int)per, a.b, a.r, j, a.P, a.G64fix,
                      nullptr, NC);
    }
  }
}

// ------------------------------------------------------------------------------
// Row GEMM for ranks r <= 32 through shared-memory tiles, with the same fused epilogues
// and partial layout as rowgemm_body.  A CTA owns TR consecutive rows of restart j:
//   1. the operand tile (X, Z = Proj[X - g/rho] or X' = Proj[Z + phi beta D]) is staged
//      with element-contiguous (coalesced) loads; B and the inputs that the epilogue
//      reads again are kept in registers,
//   2. the row product X G: TPR threads per row, each CPT columns, G (stride 32, zero
//      padded) read as 16-byte shared-memory broadcasts,
//   3. the elementwise epilogue in the same element order as step 1 (coalesced), with
//      D of each candidate staged for
//   4. <D G, D> by a second row product.
// The body has no early return and ends with a barrier.  sm: dynamic shared memory of
// rowtile_smem bytes.
// ------------------------------------------------------------------------------
template <typename T>
struct TileCfg {
  static constexpr int TR = sizeof(T) == 4 ? 128 : 64;  // rows per tile
  static constexpr int TPR = 256 / TR;                   // threads per row in the row products
  static constexpr int CPT = 32 / TPR;                   // columns per thread
  static constexpr int RS = 33;                          // tile row stride (odd: conflict free)
  static constexpr int EPT = TR * 32 / 256;              // elements per thread (r = 32)
};

template <typename T>
__host__ __device__ inline size_t rowtile_smem(int ntile) {
  return ((size_t)ntile * TileCfg<T>::TR * TileCfg<T>::RS + 32 * 32) * sizeof(T);
}

// y[u] = (row `row` of src) G[:, part*CPT + u], G (stride 32) read as 16-byte broadcasts
template <typename T>
__device__ __forceinline__ void tile_rowprod(const T* __restrict__ src, const T* __restrict__ Gs, int r, int row,
                                             int part, T* y) {
  using C = TileCfg<T>;
  using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  constexpr int W = 16 / sizeof(T);  // elements per vector
  constexpr int NVEC = C::CPT / W;
#pragma unroll
  for (int u = 0; u < C::CPT; ++u) y[u] = T(0);
  const T* xr = src + row * C::RS;
  const V* gc = reinterpret_cast<const V*>(Gs + part * C::CPT);
#pragma unroll 2
  for (int k = 0; k < r; ++k) {
    const T x0 = xr[k];
#pragma unroll
    for (int v = 0; v < NVEC; ++v) {
      const V g0 = gc[(k * 32) / W + v];
      const T* a0 = reinterpret_cast<const T*>(&g0);
#pragma unroll
      for (int w = 0; w < W; ++w) y[v * W + w] = fma(x0, a0[w], y[v * W + w]);
    }
  }
}

template <typename T, int OP, int EPI, int NC>
__device__ __forceinline__ void rowtile_body(const RowArgs& a, int j, int tile, unsigned per, T* sm) {
  using C = TileCfg<T>;
  constexpr int NV = 8;
  static_assert(NC <= 2, "tile row body: at most two candidates");
  const int r = a.r;
  const int64_t ld = a.ld;
  const int64_t jc = (int64_t)j * r;
  T* xs = sm;
  T* ys = xs + C::TR * C::RS;
  T* dsm = ys + C::TR * C::RS;                       // NC direction tiles (EPI_DIR)
  T* Gs = dsm + (EPI == EPI_DIR ? NC : 0) * C::TR * C::RS;
  __shared__ T shq[NV][8];
  __shared__ unsigned ticket;
  const Ctl& cj = a.ctl[j];
  const bool live = cj.active && !(a.run && *a.run == 0);
  T dq[NV];
#pragma unroll
  for (int m = 0; m < NV; ++m) dq[m] = T(0);
  if (live) {
    const int tid = threadIdx.x;
    const int64_t row0 = (int64_t)tile * C::TR;
    const int rows = (int)(a.n - row0 < C::TR ? a.n - row0 : C::TR);
    const int E = rows * r;
    const float inv_r = 1.0f / (float)r;
    const T* G = (const T*)a.G + (int64_t)j * r * r;
    for (int e = tid; e < 32 * 32; e += 256) {
      const int k = e >> 5, c = e & 31;
      Gs[e] = (k < r && c < r) ? G[k * r + c] : T(0);
    }
    const T inv_rho = (T)(1.0 / cj.rho);
    const T pb = (T)cj.phibeta;
    const T* X = (const T*)a.X;
    const T* gin = (const T*)a.g_in;
    const T* Zin = (const T*)a.Zin;
    const T* Din = (const T*)((OP == OP_UPD && cj.dsel) ? a.Din2 : a.Din);
    const T* B = (const T*)a.B;
    // inputs of step 1 that step 3 reads again (same buffers)
    const bool w_is_x = OP == OP_ZSTEP && a.Wcur == a.X && a.gWcur == a.g_in;
    const bool zold_is_z = OP == OP_UPD && a.Zold == a.Zin;
    T in0[C::EPT], in1[C::EPT], bq[C::EPT];
    // EPI_GRAD: the epilogue's other inputs (S, Y and increment terms) are loaded here too,
    // so that every load of the item is in flight in one round trip
    constexpr int EP = EPI == EPI_GRAD ? C::EPT : 1;
    T p0[EP], p1[EP], p2[EP];
    const bool pre_old = EPI == EPI_GRAD && a.Xold != nullptr;
    const bool pre_z = EPI == EPI_GRAD && a.Zold != nullptr;
    // 1. operand tile (and B, so that the epilogue does not wait for it)
#pragma unroll
    for (int m = 0; m < C::EPT; ++m) {
      const int e = tid + 256 * m;
      in0[m] = in1[m] = bq[m] = T(0);
      if (EPI == EPI_GRAD) p0[m % EP] = p1[m % EP] = p2[m % EP] = T(0);
      if (e < E) {
        const int row = (int)(((float)e + 0.5f) * inv_r);  // exact for e < 2^12, r <= 32
        const int col = e - row * r;
        const int64_t q = (row0 + row) * ld + jc + col;
        bq[m] = B[q];
        if (EPI == EPI_GRAD) {
          if (pre_old) { p0[m % EP] = ((const T*)a.Xold)[q]; p1[m % EP] = ((const T*)a.gold)[q]; }
          if (pre_z) p2[m % EP] = ((const T*)a.gZold)[q];
        }
        T v;
        if (OP == OP_LOAD) {
          v = X[q];
        } else if (OP == OP_ZSTEP) {
          const T x = X[q], gi = gin[q];
          const T t = x - gi * inv_rho;
          v = t > T(0) ? t : T(0);
          in0[m] = x;
          in1[m] = gi;
        } else {
          const T z = Zin[q];
          const T t = z + pb * Din[q];
          v = t > T(0) ? t : T(0);
          in0[m] = z;
        }
        xs[row * C::RS + col] = v;
      }
    }
    __syncthreads();
    // 2. Y = X G
    const int prow = tid % C::TR, part = tid / C::TR;
    if (part * C::CPT < r && prow < rows) {
      T y[C::CPT];
      tile_rowprod<T>(xs, Gs, r, prow, part, y);
#pragma unroll
      for (int u = 0; u < C::CPT; ++u)
        if (part * C::CPT + u < r) ys[prow * C::RS + part * C::CPT + u] = y[u];
    }
    __syncthreads();
    // 3. elementwise epilogue
    T alph[NC];
#pragma unroll
    for (int m = 0; m < NC; ++m) alph[m] = (T)(NC == 1 ? cj.alpha : cj.cand_alpha[m]);
#pragma unroll
    for (int m = 0; m < C::EPT; ++m) {
      const int e = tid + 256 * m;
      if (e >= E) continue;
      const int row = (int)(((float)e + 0.5f) * inv_r);
      const int col = e - row * r;
      const int64_t q = (row0 + row) * ld + jc + col;
      const int se = row * C::RS + col;
      const T xv = xs[se];
      const T g = ys[se] - bq[m];
      if (EPI == EPI_GRAD) {
        const T pgv = xv > T(0) ? g : (g < T(0) ? g : T(0));
        dq[0] += pgv * pgv;
        dq[1] += T(0.5) * (g - bq[m]) * xv;
        if (pre_old) {
          const T sv = xv - p0[m % EP];
          const T yv = g - p1[m % EP];
          dq[2] += sv * sv;
          dq[3] += sv * yv;
          dq[4] += yv * yv;
        }
        if (pre_z) {
          const T zo = zold_is_z ? in0[m] : ((const T*)a.Zold)[q];
          dq[5] += T(0.5) * (xv - zo) * (g + p2[m % EP]);
        }
        if (xv == T(0)) dq[6] += T(1);
        if (a.gout) ((T*)a.gout)[q] = g;
        if (a.Xout) ((T*)a.Xout)[q] = xv;
      } else {  // EPI_DIR
        if (a.Xout) ((T*)a.Xout)[q] = xv;
        if (a.gZout) ((T*)a.gZout)[q] = g;
        if (a.Wcur) {
          const T wv = w_is_x ? in0[m] : ((const T*)a.Wcur)[q];
          const T gw = w_is_x ? in1[m] : ((const T*)a.gWcur)[q];
          dq[2] += T(0.5) * (xv - wv) * (g + gw);
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          T d = xv - alph[c] * g;
          d = (d > T(0) ? d : T(0)) - xv;
          if (c == a.dstore) ((T*)a.Dout)[q] = d;
          if (NC == 2 && c == 1) ((T*)a.D2out)[q] = d;
          const int base = c == 0 ? 0 : 5;
          dq[base] += g * d;
          dq[base + 1] += d * d;
          dsm[c * C::TR * C::RS + se] = d;
        }
      }
    }
    // 4. <D_c G, D_c>
    if (EPI == EPI_DIR && a.want_q) {
      __syncthreads();
      if (part * C::CPT < r && prow < rows) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const T* dt = dsm + c * C::TR * C::RS;
          T y[C::CPT];
          tile_rowprod<T>(dt, Gs, r, prow, part, y);
          T qq = T(0);
#pragma unroll
          for (int u = 0; u < C::CPT; ++u)
            if (part * C::CPT + u < r) qq += y[u] * dt[prow * C::RS + part * C::CPT + u];
          dq[c == 0 ? 4 : 7] += qq;
        }
      }
    }
  }
  // one combined fixed-order reduction of the partial dots
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int m = 0; m < NV; ++m) {
    const T v = warp_sum(dq[m]);
    if (lane == 0) shq[m][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    T v = T(0);
#pragma unroll
    for (int w = 0; w < 8; ++w) v += shq[threadIdx.x][w];
    a.part[((int64_t)tile * a.b + j) * kNQ + threadIdx.x] = (double)v;
  }
  if (a.ctl_mode) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) ticket = atomicAdd(&a.counters[j], 1u);
    __syncthreads();
    if (ticket == per - 1) {
      if (threadIdx.x == 0) a.counters[j] = 0u;
      if (threadIdx.x < 32)
        fused_control(a.ctl_mode, const_cast<Ctl&>(a.ctl[j]), a.part, (int)per, a.b, a.r, j, a.P, a.G64fix,
                      nullptr, NC);
    }
  }
  __syncthreads();  // shared memory free for a following item
}

}  // namespace

}  // namespace snmf
