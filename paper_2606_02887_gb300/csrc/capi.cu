// C ABI of the SNMPBB library (declarations and argument contract in include/snmf.h).
//
// Host orchestration: every step of an iteration is a kernel on the handle's internal
// stream; one outer iteration (penalty form: W block then H block, Sec. 2.1) or one step
// (direct form) is captured once into a CUDA graph and replayed.  The per-restart FP64
// state of Algorithm 1 lives on the device (snmf::Ctl); the host reads one flag every
// few replays to stop when every restart has converged.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/snmf.h"
#include "ax_tc.cuh"
#include "batch.cuh"
#include "fp8.cuh"
#include "common.cuh"
#include "lai.cuh"
#include "rowops.cuh"

using namespace snmf;

namespace {

enum BufId {
  B_W = 0, B_HT, B_B, B_G, B_Z, B_D, B_GZ, B_XN,  // penalty
  B_AZ, B_AD, B_AWN, B_GN,                        // direct extras (B_B = AW, B_XN = Wn)
  B_LX, B_LZ, B_LD,                               // graph products
  NBUF
};

std::string g_create_err;

}  // namespace

struct snmf_ctx {
  int kind = 0, prec = SNMF_F32, tdtype = 1;
  int64_t n = 0;
  int r = 0, b = 1, N = 0;
  size_t esz = 4;
  snmf_options opt{};
  cudaStream_t user = nullptr, s = nullptr;
  cudaStream_t s2 = nullptr;                            // side branch: Gram beside the product
  cudaEvent_t evfork = nullptr, evjoin = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, evsync = nullptr;
  AxArgs A{};
  void* A_owned = nullptr;
  float* A_scale = nullptr;      // FP8: per-tile scales
  int32_t* rowptr_owned = nullptr;
  int32_t* colidx_owned = nullptr;
  void* vals_owned = nullptr;
  double normA2 = 0.0, sumA = 0.0, lam = 0.0;
  // graph regulariser
  bool graph = false;
  double gamma = 0.0;
  double normL = 0.0;  // ||L||_2 (power method), enters rho of graph-regularised blocks
  int use_tile = 0;    // row kernels through the shared-memory tile body (r <= 32)
  int use_fuse = 0;    // D step and update through rowfuse.cu (FP32, r in {16, 32, 64}, no Z / D stored)
  int row_tc = 0;      // with use_fuse: row products on the tensor cores, 1 rowtc.cu, 2 rowtma.cu (r = 64; tuned)
  int row_bm = 0;      // general row kernel, FP32: rows per CTA (0: built-in choice; autotuned)
  AxArgs L{};
  int32_t* L_rowptr = nullptr;
  int32_t* L_colidx = nullptr;
  void* L_vals = nullptr;
  bool L_implicit = false;  // L = I - D^-1/2 A D^-1/2: h->L holds -D^-1/2 A D^-1/2, applied as X + (h->L) X
  double* L_scale = nullptr;  // d_i^-1/2
  // LAI sketch
  bool lai = false;
  LaiOp lai_op{};
  // workspaces
  void* buf[NBUF] = {};
  void* ws = nullptr;
  size_t ws_elems = 0;
  double *prow = nullptr, *pax = nullptr, *pax2 = nullptr, *pax3 = nullptr, *pax4 = nullptr,
         *pclip = nullptr;
  int nrow = 0, nax = 0;
  double* gpart = nullptr;
  int nchunks = 1;
  double *G64fix = nullptr, *G64p = nullptr;  // G64p: 3 pairs [pair][b][r*r]
  void* GT = nullptr;
  Ctl* ctl = nullptr;
  int* run = nullptr;
  int* recompute = nullptr;
  unsigned* counters = nullptr;  // arrival counters of the fused Gram reduction
  int* dev_err = nullptr;        // device error code of bounded waits (tensor-core product)
  void* xh = nullptr;            // BF16 hi / lo parts of the product operand (transposed)
  void* xl = nullptr;
  int xparts = 2;                // BF16 product: X as hi + lo parts (2) or rounded to BF16 (1)
  unsigned* tcount = nullptr;    // BF16 product: arrival counters of the fused split-K epilogue
  // the split-K reduction and epilogue fused into the BF16 product (1) or the separate finish
  // pass (0)
  int fuse_epilogue = 1;
  long long budget = 2000000000LL;
  __nv_bfloat16* mlp_w = nullptr;  // learned controller weights (BF16)
  float* rec_feat = nullptr;       // record mode dataset
  float* rec_targ = nullptr;
  int* rec_count = nullptr;
  int rec_cap = 0;
  int tc_fail = 0;               // status of a failed tensor-core launch (encoder / launch error)
  double* dsc = nullptr;   // device scratch doubles
  int* h_flag = nullptr;   // pinned
  std::vector<Ctl> h_ctl;
  // captured solve phases: 0 init, 1 one iteration, 2 final evaluation
  cudaGraphExec_t exec[3] = {nullptr, nullptr, nullptr};
  int nodes[3] = {0, 0, 0};
  int axn[3] = {0, 0, 0};
  int exec_form = -1;
  cudaEvent_t evdone = nullptr;
  bool have_result = false;
  int ax_count = 0;
  BatchCtx* bt = nullptr;
  // per-iteration statistics ring (device) and an imported solver state for an exact restart
  double* ring = nullptr;
  int ring_cap = 256;
  std::vector<Ctl> resume;   // from snmf_set_state: the next solve continues from this state
  // autotuned product configuration (tuned: 1 measured here, 2 from the cache)
  TuneEntry tune{};
  int tuned = 0;          // SNMF_DENSE_BATCH handle: the uneven-batch engine
  std::string err;
};

namespace {

snmf_status fail(snmf_ctx* h, snmf_status st, const std::string& msg) {
  if (h) h->err = msg; else g_create_err = msg;
  return st;
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(h, e_ == cudaErrorMemoryAllocation ? SNMF_ERR_OOM : SNMF_ERR_CUDA,  \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                \
  } while (0)

Params make_params(const snmf_ctx* h) {
  Params P{};
  P.formulation = h->opt.formulation;
  P.memory = h->opt.nonmonotone_M;
  P.bb = h->opt.bb_variant;
  P.max_ls = h->opt.max_ls;
  P.max_iter = h->opt.max_iter;
  P.power_iters = h->opt.power_iters;
  P.controller = h->opt.step_controller;
  P.theta = h->opt.theta;
  P.phi = h->opt.phi;
  P.eta = h->opt.eta;
  P.alpha_min = h->opt.alpha_min;
  P.alpha_max = h->opt.alpha_max;
  P.beta_shrink = h->opt.beta_shrink;
  P.tol = h->opt.tol;
  P.rho_factor = h->opt.direct_rho_factor;
  P.normA2 = h->lai ? h->lai_op.normA2 : h->normA2;
  P.gamma = h->graph ? h->gamma : 0.0;
  P.mlp_w = h->mlp_w;
  P.rec_feat = (h->opt.step_controller == 2 || h->opt.step_controller == 4) ? h->rec_feat : nullptr;
  P.rec_targ = h->rec_targ;
  P.rec_count = h->rec_count;
  P.rec_cap = h->rec_cap;
  P.nr = h->n * (int64_t)h->r;
  P.ring = h->ring;
  P.ring_cap = h->ring_cap;
  P.inner = h->opt.inner_iters;
  P.branch_step = h->opt.branch_step;
  return P;
}

Dims dims(const snmf_ctx* h) {
  Dims d;
  d.n = h->n; d.r = h->r; d.b = h->b; d.N = h->N; d.ld = h->N;
  return d;
}

// Epilogue of Y = op X (+ c X2) with partials <P1, op X>, <P2, op X> fused into the BF16
// tensor-core product where its tiles allow it (dots: r a multiple of 16 dividing the tile
// width); fused = 0 otherwise (the separate finish pass runs).
TcEpilogue tc_epilogue(snmf_ctx* h, void* Y, double c, const void* X2, const void* P1, const void* P2,
                       double* part) {
  TcEpilogue e;
  // the fused epilogue moves 16-byte groups along rows: the row pitch N must be a multiple of 4
  if (!h->tcount || !h->fuse_epilogue || h->N % 4 != 0) return e;
  if (P1 || P2) {
    // the partials are reduced per 64-column chunk of a tile: r must divide 64 and the tile width
    TcPlan pl;
    const ProdTune* tn = h->tuned ? &h->tune.cfg : nullptr;
    const int a8 = h->A.a_dtype == 3;
    if (tc_plan(h->n, h->N, &pl, tn, h->xparts, a8) < 0) tc_plan(h->n, h->N, &pl, nullptr, h->xparts, a8);
    if (h->r > 64 || 64 % h->r != 0 || h->r % 4 != 0 || pl.BN % h->r != 0) return e;
  }
  e.fused = 1;
  e.Y = (float*)Y;
  e.counters = h->tcount;
  e.c = (float)c;
  e.X2 = (const float*)X2;
  e.P1 = (const float*)P1;
  e.P2 = (const float*)P2;
  e.part = part;
  e.q0 = 0;
  e.r = h->r;
  e.b = h->b;
  return e;
}

// The product kernel: CUDA cores (FP64/FP32 dense, CSR, the FP8 final evaluation) or tcgen05
// (BF16 dense; E4M3 dense, decoded to BF16 in shared memory).  Returns the number of split-K
// slices written to h->ws (1 = result in Y), or 0 when the epilogue `epi` was fused into the
// product (the result, c X2 and the partials are complete).
int product_kernel(snmf_ctx* h, const AxArgs& op, const void* X, void* Y, const int* run,
                   const TcEpilogue* epi = nullptr) {
  const ProdTune* tn = (h->tuned && &op == &h->A) ? &h->tune.cfg : nullptr;  // the tuned shape only
  if (op.kind == AX_DENSE && op.a_dtype == 3) {
    if (!op.accurate && h->xh) {
      if (epi && epi->fused) {
        if (launch_ax_tc8_fused(op.A, op.a_scale, h->n, (const float*)X, h->N, h->N, h->xh, h->xl, h->xparts,
                                (float*)h->ws, h->ws_elems, h->dev_err, h->budget, *epi, run, h->s, tn) >= 0)
          return 0;
      } else {
        const int sp = launch_ax_tc8(op.A, op.a_scale, h->n, (const float*)X, h->N, h->N, h->xh, h->xl, (float*)Y,
                                     (float*)h->ws, h->ws_elems, h->dev_err, h->budget, h->s, tn, h->xparts);
        if (sp >= 1) return sp;
      }
      // no tensor map for these codes: the CUDA-core product below
    }
    return launch_ax_fp8(op.A, op.a_scale, h->n, (const float*)X, h->N, h->N, (float*)Y, (float*)h->ws,
                         h->ws_elems, run, h->s, tn);
  }
  if (op.kind == AX_DENSE && op.a_dtype == 2 && !op.accurate) {
    if (epi && epi->fused) {
      const int rc = launch_ax_tc_fused(op.A, h->n, (const float*)X, h->N, h->N, h->xh, h->xl, h->xparts,
                                        (float*)h->ws, h->ws_elems, h->dev_err, h->budget, *epi, run, h->s, tn,
                                        op.sym);
      if (rc < 0) {
        h->tc_fail = tc_last_status();
        return 1;
      }
      return 0;
    }
    const int sp = launch_ax_tc(op.A, h->n, (const float*)X, h->N, h->N, h->xh, h->xl, (float*)Y,
                                (float*)h->ws, h->ws_elems, h->dev_err, h->budget, h->s, tn, h->xparts, op.sym);
    if (sp < 1) {
      h->tc_fail = tc_last_status();
      return 1;
    }
    return sp;
  }
  return launch_ax(op, h->tdtype, h->n, h->N, h->N, X, Y, h->ws, h->ws_elems, run, h->s, tn);
}


// Y = op X (+ c X2), dots <P1, op X> -> part q0, <P2, op X> -> q0+1 (dots_after: of the final
// Y); returns slot count.
int ax_apply(snmf_ctx* h, const AxArgs& op, bool use_lai, const void* X, void* Y, double c,
             const void* X2, const void* P1, const void* P2, double* part, const int* run,
             int dots_after = 0) {
  Dims d = dims(h);
  h->ax_count++;
  if (use_lai) {
    return lai_apply(h->lai_op, h->tdtype, d, X, Y, c, X2, P1, P2, part, run, h->s);
  }
  TcEpilogue epi;
  if (op.kind == AX_DENSE && (op.a_dtype == 2 || op.a_dtype == 3) && !op.accurate)
    epi = tc_epilogue(h, Y, c, X2, P1, P2, part);
  const int splits = product_kernel(h, op, X, Y, run, &epi);
  if (splits == 0) return (int)((h->n + kRowTile - 1) / kRowTile);  // epilogue done in the product
  return launch_ax_finish_impl(h->tdtype, d, Y, h->ws, splits, c, X2, P1, P2, part, 0, run, h->s, dots_after);
}

int ax_A(snmf_ctx* h, const void* X, void* Y, double c, const void* X2, const void* P1,
         const void* P2, double* part, const int* run) {
  return ax_apply(h, h->A, h->lai, X, Y, c, X2, P1, P2, part, run);
}

// Y = L X with <P1, L X>, <P2, L X> partials; the paper's normalized Laplacian as
// X + (-D^-1/2 A D^-1/2) X, an explicit CSR L directly.
int ax_L(snmf_ctx* h, const void* X, void* Y, const void* P1, const void* P2, double* part,
         const int* run) {
  if (h->L_implicit) return ax_apply(h, h->L, false, X, Y, 1.0, X, P1, P2, part, run, 1);
  return ax_apply(h, h->L, false, X, Y, 0.0, nullptr, P1, P2, part, run);
}

int choose_chunks(int64_t n, int b, int r) {
  // about one CTA per SM, at least 512 rows per chunk (fewer partials to reduce)
  const int ntile = (r + 63) / 64;
  const int64_t per = (int64_t)b * ntile * ntile;
  int64_t c = (152 + per - 1) / per;
  c = std::max<int64_t>(1, std::min<int64_t>(c, n / 512));
  return (int)c;
}

// Gram X^T Y per restart into G64 (+ factor-type copy GT with lam I when pair == tpair);
// inside the iteration it follows ctl[j].active and the run flag, in the initial and
// final evaluations (ctl == NULL) every restart is computed.
void gram1(snmf_ctx* h, const void* X, const void* Y, int pair, int npairs, const Ctl* ctl,
           double* G64, void* GT, int tpair, double lam) {
  launch_gram(h->tdtype, X, Y, dims(h), pair, npairs, h->gpart, h->nchunks, ctl,
              ctl ? h->run : nullptr, G64, GT, tpair, lam, h->counters, h->s);
}

RowArgs row_base(snmf_ctx* h, const Params* P = nullptr) {
  RowArgs a{};
  a.n = h->n; a.r = h->r; a.b = h->b; a.ld = h->N;
  a.G = h->GT;
  a.ctl = h->ctl;
  a.run = h->run;
  a.gamma = h->graph ? h->gamma : 0.0;
  a.part = h->prow;
  a.counters = h->counters + 16384;
  a.G64fix = h->G64fix;
  a.tile = h->use_tile;
  a.bm = h->row_bm;
  if (P) a.P = *P;
  return a;
}

// Mean time of one D-step launch and one update launch of a W block (the row kernels of
// Alg. 1 lines 2-4) on the handle's current buffers, with every restart marked live.
snmf_status time_steps(snmf_ctx* h, int iters, double* ms_dstep, double* ms_update) {
  std::vector<Ctl> live(h->b);
  for (int j = 0; j < h->b; ++j) {
    live[j] = (j < (int)h->h_ctl.size()) ? h->h_ctl[j] : Ctl{};
    live[j].active = 1;
    live[j].nan_seen = 0;
    if (!(live[j].rho > 0.0)) live[j].rho = 1.0;
    if (!(live[j].alpha > 0.0)) live[j].alpha = 1.0;
  }
  CK(cudaMemcpyAsync(h->ctl, live.data(), h->b * sizeof(Ctl), cudaMemcpyHostToDevice, h->s));
  static const int one = 1;
  CK(cudaMemcpyAsync(h->run, &one, sizeof(int), cudaMemcpyHostToDevice, h->s));
  const Params P = make_params(h);
  const int td = h->tdtype;
  const int nc = h->opt.step_controller == 1 ? 2 : (h->opt.step_controller == 2 ? kNCand : 1);
  void* X = h->buf[B_W];
  RowArgs ad = row_base(h, &P);  // the D step of a W block, as in pen_block
  ad.B = h->buf[B_B];
  ad.Dout = h->buf[B_D]; ad.gZout = h->buf[B_GZ];
  ad.Wcur = X; ad.gWcur = h->buf[B_G];
  ad.X = X; ad.g_in = h->buf[B_G]; ad.Xout = h->buf[B_Z];
  ad.want_q = 1;
  ad.ctl_mode = CTL_LS;
  ad.dstore = nc == kNCand ? 4 : 0;
  ad.D2out = h->buf[B_AD];
  RowArgs au = row_base(h, &P);  // the update of a W block
  au.B = h->buf[B_B];
  au.gout = h->buf[B_G];
  au.Xold = X; au.gold = h->buf[B_G];
  au.Zold = h->buf[B_Z]; au.gZold = h->buf[B_GZ];
  au.Xout = X;
  au.ctl_mode = CTL_UPD_W;
  au.Zin = h->buf[B_Z]; au.Din = h->buf[B_D]; au.Din2 = h->buf[B_AD];
  auto dstep = [&] {
    if (h->use_fuse && h->row_tc == 2 && launch_rowtma_dstep(ad, h->dev_err, h->s)) {
    } else if (h->use_fuse && h->row_tc) launch_rowtc_dstep(ad, h->dev_err, h->s);
    else if (h->use_fuse) launch_rowfuse_dstep(ad, h->row_bm, nc, h->s);
    else launch_rowgemm(td, OP_ZSTEP, EPI_DIR, ad, h->s, nc);
  };
  auto update = [&] {
    if (h->use_fuse && h->row_tc == 2 && launch_rowtma_update(au, h->dev_err, h->s)) {
    } else if (h->use_fuse && h->row_tc) launch_rowtc_update(au, h->dev_err, h->s);
    else if (h->use_fuse) launch_rowfuse_update(au, h->row_bm, nc, h->s);
    else launch_rowgemm(td, OP_UPD, EPI_GRAD, au, h->s);
  };
  cudaEvent_t e[4];
  for (auto& x : e) CK(cudaEventCreate(&x));
  dstep();  // warm-up
  update();
  CK(cudaEventRecord(e[0], h->s));
  for (int t = 0; t < iters; ++t) dstep();
  CK(cudaEventRecord(e[1], h->s));
  CK(cudaEventRecord(e[2], h->s));
  for (int t = 0; t < iters; ++t) update();
  CK(cudaEventRecord(e[3], h->s));
  CK(cudaStreamSynchronize(h->s));
  CK(cudaGetLastError());
  float m1 = 0.f, m2 = 0.f;
  cudaEventElapsedTime(&m1, e[0], e[1]);
  cudaEventElapsedTime(&m2, e[2], e[3]);
  for (auto& x : e) cudaEventDestroy(x);
  if (ms_dstep) *ms_dstep = m1 / iters;
  if (ms_update) *ms_update = m2 / iters;
  return SNMF_OK;
}

// Autotuner of the dense product: times every candidate configuration (CUDA events, one
// warm-up and five timed products each) and keeps the fastest; the result is cached per
// device and shape (in this process, and in opt.tune_cache when given).
snmf_status autotune_product(snmf_ctx* h) {
  if (h->kind != AX_DENSE) return SNMF_OK;
  static const char* dtn[4] = {"f64", "f32", "bf16", "fp8"};
  const std::string key = std::string("dense/") + dtn[h->A.a_dtype] + (h->A.a_dtype >= 2 && h->xparts == 1 ? "x1" : "") +
                          (h->A.sym ? "s" : "") +
                          "/n" + std::to_string(h->n) + "/r" + std::to_string(h->r) + "/N" + std::to_string(h->N);
  const std::string dev = tune_device_key();
  TuneEntry e;
  const bool tune_rows =
      (!h->use_tile || h->use_fuse) && h->tdtype == 1 && h->opt.formulation != SNMF_DIRECT && h->r <= 64;
  // rows per CTA offered to the search: the fused kernels' heights, else the general kernel's
  std::vector<int> bms;
  if (h->use_fuse) bms = h->r == 16 ? std::vector<int>{128, 256} : std::vector<int>{128, 64};
  else bms = {64, 32};
  if (tune_lookup(h->opt.tune_cache, dev, key, &e)) {
    h->tune = e;
    h->tuned = 2;
    if (tune_rows && std::find(bms.begin(), bms.end(), e.cfg.row_bm) != bms.end()) {
      h->row_bm = e.cfg.row_bm;
      if (!h->use_tile) h->nrow = rowgemm_slots(dims(h), h->tdtype, 0, h->row_bm);
    }
    const int tnc = h->opt.step_controller == 1 ? 2 : 1;
    h->row_tc = 0;
    if (tune_rows && h->use_fuse && e.cfg.row_tc == 1 && rowtc_supported(h->tdtype, h->r, tnc)) h->row_tc = 1;
    if (tune_rows && h->use_fuse && e.cfg.row_tc == 2 && rowtma_supported(h->tdtype, h->r, tnc, h->N)) h->row_tc = 2;
    return SNMF_OK;
  }
  std::vector<ProdTune> cand;
  if (h->A.a_dtype == 2 || h->A.a_dtype == 3) {
    const int rings[7][2] = {{2, 2}, {2, 3}, {2, 4}, {1, 2}, {1, 3}, {1, 4}, {1, 6}};
    const int bn0 = h->N <= 256 ? (h->N + 15) / 16 * 16 : 256;
    std::vector<int> bns{bn0};
    for (int w : {128, 64})
      if (w < bn0) bns.push_back(w);
    for (int bn : bns)
    for (auto& rg : rings)
      for (int sp : {1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 16, 19, 24, 32}) {
        ProdTune t;
        t.per_sm = rg[0];
        t.stages = rg[1];
        t.splits = sp;
        t.bn = bn;
        TcPlan pl;
        if (tc_plan(h->n, h->N, &pl, &t, h->xparts, h->A.a_dtype == 3) < 0 || pl.splits != sp) continue;
        if ((size_t)sp * h->n * h->N > h->ws_elems && sp > 1) continue;
        cand.push_back(t);
      }
  } else {
    for (int sp : {1, 2, 3, 4, 5, 6, 8, 10, 12, 16, 19, 24, 32}) {
      if (sp > 1 && ((size_t)sp * h->n * h->N > h->ws_elems || h->n / sp < 64)) continue;
      ProdTune t;
      t.splits = sp;
      cand.push_back(t);
    }
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  TuneEntry best;
  best.ms = 1e30;
  h->tuned = 1;
  // timed as the solve runs it: B = A X + lambda X (epilogue fused into the BF16 product)
  const TcEpilogue tepi = tc_epilogue(h, h->buf[B_AZ], h->lam, h->buf[B_W], nullptr, nullptr, h->pax);
  for (const ProdTune& t : cand) {
    h->tune.cfg = t;
    product_kernel(h, h->A, h->buf[B_W], h->buf[B_AZ], nullptr, &tepi);  // warm-up
    CK(cudaEventRecord(e0, h->s));
    for (int rep = 0; rep < 5; ++rep) product_kernel(h, h->A, h->buf[B_W], h->buf[B_AZ], nullptr, &tepi);
    CK(cudaEventRecord(e1, h->s));
    CK(cudaStreamSynchronize(h->s));
    if (h->tc_fail) {  // a configuration that did not launch is skipped
      h->tc_fail = 0;
      cudaGetLastError();
      continue;
    }
    CK(cudaGetLastError());
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms / 5 < best.ms) {
      best.cfg = t;
      best.ms = ms / 5;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int derr = 0;
  CK(cudaMemcpy(&derr, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (derr) {
    h->tuned = 0;
    return fail(h, SNMF_ERR_TIMEOUT, "a bounded device wait ran out while tuning the product");
  }
  if (best.ms >= 1e30) {
    h->tuned = 0;
    return SNMF_OK;
  }
  h->tune = best;
  // the general row kernel's tile height (FP32 penalty form): D step + update per inner step
  if (tune_rows) {
    double bt = 1e30;
    int bbm = 0;
    for (int bm : bms) {
      h->row_bm = bm;
      if (!h->use_tile) h->nrow = rowgemm_slots(dims(h), h->tdtype, 0, bm);
      double md = 0.0, mu = 0.0;
      const snmf_status st = time_steps(h, 5, &md, &mu);
      if (st != SNMF_OK) return st;
      if (md + mu < bt) { bt = md + mu; bbm = bm; }
    }
    h->row_bm = bbm;
    if (!h->use_tile) h->nrow = rowgemm_slots(dims(h), h->tdtype, 0, bbm);
    h->tune.cfg.row_bm = bbm;
    // the tensor-core row products (r = 64): per-CTA tiles (1) and the persistent TMA
    // pipeline (2), each kept when faster than the best so far and free of device errors
    const int tnc = h->opt.step_controller == 1 ? 2 : 1;
    h->row_tc = 0;
    for (int kind = 1; kind <= 2 && h->use_fuse; ++kind) {
      if (kind == 1 && !rowtc_supported(h->tdtype, h->r, tnc)) continue;
      if (kind == 2 && !rowtma_supported(h->tdtype, h->r, tnc, h->N)) continue;
      const int prev = h->row_tc;
      h->row_tc = kind;
      double md = 0.0, mu = 0.0;
      const snmf_status st = time_steps(h, 5, &md, &mu);
      if (st != SNMF_OK) return st;
      int derr2 = 0;
      CK(cudaMemcpy(&derr2, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
      if (derr2) {
        CK(cudaMemset(h->dev_err, 0, sizeof(int)));
        h->row_tc = prev;
      } else if (md + mu < bt) {
        bt = md + mu;
      } else {
        h->row_tc = prev;
      }
    }
    h->tune.cfg.row_tc = h->row_tc;
  }
  tune_store(h->opt.tune_cache, dev, key, h->tune);
  return SNMF_OK;
}

// ----------------------------------------------------------------------------
// penalty form (Sec. 2.1-2.2): one block of Algorithm 1 over Xvar with Xfix fixed
// ----------------------------------------------------------------------------
void pen_block(snmf_ctx* h, int xv, int xf, bool is_w, const Params& P, bool naive = false) {
  const Dims d = dims(h);
  const int td = h->tdtype;
  void* X = h->buf[xv];
  void* Xf = h->buf[xf];
  const bool gr = h->graph && !is_w;
  // The Gram and rho_0 depend on Xfix alone, so they run on the side stream beside the
  // product (a fork and a join of the captured graph); they share no buffer with it.
  // G = Xfix^T Xfix (+ lambda I in the factor-type copy); rho_0 = ||Xfix^T Xfix||_2, computed
  // by the Gram's last CTA when the restart is one tile (FP32 path), else by k_rho
  cudaEventRecord(h->evfork, h->s);
  cudaStreamWaitEvent(h->s2, h->evfork, 0);
  const bool rho_fused = td == 1 && h->r <= 64;
  // graph-regularised H block: rho_0 = ||W^T W||_2 + gamma ||L||_2 (Lipschitz constant of its gradient)
  const double shift = gr ? h->gamma * h->normL : 0.0;
  launch_gram(td, Xf, Xf, d, 0, 1, h->gpart, h->nchunks, h->ctl, h->run, h->G64fix, h->GT, 0, h->lam,
              h->counters, h->s2, rho_fused ? h->ctl : nullptr, h->opt.power_iters, 1.0, shift);
  if (!rho_fused) launch_rho(td, h->G64fix, d, h->opt.power_iters, 1.0, h->ctl, 0, h->s2, shift);
  cudaEventRecord(h->evjoin, h->s2);
  // B = A Xfix + lambda Xfix (Eq. (2.1)/(2.2))
  ax_A(h, Xf, h->buf[B_B], h->lam, Xf, nullptr, nullptr, h->pax, h->run);
  cudaStreamWaitEvent(h->s, h->evjoin, 0);
  if (gr) ax_L(h, X, h->buf[B_LX], nullptr, nullptr, h->pax2, h->run);
  {
    // gradient at the block start; its last CTA per restart runs the block-start control
    RowArgs a = row_base(h, &P);
    a.X = X; a.B = h->buf[B_B]; a.LX = gr ? h->buf[B_LX] : nullptr;
    a.gout = h->buf[B_G];
    a.ctl_mode = is_w ? CTL_START_W : CTL_START_H;
    if (h->use_fuse && h->row_tc && !gr) launch_rowtc_grad(a, h->dev_err, h->s);  // X G on tcgen05
    else launch_rowgemm(td, OP_LOAD, EPI_GRAD, a, h->s);
  }
  launch_any_active(h->ctl, h->b, h->run, nullptr, h->s);
  const int K = h->opt.inner_iters;
  const bool fused_q = h->r <= 64 && !gr;
  if (h->use_fuse && !gr) {
    // D step (g(Z) and the line search) and the update recomputing Z and D (rowfuse.cu);
    // the learned step with fallback (controller 1) carries the plain BB direction as well
    const int nc = h->opt.step_controller == 1 ? 2 : 1;
    for (int k = 0; k < K; ++k) {
      RowArgs a = row_base(h, &P);
      a.X = X; a.g_in = h->buf[B_G]; a.B = h->buf[B_B]; a.gZout = h->buf[B_GZ];
      a.ctl_mode = CTL_LS;
      if (h->row_tc == 2 && launch_rowtma_dstep(a, h->dev_err, h->s)) {
      } else if (h->row_tc) launch_rowtc_dstep(a, h->dev_err, h->s);
      else launch_rowfuse_dstep(a, h->row_bm, nc, h->s);
      RowArgs u = row_base(h, &P);
      u.Xout = X; u.gout = h->buf[B_G]; u.gZold = h->buf[B_GZ]; u.B = h->buf[B_B];
      u.ctl_mode = is_w ? (naive && k == K - 1 ? CTL_UPD_W_LAST_NAIVE : CTL_UPD_W)
                        : (k == K - 1 ? CTL_UPD_H_LAST : CTL_UPD_H);
      if (h->row_tc == 2 && launch_rowtma_update(u, h->dev_err, h->s)) {
      } else if (h->row_tc) launch_rowtc_update(u, h->dev_err, h->s);
      else launch_rowfuse_update(u, h->row_bm, nc, h->s);
    }
    return;
  }
  for (int k = 0; k < K; ++k) {
    // Z = Proj[X - g / rho_0], D = Proj[Z - alpha g(Z)] - Z   (Alg. 1 lines 2-3)
    {
      RowArgs a = row_base(h, &P);
      a.B = h->buf[B_B];
      a.Dout = h->buf[B_D]; a.gZout = h->buf[B_GZ];
      a.Wcur = X; a.gWcur = h->buf[B_G];
      if (gr) {
        launch_zstep(td, d, X, h->buf[B_G], h->buf[B_Z], h->ctl, h->s);
        ax_L(h, h->buf[B_Z], h->buf[B_LZ], nullptr, nullptr, h->pax2, h->run);
        a.X = h->buf[B_Z]; a.LX = h->buf[B_LZ];
        launch_rowgemm(td, OP_LOAD, EPI_DIR, a, h->s);
      } else {
        a.X = X; a.g_in = h->buf[B_G]; a.Xout = h->buf[B_Z];
        a.want_q = fused_q ? 1 : 0;
        a.ctl_mode = fused_q ? CTL_LS : CTL_NONE;  // line search in the last CTA of each restart
        // learned controller: proposal + plain BB direction; record mode: 9 candidates
        const int nc = h->opt.step_controller == 1 ? 2 : (h->opt.step_controller == 2 ? kNCand : 1);
        a.dstore = nc == kNCand ? 4 : 0;
        a.D2out = h->buf[B_AD];
        launch_rowgemm(td, OP_ZSTEP, EPI_DIR, a, h->s, nc);
      }
    }
    if (!fused_q) {
      // curvature of the line-search quadratic from the Gram D^T D; graph term <D, L D>
      gram1(h, h->buf[B_D], h->buf[B_D], 0, 1, h->ctl, h->G64p, nullptr, -1, 0.0);
      int nl = 0;
      if (gr) nl = ax_L(h, h->buf[B_D], h->buf[B_LD], h->buf[B_D], nullptr, h->pax3, h->run);
      launch_ctl_pen_ls(h->ctl, h->prow, h->nrow, h->pax3, gr ? nl : 0, h->b, h->r, h->G64fix, h->G64p, P,
                        gr ? 1 : 0, h->s);
    }
    // X' = Proj[Z + phi beta D], gradient, BB inner products   (Alg. 1 line 4)
    {
      RowArgs a = row_base(h, &P);
      a.B = h->buf[B_B];
      a.gout = h->buf[B_G];
      a.Xold = X; a.gold = h->buf[B_G];
      a.Zold = h->buf[B_Z]; a.gZold = h->buf[B_GZ];
      a.Xout = X;
      a.ctl_mode = is_w ? (naive && k == K - 1 ? CTL_UPD_W_LAST_NAIVE : CTL_UPD_W)
                        : (k == K - 1 ? CTL_UPD_H_LAST : CTL_UPD_H);
      if (gr) {
        launch_xupd(td, d, h->buf[B_Z], h->buf[B_D], h->buf[B_XN], nullptr, nullptr, nullptr,
                    h->ctl, h->pclip, h->s);
        ax_L(h, h->buf[B_XN], h->buf[B_LX], nullptr, nullptr, h->pax2, h->run);
        a.X = h->buf[B_XN]; a.LX = h->buf[B_LX];
        launch_rowgemm(td, OP_LOAD, EPI_GRAD, a, h->s);
      } else {
        a.Zin = h->buf[B_Z]; a.Din = h->buf[B_D]; a.Din2 = h->buf[B_AD];
        launch_rowgemm(td, OP_UPD, EPI_GRAD, a, h->s);
      }
    }
  }
}

// H gradient at the start point (enters the first joint projected gradient).
void pen_init(snmf_ctx* h, const Params& P) {
  const Dims d = dims(h);
  const int td = h->tdtype;
  launch_any_active(h->ctl, h->b, h->run, nullptr, h->s);
  ax_A(h, h->buf[B_W], h->buf[B_B], h->lam, h->buf[B_W], nullptr, nullptr, h->pax, h->run);
  gram1(h, h->buf[B_W], h->buf[B_W], 0, 1, h->ctl, h->G64fix, h->GT, 0, h->lam);
  if (h->graph) ax_L(h, h->buf[B_HT], h->buf[B_LX], nullptr, nullptr, h->pax2, h->run);
  RowArgs a = row_base(h, &P);
  a.X = h->buf[B_HT]; a.B = h->buf[B_B]; a.LX = h->graph ? h->buf[B_LX] : nullptr;
  a.gout = h->buf[B_G];
  a.ctl_mode = CTL_START_INIT;  // records the H gradient of the start
  launch_rowgemm(td, OP_LOAD, EPI_GRAD, a, h->s);
}

void pen_iteration(snmf_ctx* h, const Params& P) {
  pen_block(h, B_W, B_HT, true, P);
  pen_block(h, B_HT, B_W, false, P);
  launch_any_active(h->ctl, h->b, h->run, nullptr, h->s);
}

// The naive symmetric variant (Sec. 2.1, before the penalty form): Algorithm 1 on the W block
// with H = W^T fixed (lambda = 0), then H <- W^T.  The start needs nothing beyond the state
// the host sets; one outer iteration is the W block and the copy.
void naive_init(snmf_ctx* h) { launch_any_active(h->ctl, h->b, h->run, nullptr, h->s); }

void naive_iteration(snmf_ctx* h, const Params& P) {
  pen_block(h, B_W, B_HT, true, P, true);
  cudaMemcpyAsync(h->buf[B_HT], h->buf[B_W], (size_t)h->n * h->N * h->esz, cudaMemcpyDeviceToDevice, h->s);
  launch_any_active(h->ctl, h->b, h->run, nullptr, h->s);
}

void pen_final(snmf_ctx* h, const Params& P) {
  const Dims d = dims(h);
  const int td = h->tdtype;
  // every restart contributes to the final evaluation.  The closed-form objective
  // ||A||^2 - 2 <W, A Ht> + ... cancels to a small residual, so <W, A Ht> is taken from an
  // FP32 CUDA-core product of the stored BF16 A: the tensor-core FP32 accumulation carries
  // a relative bias of about 1e-5 over K = 8192, which that cancellation would amplify.
  AxArgs fin = h->A;
  fin.accurate = 1;
  int nax = ax_apply(h, fin, h->lai, h->buf[B_HT], h->buf[B_B], h->lam, h->buf[B_HT],
                     h->buf[B_W], nullptr, h->pax, nullptr);
  gram1(h, h->buf[B_W], h->buf[B_W], 0, 3, nullptr, h->G64p, h->GT, 1, h->lam);
  gram1(h, h->buf[B_HT], h->buf[B_HT], 1, 3, nullptr, h->G64p, h->GT, 1, h->lam);
  gram1(h, h->buf[B_W], h->buf[B_HT], 2, 3, nullptr, h->G64p, h->GT, 1, h->lam);
  // W gradient at the final point (projected-gradient statistic); uses a temporary
  // "all active" view: the row kernel is run with ctl entries forced live by the host.
  RowArgs a = row_base(h);
  a.X = h->buf[B_W]; a.B = h->buf[B_B];
  a.gout = h->buf[B_G];
  a.run = nullptr;
  a.ctl = h->ctl + h->b;  // second Ctl array: all active (set by the host)
  launch_rowgemm(td, OP_LOAD, EPI_GRAD, a, h->s);
  const int64_t rr = (int64_t)h->r * h->r * h->b;
  launch_ctl_final_pen(h->ctl, h->pax, nax, h->prow, h->nrow, h->G64p, h->G64p + rr,
                       h->G64p + 2 * rr, h->b, h->r, P, h->s);
}

// ----------------------------------------------------------------------------
// direct form (Eq. (2) with 1/4 scaling): one step of Algorithm 1
// ----------------------------------------------------------------------------
void dir_init(snmf_ctx* h, const Params& P) {
  const Dims d = dims(h);
  const int td = h->tdtype;
  int nax = ax_apply(h, h->A, h->lai, h->buf[B_W], h->buf[B_B], 0.0, nullptr, h->buf[B_W], nullptr,
                     h->pax, nullptr);
  int nlx = 0;
  if (h->graph)
    nlx = ax_L(h, h->buf[B_W], h->buf[B_LX], h->buf[B_W], nullptr, h->pax2, nullptr);
  gram1(h, h->buf[B_W], h->buf[B_W], 0, 1, nullptr, h->G64fix, h->GT, 0, 0.0);
  RowArgs a = row_base(h);
  a.X = h->buf[B_W]; a.B = h->buf[B_B]; a.LX = h->graph ? h->buf[B_LX] : nullptr;
  a.gout = h->buf[B_G];
  a.run = nullptr;
  a.ctl = h->ctl + h->b;  // all live
  launch_rowgemm(td, OP_LOAD, EPI_GRAD, a, h->s);
  launch_ctl_dir_init(h->ctl, h->pax, nax, h->prow, h->nrow, h->graph ? h->pax2 : nullptr, nlx,
                      h->G64fix, h->b, h->r, P, h->s);
  launch_any_active(h->ctl, h->b, h->run, h->recompute, h->s);
}

void dir_iteration(snmf_ctx* h, const Params& P) {
  const Dims d = dims(h);
  const int td = h->tdtype;
  const int64_t rr = (int64_t)h->r * h->r * h->b;
  void *W = h->buf[B_W], *AW = h->buf[B_B], *g = h->buf[B_G];
  void *Z = h->buf[B_Z], *AZ = h->buf[B_AZ], *D = h->buf[B_D], *AD = h->buf[B_AD];
  void *Wn = h->buf[B_XN], *AWn = h->buf[B_AWN], *gn = h->buf[B_GN];
  // rho_k = factor ||W^T W||_2 and alpha_k
  launch_rho(td, h->G64fix, d, h->opt.power_iters, h->opt.direct_rho_factor, h->ctl, 0, h->s,
             h->graph ? h->gamma * h->normL : 0.0);
  launch_ctl_dir_alpha(h->ctl, h->b, P, h->s);
  launch_zstep(td, d, W, g, Z, h->ctl, h->s);
  int nz = ax_A(h, Z, AZ, 0.0, nullptr, Z, nullptr, h->pax, h->run);
  if (h->graph) ax_L(h, Z, h->buf[B_LZ], Z, nullptr, h->pax3, h->run);
  gram1(h, Z, Z, 0, 1, h->ctl, h->G64p, h->GT, 0, 0.0);
  {
    RowArgs a = row_base(h);
    a.X = Z; a.B = AZ; a.LX = h->graph ? h->buf[B_LZ] : nullptr;
    a.Dout = D;
    launch_rowgemm(td, OP_LOAD, EPI_DIR, a, h->s);
  }
  int nd = ax_A(h, D, AD, 0.0, nullptr, Z, D, h->pax2, h->run);
  if (h->graph) ax_L(h, D, h->buf[B_LD], D, nullptr, h->pax4, h->run);
  gram1(h, Z, D, 0, 2, h->ctl, h->G64p + rr, nullptr, -1, 0.0);
  gram1(h, D, D, 1, 2, h->ctl, h->G64p + rr, nullptr, -1, 0.0);
  launch_ctl_dir_ls(h->ctl, h->pax, nz, h->prow, h->nrow, h->pax2, nd, h->G64p, h->G64p + rr,
                    h->G64p + 2 * rr, h->graph ? h->pax3 : nullptr, h->graph ? h->pax4 : nullptr,
                    h->b, h->r, P, h->s);
  int ncl = launch_xupd(td, d, Z, D, Wn, AZ, AD, AWn, h->ctl, h->pclip, h->s);
  launch_ctl_dir_clip(h->ctl, h->pclip, ncl, h->b, h->recompute, h->s);
  int nre = ax_A(h, Wn, AWn, 0.0, nullptr, Wn, nullptr, h->pax, h->recompute);
  int nlx = 0;
  if (h->graph) nlx = ax_L(h, Wn, h->buf[B_LX], Wn, nullptr, h->pax3, h->run);
  gram1(h, Wn, Wn, 0, 1, h->ctl, h->G64fix, h->GT, 0, 0.0);
  {
    RowArgs a = row_base(h);
    a.X = Wn; a.B = AWn; a.LX = h->graph ? h->buf[B_LX] : nullptr;
    a.gout = gn; a.Xold = W; a.gold = g;
    launch_rowgemm(td, OP_LOAD, EPI_GRAD, a, h->s);
  }
  launch_ctl_dir_upd(h->ctl, h->prow, h->nrow, h->pax, nre, h->graph ? h->pax3 : nullptr, nlx,
                     h->G64fix, h->recompute, h->b, h->r, P, h->s);
  launch_copy_live(td, d, Wn, W, h->ctl, h->s);
  launch_copy_live(td, d, AWn, AW, h->ctl, h->s);
  launch_copy_live(td, d, gn, g, h->ctl, h->s);
  launch_any_active(h->ctl, h->b, h->run, h->recompute, h->s);
}

void dir_final(snmf_ctx* h, const Params& P) {
  launch_ctl_final_dir(h->ctl, h->G64fix, h->b, h->r, P, h->s);
}

// Row kernels through the shared-memory tile body: r <= 32, penalty form, at most two step
// candidates, no graph term, and enough row tiles to fill the GPU (a tile holds 128 FP32 /
// 64 FP64 rows; small problems keep the general kernel's finer grid).
int tile_rule(const snmf_ctx* h) {
  const int64_t tr = h->tdtype == 0 ? 64 : 128;
  const int64_t tiles = (h->n + tr - 1) / tr * h->b;
  return (h->r <= 32 && h->opt.formulation != SNMF_DIRECT && h->opt.step_controller != 2 && !h->graph &&
          tiles >= 2 * 152) ? 1 : 0;
}

// D step and update through rowfuse.cu: FP32 factors, r in {16, 32, 64}, penalty form, the
// plain step or a learned step (with or without the fallback direction; not record mode), no
// graph term.
int fuse_rule(const snmf_ctx* h) {
  return (rowfuse_supported(h->tdtype, h->r) && h->opt.formulation != SNMF_DIRECT &&
          h->opt.step_controller != 2 && !h->graph) ? 1 : 0;
}

snmf_status alloc_buffers(snmf_ctx* h) {
  const size_t fe = (size_t)h->n * h->N;
  for (int i = 0; i < NBUF; ++i) {
    CK(cudaMalloc(&h->buf[i], fe * h->esz));
    CK(cudaMemsetAsync(h->buf[i], 0, fe * h->esz, h->s));
  }
  h->ws_elems = (h->kind == AX_DENSE) ? 8 * fe : 0;
  if (h->ws_elems) CK(cudaMalloc(&h->ws, h->ws_elems * h->esz));
  const Dims d = dims(h);
  h->nrow = rowgemm_slots(d, h->tdtype);
  h->nax = (int)((h->n + kRowTile - 1) / kRowTile);
  // room for every row-kernel layout (BM = 32 has the most slots; the tile body fewer)
  const int nrow_max = std::max(h->nrow, rowgemm_slots(d, h->tdtype, 0, 32));
  const size_t prec_n = (size_t)std::max(nrow_max, h->nax) * h->b * kNQ;
  // the shared-memory tile body where tile_rule allows it
  h->use_tile = tile_rule(h);
  if (h->use_tile) h->nrow = rowgemm_slots(d, h->tdtype, 1);
  h->use_fuse = fuse_rule(h);
  double** parts[] = {&h->prow, &h->pax, &h->pax2, &h->pax3, &h->pax4, &h->pclip};
  for (double** p : parts) {
    CK(cudaMalloc(p, prec_n * sizeof(double)));
    CK(cudaMemsetAsync(*p, 0, prec_n * sizeof(double), h->s));
  }
  h->nchunks = choose_chunks(h->n, h->b, h->r);
  const size_t rr = (size_t)h->r * h->r * h->b;
  CK(cudaMalloc(&h->gpart, (size_t)h->nchunks * 3 * rr * sizeof(double)));
  CK(cudaMalloc(&h->G64fix, rr * sizeof(double)));
  CK(cudaMalloc(&h->G64p, 3 * rr * sizeof(double)));
  CK(cudaMalloc(&h->GT, rr * h->esz));
  CK(cudaMalloc(&h->ctl, 2 * h->b * sizeof(Ctl)));
  CK(cudaMalloc(&h->run, sizeof(int)));
  CK(cudaMalloc(&h->recompute, sizeof(int)));
  CK(cudaMalloc(&h->dev_err, sizeof(int)));
  CK(cudaMemsetAsync(h->dev_err, 0, sizeof(int), h->s));
  if (h->kind == AX_DENSE && (h->prec == SNMF_BF16 || h->prec == SNMF_FP8)) {
    const size_t xb = (size_t)h->N * tc_ld(h->n) * 2;
    CK(cudaMalloc(&h->xh, xb));
    CK(cudaMalloc(&h->xl, xb));
    // one counter per output tile of any plan: 128-row tiles x tiles of >= 16 columns
    const size_t nt = (size_t)((h->n + 127) / 128) * ((h->N + 15) / 16);
    CK(cudaMalloc(&h->tcount, nt * sizeof(unsigned)));
    CK(cudaMemsetAsync(h->tcount, 0, nt * sizeof(unsigned), h->s));
  }
  if (h->opt.timeout_cycles > 0) h->budget = h->opt.timeout_cycles;
  CK(cudaMalloc(&h->counters, (16384 + 4096) * sizeof(unsigned)));  // Gram tiles, then restarts
  CK(cudaMemsetAsync(h->counters, 0, (16384 + 4096) * sizeof(unsigned), h->s));
  CK(cudaMalloc(&h->dsc, 4096 * sizeof(double)));
  CK(cudaMalloc(&h->ring, (size_t)h->b * h->ring_cap * kRingVals * sizeof(double)));
  CK(cudaMemsetAsync(h->ring, 0, (size_t)h->b * h->ring_cap * kRingVals * sizeof(double), h->s));
  CK(cudaMallocHost(&h->h_flag, sizeof(int)));
  return SNMF_OK;
}

// Structure check of a device-resident CSR matrix (launch_csr_check) on the handle's
// stream; *bad receives its flags (0 = valid).
snmf_status check_device_csr(snmf_ctx* h, const int32_t* rowptr, const int32_t* colidx, int64_t n, int64_t nnz,
                             int* bad) {
  int* dflag = nullptr;
  CK(cudaMalloc(&dflag, sizeof(int)));
  cudaError_t e = cudaMemsetAsync(dflag, 0, sizeof(int), h->s);
  if (e == cudaSuccess) {
    launch_csr_check(rowptr, colidx, n, nnz, dflag, h->s);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(bad, dflag, sizeof(int), cudaMemcpyDeviceToHost, h->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
  cudaFree(dflag);
  if (e != cudaSuccess) return fail(h, SNMF_ERR_CUDA, std::string("CSR check: ") + cudaGetErrorString(e));
  return SNMF_OK;
}

bool valid_enum(int v, int lo, int hi) { return v >= lo && v <= hi; }

snmf_status validate_options(const snmf_options& o) {
  if (!valid_enum(o.formulation, 0, 2) || !valid_enum(o.precision, 0, 3) ||
      !valid_enum(o.bb_variant, 0, 1))
    return SNMF_ERR_ARG;
  if (o.batch < 1 || o.nonmonotone_M < 0 || o.nonmonotone_M > kMaxHist || o.max_ls < 1 ||
      o.inner_iters < 1 || o.max_iter < 0 || o.power_iters < 1)
    return SNMF_ERR_ARG;
  if (!(o.theta > 0.0 && o.theta < 1.0) || !(o.phi > 0.0) || !(o.eta >= 0.0 && o.eta < 1.0) ||
      !(o.alpha_min > 0.0 && o.alpha_min < o.alpha_max) || !(o.beta_shrink > 0.0 && o.beta_shrink < 1.0) ||
      !(o.tol >= 0.0) || !(o.direct_rho_factor > 0.0))
    return SNMF_ERR_ARG;
  if (!valid_enum(o.step_controller, 0, 4) || !valid_enum(o.x_parts, 0, 2) || !valid_enum(o.sym_half, 0, 1))
    return SNMF_ERR_ARG;
  if ((o.step_controller == 1 || o.step_controller == 3) && !o.mlp_weights) return SNMF_ERR_ARG;
  if (o.step_controller == 4 && o.batch % kNCand != 0) return SNMF_ERR_ARG;
  return SNMF_OK;
}

snmf_status sync_user(snmf_ctx* h) {
  CK(cudaEventRecord(h->evsync, h->user));
  CK(cudaStreamWaitEvent(h->s, h->evsync, 0));
  return SNMF_OK;
}

}  // namespace

extern "C" {

void snmf_default_options(snmf_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->formulation = SNMF_PENALTY;
  o->precision = SNMF_F32;
  o->batch = 1;
  o->nonmonotone_M = 10;
  o->bb_variant = SNMF_BB1;
  o->max_ls = 20;
  o->inner_iters = 5;
  o->max_iter = 500;
  o->power_iters = 50;
  o->step_controller = 0;
  o->lambda_sym = -1.0;
  o->theta = 1e-3;
  o->phi = 1.7;
  o->eta = 0.85;
  o->alpha_min = 1e-10;
  o->alpha_max = 1e10;
  o->beta_shrink = 0.5;
  o->tol = 1e-4;
  o->branch_step = -1;
  o->direct_rho_factor = 3.0;
  o->init_scale = 2.0;
  o->seed = 0;
  o->mlp_weights = nullptr;
  o->timeout_cycles = 0;
  o->autotune = 0;
  o->x_parts = 0;
  o->tune_cache = nullptr;
  o->sym_half = 0;
}

snmf_status snmf_create(snmf_handle* out, const snmf_matrix* Am, int r, const snmf_options* opt,
                        void* stream) {
  snmf_ctx* h = nullptr;
  if (!out) return fail(nullptr, SNMF_ERR_ARG, "h is NULL");
  *out = nullptr;
  if (!Am) return fail(nullptr, SNMF_ERR_ARG, "A is NULL");
  snmf_options o;
  if (opt) o = *opt; else snmf_default_options(&o);
  if (validate_options(o) != SNMF_OK) return fail(nullptr, SNMF_ERR_ARG, "invalid options");
  if (Am->kind == SNMF_DENSE_BATCH) {
    std::string ve;
    if (batch_validate(Am, o, &ve) != SNMF_OK) return fail(nullptr, SNMF_ERR_ARG, ve);
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0)
      return fail(nullptr, SNMF_ERR_CUDA, "no CUDA device");
    init_kernel_attributes();
    h = new snmf_ctx();
    h->opt = o;
    h->prec = o.precision;
    h->user = (cudaStream_t)stream;
    std::string e;
    const snmf_status st = batch_create(&h->bt, Am, o, (cudaStream_t)stream, &e);
    if (st != SNMF_OK) {
      delete h;
      return fail(nullptr, st, e);
    }
    h->b = batch_nprob(h->bt);
    *out = h;
    return SNMF_OK;
  }
  if (Am->kind != SNMF_DENSE && Am->kind != SNMF_CSR) return fail(nullptr, SNMF_ERR_ARG, "unknown matrix kind");
  if (Am->dtype != SNMF_F64 && Am->dtype != SNMF_F32) return fail(nullptr, SNMF_ERR_ARG, "A dtype must be F64 or F32");
  if (Am->location != SNMF_ON_DEVICE && Am->location != SNMF_ON_HOST) return fail(nullptr, SNMF_ERR_ARG, "bad location");
  if (Am->n <= 0 || !Am->values) return fail(nullptr, SNMF_ERR_ARG, "n must be positive and values non-NULL");
  if (r < 1 || r > kMaxR || r > Am->n) return fail(nullptr, SNMF_ERR_ARG, "r out of range [1, min(n,256)]");
  if ((int64_t)r * o.batch > 4096) return fail(nullptr, SNMF_ERR_ARG, "r*batch > 4096");
  if (Am->kind == SNMF_DENSE && Am->ld < Am->n) return fail(nullptr, SNMF_ERR_ARG, "ld < n");
  if (Am->kind == SNMF_CSR) {
    if (!Am->rowptr || !Am->colidx || Am->nnz < 0) return fail(nullptr, SNMF_ERR_ARG, "CSR arrays missing");
    if (o.precision == SNMF_BF16 || o.precision == SNMF_FP8)
      return fail(nullptr, SNMF_ERR_ARG, "CSR supports F64/F32 precision");
  }
  if (o.sym_half && (Am->kind != SNMF_DENSE || o.precision != SNMF_BF16))
    return fail(nullptr, SNMF_ERR_ARG, "symmetric-half storage needs a dense A in SNMF_BF16 precision");
  if (o.step_controller && (o.formulation != SNMF_PENALTY || r > 64))
    return fail(nullptr, SNMF_ERR_ARG, "the step controller needs the penalty form and r <= 64");
  if (o.formulation == SNMF_NAIVE && o.step_controller)
    return fail(nullptr, SNMF_ERR_ARG, "the naive variant runs the plain BB step");

  h = new snmf_ctx();
  h->opt = o;
  h->kind = Am->kind == SNMF_DENSE ? AX_DENSE : AX_CSR;
  h->prec = o.precision;
  h->tdtype = (o.precision == SNMF_F64) ? 0 : 1;
  h->xparts = o.x_parts == 1 ? 1 : 2;
  h->esz = h->tdtype == 0 ? 8 : 4;
  h->n = Am->n;
  h->r = r;
  h->b = o.batch;
  h->N = r * o.batch;
  h->user = (cudaStream_t)stream;
  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0) {
    delete h;
    return fail(nullptr, SNMF_ERR_CUDA, "no CUDA device");
  }
  auto bail = [&](snmf_status st) {
    g_create_err = h->err;
    snmf_destroy(h);
    return st;
  };
#define CKC(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      h->err = std::string(#call) + ": " + cudaGetErrorString(e_);                         \
      return bail(e_ == cudaErrorMemoryAllocation ? SNMF_ERR_OOM : SNMF_ERR_CUDA);         \
    }                                                                                      \
  } while (0)
  init_kernel_attributes();
  CKC(cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking));
  CKC(cudaStreamCreateWithFlags(&h->s2, cudaStreamNonBlocking));
  CKC(cudaEventCreateWithFlags(&h->evfork, cudaEventDisableTiming));
  CKC(cudaEventCreateWithFlags(&h->evjoin, cudaEventDisableTiming));
  CKC(cudaEventCreate(&h->ev0));
  CKC(cudaEventCreate(&h->ev1));
  CKC(cudaEventCreateWithFlags(&h->evsync, cudaEventDisableTiming));
  CKC(cudaEventCreateWithFlags(&h->evdone, cudaEventDisableTiming));
  if (sync_user(h) != SNMF_OK) return bail(SNMF_ERR_CUDA);
  const int src_dt = Am->dtype == SNMF_F64 ? 0 : 1;
  const int64_t n = h->n;
  if (h->kind == AX_DENSE && o.precision == SNMF_FP8) {
    // owned E4M3 codes with a power-of-two scale per 128 x 128 tile
    const void* src = Am->values;
    void* staging = nullptr;
    const size_t sbytes = (size_t)n * Am->ld * (src_dt == 0 ? 8 : 4);
    if (Am->location == SNMF_ON_HOST) {
      CKC(cudaMalloc(&staging, sbytes));
      CKC(cudaMemcpyAsync(staging, src, sbytes, cudaMemcpyHostToDevice, h->s));
      src = staging;
    }
    const int nt = fp8_ntiles(n);
    CKC(cudaMalloc(&h->A_owned, (size_t)n * fp8_ld(n)));
    CKC(cudaMalloc(&h->A_scale, (size_t)nt * nt * sizeof(float)));
    launch_fp8_encode(src_dt, src, n, Am->ld, h->A_owned, h->A_scale, h->s);
    if (staging) {
      CKC(cudaStreamSynchronize(h->s));
      cudaFree(staging);
    }
    h->A.A = h->A_owned;
    h->A.lda = fp8_ld(n);
    h->A.a_dtype = 3;
    h->A.a_scale = h->A_scale;
    h->A.kind = AX_DENSE;
  } else if (h->kind == AX_DENSE && o.precision == SNMF_BF16) {
    // owned BF16 copy, K-major with columns padded to a multiple of 64 (tensor-core layout)
    const void* src = Am->values;
    void* staging = nullptr;
    const size_t sbytes = (size_t)n * Am->ld * (src_dt == 0 ? 8 : 4);
    if (Am->location == SNMF_ON_HOST) {
      CKC(cudaMalloc(&staging, sbytes));
      CKC(cudaMemcpyAsync(staging, src, sbytes, cudaMemcpyHostToDevice, h->s));
      src = staging;
    }
    const int64_t ldk = tc_ld(n);
    if (o.sym_half) {
      // the upper 128 x 128 tiles only (A symmetric): lda = tiles a side
      CKC(cudaMalloc(&h->A_owned, (size_t)sym_tiles(n) * 128 * 128 * 2));
      launch_to_bf16_sym(src_dt, src, n, Am->ld, h->A_owned, h->s);
    } else {
      CKC(cudaMalloc(&h->A_owned, (size_t)n * ldk * 2));
      launch_to_bf16(src_dt, src, n, Am->ld, h->A_owned, h->s);
    }
    if (staging) {
      CKC(cudaStreamSynchronize(h->s));
      cudaFree(staging);
    }
    h->A.A = h->A_owned;
    h->A.lda = o.sym_half ? (n + 127) / 128 : ldk;
    h->A.a_dtype = 2;
    h->A.sym = o.sym_half;
    h->A.kind = AX_DENSE;
  } else if (h->kind == AX_DENSE) {
    // working copy of A in the factor type unless it can be borrowed
    const bool borrow = Am->location == SNMF_ON_DEVICE && src_dt == h->tdtype;
    if (borrow) {
      h->A.A = Am->values;
      h->A.lda = Am->ld;
    } else {
      const void* src = Am->values;
      void* staging = nullptr;
      const size_t sbytes = (size_t)n * Am->ld * (src_dt == 0 ? 8 : 4);
      if (Am->location == SNMF_ON_HOST) {
        CKC(cudaMalloc(&staging, sbytes));
        CKC(cudaMemcpyAsync(staging, src, sbytes, cudaMemcpyHostToDevice, h->s));
        src = staging;
      }
      if (src_dt == h->tdtype) {
        h->A_owned = staging;
        h->A.A = staging;
        h->A.lda = Am->ld;
      } else {
        CKC(cudaMalloc(&h->A_owned, (size_t)n * n * h->esz));
        launch_convert(src_dt, h->tdtype, src, n, n, Am->ld, h->A_owned, n, h->s);
        h->A.A = h->A_owned;
        h->A.lda = n;
        if (staging) {
          CKC(cudaStreamSynchronize(h->s));
          cudaFree(staging);
        }
      }
    }
    h->A.a_dtype = h->tdtype;
    h->A.kind = AX_DENSE;
  } else if (h->kind == AX_CSR) {
    const int64_t nnz = Am->nnz;
    if (Am->location == SNMF_ON_HOST) {
      const int32_t* rp = Am->rowptr;
      if (rp[0] != 0 || rp[n] != nnz) {
        h->err = "CSR rowptr inconsistent with nnz";
        return bail(SNMF_ERR_ARG);
      }
      for (int64_t i = 0; i < n; ++i)
        if (rp[i + 1] < rp[i]) { h->err = "CSR rowptr not monotone"; return bail(SNMF_ERR_ARG); }
      for (int64_t e = 0; e < nnz; ++e)
        if (Am->colidx[e] < 0 || Am->colidx[e] >= n) { h->err = "CSR column index out of range"; return bail(SNMF_ERR_ARG); }
      CKC(cudaMalloc(&h->rowptr_owned, (n + 1) * sizeof(int32_t)));
      CKC(cudaMalloc(&h->colidx_owned, std::max<int64_t>(nnz, 1) * sizeof(int32_t)));
      CKC(cudaMalloc(&h->vals_owned, std::max<int64_t>(nnz, 1) * (src_dt == 0 ? 8 : 4)));
      CKC(cudaMemcpyAsync(h->rowptr_owned, rp, (n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, h->s));
      if (nnz) {
        CKC(cudaMemcpyAsync(h->colidx_owned, Am->colidx, nnz * sizeof(int32_t), cudaMemcpyHostToDevice, h->s));
        CKC(cudaMemcpyAsync(h->vals_owned, Am->values, nnz * (src_dt == 0 ? 8 : 4), cudaMemcpyHostToDevice, h->s));
      }
      h->A.rowptr = h->rowptr_owned;
      h->A.colidx = h->colidx_owned;
      h->A.vals = h->vals_owned;
    } else {
      // device-resident CSR: the same structure checks as for host arrays, by a device kernel
      int bad = 0;
      const snmf_status cs = check_device_csr(h, Am->rowptr, Am->colidx, n, nnz, &bad);
      if (cs != SNMF_OK) return bail(cs);
      if (bad & 1) { h->err = "CSR rowptr inconsistent with nnz or not monotone"; return bail(SNMF_ERR_ARG); }
      if (bad & 2) { h->err = "CSR column index out of range"; return bail(SNMF_ERR_ARG); }
      h->A.rowptr = Am->rowptr;
      h->A.colidx = Am->colidx;
      h->A.vals = Am->values;
    }
    h->A.v_dtype = src_dt;
    h->A.kind = AX_CSR;
    h->A.lda = nnz;
  }
  snmf_status st = alloc_buffers(h);
  if (st != SNMF_OK) return bail(st);
  if (o.step_controller == 1 || o.step_controller == 3) {
    std::vector<__nv_bfloat16> wb(kMlpParams);
    for (int i = 0; i < kMlpParams; ++i) wb[i] = __float2bfloat16_rn(o.mlp_weights[i]);  // BF16 weights
    CKC(cudaMalloc(&h->mlp_w, kMlpParams * sizeof(__nv_bfloat16)));
    CKC(cudaMemcpyAsync(h->mlp_w, wb.data(), kMlpParams * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice, h->s));
    CKC(cudaStreamSynchronize(h->s));
  }
  if (o.step_controller == 2 || o.step_controller == 4) {
    h->rec_cap = o.step_controller == 2 ? 1 << 18 : o.batch / kNCand;
    CKC(cudaMalloc(&h->rec_feat, (size_t)h->rec_cap * kMlpIn * sizeof(float)));
    CKC(cudaMalloc(&h->rec_targ, (size_t)h->rec_cap * sizeof(float)));
    CKC(cudaMalloc(&h->rec_count, sizeof(int)));
    CKC(cudaMemsetAsync(h->rec_count, 0, sizeof(int), h->s));
  }
  // ||A||_F^2 and mean(A) of the stored operator
  if (h->kind == AX_DENSE && h->A.a_dtype == 3) {
    const int nb = launch_fp8_sums(h->A.A, n, h->A.a_scale, h->dsc + 16, h->s);  // ||A~||^2 of the stored values
    launch_sum_pairs(h->dsc + 16, nb, h->dsc, h->s);
  } else if (h->kind == AX_DENSE && h->A.a_dtype == 2) {
    const int nb = h->A.sym ? launch_sums_bf16_sym(h->A.A, n, h->dsc + 16, h->s)
                            : launch_sums_bf16(h->A.A, n * h->A.lda, h->dsc + 16, h->s);  // ||A~||^2 of the stored values
    launch_sum_pairs(h->dsc + 16, nb, h->dsc, h->s);
  } else if (h->kind == AX_DENSE)
    launch_matrix_sums(AX_DENSE, h->tdtype, h->A.A, n, h->A.lda, 0, h->dsc + 16, h->dsc, h->s);
  else
    launch_matrix_sums(AX_CSR, h->A.v_dtype, h->A.vals, n, 0, h->A.lda, h->dsc + 16, h->dsc, h->s);
  double sums[2];
  CKC(cudaMemcpyAsync(sums, h->dsc, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->s));
  CKC(cudaStreamSynchronize(h->s));
  h->normA2 = sums[0];
  h->sumA = sums[1];
  if (!std::isfinite(h->normA2)) { h->err = "A has NaN/Inf entries"; return bail(SNMF_ERR_NUMERIC); }
  h->lam = o.lambda_sym >= 0.0 ? o.lambda_sym : 0.01 * std::sqrt(h->normA2);
  if (o.formulation == SNMF_NAIVE) h->lam = 0.0;  // the naive variant has no penalty term
  if (o.autotune) {
    nvtxRangePushA("snmf_create: autotune");
    const snmf_status ts = autotune_product(h);
    nvtxRangePop();
    if (ts != SNMF_OK) return bail(ts);
  }
  *out = h;
  return SNMF_OK;
#undef CKC
}

snmf_status snmf_set_graph_reg(snmf_handle h, const snmf_matrix* L, double gamma) {
  if (!h) return SNMF_ERR_STATE;
  if (h->opt.formulation == SNMF_NAIVE && gamma != 0.0)
    return fail(h, SNMF_ERR_ARG, "the naive variant has no H block for the graph term");
  if (h->bt) return fail(h, SNMF_ERR_STATE, "not available for a dense batch handle");
  if (!(gamma >= 0.0)) return fail(h, SNMF_ERR_ARG, "gamma must be >= 0");
  if (gamma == 0.0) {
    h->graph = false;
    h->gamma = 0.0;
    h->exec_form = -1;
    h->use_tile = tile_rule(h);
    h->use_fuse = fuse_rule(h);
    h->nrow = rowgemm_slots(dims(h), h->tdtype, h->use_tile, h->row_bm);
    return SNMF_OK;
  }
  if (!L) {
    // the paper's L = I - D^-1/2 A D^-1/2 (Sec. 2.2), from the handle's own A
    if (h->lai) return fail(h, SNMF_ERR_STATE, "the implicit Laplacian needs A itself, not a LAI sketch");
    if (h->kind == AX_DENSE && h->A.a_dtype > 1)
      return fail(h, SNMF_ERR_ARG, "the implicit Laplacian needs A stored in F32 or F64 precision");
    const int64_t n = h->n;
    const size_t fe = h->kind == AX_DENSE ? (size_t)n * n : (size_t)std::max<int64_t>(h->A.lda, 1);
    cudaFree(h->L_rowptr); cudaFree(h->L_colidx); cudaFree(h->L_vals); cudaFree(h->L_scale);
    h->L_rowptr = nullptr; h->L_colidx = nullptr; h->L_vals = nullptr; h->L_scale = nullptr;
    CK(cudaMalloc(&h->L_scale, (size_t)n * sizeof(double)));
    CK(cudaMalloc(&h->L_vals, fe * h->esz));
    launch_normalized_adjacency(h->A, h->tdtype, n, h->L_scale, h->L_vals, h->s);
    CK(cudaGetLastError());
    h->L = AxArgs{};
    if (h->kind == AX_DENSE) {
      h->L.kind = AX_DENSE;
      h->L.A = h->L_vals;
      h->L.lda = n;
      h->L.a_dtype = h->tdtype;
    } else {
      h->L.kind = AX_CSR;
      h->L.rowptr = h->A.rowptr;  // A's pattern (owned by the handle or borrowed for its lifetime)
      h->L.colidx = h->A.colidx;
      h->L.vals = h->L_vals;
      h->L.v_dtype = h->tdtype;
      h->L.lda = h->A.lda;
    }
    h->L_implicit = true;
  } else {
  if (L->kind != SNMF_CSR) return fail(h, SNMF_ERR_ARG, "L must be CSR");
  if (L->n != h->n) return fail(h, SNMF_ERR_ARG, "L size mismatch");
  if (L->dtype != SNMF_F64 && L->dtype != SNMF_F32) return fail(h, SNMF_ERR_ARG, "L dtype");
  const int64_t n = h->n, nnz = L->nnz;
  const size_t vb = L->dtype == SNMF_F64 ? 8 : 4;
  const cudaMemcpyKind kd = L->location == SNMF_ON_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  if (!L->rowptr || !L->colidx || !L->values || nnz < 0) return fail(h, SNMF_ERR_ARG, "L arrays missing");
  if (L->location == SNMF_ON_HOST) {
    if (L->rowptr[0] != 0 || L->rowptr[n] != nnz) return fail(h, SNMF_ERR_ARG, "L rowptr inconsistent");
    for (int64_t i = 0; i < n; ++i)
      if (L->rowptr[i + 1] < L->rowptr[i]) return fail(h, SNMF_ERR_ARG, "L rowptr not monotone");
    for (int64_t e = 0; e < nnz; ++e)
      if (L->colidx[e] < 0 || L->colidx[e] >= n) return fail(h, SNMF_ERR_ARG, "L column out of range");
  } else {
    int bad = 0;
    const snmf_status cs = check_device_csr(h, L->rowptr, L->colidx, n, nnz, &bad);
    if (cs != SNMF_OK) return cs;
    if (bad & 1) return fail(h, SNMF_ERR_ARG, "L rowptr inconsistent with nnz or not monotone");
    if (bad & 2) return fail(h, SNMF_ERR_ARG, "L column out of range");
  }
  cudaFree(h->L_rowptr); cudaFree(h->L_colidx); cudaFree(h->L_vals);
  h->L_rowptr = nullptr; h->L_colidx = nullptr; h->L_vals = nullptr;
  CK(cudaMalloc(&h->L_rowptr, (n + 1) * sizeof(int32_t)));
  CK(cudaMalloc(&h->L_colidx, std::max<int64_t>(nnz, 1) * sizeof(int32_t)));
  CK(cudaMalloc(&h->L_vals, std::max<int64_t>(nnz, 1) * vb));
  CK(cudaMemcpyAsync(h->L_rowptr, L->rowptr, (n + 1) * sizeof(int32_t), kd, h->s));
  if (nnz) {
    CK(cudaMemcpyAsync(h->L_colidx, L->colidx, nnz * sizeof(int32_t), kd, h->s));
    CK(cudaMemcpyAsync(h->L_vals, L->values, nnz * vb, kd, h->s));
  }
  CK(cudaStreamSynchronize(h->s));
  h->L = AxArgs{};
  h->L.kind = AX_CSR;
  h->L.rowptr = h->L_rowptr;
  h->L.colidx = h->L_colidx;
  h->L.vals = h->L_vals;
  h->L.v_dtype = L->dtype == SNMF_F64 ? 0 : 1;
  h->L.lda = nnz;
  h->L_implicit = false;
  }
  const int64_t n = h->n;
  h->graph = true;
  h->gamma = gamma;
  h->exec_form = -1;
  h->use_tile = 0;  // the graph term runs through the general row kernel
  h->use_fuse = 0;
  h->nrow = rowgemm_slots(dims(h), h->tdtype, 0, h->row_bm);
  // ||L||_2 by power_iters power iterations from s_i = 1 + (i mod 2) (L 1 = 0 for a
  // Laplacian, so the start must not be constant) and the Rayleigh quotient; the device
  // applies L (CSR product), the host normalises in FP64.
  {
    const size_t es = h->esz;
    std::vector<double> v(n), w(n);
    std::vector<unsigned char> buf((size_t)n * es);
    auto put = [&](const std::vector<double>& x, void* dst) -> cudaError_t {
      for (int64_t i = 0; i < n; ++i) {
        if (h->tdtype == 0) reinterpret_cast<double*>(buf.data())[i] = x[i];
        else reinterpret_cast<float*>(buf.data())[i] = (float)x[i];
      }
      return cudaMemcpyAsync(dst, buf.data(), (size_t)n * es, cudaMemcpyHostToDevice, h->s);
    };
    auto get = [&](const void* src, std::vector<double>* x) -> cudaError_t {
      const cudaError_t e = cudaMemcpyAsync(buf.data(), src, (size_t)n * es, cudaMemcpyDeviceToHost, h->s);
      if (e != cudaSuccess) return e;
      const cudaError_t e2 = cudaStreamSynchronize(h->s);
      for (int64_t i = 0; i < n; ++i)
        (*x)[i] = h->tdtype == 0 ? reinterpret_cast<double*>(buf.data())[i] : reinterpret_cast<float*>(buf.data())[i];
      return e2;
    };
    double nv = 0.0;
    for (int64_t i = 0; i < n; ++i) { v[i] = 1.0 + (double)(i & 1); nv += v[i] * v[i]; }
    for (auto& x : v) x /= std::sqrt(nv);
    double lnorm = 0.0;
    for (int it = 0; it <= h->opt.power_iters; ++it) {
      CK(put(v, h->buf[B_LZ]));
      launch_ax(h->L, h->tdtype, n, 1, 1, h->buf[B_LZ], h->buf[B_LD], nullptr, 0, nullptr, h->s);
      CK(get(h->buf[B_LD], &w));
      if (h->L_implicit)
        for (int64_t i = 0; i < n; ++i) w[i] += v[i];  // L v = v + (-D^-1/2 A D^-1/2) v
      if (it == h->opt.power_iters) {  // Rayleigh quotient v^T L v
        lnorm = 0.0;
        for (int64_t i = 0; i < n; ++i) lnorm += v[i] * w[i];
        break;
      }
      double nw = 0.0;
      for (int64_t i = 0; i < n; ++i) nw += w[i] * w[i];
      nw = std::sqrt(nw);
      if (nw == 0.0) break;
      for (int64_t i = 0; i < n; ++i) v[i] = w[i] / nw;
    }
    CK(cudaGetLastError());
    h->normL = lnorm;
  }
  return SNMF_OK;
}

snmf_status snmf_lai_sketch(snmf_handle h, int k, int oversample, int power_iters, uint64_t seed) {
  if (!h) return SNMF_ERR_STATE;
  if (h->bt) return fail(h, SNMF_ERR_STATE, "not available for a dense batch handle");
  if (k < 1 || oversample < 0 || power_iters < 0) return fail(h, SNMF_ERR_ARG, "bad sketch sizes");
  const int ell = k + oversample;
  if (ell > 128 || ell > h->n) return fail(h, SNMF_ERR_ARG, "k + oversample must be <= min(n, 128)");
  if (sync_user(h) != SNMF_OK) return SNMF_ERR_CUDA;
  std::string msg;
  const int rc = lai_build(h->lai_op, h->A, h->tdtype, h->n, k, ell, power_iters, seed, h->N, h->s, msg);
  if (rc != 0) return fail(h, rc == -3 ? SNMF_ERR_OOM : SNMF_ERR_CUDA, msg);
  h->lai = true;
  h->exec_form = -1;
  return SNMF_OK;
}

snmf_status snmf_svd_init(snmf_handle h, void* W, void* Ht, int oversample, int power_iters, uint64_t seed) {
  if (!h) return SNMF_ERR_STATE;
  if (h->bt) return fail(h, SNMF_ERR_STATE, "not available for a dense batch handle");
  if (!W || oversample < 0 || power_iters < 0) return fail(h, SNMF_ERR_ARG, "bad SVD start arguments");
  const int ell = h->r + oversample;
  if (ell > 128 || ell > h->n) return fail(h, SNMF_ERR_ARG, "r + oversample must be <= min(n, 128)");
  if (sync_user(h) != SNMF_OK) return SNMF_ERR_CUDA;
  LaiOp sk{};
  std::string msg;
  // the eigen-sketch of A itself (not of a LAI sketch set on the handle), k = r
  const int rc = lai_build(sk, h->A, h->tdtype, h->n, h->r, ell, power_iters, seed, h->r, h->s, msg);
  if (rc != 0) {
    lai_free(sk);
    return fail(h, rc == -3 ? SNMF_ERR_OOM : SNMF_ERR_CUDA, msg);
  }
  launch_svd_start(h->tdtype, sk, h->n, h->r, h->b, W, h->s);
  const size_t fbytes = (size_t)h->n * h->N * h->esz;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && Ht) e = cudaMemcpyAsync(Ht, W, fbytes, cudaMemcpyDeviceToDevice, h->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
  lai_free(sk);
  if (e != cudaSuccess) return fail(h, SNMF_ERR_CUDA, std::string("SVD start: ") + cudaGetErrorString(e));
  return SNMF_OK;
}

static snmf_status solve_impl(snmf_ctx* h, bool host, void* W, void* Ht, snmf_stats* out) {
  const size_t fbytes = (size_t)h->n * h->N * h->esz;
  const cudaMemcpyKind kin = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const cudaMemcpyKind kout = host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (sync_user(h) != SNMF_OK) return SNMF_ERR_CUDA;
  CK(cudaEventRecord(h->ev0, h->s));
  if (W) {
    CK(cudaMemcpyAsync(h->buf[B_W], W, fbytes, kin, h->s));
  } else {
    const double mean = h->sumA / ((double)h->n * (double)h->n);
    const double upper = h->opt.init_scale * std::sqrt(std::max(mean, 0.0) / h->r);
    launch_philox_uniform(h->tdtype, h->buf[B_W], h->n, h->N, h->N, h->opt.seed, upper, h->s);
  }
  const bool naive = h->opt.formulation == SNMF_NAIVE;
  const bool pen = h->opt.formulation == SNMF_PENALTY || naive;  // the naive variant runs the W block
  if (pen) {
    if (Ht && !naive) CK(cudaMemcpyAsync(h->buf[B_HT], Ht, fbytes, kin, h->s));
    else CK(cudaMemcpyAsync(h->buf[B_HT], h->buf[B_W], fbytes, cudaMemcpyDeviceToDevice, h->s));
  }
  // control state: restarts active; second array = "all live" view for final passes.  An
  // imported state (snmf_set_state) replaces the first array: its restarts continue with their
  // iteration counts, pg0 and last H-block projected gradient (the penalty blocks restart their
  // BB memory and nonmonotone reference at every block, so nothing else carries over).
  const bool resume = !h->resume.empty();
  h->h_ctl.assign(2 * h->b, Ctl{});
  for (int j = 0; j < 2 * h->b; ++j) {
    h->h_ctl[j].active = 1;
    h->h_ctl[j].lam = h->lam;
    h->h_ctl[j].rho = 1.0;
    h->h_ctl[j].mlp_mult = 1.0;
  }
  if (resume) {
    for (int j = 0; j < h->b; ++j) h->h_ctl[j] = h->resume[j];
    h->resume.clear();
  }
  CK(cudaMemcpyAsync(h->ctl, h->h_ctl.data(), 2 * h->b * sizeof(Ctl), cudaMemcpyHostToDevice, h->s));
  static const int one = 1, zero = 0;
  CK(cudaMemcpyAsync(h->run, &one, sizeof(int), cudaMemcpyHostToDevice, h->s));
  CK(cudaMemcpyAsync(h->recompute, &zero, sizeof(int), cudaMemcpyHostToDevice, h->s));
  const Params P = make_params(h);
  // capture init / iteration / final once per configuration (buffers are fixed)
  const int form = naive ? 2 : (pen ? 0 : 1);
  if (h->exec_form != form) {
    for (int g = 0; g < 3; ++g) {
      if (h->exec[g]) { cudaGraphExecDestroy(h->exec[g]); h->exec[g] = nullptr; }
      cudaGraph_t gr;
      CK(cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal));
      h->ax_count = 0;
      if (g == 0) { if (naive) naive_init(h); else if (pen) pen_init(h, P); else dir_init(h, P); }
      else if (g == 1) { if (naive) naive_iteration(h, P); else if (pen) pen_iteration(h, P); else dir_iteration(h, P); }
      else { if (pen) pen_final(h, P); else dir_final(h, P); }
      CK(cudaStreamEndCapture(h->s, &gr));
      size_t nn = 0;
      CK(cudaGraphGetNodes(gr, nullptr, &nn));
      h->nodes[g] = (int)nn;
      h->axn[g] = h->ax_count - ((!pen && g == 1) ? 1 : 0);  // direct: clipped recompute is conditional
      CK(cudaGraphInstantiate(&h->exec[g], gr, 0));
      cudaGraphDestroy(gr);
    }
    h->exec_form = form;
  }
  int64_t launches = W ? 0 : 1;
  nvtxRangePushA("snmf_solve: start");
  if (!resume) {  // a resumed solve already holds the start's statistics
    CK(cudaGraphLaunch(h->exec[0], h->s));
    launches += h->nodes[0];
  }
  nvtxRangePop();
  nvtxRangePushA("snmf_solve: iterations");
  int done = 0, launched = 0, chunk = 1;
  int done_before = 0;  // outer iterations of an imported state
  for (int j = 0; j < h->b; ++j) done_before = std::max(done_before, resume ? h->h_ctl[j].iters : 0);
  const int maxit = std::max(0, h->opt.max_iter - (h->opt.formulation == SNMF_DIRECT ? 0 : done_before));
  while (launched < maxit) {
    const int m = std::min(chunk, maxit - launched);
    for (int t = 0; t < m; ++t) CK(cudaGraphLaunch(h->exec[1], h->s));
    launched += m;
    CK(cudaMemcpyAsync(h->h_flag, h->run, sizeof(int), cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    if (*h->h_flag == 0) { done = 1; break; }
    chunk = std::min(chunk * 2, 8);
  }
  (void)done;
  nvtxRangePop();
  launches += (int64_t)h->nodes[1] * launched;
  nvtxRangePushA("snmf_solve: final evaluation");
  CK(cudaGraphLaunch(h->exec[2], h->s));
  nvtxRangePop();
  launches += h->nodes[2];
  if (W) CK(cudaMemcpyAsync(W, h->buf[B_W], fbytes, kout, h->s));
  if (pen && Ht) CK(cudaMemcpyAsync(Ht, h->buf[B_HT], fbytes, kout, h->s));
  CK(cudaEventRecord(h->ev1, h->s));
  CK(cudaMemcpyAsync(h->h_ctl.data(), h->ctl, h->b * sizeof(Ctl), cudaMemcpyDeviceToHost, h->s));
  CK(cudaEventRecord(h->evdone, h->s));
  CK(cudaStreamWaitEvent(h->user, h->evdone, 0));
  int derr = 0;
  CK(cudaMemcpyAsync(&derr, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  if (h->tc_fail) {
    const int tf = h->tc_fail;
    h->tc_fail = 0;
    cudaGetLastError();
    return fail(h, SNMF_ERR_CUDA, "tensor-core product not launched (status " + std::to_string(tf) + ")");
  }
  CK(cudaGetLastError());
  if (derr) {
    CK(cudaMemsetAsync(h->dev_err, 0, sizeof(int), h->s));
    CK(cudaStreamSynchronize(h->s));
    return fail(h, SNMF_ERR_TIMEOUT, "a bounded device wait of the tensor-core product ran out (code " +
                                         std::to_string(derr) + ")");
  }
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  h->have_result = true;
  // statistics
  int best = 0, conv = 1, lsf = 0, clip = 0, iters = 0, nan = 0, tried = 0, acc = 0;
  for (int j = 0; j < h->b; ++j) {
    const Ctl& c = h->h_ctl[j];
    if (c.fin_f < h->h_ctl[best].fin_f) best = j;
    const bool cj = c.pg0 == 0.0 || c.pg <= h->opt.tol * c.pg0;
    conv &= cj ? 1 : 0;
    lsf += c.ls_fail;
    clip += c.clipped;
    iters = std::max(iters, c.iters);
    nan |= c.nan_seen;
    tried += c.mlp_tried;
    acc += c.mlp_accept;
  }
  if (out) {
    out->iters = iters;
    out->converged = conv;
    out->ls_fail = lsf;
    out->clipped_steps = clip;
    out->best_restart = best;
    out->ax_products = h->axn[0] + h->axn[1] * launched + h->axn[2] + (pen ? 0 : clip);
    out->kernel_launches = launches;
    out->graph_replays = launched;
    out->ctl_proposals = tried;
    out->ctl_accepted = acc;
    out->f = h->h_ctl[best].fin_f;
    out->residual = h->h_ctl[best].fin_res;
    out->pg_rel = h->h_ctl[best].fin_pg;
    out->seconds = ms * 1e-3;
  }
  if (nan) return fail(h, SNMF_ERR_NUMERIC, "NaN/Inf in the scalar state");
  return conv ? SNMF_OK : SNMF_NOT_CONVERGED;
}

snmf_status snmf_solve(snmf_handle h, void* W, void* Ht, snmf_stats* out) {
  if (!h) return SNMF_ERR_STATE;
  if (h->bt) return batch_solve(h->bt, false, W, Ht, out, &h->err);
  return solve_impl(h, false, W, Ht, out);
}

snmf_status snmf_solve_host(snmf_handle h, void* W, void* Ht, snmf_stats* out) {
  if (!h) return SNMF_ERR_STATE;
  if (!W) return fail(h, SNMF_ERR_ARG, "W must not be NULL");
  if (h->bt) return batch_solve(h->bt, true, W, Ht, out, &h->err);
  return solve_impl(h, true, W, Ht, out);
}

snmf_status snmf_restart_stats(snmf_handle h, double* f, double* residual, double* pg_rel,
                               int32_t* iters) {
  if (!h) return SNMF_ERR_STATE;
  if (h->bt) return batch_problem_stats(h->bt, f, residual, pg_rel, iters, &h->err);
  if (!h->have_result) return fail(h, SNMF_ERR_STATE, "no solve has run");
  for (int j = 0; j < h->b; ++j) {
    const Ctl& c = h->h_ctl[j];
    if (f) f[j] = c.fin_f;
    if (residual) residual[j] = c.fin_res;
    if (pg_rel) pg_rel[j] = c.fin_pg;
    if (iters) iters[j] = c.iters;
  }
  return SNMF_OK;
}

snmf_status snmf_get_factors(snmf_handle h, void* W, void* Ht) {
  if (!h) return SNMF_ERR_STATE;
  if (h->bt) return batch_get_factors(h->bt, W, Ht, &h->err);
  if (!h->have_result) return fail(h, SNMF_ERR_STATE, "no solve has run");
  const size_t fbytes = (size_t)h->n * h->N * h->esz;
  if (W) CK(cudaMemcpyAsync(W, h->buf[B_W], fbytes, cudaMemcpyDeviceToDevice, h->s));
  if (Ht) CK(cudaMemcpyAsync(Ht, h->buf[h->opt.formulation == SNMF_PENALTY ? B_HT : B_W], fbytes,
                             cudaMemcpyDeviceToDevice, h->s));
  CK(cudaStreamSynchronize(h->s));
  return SNMF_OK;
}

snmf_status snmf_apply(snmf_handle h, const void* X, void* Y, int cols, double* xax) {
  if (!h) return SNMF_ERR_STATE;
  if (h->bt) return fail(h, SNMF_ERR_STATE, "not available for a dense batch handle");
  if (!X || !Y || cols < 1 || cols > h->N) return fail(h, SNMF_ERR_ARG, "bad apply arguments");
  if (sync_user(h) != SNMF_OK) return SNMF_ERR_CUDA;
  const size_t fe = (size_t)h->n * h->N;
  // stage X into the (ld = N) layout, zero-padded columns
  CK(cudaMemsetAsync(h->buf[B_Z], 0, fe * h->esz, h->s));
  CK(cudaMemcpy2DAsync(h->buf[B_Z], h->N * h->esz, X, cols * h->esz, cols * h->esz, h->n,
                       cudaMemcpyDeviceToDevice, h->s));
  int nax = ax_A(h, h->buf[B_Z], h->buf[B_AZ], 0.0, nullptr, h->buf[B_Z], nullptr, h->pax, nullptr);
  CK(cudaMemcpy2DAsync(Y, cols * h->esz, h->buf[B_AZ], h->N * h->esz, cols * h->esz, h->n,
                       cudaMemcpyDeviceToDevice, h->s));
  std::vector<double> part((size_t)nax * h->b * kNQ);
  CK(cudaMemcpyAsync(part.data(), h->pax, part.size() * sizeof(double), cudaMemcpyDeviceToHost, h->s));
  int derr = 0;
  CK(cudaMemcpyAsync(&derr, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  if (h->tc_fail) {
    const int tf = h->tc_fail;
    h->tc_fail = 0;
    cudaGetLastError();
    return fail(h, SNMF_ERR_CUDA, "tensor-core product not launched (status " + std::to_string(tf) + ")");
  }
  CK(cudaGetLastError());
  if (derr) {
    CK(cudaMemsetAsync(h->dev_err, 0, sizeof(int), h->s));
    CK(cudaStreamSynchronize(h->s));
    return fail(h, SNMF_ERR_TIMEOUT, "a bounded device wait of the tensor-core product ran out");
  }
  if (xax) {
    double s = 0.0;
    for (int t = 0; t < nax; ++t)
      for (int j = 0; j < h->b; ++j) s += part[((size_t)t * h->b + j) * kNQ];
    *xax = s;
  }
  return SNMF_OK;
}

snmf_status snmf_profile_ax(snmf_handle h, int iters, double* ms_product, double* ms_kernel) {
  if (!h) return SNMF_ERR_STATE;
  if (iters < 1) return fail(h, SNMF_ERR_ARG, "iters must be >= 1");
  if (h->bt) {
    double ms = 0.0;
    const snmf_status st = batch_profile_ax(h->bt, iters, &ms, &h->err);
    if (ms_product) *ms_product = ms;
    if (ms_kernel) *ms_kernel = ms;
    return st;
  }
  if (iters < 1) return fail(h, SNMF_ERR_ARG, "iters must be >= 1");
  if (sync_user(h) != SNMF_OK) return SNMF_ERR_CUDA;
  const Dims d = dims(h);
  cudaEvent_t e[4];
  for (auto& x : e) CK(cudaEventCreate(&x));
  // warm-up, then the full product (kernel + epilogue) and the product kernel alone
  ax_A(h, h->buf[B_W], h->buf[B_AZ], 0.0, nullptr, h->buf[B_W], nullptr, h->pax, nullptr);
  CK(cudaEventRecord(e[0], h->s));
  for (int t = 0; t < iters; ++t)
    ax_A(h, h->buf[B_W], h->buf[B_AZ], 0.0, nullptr, h->buf[B_W], nullptr, h->pax, nullptr);
  CK(cudaEventRecord(e[1], h->s));
  float m1 = 0.f, m2 = 0.f;
  if (!h->lai) {
    CK(cudaEventRecord(e[2], h->s));
    const TcEpilogue pepi = tc_epilogue(h, h->buf[B_AZ], 0.0, nullptr, h->buf[B_W], nullptr, h->pax);
    for (int t = 0; t < iters; ++t) product_kernel(h, h->A, h->buf[B_W], h->buf[B_AZ], nullptr, &pepi);
    CK(cudaEventRecord(e[3], h->s));
  }
  CK(cudaStreamSynchronize(h->s));
  CK(cudaGetLastError());
  cudaEventElapsedTime(&m1, e[0], e[1]);
  if (!h->lai) cudaEventElapsedTime(&m2, e[2], e[3]);
  for (auto& x : e) cudaEventDestroy(x);
  (void)d;
  if (ms_product) *ms_product = m1 / iters;
  if (ms_kernel) *ms_kernel = h->lai ? 0.0 : m2 / iters;
  return SNMF_OK;
}

snmf_status snmf_profile_steps(snmf_handle h, int iters, double* ms_dstep, double* ms_update) {
  if (!h) return SNMF_ERR_STATE;
  if (h->bt) return fail(h, SNMF_ERR_STATE, "not available for a dense batch handle");
  if (iters < 1) return fail(h, SNMF_ERR_ARG, "iters must be >= 1");
  if (h->opt.formulation == SNMF_DIRECT || h->graph || h->r > 64)
    return fail(h, SNMF_ERR_ARG, "step profiling needs the penalty form without graph term and r <= 64");
  if (!h->have_result) return fail(h, SNMF_ERR_STATE, "run a solve first (the step kernels read its buffers)");
  if (sync_user(h) != SNMF_OK) return SNMF_ERR_CUDA;
  return time_steps(h, iters, ms_dstep, ms_update);
}

snmf_status snmf_tuned_config(snmf_handle h, int32_t* splits, int32_t* stages, int32_t* per_sm, double* ms,
                              int32_t* from_cache) {
  if (!h) return SNMF_ERR_STATE;
  if (!h->tuned) return fail(h, SNMF_ERR_STATE, "the handle was not autotuned");
  if (splits) *splits = h->tune.cfg.splits;
  if (stages) *stages = h->tune.cfg.stages;
  if (per_sm) *per_sm = h->tune.cfg.per_sm;
  if (ms) *ms = h->tune.ms;
  if (from_cache) *from_cache = h->tuned == 2 ? 1 : 0;
  return SNMF_OK;
}

snmf_status snmf_tuned_tiles(snmf_handle h, int32_t* bn, int32_t* row_bm) {
  if (!h) return SNMF_ERR_STATE;
  if (!h->tuned) return fail(h, SNMF_ERR_STATE, "the handle was not autotuned");
  if (bn) *bn = h->tune.cfg.bn;
  if (row_bm) *row_bm = h->tune.cfg.row_bm;
  return SNMF_OK;
}

snmf_status snmf_step_config(snmf_handle h, int32_t* body, int32_t* rows_per_cta, int64_t* dstep_bytes,
                             int64_t* update_bytes) {
  if (!h) return SNMF_ERR_STATE;
  if (h->bt) return fail(h, SNMF_ERR_STATE, "not available for a dense batch handle");
  const int64_t fb = h->n * (int64_t)h->N * (int64_t)h->esz;  // one n x (r b) factor array
  const int nc = h->opt.step_controller == 1 ? 2 : (h->opt.step_controller == 2 ? kNCand : 1);
  int kind = 0, rows = 0;
  int64_t bd = 0, bu = 0;
  if (h->use_fuse) {
    kind = h->row_tc == 2 ? 4 : (h->row_tc ? 3 : 2);
    rows = h->row_tc ? 128 : rowfuse_bm(h->r, h->row_bm);
    bd = 4 * fb;  // X, g, B in; g(Z) out
    bu = 6 * fb;  // X, g, g(Z), B in; X', g(X') out
  } else {
    kind = h->use_tile ? 1 : 0;
    const Dims d = dims(h);
    rows = h->use_tile ? (int)((h->n + rowgemm_slots(d, h->tdtype, 1) - 1) / rowgemm_slots(d, h->tdtype, 1))
                       : (int)((h->n + h->nrow / ((h->r + 63) / 64) - 1) / (h->nrow / ((h->r + 63) / 64)));
    bd = (6 + (nc == 2 ? 1 : 0)) * fb;  // X, g, B in; Z, g(Z), D (+ the second direction) out
    bu = 8 * fb;                        // Z, D, B, X, g, g(Z) in; X', g(X') out
  }
  if (body) *body = kind;
  if (rows_per_cta) *rows_per_cta = rows;
  if (dstep_bytes) *dstep_bytes = bd;
  if (update_bytes) *update_bytes = bu;
  return SNMF_OK;
}

namespace {
constexpr uint32_t kStateMagic = 0x534E4D46u;  // "SNMF"
constexpr uint32_t kStateVersion = 1;
struct StateHeader {
  uint32_t magic, version, ctl_bytes, formulation;
  int32_t batch, r;
  int64_t n;
};
}  // namespace

snmf_status snmf_get_state(snmf_handle h, void* blob, int64_t capacity, int64_t* size) {
  if (!h) return SNMF_ERR_STATE;
  if (h->bt) return fail(h, SNMF_ERR_STATE, "not available for a dense batch handle");
  const int64_t need = (int64_t)sizeof(StateHeader) + (int64_t)h->b * (int64_t)sizeof(Ctl);
  if (size) *size = need;
  if (!blob) return SNMF_OK;  // size query
  if (capacity < need) return fail(h, SNMF_ERR_ARG, "state buffer too small");
  if (!h->have_result) return fail(h, SNMF_ERR_STATE, "no solve has run on this handle");
  StateHeader hd{kStateMagic, kStateVersion, (uint32_t)sizeof(Ctl), (uint32_t)h->opt.formulation, h->b, h->r, h->n};
  std::memcpy(blob, &hd, sizeof(hd));
  std::memcpy(static_cast<unsigned char*>(blob) + sizeof(hd), h->h_ctl.data(), (size_t)h->b * sizeof(Ctl));
  return SNMF_OK;
}

snmf_status snmf_set_state(snmf_handle h, const void* blob, int64_t size) {
  if (!h) return SNMF_ERR_STATE;
  if (h->bt) return fail(h, SNMF_ERR_STATE, "not available for a dense batch handle");
  if (!blob) {
    h->resume.clear();
    return SNMF_OK;
  }
  StateHeader hd{};
  if (size < (int64_t)sizeof(hd)) return fail(h, SNMF_ERR_ARG, "state blob too small");
  std::memcpy(&hd, blob, sizeof(hd));
  if (hd.magic != kStateMagic || hd.version != kStateVersion || hd.ctl_bytes != sizeof(Ctl))
    return fail(h, SNMF_ERR_ARG, "not a state blob of this library version");
  if (hd.batch != h->b || hd.r != h->r || hd.n != h->n || (int)hd.formulation != h->opt.formulation)
    return fail(h, SNMF_ERR_ARG, "state of another problem shape or formulation");
  if (size < (int64_t)sizeof(hd) + (int64_t)h->b * (int64_t)sizeof(Ctl)) return fail(h, SNMF_ERR_ARG, "state truncated");
  h->resume.resize(h->b);
  std::memcpy(h->resume.data(), static_cast<const unsigned char*>(blob) + sizeof(hd), (size_t)h->b * sizeof(Ctl));
  for (auto& c : h->resume) {
    // a restart that had stopped at the tolerance stays stopped; the others continue
    const bool conv = c.pg0 == 0.0 || c.pg <= h->opt.tol * c.pg0;
    c.active = (!conv && !c.nan_seen) ? 1 : 0;
  }
  return SNMF_OK;
}

snmf_status snmf_stats_ring(snmf_handle h, double* out, int capacity, int32_t* count) {
  if (!h) return SNMF_ERR_STATE;
  if (h->bt) return fail(h, SNMF_ERR_STATE, "not available for a dense batch handle");
  if (!out || capacity < 1) return fail(h, SNMF_ERR_ARG, "bad ring arguments");
  const int cap = std::min(capacity, h->ring_cap);
  std::vector<double> buf((size_t)h->b * h->ring_cap * kRingVals);
  CK(cudaMemcpyAsync(buf.data(), h->ring, buf.size() * sizeof(double), cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  int kept = 0;
  for (int j = 0; j < h->b; ++j) {
    const int iters = j < (int)h->h_ctl.size() ? h->h_ctl[j].iters : 0;
    const int have = std::min(std::min(iters + 1, h->ring_cap), cap);  // records 0 .. iters
    for (int t = 0; t < cap; ++t) {
      double* dst = out + ((int64_t)j * cap + t) * kRingVals;
      if (t < have) {
        const int it = iters + 1 - have + t;
        const double* src = buf.data() + ((int64_t)j * h->ring_cap + (it % h->ring_cap)) * kRingVals;
        std::memcpy(dst, src, kRingVals * sizeof(double));
      } else {
        for (int v = 0; v < kRingVals; ++v) dst[v] = -1.0;
      }
    }
    kept = std::max(kept, have);
  }
  if (count) *count = kept;
  return SNMF_OK;
}

snmf_status snmf_cluster_assign(snmf_handle h, int restart, int32_t* labels) {
  if (!h) return SNMF_ERR_STATE;
  if (h->bt) return fail(h, SNMF_ERR_STATE, "not available for a dense batch handle");
  if (!labels || restart < 0 || restart >= h->b) return fail(h, SNMF_ERR_ARG, "bad cluster_assign arguments");
  if (!h->have_result) return fail(h, SNMF_ERR_STATE, "no solve has run on this handle");
  // the paper's reading: cluster of point i = argmax over the columns of its H row
  const void* F = h->buf[h->opt.formulation == SNMF_PENALTY ? B_HT : B_W];
  launch_assign(h->tdtype, F, h->n, h->N, (int64_t)restart * h->r, h->r, labels, h->s);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->s));
  return SNMF_OK;
}

snmf_status snmf_set_timeout(snmf_handle h, int64_t cycles) {
  if (!h) return SNMF_ERR_STATE;
  if (cycles < 0) return fail(h, SNMF_ERR_ARG, "cycles must be >= 0");
  const long long c = cycles > 0 ? (long long)cycles : 2000000000LL;
  h->opt.timeout_cycles = cycles;
  h->budget = c;
  h->exec_form = -1;  // the captured solve graphs hold the old budget: capture again
  if (h->bt) batch_set_budget(h->bt, c);
  return SNMF_OK;
}

snmf_status snmf_controller_data(snmf_handle h, float* feat, float* targ, int capacity, int32_t* count) {
  if (!h) return SNMF_ERR_STATE;
  if (h->bt) return fail(h, SNMF_ERR_STATE, "not available for a dense batch handle");
  if (h->opt.step_controller != 2 && h->opt.step_controller != 4)
    return fail(h, SNMF_ERR_STATE, "the handle is not in record mode");
  if (capacity < 0 || (capacity > 0 && (!feat || !targ))) return fail(h, SNMF_ERR_ARG, "bad buffers");
  int cnt = 0;
  CK(cudaMemcpyAsync(&cnt, h->rec_count, sizeof(int), cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  cnt = std::min(cnt, h->rec_cap);
  const int m = std::min(cnt, capacity);
  if (m > 0) {
    CK(cudaMemcpyAsync(feat, h->rec_feat, (size_t)m * kMlpIn * sizeof(float), cudaMemcpyDeviceToHost, h->s));
    CK(cudaMemcpyAsync(targ, h->rec_targ, (size_t)m * sizeof(float), cudaMemcpyDeviceToHost, h->s));
  }
  CK(cudaMemsetAsync(h->rec_count, 0, sizeof(int), h->s));
  CK(cudaStreamSynchronize(h->s));
  if (count) *count = m;
  return SNMF_OK;
}

snmf_status snmf_destroy(snmf_handle h) {
  if (!h) return SNMF_OK;
  if (h->bt) {
    batch_destroy(h->bt);
    delete h;
    return SNMF_OK;
  }
  if (h->s) cudaStreamSynchronize(h->s);
  if (h->s2) cudaStreamSynchronize(h->s2);
  for (auto& e : h->exec)
    if (e) cudaGraphExecDestroy(e);
  if (h->evdone) cudaEventDestroy(h->evdone);
  for (void* p : h->buf) cudaFree(p);
  cudaFree(h->ws);
  double* parts[] = {h->prow, h->pax, h->pax2, h->pax3, h->pax4, h->pclip, h->gpart, h->G64fix,
                     h->G64p, h->dsc, h->ring};
  for (double* p : parts) cudaFree(p);
  cudaFree(h->GT);
  cudaFree(h->ctl);
  cudaFree(h->run);
  cudaFree(h->recompute);
  cudaFree(h->counters);
  cudaFree(h->dev_err);
  cudaFree(h->xh);
  cudaFree(h->xl);
  cudaFree(h->tcount);
  cudaFree(h->mlp_w);
  cudaFree(h->rec_feat);
  cudaFree(h->rec_targ);
  cudaFree(h->rec_count);
  if (h->h_flag) cudaFreeHost(h->h_flag);
  cudaFree(h->A_owned);
  cudaFree(h->A_scale);
  cudaFree(h->rowptr_owned);
  cudaFree(h->colidx_owned);
  cudaFree(h->vals_owned);
  cudaFree(h->L_rowptr);
  cudaFree(h->L_colidx);
  cudaFree(h->L_vals);
  cudaFree(h->L_scale);
  lai_free(h->lai_op);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->evsync) cudaEventDestroy(h->evsync);
  if (h->evfork) cudaEventDestroy(h->evfork);
  if (h->evjoin) cudaEventDestroy(h->evjoin);
  if (h->s2) cudaStreamDestroy(h->s2);
  if (h->s) cudaStreamDestroy(h->s);
  delete h;
  return SNMF_OK;
}

const char* snmf_last_error(snmf_handle h) {
  if (!h) return g_create_err.c_str();
  return h->err.c_str();
}

}  // extern "C"
