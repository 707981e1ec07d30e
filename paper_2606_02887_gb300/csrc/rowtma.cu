// Row kernels of an Algorithm-1 step (the D step and the update: the same arithmetic as
// rowtc.cu, bit for bit per element), persistent and warp-specialised, for FP32 penalty blocks
// with r = 64.
//
// Work unit: a tile of 128 rows of one restart (its 64 columns).  One CTA of 16 warps per SM
// walks a contiguous range of tiles.  Thread (w, lane) owns row m = 32 (w % 4) + lane of the
// tile and the 16 columns 16 (w / 4) .. + 15: TMEM lanes warp w may read, so the accumulators go
// from TMEM straight into registers; four warps per SM sub-partition hide the latency of the
// elementwise work, and 16 warps leave 128 registers a thread (a 17th warp would put five warps
// on one sub-partition and cap every thread at 96).  Thread 32 is the producer: the input slots
// are freed at the warps' votes, so it issues the TMA loads of the next tiles into a ring of
// four 32 KB shared slots (two 128 x 32 boxes each, 128-byte swizzle: the K-major layout of the
// UMMA operand tiles) as soon as a slot frees, one full-barrier per slot, and it issues the TMA
// stores; thread 0, in another warp, issues the MMAs.  A tile's statistics are summed over the
// warps (fixed order) by warp 0 after the next named-barrier vote; a CTA takes one arrival ticket per run of consecutive tiles of a
// restart, and runs the control step of each restart whose last run it completed after its
// tile range.  A restart's control scalars are read once per run.
// Row products on tcgen05 kind::tf32 with TF32 hi + lo parts (three MMAs per K step).
// Outputs leave through shared memory by TMA stores (rows past n are not written).
// Every wait is bounded: one that runs out records an error code; the warps leave the tile
// loop together at their next vote, zero partials keep the arrival counters consistent, and
// the CTA drains the copies and products it issued and frees TMEM.
#include <math.h>

#include "ax_tc.cuh"
#include "common.cuh"
#include "rowops.cuh"
#include "rowops_dev.cuh"
#include "tc_dev.cuh"

namespace snmf {

namespace {

using namespace tc;

constexpr int TR = 128;                        // rows per tile (UMMA M)
constexpr int RC = 64;                         // columns (r, UMMA N = K)
constexpr uint32_t SLOT = TR * RC * 4;         // 32 KB: one FP32 array tile
constexpr uint32_t BOX = SLOT / 2;             // 16 KB: one 128 x 32 box (an operand atom column)
constexpr int NSLOT = 4;
constexpr uint32_t G_PART = RC * RC * 4;       // 16 KB: one TF32 part of G
constexpr uint32_t OFF_AH = 0, OFF_AL = SLOT;  // operand tile parts (also output staging)
constexpr uint32_t OFF_GH = 2 * SLOT, OFF_GL = 2 * SLOT + G_PART;
constexpr uint32_t OFF_SLOT = 2 * SLOT + 2 * G_PART;
constexpr uint32_t DYN_BYTES = OFF_SLOT + NSLOT * SLOT + 1024;  // + alignment slack
constexpr int NCWARP = 16;  // warps (all compute)
constexpr int NCOMP = NCWARP * 32;
constexpr int NTHR = NCOMP;
constexpr int kMaxTodo = 32;  // runs of one CTA's tile range (the launcher checks the range length)
constexpr uint32_t kTmemCols = 512;  // two products of three 64-column accumulators (D step)
constexpr uint32_t kProd2 = 256;     // TMEM column of the D step's second product
constexpr long long kBudget = 2000000000LL;  // clock64 cycles of one wait
constexpr long long kDrain = 2000000000LL;   // of one wait on the error path

// error codes (err): 31 input slot not filled, 32 product not completed
struct RowMaps {
  CUtensorMap m[4];
};

struct RowSmem {
  uint64_t full[NSLOT], mma;
  uint32_t tmem;
  int abort;
  int ntodo;
  int todo[kMaxTodo];
  float dqs[NCWARP][8];
};

__device__ __forceinline__ bool aborted(const RowSmem& S) { return *(const volatile int*)&S.abort != 0; }

__device__ __forceinline__ void set_abort(RowSmem& S, int* err, int code) {
  if (err) atomicCAS(err, 0, code);
  *(volatile int*)&S.abort = 1;
}

// byte offset of the 16-byte chunk holding columns 4 c .. 4 c + 3 (c < 16) of row m in a
// 128 x 64 FP32 tile stored as two 128 x 32 boxes with the 128-byte swizzle
__device__ __forceinline__ uint32_t chunk_off(int m, int c) {
  return (uint32_t)((c >> 3) * BOX + m * 128 + (((c & 7) ^ (m & 7)) << 4));
}

__device__ __forceinline__ void put4(unsigned char* hi, unsigned char* lo, uint32_t off, float a, float b, float c,
                                     float d) {
  const uint32_t h0 = to_tf32(a), h1 = to_tf32(b), h2 = to_tf32(c), h3 = to_tf32(d);
  const uint32_t l0 = to_tf32(a - __uint_as_float(h0)), l1 = to_tf32(b - __uint_as_float(h1)),
                 l2 = to_tf32(c - __uint_as_float(h2)), l3 = to_tf32(d - __uint_as_float(h3));
  *reinterpret_cast<uint4*>(hi + off) = make_uint4(h0, h1, h2, h3);
  *reinterpret_cast<uint4*>(lo + off) = make_uint4(l0, l1, l2, l3);
}

__device__ __forceinline__ float4 lds4(const unsigned char* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void sts4(unsigned char* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}

__device__ __forceinline__ float zstep1(float x, float g, float inv_rho) {
  const float t = __fmaf_rn(-g, inv_rho, x);
  return t > 0.f ? t : 0.f;
}
__device__ __forceinline__ float dir1(float z, float gz, float alpha) {
  const float t = __fmaf_rn(-alpha, gz, z);
  return (t > 0.f ? t : 0.f) - z;
}
__device__ __forceinline__ float upd1(float z, float d, float pb) {
  const float t = __fmaf_rn(pb, d, z);
  return t > 0.f ? t : 0.f;
}

// G of restart j as the B operand's TF32 hi / lo parts (K-major: row n holds G[k][n] = G[n][k]);
// by the NCOMP = 512 compute threads, two chunks each
__device__ __forceinline__ void load_gram(const float* G, unsigned char* gh, unsigned char* gl) {
  static_assert(NCOMP == 512, "G is split by 512 threads");
  const int n = threadIdx.x >> 3, k0 = (threadIdx.x & 7) * 8;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int k = k0 + 4 * c;
    const float4 v = *reinterpret_cast<const float4*>(G + n * RC + k);
    const int atom = k >> 5, ch = (k & 31) >> 2;
    put4(gh, gl, (uint32_t)(atom * RC * 128 + n * 128 + ((ch ^ (n & 7)) << 4)), v.x, v.y, v.z, v.w);
  }
}

// The 24 MMAs of one 128 x 64 x 64 product as three independent accumulation chains (A_lo G_hi,
// A_hi G_lo, A_hi G_hi into TMEM columns tcol, tcol + 64, tcol + 128), interleaved so that
// consecutive MMAs do not wait on one another; the epilogue adds the three.
__device__ __forceinline__ void issue_product(uint32_t ah, uint32_t al, uint32_t bh, uint32_t bl, uint32_t tcol) {
  const uint32_t idesc = idesc_tf32(TR, RC);
#pragma unroll
  for (int kk = 0; kk < RC / 8; ++kk) {
    const uint32_t ao = (kk >> 2) * BOX + (kk & 3) * 32;
    const uint32_t bo = (kk >> 2) * (RC * 128) + (kk & 3) * 32;
    const uint32_t acc = kk > 0 ? 1u : 0u;
    mma_tf32(tcol, sdesc_sw128(al + ao), sdesc_sw128(bh + bo), idesc, acc);
    mma_tf32(tcol + 64, sdesc_sw128(ah + ao), sdesc_sw128(bl + bo), idesc, acc);
    mma_tf32(tcol + 128, sdesc_sw128(ah + ao), sdesc_sw128(bh + bo), idesc, acc);
  }
}

// this thread's 16 accumulator columns of a product at TMEM column `col`: the three chains
// summed (small terms first)
__device__ __forceinline__ void load_product(uint32_t taddr, float* v) {
  tmem_ld16(taddr, v);
  tmem_ld8_add(taddr + 64, v);
  tmem_ld8_add(taddr + 64 + 8, v + 8);
  tmem_ld8_add(taddr + 128, v);
  tmem_ld8_add(taddr + 128 + 8, v + 8);
}

__device__ __forceinline__ bool restart_live(const RowArgs& a, int j) {
  return a.ctl[j].active && !(a.run && *a.run == 0);
}

// Producer state of thread 32: the next load (tile ct, array ca, ring index q) and the busy slots.
struct Loader {
  int ct, ca, q, lj;
  bool llive;
  unsigned busy;
};

// Issue loads in ring order while the next load's slot is free (thread 0).
template <int NARR>
__device__ __forceinline__ void issue_loads(Loader& L, const RowMaps& maps, const RowArgs& a, RowSmem& S,
                                            unsigned char* base, int t1, int RT) {
  while (L.ct < t1) {
    const int j = L.ct / RT;
    if (j != L.lj) {
      L.lj = j;
      L.llive = restart_live(a, j);
    }
    if (!L.llive) {
      ++L.ct;
      L.ca = 0;
      continue;
    }
    const int s = L.q % NSLOT;
    if (L.busy & (1u << s)) return;
    L.busy |= 1u << s;
    unsigned char* dst = base + OFF_SLOT + (uint32_t)s * SLOT;
    const int rt = L.ct % RT;
    mbar_arrive_expect_tx(&S.full[s], SLOT);
    tma_load_2d(dst, &maps.m[L.ca], &S.full[s], j * RC, rt * TR);
    tma_load_2d(dst + BOX, &maps.m[L.ca], &S.full[s], j * RC + 32, rt * TR);
    ++L.q;
    if (++L.ca == NARR) {
      L.ca = 0;
      ++L.ct;
    }
  }
}

// Partials and arrival tickets (warp 0).  Partials are written in tile order; a run of
// consecutive tiles of one restart takes one ticket (an atomic add of its length) once all its
// partials are written; the CTA that completes a restart records it for its control step.
struct Tickets {
  int run_j, run_n;
};

__device__ __forceinline__ void take_ticket(const RowArgs& a, RowSmem& S, const Tickets& T, int RT, int lane) {
  __syncwarp();
  __threadfence();
  __syncwarp();
  if (lane == 0) {
    const unsigned old = atomicAdd(&a.counters[T.run_j], (unsigned)T.run_n);
    if (old + (unsigned)T.run_n == (unsigned)RT) S.todo[S.ntodo++] = T.run_j;  // <= one per run
  }
}

// partial of tile (rt, j): v on lanes 0 .. 7 (warp 0)
__device__ __forceinline__ void write_partial(const RowArgs& a, RowSmem& S, Tickets& T, int rt, int j, float v,
                                              int RT, int lane) {
  if (T.run_j >= 0 && j != T.run_j) {
    take_ticket(a, S, T, RT, lane);
    T.run_n = 0;
  }
  T.run_j = j;
  ++T.run_n;
  if (lane < 8) a.part[((int64_t)rt * a.b + j) * kNQ + lane] = (double)v;
}

// the statistics the warps left in S.dqs, summed in warp order (warp 0, after a barrier)
__device__ __forceinline__ float sum_dqs(const RowSmem& S, int lane) {
  float v = 0.f;
  if (lane < 8) {
#pragma unroll
    for (int w = 0; w < NCWARP; ++w) v += S.dqs[w][lane];
  }
  return v;
}

// each warp's sums of its threads' statistics into S.dqs
__device__ __forceinline__ void leave_dq(RowSmem& S, const float (&dq)[8], int warp, int lane) {
  float v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = warp_sum(dq[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < 8; ++q) S.dqs[warp][q] = v[q];
  }
}

// D step (KIND 0): inputs X, g, B; g(Z) out; q0 <g(Z), D>, q1 ||D||^2, q2 f(Z) - f(X),
// q4 <D G, D>.  Update (KIND 1): inputs X, g, g(Z), B; X', g(X') out in place; q0
// ||P grad f(X')||^2, q1 1/2 <g' - B, X'>, q2 <S,S>, q3 <S,Y>, q4 <Y,Y>, q5 f(X') - f(Z), q6 zero
// entries of X'.
template <int KIND>
__global__ void __launch_bounds__(NTHR, 1) k_rowtma(const __grid_constant__ RowMaps maps, RowArgs a, int* err) {
  constexpr int NARR = KIND == 0 ? 3 : 4;  // input arrays per tile
  constexpr int E = 16;                     // elements per thread: one row, 16 columns
  extern __shared__ unsigned char tma_raw[];
  __shared__ RowSmem S;
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tma_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int RT = (int)((a.n + TR - 1) / TR);
  const int T = RT * a.b;
  const int t0 = (int)((int64_t)blockIdx.x * T / gridDim.x);
  const int t1 = (int)((int64_t)(blockIdx.x + 1) * T / gridDim.x);
  const bool lead = threadIdx.x == 0;   // MMAs, partials and tickets (warp 0)
  const bool tmat = threadIdx.x == 32;  // TMA loads and stores, slot bookkeeping (warp 1)
  if (lead) {
    for (int s = 0; s < NSLOT; ++s) mbar_init(&S.full[s], 1);
    mbar_init(&S.mma, 1);
    S.abort = 0;
    S.ntodo = 0;
    mbar_init_fence();
  }
  if (warp == 0) tmem_alloc(&S.tmem, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem;
  const int m = 32 * (warp & 3) + lane, cq = warp >> 2;  // row, column quarter
  const uint32_t tl = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + 16 * cq;  // this thread's accumulator
  unsigned char* AH = base + OFF_AH;
  unsigned char* AL = base + OFF_AL;
  unsigned char* GH = base + OFF_GH;
  unsigned char* GL = base + OFF_GL;
  const uint32_t ah = smem_u32(AH), al = smem_u32(AL), gh = smem_u32(GH), gl = smem_u32(GL);

  Loader L{t0, 0, 0, -1, false, 0u};  // TMA thread
  int p_used = 0, pend = -1;           // TMA thread
  int mma_issued = 0, mma_seen = 0;    // thread 0
  if (tmat) issue_loads<NARR>(L, maps, a, S, base, t1, RT);
  Tickets tk{-1, 0};                  // warp 0
  bool have_dq = false;               // warp 0: the previous live tile's statistics wait in S.dqs
  int dq_rt = 0, dq_j = 0;
  int next_partial = t0;              // warp 0: first tile whose partial is not written

  int p = 0, nmma = 0, gj = -1, cj_idx = -1;
  bool live = false;
  float inv_rho = 0.f, alpha = 0.f, pb = 0.f;
  bool bad = false;
  auto slot = [&](int q) { return base + OFF_SLOT + (uint32_t)(q % NSLOT) * SLOT; };
  auto wait_full = [&](int q) {
    const bool ok = mbar_wait(&S.full[q % NSLOT], (uint32_t)((q / NSLOT) & 1), kBudget, &S.abort);
    if (!ok && !aborted(S)) set_abort(S, err, 31);
    if (ok && tmat) p_used = q + 1;
    return ok;
  };
  auto wait_mma = [&]() {
    const bool ok = mbar_wait(&S.mma, (uint32_t)((nmma - 1) & 1), kBudget, &S.abort);
    if (!ok && !aborted(S)) set_abort(S, err, 32);
    if (ok && lead) mma_seen = nmma;
    tc_fence_after();
    return ok;
  };
  auto release = [&](int q) { L.busy &= ~(1u << (q % NSLOT)); };
  // warp 0 after a vote: the previous live tile's statistics to its partial
  auto flush = [&]() {  // every thread tracks have_dq alike; warp 0 writes
    if (have_dq) {
      if (warp == 0) {
        write_partial(a, S, tk, dq_rt, dq_j, sum_dqs(S, lane), RT, lane);
        ++next_partial;
      }
      have_dq = false;
    }
  };
  for (int t = t0; t < t1; ++t) {
    const int j = t / RT, rt = t % RT;
    const int64_t row0 = (int64_t)rt * TR;
    const bool rv = row0 + m < a.n;
    if (j != cj_idx) {  // the restart's scalars stay fixed until its last tile has arrived
      cj_idx = j;
      live = restart_live(a, j);
      const Ctl& cj = a.ctl[j];
      inv_rho = (float)(1.0 / cj.rho);
      alpha = (float)cj.alpha;
      pb = (float)cj.phibeta;
    }
    if (!live) {
      if (have_dq) __syncthreads();  // the warps' statistics of the previous tile are in S.dqs
      flush();
      if (warp == 0) {
        write_partial(a, S, tk, rt, j, 0.f, RT, lane);
        ++next_partial;
      }
      continue;
    }
    float dq[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) dq[q] = 0.f;
    const int x0 = j * RC, y0 = (int)row0;
    if (KIND == 0) {
      // ---- D step ----
      unsigned char* sX = slot(p);
      unsigned char* sG = slot(p + 1);
      unsigned char* sB = slot(p + 2);
      bad |= !wait_full(p);
      bad |= !wait_full(p + 1);
      float x[E], g[E];
#pragma unroll
      for (int c2 = 0; c2 < 4; ++c2) {
        const uint32_t off = chunk_off(m, 4 * cq + c2);
        const float4 xv = lds4(sX + off), gv = lds4(sG + off);
        x[4 * c2] = xv.x; x[4 * c2 + 1] = xv.y; x[4 * c2 + 2] = xv.z; x[4 * c2 + 3] = xv.w;
        g[4 * c2] = gv.x; g[4 * c2 + 1] = gv.y; g[4 * c2 + 2] = gv.z; g[4 * c2 + 3] = gv.w;
      }
      if (j != gj) {
        load_gram((const float*)a.G + (int64_t)j * RC * RC, GH, GL);
        gj = j;
      }
#pragma unroll
      for (int c2 = 0; c2 < 4; ++c2)
        put4(AH, AL, chunk_off(m, 4 * cq + c2), zstep1(x[4 * c2], g[4 * c2], inv_rho),
             zstep1(x[4 * c2 + 1], g[4 * c2 + 1], inv_rho), zstep1(x[4 * c2 + 2], g[4 * c2 + 2], inv_rho),
             zstep1(x[4 * c2 + 3], g[4 * c2 + 3], inv_rho));
      fence_proxy_async();
      tc_fence_before();
      bad = bar_vote_or(1, NCOMP, bad || aborted(S));
      if (bad) break;
      flush();
      if (lead) {
        tc_fence_after();
        issue_product(ah, al, gh, gl, tmem);  // Z G
        mma_commit(&S.mma);
        mma_issued = nmma + 1;
      }
      if (tmat) {
        release(p);
        release(p + 1);
        if (pend >= 0) {  // the previous tile's g(Z) store has long read its slot
          bulk_wait_read_all();
          release(pend);
          pend = -1;
        }
        issue_loads<NARR>(L, maps, a, S, base, t1, RT);
      }
      ++nmma;
      bad |= !wait_mma();
      bad |= !wait_full(p + 2);
      float acc[E];
      load_product(tl, acc);
      // the elementwise values are recomputed from x and g (not kept from before the product)
#pragma unroll
      for (int i = 0; i < E; ++i) asm volatile("" : "+f"(x[i]), "+f"(g[i]));
      float d[E];
#pragma unroll
      for (int c2 = 0; c2 < 4; ++c2) {
        const uint32_t off = chunk_off(m, 4 * cq + c2);
        const float4 bv = lds4(sB + off);
        const float bs[4] = {bv.x, bv.y, bv.z, bv.w};
        float gz[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int i = 4 * c2 + e;
          const float z = zstep1(x[i], g[i], inv_rho);
          gz[e] = acc[i] - bs[e];
          const float dv = rv ? dir1(z, gz[e], alpha) : 0.f;
          if (rv) {
            dq[0] += gz[e] * dv;
            dq[1] += dv * dv;
            dq[2] += 0.5f * (z - x[i]) * (gz[e] + g[i]);
          }
          d[i] = dv;
        }
        sts4(sB + off, gz[0], gz[1], gz[2], gz[3]);  // g(Z) staged in place of B
        put4(AH, AL, off, d[4 * c2], d[4 * c2 + 1], d[4 * c2 + 2], d[4 * c2 + 3]);
      }
      fence_proxy_async();
      tc_fence_before();
      bad = bar_vote_or(1, NCOMP, bad || aborted(S));
      if (bad) break;
      if (lead) {
        tc_fence_after();
        issue_product(ah, al, gh, gl, tmem + kProd2);  // D G
        mma_commit(&S.mma);
        mma_issued = nmma + 1;
      }
      if (tmat) {
        tma_store_2d(&maps.m[3], sB, x0, y0);
        tma_store_2d(&maps.m[3], sB + BOX, x0 + 32, y0);
        bulk_commit();
        pend = (p + 2);  // freed at the next tile's first vote
      }
      ++nmma;
      p += 3;
      bad |= !wait_mma();
      float dg[E];
      load_product(tl + kProd2, dg);
      float qq = 0.f;
#pragma unroll
      for (int i = 0; i < E; ++i) qq = fmaf(dg[i], d[i], qq);
      dq[4] = qq;
      tc_fence_before();
    } else {
      // ---- update ----
      unsigned char* sX = slot(p);
      unsigned char* sG = slot(p + 1);
      unsigned char* sZ = slot(p + 2);
      unsigned char* sB = slot(p + 3);
      bad |= !wait_full(p);
      bad |= !wait_full(p + 1);
      bad |= !wait_full(p + 2);
      float x[E], g[E], gzo[E];
#pragma unroll
      for (int c2 = 0; c2 < 4; ++c2) {
        const uint32_t off = chunk_off(m, 4 * cq + c2);
        const float4 xv = lds4(sX + off), gv = lds4(sG + off), zv = lds4(sZ + off);
        x[4 * c2] = xv.x; x[4 * c2 + 1] = xv.y; x[4 * c2 + 2] = xv.z; x[4 * c2 + 3] = xv.w;
        g[4 * c2] = gv.x; g[4 * c2 + 1] = gv.y; g[4 * c2 + 2] = gv.z; g[4 * c2 + 3] = gv.w;
        gzo[4 * c2] = zv.x; gzo[4 * c2 + 1] = zv.y; gzo[4 * c2 + 2] = zv.z; gzo[4 * c2 + 3] = zv.w;
      }
      if (j != gj) {
        load_gram((const float*)a.G + (int64_t)j * RC * RC, GH, GL);
        gj = j;
      }
      if (tmat) bulk_wait_read_all();  // the previous tile's outputs have left the operand tile
      bad = bar_vote_or(1, NCOMP, bad || aborted(S));
      if (bad) break;
      flush();
#pragma unroll
      for (int c2 = 0; c2 < 4; ++c2) {
        float xn[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int i = 4 * c2 + e;
          const float z = zstep1(x[i], g[i], inv_rho);
          xn[e] = upd1(z, dir1(z, gzo[i], alpha), pb);
        }
        put4(AH, AL, chunk_off(m, 4 * cq + c2), xn[0], xn[1], xn[2], xn[3]);
      }
      fence_proxy_async();
      tc_fence_before();
      bad = bar_vote_or(1, NCOMP, bad || aborted(S));
      if (bad) break;
      if (lead) {
        tc_fence_after();
        issue_product(ah, al, gh, gl, tmem);  // X' G
        mma_commit(&S.mma);
        mma_issued = nmma + 1;
      }
      if (tmat) {
        release(p);
        release(p + 1);
        release(p + 2);
        issue_loads<NARR>(L, maps, a, S, base, t1, RT);
      }
      ++nmma;
      bad |= !wait_mma();
      bad |= !wait_full(p + 3);
      float acc[E];
      load_product(tl, acc);
      tc_fence_before();
      // the elementwise values are recomputed from x, g, g(Z) (not kept from before the product)
#pragma unroll
      for (int i = 0; i < E; ++i) asm volatile("" : "+f"(x[i]), "+f"(g[i]), "+f"(gzo[i]));
#pragma unroll
      for (int c2 = 0; c2 < 4; ++c2) {
        const uint32_t off = chunk_off(m, 4 * cq + c2);
        const float4 bv = lds4(sB + off);
        const float bs[4] = {bv.x, bv.y, bv.z, bv.w};
        float xo[4], go[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int i = 4 * c2 + e;
          const float z = zstep1(x[i], g[i], inv_rho);
          const float xn = upd1(z, dir1(z, gzo[i], alpha), pb);
          const float gn = acc[i] - bs[e];
          if (rv) {
            const float pgv = xn > 0.f ? gn : (gn < 0.f ? gn : 0.f);
            dq[0] += pgv * pgv;
            dq[1] += 0.5f * (gn - bs[e]) * xn;
            const float sv = xn - x[i], yv = gn - g[i];
            dq[2] += sv * sv;
            dq[3] += sv * yv;
            dq[4] += yv * yv;
            dq[5] += 0.5f * (xn - z) * (gn + gzo[i]);
            if (xn == 0.f) dq[6] += 1.f;
          }
          xo[e] = xn;
          go[e] = gn;
        }
        // X' and g(X') staged in the operand tile (its product has completed)
        sts4(AH + off, xo[0], xo[1], xo[2], xo[3]);
        sts4(AL + off, go[0], go[1], go[2], go[3]);
      }
      fence_proxy_async();
      bad = bar_vote_or(1, NCOMP, bad || aborted(S));
      if (bad) break;
      if (tmat) {
        tma_store_2d(&maps.m[0], AH, x0, y0);
        tma_store_2d(&maps.m[0], AH + BOX, x0 + 32, y0);
        tma_store_2d(&maps.m[1], AL, x0, y0);
        tma_store_2d(&maps.m[1], AL + BOX, x0 + 32, y0);
        bulk_commit();
        release(p + 3);
        issue_loads<NARR>(L, maps, a, S, base, t1, RT);
      }
      p += 4;
    }
    leave_dq(S, dq, warp, lane);
    have_dq = true;
    dq_rt = rt;
    dq_j = j;
  }
  // the last live tile's statistics, zero partials for tiles an abort left, the last run's
  // ticket, then the control steps of the restarts this CTA completed
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    if (have_dq && !aborted(S)) {
      write_partial(a, S, tk, dq_rt, dq_j, sum_dqs(S, lane), RT, lane);
      ++next_partial;
    }
    for (int t = next_partial; t < t1; ++t) write_partial(a, S, tk, t % RT, t / RT, 0.f, RT, lane);
    if (tk.run_j >= 0) take_ticket(a, S, tk, RT, lane);
    __syncwarp();
    for (int u = 0; u < S.ntodo; ++u) {
      const int jj = S.todo[u];
      if (lane == 0) a.counters[jj] = 0u;  // ready for the next launch
      fused_control(a.ctl_mode, const_cast<Ctl&>(a.ctl[jj]), a.part, RT, a.b, a.r, jj, a.P, a.G64fix, nullptr, 1);
    }
  }
  // drain after an abort: products committed but not seen complete, loads not consumed
  if (lead && aborted(S) && mma_issued > mma_seen) mbar_wait(&S.mma, (uint32_t)((mma_issued - 1) & 1), kDrain);
  if (tmat) {
    if (aborted(S))
      for (int q = p_used; q < L.q; ++q) mbar_wait(&S.full[q % NSLOT], (uint32_t)((q / NSLOT) & 1), kDrain);
    bulk_wait_all();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
  }
  return n;
}

template <int KIND>
bool launch_kind(const RowArgs& a, const void* const* arrays, int* err, cudaStream_t s) {
  RowMaps maps;
  for (int q = 0; q < 4; ++q)
    if (!make_map_f32_tile(&maps.m[q], arrays[q], a.ld, a.n, a.ld)) return false;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_rowtma<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DYN_BYTES) !=
        cudaSuccess)
      return false;
    attr = true;
  }
  const int64_t T = ((a.n + TR - 1) / TR) * a.b;
  const int grid = (int)(T < sm_count() ? T : sm_count());
  if ((T + grid - 1) / grid > kMaxTodo) return false;  // a range could hold more runs than the list
  k_rowtma<KIND><<<grid, NTHR, DYN_BYTES, s>>>(maps, a, err);
  return true;
}

}  // namespace

bool rowtma_supported(int tdtype, int r, int nc, int64_t ld) {
  return tdtype == 1 && r == RC && nc == 1 && ld % 4 == 0 && ld <= (int64_t)1 << 31;
}

bool launch_rowtma_dstep(const RowArgs& a, int* err, cudaStream_t s) {
  const void* arrays[4] = {a.X, a.g_in, a.B, a.gZout};
  return launch_kind<0>(a, arrays, err, s);
}

bool launch_rowtma_update(const RowArgs& a, int* err, cudaStream_t s) {
  const void* arrays[4] = {a.Xout, a.gout, a.gZold, a.B};
  return launch_kind<1>(a, arrays, err, s);
}

}  // namespace snmf
