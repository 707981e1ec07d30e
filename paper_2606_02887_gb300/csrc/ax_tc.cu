// Tensor-core A*X product for BF16 A on sm_103a (tcgen05 + TMA + TMEM).
//
//   Y (FP32, n x N) = A_bf16 X_hi + A_bf16 X_lo, with X_hi = bf16(X), X_lo = bf16(X - X_hi):
//   the product sees X to about 2^-17 relative while A stays in BF16 (half the HBM bytes of
//   FP32).  Both operands are K-major: A row-major (n x lda), the X parts transposed
//   (N x ldk) by k_split_x.  Tiles: BM = 128 rows (UMMA M = 128, cta_group::1), BN columns
//   (16..256), BK = 64 (one 128-byte swizzle atom).
//
//   warp 0 lane 0 : TMA producer, ring of `stages` (A tile + two X tiles) with full/empty
//                   mbarriers
//   warp 1 lane 0 : MMA issuer: per stage 4 K-steps x (hi, lo) tcgen05.mma into one TMEM
//                   accumulator, tcgen05.commit frees the stage
//   warps 0-3     : epilogue: tcgen05.ld 32 rows each, store FP32 rows (split-K slice or Y)
//
// E4M3 A (k_gemm_tc<true>): a ring stage holds the 128 x 64 code tile (unswizzled) and the X
// parts; warps 2-3 decode the codes, times the power-of-two scale of their 128 x 128 tile of
// A, into one of two BF16 A buffers outside the ring, in the layout the 128-byte swizzle gives
// (the decode is exact: an E4M3 value times 2^k has at most 4 significant bits).  The MMA
// issuer waits for the stage's TMA bytes and for the decoded buffer, and frees the buffer with
// a commit.  The MMAs and the epilogue are the BF16 kernel's.
//
// Every mbarrier wait is bounded by a clock64 budget; on expiry the kernel records an
// error code, stops issuing, releases its TMEM and returns (no unbounded spin).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <mutex>

#include "ax_tc.cuh"
#include "common.cuh"
#include "fp8.cuh"

namespace snmf {

namespace {

constexpr int BM = 128, BK = 64;
constexpr int kMaxChain = 32;  // K tiles accumulated in one TMEM accumulator at most
// Budget (clock64 cycles, about 2 s at 2 GHz) of the drain on the error path: after a wait
// ran out, the CTA still waits for every MMA and bulk copy it issued before it releases its
// TMEM and exits, so no asynchronous operation targets a finished CTA.  In-flight work
// completes in microseconds; the budget only bounds a broken pipeline.
constexpr long long kDrainBudget = 4000000000LL;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// two E4M3 codes (low byte first) -> two BF16 values times s (a power of two), packed low first
__device__ __forceinline__ uint32_t e4m3x2_to_bf16x2(uint32_t codes, float s) {
  const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(codes & 0xFFFFu), __NV_E4M3);
  const float2 f = __half22float2(__half2(hr));
  const __nv_bfloat162 b = __floats2bfloat162_rn(f.x * s, f.y * s);
  return *reinterpret_cast<const uint32_t*>(&b);
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait: true when the phase completed, false when the budget ran out
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long budget) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > budget) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
      "[%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);        // start address
  d |= (uint64_t)1 << 16;                          // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset
  d |= (uint64_t)1 << 46;                          // descriptor version
  d |= (uint64_t)2 << 61;                          // SWIZZLE_128B
  return d;
}

// shared-memory matrix descriptor: MN-major, 128-byte swizzle.  Each 8-row group along K holds
// 64 consecutive M elements per 128-byte row (one TMA box of 64 x 64 BF16 lands as 8 such
// groups, 1024 B apart); the second 64-wide M block is the next box, mn_stride bytes further.
__device__ __forceinline__ uint64_t sdesc_mn(uint32_t saddr, uint32_t mn_stride) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);        // start address
  d |= (uint64_t)((mn_stride >> 4) & 0x3FFF) << 16;  // leading byte offset: next 64-wide M block
  d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset: next 8-row K group
  d |= (uint64_t)1 << 46;                          // descriptor version
  d |= (uint64_t)2 << 61;                          // SWIZZLE_128B
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Instruction descriptor of kind::f16: D FP32, A/B BF16, both K-major, N >> 3, M >> 4.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

struct TcParams {
  int64_t n;          // rows of A (M extent) and K extent
  int N;              // columns of Y
  int BN;             // tile columns (multiple of 16, <= 256)
  int stages;
  int k_iters;        // BK-steps per split
  int tmem_cols;      // power of two >= BN, >= 32
  int xparts;         // 2: X as hi + lo BF16 parts, 1: hi only
  int comb;           // xparts 2 and 2 BN <= 256: one MMA of N = 2 BN per K step over the
                      // contiguous Xh | Xl tiles, A Xh and A Xl in TMEM columns [0, BN), [BN, 2 BN)
  int splits;         // K slices (gridDim.z)
  float* Y;           // unfused: output base (split z writes Y + z * n * ldy); fused: the slices
  int64_t ldy;
  int* err;           // error code (0 = ok)
  long long budget;   // clock64 budget per wait
  const int* run;     // device run flag of a solve (NULL: always run); 0 = stopped, skip the launch
  TcEpilogue e;       // fused epilogue (e.fused = 1)
  int sym;            // A held as its upper 128 x 128 tiles (sym_tile); mapA then has 64 x 128 boxes
                      // of a tile's columns, mapAt 64 x 64 boxes of a tile's rows (transposed use)
  int64_t nt;         // tiles per side of the symmetric storage
  const float* scales;  // E4M3 A: power-of-two scale per 128 x 128 tile, [nt8][nt8] row-major
  int nt8;              // E4M3 A: 128-wide tiles per side
};

// Fused epilogue of one 128 x BN output tile (K slice z), run by 128 threads te = 0 .. 127;
// q is the TMEM lane quadrant of the thread's warp, so the thread drains accumulator row
// 32 q + (te & 31) from trow.  The accumulator leaves TMEM in 64-column chunks through the
// shared tile T [128][kEpiTS], so every global access below is a coalesced 16-byte access
// along a row.  Split K: every slice publishes its partial tile; the last slice of the tile to
// arrive (arrival counter) sums the slices in slice order (the result does not depend on the
// arrival order) and runs the epilogue: Y = sum (+ c X2) and the per-restart partials
// <P1, A X>, <P2, A X> of the tile's two 64-row slots.  A thread reads all 16 of its rows of
// an operand before it uses them, so those reads are in flight together.  A group whose
// waits ran out (ok = false) publishes nothing but still takes its ticket, so the counter
// returns to zero for the next launch.  `sync` is a barrier over exactly these 128 threads.
constexpr int kEpiTS = 68;

template <typename Sync>
__device__ __forceinline__ void fused_tile_epilogue(const TcParams& p, float* T, uint32_t trow, int q, int te,
                                                    int n0, int m0, int z, unsigned tile, bool ok,
                                                    unsigned* s_ticket, Sync sync) {
  const int BN = p.BN;
  const int lane = te & 31;
  const int c4 = te & 15, r8 = te >> 4;  // float4 column, first row
  // 16 accumulator columns (with the combined MMA: the A Xh and A Xl halves added)
  auto acc16 = [&](uint32_t col, float* v) {
    tmem_ld16(trow + col, v);
    if (p.comb) {
      float t2[16];
      tmem_ld16(trow + col + (uint32_t)BN, t2);
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] += t2[k];
    }
  };
  auto stage_chunk = [&](int ch) {  // TMEM columns [64 ch, 64 ch + 64) -> T (rows = TMEM lanes)
    const int cw = min(64, BN - 64 * ch);
    for (int c = 0; c < cw; c += 16) {
      float v[16];
      acc16((uint32_t)(64 * ch + c), v);
      float* dst = T + (q * 32 + lane) * kEpiTS + c;
#pragma unroll
      for (int k = 0; k < 4; ++k)
        *reinterpret_cast<float4*>(dst + 4 * k) = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    }
  };
  const int nch = (BN + 63) / 64;
  bool last = ok;
  if (p.splits > 1) {
    if (ok) {
      float* Wz = p.Y + (int64_t)z * p.n * p.ldy;
      for (int ch = 0; ch < nch; ++ch) {
        stage_chunk(ch);
        sync();
        const int col = n0 + 64 * ch + 4 * c4;
        if (4 * c4 < BN - 64 * ch && col < p.N) {
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const int rr = r8 + 8 * k;
            const int64_t row_g = m0 + rr;
            if (row_g < p.n)
              *reinterpret_cast<float4*>(Wz + row_g * p.ldy + col) =
                  *reinterpret_cast<const float4*>(T + rr * kEpiTS + 4 * c4);
          }
        }
        sync();
      }
    }
    __threadfence();
    sync();
    if (te == 0) *s_ticket = atomicAdd(&p.e.counters[tile], 1u);
    sync();
    const bool arrived_last = *s_ticket == (unsigned)(p.splits - 1);
    if (arrived_last) {
      __threadfence();
      if (te == 0) p.e.counters[tile] = 0u;  // ready for the next launch
    }
    last = ok && arrived_last;
  }
  if (!last) return;
  const bool dots = p.e.P1 || p.e.P2;
  for (int ch = 0; ch < nch; ++ch) {
    stage_chunk(ch);
    sync();
    const int col = n0 + 64 * ch + 4 * c4;
    float d1[2] = {0.f, 0.f}, d2[2] = {0.f, 0.f};  // per 64-row slot (row rr: slot rr / 64 = k / 8)
    if (4 * c4 < BN - 64 * ch && col < p.N) {
      const int64_t idx0 = (int64_t)(m0 + r8) * p.ldy + col;  // row r8 + 8 k at idx0 + 8 k ldy
      const int64_t rstep = 8 * p.ldy;
      const int64_t rows_left = p.n - m0 - r8;  // rows r8 + 8 k < n - m0 exist
      const int kmax = rows_left <= 0 ? 0 : (rows_left >= 121 ? 16 : (int)((rows_left + 7) / 8));
      float4 y[16];
      if (p.splits > 1) {
        // the slices in slice order; this tile's own slice is the staged chunk
#pragma unroll
        for (int k = 0; k < 16; ++k) y[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int zz = 0; zz < p.splits; ++zz) {
          if (zz == z) {
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              const float4 v = *reinterpret_cast<const float4*>(T + (r8 + 8 * k) * kEpiTS + 4 * c4);
              y[k].x += v.x; y[k].y += v.y; y[k].z += v.z; y[k].w += v.w;
            }
          } else {
            const float* Sz = p.Y + (int64_t)zz * p.n * p.ldy + idx0;
            float4 v[16];
#pragma unroll
            for (int k = 0; k < 16; ++k)
              v[k] = k < kmax ? __ldcg(reinterpret_cast<const float4*>(Sz + k * rstep)) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              y[k].x += v[k].x; y[k].y += v[k].y; y[k].z += v[k].z; y[k].w += v[k].w;
            }
          }
        }
      } else {
#pragma unroll
        for (int k = 0; k < 16; ++k) y[k] = *reinterpret_cast<const float4*>(T + (r8 + 8 * k) * kEpiTS + 4 * c4);
      }
      // P1, P2 and X2 of 8 rows at a time in flight together: the dots use A X before c X2
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float4 w1[8], w2[8], w3[8];
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int kk = 8 * h + k;
          const int64_t off = idx0 + kk * rstep;
          w1[k] = (p.e.P1 && kk < kmax) ? *reinterpret_cast<const float4*>(p.e.P1 + off) : zero;
          w2[k] = (p.e.P2 && kk < kmax) ? *reinterpret_cast<const float4*>(p.e.P2 + off) : zero;
          w3[k] = (p.e.X2 && kk < kmax) ? *reinterpret_cast<const float4*>(p.e.X2 + off) : zero;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int kk = 8 * h + k;
          if (kk < kmax) {
            d1[h] += w1[k].x * y[kk].x + w1[k].y * y[kk].y + w1[k].z * y[kk].z + w1[k].w * y[kk].w;
            d2[h] += w2[k].x * y[kk].x + w2[k].y * y[kk].y + w2[k].z * y[kk].z + w2[k].w * y[kk].w;
            if (p.e.X2) {
              y[kk].x += p.e.c * w3[k].x; y[kk].y += p.e.c * w3[k].y; y[kk].z += p.e.c * w3[k].z;
              y[kk].w += p.e.c * w3[k].w;
            }
            *reinterpret_cast<float4*>(p.e.Y + idx0 + kk * rstep) = y[kk];
          }
        }
      }
    }
    if (dots) {
      // partials of each restart in this chunk (r divides 64, r % 4 == 0: restart jl owns the
      // g = r / 4 float4 columns c4 in [jl g, jl g + g)) and slot: a fixed shuffle tree over the
      // warp's lanes of those columns and its two row groups, then the four warps in order
      const int g = p.e.r / 4;
      float v[4] = {d1[0], d2[0], d1[1], d2[1]};
#pragma unroll
      for (int o = 1; o < 16; o <<= 1)
        if (o < g) {
#pragma unroll
          for (int t = 0; t < 4; ++t) v[t] += __shfl_xor_sync(0xffffffffu, v[t], o);
        }
#pragma unroll
      for (int t = 0; t < 4; ++t) v[t] += __shfl_xor_sync(0xffffffffu, v[t], 16);
      sync();  // every thread is done with T
      float* red = T;  // [4 warps][16 restarts][2 slots][2 dots]
      if (lane < 16 && c4 % g == 0) {
        float* rw = red + (q * 16 + c4 / g) * 4;
        rw[0] = v[0];  // slot 0: <P1, .>, <P2, .>
        rw[1] = v[1];
        rw[2] = v[2];  // slot 1
        rw[3] = v[3];
      }
      sync();
      const int cw = min(64, BN - 64 * ch);
      const int nres = cw / p.e.r;  // restarts in this chunk
      if (te < 2 * nres) {
        const int jl = te >> 1, slot_l = te & 1;
        float s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          s1 += red[(w * 16 + jl) * 4 + 2 * slot_l];
          s2 += red[(w * 16 + jl) * 4 + 2 * slot_l + 1];
        }
        const int j = (n0 + 64 * ch) / p.e.r + jl;
        const int64_t slot = 2 * (int64_t)(m0 / BM) + slot_l;
        if (j < p.e.b && slot * 64 < p.n) {
          double* qq = p.e.part + (slot * p.e.b + j) * kNQ + p.e.q0;
          qq[0] = (double)s1;
          qq[1] = (double)s2;
        }
      }
    }
    sync();  // T free for the next chunk
  }
}

template <bool FP8>
__global__ void __launch_bounds__(128, 1)
k_gemm_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapXh,
          const __grid_constant__ CUtensorMap mapXl, const __grid_constant__ CUtensorMap mapAt, TcParams p) {
  extern __shared__ unsigned char smem_raw[];
  // 1024-byte aligned ring: [stage][A 128x64 | Xh BNx64 | Xl BNx64] (bf16); E4M3 A:
  // [A buffer 0 | A buffer 1] (bf16, decoded) then the ring [stage][codes 128x64 | Xh | Xl]
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int BN = p.BN;
  const uint32_t a_bytes = BM * BK * 2;
  const uint32_t b_bytes = (uint32_t)BN * BK * 2;
  constexpr uint32_t a8_bytes = BM * BK;               // E4M3 codes of the A tile, staged by TMA
  const uint32_t xoff = FP8 ? a8_bytes : a_bytes;      // offset of the X parts in a stage
  const uint32_t stage_bytes = xoff + (uint32_t)p.xparts * b_bytes;
  unsigned char* ring = base + (FP8 ? 2 * a_bytes : 0);
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + (size_t)p.stages * stage_bytes);
  uint64_t* empty = full + p.stages;
  uint64_t* accum = empty + p.stages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
  uint64_t* conv = accum + 2;   // E4M3 A [2]: A buffer decoded (64 decoder threads arrive)
  uint64_t* afree = accum + 4;  // E4M3 A [2]: A buffer read by its MMAs (commit)
  __shared__ int s_fail, s_issued, s_consumed;
  __shared__ unsigned s_ticket;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * BN;
  const int m0 = blockIdx.y * BM;
  const int kbase = blockIdx.z * p.k_iters * BK;
  if (p.run && *p.run == 0) return;  // the solve has stopped: every CTA of the launch skips

  if (threadIdx.x == 0) {
    s_fail = 0;
    s_issued = 0;
    s_consumed = 0;
    for (int s = 0; s < p.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    if (FP8) {
      for (int j = 0; j < 2; ++j) {
        mbar_init(&conv[j], 64);
        mbar_init(&afree[j], 1);
      }
    }
    mbar_init(accum, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(p.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer
    int it = 0;
    for (; it < p.k_iters; ++it) {
      const int s = it % p.stages;
      const uint32_t ph = (uint32_t)(it / p.stages) & 1u;
      if (!mbar_wait(&empty[s], ph ^ 1u, p.budget)) { atomicExch(p.err, 1); s_fail = 1; break; }
      unsigned char* st = ring + (size_t)s * stage_bytes;
      const int kx = kbase + it * BK;
      if (FP8) {
        // the codes (64 bytes of each of 128 rows, zero filled past A), then the X parts
        mbar_expect_tx(&full[s], stage_bytes);
        tma_load_2d(st, &mapA, &full[s], kx, m0);
      } else if (!p.sym) {
        mbar_expect_tx(&full[s], stage_bytes);
        tma_load_2d(st, &mapA, &full[s], kx, m0);
      } else {
        mbar_expect_tx(&full[s], stage_bytes);
        // K block kx of row block m0 / 128: columns of the stored tile on or above the
        // diagonal, else rows kx .. kx + 63 of the stored mirror tile, as two 64-column boxes
        const int64_t i = m0 / BM, kb = kx / 128;
        const int hh = (kx / BK) & 1;
        if (kx >= p.n)  // beyond A (a short last slice): a box past the store, zero filled
          tma_load_2d(st, &mapA, &full[s], 0, (int)(p.nt * (p.nt + 1) / 2 * 128));
        else if (kb >= i)
          tma_load_2d(st, &mapA, &full[s], 64 * hh, (int)(sym_tile(i, kb, p.nt) * 128));
        else {
          const int y = (int)(sym_tile(kb, i, p.nt) * 128) + 64 * hh;
          tma_load_2d(st, &mapAt, &full[s], 0, y);
          tma_load_2d(st + a_bytes / 2, &mapAt, &full[s], 64, y);
        }
      }
      tma_load_2d(st + xoff, &mapXh, &full[s], kx, n0);
      if (p.xparts == 2) tma_load_2d(st + xoff + b_bytes, &mapXl, &full[s], kx, n0);
    }
    s_issued = it;
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t idesc = idesc_bf16(BM, p.comb ? 2 * BN : BN);
    int it = 0;
    for (; it < p.k_iters; ++it) {
      const int s = it % p.stages;
      const uint32_t ph = (uint32_t)(it / p.stages) & 1u;
      if (!mbar_wait(&full[s], ph, p.budget)) { atomicExch(p.err, 2); s_fail = 1; break; }
      if (FP8 && !mbar_wait(&conv[it & 1], (uint32_t)(it >> 1) & 1u, p.budget)) {
        atomicExch(p.err, 5);
        s_fail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t st_u = smem_u32(ring + (size_t)s * stage_bytes);
      const uint32_t sa = FP8 ? smem_u32(base + (size_t)(it & 1) * a_bytes) : st_u;
      const uint32_t sh = st_u + xoff, sl = st_u + xoff + b_bytes;
      // symmetric storage below the diagonal: A is the transposed mirror tile (MN-major)
      const int kx = kbase + it * BK;
      const bool tr = p.sym && kx < p.n && kx / 128 < m0 / BM;
      const uint32_t id = tr ? (idesc | (1u << 15)) : idesc;  // bit 15: A is MN-major
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        const uint64_t da = tr ? sdesc_mn(sa + kk * 2048, a_bytes / 2) : sdesc(sa + kk * 32);
        const uint32_t acc = (it > 0 || kk > 0) ? 1u : 0u;
        if (p.comb) {  // B = the 2 BN rows of Xh then Xl (one operand, one read of A)
          mma_bf16(tmem, da, sdesc(sh + kk * 32), id, acc);
        } else {
          mma_bf16(tmem, da, sdesc(sh + kk * 32), id, acc);
          if (p.xparts == 2) mma_bf16(tmem, da, sdesc(sl + kk * 32), id, 1u);
        }
      }
      mma_commit(&empty[s]);
      if (FP8) mma_commit(&afree[it & 1]);  // the A buffer may be decoded into again
    }
    s_consumed = it;
    mma_commit(accum);  // arrives once every MMA issued above has completed
  } else if (FP8 && warp >= 2) {
    // decoder: 16-byte chunk c of row m of the BF16 tile (8 codes) goes to chunk c ^ (m % 8)
    // of its 128-byte row, the 128-byte swizzle the MMA descriptors expect
    const int tid = threadIdx.x - 64;
    for (int it = 0; it < p.k_iters; ++it) {
      const int s = it % p.stages;
      const uint32_t ph = (uint32_t)(it / p.stages) & 1u;
      if (!mbar_wait(&full[s], ph, p.budget)) { atomicExch(p.err, 4); s_fail = 1; break; }
      // buffer it % 2, once the MMAs of its previous use (iteration it - 2) have completed
      if (!mbar_wait(&afree[it & 1], ((uint32_t)(it >> 1) & 1u) ^ 1u, p.budget)) {
        atomicExch(p.err, 6);
        s_fail = 1;
        break;
      }
      unsigned char* abuf = base + (size_t)(it & 1) * a_bytes;
      const unsigned char* a8 = ring + (size_t)s * stage_bytes;
      const int kt = (kbase + it * BK) / 128;
      const float sc = kt < p.nt8 ? __ldg(p.scales + (int64_t)(m0 / BM) * p.nt8 + kt) : 0.f;
#pragma unroll 4
      for (int i = 0; i < (BM * BK / 8) / 64; ++i) {
        const int id = tid + 64 * i;
        const int m = id >> 3, c = id & 7;
        const uint2 v = *reinterpret_cast<const uint2*>(a8 + m * 64 + c * 8);
        uint4 o;
        o.x = e4m3x2_to_bf16x2(v.x, sc);
        o.y = e4m3x2_to_bf16x2(v.x >> 16, sc);
        o.z = e4m3x2_to_bf16x2(v.y, sc);
        o.w = e4m3x2_to_bf16x2(v.y >> 16, sc);
        *reinterpret_cast<uint4*>(abuf + m * 128 + ((c ^ (m & 7)) << 4)) = o;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> the MMA's reads
      mbar_arrive(&conv[it & 1]);
    }
  }
  __syncwarp();
  __syncthreads();  // role loops finished; s_fail / s_issued / s_consumed visible
  // epilogue: all four warps, each drains its 32 TMEM lanes
  bool done = mbar_wait(accum, 0, p.budget);
  done = __all_sync(0xffffffffu, done);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!done && lane == 0) {
    atomicExch(p.err, 3);
    s_fail = 1;
  }
  __syncthreads();  // the CTA decides as one: s_fail from every warp visible
  const bool ok = !s_fail;
  const int row = m0 + warp * 32 + lane;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  // 16 accumulator columns (with the combined MMA: the A Xh and A Xl halves added)
  auto acc16 = [&](uint32_t col, float* v) {
    tmem_ld16(trow + col, v);
    if (p.comb) {
      float t[16];
      tmem_ld16(trow + col + (uint32_t)BN, t);
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] += t[i];
    }
  };
  if (ok && !p.e.fused) {
    float* Yz = p.Y + (int64_t)blockIdx.z * p.n * p.ldy;
    for (int c0 = 0; c0 < BN; c0 += 16) {
      float v[16];
      acc16((uint32_t)c0, v);
      if (row < p.n) {
        float* yr = Yz + (int64_t)row * p.ldy + n0 + c0;
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (n0 + c0 + i < p.N) yr[i] = v[i];
      }
    }
  }
  if (p.e.fused && (p.ldy & 3) == 0)  // 16-byte row groups (the launcher guarantees ldy % 4 == 0)
    // the ring is free once the accumulator is complete: it holds the epilogue tile
    fused_tile_epilogue(p, reinterpret_cast<float*>(base), trow, warp, (int)threadIdx.x, n0, m0, (int)blockIdx.z,
                        blockIdx.y * gridDim.x + blockIdx.x, ok, &s_ticket, [] { __syncthreads(); });
  __syncthreads();  // s_fail from the epilogue visible
  if (s_fail && threadIdx.x == 0) {
    // error path: drain with its own generous budget (a short wait budget that ran out
    // must not let the CTA exit with work in flight): every MMA issued above (the accum
    // commit follows them all), then the loads issued but never consumed
    const long long drain = p.budget > kDrainBudget ? p.budget : kDrainBudget;
    mbar_wait(accum, 0, drain);
    for (int it = s_consumed; it < s_issued; ++it)
      if (!mbar_wait(&full[it % p.stages], (uint32_t)(it / p.stages) & 1u, drain)) break;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols));
  }
}

// X (n x N FP32, ld) -> Xh, Xl (N x ldk BF16, transposed, zero padded in k)
__global__ void k_split_x(const float* __restrict__ X, int64_t n, int N, int64_t ld,
                          __nv_bfloat16* __restrict__ Xh, __nv_bfloat16* __restrict__ Xl, int64_t ldk) {
  __shared__ float t[32][33];
  const int64_t k0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int i = ty; i < 32; i += 8) {
    const int64_t k = k0 + i;
    const int c = c0 + tx;
    t[i][tx] = (k < n && c < N) ? X[k * ld + c] : 0.0f;
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int c = c0 + i;
    const int64_t k = k0 + tx;
    if (c < N && k < ldk) {
      const float v = t[tx][i];
      const __nv_bfloat16 hi = __float2bfloat16_rn(v);
      Xh[(int64_t)c * ldk + k] = hi;
      if (Xl) Xl[(int64_t)c * ldk + k] = __float2bfloat16_rn(v - __bfloat162float(hi));
    }
  }
}

// A (n x n, source type, lda) -> A16 (n x ldk BF16, zero padded columns)
template <typename TS>
__global__ void k_to_bf16(const TS* __restrict__ A, int64_t n, int64_t lda, __nv_bfloat16* __restrict__ A16,
                          int64_t ldk) {
  const int64_t total = n * ldk;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ldk, k = e % ldk;
    A16[e] = __float2bfloat16_rn(k < n ? (float)A[i * lda + k] : 0.0f);
  }
}

// A (source type, lda) -> its upper 128 x 128 tiles in BF16, one CTA per tile of the grid
// (blockIdx.x = column tile b, blockIdx.y = row tile a; a > b does nothing): tile (a, b) at
// sym_tile(a, b, nt) * 128 * 128, row-major, zero beyond n.  Rounding as k_to_bf16.
template <typename TS>
__global__ void k_to_bf16_sym(const TS* __restrict__ A, int64_t n, int64_t lda, __nv_bfloat16* __restrict__ out,
                              int64_t nt) {
  const int64_t a = blockIdx.y, b = blockIdx.x;
  if (a > b) return;
  __nv_bfloat16* T = out + sym_tile(a, b, nt) * 16384;
  for (int e = threadIdx.x; e < 16384; e += blockDim.x) {
    const int64_t i = a * 128 + (e >> 7), k = b * 128 + (e & 127);
    T[e] = __float2bfloat16_rn(i < n && k < n ? (float)A[i * lda + k] : 0.0f);
  }
}

// sum of squares and sum of the symmetric matrix held as its upper tiles: tiles strided over
// the CTAs, a tile above the diagonal counted twice (FP64 partial per block)
__global__ void k_sums_bf16_sym(const __nv_bfloat16* __restrict__ A, int64_t nt, double* __restrict__ part) {
  __shared__ double sh2[32], sh1[32];
  const int64_t ntiles = nt * (nt + 1) / 2;
  double s2 = 0.0, s1 = 0.0;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    // row tile a of tile t: the last a whose diagonal tile index is <= t
    const double q = 2.0 * (double)nt + 1.0;
    int64_t a = (int64_t)((q - sqrt(q * q - 8.0 * (double)t)) / 2.0);
    if (a < 0) a = 0;
    if (a > nt - 1) a = nt - 1;
    while (a > 0 && sym_tile(a, a, nt) > t) --a;
    while (a + 1 < nt && sym_tile(a + 1, a + 1, nt) <= t) ++a;
    const double w = sym_tile(a, a, nt) == t ? 1.0 : 2.0;
    double t2 = 0.0, t1 = 0.0;
    for (int e = threadIdx.x; e < 16384; e += blockDim.x) {
      const double v = (double)__bfloat162float(A[t * 16384 + e]);
      t2 += v * v;
      t1 += v;
    }
    s2 += w * t2;
    s1 += w * t1;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sh2[wid] = s2; sh1[wid] = s1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a2 = 0.0, a1 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a2 += sh2[w]; a1 += sh1[w]; }
    part[2 * blockIdx.x] = a2;
    part[2 * blockIdx.x + 1] = a1;
  }
}

// sum of squares and sum of a BF16 matrix (FP64 partial per block)
__global__ void k_sums_bf16(const __nv_bfloat16* __restrict__ A, int64_t m, double* __restrict__ part) {
  __shared__ double sh2[32], sh1[32];
  double s2 = 0.0, s1 = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)__bfloat162float(A[e]);
    s2 += v * v;
    s1 += v;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sh2[wid] = s2; sh1[wid] = s1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += sh2[w]; b += sh1[w]; }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}


// ---------------------------------------------------------------------------------------
// Grouped product of the uneven batch: CTA = one 128-row tile of one problem.  The ring
// stage holds the A tile (128 x 64) and up to 64 rows of each X part (bn / 16 boxes of 16
// rows); 3 stages, so two CTAs share an SM.  Same roles and bounded waits as k_gemm_tc.
// ---------------------------------------------------------------------------------------
constexpr int kBStages = 3;
constexpr uint32_t kBStageA = BM * BK * 2;       // 16 KB
constexpr uint32_t kBStageB = 64 * BK * 2;       // room for 64 rows of one X part
constexpr uint32_t kBStageBytes = kBStageA + 2 * kBStageB;

__device__ __forceinline__ bool item_live(const TcItem& it, const unsigned char* ctl, size_t stride,
                                          size_t off, const int* run) {
  if (run && *run == 0) return false;
  if (ctl && *reinterpret_cast<const int*>(ctl + (size_t)it.prob * stride + off) == 0) return false;
  return true;
}

__global__ void __launch_bounds__(128, 2)
k_bgemm_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapXh,
           const __grid_constant__ CUtensorMap mapXl, const TcItem* __restrict__ items,
           const int* __restrict__ cnt, const float* __restrict__ X, float* __restrict__ Y, int add_lam,
           const float* __restrict__ P1, double* __restrict__ part, int nq, const unsigned char* __restrict__ ctl,
           size_t ctl_stride, size_t active_off, const int* __restrict__ run, int* __restrict__ err,
           long long budget) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(base + (size_t)kBStages * kBStageBytes);
  uint64_t* empty = full + kBStages;
  uint64_t* accum = empty + kBStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
  __shared__ int s_fail, s_issued, s_consumed;
  __shared__ float s_red[4];
  if ((int)blockIdx.x >= *cnt) return;
  const TcItem it = items[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (!item_live(it, ctl, ctl_stride, active_off, run)) {
    if (part && threadIdx.x == 0) part[(int64_t)it.slot * nq] = 0.0;
    return;
  }
  const int bn = it.bn;
  const uint32_t stage_tx = kBStageA + 2u * (uint32_t)bn * BK * 2;
  if (threadIdx.x == 0) {
    s_fail = 0;
    s_issued = 0;
    s_consumed = 0;
    for (int s = 0; s < kBStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accum, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(64));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    int i = 0;
    for (; i < it.kt; ++i) {
      const int s = i % kBStages;
      const uint32_t ph = (uint32_t)(i / kBStages) & 1u;
      if (!mbar_wait(&empty[s], ph ^ 1u, budget)) { atomicExch(err, 11); s_fail = 1; break; }
      unsigned char* st = base + (size_t)s * kBStageBytes;
      mbar_expect_tx(&full[s], stage_tx);
      const int kx = i * BK;
      tma_load_2d(st, &mapA, &full[s], kx, (int)it.arow);
      for (int h = 0; h < bn / 16; ++h) {
        tma_load_2d(st + kBStageA + h * 16 * BK * 2, &mapXh, &full[s], kx, it.xrow + 16 * h);
        tma_load_2d(st + kBStageA + kBStageB + h * 16 * BK * 2, &mapXl, &full[s], kx, it.xrow + 16 * h);
      }
    }
    s_issued = i;
  } else if (warp == 1 && lane == 0) {
    const uint32_t idesc = idesc_bf16(BM, bn);
    int i = 0;
    for (; i < it.kt; ++i) {
      const int s = i % kBStages;
      const uint32_t ph = (uint32_t)(i / kBStages) & 1u;
      if (!mbar_wait(&full[s], ph, budget)) { atomicExch(err, 12); s_fail = 1; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = smem_u32(base + (size_t)s * kBStageBytes);
      const uint32_t sh = sa + kBStageA, sl = sa + kBStageA + kBStageB;
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        const uint64_t da = sdesc(sa + kk * 32);
        mma_bf16(tmem, da, sdesc(sh + kk * 32), idesc, (i > 0 || kk > 0) ? 1u : 0u);
        mma_bf16(tmem, da, sdesc(sl + kk * 32), idesc, 1u);
      }
      mma_commit(&empty[s]);
    }
    s_consumed = i;
    mma_commit(accum);
  }
  __syncwarp();
  __syncthreads();
  bool done = mbar_wait(accum, 0, budget);
  done = __all_sync(0xffffffffu, done);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!done && lane == 0) {
    atomicExch(err, 13);
    s_fail = 1;
  }
  __syncthreads();  // the CTA decides as one (the TMEM loads below are warp-collective)
  float d1 = 0.f;
  if (!s_fail) {
    const int row = it.m0 + warp * 32 + lane;
    const bool rv = row < it.n;
    for (int c0 = 0; c0 < bn; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (rv) {
        const int64_t rowoff = it.xoff + (int64_t)row * it.r;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int c = c0 + i;
          if (c < it.r) {
            float y = v[i];
            if (P1) d1 += P1[rowoff + c] * y;
            if (add_lam) y += it.lam * X[rowoff + c];
            Y[rowoff + c] = y;
          }
        }
      }
    }
  }
  if (part) {
    for (int o = 16; o > 0; o >>= 1) d1 += __shfl_xor_sync(0xffffffffu, d1, o);
    if (lane == 0) s_red[warp] = d1;
  }
  __syncthreads();  // s_fail from the epilogue visible
  if (s_fail && threadIdx.x == 0) {
    // error path: drain every issued MMA and unconsumed load with the generous budget
    const long long drain = budget > kDrainBudget ? budget : kDrainBudget;
    mbar_wait(accum, 0, drain);
    for (int i = s_consumed; i < s_issued; ++i)
      if (!mbar_wait(&full[i % kBStages], (uint32_t)(i / kBStages) & 1u, drain)) break;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (part && threadIdx.x == 0) part[(int64_t)it.slot * nq] = (double)(s_red[0] + s_red[1] + s_red[2] + s_red[3]);
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64));
  }
}

// X_p rows m0 .. m0 + 128 (FP32, ld r_p) -> columns of the transposed BF16 hi / lo parts
__global__ void __launch_bounds__(256)
k_bsplit_x(const TcItem* __restrict__ items, const int* __restrict__ cnt, const float* __restrict__ X,
           __nv_bfloat16* __restrict__ Xh, __nv_bfloat16* __restrict__ Xl, int64_t lda,
           const unsigned char* __restrict__ ctl, size_t ctl_stride, size_t active_off, const int* __restrict__ run) {
  __shared__ float t[BM][65];
  if ((int)blockIdx.x >= *cnt) return;
  const TcItem it = items[blockIdx.x];
  if (!item_live(it, ctl, ctl_stride, active_off, run)) return;
  const int rows = min(BM, it.n - it.m0);
  for (int e = threadIdx.x; e < rows * it.r; e += blockDim.x) {
    const int i = e / it.r, c = e % it.r;
    t[i][c] = X[it.xoff + (int64_t)(it.m0 + i) * it.r + c];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < rows * it.r; e += blockDim.x) {
    const int c = e / rows, i = e % rows;
    const float v = t[i][c];
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    const int64_t o = (int64_t)(it.xrow + c) * lda + it.m0 + i;
    Xh[o] = hi;
    Xl[o] = lo;
  }
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn get_encode() {
  static EncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  });
  return fn;
}

// 2-D BF16 tensor map: inner extent `inner` (elements, contiguous), `rows` rows, row pitch
// `ld` elements; box {64, box_rows}; 128-byte swizzle; out-of-range reads are zero.
int g_last_cu = 0;  // last CUresult of the tensor-map encoder (diagnostics)

bool make_map(CUtensorMap* m, const void* base, int64_t inner, int64_t rows, int64_t ld, int box_rows) {
  EncodeFn enc = get_encode();
  if (!enc) { g_last_cu = -1; return false; }
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  g_last_cu = (int)r;
  return r == CUDA_SUCCESS;
}

}  // namespace

// Tensor map of the E4M3 code matrix (1-byte elements, pitch ld bytes): 64 x box_rows boxes,
// unswizzled (the kernel's decoder writes the swizzled BF16 tile itself).
static bool make_map_u8(CUtensorMap* m, const void* base, int64_t inner, int64_t rows, int64_t ld, int box_rows) {
  EncodeFn enc = get_encode();
  if (!enc) { g_last_cu = -1; return false; }
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld};
  cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  g_last_cu = (int)r;
  return r == CUDA_SUCCESS;
}

int tc_last_status() { return g_last_cu; }

bool make_map_f32_tile(CUtensorMap* m, const void* base, int64_t cols, int64_t rows, int64_t ld) {
  EncodeFn enc = get_encode();
  if (!enc || !base || (reinterpret_cast<uintptr_t>(base) & 15) || (ld * 4) % 16 || cols > ld) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
  cuuint32_t box[2] = {32, 128};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int64_t tc_ld(int64_t n) { return (n + 63) / 64 * 64; }

void launch_to_bf16(int src_dtype, const void* A, int64_t n, int64_t lda, void* A16, cudaStream_t s) {
  const int64_t ldk = tc_ld(n);
  const int blocks = (int)((n * ldk + 255) / 256 < 152 * 32 ? (n * ldk + 255) / 256 : 152 * 32);
  if (src_dtype == 0)
    k_to_bf16<double><<<blocks, 256, 0, s>>>((const double*)A, n, lda, (__nv_bfloat16*)A16, ldk);
  else
    k_to_bf16<float><<<blocks, 256, 0, s>>>((const float*)A, n, lda, (__nv_bfloat16*)A16, ldk);
}

void launch_to_bf16_sym(int src_dtype, const void* A, int64_t n, int64_t lda, void* A16s, cudaStream_t s) {
  const int64_t nt = (n + 127) / 128;
  dim3 grid((unsigned)nt, (unsigned)nt);
  if (src_dtype == 0)
    k_to_bf16_sym<double><<<grid, 256, 0, s>>>((const double*)A, n, lda, (__nv_bfloat16*)A16s, nt);
  else
    k_to_bf16_sym<float><<<grid, 256, 0, s>>>((const float*)A, n, lda, (__nv_bfloat16*)A16s, nt);
}

int launch_sums_bf16_sym(const void* A16s, int64_t n, double* part, cudaStream_t s) {
  const int64_t nt = (n + 127) / 128;
  const int64_t ntiles = nt * (nt + 1) / 2;
  const int blocks = (int)(ntiles < 1024 ? ntiles : 1024);
  k_sums_bf16_sym<<<blocks, 256, 0, s>>>((const __nv_bfloat16*)A16s, nt, part);
  return blocks;
}

int launch_sums_bf16(const void* A16, int64_t elems, double* part, cudaStream_t s) {
  const int blocks = (int)((elems + 255) / 256 < 1024 ? (elems + 255) / 256 : 1024);
  k_sums_bf16<<<blocks, 256, 0, s>>>((const __nv_bfloat16*)A16, elems, part);
  return blocks;
}

int tc_plan(int64_t n, int N, TcPlan* plan, const ProdTune* tune, int xparts, int a8) {
  TcPlan pl{};
  pl.BN = N <= 256 ? ((N + 15) / 16 * 16) : 256;
  if (tune && tune->bn > 0) {
    if (tune->bn % 16 || tune->bn > 256) return -1;
    pl.BN = tune->bn < pl.BN ? tune->bn : pl.BN;
  }
  pl.tiles_n = (N + pl.BN - 1) / pl.BN;
  pl.tiles_m = (int)((n + BM - 1) / BM);
  const int64_t kiters_total = (n + BK - 1) / BK;
  // E4M3 A (a8): a stage holds the 128 x 64 code tile instead of the BF16 A tile, and the two
  // decoded BF16 A buffers sit outside the ring
  const uint32_t stage_bytes = (a8 ? BM * BK : BM * BK * 2) + (uint32_t)xparts * pl.BN * BK * 2;
  const uint32_t fixed = a8 ? 2 * BM * BK * 2 : 0;
  // two CTAs per SM with a 3-stage ring when it fits in half the SM, else one CTA with
  // as many stages as fit (at most 6)
  int per_sm = 1, stages;
  if (3 * stage_bytes + fixed + 4096 <= 110 * 1024) {
    per_sm = 2;
    stages = 3;
  } else {
    stages = (int)((200 * 1024 - fixed) / stage_bytes);
    if (stages > 6) stages = 6;
    if (stages < 2) stages = 2;
  }
  if (tune && tune->per_sm > 0 && tune->stages > 0) {  // autotuned ring
    per_sm = tune->per_sm;
    stages = tune->stages;
    const size_t cap = per_sm == 2 ? 110 * 1024 : 206 * 1024;
    if ((size_t)stage_bytes * stages + fixed + 4096 > cap || stages < 2) return -1;
  }
  pl.stages = stages;
  const int tiles = pl.tiles_n * pl.tiles_m;
  int splits = (152 * per_sm) / tiles;
  if (splits < 1) splits = 1;
  while (splits > 1 && kiters_total / splits < 8) --splits;
  // The tensor cores' FP32 accumulation loses a little in every MMA step (measured: a
  // relative bias near 2e-5 over K = 8192 in one accumulator); K slices of at most
  // kMaxChain * 64 keep it near 5e-6, below what the 1e-4 stopping test resolves.
  const int min_splits = (int)((kiters_total + kMaxChain - 1) / kMaxChain);
  if (splits < min_splits) splits = min_splits;
  if (tune && tune->splits > 0) {
    if (tune->splits < min_splits) return -1;
    splits = (int)(tune->splits < kiters_total ? tune->splits : kiters_total);
  }
  pl.splits = splits;
  pl.k_iters = (int)((kiters_total + splits - 1) / splits);
  pl.tmem_cols = 32;
  while (pl.tmem_cols < pl.BN) pl.tmem_cols *= 2;
  pl.smem = fixed + stage_bytes * stages + 1024 + 8 * (2 * stages + 2) + 64 + (a8 ? 32 : 0);
  *plan = pl;
  return 0;
}

namespace {

// Shared launcher of k_gemm_tc: fused epilogue when epi != NULL && epi->fused.
// scales8 != NULL: A16 is the E4M3 code matrix (pitch fp8_ld(n) bytes) with its tile scales.
int launch_tc_impl(const void* A16, int64_t n, const float* X, int N, int64_t ldx, void* xh, void* xl, int xparts,
                   float* Y, float* ws, size_t ws_elems, int* err, long long budget, const TcEpilogue* epi,
                   const int* run, cudaStream_t s, const ProdTune* tune, int sym, const float* scales8 = nullptr) {
  const int a8 = scales8 ? 1 : 0;
  if (a8) sym = 0;
  TcPlan pl;
  if (tc_plan(n, N, &pl, tune, xparts, a8) < 0) tc_plan(n, N, &pl, nullptr, xparts, a8);
  const int64_t ldk = tc_ld(n);
  if ((size_t)pl.splits * n * ldx > ws_elems) {
    // not enough split workspace: recompute the plan without splitting
    pl.splits = 1;
    pl.k_iters = (int)((n + BK - 1) / BK);
  }
  dim3 sg((unsigned)((ldk + 31) / 32), (unsigned)((N + 31) / 32));
  k_split_x<<<sg, 256, 0, s>>>(X, n, N, ldx, (__nv_bfloat16*)xh, xparts == 2 ? (__nv_bfloat16*)xl : nullptr,
                               ldk);
  CUtensorMap ma, mh, ml, mt;
  const int64_t nt = (n + 127) / 128;
  if (sym) {
    // the upper tiles as one (tiles x 128) x 128 array: 64-column boxes of a tile's 128 rows
    // (K-major use) and 64 x 64 boxes of its rows (the mirror's MN-major use)
    if (!make_map(&ma, A16, 128, sym_tiles(n) * 128, 128, BM) || !make_map(&mt, A16, 128, sym_tiles(n) * 128, 128, 64))
      return -1;
  } else if (a8) {
    if (!make_map_u8(&ma, A16, fp8_ld(n), n, fp8_ld(n), BM)) return -1;
  } else if (!make_map(&ma, A16, ldk, n, ldk, BM)) {
    return -1;
  }
  if (!make_map(&mh, xh, ldk, N, ldk, pl.BN) || !make_map(&ml, xparts == 2 ? xl : xh, ldk, N, ldk, pl.BN))
    return -1;
  if (!sym) mt = ma;
  static bool attr_done[2] = {false, false};
  if (!attr_done[a8]) {
    // the plan never asks for more than ~206 KB; static shared memory comes on top
    const cudaError_t ae = a8 ? cudaFuncSetAttribute(k_gemm_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     210 * 1024)
                              : cudaFuncSetAttribute(k_gemm_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     210 * 1024);
    if (ae != cudaSuccess) {
      g_last_cu = 10000 + (int)cudaGetLastError();
      return -3;
    }
    attr_done[a8] = true;
  }
  TcParams p;
  p.n = n;
  p.N = N;
  p.BN = pl.BN;
  p.stages = pl.stages;
  p.k_iters = pl.k_iters;
  p.xparts = xparts;
  p.comb = xparts == 2 && 2 * pl.BN <= 256;
  p.tmem_cols = pl.tmem_cols;
  while (p.comb && p.tmem_cols < 2 * pl.BN) p.tmem_cols *= 2;
  p.splits = pl.splits;
  p.Y = pl.splits > 1 ? ws : Y;
  p.ldy = ldx;
  p.err = err;
  p.budget = budget;
  p.run = run;
  if (epi && epi->fused) p.e = *epi;
  p.sym = sym;
  p.nt = nt;
  p.scales = scales8;
  p.nt8 = a8 ? fp8_ntiles(n) : 0;
  dim3 grid(pl.tiles_n, pl.tiles_m, pl.splits);
  if (a8)
    k_gemm_tc<true><<<grid, 128, pl.smem, s>>>(ma, mh, ml, mt, p);
  else
    k_gemm_tc<false><<<grid, 128, pl.smem, s>>>(ma, mh, ml, mt, p);
  const cudaError_t le = cudaPeekAtLastError();
  if (le != cudaSuccess) { g_last_cu = 10000 + (int)le; return -2; }
  return (epi && epi->fused) ? 0 : pl.splits;
}

}  // namespace

int launch_ax_tc(const void* A16, int64_t n, const float* X, int N, int64_t ldx, void* xh, void* xl,
                 float* Y, float* ws, size_t ws_elems, int* err, long long budget, cudaStream_t s,
                 const ProdTune* tune, int xparts, int sym) {
  return launch_tc_impl(A16, n, X, N, ldx, xh, xl, xparts, Y, ws, ws_elems, err, budget, nullptr, nullptr, s,
                        tune, sym);
}

int launch_ax_tc_fused(const void* A16, int64_t n, const float* X, int N, int64_t ldx, void* xh, void* xl,
                       int xparts, float* ws, size_t ws_elems, int* err, long long budget, const TcEpilogue& epi,
                       const int* run, cudaStream_t s, const ProdTune* tune, int sym) {
  return launch_tc_impl(A16, n, X, N, ldx, xh, xl, xparts, epi.Y, ws, ws_elems, err, budget, &epi, run, s, tune,
                        sym);
}

int launch_ax_tc8(const void* A8, const float* scales, int64_t n, const float* X, int N, int64_t ldx, void* xh,
                  void* xl, float* Y, float* ws, size_t ws_elems, int* err, long long budget, cudaStream_t s,
                  const ProdTune* tune, int xparts) {
  return launch_tc_impl(A8, n, X, N, ldx, xh, xl, xparts, Y, ws, ws_elems, err, budget, nullptr, nullptr, s, tune, 0,
                        scales);
}

int launch_ax_tc8_fused(const void* A8, const float* scales, int64_t n, const float* X, int N, int64_t ldx,
                        void* xh, void* xl, int xparts, float* ws, size_t ws_elems, int* err, long long budget,
                        const TcEpilogue& epi, const int* run, cudaStream_t s, const ProdTune* tune) {
  return launch_tc_impl(A8, n, X, N, ldx, xh, xl, xparts, epi.Y, ws, ws_elems, err, budget, &epi, run, s, tune, 0,
                        scales);
}

void launch_bsplit_x(const TcItem* items, int nitems, const int* cnt, const float* X, void* xh, void* xl,
                     int64_t lda, const void* ctl, size_t ctl_stride, size_t active_off, const int* run,
                     cudaStream_t s) {
  k_bsplit_x<<<nitems, 256, 0, s>>>(items, cnt, X, (__nv_bfloat16*)xh, (__nv_bfloat16*)xl, lda,
                                    (const unsigned char*)ctl, ctl_stride, active_off, run);
}

int launch_bgemm_tc(const void* A16, int64_t lda, int64_t rows_total, const void* xh, const void* xl,
                    int64_t xt_rows, const TcItem* items, int nitems, const int* cnt, const float* X, float* Y,
                    int add_lam,
                    const float* P1, double* part, int nq, const void* ctl, size_t ctl_stride,
                    size_t active_off, const int* run, int* err, long long budget, cudaStream_t s) {
  CUtensorMap ma, mh, ml;
  if (!make_map(&ma, A16, lda, rows_total, lda, BM) || !make_map(&mh, xh, lda, xt_rows, lda, 16) ||
      !make_map(&ml, xl, lda, xt_rows, lda, 16))
    return -1;
  const size_t smem = (size_t)kBStages * kBStageBytes + 1024 + 8 * (2 * kBStages + 2) + 64;
  static bool attr_done = false;
  if (!attr_done) {
    if (cudaFuncSetAttribute(k_bgemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      g_last_cu = 10000 + (int)cudaGetLastError();
      return -3;
    }
    attr_done = true;
  }
  k_bgemm_tc<<<nitems, 128, smem, s>>>(ma, mh, ml, items, cnt, X, Y, add_lam, P1, part, nq,
                                       (const unsigned char*)ctl, ctl_stride, active_off, run, err, budget);
  const cudaError_t le = cudaPeekAtLastError();
  if (le != cudaSuccess) { g_last_cu = 10000 + (int)le; return -2; }
  return 0;
}

}  // namespace snmf
