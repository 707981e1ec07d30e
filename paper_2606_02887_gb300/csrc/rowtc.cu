// Row kernels of an Algorithm-1 step on the tensor cores (tcgen05, kind::tf32), FP32 penalty
// blocks with r = 64: the same data flow as rowfuse.cu (the D step writes g(Z) only, the update
// recomputes Z and D from X, g, g(Z)), with the two r x r row products Z G and D G (D step) and
// X' G (update) as UMMA M = 128, N = 64, K = 64 contractions into TMEM.
//
// Precision: FP32 operands enter the tensor cores as TF32 (10 explicit mantissa bits).  Each
// operand is split into hi = tf32(v) and lo = tf32(v - hi) and the product is accumulated as
// A_hi B_hi + A_hi B_lo + A_lo B_hi (three MMAs per K step, the lo x lo term of relative size
// 2^-22 dropped), so the row products carry about FP32 accuracy.
//
// CTA: 128 rows of restart blockIdx.y, 256 threads.  Operand tiles in shared memory are K-major
// with the 128-byte swizzle (two 32-column atoms per 64-column row; 16-byte chunk c of row m
// stored at chunk c ^ (m % 8)), written from registers by the threads; one elected thread issues
// the MMAs and commits them to an mbarrier that the CTA waits on (bounded).  Global memory is
// accessed in a coalesced mapping, the accumulator read from TMEM row-wise and passed through
// shared memory (see the thread mappings below).
#include <math.h>

#include "common.cuh"
#include "rowops.cuh"
#include "rowops_dev.cuh"

namespace snmf {

namespace {

constexpr int TR = 128;           // rows per CTA (UMMA M)
constexpr int RC = 64;            // columns (r, UMMA N = K)
constexpr uint32_t A_PART = TR * RC * 4;   // 32 KB: one TF32 part of a 128 x 64 operand tile
constexpr uint32_t B_PART = RC * RC * 4;   // 16 KB: one TF32 part of G
constexpr uint32_t SMEM_BYTES = 2 * A_PART + 2 * B_PART + 1024;  // + alignment slack
constexpr long long kWait = 2000000000LL;   // clock64 budget of an MMA completion wait
constexpr long long kDrain = 4000000000LL;  // budget of the drain on the error path

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
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

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long budget) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > budget) return false;
  }
  return true;
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major, N >> 3, M >> 4.
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
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

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t t;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(x));
  return t;
}

// byte offset of the 16-byte chunk holding columns k .. k + 3 (k % 4 == 0) of row m in a
// `rows` x 64 K-major tile with the 128-byte swizzle
__device__ __forceinline__ uint32_t sw_chunk(int m, int k, int rows) {
  const int atom = k >> 5, c = (k & 31) >> 2;
  return (uint32_t)(atom * rows * 128 + m * 128 + ((c ^ (m & 7)) << 4));
}

// hi / lo TF32 parts of four consecutive values into the two operand parts
__device__ __forceinline__ void put4(unsigned char* hi_part, unsigned char* lo_part, uint32_t off, float a, float b,
                                     float c, float d) {
  const uint32_t h0 = to_tf32(a), h1 = to_tf32(b), h2 = to_tf32(c), h3 = to_tf32(d);
  const uint32_t l0 = to_tf32(a - __uint_as_float(h0)), l1 = to_tf32(b - __uint_as_float(h1)),
                 l2 = to_tf32(c - __uint_as_float(h2)), l3 = to_tf32(d - __uint_as_float(h3));
  *reinterpret_cast<uint4*>(hi_part + off) = make_uint4(h0, h1, h2, h3);
  *reinterpret_cast<uint4*>(lo_part + off) = make_uint4(l0, l1, l2, l3);
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

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

// Shared set-up of a CTA: 1024-aligned operand parts, the G parts of restart j, the mbarrier,
// the TMEM allocation (128 columns: two 64-column accumulators).
struct TcTile {
  unsigned char *ah, *al, *bh, *bl;
};

__device__ __forceinline__ TcTile carve(unsigned char* raw) {
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~static_cast<uintptr_t>(1023));
  TcTile t;
  t.ah = base;
  t.al = base + A_PART;
  t.bh = base + 2 * A_PART;
  t.bl = base + 2 * A_PART + B_PART;
  return t;
}

__device__ __forceinline__ void load_gram_parts(const float* G, const TcTile& t) {
  // thread t: row n = t / 4 of G (K-major B operand: row n holds G[n][k] = G[k][n]), 16 columns
  const int n = threadIdx.x >> 2, k0 = (threadIdx.x & 3) * 16;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int k = k0 + 4 * c;
    const float4 v = ld4(G + n * RC + k);
    put4(t.bh, t.bl, sw_chunk(n, k, RC), v.x, v.y, v.z, v.w);
  }
}

// The 24 MMAs of one 128 x 64 x 64 product (3 per K step of 8) into TMEM column `col`.
__device__ __forceinline__ void issue_product(const TcTile& t, uint32_t tmem_col) {
  const uint32_t idesc = idesc_tf32(TR, RC);
  const uint32_t ah = smem_u32(t.ah), al = smem_u32(t.al), bh = smem_u32(t.bh), bl = smem_u32(t.bl);
#pragma unroll
  for (int kk = 0; kk < RC / 8; ++kk) {
    const uint32_t ao = (kk >> 2) * TR * 128 + (kk & 3) * 32;
    const uint32_t bo = (kk >> 2) * RC * 128 + (kk & 3) * 32;
    mma_tf32(tmem_col, sdesc(al + ao), sdesc(bh + bo), idesc, kk > 0 ? 1u : 0u);
    mma_tf32(tmem_col, sdesc(ah + ao), sdesc(bl + bo), idesc, 1u);
    mma_tf32(tmem_col, sdesc(ah + ao), sdesc(bh + bo), idesc, 1u);
  }
}

// Make the threads' operand writes visible to the tensor cores, then one thread issues the
// product and commits it to `bar`.
__device__ __forceinline__ void run_product(const TcTile& t, uint32_t tmem_col, uint64_t* bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    issue_product(t, tmem_col);
    mma_commit(bar);
  }
}

// CTA-uniform wait for a committed product: false (and err set) when the budget ran out.
__device__ __forceinline__ bool wait_product(uint64_t* bar, uint32_t parity, int* s_bad, int* err) {
  const bool done = mbar_wait(bar, parity, kWait);
  if (!done) {
    *s_bad = 1;
    if (err) atomicExch(err, 21);
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return *s_bad == 0;
}

__device__ __forceinline__ void block_partials(const RowArgs& a, const float (&dq)[8], int j, int slot, unsigned per,
                                               float (*shq)[8], unsigned* ticket) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const float v = warp_sum(dq[m]);
    if (lane == 0) shq[m][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    float v = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) v += shq[threadIdx.x][w];
    a.part[((int64_t)slot * a.b + j) * kNQ + threadIdx.x] = (double)v;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) *ticket = atomicAdd(&a.counters[j], 1u);
  __syncthreads();
  if (*ticket == per - 1) {
    if (threadIdx.x == 0) a.counters[j] = 0u;
    if (threadIdx.x < 32)
      fused_control(a.ctl_mode, const_cast<Ctl&>(a.ctl[j]), a.part, (int)per, a.b, a.r, j, a.P, a.G64fix, nullptr, 1);
  }
}

// Thread mappings.  Elementwise work and every global access use the coalesced mapping: thread
// t owns float4 column c4 = t % 16 (columns 4 c4 .. 4 c4 + 3) of rows t / 16 + 16 k, k < 8, so 16
// threads read a 256-byte row segment together.  The accumulator leaves TMEM row-wise (warp w
// reads lanes 32 (w % 4) .. + 31, columns 32 (w / 4) .. + 31) into a staging tile T with the
// operand's swizzled layout, placed in the lo-part region of the operand tile, which the tensor
// cores no longer read once the product has completed.
constexpr int CM_ROWS = 8;  // rows per thread in the coalesced mapping

__device__ __forceinline__ float4 ld_sw(const unsigned char* part, int m, int k) {
  return *reinterpret_cast<const float4*>(part + sw_chunk(m, k, TR));
}

// TMEM accumulator columns [col, col + 64) -> T (swizzled like the operand tile)
__device__ __forceinline__ void stage_acc(uint32_t tacc, int col, unsigned char* T, int mrow, int c0) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    float v[16];
    tmem_ld16(tacc + (uint32_t)(col + c0 + 16 * h), v);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      *reinterpret_cast<float4*>(T + sw_chunk(mrow, c0 + 16 * h + 4 * q, TR)) =
          make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  }
}

// Set-up shared by both kernels: barrier, TMEM (128 columns), G parts.
__device__ __forceinline__ void tc_setup(uint64_t* bar, uint32_t* tmem_slot, int* s_bad, const float* G,
                                         const TcTile& t) {
  if (threadIdx.x == 0) {
    *s_bad = 0;
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(128));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  load_gram_parts(G, t);
}

// ---------------------------------------------------------------------------------------
// D step: q0 <g(Z), D>, q1 ||D||^2, q2 f(Z) - f(X), q4 <D G, D>; others zero.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 2) k_rowtc_dstep(RowArgs a, int* err) {
  extern __shared__ unsigned char tsm_raw[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_bad;
  __shared__ float shq[8][8];
  __shared__ unsigned ticket;
  const int j = blockIdx.y;
  const Ctl& cj = a.ctl[j];
  const bool live = cj.active && !(a.run && *a.run == 0);
  float dq[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) dq[m] = 0.f;
  if (live) {
    const TcTile t = carve(tsm_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mrow = 32 * (warp & 3) + lane, c0 = 32 * (warp >> 2);  // TMEM row mapping
    const int c4 = threadIdx.x & 15, rw = threadIdx.x >> 4;            // coalesced mapping
    const int64_t row_base = (int64_t)blockIdx.x * TR;
    const int64_t colg = (int64_t)j * RC + 4 * c4;
    const float* X = (const float*)a.X;
    const float* g = (const float*)a.g_in;
    const float* B = (const float*)a.B;
    float* gZo = (float*)a.gZout;
    const float inv_rho = (float)(1.0 / cj.rho);
    const float alpha = (float)cj.alpha;
    tc_setup(&bar, &tmem_slot, &s_bad, (const float*)a.G + (int64_t)j * RC * RC, t);
    // Z tile: Z = Proj[X - g / rho], hi / lo parts
#pragma unroll
    for (int k = 0; k < CM_ROWS; ++k) {
      const int m = rw + 16 * k;
      const int64_t i = row_base + m;
      float4 x4 = make_float4(0.f, 0.f, 0.f, 0.f), g4 = x4;
      if (i < a.n) {
        x4 = ld4(X + i * a.ld + colg);
        g4 = ld4(g + i * a.ld + colg);
      }
      put4(t.ah, t.al, sw_chunk(m, 4 * c4, TR), zstep1(x4.x, g4.x, inv_rho), zstep1(x4.y, g4.y, inv_rho),
           zstep1(x4.z, g4.z, inv_rho), zstep1(x4.w, g4.w, inv_rho));
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // barrier init, TMEM address
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t tacc = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    run_product(t, tmem, &bar);  // Z G -> columns 0 .. 63
    float4 b4[CM_ROWS];  // B of the thread's elements, in flight during the product
#pragma unroll
    for (int k = 0; k < CM_ROWS; ++k) {
      const int64_t i = row_base + rw + 16 * k;
      b4[k] = i < a.n ? ld4(B + i * a.ld + colg) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    int issued = 1;  // products committed to `bar` (the drain waits for the last one)
    bool ok = wait_product(&bar, 0, &s_bad, err);
    float d[CM_ROWS][4];
    if (ok) {
      stage_acc(tacc, 0, t.al, mrow, c0);  // Z G -> T (the lo part of Z is no longer read)
      __syncthreads();
#pragma unroll
      for (int k = 0; k < CM_ROWS; ++k) {
        const int m = rw + 16 * k;
        const int64_t i = row_base + m;
        const bool rv = i < a.n;
        const float4 acc = ld_sw(t.al, m, 4 * c4);
        float4 x4 = make_float4(0.f, 0.f, 0.f, 0.f), g4 = x4;
        if (rv) {
          x4 = ld4(X + i * a.ld + colg);
          g4 = ld4(g + i * a.ld + colg);
        }
        const float xs[4] = {x4.x, x4.y, x4.z, x4.w}, gs[4] = {g4.x, g4.y, g4.z, g4.w};
        const float as[4] = {acc.x, acc.y, acc.z, acc.w};
        const float bs[4] = {b4[k].x, b4[k].y, b4[k].z, b4[k].w};
        float gz[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float z = zstep1(xs[q], gs[q], inv_rho);
          gz[q] = as[q] - bs[q];
          const float dv = rv ? dir1(z, gz[q], alpha) : 0.f;
          if (rv) {
            dq[0] += gz[q] * dv;
            dq[1] += dv * dv;
            dq[2] += 0.5f * (z - xs[q]) * (gz[q] + gs[q]);
          }
          d[k][q] = dv;
        }
        if (rv) st4(gZo + i * a.ld + colg, make_float4(gz[0], gz[1], gz[2], gz[3]));
        // D into the operand tile: the same chunk this thread just read (T in the lo part)
        put4(t.ah, t.al, sw_chunk(m, 4 * c4, TR), d[k][0], d[k][1], d[k][2], d[k][3]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      run_product(t, tmem + 64, &bar);  // D G -> columns 64 .. 127
      issued = 2;
      ok = wait_product(&bar, 1, &s_bad, err);
      if (ok) {
        stage_acc(tacc, 64, t.al, mrow, c0);  // D G -> T
        __syncthreads();
        float qq = 0.f;
#pragma unroll
        for (int k = 0; k < CM_ROWS; ++k) {
          const float4 dg = ld_sw(t.al, rw + 16 * k, 4 * c4);
          qq = fmaf(dg.x, d[k][0], qq);
          qq = fmaf(dg.y, d[k][1], qq);
          qq = fmaf(dg.z, d[k][2], qq);
          qq = fmaf(dg.w, d[k][3], qq);
        }
        dq[4] = qq;
      }
    }
    if (s_bad && threadIdx.x == 0) mbar_wait(&bar, (uint32_t)(issued - 1), kDrain);  // the last product issued
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128));
  }
  block_partials(a, dq, j, blockIdx.x, gridDim.x, shq, &ticket);
}

// ---------------------------------------------------------------------------------------
// Update: q0 ||P grad f(X')||^2, q1 1/2 <g' - B, X'>, q2 <S,S>, q3 <S,Y>, q4 <Y,Y>,
// q5 f(X') - f(Z), q6 zero entries of X'; q7 zero.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 2) k_rowtc_update(RowArgs a, int* err) {
  extern __shared__ unsigned char tsm_raw[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_bad;
  __shared__ float shq[8][8];
  __shared__ unsigned ticket;
  const int j = blockIdx.y;
  const Ctl& cj = a.ctl[j];
  const bool live = cj.active && !(a.run && *a.run == 0);
  float dq[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) dq[m] = 0.f;
  if (live) {
    const TcTile t = carve(tsm_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mrow = 32 * (warp & 3) + lane, c0 = 32 * (warp >> 2);
    const int c4 = threadIdx.x & 15, rw = threadIdx.x >> 4;
    const int64_t row_base = (int64_t)blockIdx.x * TR;
    const int64_t colg = (int64_t)j * RC + 4 * c4;
    float* X = (float*)a.Xout;  // in place: X_k in, X_{k+1} out
    float* g = (float*)a.gout;  // in place: g(X_k) in, g(X_{k+1}) out
    const float* gZ = (const float*)a.gZold;
    const float* B = (const float*)a.B;
    const float inv_rho = (float)(1.0 / cj.rho);
    const float alpha = (float)cj.alpha;
    const float pb = (float)cj.phibeta;
    tc_setup(&bar, &tmem_slot, &s_bad, (const float*)a.G + (int64_t)j * RC * RC, t);
    // X' tile: X' = Proj[Z + phi beta D] with Z, D recomputed from X, g, g(Z)
#pragma unroll
    for (int k = 0; k < CM_ROWS; ++k) {
      const int m = rw + 16 * k;
      const int64_t i = row_base + m;
      float4 x4 = make_float4(0.f, 0.f, 0.f, 0.f), g4 = x4, z4 = x4;
      if (i < a.n) {
        x4 = ld4(X + i * a.ld + colg);
        g4 = ld4(g + i * a.ld + colg);
        z4 = ld4(gZ + i * a.ld + colg);
      }
      const float xs[4] = {x4.x, x4.y, x4.z, x4.w}, gs[4] = {g4.x, g4.y, g4.z, g4.w};
      const float zs[4] = {z4.x, z4.y, z4.z, z4.w};
      float xn[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float z = zstep1(xs[q], gs[q], inv_rho);
        xn[q] = upd1(z, dir1(z, zs[q], alpha), pb);
      }
      put4(t.ah, t.al, sw_chunk(m, 4 * c4, TR), xn[0], xn[1], xn[2], xn[3]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t tacc = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    run_product(t, tmem, &bar);  // X' G -> columns 0 .. 63
    float4 b4[CM_ROWS];
#pragma unroll
    for (int k = 0; k < CM_ROWS; ++k) {
      const int64_t i = row_base + rw + 16 * k;
      b4[k] = i < a.n ? ld4(B + i * a.ld + colg) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const bool ok = wait_product(&bar, 0, &s_bad, err);
    if (ok) {
      stage_acc(tacc, 0, t.al, mrow, c0);  // X' G -> T
      __syncthreads();
#pragma unroll
      for (int k = 0; k < CM_ROWS; ++k) {
        const int m = rw + 16 * k;
        const int64_t i = row_base + m;
        if (i >= a.n) continue;
        const int64_t off = i * a.ld + colg;
        const float4 acc = ld_sw(t.al, m, 4 * c4);
        const float4 x4 = ld4(X + off), g4 = ld4(g + off), z4 = ld4(gZ + off);
        const float xs[4] = {x4.x, x4.y, x4.z, x4.w}, gs[4] = {g4.x, g4.y, g4.z, g4.w};
        const float zs[4] = {z4.x, z4.y, z4.z, z4.w};
        const float as[4] = {acc.x, acc.y, acc.z, acc.w};
        const float bs[4] = {b4[k].x, b4[k].y, b4[k].z, b4[k].w};
        float xo[4], go[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float z = zstep1(xs[q], gs[q], inv_rho);
          const float xn = upd1(z, dir1(z, zs[q], alpha), pb);
          const float gn = as[q] - bs[q];
          const float pgv = xn > 0.f ? gn : (gn < 0.f ? gn : 0.f);
          dq[0] += pgv * pgv;
          dq[1] += 0.5f * (gn - bs[q]) * xn;
          const float sv = xn - xs[q], yv = gn - gs[q];
          dq[2] += sv * sv;
          dq[3] += sv * yv;
          dq[4] += yv * yv;
          dq[5] += 0.5f * (xn - z) * (gn + zs[q]);
          if (xn == 0.f) dq[6] += 1.f;
          xo[q] = xn;
          go[q] = gn;
        }
        st4(X + off, make_float4(xo[0], xo[1], xo[2], xo[3]));
        st4(g + off, make_float4(go[0], go[1], go[2], go[3]));
      }
    }
    if (s_bad && threadIdx.x == 0) mbar_wait(&bar, 0, kDrain);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128));
  }
  block_partials(a, dq, j, blockIdx.x, gridDim.x, shq, &ticket);
}

// ---------------------------------------------------------------------------------------
// Block-start gradient: g = X G - B written to gout; q0 ||P grad f(X)||^2, q1 1/2 <g - B, X>,
// q6 zero entries of X; others zero.  The last CTA of each restart runs the block-start
// control step (ctl_mode).
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 2) k_rowtc_grad(RowArgs a, int* err) {
  extern __shared__ unsigned char tsm_raw[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_bad;
  __shared__ float shq[8][8];
  __shared__ unsigned ticket;
  const int j = blockIdx.y;
  const Ctl& cj = a.ctl[j];
  const bool live = cj.active && !(a.run && *a.run == 0);
  float dq[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) dq[m] = 0.f;
  if (live) {
    const TcTile t = carve(tsm_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mrow = 32 * (warp & 3) + lane, c0 = 32 * (warp >> 2);
    const int c4 = threadIdx.x & 15, rw = threadIdx.x >> 4;
    const int64_t row_base = (int64_t)blockIdx.x * TR;
    const int64_t colg = (int64_t)j * RC + 4 * c4;
    const float* X = (const float*)a.X;
    const float* B = (const float*)a.B;
    float* g = (float*)a.gout;
    tc_setup(&bar, &tmem_slot, &s_bad, (const float*)a.G + (int64_t)j * RC * RC, t);
#pragma unroll
    for (int k = 0; k < CM_ROWS; ++k) {
      const int m = rw + 16 * k;
      const int64_t i = row_base + m;
      const float4 x4 = i < a.n ? ld4(X + i * a.ld + colg) : make_float4(0.f, 0.f, 0.f, 0.f);
      put4(t.ah, t.al, sw_chunk(m, 4 * c4, TR), x4.x, x4.y, x4.z, x4.w);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t tacc = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    run_product(t, tmem, &bar);  // X G -> columns 0 .. 63
    float4 b4[CM_ROWS];
#pragma unroll
    for (int k = 0; k < CM_ROWS; ++k) {
      const int64_t i = row_base + rw + 16 * k;
      b4[k] = i < a.n ? ld4(B + i * a.ld + colg) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const bool ok = wait_product(&bar, 0, &s_bad, err);
    if (ok) {
      stage_acc(tacc, 0, t.al, mrow, c0);  // X G -> T
      __syncthreads();
#pragma unroll
      for (int k = 0; k < CM_ROWS; ++k) {
        const int m = rw + 16 * k;
        const int64_t i = row_base + m;
        if (i >= a.n) continue;
        const int64_t off = i * a.ld + colg;
        const float4 acc = ld_sw(t.al, m, 4 * c4);
        const float4 x4 = ld4(X + off);
        const float xs[4] = {x4.x, x4.y, x4.z, x4.w};
        const float as[4] = {acc.x, acc.y, acc.z, acc.w};
        const float bs[4] = {b4[k].x, b4[k].y, b4[k].z, b4[k].w};
        float go[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float gv = as[q] - bs[q];
          const float pgv = xs[q] > 0.f ? gv : (gv < 0.f ? gv : 0.f);
          dq[0] += pgv * pgv;
          dq[1] += 0.5f * (gv - bs[q]) * xs[q];
          if (xs[q] == 0.f) dq[6] += 1.f;
          go[q] = gv;
        }
        st4(g + off, make_float4(go[0], go[1], go[2], go[3]));
      }
    }
    if (s_bad && threadIdx.x == 0) mbar_wait(&bar, 0, kDrain);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128));
  }
  block_partials(a, dq, j, blockIdx.x, gridDim.x, shq, &ticket);
}

}  // namespace

bool rowtc_supported(int tdtype, int r, int nc) { return tdtype == 1 && r == RC && nc == 1; }

void launch_rowtc_dstep(const RowArgs& a, int* err, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_rowtc_dstep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    attr = true;
  }
  dim3 grid((unsigned)((a.n + TR - 1) / TR), (unsigned)a.b);
  k_rowtc_dstep<<<grid, 256, SMEM_BYTES, s>>>(a, err);
}

void launch_rowtc_grad(const RowArgs& a, int* err, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_rowtc_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    attr = true;
  }
  dim3 grid((unsigned)((a.n + TR - 1) / TR), (unsigned)a.b);
  k_rowtc_grad<<<grid, 256, SMEM_BYTES, s>>>(a, err);
}

void launch_rowtc_update(const RowArgs& a, int* err, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_rowtc_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    attr = true;
  }
  dim3 grid((unsigned)((a.n + TR - 1) / TR), (unsigned)a.b);
  k_rowtc_update<<<grid, 256, SMEM_BYTES, s>>>(a, err);
}

}  // namespace snmf
