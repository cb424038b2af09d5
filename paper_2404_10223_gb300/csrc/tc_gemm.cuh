// Grouped GEMM on the 5th-generation tensor cores (sm_103a): C = A B with A
// (M x K) and B (N x K) both K-major FP32 in global memory, each operand tile
// brought into shared memory by TMA (128-byte swizzle), split there into a
// TF32 high part and the TF32 remainder, and multiplied as
// A_hi B_hi + A_hi B_lo + A_lo B_hi by tcgen05.mma with the FP32 accumulator in
// tensor memory (the 3-term split product keeps about 21 bits of each operand).
// One CTA computes one 128 x 256 tile of one problem; problems of different
// sizes share a launch through a tile prefix sum.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace tnqe {

constexpr int TC_BM = 128, TC_BN = 256, TC_BK = 32;
constexpr int TC_THREADS = 128;
constexpr int TC_A_BYTES = TC_BM * TC_BK * 4;                 // 16 KiB
constexpr int TC_B_BYTES = TC_BN * TC_BK * 4;                 // 32 KiB
constexpr int TC_STAGE_BYTES = 2 * (TC_A_BYTES + TC_B_BYTES);  // hi + lo of A and B
constexpr int TC_STAGES = 2;
constexpr int TC_SMEM_BYTES = TC_STAGES * TC_STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;

struct TcGemmDesc {   // CUtensorMap members carry the required alignment
  CUtensorMap mapA;     // rows M, cols K (K contiguous), box 32 x 128
  CUtensorMap mapB;     // rows N, cols K (K contiguous), box 32 x 256
  float* C;             // element (m, n) at C + m * ldc + (n / cg) * cld + n % cg
  long long ldc;
  int M, N, K;
  int cg, cld;
  int tiles_n;
  int pad[2];
};

#if defined(__CUDACC__) && defined(TNQE_DEFINE_TC_KERNEL)
namespace tcdev {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ uint32_t mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok;
}
// Bounded wait on an mbarrier phase; false if the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
  for (long long i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
      ::"r"(smem_u32(dst)), "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 32 consecutive accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// K-major operand tile, 128-byte swizzle: 128-byte rows, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)2 << 61;             // SWIZZLE_128B
  return d;
}
// kind::tf32, FP32 accumulator, A and B K-major, M = 128, N = 256
constexpr uint32_t TC_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_BN >> 3) << 17) |
                              ((uint32_t)(TC_BM >> 4) << 24);

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}

}  // namespace tcdev

// error codes written to *err
constexpr int TC_ERR_TIMEOUT = 1;

__global__ void __launch_bounds__(TC_THREADS, 1)
    gemm_tf32x3_kernel(const TcGemmDesc* __restrict__ descs, const long long* __restrict__ tile_prefix, int nprob,
                       long long max_spin, int* __restrict__ err) {
  using namespace tcdev;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + TC_STAGES * TC_STAGE_BYTES);
  uint64_t* empty = full + TC_STAGES;
  uint64_t* accb = empty + TC_STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accb + 1);
  __shared__ int s_fail;

  const long long tile = blockIdx.x;
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tile_prefix[mid] <= tile) lo = mid; else hi = mid - 1;
  }
  const TcGemmDesc* d = descs + lo;
  const long long local = tile - tile_prefix[lo];
  const int tm = (int)(local / d->tiles_n), tn = (int)(local % d->tiles_n);
  const int m0 = tm * TC_BM, n0 = tn * TC_BN;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int KT = (d->K + TC_BK - 1) / TC_BK;

  if (tid == 0) {
    s_fail = 0;
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accb, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, TC_BN);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  auto stage_a = [&](int s) { return smem + s * TC_STAGE_BYTES; };
  auto stage_alo = [&](int s) { return smem + s * TC_STAGE_BYTES + TC_A_BYTES; };
  auto stage_b = [&](int s) { return smem + s * TC_STAGE_BYTES + 2 * TC_A_BYTES; };
  auto stage_blo = [&](int s) { return smem + s * TC_STAGE_BYTES + 2 * TC_A_BYTES + TC_B_BYTES; };
  auto issue = [&](int s, int kt) {
    mbar_expect_tx(&full[s], TC_A_BYTES + TC_B_BYTES);
    tma_load_2d(stage_a(s), &d->mapA, &full[s], kt * TC_BK, m0);
    tma_load_2d(stage_b(s), &d->mapB, &full[s], kt * TC_BK, n0);
  };
  if (tid == 0)
    for (int s = 0; s < TC_STAGES && s < KT; ++s) issue(s, s);

  int fail = 0;
  for (int kt = 0; kt < KT; ++kt) {
    const int s = kt % TC_STAGES;
    const uint32_t ph = (uint32_t)((kt / TC_STAGES) & 1);
    if (!mbar_wait(&full[s], ph, max_spin)) fail = 1;
    if (__syncthreads_or(fail)) break;
    // split the raw FP32 tiles: high TF32 part in place, remainder into the lo tile
    {
      float4* a = reinterpret_cast<float4*>(stage_a(s));
      float4* alo = reinterpret_cast<float4*>(stage_alo(s));
      float4* b = reinterpret_cast<float4*>(stage_b(s));
      float4* blo = reinterpret_cast<float4*>(stage_blo(s));
      for (int i = tid; i < TC_A_BYTES / 16; i += TC_THREADS) {
        const float4 x = a[i];
        float4 h, r;
        h.x = tf32_round(x.x); r.x = x.x - h.x;
        h.y = tf32_round(x.y); r.y = x.y - h.y;
        h.z = tf32_round(x.z); r.z = x.z - h.z;
        h.w = tf32_round(x.w); r.w = x.w - h.w;
        a[i] = h;
        alo[i] = r;
      }
      for (int i = tid; i < TC_B_BYTES / 16; i += TC_THREADS) {
        const float4 x = b[i];
        float4 h, r;
        h.x = tf32_round(x.x); r.x = x.x - h.x;
        h.y = tf32_round(x.y); r.y = x.y - h.y;
        h.z = tf32_round(x.z); r.z = x.z - h.z;
        h.w = tf32_round(x.w); r.w = x.w - h.w;
        b[i] = h;
        blo[i] = r;
      }
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t ah = smem_u32(stage_a(s)), al = smem_u32(stage_alo(s));
      const uint32_t bh = smem_u32(stage_b(s)), bl = smem_u32(stage_blo(s));
#pragma unroll
      for (int k = 0; k < TC_BK / 8; ++k) {           // 8 TF32 = 32 bytes per MMA along K
        const uint64_t dah = sw128_desc(ah + 32 * k), dal = sw128_desc(al + 32 * k);
        const uint64_t dbh = sw128_desc(bh + 32 * k), dbl = sw128_desc(bl + 32 * k);
        mma_tf32(tmem, dah, dbh, TC_IDESC, (kt > 0 || k > 0) ? 1u : 0u);
        mma_tf32(tmem, dah, dbl, TC_IDESC, 1u);
        mma_tf32(tmem, dal, dbh, TC_IDESC, 1u);
      }
      mma_commit(&empty[s]);
      if (kt + TC_STAGES < KT) {
        if (!mbar_wait(&empty[s], ph, max_spin)) fail = 1;
        else issue(s, kt + TC_STAGES);
      }
    }
  }
  if (tid == 0) mma_commit(accb);
  if (!mbar_wait(accb, 0, max_spin)) fail = 1;
  tc_fence_after();
  if (fail) {
    s_fail = 1;
    atomicExch(err, TC_ERR_TIMEOUT);
  }
  __syncthreads();
  if (!s_fail) {
    const int row = m0 + warp * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < TC_BN; c0 += 32) {
      uint32_t v[32];
      tmem_ld32(lane_base + c0, v);
      if (row < d->M) {
        float* crow = d->C + (long long)row * d->ldc;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int n = n0 + c0 + j;
          if (n < d->N) crow[(long long)(n / d->cg) * d->cld + (n % d->cg)] = __uint_as_float(v[j]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, TC_BN);
  }
}
#endif

}  // namespace tnqe
