// Sliced-BF16 grouped GEMM on the 5th-generation tensor cores (sm_103a).
//
// Both operands arrive as fixed-point BF16 slices (error-free splitting in the
// manner of Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59 (2012) 95):
// row r of an operand, scaled by 2^-e_r so that every entry is below 1/2 in
// magnitude, is written as x' = v_1 + v_2 + ... + v_S with
// v_i = S_i 2^(-8 i), S_i an integer in [-128, 128].  Every v_i is exact in
// BF16, every slice product v_i^A v_j^B is exact in FP32, and the sums
//   acc0 = sum_k v_1^A v_1^B      (multiples of 2^-16, |.| <= K 2^-2)
//   acc1 = sum_k v_1^A v_2^B      (multiples of 2^-24, |.| <= K 2^-9)
//   acc2 = sum_k v_2^A v_1^B
// stay exact in FP32 for K <= 1024, so the three leading orders carry no
// rounding at all; acc3 collects the orders i + j = 4, 5 (at most 2^-16 of the
// leading term) with ordinary FP32 rounding.  The epilogue adds the four
// accumulators error-free into a double-float (hi + lo, two FP32 values) and
// scales by 2^(e_r + e_c).
//
// Persistent: one CTA per SM walks the 128 x BN tiles (BN = 128 or 64) of all
// problems of the launch.  Thread 0 issues the TMA loads (3-D boxes: 32
// K-elements x rows x S slices, 64-byte swizzle) and the tcgen05.mma
// instructions; loads run ahead into the next tile, so its first stages land
// while the current tile's epilogue runs; the four accumulators take 4 BN
// columns of tensor memory; all four warps run the epilogue, 16 columns at a
// time through a small per-warp staging buffer for row-contiguous stores.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace tnqe {

constexpr int OZ_BM = 128, OZ_BK = 32;                 // BK in BF16 elements (64 bytes)
constexpr int OZ_BN_MAX = 128;                         // N tile: 128 or 64 (chosen per GEMM by the tuner)
constexpr int OZ_MAXS = 5;                             // slices per operand
constexpr int OZ_MAXK = 1024;                          // exactness bound of acc0..acc2
constexpr int OZ_THREADS = 128;
constexpr int OZ_SLICE_BYTES = OZ_BM * OZ_BK * 2;      // 8 KiB per slice tile
constexpr int OZ_MAX_STAGES = 4;
constexpr int OZ_STAGE_AREA = 196608;                  // pipeline stages: 2 S slice tiles each
constexpr int OZ_SLD = 17;                             // staging row stride (float2): 16 columns + 1
constexpr int OZ_STAGING_BYTES = 4 * 32 * OZ_SLD * 8;  // per-warp epilogue staging, 16 columns at a time
constexpr int OZ_SMEM_BYTES = OZ_STAGE_AREA + OZ_STAGING_BYTES + 1024 /*align*/ + 256 /*barriers*/;
// bytes of one pipeline stage: S slice tiles of A (128 rows) and of B (BN rows)
__host__ __device__ constexpr int oz_stage_bytes(int S, int BN) { return S * (OZ_SLICE_BYTES + BN * OZ_BK * 2); }
// pipeline depth: as many stages as fit the stage area
__host__ __device__ constexpr int oz_stages(int S, int BN) {
  return (OZ_STAGE_AREA / oz_stage_bytes(S, BN)) < OZ_MAX_STAGES ? (OZ_STAGE_AREA / oz_stage_bytes(S, BN))
                                                                 : OZ_MAX_STAGES;
}

struct OzGemmDesc {     // CUtensorMap members carry the required alignment
  CUtensorMap mapA;     // dims {K, M, S}: slice s of row m at A + (s * M + m) * ldK, box {32, 128, S}
  CUtensorMap mapB;     // dims {K, N, S}, box {32, BN, S}
  const int* ea;        // M row exponents of A
  const int* eb;        // N row exponents of B
  float2* C;            // element (m, n) at C + m * ldc + n, as (hi, lo)
  long long ldc;
  int M, N, K;
  int tiles_n;
  int nslices;          // 2 .. 5
  int pad[3];
};

#if defined(__CUDACC__) && defined(TNQE_DEFINE_OZ_KERNEL)
namespace ozdev {

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
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
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
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 16 consecutive accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// K-major operand tile, 64-byte swizzle: 64-byte rows, 8-row groups 512 bytes apart
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;   // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;            // descriptor version
  d |= (uint64_t)4 << 61;            // SWIZZLE_64B
  return d;
}
// kind::f16 with BF16 A and B, FP32 accumulator, both K-major, M = 128, N = BN
template <int BN>
__host__ __device__ constexpr uint32_t oz_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(OZ_BM >> 4) << 24);
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// 2^e as a float for -126 <= e <= 127
__device__ __forceinline__ float pow2f(int e) {
  e = max(-126, min(127, e));
  return __int_as_float((e + 127) << 23);
}

}  // namespace ozdev

constexpr int OZ_ERR_TIMEOUT = 1;

template <int BN, int S>
__global__ void __launch_bounds__(OZ_THREADS, 1)
    gemm_bf16s_kernel(const OzGemmDesc* __restrict__ descs, const long long* __restrict__ tile_prefix, int nprob,
                      long long total_tiles, long long max_spin, int* __restrict__ err) {
  using namespace ozdev;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  float2* staging = reinterpret_cast<float2*>(smem + OZ_STAGE_AREA);          // 4 warps x 32 rows x OZ_SLD
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + OZ_STAGE_AREA + OZ_STAGING_BYTES);
  uint64_t* empty = full + OZ_MAX_STAGES;
  uint64_t* accb = empty + OZ_MAX_STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accb + 1);
  __shared__ int s_fail;
  __shared__ int s_eb[BN];
  constexpr int TMEM_COLS = 4 * BN;                      // four accumulators
  constexpr uint32_t IDESC = oz_idesc<BN>();
  constexpr int NST = oz_stages(S, BN);
  constexpr int stage_bytes = oz_stage_bytes(S, BN);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  struct Tile {
    const OzGemmDesc* d;
    int m0, n0, KT;
  };
  auto tile_of = [&](long long t) -> Tile {
    Tile r{nullptr, 0, 0, 0};
    if (t >= total_tiles) return r;
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tile_prefix[mid] <= t) lo = mid; else hi = mid - 1;
    }
    r.d = descs + lo;
    const long long local = t - tile_prefix[lo];
    r.m0 = (int)(local / r.d->tiles_n) * OZ_BM;
    r.n0 = (int)(local % r.d->tiles_n) * BN;
    r.KT = (r.d->K + OZ_BK - 1) / OZ_BK;
    return r;
  };

  if (tid == 0) {
    s_fail = 0;
    for (int s = 0; s < OZ_MAX_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accb, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // Producer / MMA state (thread 0).  Loads and consumptions are numbered over all
  // k-tiles this CTA handles; load g goes to stage g % NST.  Loads run ahead into the
  // next tile, so its first stages land while the current tile's epilogue runs.
  long long base = 0;          // global index of the current tile's first k-tile
  long long issued = 0;        // loads issued so far
  Tile cur = tile_of(blockIdx.x), nxt = tile_of(blockIdx.x + (long long)gridDim.x);
  int fail = 0;
  auto stage_a = [&](int s) { return smem + s * stage_bytes; };
  auto stage_b = [&](int s) { return smem + s * stage_bytes + S * OZ_SLICE_BYTES; };
  // issue loads while issued < limit and the load exists in the current or next tile
  auto issue_upto = [&](long long limit) {
    while (!fail && issued < limit) {
      const Tile* t;
      int kt;
      if (issued < base + cur.KT) {
        t = &cur;
        kt = (int)(issued - base);
      } else if (nxt.d && issued < base + cur.KT + nxt.KT) {
        t = &nxt;
        kt = (int)(issued - base - cur.KT);
      } else {
        return;
      }
      const int s = (int)(issued % NST);
      if (issued >= NST && !mbar_wait(&empty[s], (uint32_t)(((issued - NST) / NST) & 1), max_spin)) {
        fail = 1;
        return;
      }
      mbar_expect_tx(&full[s], (uint32_t)stage_bytes);
      tma_load_3d(stage_a(s), &t->d->mapA, &full[s], kt * OZ_BK, t->m0, 0);
      tma_load_3d(stage_b(s), &t->d->mapB, &full[s], kt * OZ_BK, t->n0, 0);
      ++issued;
    }
  };
  if (tid == 0) issue_upto(NST);

  long long ntile = 0;
  for (long long tile = blockIdx.x; tile < total_tiles; tile += gridDim.x, ++ntile) {
    const Tile me = tile_of(tile);                      // every thread: this tile's problem and origin
    // ---- mainloop (thread 0); the other warps fetch the column exponents meanwhile
    if (tid == 0 && !fail) {
      for (int kt = 0; kt < cur.KT; ++kt) {
        const long long c = base + kt;
        const int s = (int)(c % NST);
        if (!mbar_wait(&full[s], (uint32_t)((c / NST) & 1), max_spin)) {
          fail = 1;
          break;
        }
        tc_fence_after();
        const uint64_t da0 = sw64_desc(smem_u32(stage_a(s))), db0 = sw64_desc(smem_u32(stage_b(s)));
#pragma unroll
        for (int k = 0; k < OZ_BK / 16; ++k) {        // 16 BF16 = 32 bytes per MMA along K
          const uint32_t acc_on = (kt > 0 || k > 0) ? 1u : 0u;
          auto da = [&](int i) { return da0 + (uint64_t)((i * OZ_SLICE_BYTES + 32 * k) >> 4); };
          auto db = [&](int j) { return db0 + (uint64_t)((j * (BN * OZ_BK * 2) + 32 * k) >> 4); };
          mma_bf16(tmem + 0 * BN, da(0), db(0), IDESC, acc_on);
          mma_bf16(tmem + 1 * BN, da(0), db(1), IDESC, acc_on);
          mma_bf16(tmem + 2 * BN, da(1), db(0), IDESC, acc_on);
#pragma unroll
          for (int i = 0; i < S; ++i)
#pragma unroll
            for (int j = 0; j < S; ++j) {
              if (i + j < 2 || i + j > S - 1) continue;
              mma_bf16(tmem + 3 * BN, da(i), db(j), IDESC, (acc_on || i != 0 || j != 2) ? 1u : 0u);
            }
        }
        mma_commit(&empty[s]);
        if (kt >= 1) issue_upto(c - 1 + NST + 1);       // refill the stage of k-tile c - 1
      }
      mma_commit(accb);                                 // arrives once every issued MMA is done
    }
    if (warp != 0)
      for (int i = tid - 32; i < BN; i += OZ_THREADS - 32) s_eb[i] = me.n0 + i < me.d->N ? me.d->eb[me.n0 + i] : 0;
    const int row = me.m0 + warp * 32 + lane;
    const int era = row < me.d->M ? me.d->ea[row] : 0;
    if (!mbar_wait(accb, (uint32_t)(ntile & 1), max_spin)) fail = 1;
    tc_fence_after();
    if (tid == 0 && !fail) issue_upto(base + cur.KT + NST);   // every stage is free: fill them for the next tile
    if (fail) atomicExch(&s_fail, 1);
    __syncthreads();
    if (s_fail) break;
    // ---- epilogue: TMEM -> (hi, lo) -> per-warp staging -> rows of C
    {
      const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
      float2* stg = staging + warp * 32 * OZ_SLD;
      const int ncols = min(BN, me.d->N - me.n0);
      const int mrows = me.d->M;
      const long long ldc = me.d->ldc;
      float2* Ct = me.d->C + me.n0;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t v0[16], v1[16], v2[16], v3[16];
        tmem_ld16(lane_base + 0 * BN + c0, v0);
        tmem_ld16(lane_base + 1 * BN + c0, v1);
        tmem_ld16(lane_base + 2 * BN + c0, v2);
        tmem_ld16(lane_base + 3 * BN + c0, v3);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          float s, e, e2;
          two_sum(__uint_as_float(v0[j]), __uint_as_float(v1[j]), s, e);
          two_sum(s, __uint_as_float(v2[j]), s, e2);
          e += e2;
          if (S >= 3) e += __uint_as_float(v3[j]);
          const float h = s + e;
          const float l = e - (h - s);
          const int ex = era + s_eb[c0 + j];
          const float s1 = pow2f(ex / 2), s2 = pow2f(ex - ex / 2);
          stg[lane * OZ_SLD + j] = make_float2(h * s1 * s2, l * s1 * s2);
        }
        __syncwarp();
        const int col = c0 + (lane & 15);
#pragma unroll 4
        for (int rr = 0; rr < 32; rr += 2) {
          const int r = rr + (lane >> 4);
          const int grow = me.m0 + warp * 32 + r;
          if (grow < mrows && col < ncols) Ct[(long long)grow * ldc + col] = stg[r * OZ_SLD + (lane & 15)];
        }
        __syncwarp();
      }
    }
    tc_fence_before();
    __syncthreads();                                    // TMEM read out before the next tile's MMAs
    tc_fence_after();
    if (tid == 0) {
      base += cur.KT;
      cur = nxt;
      nxt = tile_of(tile + 2LL * gridDim.x);
    }
  }
  if (tid == 0 && (fail || s_fail)) {
    atomicExch(err, OZ_ERR_TIMEOUT);
    // let the loads still in flight land before the CTA leaves
    for (long long q = base; q < issued; ++q) mbar_wait(&full[q % NST], (uint32_t)((q / NST) & 1), max_spin);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// Warp-specialised variant with N = 64 tiles and two TMEM accumulator sets
// (2 x 4 x 64 = 512 columns): warp 4 (one lane) issues the TMA loads and the
// MMAs of tile t into set t % 2 while warps 0-3 read tile t - 1 out of the
// other set, so the tensor pipe keeps working through the epilogue.
constexpr int OZW_THREADS = 160;
namespace ozdev {
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
}  // namespace ozdev

template <int S>
__global__ void __launch_bounds__(OZW_THREADS, 1)
    gemm_bf16s_ws_kernel(const OzGemmDesc* __restrict__ descs, const long long* __restrict__ tile_prefix, int nprob,
                         long long total_tiles, long long max_spin, int* __restrict__ err) {
  using namespace ozdev;
  constexpr int BN = 64;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  float2* staging = reinterpret_cast<float2*>(smem + OZ_STAGE_AREA);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + OZ_STAGE_AREA + OZ_STAGING_BYTES);
  uint64_t* empty = full + OZ_MAX_STAGES;
  uint64_t* accb = empty + OZ_MAX_STAGES;           // [2]: accumulator set ready
  uint64_t* tempty = accb + 2;                      // [2]: accumulator set read out (4 warp arrivals)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
  __shared__ volatile int s_fail;
  __shared__ int s_eb[4][BN];                       // per epilogue warp
  constexpr int TMEM_COLS = 512;
  constexpr uint32_t IDESC = oz_idesc<BN>();
  constexpr int NST = oz_stages(S, BN);
  constexpr int stage_bytes = oz_stage_bytes(S, BN);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  struct Tile {
    const OzGemmDesc* d;
    int m0, n0, KT;
  };
  auto tile_of = [&](long long t) -> Tile {
    Tile r{nullptr, 0, 0, 0};
    if (t >= total_tiles) return r;
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tile_prefix[mid] <= t) lo = mid; else hi = mid - 1;
    }
    r.d = descs + lo;
    const long long local = t - tile_prefix[lo];
    r.m0 = (int)(local / r.d->tiles_n) * OZ_BM;
    r.n0 = (int)(local % r.d->tiles_n) * BN;
    r.KT = (r.d->K + OZ_BK - 1) / OZ_BK;
    return r;
  };

  if (tid == 0) {
    s_fail = 0;
    for (int s = 0; s < OZ_MAX_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accb[b], 1);
      mbar_init(&tempty[b], 4);
    }
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 4) {
    if (lane == 0) {
      // ---- producer and MMA issuer
      long long base = 0, issued = 0;
      Tile cur = tile_of(blockIdx.x), nxt = tile_of(blockIdx.x + (long long)gridDim.x);
      int fail = 0;
      auto stage_a = [&](int s) { return smem + s * stage_bytes; };
      auto stage_b = [&](int s) { return smem + s * stage_bytes + S * OZ_SLICE_BYTES; };
      auto issue_upto = [&](long long limit) {
        while (!fail && issued < limit) {
          const Tile* t;
          int kt;
          if (issued < base + cur.KT) {
            t = &cur;
            kt = (int)(issued - base);
          } else if (nxt.d && issued < base + cur.KT + nxt.KT) {
            t = &nxt;
            kt = (int)(issued - base - cur.KT);
          } else {
            return;
          }
          const int s = (int)(issued % NST);
          if (issued >= NST && !mbar_wait(&empty[s], (uint32_t)(((issued - NST) / NST) & 1), max_spin)) {
            fail = 1;
            return;
          }
          mbar_expect_tx(&full[s], (uint32_t)stage_bytes);
          tma_load_3d(stage_a(s), &t->d->mapA, &full[s], kt * OZ_BK, t->m0, 0);
          tma_load_3d(stage_b(s), &t->d->mapB, &full[s], kt * OZ_BK, t->n0, 0);
          ++issued;
        }
      };
      issue_upto(NST);
      long long lt = 0;
      for (long long tile = blockIdx.x; tile < total_tiles && !fail && !s_fail; tile += gridDim.x, ++lt) {
        const int b = (int)(lt & 1);
        if (lt >= 2 && !mbar_wait(&tempty[b], (uint32_t)(((lt - 2) >> 1) & 1), max_spin)) {
          fail = 1;
          break;
        }
        tc_fence_after();
        const uint32_t tacc = tmem + (uint32_t)(b * 4 * BN);
        for (int kt = 0; kt < cur.KT; ++kt) {
          const long long c = base + kt;
          const int s = (int)(c % NST);
          if (!mbar_wait(&full[s], (uint32_t)((c / NST) & 1), max_spin)) {
            fail = 1;
            break;
          }
          tc_fence_after();
          const uint64_t da0 = sw64_desc(smem_u32(stage_a(s))), db0 = sw64_desc(smem_u32(stage_b(s)));
#pragma unroll
          for (int k = 0; k < OZ_BK / 16; ++k) {
            const uint32_t acc_on = (kt > 0 || k > 0) ? 1u : 0u;
            auto da = [&](int i) { return da0 + (uint64_t)((i * OZ_SLICE_BYTES + 32 * k) >> 4); };
            auto db = [&](int j) { return db0 + (uint64_t)((j * (BN * OZ_BK * 2) + 32 * k) >> 4); };
            mma_bf16(tacc + 0 * BN, da(0), db(0), IDESC, acc_on);
            mma_bf16(tacc + 1 * BN, da(0), db(1), IDESC, acc_on);
            mma_bf16(tacc + 2 * BN, da(1), db(0), IDESC, acc_on);
#pragma unroll
            for (int i = 0; i < S; ++i)
#pragma unroll
              for (int j = 0; j < S; ++j) {
                if (i + j < 2 || i + j > S - 1) continue;
                mma_bf16(tacc + 3 * BN, da(i), db(j), IDESC, (acc_on || i != 0 || j != 2) ? 1u : 0u);
              }
          }
          mma_commit(&empty[s]);
          if (kt >= 1) issue_upto(c - 1 + NST + 1);
        }
        mma_commit(&accb[b]);                            // arrives once every issued MMA is done
        if (fail) break;
        issue_upto(base + cur.KT + NST - 1);             // loads that only needed earlier k-tiles
        base += cur.KT;
        cur = nxt;
        nxt = tile_of(tile + 2LL * gridDim.x);
      }
      if (fail) {
        s_fail = 1;
        atomicExch(err, OZ_ERR_TIMEOUT);
      }
      // let the loads still in flight land before the CTA leaves
      for (long long q = base; q < issued; ++q) mbar_wait(&full[q % NST], (uint32_t)((q / NST) & 1), max_spin);
    }
  } else {
    // ---- epilogue warps 0-3: TMEM set t % 2 -> (hi, lo) -> per-warp staging -> rows of C
    long long lt = 0;
    for (long long tile = blockIdx.x; tile < total_tiles; tile += gridDim.x, ++lt) {
      if (s_fail) break;
      const Tile me = tile_of(tile);
      const int b = (int)(lt & 1);
      for (int i = lane; i < BN; i += 32) s_eb[warp][i] = me.n0 + i < me.d->N ? me.d->eb[me.n0 + i] : 0;
      const int row = me.m0 + warp * 32 + lane;
      const int era = row < me.d->M ? me.d->ea[row] : 0;
      __syncwarp();
      if (!mbar_wait(&accb[b], (uint32_t)((lt >> 1) & 1), max_spin)) {
        s_fail = 1;
        atomicExch(err, OZ_ERR_TIMEOUT);
        break;
      }
      tc_fence_after();
      const uint32_t lane_base = tmem + (uint32_t)(b * 4 * BN) + ((uint32_t)(warp * 32) << 16);
      float2* stg = staging + warp * 32 * OZ_SLD;
      const int ncols = min(BN, me.d->N - me.n0);
      const int mrows = me.d->M;
      const long long ldc = me.d->ldc;
      float2* Ct = me.d->C + me.n0;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t v0[16], v1[16], v2[16], v3[16];
        tmem_ld16(lane_base + 0 * BN + c0, v0);
        tmem_ld16(lane_base + 1 * BN + c0, v1);
        tmem_ld16(lane_base + 2 * BN + c0, v2);
        tmem_ld16(lane_base + 3 * BN + c0, v3);
        tmem_wait_ld();
        if (c0 + 16 >= BN) {                             // this warp's lanes are read out: free the set
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&tempty[b]);
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          float s, e, e2;
          two_sum(__uint_as_float(v0[j]), __uint_as_float(v1[j]), s, e);
          two_sum(s, __uint_as_float(v2[j]), s, e2);
          e += e2;
          if (S >= 3) e += __uint_as_float(v3[j]);
          const float h = s + e;
          const float l = e - (h - s);
          const int ex = era + s_eb[warp][c0 + j];
          const float s1 = pow2f(ex / 2), s2 = pow2f(ex - ex / 2);
          stg[lane * OZ_SLD + j] = make_float2(h * s1 * s2, l * s1 * s2);
        }
        __syncwarp();
        const int col = c0 + (lane & 15);
#pragma unroll 4
        for (int rr = 0; rr < 32; rr += 2) {
          const int r = rr + (lane >> 4);
          const int grow = me.m0 + warp * 32 + r;
          if (grow < mrows && col < ncols) Ct[(long long)grow * ldc + col] = stg[r * OZ_SLD + (lane & 15)];
        }
        __syncwarp();
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

#endif

}  // namespace tnqe
