// Sliced-BF16 transfer contraction (tcgen05 GEMMs with exact leading-order
// accumulation; see oz_gemm.cuh) with double-float environments.
//
// Per site and pair, environments L[a][w][b] are double-floats (hi, lo FP32):
//   slice A   L rows (a,w) over b          -> BF16 slices + row exponents
//   stage 1   X[(a,w)][(k',b')] = L . ketT               sliced tcgen05 GEMM
//   stage 2   Y[(a,k)][(w',b')] = sum W X                double-float sparse MPO
//   slice B   Y columns (w',b') over (a,k) -> BF16 slices (K-major, transposed)
//   stage 3   L'[a'][(w',b')]   = braT . Yt              sliced tcgen05 GEMM
// The site tensors (FP64) are sliced once per call: ketT rows (k',b') over b,
// braT rows a' over (a,k).  Every value outside the tensor cores stays a
// double-float (about 48 significant bits); the tensor cores see only exact
// BF16 slices, so the contraction error is the slicing truncation alone.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.h"
#define TNQE_DEFINE_OZ_KERNEL
#include "oz_gemm.cuh"

namespace tnqe {
namespace {

// Error-free transforms with explicit rounding (never contracted into FMAs).
__device__ __forceinline__ void two_sum_rn(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (ah, al) += (vh, vl) * (xh, xl)
__device__ __forceinline__ void df_fma(float vh, float vl, float xh, float xl, float& ah, float& al) {
  const float p = __fmul_rn(vh, xh);
  const float pe = __fadd_rn(fmaf(vh, xh, -p), __fadd_rn(__fmul_rn(vh, xl), __fmul_rn(vl, xh)));
  float s, e;
  two_sum_rn(ah, p, s, e);
  ah = s;
  al = __fadd_rn(al, __fadd_rn(e, pe));
}
__device__ __forceinline__ float2 df_norm(float h, float l) {
  const float s = __fadd_rn(h, l);
  return make_float2(s, __fsub_rn(l, __fsub_rn(s, h)));
}
__device__ __forceinline__ int find_prob(const long long* prefix, int nprob, long long x) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}
// row exponent e with max|x| 2^-e < 1/2 (0 for an all-zero row)
__device__ __forceinline__ int row_exponent_f(float m) { return m > 0.f ? ilogbf(m) + 2 : 0; }
__device__ __forceinline__ int row_exponent_d(double m) { return m > 0.0 ? ilogb(m) + 2 : 0; }

// cp.async of 16 bytes (cp_bytes16) or 8 bytes; bytes beyond src_bytes are zero-filled
__device__ __forceinline__ void cp_async_zfill(void* dst, const void* src, int cp_bytes16, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if (cp_bytes16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}

// x 2^k: one multiplication by the exact power of two where 2^k is a normal
// float (the product is then correctly rounded, as the scaling is), ldexpf beyond
__device__ __forceinline__ float scale2(float x, int k) {
  return (k >= -126 && k <= 127) ? __fmul_rn(x, __int_as_float((127 + k) << 23)) : ldexpf(x, k);
}
// Slices of one double-float value x = hi + lo (|x| 2^-e < 1/2): out[i] = S_i 2^-(8(i+1)).
__device__ __forceinline__ void slice_df(float hi, float lo, int e, int ns, __nv_bfloat16* out, long long stride) {
  float th = scale2(hi, 8 - e), tl = scale2(lo, 8 - e);
  float unit = 1.f / 256.f;                      // 2^-8(i+1), exact
  for (int i = 0; i < ns; ++i) {
    const float S = rintf(th);
    float sh, sl;
    two_sum_rn(__fsub_rn(th, S), tl, sh, sl);
    out[i * stride] = __float2bfloat16_rn(__fmul_rn(S, unit));
    th = __fmul_rn(sh, 256.f);
    tl = __fmul_rn(sl, 256.f);
    unit = __fmul_rn(unit, 1.f / 256.f);
  }
}
// slice_df of four consecutive values, each slice stored as one 8-byte word (out 8-byte aligned)
__device__ __forceinline__ void slice_df4(const float2* x, int e, int ns, __nv_bfloat16* out, long long stride) {
  float th[4], tl[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    th[u] = scale2(x[u].x, 8 - e);
    tl[u] = scale2(x[u].y, 8 - e);
  }
  float unit = 1.f / 256.f;                      // 2^-8(i+1), exact
  for (int i = 0; i < ns; ++i) {
    unsigned short o[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float S = rintf(th[u]);
      float sh, sl;
      two_sum_rn(__fsub_rn(th[u], S), tl[u], sh, sl);
      o[u] = __bfloat16_as_ushort(__float2bfloat16_rn(__fmul_rn(S, unit)));
      th[u] = __fmul_rn(sh, 256.f);
      tl[u] = __fmul_rn(sl, 256.f);
    }
    unit = __fmul_rn(unit, 1.f / 256.f);
    uint2 w;
    w.x = (unsigned)o[0] | ((unsigned)o[1] << 16);
    w.y = (unsigned)o[2] | ((unsigned)o[3] << 16);
    *reinterpret_cast<uint2*>(out + i * stride) = w;
  }
}
__device__ __forceinline__ void slice_d(double x, int e, int ns, __nv_bfloat16* out, long long stride) {
  double t = ldexp(x, 8 - e);
  for (int i = 0; i < ns; ++i) {
    const double S = rint(t);
    out[i * stride] = __float2bfloat16_rn(ldexpf((float)S, -8 * (i + 1)));
    t = (t - S) * 256.0;
  }
}

// One warp per row: df rows over K -> slices [ns][rows][ldK] and exponents.
__global__ void __launch_bounds__(256) slice_rows_kernel(const SliceRowsDesc* __restrict__ descs,
                                                         const long long* __restrict__ prefix, int nprob,
                                                         long long total) {
  const long long task = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (task >= total) return;
  const int lane = threadIdx.x & 31;
  const int p = find_prob(prefix, nprob, task);
  const SliceRowsDesc& d = descs[p];
  const long long r = task - prefix[p];
  const float2* src = d.src + r * d.ld;
  __nv_bfloat16* dst = d.dst + r * d.ldK;
  if (d.K <= 256) {
    // the row sits in registers (four consecutive values per lane and 128-value chunk):
    // one read, and each slice leaves as 8-byte words
    float2 v[8];
    float m = 0.f;
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = 128 * j + 4 * lane + u;
        v[4 * j + u] = k < d.K ? src[k] : make_float2(0.f, 0.f);
        m = fmaxf(m, fabsf(v[4 * j + u].x));
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    const int e = row_exponent_f(m);
    if (lane == 0) d.exps[r] = e;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int k0 = 128 * j + 4 * lane;
      if (k0 + 4 <= d.K) {
        slice_df4(v + 4 * j, e, d.ns, dst + k0, d.slice_stride);
      } else {
        for (int u = 0; u < 4 && k0 + u < d.K; ++u) slice_df(v[4 * j + u].x, v[4 * j + u].y, e, d.ns, dst + k0 + u, d.slice_stride);
      }
    }
    return;
  }
  float m = 0.f;
  for (int k = lane; k < d.K; k += 32) m = fmaxf(m, fabsf(src[k].x));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  const int e = row_exponent_f(m);
  if (lane == 0) d.exps[r] = e;
  for (int k = lane; k < d.K; k += 32) {
    const float2 x = src[k];
    slice_df(x.x, x.y, e, d.ns, dst + k, d.slice_stride);
  }
}

// The same for K > 1024 (tile too large for shared memory): two passes over global memory.
__global__ void __launch_bounds__(256) slice_cols_global_kernel(const SliceColsDesc* __restrict__ descs,
                                                                const long long* __restrict__ prefix, int nprob) {
  __shared__ float2 tile[64][17];
  __shared__ float red[16][17];
  __shared__ int sexp[16];
  const long long task = blockIdx.x;
  const int p = find_prob(prefix, nprob, task);
  const SliceColsDesc& d = descs[p];
  const int c0 = (int)(task - prefix[p]) * 16;
  const int tid = threadIdx.x, cc = tid & 15, rr = tid >> 4;   // 16 columns x 16 row groups
  const int col = c0 + cc;
  float m = 0.f;
  if (col < d.ncols)
    for (int k = rr; k < d.K; k += 16) m = fmaxf(m, fabsf(d.src[(long long)k * d.ld + col].x));
  red[rr][cc] = m;
  __syncthreads();
  if (tid < 16) {
    float mm = 0.f;
    for (int i = 0; i < 16; ++i) mm = fmaxf(mm, red[i][tid]);
    const int e = row_exponent_f(mm);
    sexp[tid] = e;
    if (c0 + tid < d.ncols) d.exps[c0 + tid] = e;
  }
  __syncthreads();
  // writer mapping: column wc = tid / 16, four consecutive k per thread
  const int wc = tid >> 4, wk = (tid & 15) * 4;
  for (int k0 = 0; k0 < d.K; k0 += 64) {
    for (int i = tid; i < 64 * 16; i += 256) {
      const int k = k0 + (i >> 4), c = c0 + (i & 15);
      tile[i >> 4][i & 15] = (k < d.K && c < d.ncols) ? d.src[(long long)k * d.ld + c] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    if (c0 + wc < d.ncols) {
      __nv_bfloat16* dst = d.dst + (long long)(c0 + wc) * d.ldK;
      for (int u = 0; u < 4; ++u) {
        const int k = k0 + wk + u;
        if (k < d.K) slice_df(tile[wk + u][wc].x, tile[wk + u][wc].y, sexp[wc], d.ns, dst + k, d.slice_stride);
      }
    }
    __syncthreads();
  }
}

// Columns (w',b') of Y[(a,k)][(w',b')] over K = (a,k), transposed to K-major slices.
// One CTA per 16 columns of one problem; 256 threads.  The K x 16 tile is read
// from global memory once, by cp.async into shared memory laid out column by
// column (stride K + 1 elements, so neither the copies nor the reads of one
// column collide in the banks); the column maxima and all slices come from there.
constexpr int SLICE_COLS_SMEM_MAX = 16 * (1024 + 1) * 8;
__global__ void __launch_bounds__(256) slice_cols_kernel(const SliceColsDesc* __restrict__ descs,
                                                         const long long* __restrict__ prefix, int nprob) {
  extern __shared__ __align__(16) float2 tl[];
  __shared__ float red[16][17];
  __shared__ int sexp[16];
  const long long task = blockIdx.x;
  const int p = find_prob(prefix, nprob, task);
  const SliceColsDesc& d = descs[p];
  const int c0 = (int)(task - prefix[p]) * 16;
  const int tid = threadIdx.x, K = d.K, KS = K + 1;
  const float2* src = d.src + c0;
  for (int i = tid; i < K * 16; i += 256) {
    const int k = i >> 4, c = i & 15;
    const int bytes = c0 + c < d.ncols ? 8 : 0;
    cp_async_zfill(tl + c * KS + k, bytes ? src + (long long)k * d.ld + c : src, 0, bytes);
  }
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  const int wc = tid >> 4, lk = tid & 15;       // column, lane within the column's 16 threads
  const float2* colp = tl + wc * KS;
  float m = 0.f;
  for (int k = lk; k < K; k += 16) m = fmaxf(m, fabsf(colp[k].x));
  red[wc][lk] = m;
  __syncthreads();
  if (tid < 16) {
    float mm = 0.f;
    for (int i = 0; i < 16; ++i) mm = fmaxf(mm, red[tid][i]);
    const int e = row_exponent_f(mm);
    sexp[tid] = e;
    if (c0 + tid < d.ncols) d.exps[c0 + tid] = e;
  }
  __syncthreads();
  if (c0 + wc >= d.ncols) return;
  // four consecutive k per thread, stored as one 8-byte word per slice: the 16
  // threads of a column write 128 contiguous bytes per slice
  __nv_bfloat16* dst = d.dst + (long long)(c0 + wc) * d.ldK;
  const int e = sexp[wc];
  for (int k0 = lk * 4; k0 < K; k0 += 64) {
    if (k0 + 4 <= K) {
      slice_df4(colp + k0, e, d.ns, dst + k0, d.slice_stride);
    } else {
      for (int k = k0; k < K; ++k) slice_df(colp[k].x, colp[k].y, e, d.ns, dst + k, d.slice_stride);
    }
  }
}

// FP64 site tensors -> K-major slices.  mode 0 (ket): rows (k',b') over b of
// B[b][k'][b'];  mode 1 (bra): rows a' over (a,k) of A[a][k][a'].  Warp per row.
__global__ void __launch_bounds__(256) slice_sites_kernel(const SliceSiteDesc* __restrict__ descs,
                                                          const long long* __restrict__ prefix, int nprob,
                                                          long long total) {
  const long long task = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (task >= total) return;
  const int lane = threadIdx.x & 31;
  const int p = find_prob(prefix, nprob, task);
  const SliceSiteDesc& d = descs[p];
  const int r = (int)(task - prefix[p]);
  int K;
  long long base, step;
  if (d.mode == 0) {            // row (k', b'): element b at src[(b * 4 + k') * cr + b']
    const int kp = r / d.cr, bp = r % d.cr;
    K = d.cl;
    base = (long long)kp * d.cr + bp;
    step = 4LL * d.cr;
  } else {                      // row a': element (a, k) at src[(a * 4 + k) * cr + a']
    K = 4 * d.cl;
    base = r;
    step = d.cr;
  }
  double m = 0.0;
  for (int k = lane; k < K; k += 32) m = fmax(m, fabs(d.src[base + k * step]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  const int e = row_exponent_d(m);
  if (lane == 0) d.exps[r] = e;
  __nv_bfloat16* dst = d.dst + (long long)r * d.ldK;
  for (int k = lane; k < K; k += 32) slice_d(d.src[base + k * step], e, d.ns, dst + k, d.slice_stride);
}

// Y[a][row][0:width] = sum val * X[a][col][0:width], double-float; one warp per (a, row)
__global__ void __launch_bounds__(256) spmm_df_kernel(const SpmmDfDesc* __restrict__ descs,
                                                      const long long* __restrict__ prefix, int nprob,
                                                      long long total) {
  const long long task = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (task >= total) return;
  const int lane = threadIdx.x & 31;
  const int p = find_prob(prefix, nprob, task);
  const SpmmDfDesc& d = descs[p];
  const long long local = task - prefix[p];
  const int a = (int)(local / d.nrows), row = (int)(local % d.nrows);
  const int e0 = d.rowptr[row], e1 = d.rowptr[row + 1];
  const float2* Xa = d.X + (long long)a * d.ncols_x * d.width;
  float2* y = d.Y + ((long long)a * d.nrows + row) * d.width;
  for (int c0 = 0; c0 < d.width; c0 += 128) {
    float ah[4] = {0.f, 0.f, 0.f, 0.f}, al[4] = {0.f, 0.f, 0.f, 0.f};
    for (int e = e0; e < e1; ++e) {
      const float2 v = d.val[e];
      const float2* x = Xa + (long long)d.col[e] * d.width;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = c0 + lane + 32 * u;
        if (c < d.width) {
          const float2 xv = x[c];
          df_fma(v.x, v.y, xv.x, xv.y, ah[u], al[u]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = c0 + lane + 32 * u;
      if (c < d.width) y[c] = df_norm(ah[u], al[u]);
    }
  }
}

// (ah, al) += (vh, vl) * (xh, xl) with the cross terms fused: 12 FP32 operations
__device__ __forceinline__ void df_fma_fused(float vh, float vl, float xh, float xl, float& ah, float& al) {
  const float p = __fmul_rn(vh, xh);
  const float pe = fmaf(vh, xl, fmaf(vl, xh, fmaf(vh, xh, -p)));
  float s, e;
  two_sum_rn(ah, p, s, e);
  ah = s;
  al = __fadd_rn(al, __fadd_rn(e, pe));
}

// Y[a][row][b0:b0+BW] for every row, with X[a][:][b0:b0+BW] staged in shared
// memory once (each X element is read by every nonzero of its column).  The
// slab arrives by cp.async, 16 bytes per copy where the rows allow it, so a
// CTA keeps its whole slab in flight instead of one element per thread.  Each
// thread then owns one row and all BW columns: BW independent double-float
// accumulations share every (value, column) load, and rows go in descending
// nonzero count so the threads of a warp run loops of similar length.
constexpr int SPMM_SMEM_BYTES = 112 * 1024;
constexpr int SPMM_THREADS = 256;
template <int BW, int TPR>
__global__ void __launch_bounds__(SPMM_THREADS, 2) spmm_df_smem_kernel(const SpmmDfDesc* __restrict__ descs,
                                                                    const long long* __restrict__ prefix, int nprob) {
  extern __shared__ __align__(16) float2 xs[];
  constexpr int NC = BW / TPR;                   // columns per thread: c, c + TPR, ...
  constexpr int RPP = SPMM_THREADS / TPR;        // rows per pass
  const long long task = blockIdx.x;
  const int p = find_prob(prefix, nprob, task);
  const SpmmDfDesc& d = descs[p];
  const int nbt = (d.width + BW - 1) / BW;
  const long long local = task - prefix[p];
  const int a = (int)(local / nbt), b0 = (int)(local % nbt) * BW;
  const int tid = threadIdx.x;
  const int width = d.width, ncols = d.ncols_x;
  const float2* Xa = d.X + (long long)a * ncols * width + b0;
  if (BW >= 2 && (width & 1) == 0 && (reinterpret_cast<size_t>(Xa) & 15) == 0) {
    constexpr int CPR = BW / 2;                  // 16-byte copies per slab row
    for (int i = tid; i < ncols * CPR; i += SPMM_THREADS) {
      const int r = i / CPR, q = i - r * CPR;
      const int c0 = b0 + 2 * q;
      const int bytes = c0 + 2 <= width ? 16 : (c0 < width ? 8 : 0);
      const float2* src = bytes ? Xa + (long long)r * width + 2 * q : Xa;
      cp_async_zfill(xs + r * BW + 2 * q, src, 1, bytes);
    }
  } else {
    for (int i = tid; i < ncols * BW; i += SPMM_THREADS) {
      const int r = i / BW, c = i - r * BW;
      const int bytes = b0 + c < width ? 8 : 0;
      const float2* src = bytes ? Xa + (long long)r * width + c : Xa;
      cp_async_zfill(xs + i, src, 0, bytes);
    }
  }
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  float2* Ya = d.Y + (long long)a * d.nrows * width + b0;
  const float4* __restrict__ ent = d.ent;
  const int c = tid % TPR;
  for (int rr = tid / TPR; rr < d.nrows; rr += RPP) {
    const int row = d.rowperm[rr];
    const int e0 = d.rowptr[row], e1 = d.rowptr[row + 1];
    float ah[NC], al[NC];
#pragma unroll
    for (int u = 0; u < NC; ++u) ah[u] = al[u] = 0.f;
    for (int e = e0; e < e1; ++e) {
      const float4 en = __ldg(ent + e);
      const float2* xr = xs + __float_as_int(en.z) * BW + c;
#pragma unroll
      for (int u = 0; u < NC; ++u) {
        const float2 x = xr[u * TPR];
        df_fma_fused(en.x, en.y, x.x, x.y, ah[u], al[u]);
      }
    }
    float2* y = Ya + (long long)row * width + c;
#pragma unroll
    for (int u = 0; u < NC; ++u)
      if (b0 + c + u * TPR < width) y[u * TPR] = df_norm(ah[u], al[u]);
  }
}

__global__ void unit_env_kernel(float2* const* __restrict__ env, int n) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) env[p][0] = make_float2(1.f, 0.f);
}
__global__ void unit_env_f64_kernel(double* const* __restrict__ env, int n) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) env[p][0] = 1.0;
}
__global__ void unit_env_f32_kernel(float* const* __restrict__ env, int n) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) env[p][0] = 1.f;
}

__global__ void extract_df_kernel(const float2* const* __restrict__ fin, int npairs, double* H, double* S) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npairs) return;
  const float2 s = fin[p][0], h = fin[p][1];   // identity-string and completed-Hamiltonian channels
  S[p] = (double)s.x + (double)s.y;
  H[p] = (double)h.x + (double)h.y;
}

// H[idx[p]] = h[p], S[idx[p]] = s[p]
__global__ void scatter_pairs_kernel(const double* __restrict__ h, const double* __restrict__ s,
                                     const int* __restrict__ idx, int n, double* H, double* S) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  H[idx[p]] = h[p];
  S[idx[p]] = s[p];
}

}  // namespace

int launch_scatter_pairs(const double* h, const double* s, const int* idx, int n, double* H, double* S,
                         void* stream) {
  if (n <= 0) return 0;
  scatter_pairs_kernel<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(h, s, idx, n, H, S);
  return (int)cudaGetLastError();
}
int launch_slice_rows(const SliceRowsDesc* d, const long long* prefix, int n, long long rows, void* stream) {
  if (rows <= 0) return 0;
  slice_rows_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, (cudaStream_t)stream>>>(d, prefix, n, rows);
  return (int)cudaGetLastError();
}
int launch_slice_cols(const SliceColsDesc* d, const long long* prefix, int n, long long blocks, int max_k,
                      void* stream) {
  if (blocks <= 0) return 0;
  cudaStream_t st = (cudaStream_t)stream;
  if (max_k > 1024) {
    slice_cols_global_kernel<<<(unsigned)blocks, 256, 0, st>>>(d, prefix, n);
    return (int)cudaGetLastError();
  }
  const cudaError_t e =
      cudaFuncSetAttribute(slice_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SLICE_COLS_SMEM_MAX);
  if (e != cudaSuccess) return (int)e;
  slice_cols_kernel<<<(unsigned)blocks, 256, (size_t)16 * (max_k + 1) * sizeof(float2), st>>>(d, prefix, n);
  return (int)cudaGetLastError();
}
int launch_slice_sites(const SliceSiteDesc* d, const long long* prefix, int n, long long rows, void* stream) {
  if (rows <= 0) return 0;
  slice_sites_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, (cudaStream_t)stream>>>(d, prefix, n, rows);
  return (int)cudaGetLastError();
}
int launch_spmm_df(const SpmmDfDesc* d, const long long* prefix, int n, long long total, void* stream) {
  if (total <= 0) return 0;
  spmm_df_kernel<<<(unsigned)((total + 7) / 8), 256, 0, (cudaStream_t)stream>>>(d, prefix, n, total);
  return (int)cudaGetLastError();
}
int spmm_df_smem_width(int max_ncols_x) {
  for (int bw = 8; bw >= 1; bw >>= 1)
    if ((long long)max_ncols_x * bw * (long long)sizeof(float2) <= SPMM_SMEM_BYTES) return bw;
  return 0;
}
#ifndef TNQE_SPMM_TPR
#define TNQE_SPMM_TPR 4
#endif
template <int BW>
static cudaError_t launch_spmm_bw(const SpmmDfDesc* d, const long long* prefix, int n, long long blocks, size_t smem,
                                  cudaStream_t st) {
  constexpr int TPR = TNQE_SPMM_TPR < BW ? TNQE_SPMM_TPR : BW;
  cudaError_t e = cudaFuncSetAttribute(spmm_df_smem_kernel<BW, TPR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       SPMM_SMEM_BYTES);
  if (e == cudaSuccess) spmm_df_smem_kernel<BW, TPR><<<(unsigned)blocks, SPMM_THREADS, smem, st>>>(d, prefix, n);
  return e;
}
int launch_spmm_df_smem(const SpmmDfDesc* d, const long long* prefix, int n, long long blocks, int bw,
                        int max_ncols_x, void* stream) {
  if (blocks <= 0) return 0;
  const size_t smem = (size_t)max_ncols_x * bw * sizeof(float2);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  switch (bw) {
    case 8: e = launch_spmm_bw<8>(d, prefix, n, blocks, smem, st); break;
    case 4: e = launch_spmm_bw<4>(d, prefix, n, blocks, smem, st); break;
    case 2: e = launch_spmm_bw<2>(d, prefix, n, blocks, smem, st); break;
    default: e = launch_spmm_bw<1>(d, prefix, n, blocks, smem, st); break;
  }
  if (e != cudaSuccess) return (int)e;
  return (int)cudaGetLastError();
}

int launch_unit_env(float2* const* env, int n, void* stream) {
  if (n <= 0) return 0;
  unit_env_kernel<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(env, n);
  return (int)cudaGetLastError();
}
int launch_unit_env_f64(double* const* env, int n, void* stream) {
  if (n <= 0) return 0;
  unit_env_f64_kernel<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(env, n);
  return (int)cudaGetLastError();
}
int launch_unit_env_f32(float* const* env, int n, void* stream) {
  if (n <= 0) return 0;
  unit_env_f32_kernel<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(env, n);
  return (int)cudaGetLastError();
}
int launch_extract_df(const float2* const* fin, int npairs, double* H, double* S, void* stream) {
  if (npairs <= 0) return 0;
  extract_df_kernel<<<(npairs + 127) / 128, 128, 0, (cudaStream_t)stream>>>(fin, npairs, H, S);
  return (int)cudaGetLastError();
}
namespace {
int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        n <= 0)
      n = 148;
  }
  return n;
}
template <int BN, int S>
int launch_bf16s(const OzGemmDesc* d, const long long* tile_prefix, int nprob, long long total_tiles,
                 long long max_spin, int* err, cudaStream_t st) {
  const cudaError_t e =
      cudaFuncSetAttribute(gemm_bf16s_kernel<BN, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM_BYTES);
  if (e != cudaSuccess) return (int)e;
  const long long grid = total_tiles < sm_count() ? total_tiles : sm_count();   // persistent: one CTA per SM
  gemm_bf16s_kernel<BN, S><<<(unsigned)grid, OZ_THREADS, OZ_SMEM_BYTES, st>>>(d, tile_prefix, nprob, total_tiles,
                                                                               max_spin, err);
  return (int)cudaGetLastError();
}
template <int S>
int launch_bf16s_ws(const OzGemmDesc* d, const long long* tile_prefix, int nprob, long long total_tiles,
                    long long max_spin, int* err, cudaStream_t st) {
  const cudaError_t e =
      cudaFuncSetAttribute(gemm_bf16s_ws_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM_BYTES);
  if (e != cudaSuccess) return (int)e;
  const long long grid = total_tiles < sm_count() ? total_tiles : sm_count();
  gemm_bf16s_ws_kernel<S><<<(unsigned)grid, OZW_THREADS, OZ_SMEM_BYTES, st>>>(d, tile_prefix, nprob, total_tiles,
                                                                               max_spin, err);
  return (int)cudaGetLastError();
}
template <int BN>
int launch_bf16s_s(const OzGemmDesc* d, const long long* tile_prefix, int nprob, long long total_tiles,
                   long long max_spin, int* err, int ns, cudaStream_t st) {
  switch (ns) {
    case 2: return launch_bf16s<BN, 2>(d, tile_prefix, nprob, total_tiles, max_spin, err, st);
    case 3: return launch_bf16s<BN, 3>(d, tile_prefix, nprob, total_tiles, max_spin, err, st);
    case 4: return launch_bf16s<BN, 4>(d, tile_prefix, nprob, total_tiles, max_spin, err, st);
    case 5: return launch_bf16s<BN, 5>(d, tile_prefix, nprob, total_tiles, max_spin, err, st);
    default: return (int)cudaErrorInvalidValue;
  }
}
}  // namespace

int launch_gemm_bf16s(const OzGemmDesc* d, const long long* tile_prefix, int nprob, long long total_tiles,
                      long long max_spin, int* err, int bn, int ns, void* stream) {
  if (total_tiles <= 0) return 0;
  cudaStream_t st = (cudaStream_t)stream;
  if (bn == 128) return launch_bf16s_s<128>(d, tile_prefix, nprob, total_tiles, max_spin, err, ns, st);
  if (bn == 64) {                                   // warp-specialised, double-buffered accumulators
    switch (ns) {
      case 2: return launch_bf16s_ws<2>(d, tile_prefix, nprob, total_tiles, max_spin, err, st);
      case 3: return launch_bf16s_ws<3>(d, tile_prefix, nprob, total_tiles, max_spin, err, st);
      case 4: return launch_bf16s_ws<4>(d, tile_prefix, nprob, total_tiles, max_spin, err, st);
      case 5: return launch_bf16s_ws<5>(d, tile_prefix, nprob, total_tiles, max_spin, err, st);
      default: return (int)cudaErrorInvalidValue;
    }
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace tnqe
