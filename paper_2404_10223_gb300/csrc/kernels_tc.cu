// Split-precision (TF32x3) transfer contraction on tcgen05 tensor cores.
//
// Per site and pair, with FP32 environments L[a][w][b] (row stride ld_b, a
// multiple of 4 floats so every row starts on a 16-byte boundary for TMA):
//   stage 1  X[(a,w)][(k',b')] = L[(a,w)][b] . ketT[(k',b')][b]       tcgen05 GEMM
//   stage 2  Yt[(w',b')][(a,k)] = sum W[(w',k),(w,k')] X[(a,w)][(k',b')] sparse MPO, K-major output
//   stage 3  L'[a'][(w',b')]   = braT[a'][(a,k)] . Yt[(w',b')][(a,k)]  tcgen05 GEMM
// ketT / braT are the MPS site tensors transposed to K-major FP32.
#include <cuda_runtime.h>

#include "internal.h"
#define TNQE_DEFINE_TC_KERNEL
#include "tc_gemm.cuh"

namespace tnqe {
namespace {

// ketT[(k',b')][b] = B[b][k'][b']  (mode 0)   braT[a'][(a,k)] = A[a][k][a']  (mode 1)
__global__ void pack_sites_kernel(const PackDesc* __restrict__ descs, const long long* __restrict__ prefix, int n,
                                  long long total) {
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= total) return;
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= x) lo = mid; else hi = mid - 1;
  }
  const PackDesc& d = descs[lo];
  const long long e = x - prefix[lo];           // over the source tensor [l][k][r]
  const int r = (int)(e % d.cr);
  const int k = (int)((e / d.cr) % 4);
  const int l = (int)(e / ((long long)d.cr * 4));
  const float v = (float)d.src[e];
  if (d.mode == 0) d.dst[((long long)k * d.cr + r) * d.ld + l] = v;
  else d.dst[(long long)r * d.ld + (long long)l * 4 + k] = v;
}

// One CTA: MPO output channel w', 32 ket columns b', 32 bra rows a; all four k.
__global__ void __launch_bounds__(256) spmm_t_f32_kernel(const SpmmTDesc* __restrict__ descs,
                                                         const long long* __restrict__ prefix, int nprob) {
  __shared__ float tile[32][32 * 4 + 1];       // [b'][a * 4 + k]
  const long long task = blockIdx.x;
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= task) lo = mid; else hi = mid - 1;
  }
  const SpmmTDesc& d = descs[lo];
  long long local = task - prefix[lo];
  const int nbt = (d.width + 31) / 32, nat = (d.chi_a + 31) / 32;
  const int at = (int)(local % nat);
  local /= nat;
  const int bt = (int)(local % nbt);
  const int wp = (int)(local / nbt);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int b = bt * 32 + lane;
  const long long xrow = (long long)4 * d.width;                 // X row length (k', b')
  float acc[4][4];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[k][i] = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int row = k * d.Dout + wp;
    const int e0 = d.rowptr[row], e1 = d.rowptr[row + 1];
    for (int e = e0; e < e1; ++e) {
      const int c = d.col[e];
      const int w = c >> 2, kp = c & 3;
      const float v = d.val[e];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int a = at * 32 + warp + 8 * i;
        if (a < d.chi_a && b < d.width)
          acc[k][i] = fmaf(v, d.X[((long long)a * d.Din + w) * xrow + (long long)kp * d.width + b], acc[k][i]);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int i = 0; i < 4; ++i) tile[lane][(warp + 8 * i) * 4 + k] = acc[k][i];
  __syncthreads();
  // rows (w', b') of Yt, columns (a, k) contiguous
  const int ncol = min(32, d.chi_a - at * 32) * 4;
  for (int r = warp; r < 32; r += 8) {
    const int bb = bt * 32 + r;
    if (bb >= d.width) break;
    float* dst = d.Yt + ((long long)wp * d.width + bb) * d.ldy + (long long)at * 128;
    for (int c = lane; c < ncol; c += 32) dst[c] = tile[r][c];
  }
}

__global__ void extract_f32_kernel(const float* const* __restrict__ fin, int npairs, int ld, double* H, double* S) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npairs) return;
  S[p] = (double)fin[p][0];        // identity-string channel
  H[p] = (double)fin[p][ld];       // completed-Hamiltonian channel
}

}  // namespace

int launch_pack_sites(const PackDesc* d, const long long* prefix, int n, long long total, void* stream) {
  if (total <= 0) return 0;
  pack_sites_kernel<<<(unsigned)((total + 255) / 256), 256, 0, (cudaStream_t)stream>>>(d, prefix, n, total);
  return (int)cudaGetLastError();
}

int launch_gemm_tf32x3(const TcGemmDesc* d, const long long* tile_prefix, int nprob, long long total_tiles,
                       long long max_spin, int* err, void* stream) {
  if (total_tiles <= 0) return 0;
  const cudaError_t e = cudaFuncSetAttribute(gemm_tf32x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             TC_SMEM_BYTES);
  if (e != cudaSuccess) return (int)e;
  gemm_tf32x3_kernel<<<(unsigned)total_tiles, TC_THREADS, TC_SMEM_BYTES, (cudaStream_t)stream>>>(d, tile_prefix, nprob,
                                                                                               max_spin, err);
  return (int)cudaGetLastError();
}

int launch_spmm_t_f32(const SpmmTDesc* d, const long long* prefix, int nprob, long long total, void* stream) {
  if (total <= 0) return 0;
  spmm_t_f32_kernel<<<(unsigned)total, 256, 0, (cudaStream_t)stream>>>(d, prefix, nprob);
  return (int)cudaGetLastError();
}

int launch_extract_f32(const float* const* fin, int npairs, int ld, double* H, double* S, void* stream) {
  if (npairs <= 0) return 0;
  extract_f32_kernel<<<(npairs + 127) / 128, 128, 0, (cudaStream_t)stream>>>(fin, npairs, ld, H, S);
  return (int)cudaGetLastError();
}

}  // namespace tnqe
