// FP64 transfer-matrix contraction <MPS_i| W |MPS_j'> (Fig. 5b), one site at a
// time for every pair of a batch:
//   stage 1  X[a][w][k'][b'] = sum_b L[a][w][b] B[b][k'][b']        (grouped GEMM)
//   stage 2  Y[a][k][w'][b'] = sum W[(w',k),(w,k')] X[a][w][k'][b'] (sparse MPO)
//   stage 3  L'[a'][w'][b']  = sum_{a,k} A[a][k][a'] Y[a][k][w'][b'] (grouped GEMM, A^T)
#include <cuda_runtime.h>

#include "internal.h"

namespace tnqe {
namespace {

constexpr int TM = 64, TN = 64, TK = 16;

__device__ __forceinline__ int find_problem(const long long* prefix, int nprob, long long x) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(256) gemm_f64_grouped(const GemmDesc* __restrict__ descs,
                                                        const long long* __restrict__ prefix, int nprob) {
  __shared__ double As[TK][TM + 1];
  __shared__ double Bs[TK][TN + 1];
  const long long tile = blockIdx.x;
  const int p = find_problem(prefix, nprob, tile);
  const GemmDesc d = descs[p];
  const int tiles_n = (d.N + TN - 1) / TN;
  const long long local = tile - prefix[p];
  const int m0 = (int)(local / tiles_n) * TM, n0 = (int)(local % tiles_n) * TN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int k0 = 0; k0 < d.K; k0 += TK) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = tid + 256 * e;            // 1024 elements of each tile
      if (d.transA) {
        const int r = idx & 63, c = idx >> 6;   // A stored K x M: coalesced along m
        const int gm = m0 + r, gk = k0 + c;
        As[c][r] = (gm < d.M && gk < d.K) ? d.A[(size_t)gk * d.lda + gm] : 0.0;
      } else {
        const int c = idx & 15, r = idx >> 4;
        const int gm = m0 + r, gk = k0 + c;
        As[c][r] = (gm < d.M && gk < d.K) ? d.A[(size_t)gm * d.lda + gk] : 0.0;
      }
      const int bc = idx & 63, br = idx >> 6;
      const int gk = k0 + br, gn = n0 + bc;
      Bs[br][bc] = (gk < d.K && gn < d.N) ? d.B[(size_t)gk * d.ldb + gn] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= d.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn < d.N) d.C[(size_t)gm * d.ldc + gn] = acc[i][j];
    }
  }
}

// one warp per output row vector Y[a][row][0:width]
__global__ void __launch_bounds__(256) spmm_f64_grouped(const SpmmDesc* __restrict__ descs,
                                                        const long long* __restrict__ prefix, int nprob,
                                                        long long total) {
  const long long task = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (task >= total) return;
  const int lane = threadIdx.x & 31;
  const int p = find_problem(prefix, nprob, task);
  const SpmmDesc d = descs[p];
  const long long local = task - prefix[p];
  const int a = (int)(local / d.nrows), row = (int)(local % d.nrows);
  const int e0 = d.rowptr[row], e1 = d.rowptr[row + 1];
  const double* Xa = d.X + (size_t)a * d.ncols_x * d.width;
  double* y = d.Y + ((size_t)a * d.nrows + row) * d.width;
  for (int c0 = 0; c0 < d.width; c0 += 128) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int e = e0; e < e1; ++e) {
      const double v = d.val[e];
      const double* x = Xa + (size_t)d.col[e] * d.width;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = c0 + lane + 32 * u;
        if (c < d.width) acc[u] = fma(v, x[c], acc[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = c0 + lane + 32 * u;
      if (c < d.width) y[c] = acc[u];
    }
  }
}

__global__ void extract_kernel(const double* const* __restrict__ fin, int npairs, double* H, double* S) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npairs) return;
  S[p] = fin[p][0];   // identity-string channel
  H[p] = fin[p][1];   // completed-Hamiltonian channel
}

}  // namespace

int launch_gemm_f64(const GemmDesc* d_descs, const long long* d_tile_prefix, int nprob, long long total_tiles,
                    void* stream) {
  if (total_tiles <= 0) return 0;
  gemm_f64_grouped<<<(unsigned)total_tiles, 256, 0, (cudaStream_t)stream>>>(d_descs, d_tile_prefix, nprob);
  return (int)cudaGetLastError();
}

int launch_spmm_f64(const SpmmDesc* d_descs, const long long* d_row_prefix, int nprob, long long total_rows,
                    void* stream) {
  if (total_rows <= 0) return 0;
  const long long blocks = (total_rows + 7) / 8;
  spmm_f64_grouped<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(d_descs, d_row_prefix, nprob, total_rows);
  return (int)cudaGetLastError();
}

int launch_extract(const double* const* d_final, int npairs, double* H, double* S, void* stream) {
  if (npairs <= 0) return 0;
  extract_kernel<<<(npairs + 127) / 128, 128, 0, (cudaStream_t)stream>>>(d_final, npairs, H, S);
  return (int)cudaGetLastError();
}

}  // namespace tnqe
