// Block-sparse FP64 transfer-matrix contraction <MPS_i| W |MPS_j'> (Fig. 5b).
//
// The paper's numerics enforce particle number and S_z through block-sparse
// tensors (Sec. II C cost remark, Sec. IV A).  Every bond index carries a
// charge q = (n_alpha, n_beta) counted from the left, and every MPO channel w
// the charge change d(w) of the operator string it carries, so
//   L[a][w][b]        != 0 only if q(a) = q(b) + d(w)
//   X[a][w][k'][b']   != 0 only if q(b') = q(a) - d(w) + q(k')
//   Y[a][k][w'][b']   != 0 only if q(b') = q(a) + q(k) - d(w')
// (a nonzero W[(k, w'), (w, k')] has d(w') = d(w) + q(k) - q(k')).  The three
// stages below compute and read exactly those blocks:
//   stage 1  X = L B   one CTA per (pair, bra sector alpha of bond t, channel class c)
//   stage 2  Y = W X   one CTA per (pair, bra index a); MPO rows grouped by d(w') - q(k)
//   stage 3  L' = A^T Y one CTA per (pair, bra sector alpha' of bond t+1, channel class c')
// The arrays keep the dense capacity layout, so nothing here depends on the
// ket's sector dimensions except the sector tables the kernels read on the
// device (for a rotated ket, the ones the rotation kernel wrote).  The small
// blocks (sector dimensions of ten to a few tens) make these FP64 SIMT
// kernels: GB300 issues two FP64 FMAs per clock per SM, so one FMA per two
// operand loads (shared memory, L1) keeps the FP64 pipe the bound.
#include <cuda_runtime.h>

#include "internal.h"

namespace tnqe {
namespace {

constexpr int BS_SMEM = 6144;                 // doubles of staged operand per CTA (48 KiB)

__device__ __forceinline__ int bs_problem(const long long* prefix, int n, long long x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Sector of charge (na, nb) in a bond's table (ascending codes), -1 if absent.
__device__ __forceinline__ int bs_find(const SectorTable* T, int na, int nb) {
  if (na < 0 || nb < 0 || na >= QSTRIDE - 1 || nb >= QSTRIDE - 1) return -1;
  const int q = na * QSTRIDE + nb;
  int lo = 0, hi = T->nsec - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int v = T->q[mid];
    if (v == q) return mid;
    if (v < q) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

// ----------------------------------------------------------------------------- stage 1
// X[a][w][k'][g] = sum_{b in beta} L[a][w][b] B[b][k'][g] for a in alpha, w in class c,
// beta = q(alpha) - d(c), g in gamma_k' = beta + q(k').  Where beta is absent from the
// ket's bond t the block is zero and is written as such (stage 2 reads it).
template <int BS_THREADS>
__global__ void __launch_bounds__(BS_THREADS) bs_stage1_kernel(const BsSiteDesc* __restrict__ descs,
                                                              const long long* __restrict__ prefix, int n,
                                                              double* flops) {
  __shared__ double Bs[BS_SMEM];
  __shared__ int s_goff[4], s_gcol[5];
  __shared__ int s_info[5];
  const long long item = blockIdx.x;
  const int p = bs_problem(prefix, n, item);
  const BsSiteDesc& D = descs[p];
  const long long local = item - prefix[p];
  const int ncls = D.chL.ncls;
  const int alpha = (int)(local / ncls), c = (int)(local % ncls);
  const int tid = threadIdx.x;
  if (tid == 0) {
    const int q = D.braL->q[alpha];
    const int bna = q / QSTRIDE - D.chL.d[2 * c], bnb = q % QSTRIDE - D.chL.d[2 * c + 1];
    const int ib = bs_find(D.ketL, bna, bnb);
    s_info[0] = D.braL->off[alpha];
    s_info[1] = D.braL->dim[alpha];
    s_info[2] = ib >= 0 ? D.ketL->off[ib] : 0;
    s_info[3] = ib >= 0 ? D.ketL->dim[ib] : 0;
    int col = 0;
    for (int k = 0; k < 4; ++k) {
      const int ig = bs_find(D.ketR, bna + (k & 1), bnb + (k >> 1));
      s_gcol[k] = col;
      s_goff[k] = ig >= 0 ? D.ketR->off[ig] : 0;
      col += ig >= 0 ? D.ketR->dim[ig] : 0;
    }
    s_gcol[4] = col;
  }
  __syncthreads();
  const int offA = s_info[0], dimA = s_info[1], offB = s_info[2], dimB = s_info[3];
  const int ncol = s_gcol[4];
  const int cw0 = D.chL.off[c], Dc = D.chL.off[c + 1] - cw0;
  const int* wl = D.chL.w + cw0;
  const int nrows = dimA * Dc;
  if (ncol == 0 || nrows == 0) return;
  const int Din = D.Din, capb = D.capb, capb2 = D.capb2;
  double* __restrict__ Xo = D.X;
  const double* __restrict__ Lin = D.Lin;
  const double* __restrict__ Bt = D.B;
  auto xaddr = [&](int r, int j) -> size_t {
    const int a = offA + r / Dc, w = wl[r % Dc];
    const int k = (j >= s_gcol[1]) + (j >= s_gcol[2]) + (j >= s_gcol[3]);
    return (((size_t)a * Din + w) * 4 + k) * capb2 + s_goff[k] + (j - s_gcol[k]);
  };
  if (dimB == 0) {
    for (int o = tid; o < nrows * ncol; o += BS_THREADS) Xo[xaddr(o / ncol, o % ncol)] = 0.0;
    return;
  }
  if (tid == 0) atomicAdd(flops, 2.0 * nrows * dimB * ncol);
  const int JC = min(ncol, BS_SMEM / dimB);
  for (int j0 = 0; j0 < ncol; j0 += JC) {
    const int jn = min(JC, ncol - j0);
    for (int x = tid; x < dimB * jn; x += BS_THREADS) {
      const int b = x / jn, j = j0 + x % jn;
      const int k = (j >= s_gcol[1]) + (j >= s_gcol[2]) + (j >= s_gcol[3]);
      Bs[x] = Bt[((size_t)(offB + b) * 4 + k) * capb2 + s_goff[k] + (j - s_gcol[k])];
    }
    __syncthreads();
    for (int o = tid; o < nrows * jn; o += BS_THREADS) {
      const int r = o / jn, jj = o % jn;
      const int a = offA + r / Dc, w = wl[r % Dc];
      const double* Lr = Lin + ((size_t)a * Din + w) * capb + offB;
      double acc = 0.0;
      for (int b = 0; b < dimB; ++b) acc = fma(Lr[b], Bs[b * jn + jj], acc);
      Xo[xaddr(r, j0 + jj)] = acc;
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------- stage 2
// Y[a][row][g] = sum_e W_e X[a][col_e][g] for every MPO row (k, w'), g in the ket
// sector gamma = q(a) - (d(w') - q(k)) of bond t + 1.
template <int BS_THREADS>
__global__ void __launch_bounds__(BS_THREADS) bs_stage2_kernel(const BsSiteDesc* __restrict__ descs,
                                                              const long long* __restrict__ prefix, int n,
                                                              double* flops) {
  __shared__ int s_goff[BS_MAXRC], s_gdim[BS_MAXRC];
  __shared__ double s_fl;
  const long long item = blockIdx.x;
  const int p = bs_problem(prefix, n, item);
  const BsSiteDesc& D = descs[p];
  const int a = (int)(item - prefix[p]);
  const int tid = threadIdx.x;
  // charge of bra index a (sectors cover [0, ca) in ascending offsets)
  const SectorTable* bl = D.braL;
  int lo = 0, hi = bl->nsec - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (bl->off[mid] <= a) lo = mid; else hi = mid - 1;
  }
  const int q = bl->q[lo], na = q / QSTRIDE, nb = q % QSTRIDE;
  const int nrc = D.rows.ncls;
  if (tid == 0) s_fl = 0.0;
  __syncthreads();
  for (int r = tid; r < nrc; r += BS_THREADS) {
    const int ig = bs_find(D.ketR, na - D.rows.d[2 * r], nb - D.rows.d[2 * r + 1]);
    s_goff[r] = ig >= 0 ? D.ketR->off[ig] : 0;
    s_gdim[r] = ig >= 0 ? D.ketR->dim[ig] : 0;
    if (ig >= 0) atomicAdd(&s_fl, 2.0 * D.rows.nnz[r] * s_gdim[r]);
  }
  __syncthreads();
  if (tid == 0 && s_fl > 0.0) atomicAdd(flops + 1, s_fl);
  const int capb2 = D.capb2;
  const double* __restrict__ Xa = D.X + (size_t)a * 4 * D.Din * capb2;
  double* __restrict__ Ya = D.Y + (size_t)a * 4 * D.Dout * capb2;
  const int* __restrict__ rowptr = D.rowptr;
  const int* __restrict__ col = D.col;
  const double* __restrict__ val = D.val;
  const int* __restrict__ roff = D.rows.off;
  const int* __restrict__ rrows = D.rows.rows;
  for (int r = 0; r < nrc; ++r) {
    const int dg = s_gdim[r];
    if (dg == 0) continue;
    const int go = s_goff[r];
    const int r0 = roff[r], nr = roff[r + 1] - r0;
    for (int o = tid; o < nr * dg; o += BS_THREADS) {
      const int row = rrows[r0 + o / dg], g = go + o % dg;
      double acc = 0.0;
      const int e1 = rowptr[row + 1];
      for (int e = rowptr[row]; e < e1; ++e) acc = fma(val[e], Xa[(size_t)col[e] * capb2 + g], acc);
      Ya[(size_t)row * capb2 + g] = acc;
    }
  }
}

// ----------------------------------------------------------------------------- stage 3
// L'[a'][w'][g] = sum_k sum_{a in alpha' - q(k)} A[a][k][a'] Y[a][k][w'][g] for a' in
// alpha', w' in class c', g in beta' = q(alpha') - d(c').  Nothing is written where
// beta' is absent from the ket's bond t + 1 (no later stage reads it).
template <int BS_THREADS>
__global__ void __launch_bounds__(BS_THREADS) bs_stage3_kernel(const BsSiteDesc* __restrict__ descs,
                                                              const long long* __restrict__ prefix, int n,
                                                              double* flops) {
  __shared__ double As[BS_SMEM];
  __shared__ int s_koff[4], s_kcol[5], s_info[4];
  const long long item = blockIdx.x;
  const int p = bs_problem(prefix, n, item);
  const BsSiteDesc& D = descs[p];
  const long long local = item - prefix[p];
  const int ncls = D.chR.ncls;
  const int alpha = (int)(local / ncls), c = (int)(local % ncls);
  const int tid = threadIdx.x;
  if (tid == 0) {
    const int q = D.braR->q[alpha];
    const int na = q / QSTRIDE, nb = q % QSTRIDE;
    const int ib = bs_find(D.ketR, na - D.chR.d[2 * c], nb - D.chR.d[2 * c + 1]);
    s_info[0] = D.braR->off[alpha];
    s_info[1] = D.braR->dim[alpha];
    s_info[2] = ib >= 0 ? D.ketR->off[ib] : 0;
    s_info[3] = ib >= 0 ? D.ketR->dim[ib] : 0;
    int kc = 0;
    for (int k = 0; k < 4; ++k) {
      const int ia = bs_find(D.braL, na - (k & 1), nb - (k >> 1));
      s_kcol[k] = kc;
      s_koff[k] = ia >= 0 ? D.braL->off[ia] : 0;
      kc += ia >= 0 ? D.braL->dim[ia] : 0;
    }
    s_kcol[4] = kc;
  }
  __syncthreads();
  const int offA2 = s_info[0], dimA2 = s_info[1], offB2 = s_info[2], dimB2 = s_info[3];
  if (dimB2 == 0 || dimA2 == 0) return;
  const int cw0 = D.chR.off[c], Dc = D.chR.off[c + 1] - cw0;
  const int* wl = D.chR.w + cw0;
  const int ncol = Dc * dimB2;
  const int Kdim = s_kcol[4];
  const int Dout = D.Dout, capb2 = D.capb2, ca2 = D.ca2;
  const double* __restrict__ Yg = D.Y;
  const double* __restrict__ At = D.A;
  double* __restrict__ Lo = D.Lout;
  if (Kdim == 0) {
    for (int o = tid; o < dimA2 * ncol; o += BS_THREADS) {
      const int ap = o / ncol, j = o % ncol;
      Lo[((size_t)(offA2 + ap) * Dout + wl[j / dimB2]) * capb2 + offB2 + j % dimB2] = 0.0;
    }
    return;
  }
  if (tid == 0) atomicAdd(flops + 2, 2.0 * dimA2 * ncol * Kdim);
  const int AC = min(dimA2, BS_SMEM / Kdim);
  for (int a0 = 0; a0 < dimA2; a0 += AC) {
    const int an = min(AC, dimA2 - a0);
    for (int x = tid; x < Kdim * an; x += BS_THREADS) {
      const int kk = x / an, ap = x % an;
      const int k = (kk >= s_kcol[1]) + (kk >= s_kcol[2]) + (kk >= s_kcol[3]);
      const int a = s_koff[k] + (kk - s_kcol[k]);
      As[x] = At[((size_t)a * 4 + k) * ca2 + offA2 + a0 + ap];
    }
    __syncthreads();
    const int ngrp = (an + 3) >> 2;
    for (int o = tid; o < ngrp * ncol; o += BS_THREADS) {
      const int j = o % ncol, grp = o / ncol;
      const int wp = wl[j / dimB2], g = offB2 + j % dimB2;
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      for (int k = 0; k < 4; ++k) {
        const int kn = s_kcol[k + 1] - s_kcol[k];
        const double* yk = Yg + ((size_t)s_koff[k] * 4 + k) * Dout * capb2 + (size_t)wp * capb2 + g;
        const double* ak = As + s_kcol[k] * an + grp * 4;
        for (int x = 0; x < kn; ++x) {
          const double y = yk[(size_t)x * 4 * Dout * capb2];
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (grp * 4 + u < an) acc[u] = fma(ak[x * an + u], y, acc[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (grp * 4 + u < an) Lo[((size_t)(offA2 + a0 + grp * 4 + u) * Dout + wp) * capb2 + g] = acc[u];
    }
    __syncthreads();
  }
}

}  // namespace

// CTA sizes of the stages (launch shapes the autotuner chooses from)
#define BS_LAUNCH(kernel)                                                                                   \
  do {                                                                                                      \
    if (total <= 0) return 0;                                                                               \
    cudaStream_t st = (cudaStream_t)stream;                                                                 \
    if (threads == 64) kernel<64><<<(unsigned)total, 64, 0, st>>>(d, prefix, n, flops);                     \
    else if (threads == 256) kernel<256><<<(unsigned)total, 256, 0, st>>>(d, prefix, n, flops);             \
    else kernel<128><<<(unsigned)total, 128, 0, st>>>(d, prefix, n, flops);                                 \
    return (int)cudaGetLastError();                                                                         \
  } while (0)

int launch_bs_stage1(const BsSiteDesc* d, const long long* prefix, int n, long long total, double* flops,
                     int threads, void* stream) {
  BS_LAUNCH(bs_stage1_kernel);
}

int launch_bs_stage2(const BsSiteDesc* d, const long long* prefix, int n, long long total, double* flops,
                     int threads, void* stream) {
  BS_LAUNCH(bs_stage2_kernel);
}

int launch_bs_stage3(const BsSiteDesc* d, const long long* prefix, int n, long long total, double* flops,
                     int threads, void* stream) {
  BS_LAUNCH(bs_stage3_kernel);
}

}  // namespace tnqe
