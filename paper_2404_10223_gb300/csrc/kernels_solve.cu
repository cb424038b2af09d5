// Generalized eigenproblem H c = E S c (Eq. 9) by canonical orthogonalisation,
// the projection method of Sec. IV C / App. A2, in one warp in FP64:
// S = W L W^T (cyclic Jacobi), keep L > eps * L_max, X = W_keep L_keep^(-1/2),
// eig(X^T H X) = Y E Y^T (cyclic Jacobi), C = X Y, kappa_1 = |c_1|^2 / sqrt(E_1^2+1).
#include <cuda_runtime.h>

#include "internal.h"

namespace tnqe {
namespace {

constexpr int MS = 32;

// cyclic two-sided Jacobi on the symmetric n x n matrix A (shared), eigenvectors in V
__device__ int warp_jacobi_eig(double (*A)[MS + 1], double (*V)[MS + 1], int n, int max_sweeps) {
  const int lane = threadIdx.x;
  if (lane < n)
    for (int r = 0; r < n; ++r) V[r][lane] = (r == lane) ? 1.0 : 0.0;
  __syncwarp();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    int rotated = 0;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p][q], app = A[p][p], aqq = A[q][q];
        __syncwarp();
        if (apq == 0.0 || fabs(apq) <= 1e-17 * sqrt(fabs(app)) * sqrt(fabs(aqq))) continue;
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + hypot(theta, 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        if (s == 0.0) continue;                      // below resolution: nothing changes
        rotated = 1;
        double arp = 0.0, arq = 0.0, vrp = 0.0, vrq = 0.0;
        if (lane < n) {
          arp = A[lane][p];
          arq = A[lane][q];
          vrp = V[lane][p];
          vrq = V[lane][q];
        }
        __syncwarp();
        if (lane < n) {
          if (lane != p && lane != q) {
            const double np_ = c * arp - s * arq, nq_ = s * arp + c * arq;
            A[lane][p] = np_;
            A[p][lane] = np_;
            A[lane][q] = nq_;
            A[q][lane] = nq_;
          }
          V[lane][p] = c * vrp - s * vrq;
          V[lane][q] = s * vrp + c * vrq;
        }
        __syncwarp();
        if (lane == 0) {
          A[p][p] = app - t * apq;
          A[q][q] = aqq + t * apq;
          A[p][q] = 0.0;
          A[q][p] = 0.0;
        }
        __syncwarp();
      }
    if (!rotated) return 0;
  }
  return 1;
}

__global__ void solve_kernel(const double* __restrict__ Hin, const double* __restrict__ Sin, int M, double eps,
                             int max_sweeps, double* E, double* C, int* rank_out, double* kappa, int* status) {
  __shared__ double S[MS][MS + 1], H[MS][MS + 1], W[MS][MS + 1], X[MS][MS + 1], T[MS][MS + 1];
  double (*Y)[MS + 1] = H;                         // H is dead once T = H X is formed
  __shared__ double lam[MS], ev[MS];
  __shared__ int keep_idx[MS], order[MS];
  __shared__ int s_rank;
  const int lane = threadIdx.x;
  for (int r = 0; r < M; ++r)
    if (lane < M) {
      const int i = r < lane ? r : lane, j = r < lane ? lane : r;   // upper triangle is authoritative
      S[r][lane] = Sin[i * M + j];
      H[r][lane] = Hin[i * M + j];
    }
  __syncwarp();
  int st = warp_jacobi_eig(S, W, M, max_sweeps);
  __syncwarp();
  if (lane == 0) {
    double lmax = -1e300;
    for (int i = 0; i < M; ++i) lmax = fmax(lmax, S[i][i]);
    int r = 0;
    for (int i = 0; i < M; ++i)
      if (S[i][i] > eps * lmax) {
        keep_idx[r] = i;
        lam[r] = S[i][i];
        ++r;
      }
    s_rank = r;
  }
  __syncwarp();
  const int rk = s_rank;
  // X = W_keep diag(lam^-1/2): M x rk
  for (int c = 0; c < rk; ++c)
    if (lane < M) X[lane][c] = W[lane][keep_idx[c]] / sqrt(lam[c]);
  __syncwarp();
  // T = H X (M x rk), then Ht = X^T T (rk x rk) into H's storage
  for (int c = 0; c < rk; ++c)
    if (lane < M) {
      double acc = 0.0;
      for (int k = 0; k < M; ++k) acc = fma(H[lane][k], X[k][c], acc);
      T[lane][c] = acc;
    }
  __syncwarp();
  for (int c = 0; c < rk; ++c)
    if (lane < rk) {
      double acc = 0.0;
      for (int k = 0; k < M; ++k) acc = fma(X[k][lane], T[k][c], acc);
      S[lane][c] = acc;                            // S storage reused for X^T H X
    }
  __syncwarp();
  for (int c = 0; c < rk; ++c)
    if (lane < rk && lane < c) {
      const double m = 0.5 * (S[lane][c] + S[c][lane]);
      S[lane][c] = m;
      S[c][lane] = m;
    }
  __syncwarp();
  st |= warp_jacobi_eig(S, Y, rk, max_sweeps);
  __syncwarp();
  if (lane == 0) {
    for (int i = 0; i < rk; ++i) {
      order[i] = i;
      ev[i] = S[i][i];
    }
    for (int i = 1; i < rk; ++i) {              // insertion sort, ascending
      const int o = order[i];
      int j = i - 1;
      while (j >= 0 && ev[order[j]] > ev[o]) {
        order[j + 1] = order[j];
        --j;
      }
      order[j + 1] = o;
    }
  }
  __syncwarp();
  // C = X Y (M x rk), largest |entry| of each column positive
  for (int c = 0; c < rk; ++c)
    if (lane < M) {
      double acc = 0.0;
      for (int k = 0; k < rk; ++k) acc = fma(X[lane][k], Y[k][order[c]], acc);
      T[lane][c] = acc;
    }
  __syncwarp();
  if (lane < rk) {
    const int c = lane;
    int best = 0;
    double bv = -1.0;
    for (int r = 0; r < M; ++r)
      if (fabs(T[r][c]) > bv) {
        bv = fabs(T[r][c]);
        best = r;
      }
    const double sgn = T[best][c] < 0.0 ? -1.0 : 1.0;
    for (int r = 0; r < M; ++r) T[r][c] *= sgn;
  }
  __syncwarp();
  for (int r = 0; r < M; ++r)
    if (lane < M) C[r * M + lane] = lane < rk ? T[r][lane] : 0.0;
  if (lane < M) E[lane] = lane < rk ? ev[order[lane]] : __longlong_as_double(0x7ff8000000000000ll);
  if (lane == 0) {
    *rank_out = rk;
    double n2 = 0.0;
    for (int r = 0; r < M; ++r) n2 = fma(T[r][0], T[r][0], n2);
    const double e1 = rk > 0 ? ev[order[0]] : 0.0;
    *kappa = rk > 0 ? n2 / sqrt(e1 * e1 + 1.0) : 0.0;
    *status = st ? STATUS_NOCONV : 0;
  }
}

// Linear-dependence residuals (Sec. IV C's discard test): warp j computes
// r_j = S_jj - s^T S_<j^+ s with s = S[0:j, j] and S_<j = S[0:j, 0:j], the
// pseudo-inverse keeping eigenvalues above eps * lambda_max.  r_j is the
// squared norm of state j's component outside the span of states 0..j-1.
__global__ void dependence_kernel(const double* __restrict__ Sin, int M, double eps, int max_sweeps,
                                  double* __restrict__ resid, int* __restrict__ status) {
  __shared__ double A[MS][MS + 1], V[MS][MS + 1];
  __shared__ double sv[MS];
  const int j = blockIdx.x, lane = threadIdx.x;
  if (j >= M) return;
  for (int r = 0; r < j; ++r)
    if (lane < j) {
      const int a = r < lane ? r : lane, b = r < lane ? lane : r;   // upper triangle is authoritative
      A[r][lane] = Sin[a * M + b];
    }
  if (lane < j) sv[lane] = Sin[lane * M + j];
  __syncwarp();
  int st = 0;
  if (j > 0) st = warp_jacobi_eig(A, V, j, max_sweeps);
  __syncwarp();
  if (lane == 0) {
    double lmax = 0.0;
    for (int k = 0; k < j; ++k) lmax = fmax(lmax, A[k][k]);
    double proj = 0.0;
    for (int k = 0; k < j; ++k) {
      if (!(A[k][k] > eps * lmax)) continue;
      double wk = 0.0;
      for (int r = 0; r < j; ++r) wk = fma(V[r][k], sv[r], wk);
      proj += wk * wk / A[k][k];
    }
    resid[j] = Sin[j * M + j] - proj;
    if (st) atomicOr(status, STATUS_NOCONV);
  }
}

}  // namespace

int launch_dependence(const double* d_S, int M, double eps, int max_sweeps, double* d_resid, int* d_status,
                      void* stream) {
  dependence_kernel<<<M, 32, 0, (cudaStream_t)stream>>>(d_S, M, eps, max_sweeps, d_resid, d_status);
  return (int)cudaGetLastError();
}

int launch_solve(const double* d_H, const double* d_S, int M, double eps, int max_sweeps, double* d_E, double* d_C,
                 int* d_rank, double* d_kappa, int* d_status, void* stream) {
  solve_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(d_H, d_S, M, eps, max_sweeps, d_E, d_C, d_rank, d_kappa, d_status);
  return (int)cudaGetLastError();
}

}  // namespace tnqe
