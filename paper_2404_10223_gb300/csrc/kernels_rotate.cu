// Rotation of MPS j into the orbital basis of MPS i (Eq. 11, Sec. II D, App. A3):
// one CTA per pair walks that pair's Givens gates in order.  Per gate on sites
// (a, a+1): contract the two-site tensor, apply the 16 x 16 gate, split the
// result into particle-number blocks of the new middle bond, take an FP64
// one-sided Jacobi SVD of every block, keep the largest singular values
// globally (k <= chi_rot, sigma > cutoff * sigma_1) and write the two new site
// tensors.  The tensors stay dense in memory; only their charge-allowed blocks
// are computed, since a Givens gate conserves (n_alpha, n_beta) per spin.
#include <cuda_runtime.h>

#include "df.cuh"
#include "internal.h"

namespace tnqe {
namespace {

constexpr int ROT_THREADS = 256;
constexpr int ROT_WARPS = ROT_THREADS / 32;
constexpr int MAXSIG = 1024;       // singular values of one gate: <= 4 * min(chi_l, chi_r)

struct ThetaBlk {                  // one (left sector, k1, k2) block of the two-site tensor
  int sL, sM, sR, k1, k2, start;
};
struct NewBlk {                    // one charge block of the new middle bond
  int q, nr, nc;
  int rowsec[4], rowoff[4];        // per k1': left sector (-1 none) and row offset in block
  int colsec[4], coloff[4];        // per k2': right sector and column offset
  long long wofs, qofs;            // offsets in wbuf / qbuf
  int sofs;                        // first singular value in the gate's list
  int kept, newoff;
  double scale;                    // the block is stored divided by its largest |entry|
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int qsub(int q, int qk) {      // q - qk, -1 if a component goes negative
  int qa = q / QSTRIDE - qk / QSTRIDE, qb = q % QSTRIDE - qk % QSTRIDE;
  return (qa < 0 || qb < 0) ? -1 : qa * QSTRIDE + qb;
}
__device__ __forceinline__ int qadd(int q, int qk) {
  int qa = q / QSTRIDE + qk / QSTRIDE, qb = q % QSTRIDE + qk % QSTRIDE;
  return (qa >= QSTRIDE || qb >= QSTRIDE) ? -1 : qa * QSTRIDE + qb;
}

// pair (i, j) of round r of the circle-method tournament over n2 (even) columns
__device__ __forceinline__ void tour_pair(int r, int k, int n2, int& i, int& j) {
  const int m = n2 - 1;
  if (k == 0) {
    i = r;
    j = m;
  } else {
    i = (r + k) % m;
    j = (r - k + m) % m;
  }
}

// One-sided Jacobi on W (m x n, column-major, n <= m) accumulating Q (n x n).
// Columns become mutually orthogonal: W_final = W_0 Q.  Returns 1 if it hit the
// sweep limit.
__device__ int jacobi_block(double* W, double* Q, int m, int n, int max_sweeps, int* flag) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int idx = tid; idx < n * n; idx += ROT_THREADS) Q[idx] = ((idx / n) == (idx % n)) ? 1.0 : 0.0;
  __syncthreads();
  if (n < 2) return 0;
  const double tol = 2.220446049250313e-16 * (double)m;
  const int n2 = n + (n & 1);
  int noconv = 1;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (tid == 0) *flag = 0;
    __syncthreads();
    for (int r = 0; r < n2 - 1; ++r) {
      for (int k = warp; k < n2 / 2; k += ROT_WARPS) {
        int i, j;
        tour_pair(r, k, n2, i, j);
        if (i >= n || j >= n) continue;
        double* x = W + (size_t)i * m;
        double* y = W + (size_t)j * m;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int t = lane; t < m; t += 32) {
          const double xv = x[t], yv = y[t];
          al = fma(xv, xv, al);
          be = fma(yv, yv, be);
          ga = fma(xv, yv, ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        // columns below 1e-125 of the block's largest entry are zero at this precision
        if (ga == 0.0 || al < 1e-250 || be < 1e-250 || !(fabs(ga) > tol * sqrt(al) * sqrt(be))) continue;
        const double zeta = (be - al) / (2.0 * ga);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + hypot(1.0, zeta));
        const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        if (s == 0.0) continue;                      // rotation below resolution: nothing changes
        for (int u = lane; u < m; u += 32) {
          const double xv = x[u], yv = y[u];
          x[u] = c * xv - s * yv;
          y[u] = s * xv + c * yv;
        }
        double* qx = Q + (size_t)i * n;
        double* qy = Q + (size_t)j * n;
        for (int u = lane; u < n; u += 32) {
          const double xv = qx[u], yv = qy[u];
          qx[u] = c * xv - s * yv;
          qy[u] = s * xv + c * yv;
        }
        if (lane == 0) *flag = 1;
      }
      __syncthreads();
    }
    const int any = *flag;
    __syncthreads();
    if (!any) {
      noconv = 0;
      break;
    }
  }
  return noconv;
}

#ifndef TNQE_ROT_THREADS
#define TNQE_ROT_THREADS 1024
#endif
constexpr int RT_THREADS = TNQE_ROT_THREADS;
constexpr int MAXBLK = 1024;
#ifndef TNQE_ROT_F32_STOP                    // FP32 sweeps end once gamma^2 / (alpha beta) stays below this
#define TNQE_ROT_F32_STOP 1e-4f
#endif
// Blocks with min(rows, cols) >= this go to warp teams, the others one per warp.
// N = 14, chi = 128 with block-ordered FP32 sweeps and scaled FP64 rotations:
// 16 -> 367.9 ms rotation, 24 -> 372.9, 32 -> 405.4.
#ifndef TNQE_ROT_BIG_BLOCK_N
#define TNQE_ROT_BIG_BLOCK_N 16
#endif
constexpr int BIG_BLOCK_N = TNQE_ROT_BIG_BLOCK_N;

__device__ __forceinline__ float grp8_sum(float v, unsigned mask) {
  v += __shfl_xor_sync(mask, v, 4);
  v += __shfl_xor_sync(mask, v, 2);
  v += __shfl_xor_sync(mask, v, 1);
  return v;
}
__device__ __forceinline__ double grp8_sum(double v, unsigned mask) {
  v += __shfl_xor_sync(mask, v, 4);
  v += __shfl_xor_sync(mask, v, 2);
  v += __shfl_xor_sync(mask, v, 1);
  return v;
}

__device__ __forceinline__ float2 grp8_sum_df(float2 v, unsigned mask) {
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) {
    const float2 w = make_float2(__shfl_xor_sync(mask, v.x, o), __shfl_xor_sync(mask, v.y, o));
    v = dfa::add(v, w);
  }
  return v;
}

// 1: the first refinement sweep in double-float arithmetic (FP32 pipes), the
// later ones FP64.  Off by default: on N = 14, chi = 128 it gained 2 % of the
// step (430.7 -> 422.8 ms rotation) at unchanged oracle parity before the FP64
// sweeps used scaled rotations, and lost 10 % after (382.1 -> 425.5 ms); the
// refinement sweeps stay FP64 throughout.
#ifndef TNQE_ROT_DF_SWEEP
#define TNQE_ROT_DF_SWEEP 0
#endif
constexpr int ROT_DF_SWEEP = TNQE_ROT_DF_SWEEP;

// 2^-e for the binary exponent e of a positive normal double (integer ops only)
__device__ __forceinline__ double exp2_neg_exponent(double x) {
  const int ex = ((__double2hiint(x) >> 20) & 0x7ff) - 1023;
  return __hiloint2double((1023 - ex) << 20, 0);
}

// A team of threads that works on one SVD block: a single warp, or a group of
// whole warps with its own named barrier (barrier 0 belongs to __syncthreads).
struct WarpTeam {
  __device__ int rank() const { return threadIdx.x & 31; }
  __device__ int size() const { return 32; }
  __device__ void sync() const { __syncwarp(); }
  __device__ int any(int v) const { return __any_sync(0xffffffffu, v); }
  __device__ float max(float v) const {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
  }
};
struct SubTeam {
  int base, nthr, bar;             // first thread, thread count (multiple of 32), barrier id
  float* scratch;                  // one float of shared memory owned by the team
  __device__ int rank() const { return (int)threadIdx.x - base; }
  __device__ int size() const { return nthr; }
  __device__ void sync() const { asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nthr) : "memory"); }
  __device__ int any(int v) const {
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %1, 0;\n\tbar.red.or.pred q, %2, %3, p;\n\t"
        "selp.s32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(v), "r"(bar), "r"(nthr)
        : "memory");
    return r;
  }
  __device__ float max(float v) const {   // v >= 0
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (rank() == 0) *scratch = 0.f;
    sync();
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int*>(scratch), __float_as_int(v));
    sync();
    const float r = *scratch;
    sync();
    return r;
  }
};

// Rotation angle of a column pair from its Gram entries (alpha, beta, gamma):
// t = tan(theta) = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), zeta = (beta - alpha) / (2 gamma),
// the smaller root, so |theta| <= pi / 4.  With ROT_FAST_ANGLE the quotients and
// the root use the approximate hardware reciprocal and reciprocal square root
// (a few ulp): an angle is only the start of the next refinement, and every
// rotation built from it is orthogonal at the working precision.  N = 14,
// chi = 128: rotation 430.8 -> 421.3 ms per step.
#ifndef TNQE_ROT_FAST_ANGLE
#define TNQE_ROT_FAST_ANGLE 1
#endif
constexpr int ROT_FAST_ANGLE = TNQE_ROT_FAST_ANGLE;
__device__ __forceinline__ float jacobi_tan(float al, float be, float ga) {
  if (ROT_FAST_ANGLE) {
    const float zeta = __fdividef(be - al, 2.f * ga);
    const float az = fabsf(zeta);
    float t;
    if (az < 1e18f) {
      const float w = fmaf(zeta, zeta, 1.f);
      t = __fdividef(1.f, az + w * rsqrtf(w));
    } else {
      t = __fdividef(0.5f, az);
    }
    return copysignf(t, zeta);
  }
  const float zeta = (be - al) / (2.f * ga);
  return (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + hypotf(1.f, zeta));
}

// 1: the FP32 sweeps visit the column pairs block by block (blocks of four
// columns, a block pair per warp), with a team barrier per block round.  N = 14,
// chi = 128: 430.8 -> 421.4 ms, with the fast angles 411.0 ms.
#ifndef TNQE_ROT_F32_BLOCKED
#define TNQE_ROT_F32_BLOCKED 1
#endif
constexpr int ROT_F32_BLOCKED = TNQE_ROT_F32_BLOCKED;

// 1: the FP64 sweeps apply scaled rotations.  Column i of W and Q is held as
// d_i times the stored column; a rotation (c, s = c t) of the true columns
// becomes x <- x - t (d_j / d_i) y, y <- y + t (d_i / d_j) x on the stored ones
// (one FMA per element, as for a rotation whose cosine rounds to 1) and
// d_i <- c d_i, d_j <- c d_j; the scales are multiplied in after the last sweep.
// The first refinement sweep (angles near 1e-4, cosines below 1) then needs half
// the FP64 instructions: 413.5 -> 390.5 ms on N = 14, chi = 128.
#ifndef TNQE_ROT_SCALED
#define TNQE_ROT_SCALED 1
#endif
constexpr int ROT_SCALED = TNQE_ROT_SCALED;

// 1: the FP64 Newton-Schulz step forms E = (I - Q^T Q) / 2 in FP64 and the
// correction Q E (|E| about 1e-12 after the double-float step) in FP32, then
// Q <- Q + Q E in FP64; 0: the product Q (1.5 I - 0.5 Q^T Q) in FP64.
// 390.5 -> 382.1 ms on N = 14, chi = 128.
#ifndef TNQE_ROT_NS_SPLIT
#define TNQE_ROT_NS_SPLIT 1
#endif
constexpr int ROT_NS_SPLIT = TNQE_ROT_NS_SPLIT;

// One FP32 Jacobi rotation of columns x, y (length m) and of the accumulated
// rotation columns qx, qy (length n) by an 8-lane group (lane gl of the group,
// mask gmask).  Skipped when the pair is orthogonal to tol32 relative.
__device__ __forceinline__ void f32_pair(float* __restrict__ x, float* __restrict__ y, float* __restrict__ qx,
                                         float* __restrict__ qy, int m, int n, int gl, unsigned gmask, float tol32,
                                         float& worst, int& rot) {
  float al = 0.f, be = 0.f, ga = 0.f;
  for (int t = gl; t < m; t += 8) {
    const float xv = x[t], yv = y[t];
    al = fmaf(xv, xv, al);
    be = fmaf(yv, yv, be);
    ga = fmaf(xv, yv, ga);
  }
  al = grp8_sum(al, gmask);
  be = grp8_sum(be, gmask);
  ga = grp8_sum(ga, gmask);
  float t;
  if (ROT_FAST_ANGLE) {
    if (!(al >= 1e-30f) || !(be >= 1e-30f)) return;
    const float cs = ga * rsqrtf(al) * rsqrtf(be);     // cosine of the angle between x and y
    if (!(fabsf(cs) > tol32)) return;
    worst = fmaxf(worst, cs * cs);
    t = jacobi_tan(al, be, ga);
  } else {
    if (ga == 0.f || al < 1e-30f || be < 1e-30f || !(fabsf(ga) > tol32 * sqrtf(al) * sqrtf(be))) return;
    worst = fmaxf(worst, (ga / al) * (ga / be));
    t = jacobi_tan(al, be, ga);
  }
  const float c = rsqrtf(1.f + t * t), s = c * t;
  if (s == 0.f) return;
  for (int u = gl; u < m; u += 8) {
    const float xv = x[u], yv = y[u];
    x[u] = c * xv - s * yv;
    y[u] = s * xv + c * yv;
  }
  for (int u = gl; u < n; u += 8) {
    const float xv = qx[u], yv = qy[u];
    qx[u] = c * xv - s * yv;
    qy[u] = s * xv + c * yv;
  }
  rot = 1;
}

// > 0: in a block pair of the FP32 sweeps, a group keeps its own column
// (m <= 8 x this) in registers for the pair's four rounds; 10 covers the
// largest blocks of chi = 128 (12 spills registers and was slower).
#ifndef TNQE_ROT_F32_REGCOL
#define TNQE_ROT_F32_REGCOL 10
#endif
constexpr int ROT_F32_REGCOL = TNQE_ROT_F32_REGCOL;
template <int RC>
__device__ __forceinline__ void f32_pair_reg(float (&xr)[RC], float* __restrict__ y, float* __restrict__ qx,
                                             float* __restrict__ qy, int m, int n, int gl, unsigned gmask,
                                             float tol32, float& worst, int& rot) {
  float yr[RC];
  float al = 0.f, be = 0.f, ga = 0.f;
#pragma unroll
  for (int e = 0; e < RC; ++e) {
    const int t = gl + 8 * e;
    yr[e] = t < m ? y[t] : 0.f;
    al = fmaf(xr[e], xr[e], al);
    be = fmaf(yr[e], yr[e], be);
    ga = fmaf(xr[e], yr[e], ga);
  }
  al = grp8_sum(al, gmask);
  be = grp8_sum(be, gmask);
  ga = grp8_sum(ga, gmask);
  if (!(al >= 1e-30f) || !(be >= 1e-30f)) return;
  const float cs = ga * rsqrtf(al) * rsqrtf(be);
  if (!(fabsf(cs) > tol32)) return;
  worst = fmaxf(worst, cs * cs);
  const float t = jacobi_tan(al, be, ga);
  const float c = rsqrtf(1.f + t * t), s = c * t;
  if (s == 0.f) return;
#pragma unroll
  for (int e = 0; e < RC; ++e) {
    const float xv = xr[e], yv = yr[e];
    xr[e] = c * xv - s * yv;
    const int u = gl + 8 * e;
    if (u < m) y[u] = s * xv + c * yv;
  }
  for (int u = gl; u < n; u += 8) {
    const float xv = qx[u], yv = qy[u];
    qx[u] = c * xv - s * yv;
    qy[u] = s * xv + c * yv;
  }
  rot = 1;
}

// SVD of one block by a team (one warp, or a group of warps), mixed precision.
// Bm (m x n column-major, n <= m, scaled to max |entry| = 1) is left untouched;
// on return W = Bm Q with mutually orthogonal columns (FP64) and Q (n x n)
// orthogonal to FP64 precision.  Steps: FP32 one-sided Jacobi on a copy of Bm
// until the columns are orthogonal at FP32 level; Q = Newton-Schulz
// orthogonalisation of the FP32 rotations (double-float, then FP64); W = Bm Q
// in double-float; FP64 one-sided Jacobi sweeps from that nearly orthogonal
// start (rotation angles computed in FP32, the cosine normalised in FP64 so
// every rotation is orthogonal in FP64, applied as scaled rotations).  Column
// pairs go to the team's 8-lane groups: in the FP32 sweeps a warp takes a pair
// of four-column blocks at a time, in the FP64 sweeps a round of the column
// tournament is spread over the whole team.  Returns 1 if a phase hit the sweep
// limit.
//
// GB300 executes FP64 at 1/64 of its FP32 rate, so the FP64 sweeps take one
// dot product per column pair (gamma = x.y): the squared column norms are
// computed once and carried through every rotation by the exact 2 x 2 Gram
// update (summed again from the column where that update cancels, so each
// carried norm keeps a relative error of a few m eps per rotation), the scalar
// work of a pair runs on one thread, and a rotation whose cosine rounds to 1
// costs one FMA per element.
template <class Team>
__device__ int block_svd(const Team& tm, const double* __restrict__ Bm, double* __restrict__ W,
                         double* __restrict__ Q, float* __restrict__ W32, float* __restrict__ Q32,
                         double* __restrict__ T, int m, int n, int max_sweeps) {
  const int tr = tm.rank(), ts = tm.size();
  const int lane = threadIdx.x & 31, grp = tr >> 3, ngrp = ts >> 3, gl = tr & 7;
  const unsigned gmask = 0xffu << ((lane >> 3) * 8);
  const int n2 = n + (n & 1);
  int noconv = 0;
  // ---- FP32 phase
  for (int idx = tr; idx < m * n; idx += ts) W32[idx] = (float)Bm[idx];
  for (int idx = tr; idx < n * n; idx += ts) Q32[idx] = (idx / n == idx % n) ? 1.f : 0.f;
  tm.sync();
  if (n >= 2) {
    const float tol32 = 1.2e-7f * (float)m;
    int done = 0;
    for (int sweep = 0; sweep < max_sweeps && !done; ++sweep) {
      int rot = 0;
      float worst = 0.f;                           // largest gamma^2 / (alpha beta) of the sweep
      if (ROT_F32_BLOCKED) {
        // Columns in blocks of four.  A sweep first takes the six pairs inside every block
        // (two blocks per warp), then runs a tournament over the blocks: a warp takes the
        // block pair (I, J) and its four 8-lane groups run the four matchings
        // (I_p, J_(p+s) mod 4), s = 0..3.  Every column pair is rotated once per sweep, as
        // in the column tournament, but the warps of a team meet at a team barrier once per
        // block round (n / 4 - 1 per sweep instead of n - 1); the rounds inside a block pair
        // only need warp barriers, since no other warp touches those eight columns.
        const int wrp = tr >> 5, nwarp = ts >> 5, gw = (tr >> 3) & 3;
        const int nbk = (n + 3) >> 2, nbk2 = nbk + (nbk & 1);
        for (int b0 = 2 * wrp; b0 < nbk; b0 += 2 * nwarp) {
          const int bk = b0 + (gw >> 1), p = gw & 1;
          for (int rr = 0; rr < 3; ++rr) {
            const int a = rr == 0 ? 2 * p : p;
            const int c = rr == 0 ? 2 * p + 1 : (rr == 1 ? p + 2 : 3 - p);
            const int i = 4 * bk + a, j = 4 * bk + c;
            if (bk < nbk && j < n)
              f32_pair(W32 + (size_t)i * m, W32 + (size_t)j * m, Q32 + (size_t)i * n, Q32 + (size_t)j * n, m, n,
                       gl, gmask, tol32, worst, rot);
            __syncwarp();
          }
        }
        tm.sync();
        for (int r = 0; r < nbk2 - 1; ++r) {
          for (int k = wrp; k < nbk2 / 2; k += nwarp) {
            int I, J;
            tour_pair(r, k, nbk2, I, J);
            const bool act = I < nbk && J < nbk;
            if (ROT_F32_REGCOL > 0 && m <= 8 * ROT_F32_REGCOL) {
              constexpr int RC = ROT_F32_REGCOL > 0 ? ROT_F32_REGCOL : 1;
              const int i = 4 * I + gw;
              const bool own = act && i < n;
              float* x = W32 + (size_t)i * m;
              float xr[RC];
#pragma unroll
              for (int e = 0; e < RC; ++e) {
                const int t = gl + 8 * e;
                xr[e] = (own && t < m) ? x[t] : 0.f;
              }
              for (int s = 0; s < 4; ++s) {
                const int j = 4 * J + ((gw + s) & 3);
                if (own && j < n)
                  f32_pair_reg<RC>(xr, W32 + (size_t)j * m, Q32 + (size_t)i * n, Q32 + (size_t)j * n, m, n, gl, gmask,
                                   tol32, worst, rot);
                __syncwarp();
              }
              if (own) {
#pragma unroll
                for (int e = 0; e < RC; ++e) {
                  const int t = gl + 8 * e;
                  if (t < m) x[t] = xr[e];
                }
              }
            } else {
              for (int s = 0; s < 4; ++s) {
                const int i = 4 * I + gw, j = 4 * J + ((gw + s) & 3);
                if (act && i < n && j < n)
                  f32_pair(W32 + (size_t)i * m, W32 + (size_t)j * m, Q32 + (size_t)i * n, Q32 + (size_t)j * n, m, n,
                           gl, gmask, tol32, worst, rot);
                __syncwarp();
              }
            }
          }
          tm.sync();
        }
      } else {
        for (int r = 0; r < n2 - 1; ++r) {
          for (int k = grp; k < n2 / 2; k += ngrp) {
            int i, j;
            tour_pair(r, k, n2, i, j);
            if (i >= n || j >= n) continue;
            f32_pair(W32 + (size_t)i * m, W32 + (size_t)j * m, Q32 + (size_t)i * n, Q32 + (size_t)j * n, m, n, gl,
                     gmask, tol32, worst, rot);
          }
          tm.sync();
        }
      }
      // A sweep whose largest relative off-diagonal was below 1e-2 leaves the
      // columns orthogonal to about 1e-4 (quadratic convergence): the FP64
      // phase then still needs two sweeps (1e-4 -> 1e-8 -> below the FP64
      // criterion), as from the FP32 floor, and the last FP32 sweeps are saved.
      done = !tm.any(rot) || tm.max(worst) <= TNQE_ROT_F32_STOP;
    }
  }
  // ---- Q = orthogonalised FP32 rotations: Newton-Schulz Q <- Q (1.5 I - 0.5 Q^T Q), each step
  // squaring the orthogonality defect (about 1e-6 for the FP32 product): the first step in
  // double-float arithmetic (its result only needs 1e-12), the second in FP64.
  {
    float2* Qd = reinterpret_cast<float2*>(T);      // Q as double-float (T holds n x n doubles)
    float2* Md = reinterpret_cast<float2*>(W);      // 1.5 I - 0.5 Q^T Q (W holds m x n >= n x n doubles)
    float2* Qn = reinterpret_cast<float2*>(Q);      // the new Q, double-float, converted in place below
    for (int idx = tr; idx < n * n; idx += ts) Qd[idx] = make_float2(Q32[idx], 0.f);
    tm.sync();
    for (int idx = tr; idx < n * n; idx += ts) {
      const int i = idx % n, j = idx / n;
      const float2* qi = Qd + (size_t)i * n;
      const float2* qj = Qd + (size_t)j * n;
      float2 acc = make_float2(0.f, 0.f);
      for (int k = 0; k < n; ++k) acc = dfa::fma(qi[k], qj[k], acc);
      Md[idx] = dfa::add(make_float2(i == j ? 1.5f : 0.f, 0.f), make_float2(-0.5f * acc.x, -0.5f * acc.y));
    }
    tm.sync();
    for (int idx = tr; idx < n * n; idx += ts) {
      const int row = idx % n, col = idx / n;
      float2 acc = make_float2(0.f, 0.f);
      for (int k = 0; k < n; ++k) acc = dfa::fma(Qd[(size_t)k * n + row], Md[(size_t)col * n + k], acc);
      Qn[idx] = acc;
    }
    tm.sync();
    for (int idx = tr; idx < n * n; idx += ts) Q[idx] = dfa::to_double(Qn[idx]);   // same 8 bytes per element
    tm.sync();
  }
  {
    // Q^T Q is symmetric: one dot product per entry of its upper triangle (i <= j),
    // enumerated densely so that no lane of an FP64 instruction idles
    const int ntri = n * (n + 1) / 2;
    for (int idx = tr; idx < ntri; idx += ts) {
      int j = (int)((sqrtf(8.f * (float)idx + 1.f) - 1.f) * 0.5f);
      while (j * (j + 1) / 2 > idx) --j;
      while ((j + 1) * (j + 2) / 2 <= idx) ++j;
      const int i = idx - j * (j + 1) / 2;
      const double* qi = Q + (size_t)i * n;
      const double* qj = Q + (size_t)j * n;
      double acc = 0.0;
      for (int k = 0; k < n; ++k) acc = fma(qi[k], qj[k], acc);
      if (ROT_NS_SPLIT) {
        const float e = (float)(0.5 * ((i == j ? 1.0 : 0.0) - acc));
        Q32[(size_t)j * n + i] = e;                  // E (the FP32 rotations are no longer needed)
        Q32[(size_t)i * n + j] = e;
      } else {
        const double v = (i == j ? 1.5 : 0.0) - 0.5 * acc;
        T[(size_t)j * n + i] = v;
        T[(size_t)i * n + j] = v;
      }
    }
    if (ROT_NS_SPLIT) {
      for (int idx = tr; idx < n * n; idx += ts) W32[idx] = (float)Q[idx];   // W32 (m*n >= n*n) is free
      tm.sync();
      for (int idx = tr; idx < n * n; idx += ts) {
        const int row = idx % n, col = idx / n;
        float acc = 0.f;
        for (int k = 0; k < n; ++k) acc = fmaf(W32[(size_t)k * n + row], Q32[(size_t)col * n + k], acc);
        Q[idx] += (double)acc;                       // each thread owns its entry: no read of Q by others below
      }
      tm.sync();
    } else {
      tm.sync();
      for (int idx = tr; idx < n * n; idx += ts) {
        const int row = idx % n, col = idx / n;
        double acc = 0.0;
        for (int k = 0; k < n; ++k) acc = fma(Q[(size_t)k * n + row], T[(size_t)col * n + k], acc);
        W[idx] = acc;                                // W used as temporary (m*n >= n*n)
      }
      tm.sync();
      for (int idx = tr; idx < n * n; idx += ts) Q[idx] = W[idx];
      tm.sync();
    }
  }
  // ---- W = Bm Q in double-float: Bm converted in place (the caller no longer needs it),
  // Q copied to double-float in T; W comes back to FP64 in place.  Its error (about
  // 2^-48 relative) is far below the truncation and the FP64 sweeps keep W = Bm Q to it.
  {
    float2* Bd = reinterpret_cast<float2*>(const_cast<double*>(Bm));
    float2* Qd = reinterpret_cast<float2*>(T);
    float2* Wd = reinterpret_cast<float2*>(W);
    for (int idx = tr; idx < m * n; idx += ts) {
      const double b = Bm[idx];
      Bd[idx] = dfa::from_double(b);
    }
    for (int idx = tr; idx < n * n; idx += ts) Qd[idx] = dfa::from_double(Q[idx]);
    tm.sync();
    for (int idx = tr; idx < m * n; idx += ts) {
      const int row = idx % m, col = idx / m;
      const float2* qc = Qd + (size_t)col * n;
      float2 acc = make_float2(0.f, 0.f);
      for (int k = 0; k < n; ++k) acc = dfa::fma(Bd[(size_t)k * m + row], qc[k], acc);
      Wd[idx] = acc;
    }
    tm.sync();
    if (!(ROT_DF_SWEEP && n >= 2)) {
      for (int idx = tr; idx < m * n; idx += ts) W[idx] = dfa::to_double(Wd[idx]);
      tm.sync();
    }
  }
  if (n < 2) return noconv;
  const bool df_first = ROT_DF_SWEEP != 0;       // W is double-float here; Q joins it below
  float2* Wd = reinterpret_cast<float2*>(W);
  float2* Qd = reinterpret_cast<float2*>(Q);
  // ---- FP64 phase.  A sweep that finds no pair above 1e-7 relative leaves
  // off-diagonals near 1e-14 after its own rotations (quadratic convergence),
  // so the loop ends after that sweep without a confirming one.
  //
  // Every round takes three steps: the 8-lane groups form gamma = x.y of their
  // column pairs; one thread per pair turns (alpha, beta, gamma) into the
  // rotation and the new norms; the groups apply the rotations.  The per-pair
  // scalar FP64 work (angle, cosine, norm update) thus fills whole warp
  // instructions with 32 pairs instead of 4.
  double* nrm = T;                                 // squared column norms (T is free from here on)
  double* gam = const_cast<double*>(Bm);           // per pair of a round: gamma, then a recompute code
  double* cv = gam + n2 / 2;                       // cos, sin per pair (Bm is free: m n >= 3 n2 / 2)
  double* sv = cv + n2 / 2;
  double* dsc = T + n;                             // column scales of the scaled rotations (n * n >= 2 n)
  double* dinv = T + 2 * n;                        // their reciprocals, kept where n * n >= 3 n
  if (df_first) {
    for (int idx = tr; idx < n * n; idx += ts) Qd[idx] = dfa::from_double(Q[idx]);   // in place, same 8 bytes
    for (int j = grp; j < n; j += ngrp) {
      const float2* x = Wd + (size_t)j * m;
      float2 a = make_float2(0.f, 0.f);
      for (int t = gl; t < m; t += 8) a = dfa::fma(x[t], x[t], a);
      a = grp8_sum_df(a, gmask);
      if (gl == 0) {
        nrm[j] = dfa::to_double(a);
        dsc[j] = 1.0;
        if (n >= 3) dinv[j] = 1.0;
      }
    }
  } else {
    for (int j = grp; j < n; j += ngrp) {
      const double* x = W + (size_t)j * m;
      double a = 0.0;
      for (int t = gl; t < m; t += 8) a = fma(x[t], x[t], a);
      a = grp8_sum(a, gmask);
      if (gl == 0) {
        nrm[j] = a;
        dsc[j] = 1.0;
        if (n >= 3) dinv[j] = 1.0;
      }
    }
  }
  tm.sync();
  const double tol64 = 2.220446049250313e-16 * (double)m;
  const float tol64sq = (float)(tol64 * tol64);
  noconv = 1;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    int rot = 0;
    float worst = 0.f;                             // largest gamma^2 / (alpha beta) seen this sweep
    const bool dfw = df_first && sweep == 0;       // this sweep in double-float
    for (int r = 0; r < n2 - 1; ++r) {
      for (int k = grp; k < n2 / 2; k += ngrp) {
        int i, j;
        tour_pair(r, k, n2, i, j);
        if (i >= n || j >= n) continue;
        if (dfw) {
          const float2* x = Wd + (size_t)i * m;
          const float2* y = Wd + (size_t)j * m;
          float2 ga = make_float2(0.f, 0.f), gb = make_float2(0.f, 0.f);   // two chains
          int t = gl;
          for (; t + 8 < m; t += 16) {
            ga = dfa::fma(x[t], y[t], ga);
            gb = dfa::fma(x[t + 8], y[t + 8], gb);
          }
          if (t < m) ga = dfa::fma(x[t], y[t], ga);
          ga = grp8_sum_df(dfa::add(ga, gb), gmask);
          if (gl == 0) gam[k] = dfa::to_double(ga);
        } else {
          const double* x = W + (size_t)i * m;
          const double* y = W + (size_t)j * m;
          double ga = 0.0;
          for (int t = gl; t < m; t += 8) ga = fma(x[t], y[t], ga);
          ga = grp8_sum(ga, gmask);
          if (gl == 0) gam[k] = ga;
        }
      }
      tm.sync();
      for (int k = tr; k < n2 / 2; k += ts) {
        int i, j;
        tour_pair(r, k, n2, i, j);
        double c = 1.0, s = 0.0, code = 0.0;
        double a1 = 1.0, a2 = 0.0;                   // what the groups apply: (c, s), or the scaled (-t dj/di, t di/dj)
        if (i < n && j < n) {
          const bool scaled = ROT_SCALED != 0;
          const double al = nrm[i], be = nrm[j];
          const double ga = scaled ? gam[k] * (dsc[i] * dsc[j]) : gam[k];
          // columns below 1e-125 of the block's largest entry are zero at this precision
          if (ga != 0.0 && al >= 1e-250 && be >= 1e-250) {
            const double sc = exp2_neg_exponent(fmax(al, be));
            const float af = (float)(al * sc), bf = (float)(be * sc), gf = (float)(ga * sc);
            if (gf * gf > tol64sq * af * bf) {
              worst = fmaxf(worst, (gf * gf) / (af * bf));
              const float t32 = jacobi_tan(af, bf, gf);
              const double t = (double)t32;
              double w = 1.0;
              if (fabsf(t32) < 7.0e-9f) {            // 1 + t^2 rounds to 1: the rotation is I + t J
                s = t;
              } else {
                w = fma(t, t, 1.0);
                c = (double)rsqrtf((float)w);
                c = c * fma(-0.5 * w, c * c, 1.5);
                c = c * fma(-0.5 * w, c * c, 1.5);
                s = t * c;
              }
              if (s != 0.0) {
                rot = 1;
                // |c x - s y|^2 and |s x + c y|^2 from the Gram entries.  The update carries
                // the dot product's error (about m eps |x||y|) into the smaller norm, divided
                // by the fraction of its terms that survives: where less than half survives
                // (pairs far from orthogonal, e.g. the noise columns of a rank-deficient
                // block, which keep rotating for several sweeps) the rotating group sums that
                // norm again.
                const double cc = c * c, ss = s * s, g2 = 2.0 * c * s * ga;
                const double na = fma(cc, al, fma(ss, be, -g2));
                const double nb2 = fma(ss, al, fma(cc, be, g2));
                const bool ri = !(na > 0.5 * (cc * al + ss * be + fabs(g2)));
                const bool rj = !(nb2 > 0.5 * (ss * al + cc * be + fabs(g2)));
                nrm[i] = na;
                nrm[j] = nb2;
                code = (ri ? 1.0 : 0.0) + (rj ? 2.0 : 0.0);
                if (scaled) {
                  // d_j / d_i and d_i / d_j from the kept reciprocals (1 / c = w c)
                  const double di = dsc[i], dj = dsc[j];
                  const bool inv = n >= 3;
                  const double rji = inv ? dj * dinv[i] : dj / di, rij = inv ? di * dinv[j] : di / dj;
                  a1 = -t * rji;
                  a2 = t * rij;
                  if (c != 1.0) {
                    dsc[i] = c * di;
                    dsc[j] = c * dj;
                    if (inv) {
                      const double ic = w * c;
                      dinv[i] *= ic;
                      dinv[j] *= ic;
                    }
                  }
                } else {
                  a1 = c;
                  a2 = s;
                }
              }
            }
          }
        }
        cv[k] = a1;
        sv[k] = a2;
        gam[k] = code;
      }
      tm.sync();
      for (int k = grp; k < n2 / 2 && dfw; k += ngrp) {
        const double s = sv[k];
        if (s == 0.0) continue;
        const double c = cv[k];
        int i, j;
        tour_pair(r, k, n2, i, j);
        float2* x = Wd + (size_t)i * m;
        float2* y = Wd + (size_t)j * m;
        float2* qx = Qd + (size_t)i * n;
        float2* qy = Qd + (size_t)j * n;
        const float2 s2 = dfa::from_double(s), ms2 = make_float2(-s2.x, -s2.y), c2 = dfa::from_double(c);
        if (ROT_SCALED) {                          // c2 holds -t dj/di, s2 holds t di/dj
          for (int u = gl; u < m; u += 8) {
            const float2 xv = x[u], yv = y[u];
            x[u] = dfa::fma(c2, yv, xv);
            y[u] = dfa::fma(s2, xv, yv);
          }
          for (int u = gl; u < n; u += 8) {
            const float2 xv = qx[u], yv = qy[u];
            qx[u] = dfa::fma(c2, yv, xv);
            qy[u] = dfa::fma(s2, xv, yv);
          }
        } else if (c == 1.0) {
          for (int u = gl; u < m; u += 8) {
            const float2 xv = x[u], yv = y[u];
            x[u] = dfa::fma(ms2, yv, xv);
            y[u] = dfa::fma(s2, xv, yv);
          }
          for (int u = gl; u < n; u += 8) {
            const float2 xv = qx[u], yv = qy[u];
            qx[u] = dfa::fma(ms2, yv, xv);
            qy[u] = dfa::fma(s2, xv, yv);
          }
        } else {
          for (int u = gl; u < m; u += 8) {
            const float2 xv = x[u], yv = y[u];
            x[u] = dfa::add(dfa::mul(c2, xv), dfa::mul(ms2, yv));
            y[u] = dfa::add(dfa::mul(s2, xv), dfa::mul(c2, yv));
          }
          for (int u = gl; u < n; u += 8) {
            const float2 xv = qx[u], yv = qy[u];
            qx[u] = dfa::add(dfa::mul(c2, xv), dfa::mul(ms2, yv));
            qy[u] = dfa::add(dfa::mul(s2, xv), dfa::mul(c2, yv));
          }
        }
        const double code = gam[k];
        if (code != 0.0) {
          const int cd = (int)code;
          if (cd & 1) {
            float2 acc = make_float2(0.f, 0.f);
            for (int u = gl; u < m; u += 8) acc = dfa::fma(x[u], x[u], acc);
            acc = grp8_sum_df(acc, gmask);
            if (gl == 0) nrm[i] = ROT_SCALED ? dfa::to_double(acc) * (dsc[i] * dsc[i]) : dfa::to_double(acc);
          }
          if (cd & 2) {
            float2 acc = make_float2(0.f, 0.f);
            for (int u = gl; u < m; u += 8) acc = dfa::fma(y[u], y[u], acc);
            acc = grp8_sum_df(acc, gmask);
            if (gl == 0) nrm[j] = ROT_SCALED ? dfa::to_double(acc) * (dsc[j] * dsc[j]) : dfa::to_double(acc);
          }
        }
      }
      for (int k = grp; k < n2 / 2 && !dfw; k += ngrp) {
        const double s = sv[k];
        if (s == 0.0) continue;
        const double c = cv[k];
        int i, j;
        tour_pair(r, k, n2, i, j);
        double* x = W + (size_t)i * m;
        double* y = W + (size_t)j * m;
        double* qx = Q + (size_t)i * n;
        double* qy = Q + (size_t)j * n;
        if (ROT_SCALED) {                          // c holds -t dj/di, s holds t di/dj
          for (int u = gl; u < m; u += 8) {
            const double xv = x[u], yv = y[u];
            x[u] = fma(c, yv, xv);
            y[u] = fma(s, xv, yv);
          }
          for (int u = gl; u < n; u += 8) {
            const double xv = qx[u], yv = qy[u];
            qx[u] = fma(c, yv, xv);
            qy[u] = fma(s, xv, yv);
          }
        } else if (c == 1.0) {
          for (int u = gl; u < m; u += 8) {
            const double xv = x[u], yv = y[u];
            x[u] = fma(-s, yv, xv);
            y[u] = fma(s, xv, yv);
          }
          for (int u = gl; u < n; u += 8) {
            const double xv = qx[u], yv = qy[u];
            qx[u] = fma(-s, yv, xv);
            qy[u] = fma(s, xv, yv);
          }
        } else {
          for (int u = gl; u < m; u += 8) {
            const double xv = x[u], yv = y[u];
            x[u] = c * xv - s * yv;
            y[u] = s * xv + c * yv;
          }
          for (int u = gl; u < n; u += 8) {
            const double xv = qx[u], yv = qy[u];
            qx[u] = c * xv - s * yv;
            qy[u] = s * xv + c * yv;
          }
        }
        const double code = gam[k];
        if (code != 0.0) {
          const int cd = (int)code;
          if (cd & 1) {
            double acc = 0.0;
            for (int u = gl; u < m; u += 8) acc = fma(x[u], x[u], acc);
            acc = grp8_sum(acc, gmask);
            if (gl == 0) nrm[i] = ROT_SCALED ? acc * (dsc[i] * dsc[i]) : acc;
          }
          if (cd & 2) {
            double acc = 0.0;
            for (int u = gl; u < m; u += 8) acc = fma(y[u], y[u], acc);
            acc = grp8_sum(acc, gmask);
            if (gl == 0) nrm[j] = ROT_SCALED ? acc * (dsc[j] * dsc[j]) : acc;
          }
        }
      }
      tm.sync();
    }
    if (dfw) {
      // back to FP64; the norms summed again in FP64; at least one FP64 sweep follows
      for (int idx = tr; idx < m * n; idx += ts) W[idx] = dfa::to_double(Wd[idx]);
      for (int idx = tr; idx < n * n; idx += ts) Q[idx] = dfa::to_double(Qd[idx]);
      tm.sync();
      for (int j = grp; j < n; j += ngrp) {
        const double* x = W + (size_t)j * m;
        double a = 0.0;
        for (int t = gl; t < m; t += 8) a = fma(x[t], x[t], a);
        a = grp8_sum(a, gmask);
        if (gl == 0) nrm[j] = ROT_SCALED ? a * (dsc[j] * dsc[j]) : a;
      }
      tm.sync();
      continue;
    }
    worst = tm.max(worst);
    if (!tm.any(rot) || worst <= 1e-14f) {
      noconv = 0;
      break;
    }
  }
  if (ROT_SCALED) {                                // true columns: the stored ones times their scales
    for (int idx = tr; idx < m * n; idx += ts) W[idx] *= dsc[idx / m];
    for (int idx = tr; idx < n * n; idx += ts) Q[idx] *= dsc[idx / n];
    tm.sync();
  }
  return noconv;
}

// Large SVD blocks run concurrently on warp teams.  A configuration fixes the
// CTA size, the number of teams and the lead team (the largest block of each
// gate).  One 1024-thread CTA per SM: two 512-thread CTAs per SM (all 276
// rotated pairs of N = 20 at once instead of two waves) took 15.3 s against
// 8.7 s, since two pairs then share one SM's FP64 units.
#ifndef TNQE_ROT_TEAMS
#define TNQE_ROT_TEAMS 8                      // teams of (CTA warps) / 8 warps for the large blocks
#endif
// The lead team: 12 warps (five teams of four beside it) measured 360.0 ms
// against 365.1 ms for 16 warps on N = 14, chi = 128, together with the
// register-held columns of the FP32 block pairs.
#ifndef TNQE_ROT_LEAD_WARPS
#define TNQE_ROT_LEAD_WARPS 12
#endif
template <int THREADS, int TEAMS, int LEAD, int MINB>
struct RotCfg {
  static constexpr int threads = THREADS, warps = THREADS / 32, min_blocks = MINB;
  static constexpr int team_warps = warps / TEAMS, team_threads = team_warps * 32, lead = LEAD;
  static constexpr int rest = (warps - LEAD) / team_warps;         // teams beside the lead team
  static constexpr int slots = 1 + rest + LEAD / team_warps;       // the lead team splits into teams
  static_assert(TEAMS * team_warps == warps, "teams must tile the CTA");
  static_assert(LEAD % team_warps == 0 && LEAD <= warps, "lead team splits into teams");
  static_assert(slots <= 15, "one named barrier per team");
};
using RotWide = RotCfg<RT_THREADS, TNQE_ROT_TEAMS, TNQE_ROT_LEAD_WARPS, 1>;

template <class C>
__global__ void __launch_bounds__(C::threads, C::min_blocks) rotate_pairs_kernel(const RotDesc* __restrict__ descs) {
  constexpr int RT_THREADS = C::threads, RT_WARPS = C::warps, ROT_TEAM_WARPS = C::team_warps;
  constexpr int ROT_TEAM_THREADS = C::team_threads, ROT_LEAD_WARPS = C::lead, ROT_REST_TEAMS = C::rest;
  constexpr int ROT_SLOTS = C::slots;
  const RotDesc& D = descs[blockIdx.x];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int N = D.N;

  __shared__ int lutL[QSPACE], lutM[QSPACE], lutR[QSPACE];
  __shared__ SectorTable secL, secM, secR;
  __shared__ int gnz_n[16], gnz_k[16][16];
  __shared__ double gnz_v[16][16];
  __shared__ double sig[MAXSIG];
  __shared__ unsigned char sig_keep[MAXSIG];
  __shared__ short s_ord[QSPACE];                 // blocks of a gate: one per charge of the new bond
  __shared__ long long s_scan[QSPACE / 32][4];
  __shared__ int s_tscan[C::warps][2], s_carry[2];
  __shared__ int s_nblk, s_nnew, s_total, s_nsig, s_keep, s_status, s_nbig;
  __shared__ float s_tscr[ROT_SLOTS];
  __shared__ int s_tbi[ROT_SLOTS], s_next_big, s_next_small;
  __shared__ double s_disc, s_red[RT_WARPS], s_flops;

  ThetaBlk* tb = reinterpret_cast<ThetaBlk*>(D.meta);
  const long long tb_cap = D.meta_cap / 2 / (long long)(sizeof(ThetaBlk) / sizeof(int));
  NewBlk* nb = reinterpret_cast<NewBlk*>(D.meta + D.meta_cap / 2);
  long long nb_cap = D.meta_cap / 2 / (long long)(sizeof(NewBlk) / sizeof(int));
  if (nb_cap > MAXBLK) nb_cap = MAXBLK;

  // ---- copy the input state into the work buffer
  for (int s = 0; s < N; ++s) {
    const long long n = (long long)D.src_dims[s] * 4 * D.src_dims[s + 1];
    const double* src = D.src + D.src_off[s];
    double* dst = D.work + D.work_off[s];
    for (long long x = tid; x < n; x += RT_THREADS) dst[x] = src[x];
  }
  for (int b = tid; b <= N; b += RT_THREADS) {
    D.work_dims[b] = D.src_dims[b];
    D.work_sec[b] = D.src_sec[b];
  }
  if (tid == 0) {
    s_disc = 0.0;
    s_status = 0;
    s_flops = 0.0;
  }
  __syncthreads();

  for (int g = 0; g < D.ngates; ++g) {
    const int a = D.gate_site[g];
    const int side = D.gate_side[g];
    for (int x = tid; x < QSPACE; x += RT_THREADS) {
      lutL[x] = -1;
      lutM[x] = -1;
      lutR[x] = -1;
    }
    {
      constexpr int W4 = (int)(sizeof(SectorTable) / 4);
      const int* srcs = reinterpret_cast<const int*>(D.work_sec + a);
      int* dL = reinterpret_cast<int*>(&secL);
      int* dM = reinterpret_cast<int*>(&secM);
      int* dR = reinterpret_cast<int*>(&secR);
      for (int x = tid; x < 3 * W4; x += RT_THREADS) {
        const int v = srcs[x];
        if (x < W4) dL[x] = v; else if (x < 2 * W4) dM[x - W4] = v; else dR[x - 2 * W4] = v;
      }
    }
    __syncthreads();
    for (int x = tid; x < secL.nsec; x += RT_THREADS) lutL[secL.q[x]] = x;
    for (int x = tid; x < secM.nsec; x += RT_THREADS) lutM[secM.q[x]] = x;
    for (int x = tid; x < secR.nsec; x += RT_THREADS) lutR[secR.q[x]] = x;
    if (tid < 16) {                       // nonzero inputs of each gate row
      int c = 0;
      for (int K = 0; K < 16; ++K) {
        const double v = D.gates[(size_t)g * 256 + tid * 16 + K];
        if (v != 0.0) {
          gnz_k[tid][c] = K;
          gnz_v[tid][c] = v;
          ++c;
        }
      }
      gnz_n[tid] = c;
    }
    const int chl = D.work_dims[a], chm = D.work_dims[a + 1], chr = D.work_dims[a + 2];
    double* Lt = D.work + D.work_off[a];
    double* Rt = D.work + D.work_off[a + 1];
    __syncthreads();

    // ---- two-site tensor theta[l][k1][k2][r], charge-allowed blocks only.  The
    // block list (left sector, k1, k2 in that order) is built one item per thread,
    // its start offsets from a prefix sum over the items, chunk by chunk.
    {
      const int nitems = secL.nsec * 16;
      if (tid == 0) {
        s_carry[0] = 0;
        s_carry[1] = 0;
      }
      __syncthreads();
      for (int base = 0; base < nitems; base += C::threads) {
        const int it = base + tid;
        int ex = 0, sz = 0, sL = 0, k1 = 0, k2 = 0, sM = -1, sR = -1;
        if (it < nitems) {
          sL = it >> 4;
          k1 = (it >> 2) & 3;
          k2 = it & 3;
          const int qM = qadd(secL.q[sL], local_charge(k1));
          sM = qM < 0 ? -1 : lutM[qM];
          if (sM >= 0) {
            const int qR = qadd(qM, local_charge(k2));
            sR = qR < 0 ? -1 : lutR[qR];
            if (sR >= 0) {
              ex = 1;
              sz = secL.dim[sL] * secR.dim[sR];
            }
          }
        }
        int v0 = ex, v1 = sz;                      // inclusive scan within the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int t0 = __shfl_up_sync(0xffffffffu, v0, o), t1 = __shfl_up_sync(0xffffffffu, v1, o);
          if (lane >= o) {
            v0 += t0;
            v1 += t1;
          }
        }
        if (lane == 31) {
          s_tscan[warp][0] = v0;
          s_tscan[warp][1] = v1;
        }
        __syncthreads();
        v0 += s_carry[0];
        v1 += s_carry[1];
        for (int w = 0; w < warp; ++w) {
          v0 += s_tscan[w][0];
          v1 += s_tscan[w][1];
        }
        if (ex) {
          const int idx = v0 - 1;
          if (idx < tb_cap) tb[idx] = ThetaBlk{sL, sM, sR, k1, k2, v1 - sz};
          atomicAdd(&s_flops, 2.0 * secL.dim[sL] * secM.dim[sM] * secR.dim[sR]);   // integers: exact in any order
        }
        __syncthreads();
        if (tid == C::threads - 1) {               // the chunk's last item carries the running totals
          s_carry[0] = v0;
          s_carry[1] = v1;
        }
        __syncthreads();
      }
      if (tid == 0) {
        int nblk = s_carry[0];
        if (nblk > tb_cap) {
          s_status |= STATUS_OVERFLOW;
          nblk = (int)tb_cap;
        }
        s_nblk = nblk;
        s_total = s_carry[1];
      }
    }
    __syncthreads();
    {
      const int nblk = s_nblk, total = s_total;
      for (int idx = tid; idx < total; idx += RT_THREADS) {
        int lo = 0, hi = nblk - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (tb[mid].start <= idx) lo = mid; else hi = mid - 1;
        }
        const ThetaBlk B = tb[lo];
        const int dR = secR.dim[B.sR];
        const int li = (idx - B.start) / dR, ri = (idx - B.start) % dR;
        const int l = secL.off[B.sL] + li, r = secR.off[B.sR] + ri;
        const int m0 = secM.off[B.sM], m1 = m0 + secM.dim[B.sM];
        const double* lrow = Lt + ((size_t)l * 4 + B.k1) * chm;
        const double* rcol = Rt + (size_t)B.k2 * chr + r;
        double acc = 0.0;
        for (int m = m0; m < m1; ++m) acc = fma(lrow[m], rcol[(size_t)m * 4 * chr], acc);
        D.theta[(((size_t)l * 4 + B.k1) * 4 + B.k2) * chr + r] = acc;
      }
    }
    // ---- blocks of the new middle bond, ascending charge: one thread per charge q
    // of the new bond, offsets from prefix sums over q
    {
      static_assert(QSPACE % 32 == 0 && QSPACE <= C::threads, "one thread per charge");
      NewBlk B;
      int mm = 0, nn = 0;
      bool ex = false;
      if (tid < QSPACE) {
        const int q = tid;
        B.q = q;
        int nr = 0, nc = 0;
        for (int k = 0; k < 4; ++k) {
          const int qL = qsub(q, local_charge(k));
          const int sL = qL < 0 ? -1 : lutL[qL];
          B.rowsec[k] = sL;
          B.rowoff[k] = nr;
          if (sL >= 0) nr += secL.dim[sL];
          const int qR = qadd(q, local_charge(k));
          const int sR = qR < 0 ? -1 : lutR[qR];
          B.colsec[k] = sR;
          B.coloff[k] = nc;
          if (sR >= 0) nc += secR.dim[sR];
        }
        B.nr = nr;
        B.nc = nc;
        ex = nr > 0 && nc > 0;
        if (ex) {
          mm = nr > nc ? nr : nc;
          nn = nr > nc ? nc : nr;
        }
      }
      // inclusive scans of (block, m n, n n, n) over the charges, warp by warp
      long long v0 = ex ? 1 : 0, v1 = (long long)mm * nn, v2 = (long long)nn * nn, v3 = nn;
      if (tid < QSPACE) {
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const long long t0 = __shfl_up_sync(0xffffffffu, v0, o), t1 = __shfl_up_sync(0xffffffffu, v1, o);
          const long long t2 = __shfl_up_sync(0xffffffffu, v2, o), t3 = __shfl_up_sync(0xffffffffu, v3, o);
          if (lane >= o) {
            v0 += t0;
            v1 += t1;
            v2 += t2;
            v3 += t3;
          }
        }
        if (lane == 31) {
          s_scan[warp][0] = v0;
          s_scan[warp][1] = v1;
          s_scan[warp][2] = v2;
          s_scan[warp][3] = v3;
        }
      }
      __syncthreads();
      if (tid < QSPACE) {
        for (int w = 0; w < warp; ++w) {
          v0 += s_scan[w][0];
          v1 += s_scan[w][1];
          v2 += s_scan[w][2];
          v3 += s_scan[w][3];
        }
        if (ex) {                                  // exclusive offsets: inclusive minus own
          const int idx = (int)(v0 - 1);
          B.wofs = v1 - (long long)mm * nn;
          B.qofs = v2 - (long long)nn * nn;
          B.sofs = (int)(v3 - nn);
          B.kept = 0;
          B.newoff = 0;
          B.scale = 1.0;
          if (idx < nb_cap && v3 <= MAXSIG) nb[idx] = B;
          atomicAdd(&s_flops, 4.0 * mm * nn * nn + 8.0 * nn * nn * nn + 8.0 * mm * nn);   // integers: exact in any order
        }
        if (tid == QSPACE - 1) {
          int nnew = (int)v0, nsig = (int)v3;
          if (nnew > nb_cap || v3 > MAXSIG) {
            s_status |= STATUS_OVERFLOW;
            nnew = 0;
            nsig = 0;
          }
          s_nnew = nnew;
          s_nsig = nsig;
        }
      }
    }
    __syncthreads();
    const int nnew = s_nnew;
    // ---- largest blocks first: rank by m n^2
    for (int b = tid; b < nnew; b += RT_THREADS) {
      const NewBlk& B = nb[b];
      const long long cb = (long long)(B.nr > B.nc ? B.nr : B.nc) * (B.nr < B.nc ? B.nr : B.nc) * (B.nr < B.nc ? B.nr : B.nc);
      int rank = 0;
      for (int b2 = 0; b2 < nnew; ++b2) {
        const NewBlk& B2 = nb[b2];
        const long long cc = (long long)(B2.nr > B2.nc ? B2.nr : B2.nc) * (B2.nr < B2.nc ? B2.nr : B2.nc) * (B2.nr < B2.nc ? B2.nr : B2.nc);
        rank += (cc > cb || (cc == cb && b2 < b)) ? 1 : 0;
      }
      s_ord[rank] = (short)b;
    }
    __syncthreads();
    // ---- SVD of every block.  Large blocks go to teams of warps, each team
    // taking the next block from a shared counter (largest first); a team with
    // nothing left and every warp afterwards take the small blocks one warp per
    // block from a second counter.
    if (tid == 0) {
      int nb_big = 0;
      while (nb_big < nnew) {
        const NewBlk& B = nb[s_ord[nb_big]];
        if ((B.nr < B.nc ? B.nr : B.nc) < BIG_BLOCK_N) break;
        ++nb_big;
      }
      s_nbig = nb_big;
      s_next_big = nb_big > 0 ? 1 : 0;            // block 0, the largest, belongs to the lead team
      s_next_small = 0;
    }
    __syncthreads();
    const int nbig = s_nbig;
    {
      // Large blocks on warp teams.  The largest block of a gate (a quarter to a half
      // of the gate's SVD work at chi = 128) runs on a lead team of ROT_LEAD_WARPS
      // warps while the other warps, in teams of ROT_TEAM_WARPS, take the next large
      // blocks from the counter; the lead team then splits into teams of
      // ROT_TEAM_WARPS and joins them.  Named barrier 1 is the lead team's, 2.. the
      // other teams', the split teams' after those.
      auto run_block = [&](const SubTeam& tm, int bi) {
        const int trk = tm.rank(), tsz = tm.size();
        const int w0 = tm.base >> 5, nw = tsz >> 5, twarp = warp - w0;
        const int b = s_ord[bi];
        const NewBlk B = nb[b];
        const bool trans = B.nc > B.nr;
        const int m = trans ? B.nc : B.nr, n = trans ? B.nr : B.nc;
        double* Bm = D.bbuf + B.wofs;
        double* W = D.wbuf + B.wofs;
        float* W32 = D.w32 + B.wofs;
        double* Q = D.qbuf + B.qofs;
        double* T = D.tbuf + B.qofs;
        float* Q32 = D.q32 + B.qofs;
        double mx = 0.0;
        for (int idx = trk; idx < m * n; idx += tsz) {
          const int wi = idx % m, wj = idx / m;
          const int br = trans ? wj : wi, bc = trans ? wi : wj;
          int k1p = 3, k2p = 3;
          while (k1p > 0 && (B.rowsec[k1p] < 0 || B.rowoff[k1p] > br)) --k1p;
          while (k2p > 0 && (B.colsec[k2p] < 0 || B.coloff[k2p] > bc)) --k2p;
          const int sL = B.rowsec[k1p], sR = B.colsec[k2p];
          const int l = secL.off[sL] + (br - B.rowoff[k1p]);
          const int r = secR.off[sR] + (bc - B.coloff[k2p]);
          const int Kp = k1p * 4 + k2p;
          double acc = 0.0;
          for (int e = 0; e < gnz_n[Kp]; ++e) {
            const int K = gnz_k[Kp][e];
            const int k1 = K >> 2, k2 = K & 3;
            const int qM = qadd(secL.q[sL], local_charge(k1));
            if (qM < 0 || lutM[qM] < 0) continue;
            acc = fma(gnz_v[Kp][e], D.theta[(((size_t)l * 4 + k1) * 4 + k2) * chr + r], acc);
          }
          Bm[idx] = acc;
          mx = fmax(mx, fabs(acc));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) s_red[warp] = mx;
        tm.sync();
        double bmax = 0.0;
        for (int w2 = 0; w2 < nw; ++w2) bmax = fmax(bmax, s_red[w0 + w2]);
        const double scale = bmax > 0.0 ? bmax : 1.0;
        const double inv = 1.0 / scale;
        for (int idx = trk; idx < m * n; idx += tsz) Bm[idx] *= inv;
        if (trk == 0) nb[b].scale = scale;
        tm.sync();
        const int ncv = block_svd(tm, Bm, W, Q, W32, Q32, T, m, n, D.max_sweeps);
        if (ncv && trk == 0) atomicOr(&s_status, STATUS_NOCONV | (min(m, 4095) << 8) | (min(n, 4095) << 20));
        for (int j = twarp; j < n; j += nw) {
          double acc = 0.0;
          for (int u = lane; u < m; u += 32) {
            const double v = W[(size_t)j * m + u];
            acc = fma(v, v, acc);
          }
          acc = warp_sum(acc);
          if (lane == 0) sig[B.sofs + j] = sqrt(acc) * scale;
        }
      };
      int slot, base, nthr, bar;
      if (warp < ROT_LEAD_WARPS) {
        slot = 0;
        base = 0;
        nthr = ROT_LEAD_WARPS * 32;
        bar = 1;
      } else {
        const int t = (warp - ROT_LEAD_WARPS) / ROT_TEAM_WARPS;
        slot = 1 + t;
        base = ROT_LEAD_WARPS * 32 + t * ROT_TEAM_THREADS;
        nthr = ROT_TEAM_THREADS;
        bar = 2 + t;
      }
      if (slot == 0) {
        if (nbig > 0) run_block(SubTeam{base, nthr, bar, &s_tscr[slot]}, 0);
        const int t = warp / ROT_TEAM_WARPS;
        slot = 1 + ROT_REST_TEAMS + t;
        base = t * ROT_TEAM_THREADS;
        nthr = ROT_TEAM_THREADS;
        bar = 2 + ROT_REST_TEAMS + t;
      }
      const SubTeam tm{base, nthr, bar, &s_tscr[slot]};
      for (;;) {
        if (tm.rank() == 0) s_tbi[slot] = atomicAdd(&s_next_big, 1);
        tm.sync();
        const int bi = s_tbi[slot];
        tm.sync();
        if (bi >= nbig) break;
        run_block(tm, bi);
      }
    }
    const WarpTeam wt;
    for (;;) {
      int bi = 0;
      if (lane == 0) bi = atomicAdd(&s_next_small, 1);
      bi = __shfl_sync(0xffffffffu, bi, 0) + nbig;
      if (bi >= nnew) break;
      const int b = s_ord[bi];
      const NewBlk B = nb[b];
      const bool trans = B.nc > B.nr;                // work on B^T so that n <= m
      const int m = trans ? B.nc : B.nr, n = trans ? B.nr : B.nc;
      double* Bm = D.bbuf + B.wofs;
      double* W = D.wbuf + B.wofs;
      float* W32 = D.w32 + B.wofs;
      double* Q = D.qbuf + B.qofs;
      double* T = D.tbuf + B.qofs;
      float* Q32 = D.q32 + B.qofs;
      double mx = 0.0;
      for (int idx = lane; idx < m * n; idx += 32) {
        const int wi = idx % m, wj = idx / m;
        const int br = trans ? wj : wi, bc = trans ? wi : wj;
        int k1p = 3, k2p = 3;
        while (k1p > 0 && (B.rowsec[k1p] < 0 || B.rowoff[k1p] > br)) --k1p;
        while (k2p > 0 && (B.colsec[k2p] < 0 || B.coloff[k2p] > bc)) --k2p;
        const int sL = B.rowsec[k1p], sR = B.colsec[k2p];
        const int l = secL.off[sL] + (br - B.rowoff[k1p]);
        const int r = secR.off[sR] + (bc - B.coloff[k2p]);
        const int Kp = k1p * 4 + k2p;
        double acc = 0.0;
        for (int e = 0; e < gnz_n[Kp]; ++e) {
          const int K = gnz_k[Kp][e];
          const int k1 = K >> 2, k2 = K & 3;
          const int qM = qadd(secL.q[sL], local_charge(k1));
          if (qM < 0 || lutM[qM] < 0) continue;       // that theta block is zero
          acc = fma(gnz_v[Kp][e], D.theta[(((size_t)l * 4 + k1) * 4 + k2) * chr + r], acc);
        }
        Bm[idx] = acc;
        mx = fmax(mx, fabs(acc));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const double scale = mx > 0.0 ? mx : 1.0;
      const double inv = 1.0 / scale;
      __syncwarp();
      for (int idx = lane; idx < m * n; idx += 32) Bm[idx] *= inv;
      if (lane == 0) nb[b].scale = scale;
      __syncwarp();
      const int ncv = block_svd(wt, Bm, W, Q, W32, Q32, T, m, n, D.max_sweeps);
      if (ncv && lane == 0) atomicOr(&s_status, STATUS_NOCONV | (min(m, 4095) << 8) | (min(n, 4095) << 20));
      for (int j = 0; j < n; ++j) {
        double acc = 0.0;
        for (int u = lane; u < m; u += 32) {
          const double v = W[(size_t)j * m + u];
          acc = fma(v, v, acc);
        }
        acc = warp_sum(acc);
        if (lane == 0) sig[B.sofs + j] = sqrt(acc) * scale;
      }
    }
    __syncthreads();
    // ---- global truncation: k = min(chi_rot, #{sigma > cutoff sigma_1}), at least 1
    const int nsig = s_nsig;
    if (warp == 0) {
      double smax = 0.0;
      for (int x = lane; x < nsig; x += 32) smax = fmax(smax, sig[x]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
      const double thr = D.cutoff * smax;
      int above = 0;
      for (int x = lane; x < nsig; x += 32) above += (sig[x] > thr) ? 1 : 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) above += __shfl_xor_sync(0xffffffffu, above, o);
      if (lane == 0) {
        int keep = above < D.chi_rot ? above : D.chi_rot;
        if (keep > D.work_cap[a + 1]) keep = D.work_cap[a + 1];
        if (keep < 1) keep = 1;
        if (keep > nsig) keep = nsig;
        s_keep = keep;
      }
    }
    __syncthreads();
    {
      // rank of each singular value (ties by index).  The values are non-negative
      // (+0 or more), and for those the IEEE encodings, read as signed 64-bit
      // integers, are in numeric order: the comparisons run on the integer units.
      const long long* sk = reinterpret_cast<const long long*>(sig);
      for (int x = tid; x < nsig; x += RT_THREADS) {
        const long long v = sk[x];
        int rank = 0;
        for (int y = 0; y < nsig; ++y) {
          const long long u = sk[y];
          rank += (u > v || (u == v && y < x)) ? 1 : 0;
        }
        sig_keep[x] = rank < s_keep ? 1 : 0;
      }
    }
    __syncthreads();
    if (tid == 0) {
      double disc = 0.0;
      for (int x = 0; x < nsig; ++x)
        if (!sig_keep[x]) disc += sig[x] * sig[x];
      s_disc += disc;
      int off = 0;
      SectorTable& nt = secM;                       // reuse as the new middle table
      nt.nsec = 0;
      for (int b = 0; b < nnew; ++b) {
        int kept = 0;
        for (int j = 0; j < (nb[b].nr < nb[b].nc ? nb[b].nr : nb[b].nc); ++j) kept += sig_keep[nb[b].sofs + j];
        nb[b].kept = kept;
        nb[b].newoff = off;
        if (kept > 0) {
          nt.q[nt.nsec] = nb[b].q;
          nt.off[nt.nsec] = off;
          nt.dim[nt.nsec] = kept;
          ++nt.nsec;
        }
        off += kept;
      }
      D.work_dims[a + 1] = off;
    }
    __syncthreads();
    {
      constexpr int W4 = (int)(sizeof(SectorTable) / 4);
      const int* srcp = reinterpret_cast<const int*>(&secM);
      int* dst = reinterpret_cast<int*>(D.work_sec + a + 1);
      for (int x = tid; x < W4; x += RT_THREADS) dst[x] = srcp[x];
    }
    // ---- write the two new site tensors
    const int knew = D.work_dims[a + 1];
    for (long long x = tid; x < (long long)chl * 4 * knew; x += RT_THREADS) Lt[x] = 0.0;
    for (long long x = tid; x < (long long)knew * 4 * chr; x += RT_THREADS) Rt[x] = 0.0;
    __syncthreads();
    for (int b = warp; b < nnew; b += RT_WARPS) {
      const NewBlk B = nb[b];
      if (B.kept == 0) continue;
      const bool trans = B.nc > B.nr;
      const int m = trans ? B.nc : B.nr, n = trans ? B.nr : B.nc;
      const double* W = D.wbuf + B.wofs;
      const double* Q = D.qbuf + B.qofs;
      const double bs = B.scale;
      int newidx = B.newoff;
      for (int j = 0; j < n; ++j) {
        if (!sig_keep[B.sofs + j]) continue;
        const double sj = sig[B.sofs + j];
        const double inv = sj > 0.0 ? 1.0 / sj : 0.0;
        // left factor column over block rows (l, k1'), right factor row over block cols (k2', r)
        for (int br = lane; br < B.nr; br += 32) {
          int k1p = 3;
          while (k1p > 0 && (B.rowsec[k1p] < 0 || B.rowoff[k1p] > br)) --k1p;
          const int l = secL.off[B.rowsec[k1p]] + (br - B.rowoff[k1p]);
          double v;
          if (!trans) v = (side == 0) ? W[(size_t)j * m + br] * bs : W[(size_t)j * m + br] * bs * inv;
          else v = (side == 0) ? Q[(size_t)j * n + br] * sj : Q[(size_t)j * n + br];
          Lt[((size_t)l * 4 + k1p) * knew + newidx] = v;
        }
        for (int bc = lane; bc < B.nc; bc += 32) {
          int k2p = 3;
          while (k2p > 0 && (B.colsec[k2p] < 0 || B.coloff[k2p] > bc)) --k2p;
          const int r = secR.off[B.colsec[k2p]] + (bc - B.coloff[k2p]);
          double v;
          if (!trans) v = (side == 0) ? Q[(size_t)j * n + bc] : Q[(size_t)j * n + bc] * sj;
          else v = (side == 0) ? W[(size_t)j * m + bc] * bs * inv : W[(size_t)j * m + bc] * bs;
          Rt[((size_t)newidx * 4 + k2p) * chr + r] = v;
        }
        ++newidx;
      }
    }
    __syncthreads();
  }

  // ---- G(D): the orbital of a -1 diagonal entry flips both spins' creators
  if (D.neg_site >= 0) {
    const int s = D.neg_site;
    double* T = D.work + D.work_off[s];
    const int cl = D.work_dims[s], cr = D.work_dims[s + 1];
    for (long long x = tid; x < (long long)cl * 4 * cr; x += RT_THREADS) {
      const int k = (int)((x / cr) % 4);
      if (k == 1 || k == 2) T[x] = -T[x];
    }
    __syncthreads();
  }
  // ---- optional renormalisation to the input norm (the centre holds the norm)
  if (D.renorm && D.ngates > 0) {
    const int lastg = D.ngates - 1;
    const int c = D.gate_site[lastg] + (D.gate_side[lastg] ? 1 : 0);
    double* T = D.work + D.work_off[c];
    const long long n = (long long)D.work_dims[c] * 4 * D.work_dims[c + 1];
    const double* S0 = D.src + D.src_off[N - 1];
    const long long n0 = (long long)D.src_dims[N - 1] * 4;
    double a1 = 0.0, a0 = 0.0;
    for (long long x = tid; x < n; x += RT_THREADS) a1 = fma(T[x], T[x], a1);
    for (long long x = tid; x < n0; x += RT_THREADS) a0 = fma(S0[x], S0[x], a0);
    a1 = warp_sum(a1);
    a0 = warp_sum(a0);
    __shared__ double r1[RT_WARPS], r0[RT_WARPS];
    if (lane == 0) {
      r1[warp] = a1;
      r0[warp] = a0;
    }
    __syncthreads();
    double t1 = 0.0, t0 = 0.0;
    for (int w = 0; w < RT_WARPS; ++w) {
      t1 += r1[w];
      t0 += r0[w];
    }
    const double f = t1 > 0.0 ? sqrt(t0 / t1) : 1.0;
    for (long long x = tid; x < n; x += RT_THREADS) T[x] *= f;
  }
  // ---- optional capacity layout: site s becomes [cap_s][4][cap_{s+1}] with zeros
  // beyond the kept dimensions (staged through the theta scratch, which the host
  // sizes to hold any one site at capacity)
  if (D.pad_out) {
    __syncthreads();
    for (int s = 0; s < N; ++s) {
      const int cl = D.work_dims[s], cr = D.work_dims[s + 1];
      const int Cl = D.work_cap[s], Cr = D.work_cap[s + 1];
      if (cl == Cl && cr == Cr) continue;
      double* T = D.work + D.work_off[s];
      const long long n = (long long)cl * 4 * cr;
      for (long long x = tid; x < n; x += RT_THREADS) D.theta[x] = T[x];
      __syncthreads();
      const long long np = (long long)Cl * 4 * Cr;
      for (long long x = tid; x < np; x += RT_THREADS) {
        const int r = (int)(x % Cr);
        const long long lk = x / Cr;
        const int l = (int)(lk / 4), k = (int)(lk % 4);
        T[x] = (l < cl && r < cr) ? D.theta[((long long)l * 4 + k) * cr + r] : 0.0;
      }
      __syncthreads();
    }
  }
  if (tid == 0) {
    *D.discarded = s_disc;
    *D.status = s_status;
    *D.flops = s_flops;
  }
}



}  // namespace

int launch_rotate(const RotDesc* d_descs, int npairs, int smem_bytes, void* stream) {
  if (npairs <= 0) return 0;
  (void)smem_bytes;
  // The highest launch priority: each CTA needs a whole SM's register file, so
  // its CTAs must take their SMs before the kernels of a concurrent stream do.
  int lo = 0, hi = 0;
  cudaDeviceGetStreamPriorityRange(&lo, &hi);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)npairs);
  cfg.blockDim = dim3(RotWide::threads);
  cfg.stream = (cudaStream_t)stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributePriority;
  attr[0].val.priority = hi;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, rotate_pairs_kernel<RotWide>, d_descs);
  if (e != cudaSuccess) return (int)e;
  return (int)cudaGetLastError();
}

}  // namespace tnqe

// =============================================================================
// One Givens gate with scratch in a static device array (no allocation).
//
// For callers that cannot call cudaMalloc: host programs whose device memory
// is fully reserved up front by their own pool (a library allocation would
// fail or fragment it), and host code that must not pay the latency and
// implicit synchronisation of cudaMalloc / cudaFree inside a time-critical
// loop.  The call itself synchronises its stream (it reads the result header
// back).  The caller passes device buffers for the
// inputs and outputs; all intermediate storage of the step (two-site tensor,
// SVD blocks, block bookkeeping) lives in tnqe_gate_scratch below, which
// every GPU that loads this library holds until the process exits.
// =============================================================================

#include <cstdio>
#include <cstring>
#include <mutex>

#include <cuda.h>

#include "../../include/tnqe.h"

namespace tnqe {
namespace {

constexpr int NA_CHI = TNQE_NOALLOC_MAX_CHI;
constexpr size_t NA_HDR_BYTES = 16384;
constexpr size_t NA_META_INTS = 65536;
constexpr size_t NA_BLOCK_DOUBLES = 16ull * NA_CHI * NA_CHI;   // theta, block matrices, block rotations

struct NaHeader {
  SectorTable secL, secM, secR, secOut;
  double G[256];
  const double* A;
  const double* B;
  double* Aout;
  double* Bout;
  double cutoff;
  double disc;
  int chl, chm, chr, chi_max, side, max_sweeps;
  int k_out, status;
};
static_assert(sizeof(NaHeader) <= NA_HDR_BYTES, "header does not fit");
static_assert(NA_HDR_BYTES + NA_META_INTS * 4 + 3 * NA_BLOCK_DOUBLES * 8 == TNQE_NOALLOC_SCRATCH_BYTES,
              "scratch layout and TNQE_NOALLOC_SCRATCH_BYTES disagree");

}  // namespace

// The scratch of tnqe_apply_gate_noalloc.  Host code may only use its address
// as resolved by cudaGetSymbolAddress on the current device (gate_scratch_ptr).
static __device__ __align__(256) unsigned char tnqe_gate_scratch[TNQE_NOALLOC_SCRATCH_BYTES];

namespace {

__global__ void __launch_bounds__(ROT_THREADS) gate_static_kernel(unsigned char* __restrict__ scratch) {
  NaHeader& H = *reinterpret_cast<NaHeader*>(scratch);
  int* meta = reinterpret_cast<int*>(scratch + NA_HDR_BYTES);
  double* theta = reinterpret_cast<double*>(scratch + NA_HDR_BYTES + NA_META_INTS * 4);
  double* wbuf = theta + NA_BLOCK_DOUBLES;
  double* qbuf = wbuf + NA_BLOCK_DOUBLES;
  const int tid = threadIdx.x;
  ThetaBlk* tb = reinterpret_cast<ThetaBlk*>(meta);
  const long long tb_cap = (long long)NA_META_INTS / 2 / (long long)(sizeof(ThetaBlk) / sizeof(int));
  NewBlk* nb = reinterpret_cast<NewBlk*>(meta + NA_META_INTS / 2);
  const long long nb_cap = (long long)NA_META_INTS / 2 / (long long)(sizeof(NewBlk) / sizeof(int));

  __shared__ int lutL[QSPACE], lutM[QSPACE], lutR[QSPACE];
  __shared__ int gnz_n[16], gnz_k[16][16];
  __shared__ double gnz_v[16][16];
  __shared__ double sig[MAXSIG];
  __shared__ unsigned char sig_keep[MAXSIG];
  __shared__ int s_nblk, s_nnew, s_total, s_nsig, s_keep, s_flag, s_status;
  __shared__ double s_red[ROT_WARPS];

  const SectorTable& secL = H.secL;
  const SectorTable& secM = H.secM;
  const SectorTable& secR = H.secR;
  const int chl = H.chl, chm = H.chm, chr = H.chr, side = H.side;
  const double* Lt = H.A;
  const double* Rt = H.B;
  for (int x = tid; x < QSPACE; x += ROT_THREADS) {
    lutL[x] = -1;
    lutM[x] = -1;
    lutR[x] = -1;
  }
  if (tid == 0) s_status = 0;
  __syncthreads();
  for (int x = tid; x < secL.nsec; x += ROT_THREADS) lutL[secL.q[x]] = x;
  for (int x = tid; x < secM.nsec; x += ROT_THREADS) lutM[secM.q[x]] = x;
  for (int x = tid; x < secR.nsec; x += ROT_THREADS) lutR[secR.q[x]] = x;
  if (tid < 16) {
    int c = 0;
    for (int K = 0; K < 16; ++K) {
      const double v = H.G[tid * 16 + K];
      if (v != 0.0) {
        gnz_k[tid][c] = K;
        gnz_v[tid][c] = v;
        ++c;
      }
    }
    gnz_n[tid] = c;
  }
  __syncthreads();
  // two-site tensor, charge-allowed blocks only
  if (tid == 0) {
    int nblk = 0, start = 0;
    for (int sL = 0; sL < secL.nsec; ++sL)
      for (int k1 = 0; k1 < 4; ++k1) {
        const int qM = qadd(secL.q[sL], local_charge(k1));
        const int sM = qM < 0 ? -1 : lutM[qM];
        if (sM < 0) continue;
        for (int k2 = 0; k2 < 4; ++k2) {
          const int qR = qadd(qM, local_charge(k2));
          const int sR = qR < 0 ? -1 : lutR[qR];
          if (sR < 0) continue;
          if (nblk < tb_cap) tb[nblk] = ThetaBlk{sL, sM, sR, k1, k2, start};
          ++nblk;
          start += secL.dim[sL] * secR.dim[sR];
        }
      }
    if (nblk > tb_cap) {
      s_status |= STATUS_OVERFLOW;
      nblk = (int)tb_cap;
    }
    s_nblk = nblk;
    s_total = start;
  }
  __syncthreads();
  for (int idx = tid; idx < s_total; idx += ROT_THREADS) {
    int lo = 0, hi = s_nblk - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tb[mid].start <= idx) lo = mid; else hi = mid - 1;
    }
    const ThetaBlk B = tb[lo];
    const int dR = secR.dim[B.sR];
    const int l = secL.off[B.sL] + (idx - B.start) / dR, r = secR.off[B.sR] + (idx - B.start) % dR;
    const int m0 = secM.off[B.sM], m1 = m0 + secM.dim[B.sM];
    const double* lrow = Lt + ((size_t)l * 4 + B.k1) * chm;
    const double* rcol = Rt + (size_t)B.k2 * chr + r;
    double acc = 0.0;
    for (int m = m0; m < m1; ++m) acc = fma(lrow[m], rcol[(size_t)m * 4 * chr], acc);
    theta[(((size_t)l * 4 + B.k1) * 4 + B.k2) * chr + r] = acc;
  }
  // blocks of the new middle bond
  if (tid == 0) {
    int nnew = 0, nsig = 0;
    long long wofs = 0, qofs = 0;
    for (int q = 0; q < QSPACE; ++q) {
      NewBlk B;
      B.q = q;
      int nr = 0, nc = 0;
      for (int k = 0; k < 4; ++k) {
        const int qL = qsub(q, local_charge(k));
        const int sL = qL < 0 ? -1 : lutL[qL];
        B.rowsec[k] = sL;
        B.rowoff[k] = nr;
        if (sL >= 0) nr += secL.dim[sL];
        const int qR = qadd(q, local_charge(k));
        const int sR = qR < 0 ? -1 : lutR[qR];
        B.colsec[k] = sR;
        B.coloff[k] = nc;
        if (sR >= 0) nc += secR.dim[sR];
      }
      if (nr == 0 || nc == 0) continue;
      B.nr = nr;
      B.nc = nc;
      const int mm = nr > nc ? nr : nc, nn = nr > nc ? nc : nr;
      B.wofs = wofs;
      B.qofs = qofs;
      B.sofs = nsig;
      B.kept = 0;
      B.newoff = 0;
      B.scale = 1.0;
      wofs += (long long)mm * nn;
      qofs += (long long)nn * nn;
      nsig += nn;
      if (nnew < nb_cap && nsig <= MAXSIG) nb[nnew] = B;
      ++nnew;
    }
    if (nnew > nb_cap || nsig > MAXSIG) {
      s_status |= STATUS_OVERFLOW;
      nnew = 0;
      nsig = 0;
    }
    s_nnew = nnew;
    s_nsig = nsig;
  }
  __syncthreads();
  const int nnew = s_nnew;
  for (int b = 0; b < nnew; ++b) {
    const NewBlk B = nb[b];
    const bool trans = B.nc > B.nr;
    const int m = trans ? B.nc : B.nr, n = trans ? B.nr : B.nc;
    double* W = wbuf + B.wofs;
    double* Q = qbuf + B.qofs;
    for (int idx = tid; idx < m * n; idx += ROT_THREADS) {
      const int wi = idx % m, wj = idx / m;
      const int br = trans ? wj : wi, bc = trans ? wi : wj;
      int k1p = 3, k2p = 3;
      while (k1p > 0 && (B.rowsec[k1p] < 0 || B.rowoff[k1p] > br)) --k1p;
      while (k2p > 0 && (B.colsec[k2p] < 0 || B.coloff[k2p] > bc)) --k2p;
      const int sL = B.rowsec[k1p], sR = B.colsec[k2p];
      const int l = secL.off[sL] + (br - B.rowoff[k1p]);
      const int r = secR.off[sR] + (bc - B.coloff[k2p]);
      const int Kp = k1p * 4 + k2p;
      double acc = 0.0;
      for (int e = 0; e < gnz_n[Kp]; ++e) {
        const int K = gnz_k[Kp][e];
        const int k1 = K >> 2, k2 = K & 3;
        const int qM = qadd(secL.q[sL], local_charge(k1));
        if (qM < 0 || lutM[qM] < 0) continue;
        acc = fma(gnz_v[Kp][e], theta[(((size_t)l * 4 + k1) * 4 + k2) * chr + r], acc);
      }
      W[idx] = acc;
    }
    __syncthreads();
    double mx = 0.0;
    for (int idx = tid; idx < m * n; idx += ROT_THREADS) mx = fmax(mx, fabs(W[idx]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((tid & 31) == 0) s_red[tid >> 5] = mx;
    __syncthreads();
    double bmax = 0.0;
    for (int w = 0; w < ROT_WARPS; ++w) bmax = fmax(bmax, s_red[w]);
    const double scale = bmax > 0.0 ? bmax : 1.0;
    for (int idx = tid; idx < m * n; idx += ROT_THREADS) W[idx] *= 1.0 / scale;
    if (tid == 0) nb[b].scale = scale;
    __syncthreads();
    if (jacobi_block(W, Q, m, n, H.max_sweeps, &s_flag) && tid == 0) s_status |= STATUS_NOCONV;
    for (int j = 0; j < n; ++j) {
      double acc = 0.0;
      for (int u = tid; u < m; u += ROT_THREADS) acc = fma(W[(size_t)j * m + u], W[(size_t)j * m + u], acc);
      acc = warp_sum(acc);
      if ((tid & 31) == 0) s_red[tid >> 5] = acc;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < ROT_WARPS; ++w) t += s_red[w];
        sig[B.sofs + j] = sqrt(t) * scale;
      }
      __syncthreads();
    }
  }
  // truncation: k = min(chi_max, #{sigma > cutoff sigma_1}), at least 1
  const int nsig = s_nsig;
  if (tid == 0) {
    double smax = 0.0;
    for (int x = 0; x < nsig; ++x) smax = fmax(smax, sig[x]);
    int above = 0;
    for (int x = 0; x < nsig; ++x) above += (sig[x] > H.cutoff * smax) ? 1 : 0;
    int keep = above < H.chi_max ? above : H.chi_max;
    if (keep < 1) keep = 1;
    if (keep > nsig) keep = nsig;
    s_keep = keep;
  }
  __syncthreads();
  for (int x = tid; x < nsig; x += ROT_THREADS) {
    const double v = sig[x];
    int rank = 0;
    for (int y = 0; y < nsig; ++y) rank += (sig[y] > v || (sig[y] == v && y < x)) ? 1 : 0;
    sig_keep[x] = rank < s_keep ? 1 : 0;
  }
  __syncthreads();
  if (tid == 0) {
    double disc = 0.0;
    for (int x = 0; x < nsig; ++x)
      if (!sig_keep[x]) disc += sig[x] * sig[x];
    H.disc = disc;
    int off = 0;
    SectorTable& nt = H.secOut;
    nt.nsec = 0;
    for (int b = 0; b < nnew; ++b) {
      int kept = 0;
      for (int j = 0; j < (nb[b].nr < nb[b].nc ? nb[b].nr : nb[b].nc); ++j) kept += sig_keep[nb[b].sofs + j];
      nb[b].kept = kept;
      nb[b].newoff = off;
      if (kept > 0) {
        nt.q[nt.nsec] = nb[b].q;
        nt.off[nt.nsec] = off;
        nt.dim[nt.nsec] = kept;
        ++nt.nsec;
      }
      off += kept;
    }
    H.k_out = off;
  }
  __syncthreads();
  const int knew = H.k_out;
  double* Ao = H.Aout;
  double* Bo = H.Bout;
  for (long long x = tid; x < (long long)chl * 4 * knew; x += ROT_THREADS) Ao[x] = 0.0;
  for (long long x = tid; x < (long long)knew * 4 * chr; x += ROT_THREADS) Bo[x] = 0.0;
  __syncthreads();
  for (int b = 0; b < nnew; ++b) {
    const NewBlk B = nb[b];
    if (B.kept == 0) continue;
    const bool trans = B.nc > B.nr;
    const int m = trans ? B.nc : B.nr, n = trans ? B.nr : B.nc;
    const double* W = wbuf + B.wofs;
    const double* Q = qbuf + B.qofs;
    const double bs = B.scale;
    int newidx = B.newoff;
    for (int j = 0; j < n; ++j) {
      if (!sig_keep[B.sofs + j]) continue;
      const double sj = sig[B.sofs + j];
      const double inv = sj > 0.0 ? 1.0 / sj : 0.0;
      for (int br = tid; br < B.nr; br += ROT_THREADS) {
        int k1p = 3;
        while (k1p > 0 && (B.rowsec[k1p] < 0 || B.rowoff[k1p] > br)) --k1p;
        const int l = secL.off[B.rowsec[k1p]] + (br - B.rowoff[k1p]);
        double v;
        if (!trans) v = (side == 0) ? W[(size_t)j * m + br] * bs : W[(size_t)j * m + br] * bs * inv;
        else v = (side == 0) ? Q[(size_t)j * n + br] * sj : Q[(size_t)j * n + br];
        Ao[((size_t)l * 4 + k1p) * knew + newidx] = v;
      }
      for (int bc = tid; bc < B.nc; bc += ROT_THREADS) {
        int k2p = 3;
        while (k2p > 0 && (B.colsec[k2p] < 0 || B.coloff[k2p] > bc)) --k2p;
        const int r = secR.off[B.colsec[k2p]] + (bc - B.coloff[k2p]);
        double v;
        if (!trans) v = (side == 0) ? Q[(size_t)j * n + bc] : Q[(size_t)j * n + bc] * sj;
        else v = (side == 0) ? W[(size_t)j * m + bc] * bs * inv : W[(size_t)j * m + bc] * bs;
        Bo[((size_t)newidx * 4 + k2p) * chr + r] = v;
      }
      ++newidx;
    }
  }
  if (tid == 0) H.status = s_status;
}

constexpr int NA_MAX_DEVICES = 64;
std::mutex na_mutex;
void* na_ptr[NA_MAX_DEVICES] = {nullptr};
CUcontext na_ctx[NA_MAX_DEVICES] = {nullptr};

// The CUDA context current on the calling thread (driver entry point looked up once).
cudaError_t current_context(CUcontext* out) {
  static CUresult (*get)(CUcontext*) = nullptr;
  if (!get) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !p) return cudaErrorNotSupported;
    get = reinterpret_cast<CUresult (*)(CUcontext*)>(p);
  }
  return get(out) == CUDA_SUCCESS ? cudaSuccess : cudaErrorDeviceUninitialized;
}

// Device address of tnqe_gate_scratch on the current device.  Set up once per
// device and context: a device reset gives the device a new primary context
// (and the module a new load), so the address is looked up again then.
cudaError_t gate_scratch_ptr(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
  CUcontext ctx = nullptr;
  e = current_context(&ctx);                               // NULL before the runtime's first use of the device
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(na_mutex);
  if (!ctx || !na_ptr[dev] || na_ctx[dev] != ctx) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, tnqe_gate_scratch);      // also makes the primary context current
    if (e != cudaSuccess) return e;
    e = current_context(&ctx);
    if (e != cudaSuccess) return e;
    na_ptr[dev] = p;
    na_ctx[dev] = ctx;
  }
  *out = static_cast<unsigned char*>(na_ptr[dev]);
  return cudaSuccess;
}

bool na_sectors(const int* q, int n, SectorTable& T) {
  T.nsec = 0;
  for (int x = 0; x < n; ++x) {
    const int qa = q[x] / QSTRIDE, qb = q[x] % QSTRIDE;
    if (q[x] < 0 || qa >= QSTRIDE - 1 || qb >= QSTRIDE - 1) return false;
    if (x > 0 && q[x] < q[x - 1]) return false;           // indices must be grouped by ascending charge
    if (T.nsec == 0 || T.q[T.nsec - 1] != q[x]) {
      if (T.nsec >= MAXSEC) return false;
      T.q[T.nsec] = q[x];
      T.off[T.nsec] = x;
      T.dim[T.nsec] = 0;
      ++T.nsec;
    }
    ++T.dim[T.nsec - 1];
  }
  return true;
}

tnqe_status na_fail(char* err, int err_len, tnqe_status st, const char* msg) {
  if (err && err_len > 0) {
    std::strncpy(err, msg, (size_t)err_len - 1);
    err[err_len - 1] = '\0';
  }
  return st;
}

}  // namespace
}  // namespace tnqe

extern "C" tnqe_status tnqe_apply_gate_noalloc(const double* A, const double* B, int chi_l, int chi_m, int chi_r,
                                               const int* q_l, const int* q_m, const int* q_r, double c, double s,
                                               int sigma_side, int chi_max, double cutoff, int max_sweeps,
                                               double* A_out, double* B_out, int* q_out, int* k_out,
                                               double* discarded, void* stream, char* err, int err_len) {
  using namespace tnqe;
  if (!A || !B || !A_out || !B_out || !q_l || !q_m || !q_r || !k_out)
    return na_fail(err, err_len, TNQE_ERR_ARG, "null argument");
  if (chi_l < 1 || chi_m < 1 || chi_r < 1 || chi_max < 1 || chi_l > NA_CHI || chi_m > NA_CHI || chi_r > NA_CHI ||
      chi_max > NA_CHI)
    return na_fail(err, err_len, TNQE_ERR_ARG,
                   "bond dimensions must be in [1, TNQE_NOALLOC_MAX_CHI = 128] for the no-allocation gate");
  if (sigma_side != 0 && sigma_side != 1) return na_fail(err, err_len, TNQE_ERR_ARG, "sigma_side must be 0 or 1");
  if (!(cutoff >= 0.0) || max_sweeps < 1) return na_fail(err, err_len, TNQE_ERR_ARG, "bad cutoff or sweep limit");
  NaHeader h;
  std::memset(&h, 0, sizeof(h));
  if (!na_sectors(q_l, chi_l, h.secL) || !na_sectors(q_m, chi_m, h.secM) || !na_sectors(q_r, chi_r, h.secR))
    return na_fail(err, err_len, TNQE_ERR_ARG,
                   "bond charges must be n_alpha*16+n_beta (each below 15) in ascending order");
  gate_matrix(c, s, h.G);
  h.A = A;
  h.B = B;
  h.Aout = A_out;
  h.Bout = B_out;
  h.cutoff = cutoff;
  h.chl = chi_l;
  h.chm = chi_m;
  h.chr = chi_r;
  h.chi_max = chi_max;
  h.side = sigma_side;
  h.max_sweeps = max_sweeps;
  unsigned char* scratch = nullptr;
  cudaError_t e = gate_scratch_ptr(&scratch);
  if (e != cudaSuccess) return na_fail(err, err_len, TNQE_ERR_CUDA, cudaGetErrorString(e));
  cudaStream_t st = (cudaStream_t)stream;
  e = cudaMemcpyAsync(scratch, &h, sizeof(h), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    gate_static_kernel<<<1, ROT_THREADS, 0, st>>>(scratch);
    e = cudaGetLastError();
  }
  NaHeader r;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&r, scratch, sizeof(r), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return na_fail(err, err_len, TNQE_ERR_CUDA, cudaGetErrorString(e));
  *k_out = r.k_out;
  if (discarded) *discarded = r.disc;
  if (q_out)
    for (int t = 0; t < r.secOut.nsec; ++t)
      for (int x = 0; x < r.secOut.dim[t]; ++x) q_out[r.secOut.off[t] + x] = r.secOut.q[t];
  if (r.status & STATUS_OVERFLOW) return na_fail(err, err_len, TNQE_ERR_STATE, "gate bookkeeping overflow");
  if (r.status & STATUS_NOCONV)
    return na_fail(err, err_len, TNQE_ERR_NOCONV, "Jacobi SVD hit the sweep limit (outputs written)");
  return na_fail(err, err_len, TNQE_OK, "");
}
