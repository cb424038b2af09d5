// Rotation-proposal network (include/tnqe_mlp.h): forward, backward and Adam
// kernels in FP32 on CUDA cores.  The network is small (tens of thousands of
// parameters, batches of a few thousand rows), so every product is one tiled
// GEMM launch and the work is latency-bound rather than tensor-core shaped.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/tnqe_mlp.h"

namespace {

constexpr int GT = 16;   // GEMM tile edge

// C[M][N] (ldc) = sum_k op(A)[m][k] op(B)[k][n] (+ C if accumulate), then + bias[n] if bias.
// op(A) = A (M x K, lda) or A^T (A stored K x M); op(B) = B (K x N, ldb) or B^T (B stored N x K).
__global__ void gemm_f32(const float* __restrict__ A, const float* __restrict__ B, float* __restrict__ C, int M, int N,
                         int K, int lda, int ldb, int ldc, int transA, int transB, const float* __restrict__ bias,
                         int accumulate) {
  __shared__ float As[GT][GT + 1];
  __shared__ float Bs[GT][GT + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int m = blockIdx.y * GT + ty, n = blockIdx.x * GT + tx;
  float acc = 0.f;
  for (int k0 = 0; k0 < K; k0 += GT) {
    {
      const int am = blockIdx.y * GT + ty, ak = k0 + tx;   // As[ty][tx] = op(A)[am][ak]
      float v = 0.f;
      if (am < M && ak < K) v = transA ? A[(long long)ak * lda + am] : A[(long long)am * lda + ak];
      As[ty][tx] = v;
      const int bk = k0 + ty, bn = blockIdx.x * GT + tx;   // Bs[ty][tx] = op(B)[bk][bn]
      float u = 0.f;
      if (bk < K && bn < N) u = transB ? B[(long long)bn * ldb + bk] : B[(long long)bk * ldb + bn];
      Bs[ty][tx] = u;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GT; ++kk) acc = fmaf(As[ty][kk], Bs[kk][tx], acc);
    __syncthreads();
  }
  if (m < M && n < N) {
    float* c = C + (long long)m * ldc + n;
    float v = accumulate ? *c + acc : acc;
    if (bias) v += bias[n];
    *c = v;
  }
}

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

__global__ void gelu_kernel(const float* __restrict__ Z, float* __restrict__ A, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) A[i] = gelu_f(Z[i]);
}
// dZ = dA * gelu'(Z)
__global__ void gelu_back_kernel(const float* __restrict__ Z, const float* __restrict__ dA, float* __restrict__ dZ,
                                 long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dZ[i] = dA[i] * gelu_grad(Z[i]);
}
// dY = 2 w_b (Y - T) / (n_out W), per-row weighted squared errors into rowloss[b]
__global__ void loss_kernel(const float* __restrict__ Y, const float* __restrict__ T, const float* __restrict__ w,
                            const float* __restrict__ wsum, float* __restrict__ dY, float* __restrict__ rowloss, int B,
                            int n_out) {
  const int b = blockIdx.x;
  if (b >= B) return;
  const float wb = w ? w[b] : 1.f;
  const float scale = 1.f / (*wsum * (float)n_out);
  float acc = 0.f;
  for (int o = threadIdx.x; o < n_out; o += blockDim.x) {
    const float r = Y[(long long)b * n_out + o] - T[(long long)b * n_out + o];
    dY[(long long)b * n_out + o] = 2.f * wb * r * scale;
    acc += wb * r * r;
  }
  __shared__ float red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) rowloss[b] = red[0] * scale;
}
// out[0] = sum of x[0..n) (one block)
__global__ void sum_kernel(const float* __restrict__ x, int n, float* __restrict__ out, int ones) {
  __shared__ float red[256];
  float acc = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += x ? x[i] : (ones ? 1.f : 0.f);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}
// db[n] = sum_b dZ[b][n]
__global__ void colsum_kernel(const float* __restrict__ dZ, float* __restrict__ db, int B, int N) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float acc = 0.f;
  for (int b = 0; b < B; ++b) acc += dZ[(long long)b * N + n];
  db[n] = acc;
}
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

struct tnqe_mlp {
  int n_in = 0, n_h = 0, n_out = 0, max_batch = 0;
  long long count = 0;
  long long oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  float *P = nullptr, *G = nullptr, *Mo = nullptr, *Vo = nullptr;
  float *X = nullptr, *Z1 = nullptr, *A1 = nullptr, *Z2 = nullptr, *A2 = nullptr, *Y = nullptr;
  float *T = nullptr, *w = nullptr, *dY = nullptr, *dA = nullptr, *dZ = nullptr, *rowloss = nullptr, *scal = nullptr;
  long long step = 0;
  int launches = 0;
  std::string err;
};

namespace {

struct MlpError : std::runtime_error {
  tnqe_status st;
  MlpError(tnqe_status s, const std::string& m) : std::runtime_error(m), st(s) {}
};
void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess)
    throw MlpError(e == cudaErrorMemoryAllocation ? TNQE_ERR_NOMEM : TNQE_ERR_CUDA,
                   std::string(what) + ": " + cudaGetErrorString(e));
}
void launched(tnqe_mlp* n) {
  ++n->launches;
  ck(cudaGetLastError(), "kernel launch");
}
void gemm(tnqe_mlp* n, const float* A, const float* B, float* C, int M, int N, int K, int lda, int ldb, int ldc,
          int tA, int tB, const float* bias, int acc) {
  dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT), block(GT, GT);
  gemm_f32<<<grid, block, 0, n->stream>>>(A, B, C, M, N, K, lda, ldb, ldc, tA, tB, bias, acc);
  launched(n);
}
unsigned blocks(long long x) { return (unsigned)((x + 255) / 256); }

void check_batch(tnqe_mlp* n, const void* X, int batch) {
  if (!X || batch < 1 || batch > n->max_batch) throw MlpError(TNQE_ERR_ARG, "batch must be in [1, max_batch]");
}

void forward(tnqe_mlp* n, int B) {
  const int I = n->n_in, H = n->n_h, O = n->n_out;
  gemm(n, n->X, n->P + n->oW1, n->Z1, B, H, I, I, I, H, 0, 1, n->P + n->ob1, 0);
  gelu_kernel<<<blocks((long long)B * H), 256, 0, n->stream>>>(n->Z1, n->A1, (long long)B * H);
  launched(n);
  gemm(n, n->A1, n->P + n->oW2, n->Z2, B, H, H, H, H, H, 0, 1, n->P + n->ob2, 0);
  gelu_kernel<<<blocks((long long)B * H), 256, 0, n->stream>>>(n->Z2, n->A2, (long long)B * H);
  launched(n);
  gemm(n, n->A2, n->P + n->oW3, n->Y, B, O, H, H, H, O, 0, 1, n->P + n->ob3, 0);
}

// loss into scal[1], gradient into G
void backward(tnqe_mlp* n, int B, bool weighted) {
  const int I = n->n_in, H = n->n_h, O = n->n_out;
  float* wsum = n->scal;
  sum_kernel<<<1, 256, 0, n->stream>>>(weighted ? n->w : nullptr, B, wsum, 1);
  launched(n);
  loss_kernel<<<B, 256, 0, n->stream>>>(n->Y, n->T, weighted ? n->w : nullptr, wsum, n->dY, n->rowloss, B, O);
  launched(n);
  sum_kernel<<<1, 256, 0, n->stream>>>(n->rowloss, B, n->scal + 1, 0);
  launched(n);
  float* G = n->G;
  gemm(n, n->dY, n->A2, G + n->oW3, O, H, B, O, H, H, 1, 0, nullptr, 0);   // dW3 = dY^T A2
  colsum_kernel<<<blocks(O), 256, 0, n->stream>>>(n->dY, G + n->ob3, B, O);
  launched(n);
  gemm(n, n->dY, n->P + n->oW3, n->dA, B, H, O, O, H, H, 0, 0, nullptr, 0);   // dA2 = dY W3
  gelu_back_kernel<<<blocks((long long)B * H), 256, 0, n->stream>>>(n->Z2, n->dA, n->dZ, (long long)B * H);
  launched(n);
  gemm(n, n->dZ, n->A1, G + n->oW2, H, H, B, H, H, H, 1, 0, nullptr, 0);    // dW2 = dZ2^T A1
  colsum_kernel<<<blocks(H), 256, 0, n->stream>>>(n->dZ, G + n->ob2, B, H);
  launched(n);
  gemm(n, n->dZ, n->P + n->oW2, n->dA, B, H, H, H, H, H, 0, 0, nullptr, 0);   // dA1 = dZ2 W2
  gelu_back_kernel<<<blocks((long long)B * H), 256, 0, n->stream>>>(n->Z1, n->dA, n->dZ, (long long)B * H);
  launched(n);
  gemm(n, n->dZ, n->X, G + n->oW1, H, I, B, H, I, I, 1, 0, nullptr, 0);      // dW1 = dZ1^T X
  colsum_kernel<<<blocks(H), 256, 0, n->stream>>>(n->dZ, G + n->ob1, B, H);
  launched(n);
}

void upload_batch(tnqe_mlp* n, const float* X, const float* T, const float* w, int B) {
  ck(cudaMemcpyAsync(n->X, X, sizeof(float) * B * n->n_in, cudaMemcpyHostToDevice, n->stream), "copy X");
  if (T) ck(cudaMemcpyAsync(n->T, T, sizeof(float) * B * n->n_out, cudaMemcpyHostToDevice, n->stream), "copy T");
  if (w) {
    std::vector<float> hw(w, w + B);
    for (float x : hw)
      if (!(x >= 0.f) || !std::isfinite(x)) throw MlpError(TNQE_ERR_ARG, "row weights must be finite and >= 0");
    ck(cudaMemcpyAsync(n->w, w, sizeof(float) * B, cudaMemcpyHostToDevice, n->stream), "copy w");
  }
}

tnqe_status mlp_fail(tnqe_mlp* n, const MlpError& e) {
  if (n) n->err = e.what();
  return e.st;
}

}  // namespace

extern "C" {

tnqe_status tnqe_mlp_create(int n_in, int n_hidden, int n_out, int max_batch, void* stream, tnqe_mlp** out) {
  if (!out) return TNQE_ERR_ARG;
  *out = nullptr;
  if (n_in < 1 || n_hidden < 1 || n_out < 1 || n_in > 4096 || n_hidden > 4096 || n_out > 4096 || max_batch < 1 ||
      max_batch > 65536)
    return TNQE_ERR_ARG;
  tnqe_mlp* n = new tnqe_mlp();
  try {
    n->n_in = n_in;
    n->n_h = n_hidden;
    n->n_out = n_out;
    n->max_batch = max_batch;
    const long long I = n_in, H = n_hidden, O = n_out;
    n->oW1 = 0;
    n->ob1 = H * I;
    n->oW2 = n->ob1 + H;
    n->ob2 = n->oW2 + H * H;
    n->oW3 = n->ob2 + H;
    n->ob3 = n->oW3 + O * H;
    n->count = n->ob3 + O;
    if (stream) {
      n->stream = (cudaStream_t)stream;
    } else {
      ck(cudaStreamCreateWithFlags(&n->stream, cudaStreamNonBlocking), "stream");
      n->own_stream = true;
    }
    auto alloc = [&](float** p, long long cnt) {
      ck(cudaMalloc(p, sizeof(float) * (size_t)std::max(1LL, cnt)), "cudaMalloc");
      ck(cudaMemset(*p, 0, sizeof(float) * (size_t)std::max(1LL, cnt)), "cudaMemset");
    };
    const long long B = max_batch;
    alloc(&n->P, n->count);
    alloc(&n->G, n->count);
    alloc(&n->Mo, n->count);
    alloc(&n->Vo, n->count);
    alloc(&n->X, B * I);
    alloc(&n->Z1, B * H);
    alloc(&n->A1, B * H);
    alloc(&n->Z2, B * H);
    alloc(&n->A2, B * H);
    alloc(&n->Y, B * O);
    alloc(&n->T, B * O);
    alloc(&n->w, B);
    alloc(&n->dY, B * O);
    alloc(&n->dA, B * H);
    alloc(&n->dZ, B * H);
    alloc(&n->rowloss, B);
    alloc(&n->scal, 4);
    *out = n;
    return TNQE_OK;
  } catch (const MlpError& e) {
    tnqe_mlp_destroy(n);
    return e.st;
  }
}

long long tnqe_mlp_param_count(const tnqe_mlp* n) { return n ? n->count : 0; }

tnqe_status tnqe_mlp_set_params(tnqe_mlp* n, const float* params) {
  if (!n || !params) return TNQE_ERR_ARG;
  try {
    std::vector<float> h(params, params + n->count);
    for (float x : h)
      if (!std::isfinite(x)) throw MlpError(TNQE_ERR_ARG, "non-finite parameter");
    ck(cudaMemcpyAsync(n->P, h.data(), sizeof(float) * n->count, cudaMemcpyHostToDevice, n->stream), "copy params");
    ck(cudaMemsetAsync(n->Mo, 0, sizeof(float) * n->count, n->stream), "clear m");
    ck(cudaMemsetAsync(n->Vo, 0, sizeof(float) * n->count, n->stream), "clear v");
    ck(cudaStreamSynchronize(n->stream), "sync");
    n->step = 0;
    return TNQE_OK;
  } catch (const MlpError& e) {
    return mlp_fail(n, e);
  }
}

tnqe_status tnqe_mlp_get_params(const tnqe_mlp* n, float* params) {
  if (!n || !params) return TNQE_ERR_ARG;
  if (cudaStreamSynchronize(n->stream) != cudaSuccess) return TNQE_ERR_CUDA;
  if (cudaMemcpy(params, n->P, sizeof(float) * n->count, cudaMemcpyDeviceToHost) != cudaSuccess) return TNQE_ERR_CUDA;
  return TNQE_OK;
}

tnqe_status tnqe_mlp_forward(tnqe_mlp* n, const float* X, int batch, float* Y) {
  if (!n || !Y) return TNQE_ERR_ARG;
  try {
    check_batch(n, X, batch);
    n->launches = 0;
    upload_batch(n, X, nullptr, nullptr, batch);
    forward(n, batch);
    ck(cudaMemcpyAsync(Y, n->Y, sizeof(float) * batch * n->n_out, cudaMemcpyDeviceToHost, n->stream), "copy Y");
    ck(cudaStreamSynchronize(n->stream), "sync");
    return TNQE_OK;
  } catch (const MlpError& e) {
    return mlp_fail(n, e);
  }
}

tnqe_status tnqe_mlp_gradient(tnqe_mlp* n, const float* X, const float* T, const float* w, int batch, float* loss,
                              float* grad) {
  if (!n || !T) return TNQE_ERR_ARG;
  try {
    check_batch(n, X, batch);
    n->launches = 0;
    upload_batch(n, X, T, w, batch);
    forward(n, batch);
    backward(n, batch, w != nullptr);
    float l = 0.f;
    ck(cudaMemcpyAsync(&l, n->scal + 1, sizeof(float), cudaMemcpyDeviceToHost, n->stream), "copy loss");
    if (grad) ck(cudaMemcpyAsync(grad, n->G, sizeof(float) * n->count, cudaMemcpyDeviceToHost, n->stream), "copy grad");
    ck(cudaStreamSynchronize(n->stream), "sync");
    if (loss) *loss = l;
    return TNQE_OK;
  } catch (const MlpError& e) {
    return mlp_fail(n, e);
  }
}

tnqe_status tnqe_mlp_adam_step(tnqe_mlp* n, const float* X, const float* T, const float* w, int batch, float lr,
                               float beta1, float beta2, float eps, float* loss) {
  if (!n || !T) return TNQE_ERR_ARG;
  try {
    check_batch(n, X, batch);
    if (!(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
      throw MlpError(TNQE_ERR_ARG, "bad Adam hyper-parameters");
    n->launches = 0;
    upload_batch(n, X, T, w, batch);
    forward(n, batch);
    backward(n, batch, w != nullptr);
    ++n->step;
    const float c1 = 1.f - std::pow(beta1, (float)n->step), c2 = 1.f - std::pow(beta2, (float)n->step);
    adam_kernel<<<blocks(n->count), 256, 0, n->stream>>>(n->P, n->G, n->Mo, n->Vo, n->count, lr, beta1, beta2, eps, c1,
                                                         c2);
    launched(n);
    float l = 0.f;
    ck(cudaMemcpyAsync(&l, n->scal + 1, sizeof(float), cudaMemcpyDeviceToHost, n->stream), "copy loss");
    ck(cudaStreamSynchronize(n->stream), "sync");
    if (loss) *loss = l;
    return TNQE_OK;
  } catch (const MlpError& e) {
    return mlp_fail(n, e);
  }
}

int tnqe_mlp_last_launches(const tnqe_mlp* n) { return n ? n->launches : 0; }

const char* tnqe_mlp_last_error(const tnqe_mlp* n) { return n ? n->err.c_str() : "null network"; }

void tnqe_mlp_destroy(tnqe_mlp* n) {
  if (!n) return;
  if (n->stream) cudaStreamSynchronize(n->stream);
  float* bufs[] = {n->P, n->G, n->Mo, n->Vo, n->X, n->Z1, n->A1, n->Z2, n->A2,
                   n->Y, n->T, n->w, n->dY, n->dA, n->dZ, n->rowloss, n->scal};
  for (float* p : bufs)
    if (p) cudaFree(p);
  if (n->own_stream && n->stream) cudaStreamDestroy(n->stream);
  delete n;
}

}  // extern "C"
