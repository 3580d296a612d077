// Learned warm start: a fully connected network (FP32) that maps an instance's
// parameter vector and a mode index to initial factor profiles, with hand-written
// forward, backward and Adam kernels, and the kernel that turns predicted profiles
// into initial factor columns (the paper's Algorithm 1 starts from random values;
// this replaces them by a learned proposal).
//
// Network: n_in -> H -> ... -> H -> n_out, tanh after every hidden layer, linear
// output; loss = mean squared error over the batch and outputs.  Parameters are one
// flat FP32 array: for each layer l, W_l [out][in] row-major, then b_l [out].
#include <string.h>

#include <algorithm>

#include "taps_internal.cuh"

struct taps_mlp {
  int L;                      // linear layers
  int dims[TAPS_MLP_MAX_LAYERS + 1];
  size_t woff[TAPS_MLP_MAX_LAYERS], boff[TAPS_MLP_MAX_LAYERS];
  size_t nparams;
  float *d_p, *d_g, *d_m, *d_v;  // parameters, gradients, Adam moments
  long long t;                   // Adam step count
  cudaStream_t stream;
  int cap;                       // batch capacity of the activation buffers
  float* d_act;                  // activations A_0 .. A_L, [cap][dims[l]] each
  float* d_dact;                 // gradient buffers, same layout
  size_t aoff[TAPS_MLP_MAX_LAYERS + 1];
  float* d_loss;                 // per-block loss partials
  float* h_loss;
  int* d_status;
};

// ---------------------------------------------------------------------------------
// C[r][c] (+)= sum_k X(r,k) Y(k,c), X(r,k) = X[r*sxr + k*sxk], Y(k,c) = Y[k*syk + c*syc],
// C row-major with leading dimension ldc.  Epilogue: + bias[c] (optional), tanh
// (optional).  32 x 32 output tile, 32-wide k tile in shared memory, 256 threads with
// 4 outputs each.
// ---------------------------------------------------------------------------------
#define MT 32
__global__ void __launch_bounds__(256) mlp_gemm_kernel(const float* __restrict__ X, long long sxr, long long sxk,
                                                       const float* __restrict__ Y, long long syk, long long syc,
                                                       float* __restrict__ C, int ldc, int R, int Cn, int K,
                                                       const float* __restrict__ bias, int act_tanh) {
  __shared__ float Xs[MT][MT + 1];
  __shared__ float Ys[MT][MT + 1];
  const int r0 = blockIdx.y * MT, c0 = blockIdx.x * MT;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // ty in 0..7, 4 rows each
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k0 = 0; k0 < K; k0 += MT) {
    for (int idx = threadIdx.x; idx < MT * MT; idx += blockDim.x) {
      int a = idx / MT, b = idx % MT;
      int r = r0 + a, k = k0 + b;
      Xs[a][b] = (r < R && k < K) ? X[r * sxr + k * sxk] : 0.f;
      int kk = k0 + a, c = c0 + b;
      Ys[a][b] = (kk < K && c < Cn) ? Y[kk * syk + c * syc] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < MT; ++k) {
      float yv = Ys[k][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] += Xs[ty * 4 + q][k] * yv;
    }
    __syncthreads();
  }
  int c = c0 + tx;
  if (c >= Cn) return;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int r = r0 + ty * 4 + q;
    if (r >= R) continue;
    float v = acc[q] + (bias ? bias[c] : 0.f);
    if (act_tanh) v = tanhf(v);
    C[(size_t)r * ldc + c] = v;
  }
}

// Loss partials and dY = 2 (Y - T) / (B * n_out).
__global__ void mlp_mse_kernel(const float* __restrict__ Yp, const float* __restrict__ T, long long n, float scale,
                               float* __restrict__ dY, float* __restrict__ partial) {
  __shared__ float red[32];
  float s = 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float d = Yp[i] - T[i];
    s += d * d;
    dY[i] = 2.f * d * scale;
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// G <- G * (1 - A^2)  (tanh derivative in terms of its output A)
__global__ void mlp_tanh_back_kernel(float* __restrict__ G, const float* __restrict__ A, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) G[i] *= 1.f - A[i] * A[i];
}

// db[o] = sum_b G[b][o]
__global__ void mlp_bias_grad_kernel(const float* __restrict__ G, int B, int O, float* __restrict__ db) {
  int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= O) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += G[(size_t)b * O + o];
  db[o] = s;
}

// Adam with bias correction.
__global__ void mlp_adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                                float* __restrict__ v, long long n, float lr, float b1, float b2, float eps,
                                float c1, float c2) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = g[i];
  float mi = b1 * m[i] + (1.f - b1) * gi;
  float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Xavier-uniform weights from SplitMix64 draws keyed on (seed, parameter index); zero biases.
__global__ void mlp_init_kernel(float* __restrict__ p, long long woff, long long boff, int in, int out,
                                unsigned seed) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long nw = (long long)in * out;
  if (i < nw) {
    double u = taps_uniform_pm1(seed, 0xEE, (int)(i & 0xFFFFF), (int)((woff + (i >> 20)) & 0xFFF));
    float lim = sqrtf(6.f / (float)(in + out));
    p[woff + i] = (float)u * lim;
  } else if (i < nw + out) {
    p[boff + (i - nw)] = 0.f;
  }
}

// ---------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------
static void gemm(cudaStream_t s, const float* X, long long sxr, long long sxk, const float* Y, long long syk,
                 long long syc, float* C, int ldc, int R, int Cn, int K, const float* bias, int act) {
  dim3 grid((Cn + MT - 1) / MT, (R + MT - 1) / MT);
  mlp_gemm_kernel<<<grid, 256, 0, s>>>(X, sxr, sxk, Y, syk, syc, C, ldc, R, Cn, K, bias, act);
}

static int mlp_ensure_batch(taps_mlp* N, int B) {
  if (B <= N->cap) return TAPS_OK;
  cudaFree(N->d_act);
  cudaFree(N->d_dact);
  N->d_act = N->d_dact = nullptr;
  size_t tot = 0;
  for (int l = 0; l <= N->L; ++l) {
    N->aoff[l] = tot;
    tot += (size_t)B * N->dims[l];
  }
  TAPS_TRY(taps_alloc((void**)&N->d_act, sizeof(float) * tot));
  TAPS_TRY(taps_alloc((void**)&N->d_dact, sizeof(float) * tot));
  N->cap = B;
  return TAPS_OK;
}

extern "C" void taps_mlp_destroy(taps_mlp* N) {
  if (!N) return;
  if (N->stream) cudaStreamSynchronize(N->stream);
  cudaFree(N->d_p);
  cudaFree(N->d_g);
  cudaFree(N->d_m);
  cudaFree(N->d_v);
  cudaFree(N->d_act);
  cudaFree(N->d_dact);
  cudaFree(N->d_loss);
  cudaFree(N->d_status);
  if (N->h_loss) cudaFreeHost(N->h_loss);
  delete N;
}

extern "C" int taps_mlp_create(int n_in, int n_hidden, int hidden_layers, int n_out, unsigned seed, void* stream,
                               taps_mlp** out) {
  if (!out || n_in < 1 || n_hidden < 1 || n_out < 1 || hidden_layers < 0 ||
      hidden_layers + 1 > TAPS_MLP_MAX_LAYERS)
    return TAPS_ERR_INVALID_ARG;
  *out = nullptr;
  taps_mlp* N = new taps_mlp();
  memset((void*)N, 0, sizeof(taps_mlp));
  N->L = hidden_layers + 1;
  N->dims[0] = n_in;
  for (int l = 1; l < N->L; ++l) N->dims[l] = n_hidden;
  N->dims[N->L] = n_out;
  N->stream = (cudaStream_t)stream;
  size_t off = 0;
  for (int l = 0; l < N->L; ++l) {
    N->woff[l] = off;
    off += (size_t)N->dims[l] * N->dims[l + 1];
    N->boff[l] = off;
    off += N->dims[l + 1];
  }
  N->nparams = off;
  int st = TAPS_OK;
  do {
    if ((st = taps_alloc((void**)&N->d_p, sizeof(float) * off)) != TAPS_OK) break;
    if ((st = taps_alloc((void**)&N->d_g, sizeof(float) * off)) != TAPS_OK) break;
    if ((st = taps_alloc((void**)&N->d_m, sizeof(float) * off)) != TAPS_OK) break;
    if ((st = taps_alloc((void**)&N->d_v, sizeof(float) * off)) != TAPS_OK) break;
    if ((st = taps_alloc((void**)&N->d_loss, sizeof(float) * 256)) != TAPS_OK) break;
    if ((st = taps_alloc((void**)&N->d_status, sizeof(int))) != TAPS_OK) break;
    if (cudaMallocHost((void**)&N->h_loss, sizeof(float) * 256) != cudaSuccess) { st = TAPS_ERR_OOM; break; }
    cudaMemsetAsync(N->d_m, 0, sizeof(float) * off, N->stream);
    cudaMemsetAsync(N->d_v, 0, sizeof(float) * off, N->stream);
    cudaMemsetAsync(N->d_g, 0, sizeof(float) * off, N->stream);
    for (int l = 0; l < N->L; ++l) {
      long long n = (long long)N->dims[l] * N->dims[l + 1] + N->dims[l + 1];
      mlp_init_kernel<<<(unsigned)((n + 255) / 256), 256, 0, N->stream>>>(
          N->d_p, (long long)N->woff[l], (long long)N->boff[l], N->dims[l], N->dims[l + 1], seed + 977u * l);
    }
    if (cudaGetLastError() != cudaSuccess) { st = TAPS_ERR_CUDA; break; }
    if (cudaStreamSynchronize(N->stream) != cudaSuccess) { st = TAPS_ERR_CUDA; break; }
  } while (0);
  if (st != TAPS_OK) {
    taps_mlp_destroy(N);
    return st;
  }
  *out = N;
  return TAPS_OK;
}

extern "C" long long taps_mlp_num_params(const taps_mlp* N) { return N ? (long long)N->nparams : -1; }

extern "C" int taps_mlp_get_params(const taps_mlp* N, float* host, long long n) {
  if (!N || !host || n != (long long)N->nparams) return TAPS_ERR_INVALID_ARG;
  TAPS_CUDA(cudaMemcpyAsync(host, N->d_p, sizeof(float) * n, cudaMemcpyDeviceToHost, N->stream));
  TAPS_CUDA(cudaStreamSynchronize(N->stream));
  return TAPS_OK;
}

extern "C" int taps_mlp_set_params(taps_mlp* N, const float* host, long long n) {
  if (!N || !host || n != (long long)N->nparams) return TAPS_ERR_INVALID_ARG;
  TAPS_CUDA(cudaMemcpyAsync(N->d_p, host, sizeof(float) * n, cudaMemcpyHostToDevice, N->stream));
  TAPS_CUDA(cudaStreamSynchronize(N->stream));
  N->t = 0;
  TAPS_CUDA(cudaMemsetAsync(N->d_m, 0, sizeof(float) * n, N->stream));
  TAPS_CUDA(cudaMemsetAsync(N->d_v, 0, sizeof(float) * n, N->stream));
  return TAPS_OK;
}

// Forward pass into the activation buffers (A_0 = x); returns the output pointer.
static int mlp_forward_impl(taps_mlp* N, const float* x_dev, int B, float** yout) {
  TAPS_TRY(mlp_ensure_batch(N, B));
  cudaStream_t s = N->stream;
  TAPS_CUDA(cudaMemcpyAsync(N->d_act + N->aoff[0], x_dev, sizeof(float) * B * N->dims[0],
                            cudaMemcpyDeviceToDevice, s));
  for (int l = 0; l < N->L; ++l) {
    const int in = N->dims[l], o = N->dims[l + 1];
    const float* A = N->d_act + N->aoff[l];
    float* Z = N->d_act + N->aoff[l + 1];
    // Z[b][o] = sum_i A[b][i] W[o][i] + b[o]
    gemm(s, A, in, 1, N->d_p + N->woff[l], 1, in, Z, o, B, o, in, N->d_p + N->boff[l], l < N->L - 1);
  }
  TAPS_CUDA(cudaGetLastError());
  *yout = N->d_act + N->aoff[N->L];
  return TAPS_OK;
}

extern "C" int taps_mlp_forward(taps_mlp* N, const float* x_dev, int batch, float* y_dev) {
  if (!N || !x_dev || !y_dev || batch < 1) return TAPS_ERR_INVALID_ARG;
  float* y = nullptr;
  TAPS_TRY(mlp_forward_impl(N, x_dev, batch, &y));
  TAPS_CUDA(cudaMemcpyAsync(y_dev, y, sizeof(float) * batch * N->dims[N->L], cudaMemcpyDeviceToDevice, N->stream));
  return TAPS_OK;
}

// Loss and parameter gradients of one batch (gradients into the internal buffer).
static int mlp_grad_impl(taps_mlp* N, const float* x_dev, const float* t_dev, int B, int want_loss, float* loss) {
  float* y = nullptr;
  TAPS_TRY(mlp_forward_impl(N, x_dev, B, &y));
  cudaStream_t s = N->stream;
  const int O = N->dims[N->L];
  long long n = (long long)B * O;
  float* G = N->d_dact + N->aoff[N->L];
  mlp_mse_kernel<<<64, 256, 0, s>>>(y, t_dev, n, 1.f / (float)n, G, N->d_loss);
  for (int l = N->L - 1; l >= 0; --l) {
    const int in = N->dims[l], o = N->dims[l + 1];
    const float* A = N->d_act + N->aoff[l];
    float* Gl = N->d_dact + N->aoff[l + 1];
    // dW[o][i] = sum_b G[b][o] A[b][i]
    gemm(s, Gl, 1, o, A, in, 1, N->d_g + N->woff[l], in, o, in, B, nullptr, 0);
    mlp_bias_grad_kernel<<<(o + 127) / 128, 128, 0, s>>>(Gl, B, o, N->d_g + N->boff[l]);
    if (l > 0) {
      float* dA = N->d_dact + N->aoff[l];
      // dA[b][i] = sum_o G[b][o] W[o][i]
      gemm(s, Gl, o, 1, N->d_p + N->woff[l], in, 1, dA, in, B, in, o, nullptr, 0);
      long long na = (long long)B * in;
      mlp_tanh_back_kernel<<<(unsigned)((na + 255) / 256), 256, 0, s>>>(dA, A, na);
    }
  }
  TAPS_CUDA(cudaGetLastError());
  if (want_loss) {
    TAPS_CUDA(cudaMemcpyAsync(N->h_loss, N->d_loss, sizeof(float) * 64, cudaMemcpyDeviceToHost, s));
    TAPS_CUDA(cudaStreamSynchronize(s));
    double acc = 0.0;
    for (int b = 0; b < 64; ++b) acc += N->h_loss[b];
    *loss = (float)(acc / (double)n);
  }
  return TAPS_OK;
}

extern "C" int taps_mlp_grad(taps_mlp* N, const float* x_dev, const float* t_dev, int batch, float* loss_out,
                             float* grad_host) {
  if (!N || !x_dev || !t_dev || batch < 1) return TAPS_ERR_INVALID_ARG;
  float loss = 0.f;
  TAPS_TRY(mlp_grad_impl(N, x_dev, t_dev, batch, 1, &loss));
  if (loss_out) *loss_out = loss;
  if (grad_host) {
    TAPS_CUDA(cudaMemcpyAsync(grad_host, N->d_g, sizeof(float) * N->nparams, cudaMemcpyDeviceToHost, N->stream));
    TAPS_CUDA(cudaStreamSynchronize(N->stream));
  }
  return TAPS_OK;
}

extern "C" int taps_mlp_adam(taps_mlp* N, float lr, float beta1, float beta2, float eps) {
  if (!N) return TAPS_ERR_INVALID_ARG;
  N->t += 1;
  float c1 = 1.f - powf(beta1, (float)N->t), c2 = 1.f - powf(beta2, (float)N->t);
  long long n = (long long)N->nparams;
  mlp_adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, N->stream>>>(N->d_p, N->d_g, N->d_m, N->d_v, n, lr, beta1,
                                                                     beta2, eps, c1, c2);
  TAPS_CUDA(cudaGetLastError());
  return TAPS_OK;
}

extern "C" int taps_mlp_train(taps_mlp* N, const float* x_dev, const float* t_dev, int batch, int steps, float lr,
                              float* loss_out) {
  if (!N || !x_dev || !t_dev || batch < 1 || steps < 0) return TAPS_ERR_INVALID_ARG;
  float loss = 0.f;
  for (int it = 0; it < steps; ++it) {
    TAPS_TRY(mlp_grad_impl(N, x_dev, t_dev, batch, it == steps - 1, &loss));
    TAPS_TRY(taps_mlp_adam(N, lr, 0.9f, 0.999f, 1e-8f));
  }
  TAPS_CUDA(cudaStreamSynchronize(N->stream));
  if (loss_out) *loss_out = loss;
  return TAPS_OK;
}

// ---------------------------------------------------------------------------------
// Predicted profiles -> initial factors.  prof is [M][D * n_ref + 1] (FP32): per dim a
// profile sampled at n_ref uniform points of [lo_d, hi_d], then the mode weight.
// U_d[j, m] = linear interpolation of the profile at the free node j; the weight
// multiplies the last dim.
// ---------------------------------------------------------------------------------
struct ProfileDims {
  int nf[TAPS_MAX_DIMS], off[TAPS_MAX_DIMS], n[TAPS_MAX_DIMS];
  double* U[TAPS_MAX_DIMS];
};

__global__ void profiles_to_factors_kernel(const float* __restrict__ prof, ProfileDims pd, int D, int M, int n_ref,
                                           int d, double wscale) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int nf = pd.nf[d];
  if (idx >= nf * M) return;
  int m = idx / nf, j = idx % nf;
  int node = j + pd.off[d];
  double t = (double)node / (double)(pd.n[d] - 1) * (double)(n_ref - 1);
  int k = min((int)floor(t), n_ref - 2);
  double f = t - k;
  const float* p = prof + (size_t)m * (D * n_ref + 1) + (size_t)d * n_ref;
  double v = (1.0 - f) * (double)p[k] + f * (double)p[k + 1];
  if (d == D - 1) v *= wscale * (double)prof[(size_t)m * (D * n_ref + 1) + D * n_ref];
  pd.U[d][(size_t)m * nf + j] = v;
}

extern "C" int taps_factors_from_profiles(const taps_problem* P, taps_factors* U, int M, const float* prof_dev,
                                          int n_ref, double weight_scale) {
  if (!P || !U || !prof_dev || M < 1 || M > U->M_cap || n_ref < 2) return TAPS_ERR_INVALID_ARG;
  ProfileDims pd;
  memset(&pd, 0, sizeof(pd));
  for (int d = 0; d < P->D; ++d) {
    pd.nf[d] = P->dims[d]->nf;
    pd.off[d] = P->dims[d]->off;
    pd.n[d] = P->dims[d]->n;
    pd.U[d] = U->d_U[d];
  }
  for (int d = 0; d < P->D; ++d) {
    int n = pd.nf[d] * M;
    profiles_to_factors_kernel<<<(n + 255) / 256, 256, 0, P->stream>>>(prof_dev, pd, P->D, M, n_ref, d,
                                                                        weight_scale);
  }
  TAPS_CUDA(cudaGetLastError());
  TAPS_CUDA(cudaStreamSynchronize(P->stream));
  U->M = M;
  return TAPS_OK;
}
