// Sectional-drag surrogate: a small MLP (inputs of the branch-wise model,
// hidden layers of GELU units, one output: the sectional drag coefficient
// C_d of Eq. 2, summed over the branches by Eq. 4, Sec. 2.4) trained and
// evaluated by these kernels.  Weights are used in BF16 with FP32 accumulation; FP32 master
// weights and Adam moments are kept beside them.  Every reduction (weight
// gradients, bias gradients, loss) runs in a fixed order, so training is
// deterministic.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <new>
#include <stdexcept>

#include "internal.h"

namespace lbm {
namespace {

thread_local char g_mlp_err[256] = "";

int mlp_check(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(g_mlp_err, sizeof g_mlp_err, "%s: %s", what, cudaGetErrorString(e));
    return LBM_ECUDA;
  }
  return LBM_OK;
}

__device__ __forceinline__ float ldv(const float* p, long long i) { return p[i]; }
__device__ __forceinline__ float ldv(const __nv_bfloat16* p, long long i) { return __bfloat162float(p[i]); }

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// C[m][n] = sum_k A(m, k) B(k, n) (+ bias[n]); A(m,k) = A[m*sam + k*sak],
// B(k,n) = B[k*sbk + n*sbn].  Optional epilogue: Z = C + bias, O = GELU(Z).
// Tiles of 64 x 64 outputs, K in chunks of 16, 256 threads with 4 x 4 each.
constexpr int TM = 64, TN = 64, TK = 16;

template <typename TB, bool EPI>
__global__ void __launch_bounds__(256) k_gemm(const float* __restrict__ A, long long sam, long long sak,
                                              const TB* __restrict__ Bm, long long sbk, long long sbn, int M, int N,
                                              int K, const float* __restrict__ bias, float* __restrict__ Z,
                                              float* __restrict__ O, int act) {
  __shared__ float As[TK][TM + 1];
  __shared__ float Bs[TK][TN + 1];
  const int t = threadIdx.x;
  const int tm = (t / 16) * 4, tn = (t % 16) * 4;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += TK) {
    for (int e = t; e < TK * TM; e += 256) {
      const int kk = e / TM, mm = e % TM;
      const int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < M && k < K) ? A[(long long)m * sam + (long long)k * sak] : 0.0f;
    }
    for (int e = t; e < TK * TN; e += 256) {
      const int kk = e / TN, nn = e % TN;
      const int n = n0 + nn, k = k0 + kk;
      Bs[kk][nn] = (n < N && k < K) ? ldv(Bm, (long long)k * sbk + (long long)n * sbn) : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = As[kk][tm + i];
        b[i] = Bs[kk][tn + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + tm + i, n = n0 + tn + j;
      if (m >= M || n >= N) continue;
      float v = acc[i][j];
      if (EPI) {
        v += bias[n];
        Z[(long long)m * N + n] = v;
        O[(long long)m * N + n] = act ? gelu(v) : v;
      } else {
        O[(long long)m * N + n] = v;
      }
    }
}

// X_hat[b][i] = (X[idx ? idx[b] : b][i] - mu[i]) / sd[i]
__global__ void k_norm_in(const float* __restrict__ X, const int* __restrict__ idx, int batch, int nin,
                          const float* __restrict__ mu, const float* __restrict__ sd, float* __restrict__ Xh) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= batch * nin) return;
  const int b = t / nin, i = t % nin;
  const int r = idx ? idx[b] : b;
  Xh[t] = (X[(long long)r * nin + i] - mu[i]) / sd[i];
}

// dY = 2 (y_hat - (y - mu_y)/sd_y) / batch; per-CTA FP64 partial sums of the squared error
__global__ void __launch_bounds__(256) k_mse(const float* __restrict__ Yh, const float* __restrict__ Y,
                                             const int* __restrict__ idx, int batch, float mu, float sd,
                                             float* __restrict__ dY, double* __restrict__ partial) {
  __shared__ double s[256];
  const int t = blockIdx.x * 256 + threadIdx.x;
  double e2 = 0;
  if (t < batch) {
    const int r = idx ? idx[t] : t;
    const float d = Yh[t] - (Y[r] - mu) / sd;
    dY[t] = 2.0f * d / (float)batch;
    e2 = (double)d * d;
  }
  s[threadIdx.x] = e2;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = s[0];
}

// dZ = dA * GELU'(Z)
__global__ void k_gelu_back(const float* __restrict__ dA, const float* __restrict__ Z, long long n,
                            float* __restrict__ dZ) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) dZ[t] = dA[t] * gelu_grad(Z[t]);
}

// db[n] = sum_b dZ[b][n], one CTA per column block, fixed order
__global__ void __launch_bounds__(256) k_colsum(const float* __restrict__ dZ, int batch, int N, float* __restrict__ db) {
  __shared__ float s[256];
  const int n = blockIdx.x;
  float acc = 0;
  for (int b = threadIdx.x; b < batch; b += 256) acc += dZ[(long long)b * N + n];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[n] = s[0];
}

// y = y_hat * sd + mu
__global__ void k_denorm(const float* __restrict__ Yh, int batch, float mu, float sd, float* __restrict__ Y) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < batch) Y[t] = Yh[t] * sd + mu;
}

// ensemble mean: Y = (first ? 0 : Y) + w (y_hat sd + mu), member by member
__global__ void k_ens_acc(const float* __restrict__ Yh, int batch, float mu, float sd, float w, int first,
                          float* __restrict__ Y) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < batch) Y[t] = (first ? 0.0f : Y[t]) + w * (Yh[t] * sd + mu);
}

// Adam (Kingma & Ba 2015) on the FP32 master weights, then their BF16 copy
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1, float c2,
                       __nv_bfloat16* __restrict__ wb, const int* __restrict__ bf_map) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float gt = g[t];
  const float mt = b1 * m[t] + (1.0f - b1) * gt;
  const float vt = b2 * v[t] + (1.0f - b2) * gt * gt;
  m[t] = mt;
  v[t] = vt;
  const float wt = w[t] - lr * (mt / c1) / (sqrtf(vt / c2) + eps);
  w[t] = wt;
  const int j = bf_map[t];
  if (j >= 0) wb[j] = __float2bfloat16_rn(wt);
}

__global__ void k_to_bf16(const float* __restrict__ w, const int* __restrict__ bf_map, long long n,
                          __nv_bfloat16* __restrict__ wb) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int j = bf_map[t];
  if (j >= 0) wb[j] = __float2bfloat16_rn(w[t]);
}

unsigned nb(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

const char* mlp_error_string() { return g_mlp_err; }

// ---------------------------------------------------------------- launchers
int mlp_gemm_bias_act(const float* A, long long sam, long long sak, const __nv_bfloat16* W, long long swk,
                      long long swn, int M, int N, int K, const float* bias, float* Z, float* O, int act,
                      void* stream) {
  dim3 grid(nb(N, TN), nb(M, TM));
  k_gemm<__nv_bfloat16, true><<<grid, 256, 0, (cudaStream_t)stream>>>(A, sam, sak, W, swk, swn, M, N, K, bias, Z, O,
                                                                       act);
  return mlp_check("gemm_fwd");
}

int mlp_gemm_bf16(const float* A, long long sam, long long sak, const __nv_bfloat16* W, long long swk, long long swn,
                  int M, int N, int K, float* O, void* stream) {
  dim3 grid(nb(N, TN), nb(M, TM));
  k_gemm<__nv_bfloat16, false><<<grid, 256, 0, (cudaStream_t)stream>>>(A, sam, sak, W, swk, swn, M, N, K, nullptr,
                                                                        nullptr, O, 0);
  return mlp_check("gemm_bf16");
}

int mlp_gemm_f32(const float* A, long long sam, long long sak, const float* B, long long sbk, long long sbn, int M,
                 int N, int K, float* O, void* stream) {
  dim3 grid(nb(N, TN), nb(M, TM));
  k_gemm<float, false><<<grid, 256, 0, (cudaStream_t)stream>>>(A, sam, sak, B, sbk, sbn, M, N, K, nullptr, nullptr,
                                                                O, 0);
  return mlp_check("gemm_f32");
}

int mlp_norm_in(const float* X, const int* idx, int batch, int nin, const float* mu, const float* sd, float* Xh,
                void* stream) {
  k_norm_in<<<nb((long long)batch * nin, 256), 256, 0, (cudaStream_t)stream>>>(X, idx, batch, nin, mu, sd, Xh);
  return mlp_check("norm_in");
}

int mlp_mse(const float* Yh, const float* Y, const int* idx, int batch, float mu, float sd, float* dY,
            double* partial, int* nparts, void* stream) {
  *nparts = (int)nb(batch, 256);
  k_mse<<<*nparts, 256, 0, (cudaStream_t)stream>>>(Yh, Y, idx, batch, mu, sd, dY, partial);
  return mlp_check("mse");
}

int mlp_gelu_back(const float* dA, const float* Z, long long n, float* dZ, void* stream) {
  k_gelu_back<<<nb(n, 256), 256, 0, (cudaStream_t)stream>>>(dA, Z, n, dZ);
  return mlp_check("gelu_back");
}

int mlp_colsum(const float* dZ, int batch, int N, float* db, void* stream) {
  k_colsum<<<N, 256, 0, (cudaStream_t)stream>>>(dZ, batch, N, db);
  return mlp_check("colsum");
}

int mlp_denorm(const float* Yh, int batch, float mu, float sd, float* Y, void* stream) {
  k_denorm<<<nb(batch, 256), 256, 0, (cudaStream_t)stream>>>(Yh, batch, mu, sd, Y);
  return mlp_check("denorm");
}

int mlp_ens_acc(const float* Yh, int batch, float mu, float sd, float w, int first, float* Y, void* stream) {
  k_ens_acc<<<nb(batch, 256), 256, 0, (cudaStream_t)stream>>>(Yh, batch, mu, sd, w, first, Y);
  return mlp_check("ens_acc");
}

int mlp_adam(float* w, const float* g, float* m, float* v, long long n, float lr, float b1, float b2, float eps,
             float c1, float c2, __nv_bfloat16* wb, const int* bf_map, void* stream) {
  k_adam<<<nb(n, 256), 256, 0, (cudaStream_t)stream>>>(w, g, m, v, n, lr, b1, b2, eps, c1, c2, wb, bf_map);
  return mlp_check("adam");
}

int mlp_to_bf16(const float* w, const int* bf_map, long long n, __nv_bfloat16* wb, void* stream) {
  k_to_bf16<<<nb(n, 256), 256, 0, (cudaStream_t)stream>>>(w, bf_map, n, wb);
  return mlp_check("to_bf16");
}

}  // namespace lbm

// ---------------------------------------------------------------- C-ABI
#include <cstring>
#include <string>
#include <vector>

struct lbm_mlp {
  int n_in = 6, width = 128, hidden = 3;
  cudaStream_t stream = nullptr;
  int max_batch = 0;
  char* base = nullptr;
  size_t need = 0;
  long long P = 0, PW = 0;                      // parameters, weight entries (BF16 copy)
  std::vector<long long> w_off, b_off, wb_off;  // per layer offsets (floats / bf16 elements)
  std::vector<int> in_dim, out_dim;
  size_t o_w, o_g, o_m, o_v, o_wb, o_map, o_norm, o_xh, o_z, o_a, o_yh, o_dy, o_d0, o_d1, o_part;
  float mu_y = 0, sd_y = 1;
  long long t = 0;  // Adam steps
  std::string err;
  template <class T>
  T* dev(size_t off) const { return reinterpret_cast<T*>(base + off); }
  int layers() const { return hidden + 1; }
};

namespace {
thread_local std::string g_mlp_api_err;
int mfail(int code, const std::string& m) {
  g_mlp_api_err = m;
  return code;
}
// No C++ exception leaves the C-ABI: the one in flight (called from a catch
// handler) becomes a status and a message.
int mexception_status() {
  try {
    throw;
  } catch (const std::bad_alloc&) {
    return mfail(LBM_ENOMEM, "host memory allocation failed");
  } catch (const std::length_error&) {
    return mfail(LBM_ENOMEM, "host allocation too large");
  } catch (const std::exception& e) {
    return mfail(LBM_ESTATE, std::string("internal error: ") + e.what());
  } catch (...) {
    return mfail(LBM_ESTATE, "internal error");
  }
}
#define MCK(call)                                                             \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) return mfail(LBM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)
#define MRC(call)                                          \
  do {                                                     \
    int r_ = (call);                                       \
    if (r_) return mfail(r_, lbm::mlp_error_string());     \
  } while (0)
size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

void mlp_layout(lbm_mlp* m, int max_batch) {
  size_t off = 0;
  auto put = [&](size_t bytes) {
    size_t o = off;
    off = al(off + bytes);
    return o;
  };
  const size_t B = (size_t)max_batch, W = (size_t)m->width, H = (size_t)m->hidden;
  m->o_w = put(m->P * 4);
  m->o_g = put(m->P * 4);
  m->o_m = put(m->P * 4);
  m->o_v = put(m->P * 4);
  m->o_wb = put(m->PW * 2);
  m->o_map = put(m->P * 4);
  m->o_norm = put(2 * m->n_in * 4);
  m->o_xh = put(B * m->n_in * 4);
  m->o_z = put(H * B * W * 4);
  m->o_a = put(H * B * W * 4);
  m->o_yh = put(B * 4);
  m->o_dy = put(B * 4);
  m->o_d0 = put(B * W * 4);
  m->o_d1 = put(B * W * 4);
  m->o_part = put((B / 256 + 2) * 8);
  m->need = off;
  m->max_batch = max_batch;
}

// forward through all layers; leaves pre-activations, activations and y_hat
int mlp_forward_dev(lbm_mlp* m, const float* x, const int* idx, int batch) {
  const size_t BW = (size_t)m->max_batch * m->width;
  MRC(lbm::mlp_norm_in(x, idx, batch, m->n_in, m->dev<float>(m->o_norm), m->dev<float>(m->o_norm) + m->n_in,
                       m->dev<float>(m->o_xh), m->stream));
  const float* in = m->dev<float>(m->o_xh);
  long long ld = m->n_in;
  for (int l = 0; l < m->layers(); ++l) {
    const int ni = m->in_dim[l], no = m->out_dim[l];
    const __nv_bfloat16* W = m->dev<__nv_bfloat16>(m->o_wb) + m->wb_off[l];
    const float* b = m->dev<float>(m->o_w) + m->b_off[l];
    const bool last = l == m->layers() - 1;
    float* Z = last ? m->dev<float>(m->o_yh) : m->dev<float>(m->o_z) + l * BW;
    float* O = last ? m->dev<float>(m->o_yh) : m->dev<float>(m->o_a) + l * BW;
    // Z[b][o] = sum_i in[b][i] W[o][i] + bias[o]
    MRC(lbm::mlp_gemm_bias_act(in, ld, 1, W, 1, ni, batch, no, ni, b, Z, O, last ? 0 : 1, m->stream));
    in = O;
    ld = no;
  }
  return LBM_OK;
}

// backward from dY = d loss / d y_hat (in o_dy) into the flat gradient buffer
int mlp_backward_dev(lbm_mlp* m, int batch) {
  const size_t BW = (size_t)m->max_batch * m->width;
  float* g = m->dev<float>(m->o_g);
  float* dcur = m->dev<float>(m->o_dy);  // dZ of the current layer
  float* bufs[2] = {m->dev<float>(m->o_d0), m->dev<float>(m->o_d1)};
  int which = 0;
  for (int l = m->layers() - 1; l >= 0; --l) {
    const int ni = m->in_dim[l], no = m->out_dim[l];
    const float* X = l == 0 ? m->dev<float>(m->o_xh) : m->dev<float>(m->o_a) + (l - 1) * BW;
    // dW[o][i] = sum_b dZ[b][o] X[b][i]
    MRC(lbm::mlp_gemm_f32(dcur, 1, no, X, ni, 1, no, ni, batch, g + m->w_off[l], m->stream));
    MRC(lbm::mlp_colsum(dcur, batch, no, g + m->b_off[l], m->stream));
    if (l == 0) break;
    // dA_{l-1}[b][i] = sum_o dZ[b][o] W[o][i]; dZ_{l-1} = dA * GELU'(Z_{l-1})
    float* dA = bufs[which];
    const __nv_bfloat16* W = m->dev<__nv_bfloat16>(m->o_wb) + m->wb_off[l];
    MRC(lbm::mlp_gemm_bf16(dcur, no, 1, W, ni, 1, batch, ni, no, dA, m->stream));
    float* dZ = bufs[which ^ 1];
    MRC(lbm::mlp_gelu_back(dA, m->dev<float>(m->o_z) + (l - 1) * BW, (long long)batch * ni, dZ, m->stream));
    dcur = dZ;
    which ^= 1;
  }
  return LBM_OK;
}

int mlp_loss_grad(lbm_mlp* m, const float* x, const float* y, const int* idx, int batch, double* loss) {
  int rc = mlp_forward_dev(m, x, idx, batch);
  if (rc) return rc;
  int nparts = 0;
  MRC(lbm::mlp_mse(m->dev<float>(m->o_yh), y, idx, batch, m->mu_y, m->sd_y, m->dev<float>(m->o_dy),
                   m->dev<double>(m->o_part), &nparts, m->stream));
  rc = mlp_backward_dev(m, batch);
  if (rc) return rc;
  if (loss) {
    std::vector<double> p(nparts);
    MCK(cudaMemcpyAsync(p.data(), m->base + m->o_part, nparts * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    MCK(cudaStreamSynchronize(m->stream));
    double s = 0;
    for (double v : p) s += v;
    *loss = s / batch;
  }
  return LBM_OK;
}

bool ready(const lbm_mlp* m) { return m && m->base; }
}  // namespace

extern "C" {

int lbm_mlp_create(int n_in, int width, int hidden_layers, void* stream, lbm_mlp** out) try {
  if (!out || n_in < 1 || n_in > 64 || width < 1 || width > 1024 || hidden_layers < 1 || hidden_layers > 8)
    return mfail(LBM_EINVAL, "n_in 1..64, width 1..1024, hidden layers 1..8");
  auto* m = new (std::nothrow) lbm_mlp();
  if (!m) return mfail(LBM_ENOMEM, "host allocation");
  m->n_in = n_in;
  m->width = width;
  m->hidden = hidden_layers;
  m->stream = (cudaStream_t)stream;
  long long p = 0, pw = 0;
  for (int l = 0; l <= hidden_layers; ++l) {
    const int ni = l == 0 ? n_in : width, no = l == hidden_layers ? 1 : width;
    m->in_dim.push_back(ni);
    m->out_dim.push_back(no);
    m->w_off.push_back(p);
    m->wb_off.push_back(pw);
    p += (long long)ni * no;
    pw += (long long)ni * no;
    m->b_off.push_back(p);
    p += no;
  }
  m->P = p;
  m->PW = pw;
  *out = m;
  return LBM_OK;
} catch (...) {
  return mexception_status();
}

int lbm_mlp_memory_requirements(const lbm_mlp* m, int max_batch, size_t* bytes) try {
  if (!m || !bytes || max_batch < 1) return mfail(LBM_EINVAL, "bad argument");
  lbm_mlp tmp = *m;
  mlp_layout(&tmp, max_batch);
  *bytes = tmp.need;
  return LBM_OK;
} catch (...) {
  return mexception_status();
}

int lbm_mlp_bind_memory(lbm_mlp* m, void* dev, size_t bytes, int max_batch) try {
  if (!m || !dev || max_batch < 1) return mfail(LBM_EINVAL, "bad argument");
  if ((uintptr_t)dev & 255) return mfail(LBM_EINVAL, "buffer must be 256-byte aligned");
  mlp_layout(m, max_batch);
  if (bytes < m->need) return mfail(LBM_ENOMEM, "buffer smaller than lbm_mlp_memory_requirements");
  m->base = (char*)dev;
  std::vector<int> map(m->P, -1);
  for (int l = 0; l < m->layers(); ++l)
    for (long long k = 0; k < (long long)m->in_dim[l] * m->out_dim[l]; ++k) map[m->w_off[l] + k] = (int)(m->wb_off[l] + k);
  MCK(cudaMemcpyAsync(m->base + m->o_map, map.data(), map.size() * 4, cudaMemcpyHostToDevice, m->stream));
  std::vector<float> norm(2 * m->n_in, 0.0f);
  for (int i = 0; i < m->n_in; ++i) norm[m->n_in + i] = 1.0f;
  MCK(cudaMemcpyAsync(m->base + m->o_norm, norm.data(), norm.size() * 4, cudaMemcpyHostToDevice, m->stream));
  for (size_t o : {m->o_w, m->o_g, m->o_m, m->o_v}) MCK(cudaMemsetAsync(m->base + o, 0, m->P * 4, m->stream));
  MCK(cudaStreamSynchronize(m->stream));
  return LBM_OK;
} catch (...) {
  return mexception_status();
}

int lbm_mlp_param_count(const lbm_mlp* m, long long* n) try {
  if (!m || !n) return mfail(LBM_EINVAL, "null argument");
  *n = m->P;
  return LBM_OK;
} catch (...) {
  return mexception_status();
}

int lbm_mlp_set_params(lbm_mlp* m, const float* host, long long n) try {
  if (!ready(m) || !host || n != m->P) return mfail(LBM_EINVAL, "bind memory first; n must equal the parameter count");
  MCK(cudaMemcpyAsync(m->base + m->o_w, host, n * 4, cudaMemcpyHostToDevice, m->stream));
  MCK(cudaMemsetAsync(m->base + m->o_m, 0, n * 4, m->stream));
  MCK(cudaMemsetAsync(m->base + m->o_v, 0, n * 4, m->stream));
  MRC(lbm::mlp_to_bf16(m->dev<float>(m->o_w), m->dev<int>(m->o_map), m->P, m->dev<__nv_bfloat16>(m->o_wb),
                       m->stream));
  MCK(cudaStreamSynchronize(m->stream));
  m->t = 0;
  return LBM_OK;
} catch (...) {
  return mexception_status();
}

int lbm_mlp_get_params(lbm_mlp* m, float* host, long long n) try {
  if (!ready(m) || !host || n != m->P) return mfail(LBM_EINVAL, "bind memory first; n must equal the parameter count");
  MCK(cudaMemcpyAsync(host, m->base + m->o_w, n * 4, cudaMemcpyDeviceToHost, m->stream));
  MCK(cudaStreamSynchronize(m->stream));
  return LBM_OK;
} catch (...) {
  return mexception_status();
}

int lbm_mlp_set_normalization(lbm_mlp* m, const float* mu_x, const float* sd_x, float mu_y, float sd_y) try {
  if (!ready(m) || !mu_x || !sd_x || !(sd_y > 0)) return mfail(LBM_EINVAL, "bad argument");
  std::vector<float> norm(2 * m->n_in);
  for (int i = 0; i < m->n_in; ++i) {
    if (!(sd_x[i] > 0)) return mfail(LBM_EINVAL, "standard deviations must be positive");
    norm[i] = mu_x[i];
    norm[m->n_in + i] = sd_x[i];
  }
  MCK(cudaMemcpyAsync(m->base + m->o_norm, norm.data(), norm.size() * 4, cudaMemcpyHostToDevice, m->stream));
  MCK(cudaStreamSynchronize(m->stream));
  m->mu_y = mu_y;
  m->sd_y = sd_y;
  return LBM_OK;
} catch (...) {
  return mexception_status();
}

int lbm_mlp_forward(lbm_mlp* m, const float* x, int batch, float* y) try {
  if (!ready(m) || !x || !y || batch < 1 || batch > m->max_batch) return mfail(LBM_EINVAL, "bad argument");
  int rc = mlp_forward_dev(m, x, nullptr, batch);
  if (rc) return rc;
  MRC(lbm::mlp_denorm(m->dev<float>(m->o_yh), batch, m->mu_y, m->sd_y, y, m->stream));
  return LBM_OK;
} catch (...) {
  return mexception_status();
}

int lbm_mlp_ensemble_forward(lbm_mlp* const* nets, int n, const float* x, int batch, float* y) try {
  if (!nets || n < 1 || !x || !y || batch < 1) return mfail(LBM_EINVAL, "bad argument");
  for (int k = 0; k < n; ++k) {
    const lbm_mlp* m = nets[k];
    if (!ready(m) || batch > m->max_batch) return mfail(LBM_EINVAL, "bad member or batch above its capacity");
    if (m->n_in != nets[0]->n_in || m->stream != nets[0]->stream)
      return mfail(LBM_EINVAL, "ensemble members must share their input count and stream");
  }
  for (int k = 0; k < n; ++k) {
    lbm_mlp* m = nets[k];
    int rc = mlp_forward_dev(m, x, nullptr, batch);
    if (rc) return rc;
    MRC(lbm::mlp_ens_acc(m->dev<float>(m->o_yh), batch, m->mu_y, m->sd_y, 1.0f / (float)n, k == 0, y, m->stream));
  }
  return LBM_OK;
} catch (...) {
  return mexception_status();
}

int lbm_mlp_gradients(lbm_mlp* m, const float* x, const float* y, const int* idx, int batch, float* grad_host,
                      double* loss) try {
  if (!ready(m) || !x || !y || batch < 1 || batch > m->max_batch) return mfail(LBM_EINVAL, "bad argument");
  int rc = mlp_loss_grad(m, x, y, idx, batch, loss);
  if (rc) return rc;
  if (grad_host) {
    MCK(cudaMemcpyAsync(grad_host, m->base + m->o_g, m->P * 4, cudaMemcpyDeviceToHost, m->stream));
    MCK(cudaStreamSynchronize(m->stream));
  }
  return LBM_OK;
} catch (...) {
  return mexception_status();
}

int lbm_mlp_train_step(lbm_mlp* m, const float* x, const float* y, const int* idx, int batch, float lr,
                       double* loss) try {
  if (!ready(m) || !x || !y || batch < 1 || batch > m->max_batch || !(lr > 0)) return mfail(LBM_EINVAL, "bad argument");
  int rc = mlp_loss_grad(m, x, y, idx, batch, loss);
  if (rc) return rc;
  m->t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - std::pow(b1, (float)m->t), c2 = 1.0f - std::pow(b2, (float)m->t);
  MRC(lbm::mlp_adam(m->dev<float>(m->o_w), m->dev<float>(m->o_g), m->dev<float>(m->o_m), m->dev<float>(m->o_v),
                    m->P, lr, b1, b2, 1e-8f, c1, c2, m->dev<__nv_bfloat16>(m->o_wb), m->dev<int>(m->o_map),
                    m->stream));
  return LBM_OK;
} catch (...) {
  return mexception_status();
}

const char* lbm_mlp_last_error(void) { return g_mlp_api_err.c_str(); }

void lbm_mlp_destroy(lbm_mlp* m) { delete m; }

}  // extern "C"
