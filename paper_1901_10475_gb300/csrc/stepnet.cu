// stepnet.cu -- a small learned model of each object's time step (not in the
// paper, whose steps adapt inside the serial Alg 3-6; here the step is fixed
// per screen and predicted from the orbital elements).
//
// 8 features -> 64 -> 64 -> 1 (log of the step in seconds), ReLU hidden
// layers, BF16 weights, FP32 accumulation, FP32 master weights updated by
// AdamW.  Parameters, flat FP32: W1[8][64], b1[64], W2[64][64], b2[64],
// w3[64], b3.  Any step keeps the screen sound: every box still bounds its
// whole segment, so the network only trades boxes against candidates.
#include <cuda_bf16.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "scd_internal.cuh"

namespace scd {

constexpr int kIn = SCD_STEPNET_IN, kHid = SCD_STEPNET_HIDDEN;
constexpr int kOffW1 = 0, kOffB1 = kIn * kHid, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kHid, kParams = kOffB3 + 1;
static_assert(kParams == SCD_STEPNET_PARAMS, "parameter count");

// ---------------------------------------------------------------------------
// Features of one object, FP32 from the FP64 elements: log(a/R_E), e, sin i,
// cos i, log of perigee and apogee altitude / 100 km, log(P / 1 h), and
// log(1 + number of other objects whose semi-major axis is within 50 km).
// ---------------------------------------------------------------------------
__global__ void k_features(const scd_element *__restrict__ el, int64_t n,
                           const unsigned long long *__restrict__ asorted,
                           float *__restrict__ feat) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  scd_element x = el[i];
  double a = x.a_km, e = x.e;
  double hp = fmax(a * (1.0 - e) - kRe, 1.0), ha = fmax(a * (1.0 + e) - kRe, 1.0);
  double P = kTwoPi * sqrt(a * a * a / kMu);
  // neighbours in semi-major axis: two binary searches in the sorted axes
  double lo_a = a - 50.0, hi_a = a + 50.0;
  int64_t l = 0, h = n;
  while (l < h) {
    int64_t m = (l + h) >> 1;
    if (__longlong_as_double((long long)asorted[m]) < lo_a) l = m + 1; else h = m;
  }
  int64_t first = l;
  l = 0;
  h = n;
  while (l < h) {
    int64_t m = (l + h) >> 1;
    if (__longlong_as_double((long long)asorted[m]) <= hi_a) l = m + 1; else h = m;
  }
  double dens = (double)(l - first - 1);
  float *f = feat + kIn * i;
  f[0] = (float)log(a / kRe);
  f[1] = (float)e;
  f[2] = (float)sin(x.inc_rad);
  f[3] = (float)cos(x.inc_rad);
  f[4] = (float)log(hp / 100.0);
  f[5] = (float)log(ha / 100.0);
  f[6] = (float)log(P / 3600.0);
  f[7] = (float)log1p(fmax(dens, 0.0));
}

__global__ void k_axis_bits(const scd_element *__restrict__ el, int64_t n,
                            unsigned long long *__restrict__ abits) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) abits[i] = (unsigned long long)__double_as_longlong(el[i].a_km);
}

// ---------------------------------------------------------------------------
// Forward pass, one thread per sample; weights in shared memory as BF16.
// ---------------------------------------------------------------------------
struct NetView {
  const __nv_bfloat16 *w1, *w2, *w3;  // BF16 copies
  const float *p;                     // FP32 masters (biases read from here)
};

__global__ void __launch_bounds__(128) k_forward(NetView net, const float *__restrict__ X, int64_t n,
                                                 float *__restrict__ Y) {
  __shared__ __nv_bfloat16 w1[kIn * kHid], w2[kHid * kHid], w3[kHid];
  __shared__ float b1[kHid], b2[kHid];
  for (int k = threadIdx.x; k < kIn * kHid; k += blockDim.x) w1[k] = net.w1[k];
  for (int k = threadIdx.x; k < kHid * kHid; k += blockDim.x) w2[k] = net.w2[k];
  for (int k = threadIdx.x; k < kHid; k += blockDim.x) {
    w3[k] = net.w3[k];
    b1[k] = net.p[kOffB1 + k];
    b2[k] = net.p[kOffB2 + k];
  }
  __syncthreads();
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  float x[kIn];
#pragma unroll
  for (int k = 0; k < kIn; ++k) x[k] = X[kIn * s + k];
  float h1[kHid];
#pragma unroll 8
  for (int j = 0; j < kHid; ++j) {
    float acc = b1[j];
#pragma unroll
    for (int k = 0; k < kIn; ++k) acc = fmaf(x[k], __bfloat162float(w1[k * kHid + j]), acc);
    h1[j] = fmaxf(acc, 0.f);
  }
  float y = net.p[kOffB3];
  for (int j = 0; j < kHid; ++j) {
    float acc = b2[j];
#pragma unroll 16
    for (int k = 0; k < kHid; ++k) acc = fmaf(h1[k], __bfloat162float(w2[k * kHid + j]), acc);
    y = fmaf(fmaxf(acc, 0.f), __bfloat162float(w3[j]), y);
  }
  Y[s] = y;
}

// ---------------------------------------------------------------------------
// Forward + backward of the mean squared error over n samples.  One block of
// 128 threads owns 128 samples: activations and their gradients live in
// shared memory, and each block's weight gradients (reductions over its
// samples) are added to the global FP32 gradient with atomics.
// ---------------------------------------------------------------------------
constexpr int kTB = 128;
constexpr int kLd = kHid + 1;  // padded row: a thread walks its own row bank-free

__global__ void __launch_bounds__(kTB) k_fwd_bwd(NetView net, const float *__restrict__ X,
                                                 const float *__restrict__ T, int64_t n,
                                                 float inv_n, float *__restrict__ grad,
                                                 float *__restrict__ loss) {
  extern __shared__ float sm[];
  float *H1 = sm;                  // [kTB][kLd]
  float *H2 = H1 + kTB * kLd;      // [kTB][kLd], later dL/dpre2
  float *D1 = H2 + kTB * kLd;      // [kTB][kLd]  dL/dpre1
  float *W2 = D1 + kTB * kLd;      // [kHid][kHid] as float
  float *W1 = W2 + kHid * kHid;    // [kIn][kHid]
  float *Xs = W1 + kIn * kHid;     // [kTB][kIn]
  float *dy = Xs + kTB * kIn;      // [kTB]
  float *w3 = dy + kTB;            // [kHid]
  const int t = threadIdx.x;
  for (int k = t; k < kHid * kHid; k += kTB) W2[k] = __bfloat162float(net.w2[k]);
  for (int k = t; k < kIn * kHid; k += kTB) W1[k] = __bfloat162float(net.w1[k]);
  for (int k = t; k < kHid; k += kTB) w3[k] = __bfloat162float(net.w3[k]);
  const int64_t s = (int64_t)blockIdx.x * kTB + t;
  const bool valid = s < n;
#pragma unroll
  for (int k = 0; k < kIn; ++k) Xs[t * kIn + k] = valid ? X[kIn * s + k] : 0.f;
  __syncthreads();
  // forward
  float *h1 = H1 + t * kLd, *h2 = H2 + t * kLd, *d1 = D1 + t * kLd;
  for (int j = 0; j < kHid; ++j) {
    float acc = net.p[kOffB1 + j];
#pragma unroll
    for (int k = 0; k < kIn; ++k) acc = fmaf(Xs[t * kIn + k], W1[k * kHid + j], acc);
    h1[j] = fmaxf(acc, 0.f);
  }
  float y = net.p[kOffB3];
  for (int j = 0; j < kHid; ++j) {
    float acc = net.p[kOffB2 + j];
    for (int k = 0; k < kHid; ++k) acc = fmaf(h1[k], W2[k * kHid + j], acc);
    h2[j] = fmaxf(acc, 0.f);
    y = fmaf(h2[j], w3[j], y);
  }
  float r = valid ? y - T[s] : 0.f;
  dy[t] = 2.f * r * inv_n;
  // loss: one atomic per warp
  float l2 = r * r * inv_n;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l2 += __shfl_down_sync(0xffffffffu, l2, o);
  if ((t & 31) == 0) atomicAdd(loss, l2);
  __syncthreads();
  // output layer: dw3[j] = sum_t dy h2, db3 = sum_t dy
  if (t < kHid) {
    float acc = 0.f;
    for (int q = 0; q < kTB; ++q) acc = fmaf(dy[q], H2[q * kLd + t], acc);
    atomicAdd(grad + kOffW3 + t, acc);
  }
  if (t == kHid) {
    float acc = 0.f;
    for (int q = 0; q < kTB; ++q) acc += dy[q];
    atomicAdd(grad + kOffB3, acc);
  }
  __syncthreads();
  // dL/dpre2 in place of h2
  for (int j = 0; j < kHid; ++j) h2[j] = h2[j] > 0.f ? dy[t] * w3[j] : 0.f;
  __syncthreads();
  // dW2[k][j] = sum_t h1[t][k] dpre2[t][j]; db2[j] = sum_t dpre2[t][j]
  for (int e = t; e < kHid * kHid; e += kTB) {
    int k = e / kHid, j = e % kHid;
    float acc = 0.f;
    for (int q = 0; q < kTB; ++q) acc = fmaf(H1[q * kLd + k], H2[q * kLd + j], acc);
    atomicAdd(grad + kOffW2 + e, acc);
  }
  if (t < kHid) {
    float acc = 0.f;
    for (int q = 0; q < kTB; ++q) acc += H2[q * kLd + t];
    atomicAdd(grad + kOffB2 + t, acc);
  }
  // dL/dpre1[t][k] = (sum_j dpre2[t][j] W2[k][j]) * [h1 > 0]
  for (int k = 0; k < kHid; ++k) {
    float acc = 0.f;
    for (int j = 0; j < kHid; ++j) acc = fmaf(h2[j], W2[k * kHid + j], acc);
    d1[k] = h1[k] > 0.f ? acc : 0.f;
  }
  __syncthreads();
  // dW1[k][j] = sum_t x[t][k] dpre1[t][j]; db1[j] = sum_t dpre1[t][j]
  for (int e = t; e < kIn * kHid; e += kTB) {
    int k = e / kHid, j = e % kHid;
    float acc = 0.f;
    for (int q = 0; q < kTB; ++q) acc = fmaf(Xs[q * kIn + k], D1[q * kLd + j], acc);
    atomicAdd(grad + kOffW1 + e, acc);
  }
  if (t < kHid) {
    float acc = 0.f;
    for (int q = 0; q < kTB; ++q) acc += D1[q * kLd + t];
    atomicAdd(grad + kOffB1 + t, acc);
  }
}

constexpr size_t kFwdBwdSmem =
    sizeof(float) * (3 * kTB * kLd + kHid * kHid + kIn * kHid + kTB * kIn + kTB + kHid);

// AdamW on the FP32 masters, then the BF16 copies used by the forward pass
__global__ void k_adamw(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                        float *__restrict__ v, int step, float lr, float b1, float b2, float eps,
                        float wd, __nv_bfloat16 *__restrict__ w1, __nv_bfloat16 *__restrict__ w2,
                        __nv_bfloat16 *__restrict__ w3) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kParams) return;
  float gk = g[k];
  float mk = b1 * m[k] + (1.f - b1) * gk;
  float vk = b2 * v[k] + (1.f - b2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  float mh = mk / (1.f - powf(b1, (float)step));
  float vh = vk / (1.f - powf(b2, (float)step));
  bool is_weight = (k < kOffB1) || (k >= kOffW2 && k < kOffB2) || (k >= kOffW3 && k < kOffB3);
  float pk = p[k];
  if (is_weight) pk -= lr * wd * pk;  // decoupled weight decay (weights only)
  pk -= lr * mh / (sqrtf(vh) + eps);
  p[k] = pk;
  if (k < kOffB1) w1[k - kOffW1] = __float2bfloat16_rn(pk);
  else if (k >= kOffW2 && k < kOffB2) w2[k - kOffW2] = __float2bfloat16_rn(pk);
  else if (k >= kOffW3 && k < kOffB3) w3[k - kOffW3] = __float2bfloat16_rn(pk);
}

__global__ void k_refresh_bf16(const float *__restrict__ p, __nv_bfloat16 *__restrict__ w1,
                               __nv_bfloat16 *__restrict__ w2, __nv_bfloat16 *__restrict__ w3) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < kIn * kHid) w1[k] = __float2bfloat16_rn(p[kOffW1 + k]);
  if (k < kHid * kHid) w2[k] = __float2bfloat16_rn(p[kOffW2 + k]);
  if (k < kHid) w3[k] = __float2bfloat16_rn(p[kOffW3 + k]);
}

// per-object learned step [s]: exp of the network output, clamped to
// [P/400, P/50]
__global__ void k_learned_steps(const scd_element *__restrict__ el, const float *__restrict__ y,
                                int64_t n, float *__restrict__ ks) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a = el[i].a_km;
  double P = kTwoPi * sqrt(a * a * a / kMu);
  double k = exp((double)y[i]);
  k = fmin(fmax(k, P / 400.0), P / 50.0);
  ks[i] = (float)k;
}

}  // namespace scd

using namespace scd;

struct scd_stepnet {
  cudaStream_t stream = nullptr;
  DevBuf<float> p, g, m, v, loss;
  DevBuf<__nv_bfloat16> w1, w2, w3;
  int step = 0;
  float *h_loss = nullptr;
};

static int net_ok(const scd_stepnet *n) { return n && n->p.p; }

static NetView view(const scd_stepnet *n) {
  NetView v;
  v.w1 = n->w1.p;
  v.w2 = n->w2.p;
  v.w3 = n->w3.p;
  v.p = n->p.p;
  return v;
}

static int refresh(scd_stepnet *n) {
  k_refresh_bf16<<<(kHid * kHid + 255) / 256, 256, 0, n->stream>>>(n->p.p, n->w1.p, n->w2.p,
                                                                   n->w3.p);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? SCD_OK : SCD_ERR_CUDA;
}

extern "C" SCD_API int scd_stepnet_create(void *cuda_stream, uint64_t seed, scd_stepnet **out) {
  if (!out) return SCD_ERR_INVALID_ARG;
  *out = nullptr;
  scd_stepnet *n = new scd_stepnet();
  n->stream = (cudaStream_t)cuda_stream;
  cudaStream_t st = n->stream;
  if (!n->p.ensure(kParams, st) || !n->g.ensure(kParams, st) || !n->m.ensure(kParams, st) ||
      !n->v.ensure(kParams, st) || !n->loss.ensure(1, st) || !n->w1.ensure(kIn * kHid, st) ||
      !n->w2.ensure(kHid * kHid, st) || !n->w3.ensure(kHid, st) ||
      cudaMallocHost(&n->h_loss, sizeof(float)) != cudaSuccess) {
    scd_stepnet_destroy(n);
    return SCD_ERR_OOM;
  }
  // He-style initialisation from a host counter-based generator (splitmix64)
  std::vector<float> h(kParams, 0.f);
  uint64_t x = seed;
  auto uni = [&x]() {
    x += 0x9e3779b97f4a7c15ull;
    uint64_t z = x;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  };
  for (int k = 0; k < kIn * kHid; ++k) h[kOffW1 + k] = (float)((2 * uni() - 1) * sqrt(6.0 / kIn));
  for (int k = 0; k < kHid * kHid; ++k) h[kOffW2 + k] = (float)((2 * uni() - 1) * sqrt(6.0 / kHid));
  for (int k = 0; k < kHid; ++k) h[kOffW3 + k] = (float)((2 * uni() - 1) * sqrt(3.0 / kHid));
  int rc = scd_stepnet_set_params(n, h.data(), kParams);
  if (rc) {
    scd_stepnet_destroy(n);
    return rc;
  }
  *out = n;
  return SCD_OK;
}

extern "C" SCD_API int scd_stepnet_set_params(scd_stepnet *n, const float *host_params,
                                              int64_t count) {
  if (!net_ok(n) || !host_params || count != kParams) return SCD_ERR_INVALID_ARG;
  cudaStream_t st = n->stream;
  if (cudaMemcpyAsync(n->p.p, host_params, sizeof(float) * kParams, cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemsetAsync(n->m.p, 0, sizeof(float) * kParams, st) != cudaSuccess ||
      cudaMemsetAsync(n->v.p, 0, sizeof(float) * kParams, st) != cudaSuccess)
    return SCD_ERR_CUDA;
  n->step = 0;
  int rc = refresh(n);
  if (rc) return rc;
  return cudaStreamSynchronize(st) == cudaSuccess ? SCD_OK : SCD_ERR_CUDA;
}

extern "C" SCD_API int scd_stepnet_get_params(const scd_stepnet *n, float *host_params,
                                              int64_t count) {
  if (!net_ok(n) || !host_params || count != kParams) return SCD_ERR_INVALID_ARG;
  if (cudaMemcpyAsync(host_params, n->p.p, sizeof(float) * kParams, cudaMemcpyDeviceToHost,
                      n->stream) != cudaSuccess)
    return SCD_ERR_CUDA;
  return cudaStreamSynchronize(n->stream) == cudaSuccess ? SCD_OK : SCD_ERR_CUDA;
}

extern "C" SCD_API int scd_stepnet_features(const scd_element *d_elems, int64_t n, float *d_feat,
                                            void *cuda_stream) {
  if (!d_elems || n <= 0 || !d_feat) return SCD_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  DevBuf<unsigned long long> ab;
  SortScratch sc;
  if (!ab.ensure(n, st)) return SCD_ERR_OOM;
  k_axis_bits<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d_elems, n, ab.p);
  note_launch();
  int rc = radix_sort_u64(ab.p, nullptr, n, 64, sc, st);
  if (rc == SCD_OK) {
    k_features<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d_elems, n, ab.p, d_feat);
    note_launch();
    rc = cudaGetLastError() == cudaSuccess ? SCD_OK : SCD_ERR_CUDA;
  }
  cudaStreamSynchronize(st);
  ab.release(st);
  sc.release(st);
  return rc;
}

extern "C" SCD_API int scd_stepnet_forward(const scd_stepnet *n, const float *d_x, int64_t count,
                                           float *d_y) {
  if (!net_ok(n) || !d_x || !d_y || count < 0) return SCD_ERR_INVALID_ARG;
  if (count == 0) return SCD_OK;
  k_forward<<<(unsigned)((count + 127) / 128), 128, 0, n->stream>>>(view(n), d_x, count, d_y);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? SCD_OK : SCD_ERR_CUDA;
}

static int fwd_bwd(scd_stepnet *n, const float *d_x, const float *d_t, int64_t count) {
  cudaStream_t st = n->stream;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_fwd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdBwdSmem);
    attr = true;
  }
  if (cudaMemsetAsync(n->g.p, 0, sizeof(float) * kParams, st) != cudaSuccess ||
      cudaMemsetAsync(n->loss.p, 0, sizeof(float), st) != cudaSuccess)
    return SCD_ERR_CUDA;
  k_fwd_bwd<<<(unsigned)((count + kTB - 1) / kTB), kTB, kFwdBwdSmem, st>>>(
      view(n), d_x, d_t, count, 1.0f / (float)count, n->g.p, n->loss.p);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? SCD_OK : SCD_ERR_CUDA;
}

extern "C" SCD_API int scd_stepnet_grad(scd_stepnet *n, const float *d_x, const float *d_t,
                                        int64_t count, float *d_grad, float *loss_out) {
  if (!net_ok(n) || !d_x || !d_t || !d_grad || count <= 0) return SCD_ERR_INVALID_ARG;
  int rc = fwd_bwd(n, d_x, d_t, count);
  if (rc) return rc;
  cudaStream_t st = n->stream;
  if (cudaMemcpyAsync(d_grad, n->g.p, sizeof(float) * kParams, cudaMemcpyDeviceToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(n->h_loss, n->loss.p, sizeof(float), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SCD_ERR_CUDA;
  if (loss_out) *loss_out = *n->h_loss;
  return SCD_OK;
}

extern "C" SCD_API int scd_stepnet_train_step(scd_stepnet *n, const float *d_x, const float *d_t,
                                              int64_t count, float lr, float weight_decay,
                                              float *loss_out) {
  if (!net_ok(n) || !d_x || !d_t || count <= 0 || !(lr > 0.f) || weight_decay < 0.f)
    return SCD_ERR_INVALID_ARG;
  int rc = fwd_bwd(n, d_x, d_t, count);
  if (rc) return rc;
  n->step += 1;
  k_adamw<<<(kParams + 255) / 256, 256, 0, n->stream>>>(n->p.p, n->g.p, n->m.p, n->v.p, n->step,
                                                        lr, 0.9f, 0.999f, 1e-8f, weight_decay,
                                                        n->w1.p, n->w2.p, n->w3.p);
  note_launch();
  if (cudaGetLastError() != cudaSuccess) return SCD_ERR_CUDA;
  if (loss_out) {
    if (cudaMemcpyAsync(n->h_loss, n->loss.p, sizeof(float), cudaMemcpyDeviceToHost, n->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(n->stream) != cudaSuccess)
      return SCD_ERR_CUDA;
    *loss_out = *n->h_loss;
  }
  return SCD_OK;
}

// checkpoint: 8-byte magic, version, parameter count, AdamW step, then the
// FP32 master parameters
static const char kMagic[8] = {'S', 'C', 'D', 'N', 'E', 'T', '0', '1'};

extern "C" SCD_API int scd_stepnet_save(const scd_stepnet *n, const char *path) {
  if (!net_ok(n) || !path) return SCD_ERR_INVALID_ARG;
  std::vector<float> h(kParams);
  int rc = scd_stepnet_get_params(n, h.data(), kParams);
  if (rc) return rc;
  FILE *f = fopen(path, "wb");
  if (!f) return SCD_ERR_INVALID_ARG;
  int32_t hdr[3] = {1, kParams, n->step};
  bool ok = fwrite(kMagic, 1, 8, f) == 8 && fwrite(hdr, sizeof(int32_t), 3, f) == 3 &&
            fwrite(h.data(), sizeof(float), kParams, f) == (size_t)kParams;
  ok = (fclose(f) == 0) && ok;
  return ok ? SCD_OK : SCD_ERR_INVALID_ARG;
}

extern "C" SCD_API int scd_stepnet_load(scd_stepnet *n, const char *path) {
  if (!net_ok(n) || !path) return SCD_ERR_INVALID_ARG;
  FILE *f = fopen(path, "rb");
  if (!f) return SCD_ERR_INVALID_ARG;
  char mg[8];
  int32_t hdr[3];
  std::vector<float> h(kParams);
  bool ok = fread(mg, 1, 8, f) == 8 && memcmp(mg, kMagic, 8) == 0 &&
            fread(hdr, sizeof(int32_t), 3, f) == 3 && hdr[0] == 1 && hdr[1] == kParams &&
            fread(h.data(), sizeof(float), kParams, f) == (size_t)kParams;
  fclose(f);
  if (!ok) return SCD_ERR_INVALID_ARG;
  return scd_stepnet_set_params(n, h.data(), kParams);
}

extern "C" SCD_API void scd_stepnet_destroy(scd_stepnet *n) {
  if (!n) return;
  cudaStream_t st = n->stream;
  cudaStreamSynchronize(st);
  n->p.release(st); n->g.release(st); n->m.release(st); n->v.release(st); n->loss.release(st);
  n->w1.release(st); n->w2.release(st); n->w3.release(st);
  if (n->h_loss) cudaFreeHost(n->h_loss);
  delete n;
}

namespace scd {
// learned steps [s] of a scene's objects (LEARNED policy), into s->d_learned
int learned_steps(scd_scene *s) {
  const scd_stepnet *net = (const scd_stepnet *)s->stepnet;
  if (!net_ok(net)) return SCD_ERR_INVALID_ARG;
  cudaStream_t st = s->stream;
  if (!s->d_feat.ensure((size_t)kIn * s->n, st) || !s->d_learned.ensure(s->n, st) ||
      !s->d_ny.ensure(s->n, st))
    return SCD_ERR_OOM;
  int rc = scd_stepnet_features(s->d_el.p, s->n, s->d_feat.p, (void *)st);
  if (rc) return rc;
  // the network runs on the scene's stream
  k_forward<<<(unsigned)((s->n + 127) / 128), 128, 0, st>>>(view(net), s->d_feat.p, s->n,
                                                           s->d_ny.p);
  k_learned_steps<<<(unsigned)((s->n + 255) / 256), 256, 0, st>>>(s->d_el.p, s->d_ny.p, s->n,
                                                                   s->d_learned.p);
  note_launch(2);
  return cudaGetLastError() == cudaSuccess ? SCD_OK : SCD_ERR_CUDA;
}
}  // namespace scd

namespace scd {
__global__ void k_count_per_object(const scd_pair *__restrict__ pr, int64_t n, int64_t nobj,
                                   uint32_t *__restrict__ cnt) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  scd_pair q = pr[k];
  if ((int64_t)q.i < nobj) atomicAdd(cnt + q.i, 1u);
  if ((int64_t)q.j < nobj) atomicAdd(cnt + q.j, 1u);
}
}  // namespace scd

extern "C" SCD_API int scd_count_pairs_per_object(const scd_pair *d_pairs, int64_t n_pairs,
                                                  int64_t n_objects, uint32_t *d_counts,
                                                  void *cuda_stream) {
  if (n_pairs < 0 || n_objects <= 0 || !d_counts || (n_pairs > 0 && !d_pairs))
    return SCD_ERR_INVALID_ARG;
  if (n_pairs == 0) return SCD_OK;
  k_count_per_object<<<(unsigned)((n_pairs + 255) / 256), 256, 0, (cudaStream_t)cuda_stream>>>(
      d_pairs, n_pairs, n_objects, d_counts);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? SCD_OK : SCD_ERR_CUDA;
}
