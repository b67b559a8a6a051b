// mlp.cu -- the small FP32 network that proposes (m, s): forward, softmax
// cross-entropy with its gradient, and Adam, as plain CUDA kernels.
//
// Network: in -> hidden (ReLU) -> hidden (ReLU) -> out logits. Parameters are one
// flat float array: W1[hidden][in], b1[hidden], W2[hidden][hidden], b2[hidden],
// W3[out][hidden], b3[out] (row-major). The layers are tiny (5 -> 64 -> 64 -> 60),
// so each kernel maps one thread to one output element; weight gradients sum
// over the batch in a fixed order (deterministic, no atomics).
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace bbc {
namespace {

// Y[b][o] = act(sum_i X[b][i] W[o][i] + bias[o])
__global__ void k_linear_fwd(const float* __restrict__ X, const float* __restrict__ Wt, const float* __restrict__ bias,
                             int64_t B, int n_in, int n_out, int relu, float* __restrict__ Z,
                             float* __restrict__ H) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * n_out) return;
  const int64_t b = t / n_out;
  const int o = (int)(t % n_out);
  float acc = bias[o];
  for (int i = 0; i < n_in; ++i) acc = fmaf(X[b * n_in + i], Wt[(int64_t)o * n_in + i], acc);
  if (Z) Z[t] = acc;
  H[t] = (relu && acc < 0.f) ? 0.f : acc;
}

// G[b][k] = (softmax(logits[b])_k - [k == y_b]) / B ; loss[b] = -log softmax(logits[b])_{y_b}
__global__ void k_softmax_ce(const float* __restrict__ L, const int* __restrict__ y, int64_t B, int K,
                             float* __restrict__ G, float* __restrict__ loss) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float* l = L + b * K;
  float mx = l[0];
  for (int k = 1; k < K; ++k) mx = fmaxf(mx, l[k]);
  float sum = 0.f;
  for (int k = 0; k < K; ++k) sum += expf(l[k] - mx);
  const int yb = y[b];
  for (int k = 0; k < K; ++k) G[b * K + k] = (expf(l[k] - mx) / sum - (k == yb ? 1.f : 0.f)) / (float)B;
  loss[b] = -(l[yb] - mx - logf(sum));
}

// gW[o][i] = sum_b D[b][o] H[b][i] ; gb[o] = sum_b D[b][o]  (thread per (o, i), i == n_in -> bias)
__global__ void k_grad_weight(const float* __restrict__ D, const float* __restrict__ H, int64_t B, int n_in,
                              int n_out, float* __restrict__ gW, float* __restrict__ gb) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_out * (n_in + 1)) return;
  const int o = t / (n_in + 1), i = t % (n_in + 1);
  float acc = 0.f;
  if (i < n_in)
    for (int64_t b = 0; b < B; ++b) acc = fmaf(D[b * n_out + o], H[b * n_in + i], acc);
  else
    for (int64_t b = 0; b < B; ++b) acc += D[b * n_out + o];
  if (i < n_in) gW[(int64_t)o * n_in + i] = acc; else gb[o] = acc;
}

// Dp[b][i] = (sum_o W[o][i] D[b][o]) * [Zp[b][i] > 0]
__global__ void k_backprop(const float* __restrict__ D, const float* __restrict__ Wt, const float* __restrict__ Zp,
                           int64_t B, int n_in, int n_out, float* __restrict__ Dp) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * n_in) return;
  const int64_t b = t / n_in;
  const int i = (int)(t % n_in);
  float acc = 0.f;
  for (int o = 0; o < n_out; ++o) acc = fmaf(Wt[(int64_t)o * n_in + i], D[b * n_out + o], acc);
  Dp[t] = Zp[t] > 0.f ? acc : 0.f;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

unsigned blocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int64_t mlp_param_count(int n_in, int hid, int n_out) {
  return (int64_t)hid * n_in + hid + (int64_t)hid * hid + hid + (int64_t)n_out * hid + n_out;
}

int64_t mlp_workspace_floats(int hid, int n_out, int64_t B) { return B * (6 * (int64_t)hid + 2 * n_out); }

// Workspace layout (floats): Z1, H1, Z2, H2 [B][hid], logits [B][out], G [B][out], D2, D1 [B][hid].
struct MlpWs {
  float *z1, *h1, *z2, *h2, *lg, *g, *d2, *d1;
};
static MlpWs ws_layout(float* w, int hid, int n_out, int64_t B) {
  MlpWs s;
  s.z1 = w;
  s.h1 = s.z1 + B * hid;
  s.z2 = s.h1 + B * hid;
  s.h2 = s.z2 + B * hid;
  s.lg = s.h2 + B * hid;
  s.g = s.lg + B * n_out;
  s.d2 = s.g + B * n_out;
  s.d1 = s.d2 + B * hid;
  return s;
}

cudaError_t mlp_forward(const float* P, int n_in, int hid, int n_out, const float* X, int64_t B, float* logits,
                        float* ws, cudaStream_t st) {
  const float *W1 = P, *b1 = W1 + (int64_t)hid * n_in, *W2 = b1 + hid, *b2 = W2 + (int64_t)hid * hid;
  const float *W3 = b2 + hid, *b3 = W3 + (int64_t)n_out * hid;
  MlpWs s = ws_layout(ws, hid, n_out, B);
  k_linear_fwd<<<blocks(B * hid), 256, 0, st>>>(X, W1, b1, B, n_in, hid, 1, s.z1, s.h1);
  k_linear_fwd<<<blocks(B * hid), 256, 0, st>>>(s.h1, W2, b2, B, hid, hid, 1, s.z2, s.h2);
  k_linear_fwd<<<blocks(B * n_out), 256, 0, st>>>(s.h2, W3, b3, B, hid, n_out, 0, nullptr, logits ? logits : s.lg);
  return cudaGetLastError();
}

cudaError_t mlp_grad(const float* P, int n_in, int hid, int n_out, const float* X, const int* y, int64_t B,
                     float* grad, float* loss, float* ws, cudaStream_t st) {
  cudaError_t e = mlp_forward(P, n_in, hid, n_out, X, B, nullptr, ws, st);
  if (e != cudaSuccess) return e;
  const float *W2 = P + (int64_t)hid * n_in + hid, *W3 = W2 + (int64_t)hid * hid + hid;
  float *gW1 = grad, *gb1 = gW1 + (int64_t)hid * n_in, *gW2 = gb1 + hid, *gb2 = gW2 + (int64_t)hid * hid;
  float *gW3 = gb2 + hid, *gb3 = gW3 + (int64_t)n_out * hid;
  MlpWs s = ws_layout(ws, hid, n_out, B);
  k_softmax_ce<<<blocks(B), 256, 0, st>>>(s.lg, y, B, n_out, s.g, loss);
  k_grad_weight<<<blocks((int64_t)n_out * (hid + 1)), 256, 0, st>>>(s.g, s.h2, B, hid, n_out, gW3, gb3);
  k_backprop<<<blocks(B * hid), 256, 0, st>>>(s.g, W3, s.z2, B, hid, n_out, s.d2);
  k_grad_weight<<<blocks((int64_t)hid * (hid + 1)), 256, 0, st>>>(s.d2, s.h1, B, hid, hid, gW2, gb2);
  k_backprop<<<blocks(B * hid), 256, 0, st>>>(s.d2, W2, s.z1, B, hid, hid, s.d1);
  k_grad_weight<<<blocks((int64_t)hid * (n_in + 1)), 256, 0, st>>>(s.d1, X, B, n_in, hid, gW1, gb1);
  return cudaGetLastError();
}

cudaError_t mlp_adam(float* P, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2,
                     float eps, int step, cudaStream_t st) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_adam<<<blocks(n), 256, 0, st>>>(P, g, m, v, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

}  // namespace bbc
