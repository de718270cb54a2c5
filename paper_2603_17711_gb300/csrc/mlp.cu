// Learned rank proposer of the adaptive (ps2) sweeps: a 24-64-64-13 MLP with
// hand-written FP32 forward, backward and Adam kernels, plus the FP64 kernels
// of the randomised truncated factorisation a proposal is checked with.
//
// Network: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), z = W3 h2 + b3, loss =
// mean softmax cross-entropy; parameters packed W1, b1, W2, b2, W3, b3
// (row-major, output index first). Every reduction over the batch runs in a
// fixed order (one thread per parameter), so training is bitwise reproducible.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/ttn_heom.h"
#include "kernels.cuh"

namespace ttn {

constexpr int kIn = 24, kH = 64, kOut = 13;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kIn, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kOut * kH, kNParams = kOffB3 + kOut;
constexpr int kSamplesPerCta = 4;

// workspace (floats): h1[B*64], h2[B*64], z[B*13], dz[B*13], d2[B*64], d1[B*64], lossb[B]
size_t mlp_ws_floats(int B) { return (size_t)B * (kH + kH + kOut + kOut + kH + kH + 1); }

__global__ void k_mlp_fwd(const float* __restrict__ P, const float* __restrict__ x, int B, float* h1g, float* h2g,
                          float* zg) {
  __shared__ float sx[kSamplesPerCta][kIn], s1[kSamplesPerCta][kH], s2[kSamplesPerCta][kH];
  const int b0 = blockIdx.x * kSamplesPerCta, tid = threadIdx.x;
  for (int k = tid; k < kSamplesPerCta * kIn; k += blockDim.x) {
    const int s = k / kIn, i = k % kIn;
    sx[s][i] = b0 + s < B ? x[(int64_t)(b0 + s) * kIn + i] : 0.f;
  }
  __syncthreads();
  for (int k = tid; k < kSamplesPerCta * kH; k += blockDim.x) {
    const int s = k / kH, o = k % kH;
    float a = P[kOffB1 + o];
    for (int i = 0; i < kIn; ++i) a = fmaf(P[kOffW1 + o * kIn + i], sx[s][i], a);
    s1[s][o] = fmaxf(a, 0.f);
  }
  __syncthreads();
  for (int k = tid; k < kSamplesPerCta * kH; k += blockDim.x) {
    const int s = k / kH, o = k % kH;
    float a = P[kOffB2 + o];
    for (int i = 0; i < kH; ++i) a = fmaf(P[kOffW2 + o * kH + i], s1[s][i], a);
    s2[s][o] = fmaxf(a, 0.f);
  }
  __syncthreads();
  for (int k = tid; k < kSamplesPerCta * kOut; k += blockDim.x) {
    const int s = k / kOut, o = k % kOut;
    float a = P[kOffB3 + o];
    for (int i = 0; i < kH; ++i) a = fmaf(P[kOffW3 + o * kH + i], s2[s][i], a);
    if (b0 + s < B) zg[(int64_t)(b0 + s) * kOut + o] = a;
  }
  for (int k = tid; k < kSamplesPerCta * kH; k += blockDim.x) {
    const int s = k / kH, o = k % kH;
    if (b0 + s < B) {
      if (h1g) h1g[(int64_t)(b0 + s) * kH + o] = s1[s][o];
      if (h2g) h2g[(int64_t)(b0 + s) * kH + o] = s2[s][o];
    }
  }
}

// per sample: dz = (softmax(z) - onehot(y)) / B, loss_b, d2 = (dz W3) * [h2 > 0], d1 = (d2 W2) * [h1 > 0]
__global__ void k_mlp_back(const float* __restrict__ P, const int* __restrict__ y, int B, const float* h1g,
                           const float* h2g, const float* zg, float* dzg, float* d2g, float* d1g, float* lossb) {
  __shared__ float sdz[kSamplesPerCta][kOut], sd2[kSamplesPerCta][kH];
  const int b0 = blockIdx.x * kSamplesPerCta, tid = threadIdx.x;
  if (tid < kSamplesPerCta) {
    const int b = b0 + tid;
    if (b < B) {
      const float* z = zg + (int64_t)b * kOut;
      float zm = z[0];
      for (int o = 1; o < kOut; ++o) zm = fmaxf(zm, z[o]);
      float se = 0.f;
      for (int o = 0; o < kOut; ++o) se += expf(z[o] - zm);
      const int yb = y[b];
      lossb[b] = logf(se) + zm - z[yb];
      for (int o = 0; o < kOut; ++o) {
        const float d = (expf(z[o] - zm) / se - (o == yb ? 1.f : 0.f)) / (float)B;
        sdz[tid][o] = d;
        dzg[(int64_t)b * kOut + o] = d;
      }
    } else {
      for (int o = 0; o < kOut; ++o) sdz[tid][o] = 0.f;
    }
  }
  __syncthreads();
  for (int k = tid; k < kSamplesPerCta * kH; k += blockDim.x) {
    const int s = k / kH, i = k % kH, b = b0 + s;
    float a = 0.f;
    for (int o = 0; o < kOut; ++o) a = fmaf(sdz[s][o], P[kOffW3 + o * kH + i], a);
    const float v = (b < B && h2g[(int64_t)b * kH + i] > 0.f) ? a : 0.f;
    sd2[s][i] = v;
    if (b < B) d2g[(int64_t)b * kH + i] = v;
  }
  __syncthreads();
  for (int k = tid; k < kSamplesPerCta * kH; k += blockDim.x) {
    const int s = k / kH, i = k % kH, b = b0 + s;
    float a = 0.f;
    for (int o = 0; o < kH; ++o) a = fmaf(sd2[s][o], P[kOffW2 + o * kH + i], a);
    if (b < B) d1g[(int64_t)b * kH + i] = h1g[(int64_t)b * kH + i] > 0.f ? a : 0.f;
  }
}

// one thread per parameter, fixed-order sum over the batch
__global__ void k_mlp_wgrad(const float* __restrict__ x, int B, const float* h1g, const float* h2g, const float* dzg,
                            const float* d2g, const float* d1g, const float* lossb, float* G, float* loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0 && loss) {
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += lossb[b];
    *loss = s / (float)B;
  }
  if (p >= kNParams) return;
  const float *dout, *in;
  int nin, nout, o, i;
  bool bias;
  if (p < kOffB1) {
    dout = d1g; in = x; nin = kIn; nout = kH; o = p / kIn; i = p % kIn; bias = false;
  } else if (p < kOffW2) {
    dout = d1g; in = nullptr; nin = 0; nout = kH; o = p - kOffB1; i = 0; bias = true;
  } else if (p < kOffB2) {
    dout = d2g; in = h1g; nin = kH; nout = kH; o = (p - kOffW2) / kH; i = (p - kOffW2) % kH; bias = false;
  } else if (p < kOffW3) {
    dout = d2g; in = nullptr; nin = 0; nout = kH; o = p - kOffB2; i = 0; bias = true;
  } else if (p < kOffB3) {
    dout = dzg; in = h2g; nin = kH; nout = kOut; o = (p - kOffW3) / kH; i = (p - kOffW3) % kH; bias = false;
  } else {
    dout = dzg; in = nullptr; nin = 0; nout = kOut; o = p - kOffB3; i = 0; bias = true;
  }
  float s = 0.f;
  for (int b = 0; b < B; ++b) s = fmaf(dout[(int64_t)b * nout + o], bias ? 1.f : in[(int64_t)b * nin + i], s);
  G[p] = s;
}

__global__ void k_adam(float* P, float* M, float* V, const float* G, int n, float lr, float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const float g = G[p];
  const float m = 0.9f * M[p] + 0.1f * g;
  const float v = 0.999f * V[p] + 0.001f * g * g;
  M[p] = m;
  V[p] = v;
  P[p] -= lr * (m / c1) / (sqrtf(v / c2) + 1e-8f);
}

void launch_mlp_forward(const float* P, const float* x, int B, float* ws, float* logits, cudaStream_t s) {
  float* h1 = ws;
  float* h2 = h1 + (size_t)B * kH;
  k_mlp_fwd<<<(B + kSamplesPerCta - 1) / kSamplesPerCta, 256, 0, s>>>(P, x, B, h1, h2, logits);
}

// ---------------------------------------------------------------------------
// Randomised truncated factorisation of Theta (FP64)
// ---------------------------------------------------------------------------
// splitmix64 (Steele, Lea, Flood 2014) as a counter-based generator, two
// uniforms -> one standard complex Gaussian by Box-Muller.
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
__global__ void k_gauss(double2* O, int64_t n, uint64_t seed) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t a = splitmix64(seed ^ (2 * (uint64_t)k)), b = splitmix64(seed ^ (2 * (uint64_t)k + 1));
    const double u1 = ((a >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    const double u2 = (b >> 11) * (1.0 / 9007199254740992.0);
    const double rr = sqrt(-2.0 * log(u1)) * 0.7071067811865476;
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    O[k] = make_double2(rr * cs, rr * sn);
  }
}
void launch_gauss(double2* O, int64_t n, uint64_t seed, cudaStream_t s) {
  k_gauss<<<(int)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, s>>>(O, n, seed);
}

// C (M x N, row-major) = op(A) op(B); A is M x K (conjA: A given as K x M, use A^H),
// B is K x N row-major. One thread per output element.
__global__ void k_zgemm(const double2* A, const double2* Bm, double2* Cm, int M, int N, int K, int conjA) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)M * N;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / N), j = (int)(e % N);
    double2 acc = make_double2(0.0, 0.0);
    for (int k = 0; k < K; ++k) {
      double2 a = conjA ? A[(int64_t)k * M + i] : A[(int64_t)i * K + k];
      if (conjA) a.y = -a.y;
      const double2 b = Bm[(int64_t)k * N + j];
      acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
      acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
    }
    Cm[e] = acc;
  }
}
void launch_zgemm(const double2* A, const double2* B, double2* C, int M, int N, int K, bool conjA, cudaStream_t s) {
  const int64_t tot = (int64_t)M * N;
  k_zgemm<<<(int)std::min<int64_t>((tot + 127) / 128, 4096), 128, 0, s>>>(A, B, C, M, N, K, conjA ? 1 : 0);
}

// ||x||_2^2 in one block, fixed order
__global__ void k_norm2(const double2* x, int64_t n, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) s += x[k].x * x[k].x + x[k].y * x[k].y;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *out = t;
  }
}
void launch_norm2(const double2* x, int64_t n, double* out, cudaStream_t s) { k_norm2<<<1, 512, 0, s>>>(x, n, out); }

// Z / Cm of the randomised split. Theta ~ Q B, B (k x n) = Lb diag(sigma) Rb^H from
// the Jacobi SVD of B (computed on B^H when n > k: Lb = V (k x k), Rb_j = A_j / sigma_j).
// Left_j of Theta = Q Lb_j (length m). Layouts as in k_svd_vecs.
__global__ void k_rsvd_vecs(const double2* Q, int m, int kk, const double2* A, const double2* V, const double* sigma,
                            int n, const int* perm, int r, int g, int iso_first, double2* Z, double2* Zg, double2* Cm) {
  const bool tr = n > kk;
  const int nr = tr ? n : kk, nc = tr ? kk : n;
  const int rows_iso = iso_first ? m : n, rows_c = iso_first ? n : m;
  const int64_t nz = (int64_t)rows_iso * r, ncm = (int64_t)rows_c * r;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nz + ncm; e += (int64_t)gridDim.x * blockDim.x) {
    const bool zpart = e < nz;
    const int64_t q = zpart ? e : e - nz;
    const int a = (int)(q % r), row = (int)(q / r);
    const int j = perm[a];
    const double sj = sigma[j];
    const bool good = a < g;
    auto lb = [&](int t) -> double2 {  // Lb[t][j]
      if (tr) return V[(int64_t)j * nc + t];
      const double2 v = A[(int64_t)j * nr + t];
      return make_double2(v.x / sj, v.y / sj);
    };
    auto left = [&](int i) -> double2 {
      double2 acc = make_double2(0.0, 0.0);
      for (int t = 0; t < kk; ++t) {
        const double2 qv = Q[(int64_t)i * kk + t], l = lb(t);
        acc.x = fma(qv.x, l.x, fma(-qv.y, l.y, acc.x));
        acc.y = fma(qv.x, l.y, fma(qv.y, l.x, acc.y));
      }
      return acc;
    };
    auto right = [&](int i) -> double2 {
      if (!tr) return V[(int64_t)j * nc + i];
      const double2 v = A[(int64_t)j * nr + i];
      return make_double2(v.x / sj, v.y / sj);
    };
    double2 v = make_double2(0.0, 0.0);
    if (zpart) {
      if (good) {
        v = iso_first ? left(row) : right(row);
        if (!iso_first) v.y = -v.y;
      }
      Z[q] = v;
      Zg[q] = v;
    } else {
      if (good) {
        double2 w = iso_first ? right(row) : left(row);
        if (iso_first) w.y = -w.y;
        v = make_double2(sj * w.x, sj * w.y);
      }
      if (iso_first)
        Cm[(int64_t)a * rows_c + row] = v;
      else
        Cm[(int64_t)row * r + a] = v;
    }
  }
}
void launch_rsvd_vecs(const double2* Q, int m, int kk, const double2* A, const double2* V, const double* sigma, int n,
                      const int* perm, int r, int g, bool iso_first, double2* Z, double2* Zg, double2* Cm,
                      cudaStream_t s) {
  const int64_t tot = (int64_t)(m + n) * r;
  k_rsvd_vecs<<<(int)std::min<int64_t>((tot + 127) / 128, 2048), 128, 0, s>>>(Q, m, kk, A, V, sigma, n, perm, r, g,
                                                                           iso_first ? 1 : 0, Z, Zg, Cm);
}

}  // namespace ttn

// ---------------------------------------------------------------------------
// C ABI of the network (see include/ttn_heom.h)
// ---------------------------------------------------------------------------
extern "C" {

ttn_status ttn_mlp_n_params(int32_t* n) {
  if (!n) return TTN_EINVAL;
  *n = ttn::kNParams;
  return TTN_OK;
}

ttn_status ttn_mlp_workspace_size(int32_t batch, size_t* bytes) {
  if (!bytes || batch < 1) return TTN_EINVAL;
  *bytes = ttn::mlp_ws_floats(batch) * sizeof(float);
  return TTN_OK;
}

ttn_status ttn_mlp_forward(const float* params, const float* x, int32_t batch, float* logits, void* ws, void* stream) {
  if (!params || !x || !logits || !ws || batch < 1) return TTN_EINVAL;
  ttn::launch_mlp_forward(params, x, batch, (float*)ws, logits, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? TTN_OK : TTN_ECUDA;
}

ttn_status ttn_mlp_grad(const float* params, const float* x, const int32_t* labels, int32_t batch, float* grads,
                        float* loss, void* ws, void* stream) {
  using namespace ttn;
  if (!params || !x || !labels || !grads || !ws || batch < 1) return TTN_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int B = batch;
  float* h1 = (float*)ws;
  float* h2 = h1 + (size_t)B * kH;
  float* z = h2 + (size_t)B * kH;
  float* dz = z + (size_t)B * kOut;
  float* d2 = dz + (size_t)B * kOut;
  float* d1 = d2 + (size_t)B * kH;
  float* lb = d1 + (size_t)B * kH;
  const int nb = (B + kSamplesPerCta - 1) / kSamplesPerCta;
  k_mlp_fwd<<<nb, 256, 0, s>>>(params, x, B, h1, h2, z);
  k_mlp_back<<<nb, 256, 0, s>>>(params, labels, B, h1, h2, z, dz, d2, d1, lb);
  k_mlp_wgrad<<<(kNParams + 255) / 256, 256, 0, s>>>(x, B, h1, h2, dz, d2, d1, lb, grads, loss);
  return cudaGetLastError() == cudaSuccess ? TTN_OK : TTN_ECUDA;
}

ttn_status ttn_mlp_adam(float* params, float* m, float* v, const float* grads, int32_t t, float lr, void* stream) {
  if (!params || !m || !v || !grads || t < 1 || !(lr > 0)) return TTN_EINVAL;
  const float c1 = 1.f - powf(0.9f, (float)t), c2 = 1.f - powf(0.999f, (float)t);
  ttn::k_adam<<<(ttn::kNParams + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, m, v, grads, ttn::kNParams, lr,
                                                                              c1, c2);
  return cudaGetLastError() == cudaSuccess ? TTN_OK : TTN_ECUDA;
}

}  // extern "C"
