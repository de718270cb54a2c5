// Kernels of the direct integration (vmf, Sec. 2.3 and Sec. 7.5), FP64.
//
// The node equations of the multilayer-MCTDH form need, on every edge p -> c,
// the single-hole density matrix rho and the mean fields M(kappa) of the part
// of the tree above c, weighted by the root. With the upper part brought into
// an orthonormal basis by a QR gauge move toward c (V_p = Q R), they are
//     rho = R^H R,   M(kappa) = R^H E(kappa) R,
// E(kappa) the ordinary (isometric) environment of class kappa. The equation
// of c, rho_reg dU_c/dt = (1 - P_c) G_c with rho_reg = rho + vmf_atol * 1, is
// evaluated as
//     dU_c/dt = (1 - P_c) [ H~ U_c + (D - 1) x_parent G_down ],
//     H~      = the node operator with E~(kappa) = rho_reg^-1 M(kappa) on the
//               parent leg, D = rho_reg^-1 rho,
// G_down the part of the node operator without a parent-leg factor (rho_reg^-1
// then multiplies rho, not the identity, for those terms). P_c projects onto
// the span of U_c's rows (parent index fixed): (1 - P) X = X - (X U^H) U.
//
//  k_vmf_rho    one CTA: rho = R^H R, the augmented [rho + eps 1 | 1 | rho]
//  k_vmf_gj     one CTA: Gauss-Jordan elimination with partial pivoting of the
//               augmented matrix -> [1 | rho_reg^-1 | D]; D - 1 stored
//  k_vmf_class  one CTA per class: E~ = rho_reg^-1 (R^H (E R)), in place
//  k_vmf_dmi    K += (D - 1) x_0 G_down
//  k_vmf_px     X = K U^H (one CTA per entry, fixed-order sums)
//  k_vmf_psub   K -= X U
//  k_vmf_stage  out = y + sum_l c_l K_l over the flat state
//  k_vmf_err    scaled squared error of the embedded pair, block partials;
//  k_vmf_sum    the partials added in order
#include <algorithm>

#include "kernels.cuh"

namespace ttn {

namespace {

constexpr int kT = 256;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // conj(a) b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// aug: r x 3r row-major: [rho + eps 1 | 1 | rho]
__global__ void k_vmf_rho(const double2* __restrict__ R, int r, double eps, double2* __restrict__ aug) {
  const int w = 3 * r;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e % r;
    double2 s = make_double2(0.0, 0.0);
    for (int k = 0; k < r; ++k) s = cadd(s, cmulc(R[k * r + i], R[k * r + j]));  // (R^H R)[i][j]
    aug[i * w + j] = make_double2(s.x + (i == j ? eps : 0.0), s.y);
    aug[i * w + r + j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    aug[i * w + 2 * r + j] = s;
  }
}

// Gauss-Jordan on the r x 3r augmented matrix: pivot column j, the row of the
// largest |entry| at or below j (lowest index on ties) swapped up, scaled, and
// eliminated from every other row. Leaves [1 | rho_reg^-1 | D]; dmi = D - 1.
__global__ void k_vmf_gj(double2* aug, int r, double2* __restrict__ dmi) {
  __shared__ int s_piv;
  __shared__ double2 s_inv;
  const int w = 3 * r, tid = threadIdx.x;
  for (int j = 0; j < r; ++j) {
    if (tid < 32) {
      double best = -1.0;
      int bi = j;
      for (int i = j + tid; i < r; i += 32) {
        const double a = fabs(aug[i * w + j].x) + fabs(aug[i * w + j].y);
        if (a > best) {
          best = a;
          bi = i;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (tid == 0) s_piv = bi;
    }
    __syncthreads();
    const int pv = s_piv;
    if (pv != j)
      for (int c = tid; c < w; c += blockDim.x) {
        const double2 t = aug[j * w + c];
        aug[j * w + c] = aug[pv * w + c];
        aug[pv * w + c] = t;
      }
    __syncthreads();
    if (tid == 0) {
      const double2 p = aug[j * w + j];
      const double n = p.x * p.x + p.y * p.y;
      s_inv = make_double2(p.x / n, -p.y / n);
    }
    __syncthreads();
    for (int c = tid; c < w; c += blockDim.x) aug[j * w + c] = cmul(s_inv, aug[j * w + c]);
    __syncthreads();
    for (int e = tid; e < r * w; e += blockDim.x) {
      const int i = e / w, c = e % w;
      if (i == j || c == j) continue;
      const double2 f = aug[i * w + j];
      const double2 v = cmul(f, aug[j * w + c]);
      aug[i * w + c] = make_double2(aug[i * w + c].x - v.x, aug[i * w + c].y - v.y);
    }
    __syncthreads();
    for (int i = tid; i < r; i += blockDim.x)
      if (i != j) aug[i * w + j] = make_double2(0.0, 0.0);
    __syncthreads();
  }
  for (int e = tid; e < r * r; e += blockDim.x) {
    const int i = e / r, c = e % r;
    const double2 d = aug[i * w + 2 * r + c];
    dmi[e] = make_double2(d.x - (i == c ? 1.0 : 0.0), d.y);
  }
}

// E~ = rho_reg^-1 (R^H (E R)) for the class matrix of this CTA, in place; the
// two intermediate products in `tmp` (2 r^2 per CTA).
__global__ void k_vmf_class(double2* const* mats, const int* __restrict__ slots, const double2* __restrict__ R,
                            const double2* __restrict__ aug, int r, double2* __restrict__ tmp) {
  double2* E = mats[slots[blockIdx.x]];
  double2* A = tmp + (size_t)blockIdx.x * 2 * r * r;  // E R
  double2* B = A + r * r;                              // R^H E R
  const int w = 3 * r;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e % r;
    double2 s = make_double2(0.0, 0.0);
    for (int k = 0; k < r; ++k) s = cadd(s, cmul(E[i * r + k], R[k * r + j]));
    A[e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e % r;
    double2 s = make_double2(0.0, 0.0);
    for (int k = 0; k < r; ++k) s = cadd(s, cmulc(R[k * r + i], A[k * r + j]));
    B[e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e % r;
    double2 s = make_double2(0.0, 0.0);
    for (int k = 0; k < r; ++k) s = cadd(s, cmul(aug[i * w + r + k], B[k * r + j]));
    E[e] = s;
  }
}

// K (r x nc) += dmi (r x r) G (r x nc)
__global__ void k_vmf_dmi(double2* __restrict__ K, const double2* __restrict__ G, const double2* __restrict__ dmi,
                          int r, int64_t nc) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)r * nc;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t c;
    const int a = (int)idivmod(e, nc, c);
    double2 s = K[e];
    for (int b = 0; b < r; ++b) s = cadd(s, cmul(dmi[a * r + b], G[(int64_t)b * nc + c]));
    K[e] = s;
  }
}

// X[a][b] = sum_c K[a][c] conj(U[b][c]); one CTA per entry
__global__ void k_vmf_px(const double2* __restrict__ K, const double2* __restrict__ U, int r, int64_t nc,
                         double2* __restrict__ X) {
  __shared__ double2 red[kT / 32];
  const int a = blockIdx.x / r, b = blockIdx.x % r;
  double2 s = make_double2(0.0, 0.0);
  for (int64_t c = threadIdx.x; c < nc; c += blockDim.x)
    s = cadd(s, cmulc(U[(int64_t)b * nc + c], K[(int64_t)a * nc + c]));
  for (int o = 16; o > 0; o >>= 1) {
    s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
    s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 t = make_double2(0.0, 0.0);
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t = cadd(t, red[q]);
    X[blockIdx.x] = t;
  }
}

// K[a][c] -= sum_b X[a][b] U[b][c]
__global__ void k_vmf_psub(double2* __restrict__ K, const double2* __restrict__ U, const double2* __restrict__ X, int r,
                           int64_t nc) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)r * nc;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t c;
    const int a = (int)idivmod(e, nc, c);
    double2 s = make_double2(0.0, 0.0);
    for (int b = 0; b < r; ++b) s = cadd(s, cmul(X[a * r + b], U[(int64_t)b * nc + c]));
    K[e] = make_double2(K[e].x - s.x, K[e].y - s.y);
  }
}

__global__ void k_vmf_stage(double2* __restrict__ out, const double2* __restrict__ y, VmfComb cb, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double2 s = y[e];
    for (int l = 0; l < cb.n; ++l) {
      const double2 k = cb.K[l][e];
      s.x = fma(cb.c[l], k.x, s.x);
      s.y = fma(cb.c[l], k.y, s.y);
    }
    out[e] = s;
  }
}

constexpr int kErrBlocks = 1024;
__global__ void k_vmf_err(const double2* __restrict__ y, const double2* __restrict__ y5, VmfComb cb, double rtol,
                          double atol, int64_t n, double* __restrict__ part) {
  __shared__ double red[kT / 32];
  double acc = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double ex = 0.0, ey = 0.0;
    for (int l = 0; l < cb.n; ++l) {
      const double2 k = cb.K[l][e];
      ex = fma(cb.c[l], k.x, ex);
      ey = fma(cb.c[l], k.y, ey);
    }
    const double a = sqrt(y[e].x * y[e].x + y[e].y * y[e].y), b = sqrt(y5[e].x * y5[e].x + y5[e].y * y5[e].y);
    const double sc = atol + rtol * fmax(a, b);
    acc += (ex * ex + ey * ey) / (sc * sc);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kT / 32; ++q) t += red[q];
    part[blockIdx.x] = t;
  }
}
__global__ void k_vmf_sum(const double* __restrict__ part, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < n; ++i) t += part[i];
    out[0] = t;
  }
}

int grid_of(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + kT - 1) / kT, 4096)); }

}  // namespace

void launch_vmf_edge(double2* const* mats_dev, const int* slots_dev, int n_classes, const double2* R, int r,
                     double eps, double2* aug, double2* dmi, double2* tmp, cudaStream_t s) {
  k_vmf_rho<<<1, kT, 0, s>>>(R, r, eps, aug);
  k_vmf_gj<<<1, kT, 0, s>>>(aug, r, dmi);
  if (n_classes > 0) k_vmf_class<<<n_classes, kT, 0, s>>>(mats_dev, slots_dev, R, aug, r, tmp);
}

void launch_vmf_finish(double2* K, const double2* Gdown, const double2* dmi, const double2* U, int r, int64_t nc,
                       double2* X, cudaStream_t s) {
  k_vmf_dmi<<<grid_of((int64_t)r * nc), kT, 0, s>>>(K, Gdown, dmi, r, nc);
  k_vmf_px<<<r * r, kT, 0, s>>>(K, U, r, nc, X);
  k_vmf_psub<<<grid_of((int64_t)r * nc), kT, 0, s>>>(K, U, X, r, nc);
}

void launch_vmf_stage(double2* out, const double2* y, const VmfComb& cb, int64_t n, cudaStream_t s) {
  k_vmf_stage<<<grid_of(n), kT, 0, s>>>(out, y, cb, n);
}

void launch_vmf_err(const double2* y, const double2* y5, const VmfComb& cb, double rtol, double atol, int64_t n,
                    double* part, double* out, cudaStream_t s) {
  k_vmf_err<<<kErrBlocks, kT, 0, s>>>(y, y5, cb, rtol, atol, n, part);
  k_vmf_sum<<<1, 32, 0, s>>>(part, kErrBlocks, out);
}

}  // namespace ttn
