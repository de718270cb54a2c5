// Householder QR of a node tensor spread over a thread-block cluster (FP64).
//
// On GB300 a single SM retires about 2 FP64 FMA per clock, so a one-CTA
// Householder QR of a 400 x 20 complex matricisation takes ~170 us. Here the
// m rows are split over C <= 16 CTAs of one cluster; each CTA keeps its row
// block in shared memory and the per-column reductions (the column norm and the
// dot products with the trailing columns) are exchanged through distributed
// shared memory with two cluster barriers per column. Q is then formed from
// the compact WY representation H_0..H_{n-1} = I - V T V^H (Schreiber-Van Loan),
// which costs one Gram reduction instead of n sequential reflector passes.
//
// The arithmetic convention is the one of the CPU oracle and of the one-CTA
// kernel: for column j with remainder x of norm alpha, alpha <= tol*||A||_F
// means no reflector (R_jj = 0, Q column H_0..H_{j-1} e_j); otherwise
// v = x + phi*alpha*e_0, phi = x_0/|x_0| (1 if x_0 = 0), beta = 1/(alpha(alpha+|x_0|)),
// and finally row j of R / column j of Q are rescaled by the phase -phi so
// that diag(R) >= 0. All reductions run in a fixed order, so results are
// bitwise reproducible.
#include <cooperative_groups.h>

#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace ttn {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double2 cfma_c(double2 a, double2 b, double2 c) {  // a*b + c
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ double2 cfmaj(double2 a, double2 b, double2 c) {  // conj(a)*b + c
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(-a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double2 wsum2(double2 v) {
  v.x = wsum(v.x);
  v.y = wsum(v.y);
  return v;
}
// block sum in a fixed order; every thread gets the result
__device__ double bsum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = wsum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < nw; ++w) s += red[w];
  __syncthreads();
  return s;
}

}  // namespace

// Shared-memory layout (dynamic, double2 units):
//   A   [n][rp]  my row block, column-major (v_j overwrites rows >= j of column j)
//   P2  [2][n]   per-parity partial dot products w_k
//   G   [n][n]   partial Gram V^H V of my rows, then the full Gram
//   T   [n][n]   WY factor
//   MM  [n][n]   T V_top^H
__global__ void __launch_bounds__(kThreads) k_qr_cluster(double2* U, int d0, int d1, int d2, int leg,
                                                         double tol, double2* R, int* flag, float2* U_lo,
                                                         float2* R_lo) {
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int me = (int)cluster.block_rank();
  const int dd[3] = {d0, d1, d2};
  const int64_t st[3] = {(int64_t)d1 * d2, d2, 1};
  const int n = dd[leg];
  const int la = leg == 0 ? 1 : 0, lb = leg == 2 ? 1 : 2;
  const int m = dd[la] * dd[lb];
  const int rp = (m + C - 1) / C;
  const int r0 = me * rp;
  const int nr = max(0, min(m, r0 + rp) - r0);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;

  extern __shared__ double2 smem[];
  double2* A = smem;
  double2* P2 = A + (size_t)n * rp;
  double2* G = P2 + 2 * n;
  double2* T = G + n * n;
  double2* MM = T + n * n;
  __shared__ double red[kThreads / 32];
  __shared__ double s_part[2];     // per-parity partial norm^2
  __shared__ double2 s_x0[2];      // per-parity x_0 (owner of row j only)
  __shared__ double s_beta[kQrClusterMaxN], s_alpha[kQrClusterMaxN];
  __shared__ int s_skip[kQrClusterMaxN];
  __shared__ double2 s_phase[kQrClusterMaxN];
  __shared__ double s_bcast[2];
  __shared__ double2 s_bx0;

  // gather my rows: A[c][i] = U[.. row r0+i, column c ..]
  double fro = 0.0;
  for (int k = tid; k < n * rp; k += nt) {
    const int c = k / rp, i = k % rp;
    double2 v = make_double2(0.0, 0.0);
    if (i < nr) {
      const int r = r0 + i;
      v = U[c * st[leg] + (int64_t)(r / dd[lb]) * st[la] + (int64_t)(r % dd[lb]) * st[lb]];
    }
    A[k] = v;
    fro += v.x * v.x + v.y * v.y;
  }
  fro = bsum(fro, red);
  if (tid == 0) s_part[0] = fro;
  cluster.sync();
  if (wid == 0) {  // lane c reads CTA c's partial; fixed butterfly order
    double v = lane < C ? *cluster.map_shared_rank(&s_part[0], lane) : 0.0;
    v = wsum(v);
    if (lane == 0) s_bcast[0] = sqrt(v);
  }
  __syncthreads();
  const double frob = s_bcast[0];
  if (!isfinite(frob)) {  // uniform across the cluster
    if (tid == 0 && me == 0) atomicOr(flag, 1);
    cluster.sync();
    return;
  }
  const double thr = tol * frob;
  cluster.sync();  // everyone has read s_part[0] before it is reused

  for (int j = 0; j < n; ++j) {
    const int par = j & 1;
    double2* x = A + (size_t)j * rp;
    const int i0 = max(0, j - r0);  // first local row with global index >= j
    double ss = 0.0;
    for (int i = i0 + tid; i < nr; i += nt) ss += x[i].x * x[i].x + x[i].y * x[i].y;
    ss = bsum(ss, red);
    const int owner = j / rp;
    if (tid == 0) {
      s_part[par] = ss;
      if (owner == me) s_x0[par] = x[j - r0];
    }
    cluster.sync();
    if (wid == 0) {
      double v = lane < C ? *cluster.map_shared_rank(&s_part[par], lane) : 0.0;
      v = wsum(v);
      if (lane == 0) {
        s_bcast[1] = sqrt(v);
        s_bx0 = *cluster.map_shared_rank(&s_x0[par], owner);
      }
    }
    __syncthreads();
    const double alpha = s_bcast[1];
    const double2 x0 = s_bx0;
    if (alpha <= thr) {
      for (int i = i0 + tid; i < nr; i += nt) x[i] = make_double2(0.0, 0.0);
      if (tid == 0) {
        s_skip[j] = 1;
        s_beta[j] = 0.0;
        s_alpha[j] = 0.0;
        s_phase[j] = make_double2(1.0, 0.0);
      }
      __syncthreads();
      continue;  // uniform: every CTA takes this branch
    }
    const double ax0 = hypot(x0.x, x0.y);
    const double2 phi = ax0 > 0.0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
    const double beta = 1.0 / (alpha * (alpha + ax0));
    if (tid == 0) {
      if (owner == me) x[j - r0] = make_double2(x0.x + phi.x * alpha, x0.y + phi.y * alpha);
      s_skip[j] = 0;
      s_beta[j] = beta;
      s_alpha[j] = alpha;
      s_phase[j] = make_double2(-phi.x, -phi.y);
    }
    __syncthreads();
    // partial dots w_k = sum_{my rows >= j} conj(v) a_k, one warp per column
    double2* pw = P2 + par * n;
    for (int k = j + 1 + wid; k < n; k += nw) {
      const double2* a = A + (size_t)k * rp;
      double2 w = make_double2(0.0, 0.0);
      for (int i = i0 + lane; i < nr; i += 32) w = cfmaj(x[i], a[i], w);
      w = wsum2(w);
      if (lane == 0) pw[k] = w;
    }
    cluster.sync();
    for (int k = j + 1 + wid; k < n; k += nw) {
      double2 w = make_double2(0.0, 0.0);
      if (lane < C) w = *cluster.map_shared_rank(&pw[k], lane);
      w = wsum2(w);  // fixed butterfly order, identical in every CTA
      const double2 bw = make_double2(beta * w.x, beta * w.y);
      double2* a = A + (size_t)k * rp;
      for (int i = i0 + lane; i < nr; i += 32) {
        const double2 t = make_double2(x[i].x * bw.x - x[i].y * bw.y, x[i].x * bw.y + x[i].y * bw.x);
        a[i] = make_double2(a[i].x - t.x, a[i].y - t.y);
      }
    }
    __syncthreads();
  }
  cluster.sync();  // all reflectors final everywhere

  // R rows owned here (global rows < n), diag(R) = alpha >= 0 after the phase fix
  for (int k = tid; k < n * n; k += nt) {
    const int i = k / n, c = k % n;
    if (i < r0 || i >= r0 + nr) continue;
    double2 v = make_double2(0.0, 0.0);
    if (c == i) {
      v = make_double2(s_skip[i] ? 0.0 : s_alpha[i], 0.0);
    } else if (c > i) {
      const double2 a = A[(size_t)c * rp + (i - r0)];
      const double2 p = s_phase[i];
      v = make_double2(a.x * p.x + a.y * p.y, a.y * p.x - a.x * p.y);  // conj(p) * a
    }
    R[k] = v;
    if (R_lo) R_lo[k] = make_float2((float)v.x, (float)v.y);
  }
  // partial Gram G[a][b] = sum_{my rows} conj(v_a) v_b, v_a = 0 above the diagonal and for skipped a
  for (int k = tid; k < n * n; k += nt) {
    const int a = k / n, b = k % n;
    double2 g = make_double2(0.0, 0.0);
    if (!s_skip[a] && !s_skip[b]) {
      const int lo = max(max(a, b) - r0, 0);
      const double2* va = A + (size_t)a * rp;
      const double2* vb = A + (size_t)b * rp;
      for (int i = lo; i < nr; ++i) g = cfmaj(va[i], vb[i], g);
    }
    G[k] = g;
  }
  cluster.sync();
  // full Gram (fixed order over CTAs) into T's storage temporarily
  for (int k = tid; k < n * n; k += nt) {
    double2 v[16];  // all remote loads in flight before the fixed-order sum
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = c < C ? cluster.map_shared_rank(G, c)[k] : make_double2(0.0, 0.0);
    double2 g = make_double2(0.0, 0.0);
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      g.x += v[c].x;
      g.y += v[c].y;
    }
    T[k] = g;
  }
  // gather V_top[c][b] = v_b[row c] for rows c < n into MM (remote reads)
  for (int k = tid; k < n * n; k += nt) {
    const int c = k / n, b = k % n;
    double2 v = make_double2(0.0, 0.0);
    if (!s_skip[b] && c >= b) {
      const int own = c / rp;
      v = cluster.map_shared_rank(A, own)[(size_t)b * rp + (c - own * rp)];
    }
    MM[k] = v;
  }
  cluster.sync();  // remote reads of G and A done; G may be overwritten
  // WY factor: T[j][j] = beta_j, T[0:j, j] = -beta_j T[0:j, 0:j] Gram[0:j, j]
  // (Gram in T's storage is copied to G first, T built in place column by column)
  for (int k = tid; k < n * n; k += nt) G[k] = T[k];
  __syncthreads();
  for (int k = tid; k < n * n; k += nt) T[k] = make_double2(0.0, 0.0);
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (s_skip[j]) continue;
    const double bj = s_beta[j];
    for (int a = tid; a < j; a += nt) {
      double2 acc = make_double2(0.0, 0.0);
      for (int b = a; b < j; ++b) acc = cfma_c(T[a * n + b], G[b * n + j], acc);
      T[a * n + j] = make_double2(-bj * acc.x, -bj * acc.y);
    }
    if (tid == 0) T[j * n + j] = make_double2(bj, 0.0);
    __syncthreads();
  }
  // M = T V_top^H: M[a][c] = sum_b T[a][b] conj(V_top[c][b]); G's storage reused for M
  for (int k = tid; k < n * n; k += nt) {
    const int a = k / n, c = k % n;
    double2 acc = make_double2(0.0, 0.0);
    for (int b = a; b < n; ++b) {
      const double2 t = T[a * n + b], v = MM[c * n + b];
      acc.x = fma(t.x, v.x, fma(t.y, v.y, acc.x));
      acc.y = fma(t.y, v.x, fma(-t.x, v.y, acc.y));
    }
    G[k] = acc;
  }
  __syncthreads();
  // Q rows: Q[r][c] = delta_rc - sum_a v_a[r] M[a][c], column c scaled by phase_c, scattered to U
  for (int k = tid; k < n * nr; k += nt) {
    const int c = k / nr, i = k % nr;
    const int r = r0 + i;
    double2 q = make_double2(r == c ? 1.0 : 0.0, 0.0);
    for (int a = 0; a < n && a <= r; ++a) {
      if (s_skip[a]) continue;
      const double2 v = A[(size_t)a * rp + i];
      const double2 mm = G[a * n + c];
      q.x -= v.x * mm.x - v.y * mm.y;
      q.y -= v.x * mm.y + v.y * mm.x;
    }
    const double2 p = s_phase[c];
    const double2 qp = make_double2(q.x * p.x - q.y * p.y, q.x * p.y + q.y * p.x);
    const int64_t at = c * st[leg] + (int64_t)(r / dd[lb]) * st[la] + (int64_t)(r % dd[lb]) * st[lb];
    U[at] = qp;
    if (U_lo) U_lo[at] = make_float2((float)qp.x, (float)qp.y);
  }
  cluster.sync();  // keep shared memory alive until every remote read has finished
}

size_t qr_cluster_smem(int m, int n, int C) {
  const int rp = (m + C - 1) / C;
  return sizeof(double2) * ((size_t)n * rp + 2 * n + 3 * (size_t)n * n);
}

int qr_cluster_size(int m, int n) {
  if (n > kQrClusterMaxN) return 0;
  int C = (m + 7) / 8;  // about 8 rows per CTA: the factorisation is FP64-issue bound
  C = C < 1 ? 1 : (C > 16 ? 16 : C);
  while (C > 1 && qr_cluster_smem(m, n, C) > 160 * 1024) --C;  // not expected for C <= 16
  if (qr_cluster_smem(m, n, C) > 160 * 1024) return 0;
  return C;
}

bool launch_qr_cluster(double2* U, int d0, int d1, int d2, int leg, double tol, double2* R, int* flag,
                       float2* U_lo, float2* R_lo, cudaStream_t s) {
  const int dd[3] = {d0, d1, d2};
  const int n = dd[leg];
  const int m = (int)((int64_t)d0 * d1 * d2 / n);
  const int C = qr_cluster_size(m, n);
  if (C == 0) return false;
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(k_qr_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(k_qr_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    attr_done = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = qr_cluster_smem(m, n, C);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_qr_cluster, U, d0, d1, d2, leg, tol, R, flag, U_lo, R_lo) == cudaSuccess;
}

}  // namespace ttn
