// Blocked Householder QR for node matricisations too tall for one cluster's
// shared memory (e.g. 4096 x 64 at bond rank 64), FP64.
//
// Same convention and, in exact arithmetic, the same result as the unblocked
// kernels: the column loop is the cluster kernel run on panels of kQrPanelMaxNb
// columns (rows from the panel's first pivot down), with the threshold
// tol*||A||_F of the WHOLE matrix; the panel's reflectors are then applied to
// the trailing columns in compact WY form, A2 -= V T^H (V^H A2), and Q is formed
// by applying the panels in reverse order to the first n columns of the
// identity, X -= V T (V^H X). A skipped column has no reflector (zero v, zero
// rows and columns of T), so the deterministic completion H_0..H_{j-1} e_j comes
// out of the reverse accumulation by itself. Every reduction runs in a fixed
// order (row blocks summed in block order), so results are reproducible.
//
// The trailing and Q updates are spread over one CTA per SM (rows split evenly,
// at most kRB per CTA): they are bound by the FP64 issue rate of each SM, so
// an even split over all SMs is what shortens them. Only the panels run on
// one cluster.
#include <algorithm>

#include "kernels.cuh"

namespace ttn {

namespace {

constexpr int kRB = 32;                // most rows per CTA of the update kernels
constexpr int kNB = kQrPanelMaxNb;     // panel width
constexpr int kGatherMax = 1024;       // CTAs of the gather / norm partials
constexpr int kBlkCap = 256;           // most CTAs of a balanced row partition

// The update kernels are bound by the SM's FP64 issue rate, so the rows are
// split into one block per SM (at most kRB rows each, at least one row).
int rows_per_block(int64_t rows, int sms) {
  const int64_t s = std::max(1, std::min(sms, kBlkCap));
  return (int)std::max<int64_t>(1, std::min<int64_t>(kRB, (rows + s - 1) / s));
}
int64_t max_blocks(int64_t m) { return std::max<int64_t>(kBlkCap, (m + kRB - 1) / kRB); }

int64_t round16(int64_t x) { return (x + 15) / 16 * 16; }

// Offsets (complex elements) of the blocked-QR scratch inside `work`.
struct QbLayout {
  int64_t A, part, sc, beta, alpha, phase, skip, T, Y, Z, total;
};
QbLayout qb_layout(int64_t m, int64_t n) {
  QbLayout L;
  int64_t o = 0;
  auto take = [&](int64_t e) {
    const int64_t r = o;
    o += round16(e);
    return r;
  };
  L.A = take(m * n);
  L.part = take(kGatherMax / 2);
  L.sc = take(8);
  L.beta = take((n + 1) / 2);
  L.alpha = take((n + 1) / 2);
  L.phase = take(n);
  L.skip = take((n + 3) / 4);
  L.T = take((n + kNB - 1) / kNB * kNB * kNB);
  L.Y = take(max_blocks(m) * kNB * n);
  L.Z = take(kNB * n);
  L.total = o;
  return L;
}

__device__ __forceinline__ double2 cfmaj(double2 a, double2 b, double2 c) {  // conj(a)*b + c
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(-a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {  // a*b + c
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ bool aborted(const double* sc) { return !isfinite(sc[0]); }

// Acm[c*m + r] = U[row r, column c of the matricisation toward `leg`];
// part[block] = sum |a|^2 of the block's elements (fixed order).
__global__ void __launch_bounds__(256) k_qb_gather(const double2* U, int d0, int d1, int d2, int leg,
                                                   double2* Acm, int64_t m, int64_t n, double* part) {
  __shared__ double red[8];
  const int dd[3] = {d0, d1, d2};
  const int64_t st[3] = {(int64_t)d1 * d2, d2, 1};
  const int la = leg == 0 ? 1 : 0, lb = leg == 2 ? 1 : 2;
  double ss = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m * n; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = k / m, r = k % m;
    const double2 v = U[c * st[leg] + (r / dd[lb]) * st[la] + (r % dd[lb]) * st[lb]];
    Acm[k] = v;
    ss = fma(v.x, v.x, fma(v.y, v.y, ss));
  }
  ss = wsum(ss);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

// sc[0] = tol * ||A||_F (NaN and flag bit 1 when the norm is not finite)
__global__ void k_qb_norm(const double* part, int np, double tol, double* sc, int* flag) {
  double t = 0.0;
  for (int i = threadIdx.x; i < np; i += 32) t += part[i];
  t = wsum(t);
  if (threadIdx.x == 0) {
    const double f = sqrt(t);
    if (isfinite(f)) {
      sc[0] = tol * f;
    } else {
      sc[0] = __longlong_as_double(0x7ff8000000000000ll);
      atomicOr(flag, 1);
    }
  }
}

// Ypart[b][i][k] = sum over rows r of block b (rows from c0, rbs rows per
// block) with r >= c0+i of conj(V[r][c0+i]) * S[r][k], for i < nb and
// k0 <= k < n. V = column block of A.
__global__ void __launch_bounds__(256) k_qb_ypart(const double2* A, const double2* S, int64_t m, int c0, int nb,
                                                  int k0, int n, int rbs, double2* Ypart, const double* sc) {
  __shared__ double2 Vs[kNB][kRB];
  __shared__ double2 Ss[kRB][kQrClusterMaxN + 1];
  if (aborted(sc)) return;
  const int b = blockIdx.x;
  const int64_t rb = c0 + (int64_t)b * rbs;
  const int nk = n - k0;
  for (int t = threadIdx.x; t < nb * rbs; t += blockDim.x) {
    const int i = t / rbs, rr = t % rbs;
    const int64_t r = rb + rr;
    Vs[i][rr] = (r < m && r >= c0 + i) ? A[(int64_t)(c0 + i) * m + r] : make_double2(0.0, 0.0);
  }
  for (int t = threadIdx.x; t < nk * rbs; t += blockDim.x) {
    const int kk = t / rbs, rr = t % rbs;
    const int64_t r = rb + rr;
    Ss[rr][kk] = r < m ? S[(int64_t)(k0 + kk) * m + r] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nb * nk; t += blockDim.x) {
    const int i = t / nk, kk = t % nk;
    double2 y = make_double2(0.0, 0.0);
#pragma unroll 4
    for (int rr = 0; rr < rbs; ++rr) y = cfmaj(Vs[i][rr], Ss[rr][kk], y);
    Ypart[((int64_t)b * kNB + i) * n + k0 + kk] = y;
  }
}

// One CTA per column k: Y[i] = sum over blocks (in block order), then
// Z[i][k] = sum_j T'[i][j] Y[j] with T' = T^H (trans) or T.
__global__ void __launch_bounds__(256) k_qb_zsum(const double2* Ypart, int nblk, int nb, int k0, int n,
                                                 const double2* T, int trans, double2* Z, const double* sc) {
  __shared__ double2 y[kNB];
  __shared__ double2 Ts[kNB * kNB];  // T'[i][j], loaded while the block sums run
  if (aborted(sc)) return;
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int i = t / nb, j = t % nb;
    Ts[t] = trans ? make_double2(T[j * nb + i].x, -T[j * nb + i].y) : T[t];
  }
  const int k = k0 + blockIdx.x;
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int w = threadIdx.x >> 5; w < nb; w += nw) {  // warp-uniform
    double2 a = make_double2(0.0, 0.0);
    for (int b = lane; b < nblk; b += 32) {
      const double2 v = Ypart[((int64_t)b * kNB + w) * n + k];
      a.x += v.x;
      a.y += v.y;
    }
    a.x = wsum(a.x);
    a.y = wsum(a.y);
    if (lane == 0) y[w] = a;
  }
  __syncthreads();
  if ((int)threadIdx.x < nb) {
    const int i = threadIdx.x;
    double2 z = make_double2(0.0, 0.0);
    for (int j = 0; j < nb; ++j) z = cfma(Ts[i * nb + j], y[j], z);
    Z[(int64_t)i * n + k] = z;
  }
}

// D[r][k] -= sum_i V[r][c0+i] Z[i][k] for the rows of block b (rbs rows per
// block) and k0 <= k < n.
__global__ void __launch_bounds__(256) k_qb_update(const double2* A, double2* D, int64_t m, int c0, int nb, int k0,
                                                   int n, int rbs, const double2* Z, const double* sc) {
  __shared__ double2 Vs[kNB][kRB];
  __shared__ double2 Zs[kNB][kQrClusterMaxN];
  if (aborted(sc)) return;
  const int64_t rb = c0 + (int64_t)blockIdx.x * rbs;
  const int nk = n - k0;
  for (int t = threadIdx.x; t < nb * rbs; t += blockDim.x) {
    const int i = t / rbs, rr = t % rbs;
    const int64_t r = rb + rr;
    Vs[i][rr] = (r < m && r >= c0 + i) ? A[(int64_t)(c0 + i) * m + r] : make_double2(0.0, 0.0);
  }
  for (int t = threadIdx.x; t < nb * nk; t += blockDim.x) {
    const int i = t / nk, kk = t % nk;
    Zs[i][kk] = Z[(int64_t)i * n + k0 + kk];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nk * rbs; t += blockDim.x) {
    const int kk = t / rbs, rr = t % rbs;
    const int64_t r = rb + rr;
    if (r >= m) continue;
    double2* d = D + (int64_t)(k0 + kk) * m + r;
    double2 v = *d;
    for (int i = 0; i < nb; ++i) {
      const double2 a = Vs[i][rr], z = Zs[i][kk];
      v.x = fma(-a.x, z.x, fma(a.y, z.y, v.x));
      v.y = fma(-a.x, z.y, fma(-a.y, z.x, v.y));
    }
    *d = v;
  }
}

__global__ void k_qb_identity(double2* X, int64_t m, int64_t n, const double* sc) {
  if (aborted(sc)) return;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m * n; k += (int64_t)gridDim.x * blockDim.x)
    X[k] = make_double2((k % m) == (k / m) ? 1.0 : 0.0, 0.0);
}

// R (row-major n x n, row i scaled by conj(phase_i), diag alpha) and
// Q = X with column c scaled by phase_c, scattered into U's layout.
__global__ void k_qb_finish(const double2* A, const double2* X, int64_t m, int64_t n, const double* alpha,
                            const double2* phase, const int* skip, double2* U, int d0, int d1, int d2, int leg,
                            double2* R, float2* U_lo, float2* R_lo, const double* sc) {
  if (aborted(sc)) return;
  const int dd[3] = {d0, d1, d2};
  const int64_t st[3] = {(int64_t)d1 * d2, d2, 1};
  const int la = leg == 0 ? 1 : 0, lb = leg == 2 ? 1 : 2;
  const int64_t g0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, gs = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = g0; k < n * n; k += gs) {
    const int64_t i = k / n, c = k % n;
    double2 v = make_double2(0.0, 0.0);
    if (c == i) {
      v = make_double2(skip[i] ? 0.0 : alpha[i], 0.0);
    } else if (c > i) {
      const double2 a = A[c * m + i], p = phase[i];
      v = make_double2(a.x * p.x + a.y * p.y, a.y * p.x - a.x * p.y);
    }
    R[k] = v;
    if (R_lo) R_lo[k] = make_float2((float)v.x, (float)v.y);
  }
  for (int64_t k = g0; k < m * n; k += gs) {
    const int64_t c = k / m, r = k % m;
    const double2 q = X[k], p = phase[c];
    const double2 qp = make_double2(q.x * p.x - q.y * p.y, q.x * p.y + q.y * p.x);
    const int64_t at = c * st[leg] + (r / dd[lb]) * st[la] + (r % dd[lb]) * st[lb];
    U[at] = qp;
    if (U_lo) U_lo[at] = make_float2((float)qp.x, (float)qp.y);
  }
}

}  // namespace

int64_t qr_blocked_elems(int64_t m, int64_t n) { return qb_layout(m, n).total; }

bool launch_qr_blocked(double2* U, int d0, int d1, int d2, int leg, double tol, double2* work,
                       int64_t work_elems, double2* qbuf, double2* R, int* flag, float2* U_lo, float2* R_lo,
                       cudaStream_t s) {
  const int dd[3] = {d0, d1, d2};
  const int n = dd[leg];
  const int64_t m = (int64_t)d0 * d1 * d2 / n;
  if (n < 1 || n > kQrClusterMaxN || m < n) return false;
  const QbLayout L = qb_layout(m, n);
  if (L.total > work_elems) return false;
  if (qr_panel_cluster((int)m, std::min(n, kNB)) == 0) return false;  // the first panel is the tallest
  double2* A = work + L.A;
  double* part = (double*)(work + L.part);
  double* sc = (double*)(work + L.sc);
  double* beta = (double*)(work + L.beta);
  double* alpha = (double*)(work + L.alpha);
  double2* phase = work + L.phase;
  int* skip = (int*)(work + L.skip);
  double2* T = work + L.T;
  double2* Y = work + L.Y;
  double2* Z = work + L.Z;
  double2* X = qbuf;

  static int sms = 0;  // SMs of the device (the update kernels use one CTA per SM)
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 1;
  }
  const int g1 = (int)std::min<int64_t>(kGatherMax, (m * n + 255) / 256);
  k_qb_gather<<<g1, 256, 0, s>>>(U, d0, d1, d2, leg, A, m, n, part);
  k_qb_norm<<<1, 32, 0, s>>>(part, g1, tol, sc, flag);
  // factorisation: panel, then its reflectors on the trailing columns
  for (int c0 = 0; c0 < n; c0 += kNB) {
    const int nb = std::min(kNB, n - c0);
    QrPanel pn{nullptr, A, (int)m, n, c0, nb, sc, beta, alpha, phase, skip, T + (int64_t)(c0 / kNB) * kNB * kNB};
    if (!launch_qr_panel(pn, s)) return false;
    const int k0 = c0 + nb;
    if (k0 >= n) break;
    const int rbs = rows_per_block(m - c0, sms);
    const int nblk = (int)((m - c0 + rbs - 1) / rbs);
    k_qb_ypart<<<nblk, 256, 0, s>>>(A, A, m, c0, nb, k0, n, rbs, Y, sc);
    k_qb_zsum<<<n - k0, 256, 0, s>>>(Y, nblk, nb, k0, n, pn.T, 1, Z, sc);
    k_qb_update<<<nblk, 256, 0, s>>>(A, A, m, c0, nb, k0, n, rbs, Z, sc);
  }
  // Q = H_0 .. H_{n-1} [I_n; 0], panels applied last to first
  const int gi = (int)std::min<int64_t>(2048, (m * n + 255) / 256);
  k_qb_identity<<<gi, 256, 0, s>>>(X, m, n, sc);
  for (int c0 = (n - 1) / kNB * kNB; c0 >= 0; c0 -= kNB) {
    const int nb = std::min(kNB, n - c0);
    const double2* Tp = T + (int64_t)(c0 / kNB) * kNB * kNB;
    const int rbs = rows_per_block(m - c0, sms);
    const int nblk = (int)((m - c0 + rbs - 1) / rbs);
    k_qb_ypart<<<nblk, 256, 0, s>>>(A, X, m, c0, nb, c0, n, rbs, Y, sc);
    k_qb_zsum<<<n - c0, 256, 0, s>>>(Y, nblk, nb, c0, n, Tp, 0, Z, sc);
    k_qb_update<<<nblk, 256, 0, s>>>(A, X, m, c0, nb, c0, n, rbs, Z, sc);
  }
  k_qb_finish<<<gi, 256, 0, s>>>(A, X, m, n, alpha, phase, skip, U, d0, d1, d2, leg, R, U_lo, R_lo, sc);
  return true;
}

}  // namespace ttn
