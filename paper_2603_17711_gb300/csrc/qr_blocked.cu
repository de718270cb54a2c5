// Blocked Householder QR for node matricisations too tall for one cluster's
// shared memory (e.g. 4096 x 64 at bond rank 64), FP64.
//
// Same convention and, in exact arithmetic, the same result as the unblocked
// kernels: the column loop runs on panels of kQrPanelMaxNb columns (rows from
// the panel's first pivot down) with the threshold tol*||A||_F of the WHOLE
// matrix -- over the whole GPU (k_qb_panel_grid, a cooperative launch with one
// grid exchange per column) where the device supports cooperative launches,
// else as the cluster kernel in panel mode; the panel's reflectors are then applied to
// the trailing columns in compact WY form, A2 -= V T^H (V^H A2), and Q is formed
// by applying the panels in reverse order to the first n columns of the
// identity, X -= V T (V^H X). A skipped column has no reflector (zero v, zero
// rows and columns of T), so the deterministic completion H_0..H_{j-1} e_j comes
// out of the reverse accumulation by itself. Every reduction runs in a fixed
// order (row blocks summed in block order), so results are reproducible.
//
// The trailing and Q updates are spread over one CTA per SM (rows split evenly,
// at most kRB per CTA): they are bound by the FP64 issue rate of each SM, so
// an even split over all SMs is what shortens them.
#include <algorithm>

#include "kernels.cuh"

namespace ttn {

namespace {

constexpr int kRB = 32;                // most rows per CTA of the update kernels
constexpr int kNB = kQrPanelMaxNb;     // panel width
constexpr int kGatherMax = 1024;       // CTAs of the gather / norm partials
constexpr int kBlkCap = 256;           // most CTAs of a balanced row partition
constexpr int kNpair = kNB * (kNB - 1) / 2;  // strictly-upper Gram entries of a panel
constexpr int kPgRows = 64;            // most panel rows per CTA of the grid panel kernel
constexpr int kMaxPanels = (kQrClusterMaxN + kNB - 1) / kNB;

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
  int64_t A, part, sc, beta, alpha, phase, skip, T, Y, Z, rec, own, gp, gf, bar, total;
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
  L.rec = take((int64_t)kNB * kBlkCap * kNB);
  L.own = take(kNB * kNB);
  L.gp = take((int64_t)kBlkCap * kNpair);
  L.gf = take(kNpair);
  L.bar = take(kMaxPanels * 8 / 4);  // kBarLanes (8) 32-bit grid-barrier counters per panel
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
__device__ __forceinline__ double2 cfms(double2 a, double2 b, double2 c) {  // c - a*b
  c.x = fma(-a.x, b.x, c.x);
  c.x = fma(a.y, b.y, c.x);
  c.y = fma(-a.x, b.y, c.y);
  c.y = fma(-a.y, b.x, c.y);
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
    int64_t r, rb;
    const int64_t c = idivmod(k, m, r);
    const int64_t ra = idivmod(r, dd[lb], rb);
    const double2 v = U[c * st[leg] + ra * st[la] + rb * st[lb]];
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

// sc[0] = tol * ||A||_F (NaN and flag bit 1 when the norm is not finite);
// the panels' grid-barrier counters start at zero
__global__ void k_qb_norm(const double* part, int np, double tol, double* sc, int* flag, unsigned* bar) {
  if (threadIdx.x < kMaxPanels * 8) bar[threadIdx.x] = 0u;
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

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Grid barrier of a cooperative launch over kBarLanes counters (CTA c adds
// one to bar[c % kBarLanes], so the arrivals do not all serialise on one
// address); a waiting CTA polls the counters with one warp until their sum
// reaches target. The wait is bounded by the kernel-wide deadline; on expiry
// bit 2 of *flag is set and false returned.
constexpr int kBarLanes = 8;
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// The CTA barrier orders the CTA's earlier writes before thread 0's release;
// the acquire of the counters plus the CTA barrier after it order the other
// CTAs' writes before this CTA's later reads.
__device__ bool grid_arrive_wait(unsigned* bar, unsigned target, bool wait, uint64_t deadline, int* flag) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    if (lane == 0) red_release_add(bar + blockIdx.x % kBarLanes, 1u);
    int ok = 1;
    if (wait) {
      for (;;) {
        unsigned v = lane < kBarLanes ? ld_acquire(bar + lane) : 0u;
        for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (__shfl_sync(0xffffffffu, v, 0) >= target) break;
        if (__shfl_sync(0xffffffffu, (int)(gtimer() > deadline), 0)) {  // warp-uniform decision
          if (lane == 0) atomicOr(flag, 2);
          ok = 0;
          break;
        }
      }
    }
    if (lane == 0) s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Panel factorisation over the whole GPU (cooperative launch, G <= SMs CTAs):
// the rows [c0, m) of the nb panel columns are split over the CTAs (rp <=
// kPgRows each, kept in shared memory) and column j costs one grid barrier.
// Before it every CTA writes its record rec[j][cta] = (|x_j|^2 over its rows,
// u_k = x_j^H a_k for k > j) and the owner of row j writes own[j] = (x_0,
// a_k[j]); after it every CTA adds the G records in the same fixed order, so
// all CTAs hold bitwise the same alpha, phi, beta and w_k = sum u_k + alpha
// conj(phi) a_k[j], and updates its own rows. Convention, skipping rule and
// outputs are those of the cluster kernel in panel mode: v below the diagonal
// and R entries above written back to A, per-column beta / alpha / phase /
// skip, and the panel's WY factor T from T^{-1} = diag(1/beta) +
// strictly-upper(V^H V) (partial Grams reduced over the grid, back substitution
// in CTA 0). Every wait is bounded (wait_ns from the kernel's start, 2 s by
// default): bit 2 of *flag on expiry; the CTA then skips its remaining waits
// and runs to its end (it only exchanges through global memory, so no peer
// can still be writing into its shared memory when it exits).
__global__ void __launch_bounds__(256) k_qb_panel_grid(double2* A, int64_t m, int c0, int nb, const double* sc,
                                                       double* beta, double* alpha, double2* phase, int* skip,
                                                       double2* T, double2* rec, double2* own, double2* gp,
                                                       double2* gf, unsigned* bar, int* flag, uint64_t wait_ns) {
  __shared__ double2 X[kNB][kPgRows];  // my rows of the panel, column-major
  __shared__ double2 red[kNB];         // this column's summed record: [0].x = |x|^2, [t] = sum u_{j+t}
  __shared__ double2 s_own[kNB];       // [0] = x_0, [t] = a_{j+t}[j]
  __shared__ double s_beta[kNB], s_alpha[kNB];
  __shared__ double2 s_phase[kNB], s_gam;
  __shared__ int s_skip[kNB];
  __shared__ double2 s_gf[kNpair];
  if (aborted(sc)) return;  // uniform over the grid
  const double thr = sc[0];
  const int G = gridDim.x, me = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t Rrows = m - c0;
  const int rp = (int)((Rrows + G - 1) / G);
  const int64_t r0 = (int64_t)me * rp;
  const int nr = (int)max((int64_t)0, min(Rrows, r0 + rp) - r0);
  const uint64_t deadline = gtimer() + wait_ns;
  bool alive = true;
  for (int t = tid; t < nb * rp; t += blockDim.x) {
    const int c = t / rp, i = t % rp;
    X[c][i] = i < nr ? A[(int64_t)(c0 + c) * m + c0 + r0 + i] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    const int i0 = (int)max((int64_t)0, (int64_t)j - r0);
    const bool ownr = j >= r0 && j < r0 + nr;
    const int lrow = (int)(j - r0);
    // record of my rows: task 0 = |x_j|^2, task t = u_{j+t}
    for (int task = wid; task < nb - j; task += 8) {
      double2 u = make_double2(0.0, 0.0);
      if (task == 0) {
        for (int i = i0 + lane; i < nr; i += 32) u.x = fma(X[j][i].x, X[j][i].x, fma(X[j][i].y, X[j][i].y, u.x));
      } else {
        const int k = j + task;
        for (int i = i0 + lane; i < nr; i += 32) u = cfmaj(X[j][i], X[k][i], u);
      }
      u.x = wsum(u.x);
      u.y = wsum(u.y);
      if (lane == 0) rec[((int64_t)j * kBlkCap + me) * kNB + task] = u;
    }
    if (ownr)
      for (int k = j + tid; k < nb; k += blockDim.x) own[j * kNB + k] = X[k][lrow];
    if (alive) alive = grid_arrive_wait(bar, (unsigned)((j + 1) * G), true, deadline, flag);
    {  // sum the G records in a fixed order: 16 threads per task, then a butterfly
      const int task = tid >> 4, sub = tid & 15;
      // the owner's record, loaded together with the CTA records
      const double2 ow = tid < nb - j ? __ldcg(&own[j * kNB + j + tid]) : make_double2(0.0, 0.0);
      double2 v = make_double2(0.0, 0.0);
      if (task < nb - j) {
        double2 a[kBlkCap / 16];
#pragma unroll
        for (int q = 0; q < kBlkCap / 16; ++q) {
          const int c = sub + 16 * q;
          a[q] = c < G ? __ldcg(&rec[((int64_t)j * kBlkCap + c) * kNB + task]) : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int h = kBlkCap / 32; h > 0; h >>= 1)  // pairwise, fixed order
#pragma unroll
          for (int q = 0; q < h; ++q) {
            a[q].x += a[q + h].x;
            a[q].y += a[q + h].y;
          }
        v = a[0];
      }
      for (int o = 8; o > 0; o >>= 1) {  // within each group of 16 lanes
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
      }
      if (sub == 0 && task < nb - j) red[task] = v;
      if (tid < nb - j) s_own[tid] = ow;
    }
    __syncthreads();
    if (wid == 0) {  // alpha, phi, beta as in the cluster kernel (two lanes share a sqrt and a division)
      const double a2 = red[0].x;
      const double2 x0 = s_own[0];
      const double rt = sqrt(lane == 1 ? fma(x0.x, x0.x, x0.y * x0.y) : a2);
      const double al = __shfl_sync(0xffffffffu, rt, 0);
      const double ax0 = __shfl_sync(0xffffffffu, rt, 1);
      if (!(al > thr)) {
        if (lane == 0) {
          s_skip[j] = 1;
          s_beta[j] = 0.0;
          s_alpha[j] = 0.0;
          s_phase[j] = make_double2(1.0, 0.0);
        }
      } else {
        const double rc = 1.0 / (lane == 1 ? al * (al + ax0) : ax0);
        const double inv = __shfl_sync(0xffffffffu, rc, 0);
        const double be = __shfl_sync(0xffffffffu, rc, 1);
        const double2 phi = ax0 > 0.0 ? make_double2(x0.x * inv, x0.y * inv) : make_double2(1.0, 0.0);
        if (lane == 0) {
          s_skip[j] = 0;
          s_beta[j] = be;
          s_alpha[j] = al;
          s_phase[j] = make_double2(-phi.x, -phi.y);
          s_gam = make_double2(al * phi.x, -al * phi.y);
          if (ownr) X[j][lrow] = make_double2(fma(phi.x, al, x0.x), fma(phi.y, al, x0.y));
        }
      }
    }
    __syncthreads();
    if (s_skip[j]) {
      for (int i = i0 + tid; i < nr; i += blockDim.x) X[j][i] = make_double2(0.0, 0.0);
    } else {
      const double be = s_beta[j];
      const double2 gam = s_gam;
      const int nk = nb - j - 1, len = nr - i0;
      for (int t = tid; len > 0 && t < nk * len; t += blockDim.x) {
        const int k = j + 1 + t / len, i = i0 + t % len;
        const double2 rj = s_own[k - j];
        double2 w = red[k - j];
        w.x = fma(gam.x, rj.x, fma(-gam.y, rj.y, w.x));
        w.y = fma(gam.x, rj.y, fma(gam.y, rj.x, w.y));
        const double2 bw = make_double2(be * w.x, be * w.y);
        X[k][i] = cfms(X[j][i], bw, X[k][i]);
      }
    }
    __syncthreads();
  }
  // write back: v below the diagonal, R entries above; per-column scalars
  for (int t = tid; t < nb * nr; t += blockDim.x) {
    const int c = t / nr, i = t % nr;
    A[(int64_t)(c0 + c) * m + c0 + r0 + i] = X[c][i];
  }
  if (me == 0)
    for (int c = tid; c < nb; c += blockDim.x) {
      beta[c0 + c] = s_beta[c];
      alpha[c0 + c] = s_alpha[c];
      phase[c0 + c] = s_phase[c];
      skip[c0 + c] = s_skip[c];
    }
  // partial strictly-upper Gram of my rows (v_a vanishes above row a)
  const int npair = nb * (nb - 1) / 2;
  for (int pq = tid; pq < npair; pq += blockDim.x) {
    int b = 1;
    while ((b + 1) * b / 2 <= pq) ++b;
    const int a = pq - b * (b - 1) / 2;
    double2 g = make_double2(0.0, 0.0);
    for (int i = (int)max((int64_t)0, (int64_t)b - r0); i < nr; ++i) g = cfmaj(X[a][i], X[b][i], g);
    gp[(int64_t)me * kNpair + pq] = g;
  }
  if (alive) alive = grid_arrive_wait(bar, (unsigned)((nb + 1) * G), true, deadline, flag);
  // full Gram entry pq (CTA pq mod G, warp 0): the G partials in a fixed order
  for (int pq = me; pq < npair; pq += G) {
    if (wid == 0) {
      double2 g = make_double2(0.0, 0.0);
      for (int c = lane; c < G; c += 32) {
        const double2 v = __ldcg(&gp[(int64_t)c * kNpair + pq]);
        g.x += v.x;
        g.y += v.y;
      }
      g.x = wsum(g.x);
      g.y = wsum(g.y);
      if (lane == 0) gf[pq] = g;
    }
  }
  // CTA 0 waits for the whole Gram, then solves T column by column
  if (alive) alive = grid_arrive_wait(bar, (unsigned)((nb + 2) * G), me == 0, deadline, flag);
  if (me != 0) return;
  for (int pq = tid; pq < npair; pq += blockDim.x) s_gf[pq] = __ldcg(&gf[pq]);
  __syncthreads();
  for (int c = wid; c < nb; c += 8) {
    double2 acc = make_double2(lane == c ? 1.0 : 0.0, 0.0);
    for (int a = c; a >= 0; --a) {
      const double ba = s_beta[a];
      double2 ta = make_double2(ba * acc.x, ba * acc.y);
      ta.x = __shfl_sync(0xffffffffu, ta.x, a);
      ta.y = __shfl_sync(0xffffffffu, ta.y, a);
      if (lane == a) T[a * nb + c] = ta;
      if (lane < a) acc = cfms(s_gf[a * (a - 1) / 2 + lane], ta, acc);
    }
    for (int a = c + 1 + lane; a < nb; a += 32) T[a * nb + c] = make_double2(0.0, 0.0);
  }
}

__global__ void k_qb_identity(double2* X, int64_t m, int64_t n, const double* sc) {
  if (aborted(sc)) return;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m * n; k += (int64_t)gridDim.x * blockDim.x)
  {
    int64_t r;
    const int64_t c = idivmod(k, m, r);
    X[k] = make_double2(r == c ? 1.0 : 0.0, 0.0);
  }
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
    int64_t c;
    const int64_t i = idivmod(k, n, c);
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
    int64_t r, rb;
    const int64_t c = idivmod(k, m, r);
    const double2 q = X[k], p = phase[c];
    const double2 qp = make_double2(q.x * p.x - q.y * p.y, q.x * p.y + q.y * p.x);
    const int64_t ra = idivmod(r, dd[lb], rb);
    const int64_t at = c * st[leg] + ra * st[la] + rb * st[lb];
    U[at] = qp;
    if (U_lo) U_lo[at] = make_float2((float)qp.x, (float)qp.y);
  }
}

}  // namespace

int64_t qr_blocked_elems(int64_t m, int64_t n) { return qb_layout(m, n).total; }

bool launch_qr_blocked(double2* U, int d0, int d1, int d2, int leg, double tol, double2* work,
                       int64_t work_elems, double2* qbuf, double2* R, int* flag, float2* U_lo, float2* R_lo,
                       cudaStream_t s, uint64_t grid_wait_ns) {
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
  unsigned* bar = (unsigned*)(work + L.bar);

  static int sms = 0, coop = 0, occ = 0;  // SMs (one CTA each for the FP64-bound kernels), cooperative launch
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 1;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess) coop = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_qb_panel_grid, 256, 0) != cudaSuccess) occ = 0;
  }
  // a panel over the whole GPU (one grid barrier per column) when the device
  // guarantees co-residency; else on one cluster
  auto panel = [&](const QrPanel& pn, int idx) -> bool {
    const int64_t rows = m - pn.c0;
    const int G = (int)std::min<int64_t>(std::min(sms, kBlkCap), (rows + 7) / 8);
    if (coop && occ >= 1 && G >= 1 && (rows + G - 1) / G <= kPgRows) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(G, 1, 1);
      cfg.blockDim = dim3(256, 1, 1);
      cfg.stream = s;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeCooperative;
      at[0].val.cooperative = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      return cudaLaunchKernelEx(&cfg, k_qb_panel_grid, A, (int64_t)m, pn.c0, pn.nb, (const double*)sc, beta, alpha,
                                phase, skip, pn.T, work + L.rec, work + L.own, work + L.gp, work + L.gf, bar + 8 * idx,
                                flag, grid_wait_ns) == cudaSuccess;
    }
    return launch_qr_panel(pn, s);
  };
  const int g1 = (int)std::min<int64_t>(kGatherMax, (m * n + 255) / 256);
  k_qb_gather<<<g1, 256, 0, s>>>(U, d0, d1, d2, leg, A, m, n, part);
  k_qb_norm<<<1, 32, 0, s>>>(part, g1, tol, sc, flag, bar);
  // factorisation: panel, then its reflectors on the trailing columns
  for (int c0 = 0; c0 < n; c0 += kNB) {
    const int nb = std::min(kNB, n - c0);
    QrPanel pn{nullptr, A, (int)m, n, c0, nb, sc, beta, alpha, phase, skip, T + (int64_t)(c0 / kNB) * kNB * kNB};
    if (!panel(pn, c0 / kNB)) return false;
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
