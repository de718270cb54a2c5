// Householder QR of a node tensor spread over a thread-block cluster (FP64).
//
// GB300 retires FP64 at a small fraction of its FP32 rate: a warp issues one
// FP64 instruction per ~64 cycles, an SM about one per ~19 cycles, and an FP64
// square root or division costs ~600 cycles. The kernel is therefore laid out
// to keep the number of FP64 warp instructions on the critical path small:
//
//  * the m rows are split over C <= 16 CTAs of one cluster, each keeping its
//    row block in shared memory;
//  * a column costs ONE exchange: every CTA pushes (st.async into the other
//    CTAs' shared memory, completing bytes on their mbarrier) its partial
//    squared norm of column j and its partial dots u_k = x_j^H a_k, k > j, and
//    the CTA owning row j adds x_0 and row j of the trailing columns. With
//    v = x + phi*alpha*e_0 the reflector dot is then w_k = sum u_k + alpha
//    conj(phi) a_k[j], so norm and dots need no second round trip;
//  * alpha, phi and beta are computed by one warp (two lanes share each sqrt
//    and division) while the other warps sum the pushed dot partials;
//  * the update and the next column's partials use groups of 8 lanes per
//    trailing column (rows strided over the group), so each warp instruction
//    covers 4 columns;
//  * Q is formed from the compact WY form H_0..H_{n-1} = I - V T V^H, but
//    instead of the sequential recurrence for T, M = T V_top^H is obtained by
//    back substitution with T^{-1} = diag(1/beta) + strictly-upper(V^H V)
//    (Joffrain, Low, Quintana-Orti, van de Geijn, Van Zee 2006), one column of
//    M per warp, spread over the cluster.
//
// The arithmetic convention is the one of the CPU oracle and of the one-CTA
// kernel: for column j with remainder x of norm alpha, alpha <= tol*||A||_F
// means no reflector (R_jj = 0, Q column H_0..H_{j-1} e_j); otherwise
// v = x + phi*alpha*e_0, phi = x_0/|x_0| (1 if x_0 = 0), beta = 1/(alpha(alpha+|x_0|)),
// and finally row j of R / column j of Q are rescaled by the phase -phi so
// that diag(R) >= 0. All reductions run in a fixed order, so results are
// bitwise reproducible. Every wait on a peer is bounded (2 s from the kernel
// start): on expiry bit 2 of *flag is set and the kernel runs to its end
// without further exchanges.
#include <cooperative_groups.h>

#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace ttn {

namespace {

constexpr int kThreads = 256;
constexpr int kNW = kThreads / 32;
// G = lanes per trailing-column group (8 for whole small matrices, 32 for
// panels of tall matrices, whose row blocks are long)
template <int G> struct Grp {
  static constexpr int kGPW = 32 / G;             // column groups per warp
  static constexpr int kSlots = (kNW - 1) * kGPW;  // column groups of warps 1..7
  static constexpr int kMaxPass = (kQrClusterMaxN - 1 + kSlots - 1) / kSlots;
};
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double2 cfmaj(double2 a, double2 b, double2 c) {  // conj(a)*b + c
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(-a.y, b.x, c.y);
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
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
// sum over aligned groups of G lanes; every lane of a group gets the same bits
template <int G>
__device__ __forceinline__ double2 gsum2(double2 v) {
  for (int o = G / 2; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(kFull, v.x, o);
    v.y += __shfl_xor_sync(kFull, v.y, o);
  }
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

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// address of the same shared variable in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t mapa(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_init(uint64_t* mb, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mb)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* mb, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mb)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* mb, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(mb)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for the phase of the given parity; false (and bit 2 of *flag) once the
// kernel-wide deadline has passed.
__device__ __forceinline__ bool mbar_wait(uint64_t* mb, uint32_t parity, uint64_t deadline, int* flag) {
  while (!mbar_try(mb, parity)) {
    if (gtimer() > deadline) {
      atomicOr(flag, 2);
      return false;
    }
  }
  return true;
}
// remote stores into another CTA's shared memory that complete bytes on its mbarrier
__device__ __forceinline__ void push_f64(uint32_t raddr, double v, uint32_t rmb) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f64 [%0], %1, [%2];" ::"r"(raddr), "d"(v),
               "r"(rmb)
               : "memory");
}
__device__ __forceinline__ void push_c64(uint32_t raddr, double2 v, uint32_t rmb) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];" ::"r"(raddr),
               "d"(v.x), "d"(v.y), "r"(rmb)
               : "memory");
}

}  // namespace

// Shared-memory layout (dynamic, double2 units):
//   A   [n][rp]     my row block, column-major (v_j overwrites rows >= j of column j)
//   SU  [2][16][n]  per-parity dot partials u_k pushed by each CTA
//   RJ  [2][n]      per-parity row j of the trailing columns (from the owner of row j)
//   G   [n][n]      partial strictly-upper Gram of my rows, later the gathered M
//   GF  [n][n]      full strictly-upper Gram
//   MM  [n][n]      the columns of M solved by this CTA
template <int GL>
__global__ void __launch_bounds__(kThreads) k_qr_cluster(double2* U, int d0, int d1, int d2, int leg,
                                                         double tol, double2* R, int* flag, float2* U_lo,
                                                         float2* R_lo, QrPanel pn) {
  using Gp = Grp<GL>;
  constexpr int kGPW = Gp::kGPW, kSlots = Gp::kSlots, kMaxPass = Gp::kMaxPass;
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int me = (int)cluster.block_rank();
  const int dd[3] = {d0, d1, d2};
  const int64_t st[3] = {(int64_t)d1 * d2, d2, 1};
  const int la = leg == 0 ? 1 : 0, lb = leg == 2 ? 1 : 2;
  // panel mode: factor columns [c0, c0+nb) of the column-major m x n matrix
  // pn.A over rows [c0, m) -- an (m - c0) x nb matrix in its own right
  const bool panel = pn.A != nullptr;
  const int n = panel ? pn.nb : dd[leg];
  const int m = panel ? pn.m - pn.c0 : dd[la] * dd[lb];
  const int rp = (m + C - 1) / C;
  const int r0 = me * rp;
  const int nr = max(0, min(m, r0 + rp) - r0);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5;
  const uint64_t deadline = gtimer() + 2000000000ull;

  extern __shared__ double2 smem[];
  double2* A = smem;
  double2* SU = A + (size_t)n * rp;
  double2* RJ = SU + 32 * (size_t)n;
  // Gram / M buffers: shared memory, or (large n) per-CTA regions of pn.gtail
  const bool gt = !panel && pn.gtail != nullptr;
  const size_t n2 = (size_t)n * n;
  double2* G = gt ? pn.gtail + (size_t)me * n2 : RJ + 2 * (size_t)n;
  double2* GF = gt ? pn.gtail + (size_t)(C + me) * n2 : G + n2;
  double2* MM = gt ? pn.gtail + (size_t)(2 * C + me) * n2 : GF + n2;
  // the partial Gram / M of CTA c, as seen from this CTA
  auto G_of = [&](int c) -> const double2* { return gt ? pn.gtail + (size_t)c * n2 : cluster.map_shared_rank(G, c); };
  auto MM_of = [&](int c) -> const double2* {
    return gt ? pn.gtail + (size_t)(2 * C + c) * n2 : cluster.map_shared_rank(MM, c);
  };
  __shared__ __align__(8) uint64_t mb[2];
  __shared__ double SN[2][16];
  __shared__ double2 SX[2];
  __shared__ double red[kNW];
  __shared__ double s_part, s_frob;
  __shared__ double s_beta[kQrClusterMaxN], s_alpha[kQrClusterMaxN];
  __shared__ int s_skip[kQrClusterMaxN];
  __shared__ double2 s_phase[kQrClusterMaxN];
  __shared__ double2 s_gam;
  if (tid == 0) {
    mbar_init(&mb[0], 1);
    mbar_init(&mb[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }

  // gather my rows: A[c][i] = U[.. row r0+i, column c ..] (panel: pn.A[c0+c][c0+r0+i])
  double fro = 0.0;
  for (int k = tid; k < n * rp; k += nt) {
    const int c = k / rp, i = k % rp;
    double2 v = make_double2(0.0, 0.0);
    if (i < nr) {
      const int r = r0 + i;
      v = panel ? pn.A[(int64_t)(pn.c0 + c) * pn.m + pn.c0 + r]
                : U[c * st[leg] + (int64_t)(r / dd[lb]) * st[la] + (int64_t)(r % dd[lb]) * st[lb]];
    }
    A[k] = v;
    fro = fma(v.x, v.x, fma(v.y, v.y, fro));
  }
  fro = bsum(fro, red);
  if (tid == 0) s_part = fro;
  cluster.sync();  // partial norms visible, mbarriers initialised cluster-wide
  if (wid == 0) {  // lane c reads CTA c's partial; fixed butterfly order
    double v = lane < C ? *cluster.map_shared_rank(&s_part, lane) : 0.0;
    v = wsum(v);
    if (lane == 0) s_frob = sqrt(v);
  }
  __syncthreads();
  // the threshold of a panel is the one of the whole matrix (NaN: abort)
  const double frob = panel ? *pn.thr : s_frob;
  if (!isfinite(frob)) {  // uniform across the cluster
    if (tid == 0 && me == 0 && !panel) atomicOr(flag, 1);
    cluster.sync();
    return;
  }
  const double thr = panel ? frob : tol * frob;  // s_part stays untouched until the final cluster barrier
  bool alive = true;

  // Partials of step j over my rows >= j, pushed into every CTA's slots of
  // parity j&1: ||x_j||^2 (warp 0), u_k = x_j^H a_k for k > j (column groups);
  // the CTA owning row j also pushes x_0 and a_k[j].
  auto push_partials = [&](int j) {
    const int p = j & 1;
    const int i0 = max(0, j - r0);
    const double2* x = A + (size_t)j * rp;
    const bool own = j >= r0 && j < r0 + nr;
    const int lrow = j - r0;
    if (tid == 0) {
      const uint32_t nk = (uint32_t)(n - j - 1);
      mbar_arrive_tx(&mb[p], 8u * C + 16u * C * nk + (j < m ? 16u + 16u * nk : 0u));
    }
    if (wid == 0) {
      double ss = 0.0;
      for (int i = i0 + lane; i < nr; i += 32) ss = fma(x[i].x, x[i].x, fma(x[i].y, x[i].y, ss));
      ss = wsum(ss);
      if (alive && lane < C) {
        const uint32_t rmb = mapa(smem_u32(&mb[p]), lane);
        push_f64(mapa(smem_u32(&SN[p][me]), lane), ss, rmb);
        if (own) push_c64(mapa(smem_u32(&SX[p]), lane), x[lrow], rmb);
      }
    } else {
      const int q = (wid - 1) * kGPW + lane / GL, sl = lane % GL;
      for (int kb = j + 1; kb < n; kb += kSlots) {  // block-uniform trip count
        const int k = kb + q;
        const double2* a = A + (size_t)min(k, n - 1) * rp;
        double2 u = make_double2(0.0, 0.0);
        if (k < n)
          for (int i = i0 + sl; i < nr; i += GL) u = cfmaj(x[i], a[i], u);
        u = gsum2<GL>(u);
        if (alive && k < n) {
          const uint32_t su = smem_u32(&SU[((size_t)p * 16 + me) * n + k]);
          const uint32_t rj = smem_u32(&RJ[(size_t)p * n + k]);
          const uint32_t lmb = smem_u32(&mb[p]);
          for (int c = sl; c < C; c += GL) {
            const uint32_t rmb = mapa(lmb, c);
            push_c64(mapa(su, c), u, rmb);
            if (own) push_c64(mapa(rj, c), a[lrow], rmb);
          }
        }
      }
    }
  };

  // Column loop (see the header): wait for step j's partials, scalars in warp
  // 0 / dot sums in warps 1..7, barrier, update, barrier, push step j+1.
  // A push for step j+2 (same parity as j) can only leave a CTA after every
  // CTA has pushed for step j+1, i.e. after all threads here have passed the
  // second barrier of step j and are done with step j's slots and phase.
  push_partials(0);
  uint32_t ph[2] = {0u, 0u};
  for (int j = 0; j < n; ++j) {
    const int p = j & 1;
    const int i0 = max(0, j - r0);
    double2* x = A + (size_t)j * rp;
    const bool own = j >= r0 && j < r0 + nr;
    const int lrow = j - r0;
    if (alive) alive = mbar_wait(&mb[p], ph[p], deadline, flag);
    ph[p] ^= 1u;
    double2 W[kMaxPass];
    if (wid == 0) {
      double a2 = lane < C ? SN[p][lane] : 0.0;  // C <= 16: lanes 0..15 carry the sum
      for (int o = 8; o > 0; o >>= 1) a2 += __shfl_xor_sync(kFull, a2, o);
      const double2 x0 = j < m ? SX[p] : make_double2(0.0, 0.0);
      // lane 0: alpha = sqrt(sum), lane 1: |x_0| (one sqrt for both)
      const double rt = sqrt(lane == 1 ? fma(x0.x, x0.x, x0.y * x0.y) : a2);
      const double alpha = __shfl_sync(kFull, rt, 0);
      const double ax0 = __shfl_sync(kFull, rt, 1);
      if (!(alpha > thr)) {
        for (int i = i0 + lane; i < nr; i += 32) x[i] = make_double2(0.0, 0.0);
        if (lane == 0) {
          s_skip[j] = 1;
          s_beta[j] = 0.0;
          s_alpha[j] = 0.0;
          s_phase[j] = make_double2(1.0, 0.0);
        }
      } else {
        // lane 0: 1/|x_0|, lane 1: beta (one division for both)
        const double rc = 1.0 / (lane == 1 ? alpha * (alpha + ax0) : ax0);
        const double inv = __shfl_sync(kFull, rc, 0);
        const double beta = __shfl_sync(kFull, rc, 1);
        const double2 phi = ax0 > 0.0 ? make_double2(x0.x * inv, x0.y * inv) : make_double2(1.0, 0.0);
        if (lane == 0) {
          s_skip[j] = 0;
          s_beta[j] = beta;
          s_alpha[j] = alpha;
          s_phase[j] = make_double2(-phi.x, -phi.y);
          s_gam = make_double2(alpha * phi.x, -alpha * phi.y);
          if (own) x[lrow] = make_double2(fma(phi.x, alpha, x0.x), fma(phi.y, alpha, x0.y));
        }
      }
    } else {
      const int q = (wid - 1) * kGPW + lane / GL, sl = lane % GL;
#pragma unroll
      for (int ps = 0; ps < kMaxPass; ++ps) {
        const int k = j + 1 + ps * kSlots + q;
        if (j + 1 + ps * kSlots >= n) break;  // block-uniform
        double2 w = make_double2(0.0, 0.0);
        if (k < n)
          for (int c = sl; c < C; c += GL) {
            const double2 t = SU[((size_t)p * 16 + c) * n + k];
            w.x += t.x;
            w.y += t.y;
          }
        W[ps] = gsum2<GL>(w);
      }
    }
    __syncthreads();
    if (wid > 0 && !s_skip[j]) {
      const double beta = s_beta[j];
      const double2 gam = s_gam;
      const int q = (wid - 1) * kGPW + lane / GL, sl = lane % GL;
#pragma unroll
      for (int ps = 0; ps < kMaxPass; ++ps) {
        const int k = j + 1 + ps * kSlots + q;
        if (j + 1 + ps * kSlots >= n) break;
        if (k < n) {
          const double2 rj = RJ[(size_t)p * n + k];
          double2 w = W[ps];
          w.x = fma(gam.x, rj.x, fma(-gam.y, rj.y, w.x));
          w.y = fma(gam.x, rj.y, fma(gam.y, rj.x, w.y));
          const double2 bw = make_double2(beta * w.x, beta * w.y);
          double2* a = A + (size_t)k * rp;
          for (int i = i0 + sl; i < nr; i += GL) a[i] = cfms(x[i], bw, a[i]);
        }
      }
    }
    __syncthreads();
    if (j + 1 < n) push_partials(j + 1);
  }
  cluster.sync();  // all reflectors final everywhere, every pushed slot consumed
  if (panel) {
    // write the panel back (v below the diagonal, R entries above), the
    // per-column scalars, and the WY factor T of the panel:
    // T^{-1} = diag(1/beta) + strictly-upper(V^H V), column c of T solved by
    // back substitution from e_c (skipped reflectors give zero rows/columns)
    for (int k = tid; k < n * nr; k += nt) {
      const int c = k / nr, i = k % nr;
      pn.A[(int64_t)(pn.c0 + c) * pn.m + pn.c0 + r0 + i] = A[(size_t)c * rp + i];
    }
    if (me == 0)
      for (int c = tid; c < n; c += nt) {
        pn.beta[pn.c0 + c] = s_beta[c];
        pn.alpha[pn.c0 + c] = s_alpha[c];
        pn.phase[pn.c0 + c] = s_phase[c];
        pn.skip[pn.c0 + c] = s_skip[c];
      }
  }

  // R rows owned here (global rows < n), diag(R) = alpha >= 0 after the phase fix
  for (int k = tid; !panel && k < n * n; k += nt) {
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
  // partial strictly-upper Gram of my rows, one thread per pair a < b
  // (v_a vanishes above row a; skipped reflectors are zero columns)
  const int npair = n * (n - 1) / 2;
  for (int t = tid; t < npair; t += nt) {
    int b = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)t)) * 0.5f);  // t = b(b-1)/2 + a
    while (b * (b - 1) / 2 > t) --b;
    while ((b + 1) * b / 2 <= t) ++b;
    const int a = t - b * (b - 1) / 2;
    double2 g = make_double2(0.0, 0.0);
    const double2* va = A + (size_t)a * rp;
    const double2* vb = A + (size_t)b * rp;
    for (int i = max(b - r0, 0); i < nr; ++i) g = cfmaj(va[i], vb[i], g);
    G[a * n + b] = g;
  }
  cluster.sync();
  // full Gram: fixed-order sum of the CTAs' partials
  for (int t = tid; t < npair; t += nt) {
    int b = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)t)) * 0.5f);
    while (b * (b - 1) / 2 > t) --b;
    while ((b + 1) * b / 2 <= t) ++b;
    const int a = t - b * (b - 1) / 2;
    double2 v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c)
      v[c] = c < C ? G_of(c)[a * n + b] : make_double2(0.0, 0.0);
    double2 g = make_double2(0.0, 0.0);
#pragma unroll
    for (int c = 0; c < 16; ++c)
      if (c < C) {
        g.x += v[c].x;
        g.y += v[c].y;
      }
    GF[a * n + b] = g;
  }
  __syncthreads();
  if (panel) {
    for (int c = me + C * wid; c < n; c += C * kNW) {
      double2 acc0 = make_double2(lane == c ? 1.0 : 0.0, 0.0), acc1 = make_double2(lane + 32 == c ? 1.0 : 0.0, 0.0);
      for (int a = c; a >= 0; --a) {
        const double ba = s_beta[a];
        const double2 src = a < 32 ? acc0 : acc1;
        double2 ta = make_double2(ba * src.x, ba * src.y);
        ta.x = __shfl_sync(kFull, ta.x, a & 31);
        ta.y = __shfl_sync(kFull, ta.y, a & 31);
        if (lane == (a & 31)) pn.T[a * n + c] = ta;
        if (lane < a) acc0 = cfms(GF[lane * n + a], ta, acc0);
        if (a > 32 && lane + 32 < a) acc1 = cfms(GF[(lane + 32) * n + a], ta, acc1);
      }
      for (int a = c + 1 + lane; a < n; a += 32) pn.T[a * n + c] = make_double2(0.0, 0.0);
    }
    cluster.sync();  // keep shared memory alive until every remote read has finished
    return;
  }
  // M = T V_top^H column by column: T^{-1} M[:, c] = conj(V_top[c, :])^T, with
  // T^{-1} = diag(1/beta) + strictly-upper Gram; back substitution from a = c
  // down (M[a][c] = 0 for a > c). Column c is solved by CTA c mod C, one warp.
  for (int c = me + C * wid; c < n; c += C * kNW) {
    double2 acc0 = make_double2(0.0, 0.0), acc1 = make_double2(0.0, 0.0);
    if (c < m) {
      const int oc = c / rp;
      const double2* Ar = cluster.map_shared_rank(A, oc);
      const int lr = c - oc * rp;
      if (lane <= c && lane < n && !s_skip[lane]) {
        const double2 v = Ar[(size_t)lane * rp + lr];
        acc0 = make_double2(v.x, -v.y);
      }
      if (lane + 32 <= c && lane + 32 < n && !s_skip[lane + 32]) {
        const double2 v = Ar[(size_t)(lane + 32) * rp + lr];
        acc1 = make_double2(v.x, -v.y);
      }
    }
    for (int a = c; a >= 0; --a) {
      const double ba = s_beta[a];
      const double2 src = a < 32 ? acc0 : acc1;
      double2 ma = make_double2(ba * src.x, ba * src.y);
      ma.x = __shfl_sync(kFull, ma.x, a & 31);
      ma.y = __shfl_sync(kFull, ma.y, a & 31);
      if (lane == (a & 31)) MM[a * n + c] = ma;
      if (lane < a) acc0 = cfms(GF[lane * n + a], ma, acc0);
      if (a > 32 && lane + 32 < a) acc1 = cfms(GF[(lane + 32) * n + a], ma, acc1);
    }
    for (int a = c + 1 + lane; a < n; a += 32) MM[a * n + c] = make_double2(0.0, 0.0);
  }
  cluster.sync();  // every column of M solved; partial Grams no longer read
  // gather M into G (column c from CTA c mod C)
  for (int t = tid; t < n * n; t += nt) G[t] = MM_of((t % n) % C)[t];
  __syncthreads();
  // Q rows: Q[r][c] = delta_rc - sum_{a <= min(r,c)} v_a[r] M[a][c], column c scaled by phase_c
  const int nch = (nr + 31) / 32;
  for (int task = wid; task < n * nch; task += kNW) {
    const int c = task / nch, i = (task % nch) * 32 + lane;
    if (i >= nr) continue;
    const int r = r0 + i;
    double2 q = make_double2(r == c ? 1.0 : 0.0, 0.0);
    const int amax = min(c, r);
    for (int a = 0; a <= amax; ++a) q = cfms(A[(size_t)a * rp + i], G[a * n + c], q);
    const double2 p = s_phase[c];
    const double2 qp = make_double2(q.x * p.x - q.y * p.y, q.x * p.y + q.y * p.x);
    const int64_t at = c * st[leg] + (int64_t)(r / dd[lb]) * st[la] + (int64_t)(r % dd[lb]) * st[lb];
    U[at] = qp;
    if (U_lo) U_lo[at] = make_float2((float)qp.x, (float)qp.y);
  }
  cluster.sync();  // keep shared memory alive until every remote read has finished
}

constexpr size_t kQrSmemCap = 200 * 1024;

size_t qr_cluster_smem(int m, int n, int C, bool gtail) {
  const int rp = (m + C - 1) / C;
  return sizeof(double2) * ((size_t)n * rp + 34 * (size_t)n + (gtail ? 0 : 3 * (size_t)n * n));
}
size_t qr_cluster_smem(int m, int n, int C) { return qr_cluster_smem(m, n, C, false); }

// Cluster size for an m x n QR (0: does not fit); *gtail set when the Gram / M
// buffers have to live in global memory.
int qr_cluster_size(int m, int n, bool* gtail) {
  *gtail = false;
  if (n > kQrClusterMaxN) return 0;
  int C = (m + 7) / 8;  // about 8 rows per CTA: the factorisation is FP64-issue bound
  C = C < 1 ? 1 : (C > 16 ? 16 : C);
  if (qr_cluster_smem(m, n, C, false) <= kQrSmemCap) return C;
  if (qr_cluster_smem(m, n, C, true) <= kQrSmemCap) {
    *gtail = true;
    return C;
  }
  return 0;
}
int qr_cluster_size(int m, int n) {
  bool gt;
  const int C = qr_cluster_size(m, n, &gt);
  return gt ? 0 : C;
}

template <int G>
static bool launch_cluster(double2* U, int d0, int d1, int d2, int leg, double tol, double2* R, int* flag,
                           float2* U_lo, float2* R_lo, const QrPanel& pn, int m, int n, int C, cudaStream_t s) {
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(k_qr_cluster<G>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(k_qr_cluster<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kQrSmemCap);
    attr_done = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = qr_cluster_smem(m, n, C, !pn.A && pn.gtail);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_qr_cluster<G>, U, d0, d1, d2, leg, tol, R, flag, U_lo, R_lo, pn) == cudaSuccess;
}

bool launch_qr_cluster(double2* U, int d0, int d1, int d2, int leg, double tol, double2* R, int* flag,
                       float2* U_lo, float2* R_lo, double2* scratch, int64_t scratch_elems, cudaStream_t s) {
  const int dd[3] = {d0, d1, d2};
  const int n = dd[leg];
  const int m = (int)((int64_t)d0 * d1 * d2 / n);
  bool gt = false;
  const int C = qr_cluster_size(m, n, &gt);
  if (C == 0) return false;
  QrPanel pn = {};
  if (gt) {
    if (!scratch || scratch_elems < 3 * (int64_t)C * n * n) return false;
    pn.gtail = scratch;
  }
  return launch_cluster<8>(U, d0, d1, d2, leg, tol, R, flag, U_lo, R_lo, pn, m, n, C, s);
}

int qr_panel_cluster(int m_act, int nb) {
  int C = (m_act + 7) / 8;
  C = C < 1 ? 1 : (C > 16 ? 16 : C);
  return qr_cluster_smem(m_act, nb, C) > kQrSmemCap ? 0 : C;
}

bool launch_qr_panel(const QrPanel& pn, cudaStream_t s) {
  const int m_act = pn.m - pn.c0;
  const int C = qr_panel_cluster(m_act, pn.nb);
  if (C == 0 || pn.nb > kQrPanelMaxNb) return false;
  return launch_cluster<32>(nullptr, 1, 1, 1, 0, 0.0, nullptr, nullptr, nullptr, nullptr, pn, m_act, pn.nb, C, s);
}

}  // namespace ttn
