// One-sided (Hestenes) Jacobi SVD spread over several CTAs, FP64 -- the
// factorisation that splits a merged pair in the adaptive-rank scheme (Sec. 2.3,
// last paragraph), for matrices too wide for one CTA.
//
// The working matrix holds the columns of Theta (or of Theta^H when Theta is
// wider than tall), column-major; V starts as the identity. A sweep visits every
// column pair once, in the rounds of the circle method: the pairs of one round
// are disjoint, so they are dealt to the CTAs and the round ends with one
// barrier -- the hardware barrier of a thread-block cluster when the pairs fit
// one cluster (at most 16 CTAs), else a grid barrier of one cooperative launch.
// A pair is handled by one CTA: its threads split the rows, the three Gram
// entries a = |x|^2, b = |y|^2, c = x^H y are summed in a fixed order (threads
// -> warps -> warp order), thread 0 computes the complex rotation
// (jacobi_rotation: skipped when |c| <= tol sqrt(a b) or a column is rounding
// noise) and the threads apply it to the pair's rows of the working matrix and
// of V. GB300 retires about one FP64 warp instruction per 19 cycles per SM, and
// a square root or quotient is a dozen of them: computing the rotation in one
// thread instead of all eight warps keeps the FP64 pipe for the rows.
// A sweep without any rotation ends the iteration: every CTA reads the sweep's
// rotation count after the sweep's last barrier. Which CTA handles a pair, and
// which barrier ends a round, does not change the arithmetic, so the result
// does not depend on the launch shape.
//
// The convergence threshold tol = 2 sqrt(max(rows, 64)) * DBL_EPSILON sits above
// the rounding noise of the Gram entries summed over the rows, so a converged
// matrix stops rotating; a run that reaches max_sweeps reports it (info[0] ==
// max_sweeps) and the host refuses the result.
//
// Every grid wait is bounded (wait_ns from the moment the CTA starts waiting);
// a CTA whose wait gives up sets bit 4 (value 16) of *flag and returns. Nothing
// is in flight when it does (plain loads and stores only), so any CTA may leave
// at any time; the others give up at their next barrier. The cluster barrier is
// the hardware's: all CTAs of a cluster are resident together and every CTA
// passes the same number of barriers.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include <cooperative_groups.h>

#include "../../include/ttn_heom.h"
#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace ttn {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kBarLanes = 8;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier: CTA c adds one to lane c % kBarLanes after a CTA barrier (which
// orders the CTA's writes before thread 0's release); warp 0 polls the lanes
// with acquire loads until their sum reaches target, then a CTA barrier orders
// the other CTAs' writes before this CTA's later reads. Returns false when the
// wait gave up.
__device__ bool grid_sync(unsigned* lanes, unsigned target, uint64_t wait_ns, int* flag) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    if (lane == 0) red_release_add(lanes + blockIdx.x % kBarLanes, 1u);
    const uint64_t t0 = now_ns();
    int ok = 1;
    for (;;) {
      unsigned v = lane < kBarLanes ? ld_acquire(lanes + lane) : 0u;
      for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (__shfl_sync(0xffffffffu, v, 0) >= target) break;
      if (__shfl_sync(0xffffffffu, (int)(now_ns() - t0 >= wait_ns), 0)) {  // wait_ns = 0: one poll
        if (lane == 0) atomicOr(flag, 16);
        ok = 0;
        break;
      }
    }
    if (lane == 0) s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Circle-method pair p of round rd among N (even) columns.
__device__ __forceinline__ void round_pair(int N, int rd, int p, int& i, int& j) {
  if (p == 0) {
    i = 0;
    j = 1 + rd;
  } else {
    i = 1 + (rd + p) % (N - 1);
    j = 1 + (rd - p + N - 1) % (N - 1);
  }
  if (i > j) {
    const int t = i;
    i = j;
    j = t;
  }
}

// Working matrix A (nr x nc, column-major) from theta (m x n, row-major): the
// columns of theta, or of theta^H when n > m. V = identity (nc x nc).
__global__ void k_svd_load(const double2* __restrict__ theta, int m, int n, double2* __restrict__ A,
                           double2* __restrict__ V) {
  const bool tr = n > m;
  const int nr = tr ? n : m, nc = tr ? m : n;
  const int64_t na = (int64_t)nr * nc, nv = (int64_t)nc * nc;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < na + nv;
       k += (int64_t)gridDim.x * blockDim.x) {
    if (k < na) {
      int64_t r;
      const int64_t c = idivmod(k, nr, r);
      A[k] = tr ? cconj(theta[c * n + r]) : theta[r * n + c];
    } else {
      const int64_t kv = k - na;
      int64_t rr;
      const int64_t cc = idivmod(kv, nc, rr);
      V[kv] = make_double2(rr == cc ? 1.0 : 0.0, 0.0);
    }
  }
}

// Barrier at the end of a phase: the hardware barrier of the cluster (release /
// acquire at cluster scope, which orders the global-memory writes of A and V
// too), or the grid barrier of a cooperative launch.
template <bool kCluster>
__device__ __forceinline__ bool phase_sync(unsigned* lanes, unsigned target, uint64_t wait_ns, int* flag) {
  if constexpr (kCluster) {
    cg::this_cluster().sync();
    return true;
  } else {
    return grid_sync(lanes, target, wait_ns, flag);
  }
}

// sync: [0, 8) barrier lanes, [8, 8 + max_sweeps) rotations per sweep; zeroed
// before the launch. kCluster: the CTAs form one thread-block cluster.
template <bool kCluster>
__global__ void __launch_bounds__(kThreads) k_jacobi_grid(double2* __restrict__ A, double2* __restrict__ V, int nr,
                                                          int nc, double* __restrict__ sigma, int* __restrict__ info,
                                                          unsigned* sync, int* flag, double tol, int max_sweeps,
                                                          int tr, uint64_t wait_ns) {
  static_assert(kWarps * 4 == 32, "warp 0 adds four sums of each warp, one per lane");
  __shared__ double s_red[kWarps][4];
  __shared__ double s_par[4];
  __shared__ int s_go;
  __shared__ unsigned s_total;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int G = gridDim.x;
  const int N = nc + (nc & 1), npairs = N / 2;
  unsigned nbar = 0;
  bool ok = true;
  // ||A||_F^2: column norms of columns jc = blockIdx.x (mod G) into sigma[]
  // (overwritten at the end), one barrier, then every CTA adds them in order
  for (int jc = blockIdx.x; jc < nc; jc += G) {
    const double2* x = A + (int64_t)jc * nr;
    double f = 0.0;
    for (int r = tid; r < nr; r += kThreads) f = fma(x[r].x, x[r].x, fma(x[r].y, x[r].y, f));
    f = wsum(f);
    if (lane == 0) s_red[wid][0] = f;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < kWarps; ++w) t += s_red[w][0];
      sigma[jc] = t;
    }
    __syncthreads();
  }
  ++nbar;
  ok = phase_sync<kCluster>(sync, nbar * (unsigned)G, wait_ns, flag);
  if (!ok) return;
  double fro2 = 0.0;
  for (int jc = 0; jc < nc; ++jc) fro2 += sigma[jc];
  const double tiny2 = jacobi_negligible(nr, fro2);
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    unsigned rot = 0;
    for (int rd = 0; rd < N - 1 && ok; ++rd) {
      for (int p = blockIdx.x; p < npairs; p += G) {
        int i, j;
        round_pair(N, rd, p, i, j);
        if (j >= nc) continue;  // the dummy column of an odd count
        double2* x = A + (int64_t)i * nr;
        double2* y = A + (int64_t)j * nr;
        double a = 0.0, b = 0.0, cr = 0.0, ci = 0.0;
        for (int r = tid; r < nr; r += kThreads) {
          const double2 xv = x[r], yv = y[r];
          a = fma(xv.x, xv.x, fma(xv.y, xv.y, a));
          b = fma(yv.x, yv.x, fma(yv.y, yv.y, b));
          cr = fma(xv.x, yv.x, fma(xv.y, yv.y, cr));  // Re conj(x) y
          ci = fma(xv.x, yv.y, fma(-xv.y, yv.x, ci));  // Im conj(x) y
        }
        const double sum = warp_sum4(a, b, cr, ci);
        if ((lane & 7) == 0) s_red[wid][lane >> 3] = sum;
        __syncthreads();
        if (wid == 0) {  // the rotation, once per pair: warp 0 adds the warps' sums, lane 0 rotates
          // lane l holds quantity l & 3 of warp l >> 2; a fixed butterfly over the warp bits
          double v = s_red[lane >> 2][lane & 3];
          for (int o = 4; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          const double ga = __shfl_sync(0xffffffffu, v, 0), gb = __shfl_sync(0xffffffffu, v, 1);
          const double gr = __shfl_sync(0xffffffffu, v, 2), gi = __shfl_sync(0xffffffffu, v, 3);
          if (lane == 0) {
            double cs, sn;
            double2 e;
            s_go = jacobi_rotation(ga, gb, gr, gi, tol, tiny2, cs, sn, e) ? 1 : 0;
            s_par[0] = cs;
            s_par[1] = sn;
            s_par[2] = e.x;
            s_par[3] = e.y;
          }
        }
        __syncthreads();  // s_red and s_par are rewritten only after the next pair's sums
        if (!s_go) continue;
        const double cs = s_par[0], sn = s_par[1];
        const double2 e = make_double2(s_par[2], s_par[3]);
        for (int r = tid; r < nr; r += kThreads) {
          const double2 xv = x[r], yv = cmul(e, y[r]);
          x[r] = make_double2(cs * xv.x - sn * yv.x, cs * xv.y - sn * yv.y);
          y[r] = make_double2(sn * xv.x + cs * yv.x, sn * xv.y + cs * yv.y);
        }
        double2* vx = V + (int64_t)i * nc;
        double2* vy = V + (int64_t)j * nc;
        for (int r = tid; r < nc; r += kThreads) {
          const double2 xv = vx[r], yv = cmul(e, vy[r]);
          vx[r] = make_double2(cs * xv.x - sn * yv.x, cs * xv.y - sn * yv.y);
          vy[r] = make_double2(sn * xv.x + cs * yv.x, sn * xv.y + cs * yv.y);
        }
        ++rot;
      }
      // the sweep's rotation count is published before its last barrier
      if (rd == N - 2 && tid == 0 && rot > 0) atomicAdd(sync + kBarLanes + sweep, rot);
      ++nbar;
      ok = phase_sync<kCluster>(sync, nbar * (unsigned)G, wait_ns, flag);
    }
    if (!ok) break;
    if (tid == 0) s_total = ld_acquire(sync + kBarLanes + sweep);
    __syncthreads();
    if (s_total == 0) break;
  }
  if (!ok) return;
  // sigma_j = |column j|, fixed-order sums; columns dealt round-robin to CTAs
  for (int jc = blockIdx.x; jc < nc; jc += G) {
    const double2* x = A + (int64_t)jc * nr;
    double a = 0.0;
    for (int r = tid; r < nr; r += kThreads) a = fma(x[r].x, x[r].x, fma(x[r].y, x[r].y, a));
    a = wsum(a);
    if (lane == 0) s_red[wid][0] = a;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < kWarps; ++w) t += s_red[w][0];
      sigma[jc] = sqrt(t);
    }
    __syncthreads();
  }
  if (blockIdx.x == 0 && tid == 0) {
    info[0] = sweep;
    info[1] = tr;
  }
}

struct GridInfo {
  int sms = 0, coop = 0, occ = 0;
  bool cluster16 = false;
};
GridInfo grid_info() {
  static std::once_flag once;
  static GridInfo gi;
  std::call_once(once, [] {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&gi.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      gi.sms = 1;
    if (cudaDeviceGetAttribute(&gi.coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess) gi.coop = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&gi.occ, k_jacobi_grid<false>, kThreads, 0) != cudaSuccess)
      gi.occ = 0;
    gi.cluster16 = cudaFuncSetAttribute(k_jacobi_grid<true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                   cudaSuccess;
  });
  return gi;
}

}  // namespace

double jacobi_tol(int m, int n) {
  const int nr = std::max(m, n);
  return 2.0 * std::sqrt((double)std::max(nr, 64)) * DBL_EPSILON;
}

bool launch_jacobi_svd_grid(const double2* theta, int m, int n, double2* A, double2* V, double* sigma, int* info,
                            unsigned* sync, int* flag, uint64_t wait_ns, cudaStream_t s) {
  const int nc = std::min(m, n), nr = std::max(m, n);
  const GridInfo gi = grid_info();
  const int npairs = (nc + 1) / 2;
  const bool cluster = npairs <= (gi.cluster16 ? kJacClusterMax : 8);  // one pair per CTA, one cluster
  if (nc <= kJacOneCtaMaxCols || (!cluster && (!gi.coop || gi.occ < 1))) {
    launch_jacobi_svd(theta, m, n, A, V, sigma, info, s);
    return cudaGetLastError() == cudaSuccess;
  }
  const int64_t tot = (int64_t)nr * nc + (int64_t)nc * nc;
  k_svd_load<<<(int)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, s>>>(theta, m, n, A, V);
  if (cudaMemsetAsync(sync, 0, kSvdSyncInts * sizeof(unsigned), s) != cudaSuccess) return false;
  const int tr = n > m ? 1 : 0;
  const double tol = jacobi_tol(m, n);
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (cluster) {  // one pair per CTA, the CTAs one cluster
    cfg.gridDim = dim3(npairs, 1, 1);
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = npairs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    return cudaLaunchKernelEx(&cfg, k_jacobi_grid<true>, A, V, nr, nc, sigma, info, sync, flag, tol, kJacMaxSweeps, tr,
                              wait_ns) == cudaSuccess;
  }
  const int G = std::max(1, std::min(npairs, gi.sms * std::min(gi.occ, 2)));
  cfg.gridDim = dim3(G, 1, 1);
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  return cudaLaunchKernelEx(&cfg, k_jacobi_grid<false>, A, V, nr, nc, sigma, info, sync, flag, tol, kJacMaxSweeps, tr,
                            wait_ns) == cudaSuccess;
}

namespace {

// U (m x k) and Vh (k x n), row-major, from the converged working matrix, V and
// the descending order perm of sigma; columns whose sigma is 0 are left 0.
__global__ void k_svd_write(const double2* __restrict__ A, const double2* __restrict__ V,
                            const double* __restrict__ sigma, const int* __restrict__ perm, int m, int n,
                            double2* __restrict__ U, double2* __restrict__ Vh) {
  const bool tr = n > m;
  const int nr = tr ? n : m, nc = tr ? m : n, k = nc;
  const int64_t nu = (int64_t)m * k, nvh = (int64_t)k * n;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nu + nvh;
       q += (int64_t)gridDim.x * blockDim.x) {
    const bool upart = q < nu;
    const int64_t qq = upart ? q : q - nu;
    int row, a;
    int64_t rem;
    if (upart) {
      row = (int)idivmod(qq, k, rem);
      a = (int)rem;
    } else {
      a = (int)idivmod(qq, n, rem);
      row = (int)rem;
    }
    const int j = perm[a];
    const double sj = sigma[j];
    double2 v = make_double2(0.0, 0.0);
    if (upart) {  // left vector entry `row` (length m)
      if (tr)
        v = V[(int64_t)j * nc + row];
      else if (sj > 0.0)
        v = make_double2(A[(int64_t)j * nr + row].x / sj, A[(int64_t)j * nr + row].y / sj);
      U[qq] = v;
    } else {  // conj of right vector entry `row` (length n)
      if (!tr)
        v = cconj(V[(int64_t)j * nc + row]);
      else if (sj > 0.0)
        v = make_double2(A[(int64_t)j * nr + row].x / sj, -A[(int64_t)j * nr + row].y / sj);
      Vh[qq] = v;
    }
  }
}

struct SvdWs {
  int64_t A, V, sigma, perm, info, sync, flag, total;
};
SvdWs svd_ws(int m, int n) {
  const int64_t nr = std::max(m, n), nc = std::min(m, n);
  SvdWs L;
  int64_t o = 0;
  auto take = [&](int64_t bytes) {
    const int64_t r = o;
    o += (bytes + 255) / 256 * 256;
    return r;
  };
  L.A = take(nr * nc * 16);
  L.V = take(nc * nc * 16);
  L.sigma = take(nc * 8);
  L.perm = take(nc * 4);
  L.info = take(4 * 4);
  L.sync = take(kSvdSyncInts * 4);
  L.flag = take(4);
  L.total = o;
  return L;
}

}  // namespace

}  // namespace ttn

extern "C" ttn_status ttn_svd_workspace_size(int32_t m, int32_t n, size_t* bytes) {
  if (!bytes || m < 1 || n < 1) return TTN_EINVAL;
  *bytes = (size_t)ttn::svd_ws(m, n).total;
  return TTN_OK;
}

extern "C" ttn_status ttn_svd(const void* a_dev, int32_t m, int32_t n, void* u_dev, double* sigma_host, void* vh_dev,
                              void* ws_dev, size_t ws_bytes, double wait_s, int32_t* sweeps_out, void* stream) {
  using namespace ttn;
  if (!a_dev || !u_dev || !sigma_host || !vh_dev || !ws_dev || m < 1 || n < 1 || !(wait_s >= 0.0)) return TTN_EINVAL;
  const SvdWs L = svd_ws(m, n);
  if (ws_bytes < (size_t)L.total || ((uintptr_t)ws_dev & 255)) return TTN_ENOMEM;
  cudaStream_t s = (cudaStream_t)stream;
  char* base = (char*)ws_dev;
  double2* A = (double2*)(base + L.A);
  double2* V = (double2*)(base + L.V);
  double* sigma = (double*)(base + L.sigma);
  int* perm = (int*)(base + L.perm);
  int* info = (int*)(base + L.info);
  unsigned* sync = (unsigned*)(base + L.sync);
  int* flag = (int*)(base + L.flag);
  const int nc = std::min(m, n);
  if (cudaMemsetAsync(flag, 0, sizeof(int), s) != cudaSuccess) return TTN_ECUDA;
  const double wns = std::min(wait_s, 60.0) * 1e9;
  if (!launch_jacobi_svd_grid((const double2*)a_dev, m, n, A, V, sigma, info, sync, flag, (uint64_t)wns, s))
    return TTN_ECUDA;
  std::vector<double> sig(nc);
  int hinfo[2] = {0, 0}, hflag = 0;
  if (cudaMemcpyAsync(sig.data(), sigma, nc * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(hinfo, info, sizeof(hinfo), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return TTN_ECUDA;
  if (hflag & 16) return TTN_ETIMEOUT;
  if (sweeps_out) *sweeps_out = hinfo[0];
  if (hinfo[0] >= kJacMaxSweeps) return TTN_ENUMERIC;
  std::vector<int> pm(nc);
  for (int i = 0; i < nc; ++i) pm[i] = i;
  std::stable_sort(pm.begin(), pm.end(), [&](int a, int b) { return sig[a] > sig[b]; });
  for (int i = 0; i < nc; ++i) sigma_host[i] = sig[pm[i]];
  if (cudaMemcpyAsync(perm, pm.data(), nc * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess) return TTN_ECUDA;
  const int64_t tot = (int64_t)(m + n) * nc;
  k_svd_write<<<(int)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, s>>>(A, V, sigma, perm, m, n,
                                                                             (double2*)u_dev, (double2*)vh_dev);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return TTN_ECUDA;
  return TTN_OK;
}
