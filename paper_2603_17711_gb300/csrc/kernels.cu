// Device kernels of the TTN-HEOM library, FP64 path (sm_103a).
//
// On GB300 the FP64 pipe issues about 2 FMA per SM per clock, so every kernel
// here is bound by FP64 issue, not by memory: the data (node tensors of at most
// a few hundred KB, environments of r x r) stays in L2 and L1.
#include <algorithm>
#include <cooperative_groups.h>
#include <mutex>

#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace ttn {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {  // a*b + c
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ double2 cfma_conj(double2 a, double2 b, double2 c) {  // conj(a)*b + c
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(-a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }

// ---------------------------------------------------------------------------
// Complex arithmetic in the contraction type (double2 or float2).
// ---------------------------------------------------------------------------
template <typename R> struct Cx;
template <> struct Cx<double> {
  using T = double2;
  __device__ static T zero() { return make_double2(0.0, 0.0); }
  __device__ static T fma(T a, T b, T c) { return cfma(a, b, c); }
  __device__ static T fmaj(T a, T b, T c) { return cfma_conj(a, b, c); }
  __device__ static T add(T a, T b) { return cadd(a, b); }
  __device__ static double2 wide(T a) { return a; }
  __device__ static T narrow(double2 a) { return a; }
};
template <> struct Cx<float> {
  using T = float2;
  __device__ static T zero() { return make_float2(0.f, 0.f); }
  __device__ static T fma(T a, T b, T c) {
    c.x = fmaf(a.x, b.x, c.x);
    c.x = fmaf(-a.y, b.y, c.x);
    c.y = fmaf(a.x, b.y, c.y);
    c.y = fmaf(a.y, b.x, c.y);
    return c;
  }
  __device__ static T fmaj(T a, T b, T c) {
    c.x = fmaf(a.x, b.x, c.x);
    c.x = fmaf(a.y, b.y, c.x);
    c.y = fmaf(a.x, b.y, c.y);
    c.y = fmaf(-a.y, b.x, c.y);
    return c;
  }
  __device__ static T add(T a, T b) { return make_float2(a.x + b.x, a.y + b.y); }
  __device__ static double2 wide(T a) { return make_double2(a.x, a.y); }
  __device__ static T narrow(double2 a) { return make_float2((float)a.x, (float)a.y); }
};

// ---------------------------------------------------------------------------
// Sum of mode products: out_o[idx] = sum_t M_t x_{leg_t} src_t.
// An output tile is 32 consecutive elements (one per lane). Its work is cut
// into units -- an identity term, or kApChunk consecutive positions x of one
// mode product -- dealt round-robin to the NW*k warps of the k CTAs (one
// thread-block cluster) that share the tile. Each warp sums its units in
// order, the CTA sums its warps in order, and CTA 0 of the cluster sums the
// CTAs in order (through distributed shared memory), so results are bitwise
// reproducible for a given tile shape (NW, k). GB300 issues one FP64
// instruction per warp every ~64 cycles, so short dependency chains (4
// positions per unit, loads issued before the FMAs) and many warps per tile
// make a small contraction fast; when many lists run at once (batched
// instances) fewer warps per tile waste less on idle warps and reductions.
// NW (warps per CTA: 2, 4 or 8) and k are chosen per list (ApList::w, k).
// ---------------------------------------------------------------------------

// Leg geometry of one output element (kept in registers: selected by switch,
// never indexed dynamically).
struct Geo {
  int d0, d1, d2, d3;
  int i0, i1, i2, i3;
  int64_t s0, s1, s2;  // s3 = 1
};

template <typename R>
__device__ __forceinline__ int term_dim(const ApTerm& term, const Geo& g) {
  switch (term.leg) {
    case 0: return g.d0;
    case 1: return g.d1;
    case 2: return g.d2;
    default: return g.d3;
  }
}

// contribution of positions [x0, x0 + kApChunk) of one term (the whole term if identity)
template <typename R>
__device__ __forceinline__ typename Cx<R>::T unit_dot(const ApTerm& term, const DevTables& T, int64_t idx,
                                                      const Geo& g, int x0) {
  using C = Cx<R>;
  using V = typename C::T;
  const V* __restrict__ src = (const V*)T.bufs[term.src];
  if (term.mat < 0) return src[idx];
  const V* __restrict__ M = (const V*)T.mats[term.mat];
  int dl, il;
  int64_t stride;
  switch (term.leg) {
    case 0: dl = g.d0; il = g.i0; stride = g.s0; break;
    case 1: dl = g.d1; il = g.i1; stride = g.s1; break;
    case 2: dl = g.d2; il = g.i2; stride = g.s2; break;
    default: dl = g.d3; il = g.i3; stride = 1; break;
  }
  const V* __restrict__ row = M + (int64_t)il * dl;
  const V* __restrict__ col = src + (idx - (int64_t)il * stride);
  V mv[kApChunk], sv[kApChunk];
#pragma unroll
  for (int k = 0; k < kApChunk; ++k) {
    const int x = x0 + k;
    if (x < dl) {
      mv[k] = row[x];
      sv[k] = col[(int64_t)x * stride];
    }
  }
  V acc = C::zero();
#pragma unroll
  for (int k = 0; k < kApChunk; ++k)
    if (x0 + k < dl) acc = C::fma(mv[k], sv[k], acc);
  return acc;
}

// Sum of one output tile over the units of CTA `rank` of the k sharing it;
// the CTA's total (fixed order over warps) is returned in warp 0.
template <typename R, int NW>
__device__ __forceinline__ typename Cx<R>::T tile_sum(const DevTables& T, const ApList& L, int tile, int rank, int K,
                                                      typename Cx<R>::T (*part)[32], ApOut& out, int64_t& idx,
                                                      int64_t& P) {
  using C = Cx<R>;
  using V = typename C::T;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  out = T.outs[list_output(T.outs, L.out_begin, L.out_end, L.tpo, tile)];
  Geo g;
  g.d0 = out.d0; g.d1 = out.d1; g.d2 = out.d2; g.d3 = out.d3;
  g.s2 = g.d3;
  g.s1 = (int64_t)g.d2 * g.d3;
  g.s0 = g.s1 * g.d1;
  P = g.s0 * g.d0;
  idx = (int64_t)(tile - out.tile0) * kApTile + lane;
  V acc = C::zero();
  if (idx < P) {
    if (P <= 0x7fffffff) {  // every tensor of these trees: 32-bit index arithmetic
      const unsigned x = (unsigned)idx, s1 = (unsigned)g.s1, s2 = (unsigned)g.s2;
      const unsigned q2 = x / s2, q1 = x / s1;
      g.i0 = (int)(x / (unsigned)g.s0);
      g.i1 = (int)(q1 % (unsigned)g.d1);
      g.i2 = (int)(q2 % (unsigned)g.d2);
      g.i3 = (int)(x - q2 * s2);
    } else {
      g.i0 = (int)(idx / g.s0);
      g.i1 = (int)((idx / g.s1) % g.d1);
      g.i2 = (int)((idx / g.s2) % g.d2);
      g.i3 = (int)(idx % g.d3);
    }
    const int W = K * NW, me = rank * NW + wid;
    int u = 0;  // index of the term's first unit in the tile's unit list
    for (int t = out.term_begin; t < out.term_end; ++t) {
      const ApTerm term = T.terms[t];
      const int nch = term.mat < 0 ? 1 : (term_dim<R>(term, g) + kApChunk - 1) / kApChunk;
      for (int c = ((me - u) % W + W) % W; c < nch; c += W)
        acc = C::add(acc, unit_dot<R>(term, T, idx, g, c * kApChunk));
      u += nch;
    }
  }
  part[wid][lane] = acc;
  __syncthreads();
  if (wid == 0) {
    acc = part[0][lane];
    for (int w = 1; w < NW; ++w) acc = C::add(acc, part[w][lane]);
  }
  __syncthreads();  // part may be reused by the caller's next tile
  return acc;
}

// Epilogue of one output element (warp 0 of the CTA owning the tile).
template <typename R>
__device__ __forceinline__ void tile_store(const DevTables& T, const ApOut& out, const Epi& ep, int64_t idx,
                                           typename Cx<R>::T acc) {
  using C = Cx<R>;
  using V = typename C::T;
  if (ep.mode == EPI_STORE) {
    ((V*)T.bufs[out.dst])[idx] = acc;
    return;
  }
  const double2 k = C::wide(acc);
  double2* __restrict__ y = ep.y;
  double2* __restrict__ ac = ep.acc;
  V* __restrict__ ys = (V*)ep.ys;
  const double h = ep.h;
  switch (ep.mode) {
    case EPI_RK1:
      ac[idx] = k;
      ys[idx] = C::narrow(cadd(y[idx], cscale(0.5 * h, k)));
      break;
    case EPI_RK2:
      ac[idx] = cadd(ac[idx], cscale(2.0, k));
      ys[idx] = C::narrow(cadd(y[idx], cscale(0.5 * h, k)));
      break;
    case EPI_RK3:
      ac[idx] = cadd(ac[idx], cscale(2.0, k));
      ys[idx] = C::narrow(cadd(y[idx], cscale(h, k)));
      break;
    default: {
      const double2 yn = cadd(y[idx], cscale(h / 6.0, cadd(ac[idx], k)));
      y[idx] = yn;
      if ((void*)ep.y_lo != (void*)ep.y) ((V*)ep.y_lo)[idx] = C::narrow(yn);
      break;
    }
  }
}

template <typename R, int NW>
__global__ void __launch_bounds__(32 * NW, 32 / NW) k_apply(DevTables T, ApList L, Epi ep) {
  using C = Cx<R>;
  using V = typename C::T;
  __shared__ V part[NW][32];
  __shared__ V slot[kMaxSplit][32];
  const int K = L.k;
  const int tile = blockIdx.x / K, rank = blockIdx.x % K;  // rank == block rank in the cluster
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  ApOut out;
  int64_t idx, P;
  V acc = tile_sum<R, NW>(T, L, tile, rank, K, part, out, idx, P);
  if (K > 1) {
    cg::cluster_group cluster = cg::this_cluster();
    if (wid == 0 && rank > 0) cluster.map_shared_rank(&slot[0][0], 0)[rank * 32 + lane] = acc;
    cluster.sync();
    if (rank > 0) return;
    if (wid == 0)
      for (int r = 1; r < K; ++r) acc = C::add(acc, slot[r][lane]);
  }
  if (wid != 0 || idx >= P) return;
  tile_store<R>(T, out, ep, idx, acc);
}

// Launch n_tiles * k CTAs; k > 1 makes every k consecutive CTAs one cluster.
template <typename Kern, typename... Args>
static void launch_split(Kern kern, int n_tiles, int k, int warps, cudaStream_t s, Args... args) {
  if (k <= 1) {
    kern<<<n_tiles, 32 * warps, 0, s>>>(args...);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n_tiles * k), 1, 1);
  cfg.blockDim = dim3(32 * warps, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)k;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, args...);
}

template <typename R>
static void launch_apply_w(const DevTables& T, const ApList& L, const Epi& e, cudaStream_t s) {
  switch (L.w) {
    case 2: launch_split(k_apply<R, 2>, L.n_tiles, L.k, 2, s, T, L, e); break;
    case 4: launch_split(k_apply<R, 4>, L.n_tiles, L.k, 4, s, T, L, e); break;
    default: launch_split(k_apply<R, 8>, L.n_tiles, L.k, 8, s, T, L, e); break;
  }
}

void launch_apply(int prec, const DevTables& T, const ApList& L, const Epi& e, cudaStream_t s) {
  if (L.n_tiles <= 0) return;
  if (prec == PREC_F32)
    launch_apply_w<float>(T, L, e, s);
  else
    launch_apply_w<double>(T, L, e, s);
}

// ---------------------------------------------------------------------------
// Environment projection E[x', x] = sum_r conj(U[.. x' ..]) W[.. x ..] over all
// legs except `leg`. A tile is 32 output entries (one per lane); the reduction
// range r is dealt round-robin to the 8*k warps of the k CTAs (one cluster)
// sharing the tile, four positions per batch with loads issued first, and the
// partial sums are added in a fixed order (warps, then CTAs via distributed
// shared memory).
// ---------------------------------------------------------------------------
constexpr int kPjWarps = kSplitWarps;

template <typename R>
__global__ void __launch_bounds__(32 * kPjWarps, 4) k_project(DevTables T, PjList L) {
  using C = Cx<R>;
  using V = typename C::T;
  __shared__ V part[kPjWarps][32];
  __shared__ V slot[kMaxSplit][32];
  const int K = L.k;
  const int tile = blockIdx.x / K, rank = blockIdx.x % K;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const PjOut pj = T.pjs[list_output(T.pjs, L.out_begin, L.out_end, L.tpo, tile)];
  const int dd[3] = {pj.d0, pj.d1, pj.d2};
  const int64_t st[3] = {(int64_t)pj.d1 * pj.d2, pj.d2, 1};
  const int l = pj.leg;
  const int d = dd[l];
  const int e = (tile - pj.tile0) * kPjTile + lane;
  const int la = l == 0 ? 1 : 0, lb = l == 2 ? 1 : 2;  // the two other legs
  const int nrest = dd[la] * dd[lb];
  V acc = C::zero();
  if (e < d * d) {
    const int xp = e / d, x = e % d;
    const V* __restrict__ U = (const V*)T.bufs[pj.u_buf] + (int64_t)xp * st[l];
    const V* __restrict__ Wt = (const V*)T.bufs[pj.w_buf] + (int64_t)x * st[l];
    const int W = K * kPjWarps, me = rank * kPjWarps + wid;
    for (int r0 = me; r0 < nrest; r0 += 4 * W) {
      V uv[4], wv[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int r = r0 + k * W;
        if (r < nrest) {
          const int64_t off = (int64_t)(r / dd[lb]) * st[la] + (int64_t)(r % dd[lb]) * st[lb];
          uv[k] = U[off];
          wv[k] = Wt[off];
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (r0 + k * W < nrest) acc = C::fmaj(uv[k], wv[k], acc);
    }
  }
  part[wid][lane] = acc;
  __syncthreads();
  if (wid == 0) {
    acc = part[0][lane];
    for (int w = 1; w < kPjWarps; ++w) acc = C::add(acc, part[w][lane]);
  }
  if (K > 1) {
    cg::cluster_group cluster = cg::this_cluster();
    if (wid == 0 && rank > 0) cluster.map_shared_rank(&slot[0][0], 0)[rank * 32 + lane] = acc;
    cluster.sync();
    if (rank > 0) return;
    if (wid == 0)
      for (int r = 1; r < K; ++r) acc = C::add(acc, slot[r][lane]);
  }
  if (wid != 0 || e >= d * d) return;
  ((V*)T.mats[pj.dst_mat])[e] = acc;
}

// Projection of wide bonds (d >= 32, reduction range >= 1024): 32 x 32 output
// tiles, reduction range in chunks of 32 staged through shared memory with
// coalesced loads (along the reduction index, or along the leg when the leg
// is the contiguous one), 2 x 2 outputs per thread. The range is split over
// KS CTAs of one cluster, whose partial tiles CTA 0 adds in rank order
// through distributed shared memory, so results are reproducible.
constexpr int kPtT = 32;  // output tile edge
constexpr int kPtR = 32;  // reduction chunk

template <typename R>
__global__ void __launch_bounds__(256) k_project_tiled(DevTables T, PjList L, int ntx, int KS) {
  using C = Cx<R>;
  using V = typename C::T;
  extern __shared__ __align__(16) unsigned char psm[];
  V(*Us)[kPtR + 1] = (V(*)[kPtR + 1])psm;
  V(*Ws)[kPtR + 1] = Us + kPtT;
  V* slot = (V*)(Ws + kPtT);  // CTA 0: [KS-1][kPtT * kPtT] partial tiles of the other ranks
  __shared__ int64_t base[kPtR];
  const int tid = threadIdx.x;
  const int rank = blockIdx.x % KS, item = blockIdx.x / KS;
  const int per_out = ntx * ntx;
  const int o = L.out_begin + item / per_out, tt = item % per_out;
  const PjOut pj = T.pjs[o];
  const int dd[3] = {pj.d0, pj.d1, pj.d2};
  const int64_t st[3] = {(int64_t)pj.d1 * pj.d2, pj.d2, 1};
  const int l = pj.leg, d = dd[l];
  const int la = l == 0 ? 1 : 0, lb = l == 2 ? 1 : 2;
  const int nrest = dd[la] * dd[lb];
  const int X0 = (tt / ntx) * kPtT, Y0 = (tt % ntx) * kPtT;  // rows x' (conjugated side), columns x
  const V* __restrict__ U = (const V*)T.bufs[pj.u_buf];
  const V* __restrict__ W = (const V*)T.bufs[pj.w_buf];
  const int nch = (nrest + kPtR - 1) / kPtR;
  const int c0 = (int)((int64_t)rank * nch / KS), c1 = (int)((int64_t)(rank + 1) * nch / KS);
  const bool leg_fast = l == 2;  // the leg index is the contiguous one
  const int ty = (tid >> 4) * 2, tx = (tid & 15) * 2;
  V acc[2][2] = {{C::zero(), C::zero()}, {C::zero(), C::zero()}};
  for (int c = c0; c < c1; ++c) {
    const int r0 = c * kPtR;
    if (tid < kPtR) {
      const int r = r0 + tid;
      base[tid] = r < nrest ? (int64_t)(r / dd[lb]) * st[la] + (int64_t)(r % dd[lb]) * st[lb] : 0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < (kPtT * kPtR) / 256; ++q) {
      const int e = tid + q * 256;
      const int row = leg_fast ? (e & 31) : (e >> 5), rr = leg_fast ? (e >> 5) : (e & 31);
      const bool rin = r0 + rr < nrest;
      const int xu = X0 + row, xw = Y0 + row;
      Us[row][rr] = (xu < d && rin) ? U[(int64_t)xu * st[l] + base[rr]] : C::zero();
      Ws[row][rr] = (xw < d && rin) ? W[(int64_t)xw * st[l] + base[rr]] : C::zero();
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < kPtR; ++rr) {
      const V u0 = Us[ty][rr], u1 = Us[ty + 1][rr], w0 = Ws[tx][rr], w1 = Ws[tx + 1][rr];
      acc[0][0] = C::fmaj(u0, w0, acc[0][0]);
      acc[0][1] = C::fmaj(u0, w1, acc[0][1]);
      acc[1][0] = C::fmaj(u1, w0, acc[1][0]);
      acc[1][1] = C::fmaj(u1, w1, acc[1][1]);
    }
    __syncthreads();
  }
  if (KS > 1) {
    cg::cluster_group cluster = cg::this_cluster();
    if (rank > 0) {
      V* dst = cluster.map_shared_rank(slot, 0) + (size_t)(rank - 1) * kPtT * kPtT;
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) dst[(ty + i) * kPtT + tx + j] = acc[i][j];
    }
    cluster.sync();
    if (rank > 0) return;
    for (int r = 1; r < KS; ++r)
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) acc[i][j] = C::add(acc[i][j], slot[(size_t)(r - 1) * kPtT * kPtT + (ty + i) * kPtT + tx + j]);
  }
  V* E = (V*)T.mats[pj.dst_mat];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      const int xp = X0 + ty + i, x = Y0 + tx + j;
      if (xp < d && x < d) E[xp * d + x] = acc[i][j];
    }
}

bool launch_project_tiled(int prec, const DevTables& T, const PjList& L, int d, int64_t nrest, int sm_count,
                          cudaStream_t s) {
  const int n_outs = L.out_end - L.out_begin;
  // FP64 projections are bound by FP64 issue either way and measured faster
  // on the per-entry kernel (rank-64 env update 100 vs 117 ms/step)
  if (prec != PREC_F32 || n_outs <= 0 || d < 32 || nrest < 1024) return false;
  const int ntx = (d + kPtT - 1) / kPtT;
  const int items = n_outs * ntx * ntx;
  const int nch = (int)((nrest + kPtR - 1) / kPtR);
  const int kmax = prec == PREC_F32 ? 8 : 4;
  int KS = 1;
  while (KS < kmax && KS < nch && items * KS < 2 * sm_count) ++KS;
  const size_t vb = prec == PREC_F32 ? sizeof(float2) : sizeof(double2);
  const size_t smem = vb * (2 * kPtT * (kPtR + 1) + (size_t)(KS - 1) * kPtT * kPtT);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_project_tiled<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    cudaFuncSetAttribute(k_project_tiled<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    attr = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(items * KS), 1, 1);
  cfg.blockDim = dim3(256, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr1[1];
  attr1[0].id = cudaLaunchAttributeClusterDimension;
  attr1[0].val.clusterDim.x = (unsigned)KS;
  attr1[0].val.clusterDim.y = 1;
  attr1[0].val.clusterDim.z = 1;
  cfg.attrs = attr1;
  cfg.numAttrs = 1;
  if (prec == PREC_F32) return cudaLaunchKernelEx(&cfg, k_project_tiled<float>, T, L, ntx, KS) == cudaSuccess;
  return cudaLaunchKernelEx(&cfg, k_project_tiled<double>, T, L, ntx, KS) == cudaSuccess;
}

void launch_project(int prec, const DevTables& T, const PjList& L, cudaStream_t s) {
  if (L.n_tiles <= 0) return;
  if (prec == PREC_F32)
    launch_split(k_project<float>, L.n_tiles, L.k, kPjWarps, s, T, L);
  else
    launch_split(k_project<double>, L.n_tiles, L.k, kPjWarps, s, T, L);
}

// Clusters of more than 8 CTAs are non-portable: allowed once per process for
// every contraction and projection kernel, before any launch (and outside any
// graph capture).
void allow_wide_splits() {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_apply<double, 8>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(k_apply<double, 4>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(k_apply<double, 2>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(k_apply<float, 8>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(k_apply<float, 4>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(k_apply<float, 2>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(k_project<double>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(k_project<float>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaGetLastError();
  });
}


// ---------------------------------------------------------------------------
// Householder QR (one CTA). A (m x n, m = P / d_leg, n = d_leg) is gathered
// column-major into `work`; rows enumerate the two other legs in order.
// Convention (identical to the CPU oracle): for column j with remainder x of
// norm alpha, alpha <= tol*||A||_F means no reflector (R_jj = 0, Q column
// H_0..H_{j-1} e_j); otherwise v = x + phi*alpha*e_0 with phi = x_0/|x_0|
// (1 if x_0 = 0), H = I - beta v v^H, beta = 2 / (v^H v) = 1/(alpha(alpha+|x_0|)).
// Afterwards rows of R and columns of Q are rescaled so that diag(R) >= 0.
// ---------------------------------------------------------------------------
constexpr int kQrThreads = 512;
constexpr int kQrMaxN = 256;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double2 warp_sum2(double2 v) {
  v.x = warp_sum(v.x);
  v.y = warp_sum(v.y);
  return v;
}
// Block-wide sum with a fixed reduction order (deterministic).
__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < nw; ++w) s += red[w];
  return s;
}

__global__ void __launch_bounds__(kQrThreads) k_qr(double2* U, int d0, int d1, int d2, int leg,
                                                   double tol, double2* A, double2* Q, double2* R, int* flag,
                                                   float2* U_lo, float2* R_lo) {
  __shared__ double red[kQrThreads / 32];
  __shared__ double s_beta[kQrMaxN];
  __shared__ int s_skip[kQrMaxN];
  __shared__ double2 s_rdiag[kQrMaxN];
  __shared__ double2 s_phase[kQrMaxN];
  const int dd[3] = {d0, d1, d2};
  const int64_t st[3] = {(int64_t)d1 * d2, d2, 1};
  const int n = dd[leg];
  const int la = leg == 0 ? 1 : 0, lb = leg == 2 ? 1 : 2;
  const int64_t m = (int64_t)dd[la] * dd[lb];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  // gather A[r, c] (column-major), r = (a, b) over the two other legs
  double fro = 0.0;
  for (int64_t k = tid; k < m * n; k += nt) {
    const int64_t c = k / m, r = k % m;
    const int64_t a = r / dd[lb], b = r % dd[lb];
    const double2 v = U[c * st[leg] + a * st[la] + b * st[lb]];
    A[k] = v;
    fro += v.x * v.x + v.y * v.y;
  }
  fro = sqrt(block_sum(fro, red));
  if (!isfinite(fro)) {  // non-finite or overflowing input: report, leave U untouched
    if (tid == 0) atomicOr(flag, 1);
    return;
  }
  const double thr = tol * fro;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    double2* x = A + (int64_t)j * m;
    double ss = 0.0;
    for (int64_t r = j + tid; r < m; r += nt) ss += x[r].x * x[r].x + x[r].y * x[r].y;
    const double alpha = sqrt(block_sum(ss, red));
    if (alpha <= thr) {
      for (int64_t r = j + tid; r < m; r += nt) x[r] = make_double2(0.0, 0.0);
      if (tid == 0) {
        s_skip[j] = 1;
        s_beta[j] = 0.0;
        s_rdiag[j] = make_double2(0.0, 0.0);
        s_phase[j] = make_double2(1.0, 0.0);
      }
      __syncthreads();
      continue;
    }
    const double2 x0 = x[j];
    const double ax0 = hypot(x0.x, x0.y);
    const double2 phi = ax0 > 0.0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
    const double beta = 1.0 / (alpha * (alpha + ax0));
    __syncthreads();
    if (tid == 0) {
      x[j] = make_double2(x0.x + phi.x * alpha, x0.y + phi.y * alpha);  // v_0
      s_skip[j] = 0;
      s_beta[j] = beta;
      s_rdiag[j] = make_double2(-phi.x * alpha, -phi.y * alpha);
      s_phase[j] = make_double2(-phi.x, -phi.y);  // R_jj / |R_jj|
    }
    __syncthreads();
    // apply H_j to the remaining columns: one warp per column
    for (int k = j + 1 + wid; k < n; k += nw) {
      double2* a = A + (int64_t)k * m;
      double2 w = make_double2(0.0, 0.0);
      for (int64_t r = j + lane; r < m; r += 32) w = cfma_conj(x[r], a[r], w);
      w = warp_sum2(w);
      const double2 bw = cscale(beta, w);
      for (int64_t r = j + lane; r < m; r += 32) {
        const double2 t = cmul(x[r], bw);
        a[r] = make_double2(a[r].x - t.x, a[r].y - t.y);
      }
    }
    __syncthreads();
  }
  // R (row-major n x n) with diag(R) real >= 0: row j scaled by conj(phase_j)
  for (int k = tid; k < n * n; k += nt) {
    const int i = k / n, c = k % n;
    double2 v = make_double2(0.0, 0.0);
    if (c == i) {
      v = s_skip[i] ? make_double2(0.0, 0.0) : make_double2(hypot(s_rdiag[i].x, s_rdiag[i].y), 0.0);
    } else if (c > i) {
      const double2 a = A[(int64_t)c * m + i];
      const double2 p = s_phase[i];
      v = make_double2(a.x * p.x + a.y * p.y, a.y * p.x - a.x * p.y);  // conj(p) * a
    }
    R[k] = v;
    if (R_lo) R_lo[k] = make_float2((float)v.x, (float)v.y);
  }
  // Q = H_0 ... H_{n-1} [I; 0], column-major in Q
  for (int64_t k = tid; k < m * n; k += nt) {
    const int64_t c = k / m, r = k % m;
    Q[k] = make_double2(r == c ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int j = n - 1; j >= 0; --j) {
    if (s_skip[j]) continue;
    const double2* v = A + (int64_t)j * m;
    const double beta = s_beta[j];
    for (int k = j + wid; k < n; k += nw) {
      double2* q = Q + (int64_t)k * m;
      double2 w = make_double2(0.0, 0.0);
      for (int64_t r = j + lane; r < m; r += 32) w = cfma_conj(v[r], q[r], w);
      w = warp_sum2(w);
      const double2 bw = cscale(beta, w);
      for (int64_t r = j + lane; r < m; r += 32) {
        const double2 t = cmul(v[r], bw);
        q[r] = make_double2(q[r].x - t.x, q[r].y - t.y);
      }
    }
    __syncthreads();
  }
  // scatter Q (columns scaled by phase) back into the node layout
  for (int64_t k = tid; k < m * n; k += nt) {
    const int64_t c = k / m, r = k % m;
    const int64_t a = r / dd[lb], b = r % dd[lb];
    const double2 q = cmul(Q[k], s_phase[c]);
    const int64_t at = c * st[leg] + a * st[la] + b * st[lb];
    U[at] = q;
    if (U_lo) U_lo[at] = make_float2((float)q.x, (float)q.y);
  }
}

void launch_qr(double2* U, int d0, int d1, int d2, int leg, double tol, double2* work, int64_t work_elems,
               double2* qbuf, double2* R, int* flag, float2* U_lo, float2* R_lo, cudaStream_t s,
               uint64_t grid_wait_ns) {
  if (launch_qr_cluster(U, d0, d1, d2, leg, tol, R, flag, U_lo, R_lo, work, work_elems, s)) return;
  if (launch_qr_blocked(U, d0, d1, d2, leg, tol, work, work_elems, qbuf, R, flag, U_lo, R_lo, s, grid_wait_ns))
    return;
  k_qr<<<1, kQrThreads, 0, s>>>(U, d0, d1, d2, leg, tol, work, qbuf, R, flag, U_lo, R_lo);
}

__global__ void k_copy(double2* dst, float2* dst_lo, const double2* src, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = src[i];
    dst[i] = v;
    if (dst_lo) dst_lo[i] = make_float2((float)v.x, (float)v.y);
  }
}
void launch_copy(double2* dst, float2* dst_lo, const double2* src, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 1024);
  k_copy<<<blocks, 256, 0, s>>>(dst, dst_lo, src, n);
}

// ---------------------------------------------------------------------------
// Reduced density matrix (rho_S = <0|Omega>): contraction of one node with
// the vectors of its two child legs (the n = 0 unit vector on open legs).
// ---------------------------------------------------------------------------
// One CTA per output; warp w takes the rows b = w, w + 8, ... of the output's
// slice (for the root: one row, the output itself), the lanes split the row
// over c and a fixed butterfly adds them, and the warps' sums are added in warp
// order, so the result is reproducible.
__global__ void __launch_bounds__(256) k_rdm_node(const double2* U, int d0, int d1, int d2, int root,
                                                  const double2* w1, const double2* w2, double2* out) {
  // root: out[i*d1 + j] = sum_c U[i, j, c] w2[c]; else out[a] = sum_{b,c} U[a,b,c] w1[b] w2[c]
  __shared__ double2 part[8];
  const int e = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nrow = root ? 1 : (w1 ? d1 : 1);
  const double2* blk = U + (int64_t)e * (root ? d2 : (int64_t)d1 * d2);
  double2 acc = make_double2(0.0, 0.0);
  for (int b = warp; b < nrow; b += 8) {
    const double2* row = blk + (int64_t)b * d2;
    double2 inner = make_double2(0.0, 0.0);
    if (w2) {
      for (int c = lane; c < d2; c += 32) inner = cfma(row[c], w2[c], inner);
      for (int o = 16; o > 0; o >>= 1) {
        inner.x += __shfl_xor_sync(0xffffffffu, inner.x, o);
        inner.y += __shfl_xor_sync(0xffffffffu, inner.y, o);
      }
    } else {
      inner = row[0];
    }
    acc = (!root && w1) ? cfma(w1[b], inner, acc) : inner;
  }
  if (lane == 0) part[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 t = part[0];
    for (int w = 1; w < 8 && w < nrow; ++w) {
      t.x += part[w].x;
      t.y += part[w].y;
    }
    out[e] = t;
  }
}
void launch_rdm_node(const double2* U, int d0, int d1, int d2, bool root, const double2* w1,
                     const double2* w2, double2* out, cudaStream_t s) {
  const int nout = root ? d0 * d1 : d0;
  if (nout > 0) k_rdm_node<<<nout, 256, 0, s>>>(U, d0, d1, d2, root ? 1 : 0, w1, w2, out);
}

__global__ void k_drive(double2* const* mats, float2* const* mats32, const DriveMat* list, int n, DriveArgs g) {
  const DriveMat dm = list[blockIdx.x];
  const int dd = dm.d * dm.d;
  double2* cur = mats[dm.cur];
  float2* cur32 = mats32 ? mats32[dm.cur] : nullptr;
  const double2* st = mats[dm.stat];
  for (int e = threadIdx.x; e < dd; e += blockDim.x) {
    double2 v = st[e];
    for (int d = 0; d < kMaxDrives; ++d)
      if (dm.part[d] >= 0) {
        const double2 p = mats[dm.part[d]][e];
        v.x += g.g[d] * p.x;
        v.y += g.g[d] * p.y;
      }
    cur[e] = v;
    if (cur32) cur32[e] = make_float2((float)v.x, (float)v.y);
  }
}
void launch_drive(double2* const* mats_dev, float2* const* mats32, const DriveMat* list, int n,
                  const DriveArgs& g, cudaStream_t s) {
  if (n <= 0) return;
  k_drive<<<n, 128, 0, s>>>(mats_dev, mats32, list, n, g);
}

__global__ void k_check_finite(const double2* x, int64_t n, int* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = x[i];
    if (!isfinite(v.x) || !isfinite(v.y)) atomicOr(flag, 1);
  }
}
void launch_check_finite(const double2* x, int64_t n, int* flag, cudaStream_t s) {
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 64);
  k_check_finite<<<blocks, 256, 0, s>>>(x, n, flag);
}

}  // namespace ttn
