// Mode products of the mixed-precision form on the 5th-generation tensor cores
// (tcgen05, kind::tf32, accumulator in tensor memory).
//
// One term Y += M x_l X (M complex d x d, d = d_l <= 64) is a real GEMM through
// the 2x2 embedding of every complex entry,
//     (Re Y, Im Y) = [[Re M, -Im M], [Im M, Re M]] . (Re X, Im X),
// with real and imaginary parts interleaved along both the MMA's M dimension
// (2d <= 128 rows, zero-padded) and K (2d, in chunks of 32); n, the positions
// of the two other legs, is the N dimension (tiles of 64). All terms of an output on the same leg accumulate into one
// tensor-memory tile; the legs are separate launches (0, 1, 2) so that the
// first writes the output and the later ones add to it, in that fixed order.
// Precision: every FP32 operand is split into tf32 hi + lo, and the three
// products hi*hi + hi*lo + lo*hi are accumulated in FP32 ("3xTF32"), which
// keeps the error at the level of FP32 CUDA-core arithmetic.
//
// The operator operand comes pre-split from a pool that every writer of an
// operator matrix refreshes (launch_tc_embed) and is copied into shared memory
// with one bulk asynchronous copy per chunk; the tensor operand is staged by
// the threads (the 2x2 embedding and the hi/lo split happen on the way) into
// shared memory in the K-major, unswizzled canonical
// layout: 8-row x 16-byte core matrices, K-adjacent core matrices 128 B apart
// (leading byte offset), 8-row groups 1024 B apart (stride byte offset). Two
// stages alternate so that staging chunk c+1 overlaps the MMAs of chunk c;
// one thread issues the MMAs and commits them to the stage's mbarrier.
#include <algorithm>
#include <cstdint>

#include "kernels.cuh"

namespace ttn {

namespace {

constexpr int kTcThreads = 256;
constexpr int kTcM = 128;  // MMA rows (2d, zero-padded)
constexpr int kTcN = 64;   // positions per tile (MMA N)
constexpr int kTcK = 32;   // K per staged chunk (4 MMAs of K = 8)
constexpr int kAElems = kTcM * kTcK;  // floats per A chunk (hi or lo)
constexpr int kBElems = kTcN * kTcK;
constexpr int kStageFloats = 2 * kAElems + 2 * kBElems;
constexpr size_t kTcSmem = 2 * kStageFloats * sizeof(float);  // 96 KB
constexpr int64_t kTcMinElems = 16384;  // smaller lists stay on the CUDA cores
constexpr int kTcMaxSplit = 8;          // most parts a leg's terms are cut into

// CTA ranges, term parts and first plane of each leg of a one-output launch
struct TcLegs {
  int lt[4];  // leg l: CTAs [lt[l], lt[l+1]), ks[l] parts x its tiles
  int ks[3];
  int pb[3];
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// float offset of element (r, k) of an R x kTcK chunk in the canonical layout
__device__ __forceinline__ int cm_off(int r, int k) { return ((r >> 3) * (kTcK / 4) + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3); }
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)(128 >> 4) << 16;                  // leading byte offset: next core matrix along K
  d |= (uint64_t)((kTcK / 4 * 128) >> 4) << 32;     // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                           // descriptor version; base offset 0, no swizzle
  return d;
}
__device__ __forceinline__ float tf32_hi(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}
__device__ __forceinline__ bool mbar_done(uint64_t* mb, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
               : "=r"(ok)
               : "r"(smem_u32(mb)), "r"(parity)
               : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* mb, uint32_t parity, uint64_t deadline) {
  while (!mbar_done(mb, parity))
    if (gtimer() > deadline) return false;
  return true;
}

struct Geo3 {
  int d[3];
  int64_t st[3];
};
__device__ __forceinline__ Geo3 geo_of(const ApOut& o) {
  Geo3 g;
  g.d[0] = o.d0;
  g.d[1] = o.d1;
  g.d[2] = o.d2;
  g.st[0] = (int64_t)o.d1 * o.d2;
  g.st[1] = o.d2;
  g.st[2] = 1;
  return g;
}
// Embedded operands interleave real and imaginary parts: row 2i + c of A is
// component c of output index i, column 2x + c' pairs with component c' of X
// at leg index x, so A[2i+c][2x+c'] = (Re M, -Im M; Im M, Re M)[c][c'] at
// M[i][x] and B[n][2x+c'] = component c' of X at (x, position n). A chunk of
// 32 K columns covers 16 leg indices x; each complex value is read once.
// base[nn]: offset of tile position nn over the two other legs.
constexpr int kAq = (kTcM / 2) * (kTcK / 2) / kTcThreads;  // complex operator entries per thread and chunk
// The tensor operand is staged in items of one tile position nn and a pair
// of leg indices (2 xp, 2 xp + 1): their four floats (re, im, re, im) are one
// 16-byte row of a core matrix, written with one vector store per hi / lo
// plane; eight consecutive positions fill 128 contiguous bytes, so a warp's
// store touches each bank once per 128 bytes.
constexpr int kBp = kTcN * (kTcK / 4) / kTcThreads;  // (position, leg pair) items per thread and chunk
static_assert(kTcK / 4 == 8 && kTcN % 8 == 0, "item mapping below");
struct ChunkRegs {
  float2 m[kAq], x[2 * kBp];
};
// item e -> (nn, xp). Leg contiguous in X (x_fast): eight consecutive items
// are eight positions (one 128-byte smem segment), the next bits the pair;
// otherwise consecutive items are consecutive positions (contiguous in X).
__device__ __forceinline__ void b_item(int e, bool x_fast, int& nn, int& xp) {
  if (x_fast) {
    nn = ((e >> 6) << 3) | (e & 7);
    xp = (e >> 3) & 7;
  } else {
    nn = e % kTcN;
    xp = e / kTcN;
  }
}

// Load this thread's share of chunk kc (one L2 round trip; the values are
// split and stored later, so the loads overlap the MMAs of the previous chunk).
__device__ __forceinline__ void load_chunk(ChunkRegs& r, const float2* __restrict__ M, const float2* __restrict__ X,
                                           int d, int64_t st_l, bool x_fast, const int64_t* base, int nvalid,
                                           int kc, bool with_a) {
  const int x0 = kc * (kTcK / 2);
#pragma unroll
  for (int q = 0; q < kAq && with_a; ++q) {
    const int e = threadIdx.x + q * kTcThreads, i = e >> 4, x = x0 + (e & 15);
    r.m[q] = (i < d && x < d) ? M[i * d + x] : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int q = 0; q < kBp; ++q) {
    int nn, xp;
    b_item(threadIdx.x + q * kTcThreads, x_fast, nn, xp);
    const int x = x0 + 2 * xp;
    const bool ok = nn < nvalid;
    r.x[2 * q] = (ok && x < d) ? X[(int64_t)x * st_l + base[nn]] : make_float2(0.f, 0.f);
    r.x[2 * q + 1] = (ok && x + 1 < d) ? X[(int64_t)(x + 1) * st_l + base[nn]] : make_float2(0.f, 0.f);
  }
}
// Split into tf32 hi / lo, embed, and store into one stage buffer.
__device__ __forceinline__ void store_chunk(float* buf, const ChunkRegs& r, bool x_fast, bool with_a,
                                            bool with_b = true) {
  float* Ah = buf;
  float* Al = buf + kAElems;
  float* Bh = buf + 2 * kAElems;
  float* Bl = Bh + kBElems;
#pragma unroll
  for (int q = 0; q < kAq && with_a; ++q) {
    const int e = threadIdx.x + q * kTcThreads, i = e >> 4, xl = e & 15;
    const float v[4] = {r.m[q].x, -r.m[q].y, r.m[q].y, r.m[q].x};  // (c, c') = (0,0), (0,1), (1,0), (1,1)
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int o = cm_off(2 * i + (t >> 1), 2 * xl + (t & 1));
      const float h = tf32_hi(v[t]);
      Ah[o] = h;
      Al[o] = tf32_hi(v[t] - h);
    }
  }
#pragma unroll
  for (int q = 0; q < kBp && with_b; ++q) {
    int nn, xp;
    b_item(threadIdx.x + q * kTcThreads, x_fast, nn, xp);
    const int o = cm_off(nn, 4 * xp);  // K positions 4 xp .. 4 xp + 3: one 16-byte row
    const float2 a = r.x[2 * q], b = r.x[2 * q + 1];
    const float4 h = make_float4(tf32_hi(a.x), tf32_hi(a.y), tf32_hi(b.x), tf32_hi(b.y));
    *reinterpret_cast<float4*>(Bh + o) = h;
    *reinterpret_cast<float4*>(Bl + o) =
        make_float4(tf32_hi(a.x - h.x), tf32_hi(a.y - h.y), tf32_hi(b.x - h.z), tf32_hi(b.y - h.w));
  }
}

// Pre-split operator matrices: the A operand of every K chunk of a matrix,
// embedded and split exactly as the staging above would (hi then lo, each
// kTcM x kTcK floats in the canonical layout), so the apply kernel can copy a
// chunk with one bulk asynchronous copy. One CTA per (job, chunk).
__global__ void k_tc_embed(void* const* mats32, TcEmbedBatch jb, float* pool) {
  const TcEmbedJob j = jb.job[blockIdx.x];
  const int kc = blockIdx.y;
  if (kc >= (2 * j.d + kTcK - 1) / kTcK) return;
  const float2* M = (const float2*)mats32[j.mat];
  float* out = pool + j.off + (int64_t)kc * 2 * kAElems;
  ChunkRegs r;
  const int x0 = kc * (kTcK / 2);
#pragma unroll
  for (int q = 0; q < kAq; ++q) {
    const int e = threadIdx.x + q * kTcThreads, i = e >> 4, x = x0 + (e & 15);
    r.m[q] = (i < j.d && x < j.d) ? M[i * j.d + x] : make_float2(0.f, 0.f);
  }
  store_chunk(out, r, false, true, false);  // the A hi / lo halves only
}

// One CTA = one (output, 64-position tile) of one leg: Y_o (+)= sum over the
// output's terms on this leg of M_t x_leg X_t.
//  * leg >= 0 (lists of several outputs): every CTA works on `leg`; Y_o is the
//    STORE destination, the first leg with terms writes, later legs add
//    (separate launches in leg order).
//  * leg < 0 (lists of one output): the legs run in one launch, CTAs
//    [lg.lt[l], lg.lt[l+1]) on leg l; leg l's terms are cut into lg.ks[l]
//    contiguous parts, part j of a tile writing its own plane
//    part + (lg.pb[l] + j) * pstride; the epilogue adds the planes in order.
// Flag bit 3 on a timed-out MMA wait.
constexpr int kTcMaxTerms = 64;  // terms of one leg held in shared memory
__global__ void __launch_bounds__(kTcThreads) k_tc_apply(DevTables T, ApList L, int leg, TcLegs lg, float2* part,
                                                        int64_t pstride, int* flag, const float* pool,
                                                        const int64_t* pool_off) {
  extern __shared__ __align__(128) float tsm[];
  __shared__ __align__(8) uint64_t mbar[2], lbar[2];  // MMA commits, bulk A copies
  __shared__ uint32_t tmem_base;
  __shared__ int64_t base[kTcN];
  __shared__ int s_terms[kTcMaxTerms];  // this leg's terms, in list order
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool planes = leg < 0;
  // The job tables are read with parallel loads (one L2 round trip each
  // instead of one per output and per term): locate the output and tile of
  // this CTA, then list this leg's terms with their operands.
  __shared__ int s_o, s_tile, s_n, s_earlier;
  __shared__ ApTerm s_all[kTcMaxTerms];
  __shared__ const float2* s_M[kTcMaxTerms];
  __shared__ const float2* s_X[kTcMaxTerms];
  __shared__ int64_t s_poff[kTcMaxTerms];
  int o = L.out_begin, tile = blockIdx.x;
  int split = 0, nsplit = 1;
  if (planes) {
    const int bx = (int)blockIdx.x;
    leg = bx >= lg.lt[2] ? 2 : bx >= lg.lt[1] ? 1 : 0;
    nsplit = lg.ks[leg];
    const int ntile = (lg.lt[leg + 1] - lg.lt[leg]) / nsplit;
    split = (bx - lg.lt[leg]) / ntile;
    tile = (bx - lg.lt[leg]) % ntile;
  } else {
    if (warp == 0) {
      int found = -1, left = tile;
      for (int o0 = L.out_begin; o0 < L.out_end && found < 0; o0 += 32) {
        int nt = 0;
        if (o0 + lane < L.out_end) {
          const ApOut u = T.outs[o0 + lane];
          const int dl = leg == 0 ? u.d0 : leg == 1 ? u.d1 : u.d2;
          nt = (int)(((int64_t)u.d0 * u.d1 * u.d2 / dl + kTcN - 1) / kTcN);
        }
        int inc = nt;  // inclusive prefix sum over the lanes
        for (int k = 1; k < 32; k <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, inc, k);
          if (lane >= k) inc += v;
        }
        const unsigned hit = __ballot_sync(0xffffffffu, left < inc);
        if (hit) {
          const int fl = __ffs(hit) - 1;
          found = o0 + fl;
          left -= __shfl_sync(0xffffffffu, inc - nt, fl);
        } else {
          left -= __shfl_sync(0xffffffffu, inc, 31);
        }
      }
      if (lane == 0) {
        s_o = found;
        s_tile = left;
      }
    }
    __syncthreads();
    if (s_o < 0) return;  // uniform: past the last tile
    o = s_o;
    tile = s_tile;
  }
  const ApOut out = T.outs[o];
  const Geo3 g = geo_of(out);
  const int64_t rest = (int64_t)out.d0 * out.d1 * out.d2 / g.d[leg];
  const int n_all = out.term_end - out.term_begin;
  int n_here = 0;
  bool earlier = false;
  if (n_all <= kTcMaxTerms) {
    if (tid < n_all) s_all[tid] = T.terms[out.term_begin + tid];
    __syncthreads();
    if (tid == 0) {
      int n = 0, e = 0;
      for (int t = 0; t < n_all; ++t) {
        const ApTerm tm = s_all[t];
        if (tm.mat < 0) continue;
        if (tm.leg == leg) s_terms[n++] = out.term_begin + t;
        if (tm.leg < leg) e = 1;
      }
      s_n = n;
      s_earlier = e;
    }
    __syncthreads();
    n_here = s_n;
    earlier = s_earlier != 0;
  } else {
    for (int t = out.term_begin; t < out.term_end; ++t) {
      const ApTerm tm = T.terms[t];
      if (tm.mat < 0) continue;
      if (tm.leg == leg) {
        if (tid == 0 && n_here < kTcMaxTerms) s_terms[n_here] = t;
        ++n_here;
      }
      if (tm.leg < leg) earlier = true;
    }
  }
  __syncthreads();  // s_terms complete (both paths)
  if (tid < n_here && tid < kTcMaxTerms) {
    const ApTerm tm = T.terms[s_terms[tid]];
    s_M[tid] = (const float2*)T.mats[tm.mat];
    s_X[tid] = (const float2*)T.bufs[tm.src];
    s_poff[tid] = pool_off ? pool_off[tm.mat] : -1;
  }
  if (planes) earlier = false;  // own plane
  if (n_here == 0) return;  // uniform over the CTA
  const int d = g.d[leg];
  const int nkc = (2 * d + kTcK - 1) / kTcK;
  // this CTA's part of the leg's terms: [k_begin, k_begin + n_mine)
  const int k_begin = split * n_here / nsplit;
  const int n_mine = (split + 1) * n_here / nsplit - k_begin;
  const int nchunks = n_mine * nkc;
  const int64_t n0 = (int64_t)tile * kTcN;
  const int nvalid = rest - n0 < kTcN ? (int)(rest - n0) : kTcN;
  {
    const int la = leg == 0 ? 1 : 0, lb = leg == 2 ? 1 : 2;
    for (int nn = tid; nn < kTcN; nn += kTcThreads) {
      int64_t nb;
      const int64_t na = idivmod(n0 + nn, g.d[lb], nb);
      base[nn] = na * g.st[la] + nb * g.st[lb];
    }
  }
  __syncthreads();
  float2* Y = part ? part + (planes ? (int64_t)(lg.pb[leg] + split) * pstride : 0) : (float2*)T.bufs[out.dst];

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&lbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&lbar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(smem_u32(&tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // instruction descriptor: D f32, A/B tf32, both K-major, N = 64, M = 128
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
  const uint64_t deadline = gtimer() + 1000000000ull;
  bool ok = true;
  uint32_t ph[2] = {0u, 0u}, lph[2] = {0u, 0u};
  // asynchronous operations thread 0 issued and nobody has waited for yet: the
  // MMA commit of each stage and the bulk copy into each stage. A wait that
  // gives up stops thread 0 from issuing more; before the CTA frees its tensor
  // memory and leaves, thread 0 waits (bounded again) for whatever is pending.
  bool pend_m[2] = {false, false}, pend_l[2] = {false, false};

  // chunk ci -> (operator, tensor, K chunk); poff: pre-split operator offset or -1
  auto chunk_src = [&](int ci, const float2*& M, const float2*& X, int& kc, int64_t& poff) {
    int k = k_begin + ci / nkc;
    kc = ci % nkc;
    int tt = -1;
    if (n_here <= kTcMaxTerms) {
      M = s_M[k];
      X = s_X[k];
      poff = s_poff[k];
      return;
    } else {
      for (int t = out.term_begin; t < out.term_end; ++t) {
        const ApTerm tm = T.terms[t];
        if (tm.mat < 0 || tm.leg != leg) continue;
        if (k-- == 0) {
          tt = t;
          break;
        }
      }
    }
    const ApTerm tm = T.terms[tt];
    M = (const float2*)T.mats[tm.mat];
    X = (const float2*)T.bufs[tm.src];
    poff = pool_off ? pool_off[tm.mat] : -1;
  };
  // A chunk by one bulk copy from the pre-split pool (thread 0 issues it)
  auto bulk_a = [&](float* buf, int64_t poff, int kc, int b) {
    pend_l[b] = true;
    if (tid == 0) {
      const uint32_t bytes = 2u * kAElems * 4u;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&lbar[b])), "r"(bytes)
                   : "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_u32(buf)),
          "l"(pool + poff + (int64_t)kc * 2 * kAElems), "r"(bytes), "r"(smem_u32(&lbar[b]))
          : "memory");
    }
  };
  // Chunk ci is staged in stage ci & 1. Its tensor operand is loaded into
  // registers two iterations ahead (two register sets), so a chunk's loads
  // overlap the MMAs of the two chunks before it.
  bool bulk[2] = {false, false};  // does the A of the chunk of slot ci & 1 come from a bulk copy
  int64_t poffs[2] = {-1, -1};
  int kcs[2] = {0, 0};
  ChunkRegs R0, R1;
  const int64_t st_l = g.st[leg];  // stride of the contracted leg, read once
  // slot = ci & 1, passed as a literal so that these small arrays stay in registers
  auto fetch = [&](int ci, ChunkRegs& R, int slot) {
    const float2 *M, *X;
    int kc;
    int64_t poff;
    chunk_src(ci, M, X, kc, poff);
    bulk[slot] = poff >= 0;
    poffs[slot] = poff;
    kcs[slot] = kc;
    load_chunk(R, M, X, d, st_l, leg == 2, base, nvalid, kc, !bulk[slot]);
  };
  fetch(0, R0, 0);
  if (bulk[0]) bulk_a(tsm, poffs[0], kcs[0], 0);
  store_chunk(tsm, R0, leg == 2, !bulk[0]);
  if (nchunks > 1) fetch(1, R1, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  // one iteration: MMAs of chunk ci; loads of chunk ci+2 into Rld; chunk ci+1
  // (in Rst since the previous iteration) stored into the other stage
  auto step = [&](int ci, ChunkRegs& Rst, ChunkRegs& Rld, int b) {  // b = ci & 1, a literal
    float* buf = tsm + b * kStageFloats;
    // make the staged operands visible to the tensor core, then issue
    if (bulk[b] && ok) {
      ok = mbar_wait(&lbar[b], lph[b], deadline);
      if (ok) {
        lph[b] ^= 1u;
        pend_l[b] = false;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0 && ok) {
      const uint32_t ah = smem_u32(buf), al = ah + kAElems * 4, bh = al + kAElems * 4, bl = bh + kBElems * 4;
      const uint32_t a_op[3] = {ah, ah, al}, b_op[3] = {bh, bl, bh};
#pragma unroll
      for (int pass = 0; pass < 3; ++pass)
#pragma unroll
        for (int ks = 0; ks < kTcK / 8; ++ks) {
          const uint64_t ad = sdesc(a_op[pass] + ks * 256), bd = sdesc(b_op[pass] + ks * 256);
          const uint32_t accum = (ci > 0 || pass > 0 || ks > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
              : "memory");
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mbar[b]))
                   : "memory");
      pend_m[b] = true;
    }
    if (ci + 2 < nchunks) fetch(ci + 2, Rld, b);
    if (ci + 1 < nchunks) {
      // the other stage is free once the MMAs of chunk ci-1 have completed
      if (ci >= 1 && ok) {
        ok = mbar_wait(&mbar[b ^ 1], ph[b ^ 1], deadline);
        if (ok) {
          ph[b ^ 1] ^= 1u;
          pend_m[b ^ 1] = false;
        }
      }
      if (bulk[b ^ 1] && ok) bulk_a(tsm + (b ^ 1) * kStageFloats, poffs[b ^ 1], kcs[b ^ 1], b ^ 1);
      store_chunk(tsm + (b ^ 1) * kStageFloats, Rst, leg == 2, !bulk[b ^ 1]);
    }
  };
  for (int ci = 0; ci < nchunks; ci += 2) {
    step(ci, R1, R0, 0);
    if (ci + 1 < nchunks) step(ci + 1, R0, R1, 1);
  }
  // all MMAs done once the last commit has landed (they complete in order)
  if (ok) {
    const bool odd = ((nchunks - 1) & 1) != 0;
    ok = mbar_wait(odd ? &mbar[1] : &mbar[0], odd ? ph[1] : ph[0], deadline);
    if (ok) pend_m[odd ? 1 : 0] = false;
  }
  ok = __syncthreads_and(ok) != 0;  // CTA-uniform: tcgen05.ld below is warp-collective
  if (!ok && tid == 0) {
    atomicOr(flag, 8);
    // drain: no MMA may still write tensor memory, and no bulk copy may still
    // land in shared memory, once the CTA deallocates and exits
    const uint64_t drain = gtimer() + 1000000000ull;
    for (int b = 0; b < 2; ++b) {
      if (pend_m[b]) mbar_wait(&mbar[b], ph[b], drain);
      if (pend_l[b]) mbar_wait(&lbar[b], lph[b], drain);
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // tensor memory -> shared (rows = embedded output rows, 64 columns)
  float* Ds = tsm;  // [128][65]
  if (ok) {
    const int q = warp & 3, h = warp >> 2;
    uint32_t r[32];
    const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * h);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const int row = 32 * q + lane;
#pragma unroll
    for (int j = 0; j < 32; ++j) Ds[row * 65 + 32 * h + j] = __uint_as_float(r[j]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
  if (!ok) return;
  // write (or add) the complex outputs: Y(i, n) = Ds[2i][n] + i Ds[2i+1][n]
  for (int e = tid; e < d * kTcN; e += kTcThreads) {
    const int i = e / kTcN, nn = e % kTcN;
    if (nn >= nvalid) continue;
    const int64_t at = (int64_t)i * g.st[leg] + base[nn];
    float2 v = make_float2(Ds[(2 * i) * 65 + nn], Ds[(2 * i + 1) * 65 + nn]);
    if (earlier) {
      const float2 y = Y[at];
      v.x += y.x;
      v.y += y.y;
    }
    Y[at] = v;
  }
}

// Identity terms and the epilogue (RK4 stage update or nothing) of a list
// whose mode products ran on the tensor cores: the tiles of the apply kernel
// (32 elements), one thread per element. nplanes > 0 (one-output lists): the
// mode products are in the planes acc + q*pstride, q < nplanes, added here in
// plane order (leg by leg, each leg's term parts in order); otherwise in acc
// (RK) or the destination (store).
__global__ void k_tc_epilogue(DevTables T, ApList L, Epi ep, const float2* acc, int nplanes, int64_t pstride) {
  const int tile = blockIdx.x;
  const ApOut out = T.outs[list_output(T.outs, L.out_begin, L.out_end, L.tpo, tile)];
  const int64_t P = (int64_t)out.d0 * out.d1 * out.d2;
  const int64_t e = (int64_t)(tile - out.tile0) * kApTile + threadIdx.x;
  if (e >= P) return;
  bool any = false;
  float2 s = make_float2(0.f, 0.f);
  for (int t = out.term_begin; t < out.term_end; ++t) {
    const ApTerm tm = T.terms[t];
    if (tm.mat >= 0) {
      any = true;
      continue;
    }
    const float2 v = ((const float2*)T.bufs[tm.src])[e];
    s.x += v.x;
    s.y += v.y;
  }
  const bool rk = ep.mode != EPI_STORE;
  float2* Y = rk ? const_cast<float2*>(acc) : (float2*)T.bufs[out.dst];
  if (any) {
    float2 y = make_float2(0.f, 0.f);
    if (nplanes > 0) {
      y = acc[e];
      for (int q = 1; q < nplanes; ++q) {  // same order and operands as the adds of leg-by-leg launches
        const float2 v = acc[(int64_t)q * pstride + e];
        y.x = v.x + y.x;
        y.y = v.y + y.y;
      }
    } else {
      y = Y[e];
    }
    s.x += y.x;
    s.y += y.y;
  }
  if (!rk) {
    Y[e] = s;
    return;
  }
  const double2 k = make_double2(s.x, s.y);
  double2* y = ep.y;
  double2* ac = ep.acc;
  float2* ys = (float2*)ep.ys;
  const double h = ep.h;
  switch (ep.mode) {
    case EPI_RK1:
      ac[e] = k;
      ys[e] = make_float2((float)(y[e].x + 0.5 * h * k.x), (float)(y[e].y + 0.5 * h * k.y));
      break;
    case EPI_RK2:
      ac[e] = make_double2(ac[e].x + 2.0 * k.x, ac[e].y + 2.0 * k.y);
      ys[e] = make_float2((float)(y[e].x + 0.5 * h * k.x), (float)(y[e].y + 0.5 * h * k.y));
      break;
    case EPI_RK3:
      ac[e] = make_double2(ac[e].x + 2.0 * k.x, ac[e].y + 2.0 * k.y);
      ys[e] = make_float2((float)(y[e].x + h * k.x), (float)(y[e].y + h * k.y));
      break;
    default: {
      const double2 yn = make_double2(y[e].x + h / 6.0 * (ac[e].x + k.x), y[e].y + h / 6.0 * (ac[e].y + k.y));
      y[e] = yn;
      ((float2*)ep.y_lo)[e] = make_float2((float)yn.x, (float)yn.y);
      break;
    }
  }
}

// ---------------------------------------------------------------------------
// Pre-split tensor operand and the bulk-copy ring.
//
// k_tc_split writes, for one (source tensor, contracted leg) pair, the B
// operand of every (64-position tile, 32-float K chunk) block exactly as the
// staging above lays it out in shared memory: hi then lo, each kTcN x kTcK
// floats in the canonical K-major layout, one contiguous 16 KB block per
// (tile, chunk). k_tc_apply_ring then moves both operands of a chunk with two
// bulk asynchronous copies (32 KB of operator, 16 KB of tensor) into a ring
// of kRing stages: one producer thread issues the copies (completing on the
// stage's `full` mbarrier), one MMA thread waits for `full`, issues the 12
// MMAs of the chunk and commits them to the stage's `empty` mbarrier, which
// the producer waits on before it refills the stage. No CTA barrier runs in
// the chunk loop; the other warps join for the epilogue only.
// ---------------------------------------------------------------------------
constexpr int kRing = 4;
constexpr size_t kRingSmem = (size_t)kRing * kStageFloats * sizeof(float);  // 192 KB
constexpr int kTcMaxSplitJobs = 96;
struct TcSplitJob {
  int32_t src, leg, d0, d1, d2, tiles, nkc, pad;
  int64_t off;  // float offset of the pair's blocks in the split buffer
};
struct TcSplitJobs {
  int n;
  int start[kTcMaxSplitJobs + 1];  // first block of each job (prefix sums of tiles * nkc)
  TcSplitJob job[kTcMaxSplitJobs];
};
constexpr int kTcMaxListTerms = 320;
struct TcBOff {
  int t0, n;                       // terms t0 .. t0 + n - 1 of the global table
  int64_t off[kTcMaxListTerms];    // float offset of each term's split tensor operand (-1: none)
};

__global__ void __launch_bounds__(kTcThreads) k_tc_split(DevTables T, TcSplitJobs J, float* __restrict__ bs) {
  const int b = blockIdx.x;
  if (b >= J.start[J.n]) return;
  int j = 0;
  while (j + 1 < J.n && J.start[j + 1] <= b) ++j;
  const TcSplitJob jb = J.job[j];
  const int local = b - J.start[j];
  const int tile = local / jb.nkc, kc = local % jb.nkc;
  const float2* __restrict__ X = (const float2*)T.bufs[jb.src];
  const int d[3] = {jb.d0, jb.d1, jb.d2};
  const int64_t st[3] = {(int64_t)jb.d1 * jb.d2, jb.d2, 1};
  const int l = jb.leg, la = l == 0 ? 1 : 0, lb = l == 2 ? 1 : 2;
  const int dl = d[l];
  const int64_t rest = (int64_t)jb.d0 * jb.d1 * jb.d2 / dl;
  float* Bh = bs + jb.off + ((int64_t)tile * jb.nkc + kc) * 2 * kBElems;
  float* Bl = Bh + kBElems;
  const int x0 = kc * (kTcK / 2);
#pragma unroll
  for (int q = 0; q < kBp; ++q) {
    int nn, xp;
    b_item(threadIdx.x + q * kTcThreads, l == 2, nn, xp);
    const int64_t n = (int64_t)tile * kTcN + nn;
    const int x = x0 + 2 * xp;
    float2 a = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
    if (n < rest) {
      int64_t nb;
      const int64_t base = idivmod(n, d[lb], nb) * st[la] + nb * st[lb];
      if (x < dl) a = X[(int64_t)x * st[l] + base];
      if (x + 1 < dl) c = X[(int64_t)(x + 1) * st[l] + base];
    }
    const int o = cm_off(nn, 4 * xp);
    const float4 h = make_float4(tf32_hi(a.x), tf32_hi(a.y), tf32_hi(c.x), tf32_hi(c.y));
    *reinterpret_cast<float4*>(Bh + o) = h;
    *reinterpret_cast<float4*>(Bl + o) =
        make_float4(tf32_hi(a.x - h.x), tf32_hi(a.y - h.y), tf32_hi(c.x - h.z), tf32_hi(c.y - h.w));
  }
}

__device__ __forceinline__ void bulk_g2s(float* dst, const float* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Same CTA -> (output, leg, tile, term part) mapping and outputs as
// k_tc_apply; every term needs its operator in the pool and its tensor
// operand in the split buffer (the host checks both).
__global__ void __launch_bounds__(kTcThreads) k_tc_apply_ring(DevTables T, ApList L, int leg, TcLegs lg, float2* part,
                                                             int64_t pstride, int* flag, const float* pool,
                                                             const int64_t* pool_off, const float* bsplit,
                                                             TcBOff boff) {
  extern __shared__ __align__(128) float tsm[];
  __shared__ __align__(8) uint64_t full[kRing], empty[kRing], done;
  __shared__ uint32_t tmem_base;
  __shared__ int64_t base[kTcN];
  __shared__ int s_terms[kTcMaxTerms];
  __shared__ int s_o, s_tile, s_n, s_earlier;
  __shared__ ApTerm s_all[kTcMaxTerms];
  __shared__ int64_t s_poff[kTcMaxTerms], s_boff[kTcMaxTerms];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool planes = leg < 0;
  int o = L.out_begin, tile = blockIdx.x;
  int split = 0, nsplit = 1;
  if (planes) {
    const int bx = (int)blockIdx.x;
    leg = bx >= lg.lt[2] ? 2 : bx >= lg.lt[1] ? 1 : 0;
    nsplit = lg.ks[leg];
    const int ntile = (lg.lt[leg + 1] - lg.lt[leg]) / nsplit;
    split = (bx - lg.lt[leg]) / ntile;
    tile = (bx - lg.lt[leg]) % ntile;
  } else {
    if (warp == 0) {
      int found = -1, left = tile;
      for (int o0 = L.out_begin; o0 < L.out_end && found < 0; o0 += 32) {
        int nt = 0;
        if (o0 + lane < L.out_end) {
          const ApOut u = T.outs[o0 + lane];
          const int dl = leg == 0 ? u.d0 : leg == 1 ? u.d1 : u.d2;
          nt = (int)(((int64_t)u.d0 * u.d1 * u.d2 / dl + kTcN - 1) / kTcN);
        }
        int inc = nt;
        for (int k = 1; k < 32; k <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, inc, k);
          if (lane >= k) inc += v;
        }
        const unsigned hit = __ballot_sync(0xffffffffu, left < inc);
        if (hit) {
          const int fl = __ffs(hit) - 1;
          found = o0 + fl;
          left -= __shfl_sync(0xffffffffu, inc - nt, fl);
        } else {
          left -= __shfl_sync(0xffffffffu, inc, 31);
        }
      }
      if (lane == 0) {
        s_o = found;
        s_tile = left;
      }
    }
    __syncthreads();
    if (s_o < 0) return;
    o = s_o;
    tile = s_tile;
  }
  const ApOut out = T.outs[o];
  const Geo3 g = geo_of(out);
  const int64_t rest = (int64_t)out.d0 * out.d1 * out.d2 / g.d[leg];
  const int n_all = out.term_end - out.term_begin;  // <= kTcMaxTerms (host check)
  if (tid < n_all) s_all[tid] = T.terms[out.term_begin + tid];
  __syncthreads();
  if (tid == 0) {
    int n = 0, e = 0;
    for (int t = 0; t < n_all; ++t) {
      const ApTerm tm = s_all[t];
      if (tm.mat < 0) continue;
      if (tm.leg == leg) s_terms[n++] = out.term_begin + t;
      if (tm.leg < leg) e = 1;
    }
    s_n = n;
    s_earlier = e;
  }
  __syncthreads();
  const int n_here = s_n;
  const bool earlier = planes ? false : s_earlier != 0;
  if (tid < n_here) {
    const int t = s_terms[tid];
    s_poff[tid] = pool_off[T.terms[t].mat];
    s_boff[tid] = boff.off[t - boff.t0];
  }
  if (n_here == 0) return;  // uniform
  const int d = g.d[leg];
  const int nkc = (2 * d + kTcK - 1) / kTcK;
  const int k_begin = split * n_here / nsplit;
  const int n_mine = (split + 1) * n_here / nsplit - k_begin;
  const int nchunks = n_mine * nkc;
  const int64_t n0 = (int64_t)tile * kTcN;
  const int nvalid = rest - n0 < kTcN ? (int)(rest - n0) : kTcN;
  {
    const int la = leg == 0 ? 1 : 0, lb = leg == 2 ? 1 : 2;
    for (int nn = tid; nn < kTcN; nn += kTcThreads) {
      int64_t nb;
      const int64_t na = idivmod(n0 + nn, g.d[lb], nb);
      base[nn] = na * g.st[la] + nb * g.st[lb];
    }
  }
  float2* Y = part ? part + (planes ? (int64_t)(lg.pb[leg] + split) * pstride : 0) : (float2*)T.bufs[out.dst];
  if (tid == 0) {
    for (int s = 0; s < kRing; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(smem_u32(&tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
  const uint64_t deadline = gtimer() + 1000000000ull;
  bool ok = true;
  // producer: thread 0; issued[s] = copies into stage s so far (the k-th
  // completes phase k - 1 of full[s]). MMA thread: warp 1 lane 0.
  int issued[kRing] = {0, 0, 0, 0};
  bool mma_pending = false;  // MMAs issued (the drain commits and waits for them)
  // lanes 1..31 of the two role warps park at __syncwarp (no spinning next
  // to their lane 0); the other warps wait for `done` below
  if (tid == 0) {
    for (int ci = 0; ci < nchunks && ok; ++ci) {
      const int s = ci % kRing;
      if (ci >= kRing) ok = mbar_wait(&empty[s], (uint32_t)(((ci / kRing) - 1) & 1), deadline);
      if (!ok) break;
      const int k = k_begin + ci / nkc, kc = ci % nkc;
      float* buf = tsm + s * kStageFloats;
      const uint32_t abytes = 2u * kAElems * 4u, bbytes = 2u * kBElems * 4u;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&full[s])),
                   "r"(abytes + bbytes)
                   : "memory");
      bulk_g2s(buf, pool + s_poff[k] + (int64_t)kc * 2 * kAElems, abytes, &full[s]);
      bulk_g2s(buf + 2 * kAElems, bsplit + s_boff[k] + ((int64_t)tile * nkc + kc) * 2 * kBElems, bbytes, &full[s]);
      ++issued[s];
    }
  } else if (tid == 32) {
    for (int ci = 0; ci < nchunks && ok; ++ci) {
      const int s = ci % kRing;
      ok = mbar_wait(&full[s], (uint32_t)((ci / kRing) & 1), deadline);
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ah = smem_u32(tsm + s * kStageFloats), al = ah + kAElems * 4, bh = al + kAElems * 4,
                     bl = bh + kBElems * 4;
      const uint32_t a_op[3] = {ah, ah, al}, b_op[3] = {bh, bl, bh};
#pragma unroll
      for (int pass = 0; pass < 3; ++pass)
#pragma unroll
        for (int ks = 0; ks < kTcK / 8; ++ks) {
          const uint64_t ad = sdesc(a_op[pass] + ks * 256), bd = sdesc(b_op[pass] + ks * 256);
          const uint32_t accum = (ci > 0 || pass > 0 || ks > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
              : "memory");
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&empty[s]))
                   : "memory");
      mma_pending = true;
    }
    if (ok) {
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&done))
                   : "memory");
    }
  }
  if (warp < 2) __syncwarp();
  // every thread: the accumulator is complete once `done` has fired
  if (ok) ok = mbar_wait(&done, 0u, deadline);
  ok = __syncthreads_and(ok) != 0;
  if (!ok) {
    if (tid == 0) atomicOr(flag, 8);
    // drain: no copy may still land in shared memory and no MMA may still run
    // once the CTA frees its tensor memory and exits
    const uint64_t drain = gtimer() + 1000000000ull;
    if (tid == 0)
      for (int s = 0; s < kRing; ++s)
        if (issued[s] > 0) mbar_wait(&full[s], (uint32_t)((issued[s] - 1) & 1), drain);
    if (tid == 32 && mma_pending) {
      // a commit tracks every MMA this thread issued before it
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&done))
                   : "memory");
      mbar_wait(&done, 0u, drain);
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  float* Ds = tsm;  // [128][65], the ring is idle now
  if (ok) {
    const int q = warp & 3, h = warp >> 2;
    uint32_t r[32];
    const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * h);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const int row = 32 * q + lane;
#pragma unroll
    for (int j = 0; j < 32; ++j) Ds[row * 65 + 32 * h + j] = __uint_as_float(r[j]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
  if (!ok) return;
  for (int e = tid; e < d * kTcN; e += kTcThreads) {
    const int i = e / kTcN, nn = e % kTcN;
    if (nn >= nvalid) continue;
    const int64_t at = (int64_t)i * g.st[leg] + base[nn];
    float2 v = make_float2(Ds[(2 * i) * 65 + nn], Ds[(2 * i + 1) * 65 + nn]);
    if (earlier) {
      const float2 y = Y[at];
      v.x += y.x;
      v.y += y.y;
    }
    Y[at] = v;
  }
}

// Split plan of a list for the ring kernel: the distinct (source, leg) pairs of
// its tensor-core terms, their blocks in the split buffer, and every term's
// offset. False when the list does not fit the kernel's tables (more than
// kTcMaxTerms terms on an output, kTcMaxListTerms in the list, kTcMaxSplitJobs
// pairs) or some operator has no pre-split copy (pool_off_host < 0).
bool tc_ring_plan(const ApList& L, const ApOut* outs, const ApTerm* terms, const int64_t* pool_off_host,
                  TcSplitJobs* J, TcBOff* B, int64_t* floats) {
  int t0 = 1 << 30, t1 = 0;
  for (int o = L.out_begin; o < L.out_end; ++o) {
    const ApOut& u = outs[o];
    if (u.term_end - u.term_begin > kTcMaxTerms) return false;
    t0 = std::min(t0, u.term_begin);
    t1 = std::max(t1, u.term_end);
  }
  if (t1 <= t0 || t1 - t0 > kTcMaxListTerms) return false;
  B->t0 = t0;
  B->n = t1 - t0;
  for (int i = 0; i < kTcMaxListTerms; ++i) B->off[i] = -1;
  J->n = 0;
  int64_t off = 0;
  for (int o = L.out_begin; o < L.out_end; ++o) {
    const ApOut& u = outs[o];
    const int dd[3] = {u.d0, u.d1, u.d2};
    const int64_t P = (int64_t)u.d0 * u.d1 * u.d2;
    for (int t = u.term_begin; t < u.term_end; ++t) {
      const ApTerm& tm = terms[t];
      if (tm.mat < 0) continue;
      if (!pool_off_host || pool_off_host[tm.mat] < 0) return false;
      int j = 0;
      for (; j < J->n; ++j) {
        const TcSplitJob& q = J->job[j];
        if (q.src == tm.src && q.leg == tm.leg && q.d0 == u.d0 && q.d1 == u.d1 && q.d2 == u.d2) break;
      }
      if (j == J->n) {
        if (J->n == kTcMaxSplitJobs) return false;
        TcSplitJob q{};
        q.src = tm.src;
        q.leg = tm.leg;
        q.d0 = u.d0;
        q.d1 = u.d1;
        q.d2 = u.d2;
        q.tiles = (int)((P / dd[tm.leg] + kTcN - 1) / kTcN);
        q.nkc = (2 * dd[tm.leg] + kTcK - 1) / kTcK;
        q.off = off;
        off += (int64_t)q.tiles * q.nkc * 2 * kBElems;
        J->job[J->n++] = q;
      }
      B->off[t - t0] = J->job[j].off;
    }
  }
  J->start[0] = 0;
  for (int j = 0; j < J->n; ++j) J->start[j + 1] = J->start[j] + J->job[j].tiles * J->job[j].nkc;
  *floats = off;
  return true;
}

}  // namespace

int64_t tc_split_floats(const ApList& L, const ApOut* outs_host, const ApTerm* terms_host,
                        const int64_t* pool_off_host) {
  thread_local TcSplitJobs J;
  thread_local TcBOff B;
  int64_t f = 0;
  return tc_ring_plan(L, outs_host, terms_host, pool_off_host, &J, &B, &f) ? f : 0;
}

bool launch_apply_tc(const DevTables& T, const ApList& L, const Epi& e, const ApOut* outs_host,
                     const ApTerm* terms_host, float2* acc, int64_t acc_elems, int* flag, const float* pool,
                     const int64_t* pool_off, cudaStream_t s, const int64_t* pool_off_host, float* bsplit,
                     int64_t bsplit_floats, bool* used_ring) {
  if (used_ring) *used_ring = false;
  if (L.n_tiles <= 0) return true;
  // the bulk-copy ring when both operands of every term can arrive pre-split
  thread_local TcSplitJobs J;  // kernel arguments (copied at launch); per thread: handles are independent
  thread_local TcBOff B;
  int64_t need = 0;
  const bool ring = pool && pool_off && bsplit &&
                    tc_ring_plan(L, outs_host, terms_host, pool_off_host, &J, &B, &need) && need <= bsplit_floats;
  static bool ring_attr = false;
  if (ring && !ring_attr) {
    cudaFuncSetAttribute(k_tc_apply_ring, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingSmem);
    ring_attr = true;
  }
  if (ring && J.start[J.n] > 0) k_tc_split<<<J.start[J.n], kTcThreads, 0, s>>>(T, J, bsplit);
  if (used_ring) *used_ring = ring;
  const bool rk = e.mode != EPI_STORE;
  const bool one = L.out_end - L.out_begin == 1;
  if (rk && (!one || !acc)) return false;
  int tiles[3] = {0, 0, 0};
  bool has[3] = {false, false, false}, ident = false;
  int64_t P = 0;
  for (int o = L.out_begin; o < L.out_end; ++o) {
    const ApOut& u = outs_host[o];
    const int dd[3] = {u.d0, u.d1, u.d2};
    P = (int64_t)u.d0 * u.d1 * u.d2;
    for (int l = 0; l < 3; ++l) tiles[l] += (int)((P / dd[l] + kTcN - 1) / kTcN);
    for (int t = u.term_begin; t < u.term_end; ++t) {
      if (terms_host[t].mat < 0)
        ident = true;
      else
        has[terms_host[t].leg] = true;
    }
  }
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_tc_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    attr = true;
  }
  // one output whose leg planes fit the scratch: all legs in one launch, a
  // leg's terms cut into parts while that shortens the longest per-CTA chain
  // and the launch stays within about two CTAs per SM
  if (one && acc && 3 * P <= acc_elems) {
    static int sms = 0;
    if (sms == 0) {
      int dev = 0;
      if (cudaGetDevice(&dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 1;
    }
    const ApOut& u = outs_host[L.out_begin];
    const int dd[3] = {u.d0, u.d1, u.d2};
    int nterm[3] = {0, 0, 0};
    for (int t = u.term_begin; t < u.term_end; ++t)
      if (terms_host[t].mat >= 0) ++nterm[terms_host[t].leg];
    TcLegs lg{};
    int ctas = 0, planes = 0;
    for (int l = 0; l < 3; ++l) {
      lg.ks[l] = 1;
      if (has[l]) {
        ctas += tiles[l];
        ++planes;
      }
    }
    for (;;) {
      int best = -1;
      int64_t chain = 0;
      for (int l = 0; l < 3; ++l) {
        if (!has[l]) continue;
        const int64_t c = (int64_t)((nterm[l] + lg.ks[l] - 1) / lg.ks[l]) * ((2 * dd[l] + kTcK - 1) / kTcK);
        if (c > chain) {
          chain = c;
          best = l;
        }
      }
      if (best < 0 || lg.ks[best] >= std::min(nterm[best], kTcMaxSplit)) break;
      if (ctas + tiles[best] > 2 * sms || (int64_t)(planes + 1) * P > acc_elems) break;
      ++lg.ks[best];
      ctas += tiles[best];
      ++planes;
    }
    int q = 0;
    lg.lt[0] = 0;
    for (int l = 0; l < 3; ++l) {
      lg.pb[l] = q;
      const int n = has[l] ? tiles[l] * lg.ks[l] : 0;
      lg.lt[l + 1] = lg.lt[l] + n;
      if (has[l]) q += lg.ks[l];
    }
    if (lg.lt[3] > 0) {
      if (ring)
        k_tc_apply_ring<<<lg.lt[3], kTcThreads, kRingSmem, s>>>(T, L, -1, lg, acc, P, flag, pool, pool_off, bsplit,
                                                                B);
      else
        k_tc_apply<<<lg.lt[3], kTcThreads, kTcSmem, s>>>(T, L, -1, lg, acc, P, flag, pool, pool_off);
    }
    k_tc_epilogue<<<L.n_tiles, 32, 0, s>>>(T, L, e, acc, q, P);
    return true;
  }
  const TcLegs none{};
  for (int l = 0; l < 3; ++l)
    if (has[l]) {
      float2* part = rk ? acc : nullptr;  // RK lists: the single output's sum goes to acc
      if (ring)
        k_tc_apply_ring<<<tiles[l], kTcThreads, kRingSmem, s>>>(T, L, l, none, part, 0, flag, pool, pool_off, bsplit,
                                                                B);
      else
        k_tc_apply<<<tiles[l], kTcThreads, kTcSmem, s>>>(T, L, l, none, part, 0, flag, pool, pool_off);
    }
  if (rk || ident) k_tc_epilogue<<<L.n_tiles, 32, 0, s>>>(T, L, e, acc, 0, 0);
  return true;
}

int64_t tc_pool_floats(int d) { return d > kTcM / 2 ? 0 : (int64_t)((2 * d + kTcK - 1) / kTcK) * 2 * kAElems; }

void launch_tc_embed(void* const* mats32, const TcEmbedJob* jobs, int n, float* pool, cudaStream_t s) {
  for (int i0 = 0; i0 < n; i0 += kTcEmbedBatch) {
    TcEmbedBatch b{};
    b.n = std::min(kTcEmbedBatch, n - i0);
    for (int i = 0; i < b.n; ++i) b.job[i] = jobs[i0 + i];
    k_tc_embed<<<dim3(b.n, (kTcM + kTcK - 1) / kTcK), kTcThreads, 0, s>>>(mats32, b, pool);
  }
}

bool tc_applicable(const ApList& L, const ApOut* outs_host, const ApTerm* terms_host) {
  int64_t pmax = 0;
  for (int o = L.out_begin; o < L.out_end; ++o) {
    const ApOut& u = outs_host[o];
    if (u.d3 != 1) return false;
    const int dd[3] = {u.d0, u.d1, u.d2};
    pmax = std::max<int64_t>(pmax, (int64_t)u.d0 * u.d1 * u.d2);
    for (int t = u.term_begin; t < u.term_end; ++t) {
      const ApTerm& tm = terms_host[t];
      if (tm.mat < 0) continue;
      if (tm.leg < 0 || tm.leg > 2 || dd[tm.leg] > kTcM / 2) return false;
    }
  }
  return pmax >= kTcMinElems;
}

}  // namespace ttn
