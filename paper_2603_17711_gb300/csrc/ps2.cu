// Kernels of the adaptive-rank (ps2) two-site update, FP64.
//
//  k_merge      Theta = U_first contracted with U_second over their shared bond
//               (legs: first's other legs, then second's other legs).
//  k_jacobi     one-sided (Hestenes) Jacobi SVD of Theta matricised as
//               (first's legs) x (second's legs), on the smaller side; sweeps of
//               the round-robin (circle-method) pairing, one warp per column
//               pair, complex rotations that make the pair orthogonal.
//  k_svd_vecs   kept singular triplets -> the isometry side's basis Z (columns,
//               normalised) and the centre side's factor (sigma times the other
//               singular vectors); numerically undetermined triplets get zero.
//  k_write_pair new node tensors (canonical leg order) from Z and the centre factor.
#include "kernels.cuh"

namespace ttn {

namespace {

__device__ __forceinline__ double2 cm(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double ws(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// the two legs of a 3-leg node other than `skip`, in order
__device__ __forceinline__ void others(int skip, int& l0, int& l1) {
  l0 = skip == 0 ? 1 : 0;
  l1 = skip == 2 ? 1 : 2;
}

}  // namespace

__global__ void k_merge(const double2* Uf, int f0, int f1, int f2, int lf, const double2* Us, int s0, int s1,
                        int s2, int ls, double2* theta, float2* theta_lo) {
  const int fd[3] = {f0, f1, f2}, sd[3] = {s0, s1, s2};
  const int64_t fs[3] = {(int64_t)f1 * f2, f2, 1}, ss[3] = {(int64_t)s1 * s2, s2, 1};
  int fa, fb, sa, sb;
  others(lf, fa, fb);
  others(ls, sa, sb);
  const int r = fd[lf];
  const int64_t n = (int64_t)fd[fa] * fd[fb] * sd[sa] * sd[sb];
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t i3, i2, i1;
    int64_t q = idivmod(idx, sd[sb], i3);
    q = idivmod(q, sd[sa], i2);
    const int64_t i0 = idivmod(q, fd[fb], i1);
    const double2* pf = Uf + i0 * fs[fa] + i1 * fs[fb];
    const double2* ps = Us + i2 * ss[sa] + i3 * ss[sb];
    double2 acc = make_double2(0.0, 0.0);
    for (int a = 0; a < r; ++a) {
      const double2 x = pf[a * fs[lf]], y = ps[a * ss[ls]];
      acc.x = fma(x.x, y.x, fma(-x.y, y.y, acc.x));
      acc.y = fma(x.x, y.y, fma(x.y, y.x, acc.y));
    }
    theta[idx] = acc;
    if (theta_lo) theta_lo[idx] = make_float2((float)acc.x, (float)acc.y);
  }
}

void launch_merge(const double2* Uf, const int* fd, int lf, const double2* Us, const int* sd, int ls,
                  double2* theta, float2* theta_lo, cudaStream_t s) {
  const int64_t n = (int64_t)fd[0] * fd[1] * fd[2] / fd[lf] * ((int64_t)sd[0] * sd[1] * sd[2] / sd[ls]);
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 2048);
  k_merge<<<blocks, 256, 0, s>>>(Uf, fd[0], fd[1], fd[2], lf, Us, sd[0], sd[1], sd[2], ls, theta, theta_lo);
}

constexpr int kJacThreads = 512;
constexpr int kJacChunk = 128;  // pairs of one round whose Gram entries and rotations sit in shared memory

// One round of pairs is handled in three phases, chunk by chunk: each warp sums
// the Gram entries of its pairs (lanes split the rows), one lane per pair then
// computes the rotations of the whole chunk (so the square roots and quotients
// cost one warp instruction stream instead of one per pair), and the warps
// apply them to their pairs' columns of A and V.
__global__ void __launch_bounds__(kJacThreads) k_jacobi(const double2* theta, int m, int n, double2* A, double2* V,
                                                        double* sigma, int* info, double tol, int max_sweeps) {
  __shared__ int s_rot;
  __shared__ double s_g[kJacChunk][4];
  __shared__ double s_r[kJacChunk][4];
  __shared__ int s_go[kJacChunk];
  const bool tr = n > m;
  const int nr = tr ? n : m, nc = tr ? m : n;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  for (int64_t k = tid; k < (int64_t)nr * nc; k += blockDim.x) {
    const int r = (int)(k % nr), c = (int)(k / nr);
    A[k] = tr ? cj(theta[(int64_t)c * n + r]) : theta[(int64_t)r * n + c];
  }
  for (int64_t k = tid; k < (int64_t)nc * nc; k += blockDim.x)
    V[k] = make_double2((k % nc) == (k / nc) ? 1.0 : 0.0, 0.0);
  __syncthreads();
  // ||A||_F^2 (fixed-order sums): columns at the rounding floor of the matrix
  // are not rotated (see jacobi_negligible)
  __shared__ double s_fro[kJacThreads / 32];
  {
    double f = 0.0;
    for (int64_t k = tid; k < (int64_t)nr * nc; k += blockDim.x) f += A[k].x * A[k].x + A[k].y * A[k].y;
    f = ws(f);
    if (lane == 0) s_fro[wid] = f;
    __syncthreads();
  }
  double fro2 = 0.0;
  for (int w = 0; w < nw; ++w) fro2 += s_fro[w];
  const double tiny2 = jacobi_negligible(nr, fro2);
  const int N = nc + (nc & 1), npairs = N / 2;
  auto pair_of = [&](int rd, int p, int& i, int& j) {
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
  };
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int rd = 0; rd < N - 1; ++rd) {
      for (int p0 = 0; p0 < npairs; p0 += kJacChunk) {
        const int np = min(kJacChunk, npairs - p0);
        for (int q = wid; q < np; q += nw) {  // Gram entries
          int i, j;
          pair_of(rd, p0 + q, i, j);
          if (j >= nc) continue;
          const double2* x = A + (int64_t)i * nr;
          const double2* y = A + (int64_t)j * nr;
          double a = 0.0, b = 0.0, cr = 0.0, ci = 0.0;
          for (int r = lane; r < nr; r += 32) {
            const double2 xv = x[r], yv = y[r];
            a += xv.x * xv.x + xv.y * xv.y;
            b += yv.x * yv.x + yv.y * yv.y;
            cr += xv.x * yv.x + xv.y * yv.y;  // conj(x) y
            ci += xv.x * yv.y - xv.y * yv.x;
          }
          const double sum = warp_sum4(a, b, cr, ci);
          if ((lane & 7) == 0) s_g[q][lane >> 3] = sum;
        }
        __syncthreads();
        for (int q = tid; q < np; q += blockDim.x) {  // rotations, one lane per pair
          int i, j;
          pair_of(rd, p0 + q, i, j);
          double cs = 1.0, sn = 0.0;
          double2 e = make_double2(1.0, 0.0);
          const int go = j < nc && jacobi_rotation(s_g[q][0], s_g[q][1], s_g[q][2], s_g[q][3], tol, tiny2, cs, sn, e);
          s_r[q][0] = cs;
          s_r[q][1] = sn;
          s_r[q][2] = e.x;
          s_r[q][3] = e.y;
          s_go[q] = go;
          if (go) atomicAdd(&s_rot, 1);
        }
        __syncthreads();
        for (int q = wid; q < np; q += nw) {  // apply
          if (!s_go[q]) continue;
          int i, j;
          pair_of(rd, p0 + q, i, j);
          const double cs = s_r[q][0], sn = s_r[q][1];
          const double2 e = make_double2(s_r[q][2], s_r[q][3]);
          double2* x = A + (int64_t)i * nr;
          double2* y = A + (int64_t)j * nr;
          for (int r = lane; r < nr; r += 32) {
            const double2 xv = x[r], yv = cm(e, y[r]);
            x[r] = make_double2(cs * xv.x - sn * yv.x, cs * xv.y - sn * yv.y);
            y[r] = make_double2(sn * xv.x + cs * yv.x, sn * xv.y + cs * yv.y);
          }
          double2* vx = V + (int64_t)i * nc;
          double2* vy = V + (int64_t)j * nc;
          for (int r = lane; r < nc; r += 32) {
            const double2 xv = vx[r], yv = cm(e, vy[r]);
            vx[r] = make_double2(cs * xv.x - sn * yv.x, cs * xv.y - sn * yv.y);
            vy[r] = make_double2(sn * xv.x + cs * yv.x, sn * xv.y + cs * yv.y);
          }
        }
        __syncthreads();
      }
    }
    const int rot = s_rot;
    __syncthreads();
    if (rot == 0) break;
  }
  for (int j = wid; j < nc; j += nw) {
    const double2* x = A + (int64_t)j * nr;
    double a = 0.0;
    for (int r = lane; r < nr; r += 32) a += x[r].x * x[r].x + x[r].y * x[r].y;
    a = ws(a);
    if (lane == 0) sigma[j] = sqrt(a);
  }
  if (tid == 0) {
    info[0] = sweep;
    info[1] = tr ? 1 : 0;
  }
}

void launch_jacobi_svd(const double2* theta, int m, int n, double2* A, double2* V, double* sigma, int* info,
                       cudaStream_t s) {
  k_jacobi<<<1, kJacThreads, 0, s>>>(theta, m, n, A, V, sigma, info, jacobi_tol(m, n), kJacMaxSweeps);
}

// Z (rows_iso x r, row-major) and the centre factor Cm (row-major: first side
// rows x r when the centre is the first node, r x cols when it is the second).
// Left_j / Right_j are the singular vectors of Theta = Left diag(sigma) Right^H.
__global__ void k_svd_vecs(const double2* A, const double2* V, const double* sigma, int m, int n,
                           const int* perm, int r, int g, int iso_first, double2* Z, double2* Zg, double2* Cm) {
  const bool tr = n > m;
  const int nr = tr ? n : m, nc = tr ? m : n;
  const int rows_iso = iso_first ? m : n, rows_c = iso_first ? n : m;
  const int64_t nz = (int64_t)rows_iso * r, ncm = (int64_t)rows_c * r;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nz + ncm;
       k += (int64_t)gridDim.x * blockDim.x) {
    const bool zpart = k < nz;
    const int64_t kk = zpart ? k : k - nz;
    const int a = (int)(kk % r);
    const int row = (int)(kk / r);
    const int j = perm[a];
    const double sj = sigma[j];
    const bool good = a < g;
    // left (length m) and right (length n) singular vector entries
    auto left = [&](int i) -> double2 {
      if (tr) return V[(int64_t)j * nc + i];
      const double2 v = A[(int64_t)j * nr + i];
      return make_double2(v.x / sj, v.y / sj);
    };
    auto right = [&](int i) -> double2 {
      if (!tr) return V[(int64_t)j * nc + i];
      const double2 v = A[(int64_t)j * nr + i];
      return make_double2(v.x / sj, v.y / sj);
    };
    if (zpart) {
      double2 v = make_double2(0.0, 0.0);
      if (good) v = iso_first ? left(row) : cj(right(row));
      Z[kk] = v;
      Zg[kk] = v;
    } else {
      double2 v = make_double2(0.0, 0.0);
      if (good) {
        if (iso_first) {  // centre = second: Cm[a][col] = sigma conj(right)
          const double2 w = cj(right(row));
          v = make_double2(sj * w.x, sj * w.y);
        } else {  // centre = first: Cm[row][a] = sigma left
          const double2 w = left(row);
          v = make_double2(sj * w.x, sj * w.y);
        }
      }
      // storage: centre second -> [a][col]; centre first -> [row][a]
      if (iso_first)
        Cm[(int64_t)a * rows_c + row] = v;
      else
        Cm[(int64_t)row * r + a] = v;
    }
  }
}

void launch_svd_vecs(const double2* A, const double2* V, const double* sigma, int m, int n, const int* perm, int r,
                     int g, bool iso_first, double2* Z, double2* Zg, double2* Cm, cudaStream_t s) {
  const int64_t tot = (int64_t)(m + n) * r;
  const int blocks = (int)std::min<int64_t>((tot + 255) / 256, 1024);
  k_svd_vecs<<<blocks, 256, 0, s>>>(A, V, sigma, m, n, perm, r, g, iso_first ? 1 : 0, Z, Zg, Cm);
}

// Z[:, a] := Zg[:, a] for a < g (restore the determined columns after the QR completion).
__global__ void k_restore_cols(double2* Z, const double2* Zg, int rows, int r, int g) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < (int64_t)rows * r;
       k += (int64_t)gridDim.x * blockDim.x)
    if ((int)(k % r) < g) Z[k] = Zg[k];
}

void launch_restore_cols(double2* Z, const double2* Zg, int rows, int r, int g, cudaStream_t s) {
  const int64_t tot = (int64_t)rows * r;
  k_restore_cols<<<(int)std::min<int64_t>((tot + 255) / 256, 1024), 256, 0, s>>>(Z, Zg, rows, r, g);
}

// New node tensors of the pair (canonical leg order, bond of new rank r at
// leg lf of `first` and leg ls of `second`). The isometry side reads Z, the
// centre side Cm (layouts as written by k_svd_vecs).
__global__ void k_write_pair(double2* Uf, float2* Uf_lo, int f0, int f1, int f2, int lf, double2* Us, float2* Us_lo,
                             int s0, int s1, int s2, int ls, const double2* Z, const double2* Cm, int r, int iso_first) {
  const int fd[3] = {f0, f1, f2}, sd[3] = {s0, s1, s2};
  const int64_t nf = (int64_t)f0 * f1 * f2, ns = (int64_t)s0 * s1 * s2;
  int fa, fb, sa, sb;
  others(lf, fa, fb);
  others(ls, sa, sb);
  const int rows_f = fd[fa] * fd[fb], cols_s = sd[sa] * sd[sb];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nf + ns;
       k += (int64_t)gridDim.x * blockDim.x) {
    if (k < nf) {
      int id[3];
      id[0] = (int)(k / ((int64_t)f1 * f2));
      id[1] = (int)((k / f2) % f1);
      id[2] = (int)(k % f2);
      const int a = id[lf], row = id[fa] * fd[fb] + id[fb];
      const double2 v = iso_first ? Z[(int64_t)row * r + a] : Cm[(int64_t)row * r + a];
      Uf[k] = v;
      if (Uf_lo) Uf_lo[k] = make_float2((float)v.x, (float)v.y);
    } else {
      const int64_t kk = k - nf;
      int id[3];
      id[0] = (int)(kk / ((int64_t)s1 * s2));
      id[1] = (int)((kk / s2) % s1);
      id[2] = (int)(kk % s2);
      const int a = id[ls], col = id[sa] * sd[sb] + id[sb];
      const double2 v = iso_first ? Cm[(int64_t)a * cols_s + col] : Z[(int64_t)col * r + a];
      Us[kk] = v;
      if (Us_lo) Us_lo[kk] = make_float2((float)v.x, (float)v.y);
    }
  }
  (void)rows_f;
}

void launch_write_pair(double2* Uf, float2* Uf_lo, const int* fd, int lf, double2* Us, float2* Us_lo, const int* sd,
                       int ls, const double2* Z, const double2* Cm, int r, bool iso_first, cudaStream_t s) {
  const int64_t tot = (int64_t)fd[0] * fd[1] * fd[2] + (int64_t)sd[0] * sd[1] * sd[2];
  k_write_pair<<<(int)std::min<int64_t>((tot + 255) / 256, 2048), 256, 0, s>>>(
      Uf, Uf_lo, fd[0], fd[1], fd[2], lf, Us, Us_lo, sd[0], sd[1], sd[2], ls, Z, Cm, r, iso_first ? 1 : 0);
}

}  // namespace ttn
