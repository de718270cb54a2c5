// Device kernels of the TTN-HEOM library (sm_103a). Complex numbers are
// double2 (x = real, y = imaginary).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "plan.hpp"

namespace ttn {

// Precision of the node/bond/environment contractions. The state (node
// tensors, bond matrices), RK4 accumulation, QR, absorb and RDM are FP64 in
// both modes; PREC_F32 runs the contractions in FP32 on FP32 shadow copies.
enum Prec : int { PREC_F64 = 0, PREC_F32 = 1 };

// Device-side view of the job tables. Element type of bufs/mats is the
// contraction type of the table (double2 or float2).
struct DevTables {
  void* const* bufs;   // buffer id -> tensor base
  void* const* mats;   // matrix id -> d x d matrix
  const ApTerm* terms;
  const ApOut* outs;
  const PjOut* pjs;
};

// q = a / b and r = a - q b for a >= 0, b > 0, in 32-bit arithmetic when both
// fit: a 64-bit integer division is a long instruction sequence on the GPU,
// and index decompositions sit in the inner loops of the gather, scatter and
// contraction kernels.
__device__ __forceinline__ int64_t idivmod(int64_t a, int64_t b, int64_t& r) {
  if (((a | b) >> 31) == 0) {
    const unsigned q = (unsigned)a / (unsigned)b;
    r = a - (int64_t)q * b;
    return q;
  }
  const int64_t q = a / b;
  r = a - q * b;
  return q;
}

// Output of a job list that holds output tile `tile` (tile0 ascending over the
// list): one division when all outputs have the same number of tiles (tpo),
// else a binary search -- a few dependent table loads instead of one per
// earlier output.
template <typename Out>
__device__ __forceinline__ int list_output(const Out* outs, int out_begin, int out_end, int tpo, int tile) {
  if (tpo > 0) return out_begin + tile / tpo;
  int lo = out_begin, hi = out_end - 1;  // the last output with tile0 <= tile
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (outs[mid].tile0 <= tile)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Epilogue of the apply kernel. STORE writes each output to its dst buffer;
// RKs (s = 1..4) fuse the classical RK4 stage update of the FP64 state y with
// step h (k = the computed sum, acc and y in FP64, ys in the contraction type):
//   s=1: acc = k;      ys = y + h/2 k      s=3: acc += 2k; ys = y + h k
//   s=2: acc += 2k;    ys = y + h/2 k      s=4: y += h/6 (acc + k), y_lo = y
enum EpiMode : int { EPI_STORE = 0, EPI_RK1 = 1, EPI_RK2 = 2, EPI_RK3 = 3, EPI_RK4 = 4 };
struct Epi {
  int mode;
  double2* y;    // FP64 state
  void* y_lo;    // contraction-type copy of y refreshed at s = 4 (== y in FP64 mode)
  void* ys;      // stage input (contraction type)
  double2* acc;  // FP64 stage accumulator
  double h;
};

// One time-dependent open-leg matrix: cur = stat + sum_d g_d * part_d.
constexpr int kMaxDrives = 8;
struct DriveMat {
  int d;
  int cur, stat;         // ids in the FP64 matrix table
  int part[kMaxDrives];  // FP64 matrix ids, -1 if the drive has no part here
};
struct DriveArgs {
  double g[kMaxDrives];
};

void launch_apply(int prec, const DevTables& T, const ApList& L, const Epi& e, cudaStream_t s);
// Allows the contraction and projection kernels clusters of up to kMaxSplit
// (16) CTAs; called once before the first launch.
void allow_wide_splits();

// Mixed form: the same list with its mode products on the tcgen05 tensor
// cores (tc_apply.cu, 3xTF32). outs_host/terms_host: host copies of the job
// tables; acc: FP32 scratch of acc_elems complex values (RK epilogue lists;
// one-output lists run their three legs in one launch when 3 planes of the
// output fit); flag bit 3 on a timed-out MMA wait. tc_applicable: 3-leg outputs, contracted
// legs of dimension <= 64, largest output >= 16384 elements.
// pool/pool_off (nullable): pre-split operator matrices (launch_tc_embed),
// pool_off[mat] the float offset of a matrix or -1 (staged by the threads).
bool tc_applicable(const ApList& L, const ApOut* outs_host, const ApTerm* terms_host);
// pool_off_host: host copy of pool_off. bsplit (nullable, bsplit_floats floats):
// buffer of the pre-split tensor operands; when every term of the list has a
// pre-split operator and the list's split operands fit (tc_split_floats), the
// tensor operands are split there first (k_tc_split) and both operands stream
// into a 4-stage ring by bulk copies (k_tc_apply_ring); otherwise the threads
// stage the tensor operand (k_tc_apply).
bool launch_apply_tc(const DevTables& T, const ApList& L, const Epi& e, const ApOut* outs_host,
                     const ApTerm* terms_host, float2* acc, int64_t acc_elems, int* flag, const float* pool,
                     const int64_t* pool_off, cudaStream_t s, const int64_t* pool_off_host = nullptr,
                     float* bsplit = nullptr, int64_t bsplit_floats = 0, bool* used_ring = nullptr);
// Floats of pre-split tensor operands a list needs on the ring path (0: not eligible).
int64_t tc_split_floats(const ApList& L, const ApOut* outs_host, const ApTerm* terms_host,
                        const int64_t* pool_off_host);
// Pre-split copies of FP32 operator matrices for the tensor-core path: for
// each job, matrix `mat` (d x d, d <= 64) of the FP32 matrix table is embedded
// and split into tf32 hi / lo in the layout the apply kernel stages, at float
// offset `off` of pool (tc_pool_floats(d) floats, 0 when d > 64).
struct TcEmbedJob {
  int mat, d;
  int64_t off;
};
constexpr int kTcEmbedBatch = 32;
struct TcEmbedBatch {
  int n;
  TcEmbedJob job[kTcEmbedBatch];
};
int64_t tc_pool_floats(int d);
void launch_tc_embed(void* const* mats32, const TcEmbedJob* jobs, int n, float* pool, cudaStream_t s);
void launch_project(int prec, const DevTables& T, const PjList& L, cudaStream_t s);
// The same projections for wide bonds in the FP32 form (every output d x d
// with d >= 32 and a reduction range of >= 1024 positions, all outputs of the
// list alike):
// shared-memory tiled, range split over a cluster. Returns false (nothing
// launched) when the list does not qualify or the launch fails.
bool launch_project_tiled(int prec, const DevTables& T, const PjList& L, int d, int64_t nrest, int sm_count,
                          cudaStream_t s);
// Householder QR of node tensor U (dims d[3]) matricised toward leg `leg`.
// U is overwritten with Q (same layout), R (d_leg x d_leg, row-major) written to R.
// work: >= P complex, qbuf: >= P complex. A non-finite ||U||_F sets *flag and
// leaves U unchanged. U_lo / R_lo (nullable) receive FP32 copies of Q and R.
// work_elems: capacity of work (the blocked path for tall matrices needs
// qr_blocked_elems(m, n) of it; otherwise P suffices). Tried in order: the
// cluster kernel (n <= 64, rows fit a cluster), the blocked path (n <= 64),
// the one-CTA kernel (any n).
// grid_wait_ns: bound of the grid barriers of the blocked path's panels over
// the whole GPU, counted from the panel kernel's start (the cluster kernel's
// exchanges keep a fixed 2 s: a CTA that gave up there could leave a peer's
// asynchronous store into its shared memory in flight).
void launch_qr(double2* U, int d0, int d1, int d2, int leg, double tol, double2* work, int64_t work_elems,
               double2* qbuf, double2* R, int* flag, float2* U_lo, float2* R_lo, cudaStream_t s,
               uint64_t grid_wait_ns = 2000000000ull);
// Cluster-parallel variant (qr.cu); returns false when the shape does not fit
// (bond dim > kQrClusterMaxN or the row blocks exceed shared memory).
constexpr int kQrClusterMaxN = 64;
// scratch/scratch_elems: global memory the kernel may use for its Gram / M
// buffers when shared memory cannot hold them (bond dimensions above ~40).
bool launch_qr_cluster(double2* U, int d0, int d1, int d2, int leg, double tol, double2* R, int* flag,
                       float2* U_lo, float2* R_lo, double2* scratch, int64_t scratch_elems, cudaStream_t s);
// Panel of the blocked QR (qr_blocked.cu): the cluster kernel factors columns
// [c0, c0+nb) of the column-major m x n matrix A over rows [c0, m) with the
// threshold *thr of the whole matrix (NaN: do nothing), writes V / R entries
// back in place, beta/alpha/phase/skip of those columns at index c0.., and the
// panel's WY factor T (nb x nb, row-major) with H_c0..H_{c0+nb-1} = I - V T V^H.
struct QrPanel {
  double2* gtail;  // full mode: global scratch (3*C*n*n) for the Gram / M buffers, or null
  double2* A;
  int m, n, c0, nb;
  const double* thr;
  double* beta;
  double* alpha;
  double2* phase;
  int* skip;
  double2* T;
};
constexpr int kQrPanelMaxNb = 16;
bool launch_qr_panel(const QrPanel& pn, cudaStream_t s);
int qr_panel_cluster(int m_act, int nb);  // cluster size of a panel, 0 if it does not fit
// Blocked Householder QR for matrices the cluster kernel cannot hold; same
// convention and result as launch_qr. Panels run over the whole GPU (a
// cooperative launch, bounded waits -> bit 2 of *flag) where the device
// supports it, else on one cluster. work needs qr_blocked_elems(m, n)
// complex values; returns false (nothing launched) when it does not apply.
int64_t qr_blocked_elems(int64_t m, int64_t n);
bool launch_qr_blocked(double2* U, int d0, int d1, int d2, int leg, double tol, double2* work,
                       int64_t work_elems, double2* qbuf, double2* R, int* flag, float2* U_lo, float2* R_lo,
                       cudaStream_t s, uint64_t grid_wait_ns = 2000000000ull);
// dst = src (FP64); dst_lo (nullable) = FP32 copy.
void launch_copy(double2* dst, float2* dst_lo, const double2* src, int64_t n, cudaStream_t s);
// rho / vector contraction for one node: out[a] (non-root) or out[i*d1+j] (root)
// = sum U[...] w1[.] w2[.] (w = nullptr means the n = 0 unit vector).
void launch_rdm_node(const double2* U, int d0, int d1, int d2, bool root, const double2* w1,
                     const double2* w2, double2* out, cudaStream_t s);
// cur = stat + sum_d g_d part_d in the FP64 table; mats32 (nullable) receives
// the FP32 copy of cur (same matrix id in the FP32 table).
void launch_drive(double2* const* mats_dev, float2* const* mats32, const DriveMat* list, int n,
                  const DriveArgs& g, cudaStream_t s);
void launch_check_finite(const double2* x, int64_t n, int* flag, cudaStream_t s);

// ps2 two-site kernels (ps2.cu), FP64. fd/sd: dims of the first/second node,
// lf/ls: the leg of each facing the other.
void launch_merge(const double2* Uf, const int* fd, int lf, const double2* Us, const int* sd, int ls,
                  double2* theta, float2* theta_lo, cudaStream_t s);
// One-sided Jacobi SVD of theta (m x n row-major). A: >= m*n, V: >= min(m,n)^2,
// sigma: min(m,n) (unsorted), info[0] = sweeps, info[1] = 1 if Theta^H was used.
void launch_jacobi_svd(const double2* theta, int m, int n, double2* A, double2* V, double* sigma, int* info,
                       cudaStream_t s);
// Convergence threshold of both Jacobi kernels: |x^H y| > tol |x| |y| rotates,
// tol = 2 sqrt(max(rows, 64)) DBL_EPSILON (above the rounding noise of the
// summed Gram entries); a run that reaches kJacMaxSweeps is not converged.
double jacobi_tol(int m, int n);
// A column whose squared norm is at most 16 rows eps^2 ||A||_F^2 is rounding
// noise of the matrix (an exactly dependent column leaves one after its
// rotation); rotating it against the others would go on forever, each rotation
// only shrinking the noise. Such pairs are not rotated: the singular values
// they leave are below sqrt(16 rows) eps ||A||_F, far under the svd_tol
// cut that replaces them by the deterministic completion.
__host__ __device__ inline double jacobi_negligible(int rows, double fro2) {
  return 16.0 * rows * 2.220446049250313e-16 * 2.220446049250313e-16 * fro2;
}
constexpr int kJacMaxSweeps = 60;

// Rotation of one column pair of the one-sided Jacobi SVD from its Gram
// entries a = |x|^2, b = |y|^2 and c = x^H y = cr + i ci. Returns false when
// the pair is left alone: |c|^2 <= tol^2 a b (orthogonal to working accuracy),
// c = 0, or a column is rounding noise (min(a, b) <= tiny2, jacobi_negligible).
// Otherwise the complex rotation
//     x' = cs x - sn e y,   y' = sn x + cs e y,   e = conj(c) / |c|
// makes the pair orthogonal; t = sn / cs is the root of smaller modulus of
// t^2 + 2 zeta t - 1 = 0, zeta = (b - a) / (2 |c|), i.e. with d = b - a,
//     r = sqrt(d^2 + 4 |c|^2),  u = |d| + r,  t = sign(d) 2|c| / u,
// and cs = 1 / sqrt(1 + t^2) = u w, sn = t cs = sign(d) 2|c| w with
// w = 1 / sqrt(u^2 + 4 |c|^2): no quotient, and the dependent chain is one
// square root and one reciprocal square root (1/|c| is taken beside r).
__device__ __forceinline__ bool jacobi_rotation(double a, double b, double cr, double ci, double tol, double tiny2,
                                                double& cs, double& sn, double2& e) {
  const double c2 = cr * cr + ci * ci;
  if (!(c2 > tol * tol * a * b) || c2 == 0.0 || !(fmin(a, b) > tiny2)) return false;
  const double d = b - a;
  const double ic = rsqrt(c2);  // 1 / |c|
  const double r = sqrt(fma(d, d, 4.0 * c2));
  const double u = fabs(d) + r;
  const double w = rsqrt(fma(u, u, 4.0 * c2));
  const double ac2 = 2.0 * (c2 * ic);  // 2 |c|
  cs = u * w;
  sn = d >= 0.0 ? ac2 * w : -ac2 * w;
  e = make_double2(cr * ic, -ci * ic);
  return true;
}

// Sums of four per-lane values over a warp in a fixed order (reduce-scatter:
// 6 additions instead of 20). On return lanes 0-7 hold the sum of v0, lanes
// 8-15 of v1, lanes 16-23 of v2 and lanes 24-31 of v3.
__device__ __forceinline__ double warp_sum4(double v0, double v1, double v2, double v3) {
  const int lane = threadIdx.x & 31;
  const bool hi = (lane & 16) != 0;
  double k0 = hi ? v2 : v0, k1 = hi ? v3 : v1;
  const double s0 = hi ? v0 : v2, s1 = hi ? v1 : v3;
  k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
  k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
  const bool h8 = (lane & 8) != 0;
  double k = h8 ? k1 : k0;
  k += __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, 8);
  for (int o = 4; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
  return k;
}
// The same SVD spread over several CTAs (svd.cu): pairs of a circle-method
// round dealt to the CTAs, one barrier per round -- the hardware barrier of
// one thread-block cluster for up to 2 * kJacClusterMax columns, else a grid
// barrier of one cooperative launch. Used when the smaller side has more than
// kJacOneCtaMaxCols columns (else the one-CTA kernel). sync: kSvdSyncInts device
// ints (cleared by the launch); a grid wait longer than wait_ns sets bit 4 (16)
// of *flag. Same outputs as launch_jacobi_svd.
constexpr int kJacOneCtaMaxCols = 16;
constexpr int kJacClusterMax = 16;
constexpr int kSvdSyncInts = 128;
bool launch_jacobi_svd_grid(const double2* theta, int m, int n, double2* A, double2* V, double* sigma, int* info,
                            unsigned* sync, int* flag, uint64_t wait_ns, cudaStream_t s);
void launch_svd_vecs(const double2* A, const double2* V, const double* sigma, int m, int n, const int* perm, int r,
                     int g, bool iso_first, double2* Z, double2* Zg, double2* Cm, cudaStream_t s);
void launch_restore_cols(double2* Z, const double2* Zg, int rows, int r, int g, cudaStream_t s);
// rank-proposer network and the randomised factorisation (mlp.cu)
size_t mlp_ws_floats(int B);
void launch_mlp_forward(const float* P, const float* x, int B, float* ws, float* logits, cudaStream_t s);
void launch_gauss(double2* O, int64_t n, uint64_t seed, cudaStream_t s);
void launch_zgemm(const double2* A, const double2* B, double2* C, int M, int N, int K, bool conjA, cudaStream_t s);
void launch_norm2(const double2* x, int64_t n, double* out, cudaStream_t s);
void launch_rsvd_vecs(const double2* Q, int m, int kk, const double2* A, const double2* V, const double* sigma, int n,
                      const int* perm, int r, int g, bool iso_first, double2* Z, double2* Zg, double2* Cm,
                      cudaStream_t s);
void launch_write_pair(double2* Uf, float2* Uf_lo, const int* fd, int lf, double2* Us, float2* Us_lo, const int* sd,
                       int ls, const double2* Z, const double2* Cm, int r, bool iso_first, cudaStream_t s);

// Direct integration (vmf.cu), FP64. launch_vmf_edge: on edge p -> c with the
// QR factor R (r x r, row-major) of the upper part and the class matrices at
// slots_dev[0..n_classes) (isometric environments on entry): rho = R^H R,
// rho_reg = rho + eps 1, E~ = rho_reg^-1 R^H E R in place, dmi = rho_reg^-1 rho - 1.
// aug: 3 r^2, tmp: 2 r^2 per class. launch_vmf_finish: K (node derivative, r x
// nc, row-major over the parent index) += dmi G_down, then K := (1 - P) K with
// P the projector onto the rows of U (X: r^2 scratch).
void launch_vmf_edge(double2* const* mats_dev, const int* slots_dev, int n_classes, const double2* R, int r,
                     double eps, double2* aug, double2* dmi, double2* tmp, cudaStream_t s);
void launch_vmf_finish(double2* K, const double2* Gdown, const double2* dmi, const double2* U, int r, int64_t nc,
                       double2* X, cudaStream_t s);
// out = y + sum_l c[l] K[l] (flat), and the embedded-pair error
// sum |sum_l c[l] K[l]|^2 / (atol + rtol max(|y|, |y5|))^2 into *out (block
// partials in part, 1024 doubles, added in order).
struct VmfComb {
  int n;
  double c[7];
  const double2* K[7];
};
void launch_vmf_stage(double2* out, const double2* y, const VmfComb& cb, int64_t n, cudaStream_t s);
void launch_vmf_err(const double2* y, const double2* y5, const VmfComb& cb, double rtol, double atol, int64_t n,
                    double* part, double* out, cudaStream_t s);

}  // namespace ttn
