// Device kernels of the TTN-HEOM library (sm_103a). Complex numbers are
// double2 (x = real, y = imaginary).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "plan.hpp"

namespace ttn {

// Device-side view of the job tables (all pointers into the workspace).
struct DevTables {
  double2* const* bufs;   // buffer id -> tensor base
  double2* const* mats;   // matrix id -> d x d matrix
  const ApTerm* terms;
  const ApOut* outs;
  const PjOut* pjs;
};

// Epilogue of the apply kernel. STORE writes each output to its dst buffer;
// RKs (s = 1..4) fuse the classical RK4 stage update of y with step h:
//   s=1: acc = k;      ys = y + h/2 k      s=3: acc += 2k; ys = y + h k
//   s=2: acc += 2k;    ys = y + h/2 k      s=4: y += h/6 (acc + k)
enum EpiMode : int { EPI_STORE = 0, EPI_RK1 = 1, EPI_RK2 = 2, EPI_RK3 = 3, EPI_RK4 = 4 };
struct Epi {
  int mode;
  int y, ys, acc;  // buffer ids
  double h;
};

// One time-dependent open-leg matrix: cur = stat + sum_d g_d * part_d.
constexpr int kMaxDrives = 8;
struct DriveMat {
  int d;
  int cur, stat;
  int part[kMaxDrives];  // matrix ids, -1 if the drive has no part here
};
struct DriveArgs {
  double g[kMaxDrives];
};

void launch_apply(const DevTables& T, const ApList& L, const Epi& e, cudaStream_t s);
void launch_project(const DevTables& T, const PjList& L, cudaStream_t s);
// Householder QR of node tensor U (dims d[3]) matricised toward leg `leg`.
// U is overwritten with Q (same layout), R (d_leg x d_leg, row-major) written to R.
// work: >= P complex, qbuf: >= P complex. A non-finite ||U||_F sets *flag and
// leaves U unchanged.
void launch_qr(double2* U, int d0, int d1, int d2, int leg, double tol, double2* work,
               double2* qbuf, double2* R, int* flag, cudaStream_t s);
// Cluster-parallel variant (qr.cu); returns false when the shape does not fit
// (bond dim > kQrClusterMaxN or the row blocks exceed shared memory).
constexpr int kQrClusterMaxN = 64;
bool launch_qr_cluster(double2* U, int d0, int d1, int d2, int leg, double tol, double2* R, int* flag,
                       cudaStream_t s);
void launch_copy(double2* dst, const double2* src, int64_t n, cudaStream_t s);
// rho / vector contraction for one node: out[a] (non-root) or out[i*d1+j] (root)
// = sum U[...] w1[.] w2[.] (w = nullptr means the n = 0 unit vector).
void launch_rdm_node(const double2* U, int d0, int d1, int d2, bool root, const double2* w1,
                     const double2* w2, double2* out, cudaStream_t s);
void launch_drive(double2* const* mats_dev, const DriveMat* list, int n, const DriveArgs& g,
                  cudaStream_t s);
void launch_check_finite(const double2* x, int64_t n, int* flag, cudaStream_t s);

}  // namespace ttn
