// C ABI of the TTN-HEOM library (include/ttn_heom.h): handle, workspace layout
// and the host-side sweep executor that issues the kernels of kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <exception>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/ttn_heom.h"
#include "kernels.cuh"
#include "plan.hpp"

using namespace ttn;

namespace {

struct DriveSlot {
  ttn_drive_fn fn = nullptr;
  void* user = nullptr;
  double bound = 1.0;
};

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

}  // namespace

struct ttn_ctx {
  Plan plan;
  int precision = TTN_FP64;
  ttn_params params{1e-9, 2.5, 1e-7, 2.0, 32, 1e-12, kMaxSplit, 1, 2.0, 1e-5, 1e-7, 1e-10, 0};
  bool sop_loaded = false;
  bool ws_bound = false;
  bool envs_dirty = true;
  std::vector<DriveSlot> drives;
  cudaStream_t stream = nullptr;
  std::string err;
  double t = 0.0;

  // workspace
  char* ws = nullptr;
  size_t ws_bytes = 0;
  std::vector<double2*> h_bufs;  // FP64 device addresses per buffer id
  std::vector<double2*> h_mats;  // FP64 device addresses per matrix id
  std::vector<void*> h_bufs_lo;  // contraction-type addresses (== h_bufs in FP64 mode)
  std::vector<void*> h_mats_lo;
  double2* pool = nullptr;
  int prec = PREC_F64;
  double2* qr_work = nullptr;
  int64_t qr_elems = 0;
  float2* tc_acc = nullptr;  // FP32 scratch of the tensor-core path (mixed form)
  float* tc_bsplit = nullptr;  // pre-split tensor operands of the tensor-core ring kernel
  int64_t tc_bsplit_floats = 0;
  int64_t tc_acc_elems = 0;  // its capacity: three node-sized leg planes
  // pre-split operator matrices of the tensor-core path: on when some job list
  // was tensor-core eligible at bind time; every writer of those matrices
  // then refreshes their pool copies
  bool tc_pool_on = false;
  float* tc_pool = nullptr;
  int64_t* tc_off_dev = nullptr;
  std::vector<int64_t> tc_off;
  // ps2 scratch
  double2 *svd_A = nullptr, *svd_V = nullptr, *svd_Z = nullptr, *svd_Zg = nullptr, *svd_C = nullptr;
  double* svd_sigma = nullptr;
  int* svd_perm = nullptr;
  int* svd_info = nullptr;
  unsigned* svd_sync = nullptr;  // barrier counters of the grid Jacobi SVD
  // direct integration (vmf), FP64 form only
  double2 *vmf_y = nullptr, *vmf_save = nullptr, *vmf_tmp = nullptr, *vmf_r = nullptr, *vmf_aug = nullptr,
          *vmf_dmi = nullptr, *vmf_x = nullptr, *vmf_ctmp = nullptr;
  double2* vmf_k[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int* vmf_slots = nullptr;
  double* vmf_err = nullptr;
  int64_t vmf_n = 0;                 // complex elements of the flat node region
  std::vector<int64_t> node_off, vmf_r_off;
  std::vector<int> vmf_slot_off;
  double vmf_h = 0.0;                // dopri5 trial step carried between calls
  int64_t vmf_acc = 0, vmf_rej = 0;  // dopri5 steps accepted / rejected
  bool mix_switched = false;         // TTN_MIX: ps2 phase over
  std::vector<double> discarded;  // discarded weight of every ps2 split (host log)
  std::vector<int> init_ranks;
  // learned rank proposer
  const float* proposer = nullptr;  // device parameters (caller-owned), nullptr = off
  int64_t n_proposed = 0, n_accepted = 0;
  std::vector<float> log_feats;     // split records: 24 features each
  std::vector<int32_t> log_labels;  // class = clamp(r_svd - r_cur, -4, 8) + 4
  std::vector<std::vector<double>> edge_sig;   // per child node: last normalised spectrum (top 16)
  std::vector<std::vector<double>> edge_disc;  // per child node: last discarded weights (newest first)
  double2 *rs_omega = nullptr, *rs_Y = nullptr, *rs_B = nullptr;
  float *mlp_x = nullptr, *mlp_ws = nullptr, *mlp_logits = nullptr;
  double* rs_norm = nullptr;
  uint64_t n_splits = 0;
  double2* rdm_vec = nullptr;
  double2* rho_dev = nullptr;
  int* flag_dev = nullptr;
  DriveMat* drive_list_dev = nullptr;
  std::vector<DriveMat> drive_list;
  std::vector<int64_t> rdm_off;  // per node offset into rdm_vec
  DevTables T{};    // FP64 table (absorb; everything in FP64 mode)
  DevTables Tlo{};  // contraction table (== T in FP64 mode)

  // kernel accounting (ttn_stats / ttn_profile)
  int64_t n_launch[4] = {0, 0, 0, 0};
  int64_t n_ring = 0;  // job lists issued on the tensor-core ring path (counted at issue, ttn_stats kind 4)
  double n_flops[4] = {0, 0, 0, 0};
  bool profiling = false;  // per-launch events (mode 1) or event nodes in the step graph (mode 2)
  int prof_mode = 0;
  bool capturing = false;   // inside ensure_graph's stream capture
  int graph_prof = 0;       // prof_mode the current step graph was captured with
  struct Mark {
    int kind;
    cudaEvent_t a, b;
  };
  static_assert(sizeof(Mark) > 0, "");
  std::vector<cudaEvent_t> ev_free;
  std::vector<Mark> marks;
  double prof_ms[4] = {0, 0, 0, 0};

  // one ps1 step captured as a CUDA graph (autonomous generators, non-default stream)
  cudaGraphExec_t graph = nullptr;
  cudaGraph_t graph_src = nullptr;  // kept for composition by ttn_batch_step
  double graph_dt = 0.0;
  bool graph_disabled = false;
  int64_t graph_launch[4] = {0, 0, 0, 0};
  double graph_flops[4] = {0, 0, 0, 0};
  // batch graph owned by the first handle of the last ttn_batch_step call
  cudaGraphExec_t batch_exec = nullptr;
  std::vector<ttn_ctx*> batch_members;
  std::vector<cudaGraphExec_t> batch_member_graphs;
  double batch_dt = 0.0;
  void drop_batch() {
    if (batch_exec) cudaGraphExecDestroy(batch_exec);
    batch_exec = nullptr;
    batch_members.clear();
    batch_member_graphs.clear();
  }
  void drop_graph() {
    if (graph) cudaGraphExecDestroy(graph);
    if (graph_src) cudaGraphDestroy(graph_src);
    graph = nullptr;
    graph_src = nullptr;
    for (auto& m : graph_marks) {
      ev_free.push_back(m.a);
      ev_free.push_back(m.b);
    }
    graph_marks.clear();
  }
  // event pairs recorded by every replay of the step graph (profile mode 2)
  std::vector<struct Mark> graph_marks;
  // after a replay: fold the graph's event pairs into prof_ms
  cudaError_t read_graph_marks() {
    if (graph_marks.empty()) return cudaSuccess;
    cudaError_t err = cudaEventSynchronize(graph_marks.back().b);
    if (err != cudaSuccess) return err;
    for (auto& m : graph_marks) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess) prof_ms[m.kind] += ms;
    }
    return cudaSuccess;
  }

  ~ttn_ctx() {
    // the caller frees the workspace once ttn_destroy returns: nothing queued on
    // the handle's stream may still touch it (a step that failed part-way can
    // leave launches behind)
    if (stream) cudaStreamSynchronize(stream);
    drop_batch();
    drop_graph();
    for (auto& m : marks) {
      cudaEventDestroy(m.a);
      cudaEventDestroy(m.b);
    }
    for (auto e : ev_free) cudaEventDestroy(e);
  }
  cudaEvent_t get_event() {
    if (!ev_free.empty()) {
      cudaEvent_t e = ev_free.back();
      ev_free.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  // synchronise and fold recorded event pairs into prof_ms
  cudaError_t drain_marks() {
    if (marks.empty()) return cudaSuccess;
    cudaError_t err = cudaEventSynchronize(marks.back().b);
    if (err != cudaSuccess) return err;
    for (auto& m : marks) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess) prof_ms[m.kind] += ms;
      ev_free.push_back(m.a);
      ev_free.push_back(m.b);
    }
    marks.clear();
    return cudaSuccess;
  }

  ttn_status fail(ttn_status s, const std::string& m) {
    err = m;
    return s;
  }
};

namespace {

ttn_status cuda_fail(ttn_t h, cudaError_t e, const char* what) {
  return h->fail(TTN_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CUDA_TRY(h, call)                                   \
  do {                                                      \
    cudaError_t _e = (call);                                \
    if (_e != cudaSuccess) return cuda_fail(h, _e, #call);  \
  } while (0)

// ---------------------------------------------------------------------------
// Workspace layout
// ---------------------------------------------------------------------------
struct Layout {
  size_t nodes, pool, scratch, qr, rdm, rho, bufs_tab, mats_tab, terms, outs, pjs, drives, flag, total;
  size_t nodes32 = 0, pool32 = 0, scratch32 = 0, bufs_tab_lo = 0, mats_tab_lo = 0, tc_acc = 0, tc_bsplit = 0;
  int64_t tc_bsplit_floats = 0;  // FP32 mode only
  size_t tc_pool = 0, tc_off = 0;
  std::vector<int64_t> tc_off_host;  // float offset of each matrix in tc_pool, -1 if none
  size_t svd_small = 0, rsvd = 0, mlp = 0;
  // direct integration (vmf): committed state, per-node saves, 7 stage
  // derivatives (all as flat copies of the node region), edge scratch
  size_t vmf_y = 0, vmf_save = 0, vmf_k = 0, vmf_tmp = 0, vmf_r = 0, vmf_aug = 0, vmf_dmi = 0, vmf_x = 0,
         vmf_ctmp = 0, vmf_slots = 0, vmf_err = 0;
  int64_t nodes_elems = 0;
  std::vector<int64_t> vmf_r_off;   // complex offset of each bond's R in vmf_r
  std::vector<int> vmf_slot_off;    // offset of each directed edge's class slots in vmf_slots
  std::vector<int> vmf_slot_host;   // the class slots themselves
  std::vector<int64_t> node_off;  // complex elements from `nodes`
  std::vector<int64_t> rdm_off;
  int64_t scratch_elems = 0, qr_elems = 0, rdm_elems = 0;
};

Layout layout_of(const Plan& p, int prec) {
  Layout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += align_up(std::max<size_t>(bytes, 1));
    return o;
  };
  const int n = p.tree.n_nodes;
  L.node_off.resize(n);
  int64_t acc = 0;
  for (int u = 0; u < n; ++u) {
    L.node_off[u] = acc;
    acc += (p.P_cap[u] + 15) / 16 * 16;
  }
  const int64_t S = std::max(p.P_cap_max, p.theta_cap);  // node-sized scratch capacity
  L.nodes = take(acc * sizeof(double2));
  L.pool = take(std::max<int64_t>(p.mat_pool, 1) * sizeof(double2));
  const int64_t r2 = (int64_t)p.r_cap_max * p.r_cap_max;
  const int64_t nP = (int64_t)(4 + p.buf.n_t + p.buf.n_w) * S;
  L.scratch_elems = nP + 4 * r2 + 4 * p.theta_cap + 5 * p.theta_cap;
  L.scratch = take(L.scratch_elems * sizeof(double2));
  // QR scratch: the one-CTA kernel needs S; the blocked path for tall
  // matricisations (m x n, m*n <= S, n <= r_cap_max) needs its own layout
  L.qr_elems = S;
  for (int u = 0; u < n; ++u)
    for (int l = 0; l < 3; ++l) {
      const int64_t nn = p.cap_dims[u][l];
      if (nn < 1 || nn > kQrClusterMaxN) continue;
      L.qr_elems = std::max<int64_t>(L.qr_elems, qr_blocked_elems(p.P_cap[u] / nn, nn));
    }
  L.qr = take(L.qr_elems * sizeof(double2));
  L.rdm_off.resize(n);
  int64_t ra = 0;
  for (int u = 0; u < n; ++u) {
    L.rdm_off[u] = ra;
    ra += p.cap_dims[u][0];
  }
  L.rdm_elems = ra;
  L.rdm = take(ra * sizeof(double2));
  L.rho = take((size_t)p.leg_dims[0] * p.leg_dims[0] * sizeof(double2));
  L.bufs_tab = take(p.buf.n_bufs * sizeof(double2*));
  L.mats_tab = take(p.mats.size() * sizeof(double2*));
  L.terms = take(p.ap_terms.size() * sizeof(ApTerm));
  L.outs = take(p.ap_outs.size() * sizeof(ApOut));
  L.pjs = take(p.pj_outs.size() * sizeof(PjOut));
  L.drives = take(p.locals.size() * sizeof(DriveMat));
  L.svd_small = take(p.theta_cap * sizeof(double) + (p.theta_cap + 4 + kSvdSyncInts) * sizeof(int));
  L.rsvd = take(3 * p.theta_cap * sizeof(double2));
  L.mlp = take((24 + 13 + mlp_ws_floats(1) + 8) * sizeof(float) + 2 * sizeof(double));
  L.flag = take(sizeof(int) * 4);
  if (prec == PREC_F64) {
    L.nodes_elems = acc;
    L.vmf_y = take(acc * sizeof(double2));
    L.vmf_save = take(acc * sizeof(double2));
    L.vmf_k = take(7 * acc * sizeof(double2));
    L.vmf_tmp = take(p.P_cap_max * sizeof(double2));
    L.vmf_r_off.assign(n, 0);
    int64_t ro = 0;
    int max_cls = 0;
    for (int c = 1; c < n; ++c) {
      L.vmf_r_off[c] = ro;
      ro += (int64_t)p.caps[c] * p.caps[c];
    }
    L.vmf_r = take(std::max<int64_t>(ro, 1) * sizeof(double2));
    const int64_t r2 = (int64_t)p.r_cap_max * p.r_cap_max;
    L.vmf_aug = take(3 * r2 * sizeof(double2));
    L.vmf_dmi = take(r2 * sizeof(double2));
    L.vmf_x = take(r2 * sizeof(double2));
    L.vmf_slot_off.assign(2 * n + 1, 0);
    for (int e = 0; e < 2 * n; ++e) {
      L.vmf_slot_off[e] = (int)L.vmf_slot_host.size();
      for (int sl : p.dir_slots[e]) L.vmf_slot_host.push_back(sl);
      max_cls = std::max(max_cls, (int)p.dir_slots[e].size());
    }
    L.vmf_slot_off[2 * n] = (int)L.vmf_slot_host.size();
    L.vmf_ctmp = take(std::max<int64_t>(2 * r2 * max_cls, 1) * sizeof(double2));
    L.vmf_slots = take(std::max<size_t>(L.vmf_slot_host.size(), 1) * sizeof(int));
    L.vmf_err = take(1025 * sizeof(double));
  }
  if (prec == PREC_F32) {
    L.nodes32 = take(acc * sizeof(float2));
    L.pool32 = take(std::max<int64_t>(p.mat_pool, 1) * sizeof(float2));
    // ys, T_g, W_c and the bond shadow / stage input in FP32
    L.scratch32 = take(((int64_t)(2 + p.buf.n_t + p.buf.n_w) * S + 3 * r2 + 3 * p.theta_cap) * sizeof(float2));
    L.bufs_tab_lo = take(p.buf.n_bufs * sizeof(void*));
    L.tc_acc = take(3 * S * sizeof(float2));
    // pre-split copies of the operator matrices the job lists use (not the bond matrix)
    L.tc_off_host.assign(p.mats.size(), -1);
    std::vector<char> used(p.mats.size(), 0);
    for (const ApTerm& t : p.ap_terms)
      if (t.mat >= 0) used[t.mat] = 1;
    int64_t pf = 0;
    for (size_t i = 0; i < p.mats.size(); ++i) {
      if (!used[i] || (int)i == p.bond_mat) continue;
      const int64_t f = tc_pool_floats(p.mats[i].d);
      if (f == 0) continue;
      L.tc_off_host[i] = pf;
      pf += f;
    }
    L.tc_pool = take(std::max<int64_t>(pf, 1) * sizeof(float));
    L.tc_off = take(p.mats.size() * sizeof(int64_t));
    // pre-split tensor operands of the ring kernel: the largest need of a
    // tensor-core list (the lists run one after another on the stream)
    for (const ApList& al : p.ap_lists)
      if (al.n_tiles > 0 && tc_applicable(al, p.ap_outs.data(), p.ap_terms.data()))
        L.tc_bsplit_floats =
            std::max(L.tc_bsplit_floats, tc_split_floats(al, p.ap_outs.data(), p.ap_terms.data(), L.tc_off_host.data()));
    L.tc_bsplit = take(std::max<int64_t>(L.tc_bsplit_floats, 1) * sizeof(float));
    L.mats_tab_lo = take(p.mats.size() * sizeof(void*));
  }
  L.total = off;
  return L;
}

// ---------------------------------------------------------------------------
// Executor: the ps1 sweep of the oracle, issued as kernels on h->stream
// ---------------------------------------------------------------------------
struct Exec {
  ttn_t h;
  Plan& p;
  cudaStream_t s;
  explicit Exec(ttn_t hh) : h(hh), p(hh->plan), s(hh->stream) {}

  // account one kernel launch of class `kind` and, when profiling, bracket it
  // with CUDA events on the handle's stream
  template <typename F>
  void run(int kind, double flops, F&& launch) {
    if (err != cudaSuccess || fail_st != TTN_OK) return;  // a failed step launches nothing more
    h->n_launch[kind] += 1;
    h->n_flops[kind] += flops;
    if (h->prof_mode == 0) {
      launch();
      return;
    }
    cudaEvent_t a = h->get_event(), b = h->get_event();
    if (h->capturing) {  // profile mode 2: event-record nodes inside the step graph
      cudaEventRecordWithFlags(a, s, cudaEventRecordExternal);
      launch();
      cudaEventRecordWithFlags(b, s, cudaEventRecordExternal);
      h->graph_marks.push_back({kind, a, b});
      return;
    }
    cudaEventRecord(a, s);
    launch();
    cudaEventRecord(b, s);
    h->marks.push_back({kind, a, b});
    if (h->marks.size() > 100000) h->drain_marks();
  }
  void apply(int kind, int list, const Epi& e) {
    if (list < 0) return;
    const ApList& L = p.ap_lists[list];
    if (h->prec == PREC_F32 && h->params.tensor_cores && h->tc_acc &&
        tc_applicable(L, p.ap_outs.data(), p.ap_terms.data())) {
      run(kind, L.flops, [&] {
        const bool ring = h->params.tensor_cores == 2;  // 1: thread-staged tensor operand
        bool used_ring = false;
        if (!launch_apply_tc(h->Tlo, L, e, p.ap_outs.data(), p.ap_terms.data(), h->tc_acc, h->tc_acc_elems, h->flag_dev,
                             h->tc_pool_on ? h->tc_pool : nullptr, h->tc_pool_on ? h->tc_off_dev : nullptr, s,
                             h->tc_off.data(), ring ? h->tc_bsplit : nullptr, ring ? h->tc_bsplit_floats : 0,
                             &used_ring))
          launch_apply(h->prec, h->Tlo, L, e, s);
        if (used_ring) ++h->n_ring;
      });
      return;
    }
    run(kind, L.flops, [&] { launch_apply(h->prec, h->Tlo, L, e, s); });
  }
  void store(int kind, int list) { apply(kind, list, Epi{EPI_STORE, nullptr, nullptr, nullptr, nullptr, 0.0}); }

  void env(int a, int b) {
    const EnvLists& E = p.env[p.dir_id(a, b)];
    store(1, E.first);
    store(1, E.classes);
    if (E.project >= 0) {
      const PjList& L = p.pj_lists[E.project];
      // wide bonds: the tiled kernel (all classes of one edge share U and its dims)
      const PjOut& q = p.pj_outs[L.out_begin];
      const int dq = q.leg == 0 ? q.d0 : q.leg == 1 ? q.d1 : q.d2;
      const int64_t nrest = (int64_t)q.d0 * q.d1 * q.d2 / dq;
      run(1, L.flops, [&] {
        if (!launch_project_tiled(h->prec, h->Tlo, L, dq, nrest, p.sm_count, s)) launch_project(h->prec, h->Tlo, L, s);
      });
      if (h->tc_pool_on) {
        const int d = p.dims[a][p.tree.leg_index(a, b)];  // current rank of the bond
        std::vector<TcEmbedJob> jobs;
        for (int slot : p.dir_slots[p.dir_id(a, b)])
          if (slot >= 0 && h->tc_off[slot] >= 0) jobs.push_back(TcEmbedJob{slot, d, h->tc_off[slot]});
        run(1, 0.0, [&] { launch_tc_embed(h->Tlo.mats, jobs.data(), (int)jobs.size(), h->tc_pool, s); });
      }
    }
  }
  // U_u := Q (semi-unitary toward neighbour v), R -> bond buffer
  void qr(int u, int v) {
    const int li = p.tree.leg_index(u, v);
    const auto& d = p.dims[u];
    const double n = d[li], m = (double)p.P[u] / n;
    // Householder factorisation + explicit Q: 2 (2 m n^2 - 2 n^3 / 3) complex MACs
    const double flops = 8.0 * 2.0 * (2.0 * m * n * n - 2.0 * n * n * n / 3.0);
    run(2, flops, [&] {
      launch_qr(h->h_bufs[u], d[0], d[1], d[2], li, h->params.qr_tol, h->qr_work, h->qr_elems,
                h->h_bufs[p.buf.tmp], h->h_bufs[p.buf.bond_y], h->flag_dev, lo_copy(u), lo_copy(p.buf.bond_y), s,
                wait_ns());
    });
  }
  // FP32 shadow of an FP64 buffer (nullptr in FP64 mode, where they coincide)
  float2* lo_copy(int buf) { return h->prec == PREC_F32 ? (float2*)h->h_bufs_lo[buf] : nullptr; }
  // U_v := R x_(leg of v facing u) U_v, in FP64 (a gauge move), shadow refreshed
  void absorb(int v, int u) {
    const int li = p.tree.leg_index(v, u);
    const ApList& L = p.ap_lists[p.absorb[v][li]];
    run(3, L.flops, [&] {
      launch_apply(PREC_F64, h->T, L, Epi{EPI_STORE, nullptr, nullptr, nullptr, nullptr, 0.0}, s);
    });
    run(3, 0.0, [&] { launch_copy(h->h_bufs[v], lo_copy(v), h->h_bufs[p.buf.tmp], p.P[v], s); });
  }
  // Stage inputs alternate between two buffers: stage 1 reads y and writes A,
  // stage 2 reads A and writes B, stage 3 reads B and writes A, stage 4 reads A
  // and updates y. A kernel never writes the buffer it reads.
  void rk4(const FlowLists& F, int y, int ysA, int ysB, int acc, double tau) {
    const int m = p.n_sub(tau, h->params.kappa);
    const double hs = tau / m;
    static const int src_var[5] = {0, 0, 1, 2, 1};
    for (int sub = 0; sub < m; ++sub)
      for (int st = 1; st <= 4; ++st) {
        const int var = src_var[st];
        const int dst = st == 2 ? ysB : ysA;  // stage input written by this stage (unused at st = 4)
        store(0, F.first[var]);
        apply(0, F.combine[var], Epi{st, h->h_bufs[y], h->h_bufs_lo[y], h->h_bufs_lo[dst], h->h_bufs[acc], hs});
      }
  }
  void node_flow(int u, double tau) { rk4(p.node_flow[u], u, p.buf.ys, p.buf.ys2, p.buf.acc, tau); }
  void bond_flow(int a, int b, double tau) {
    rk4(p.bond_flow[p.dir_id(a, b)], p.buf.bond_y, p.buf.bond_ys, p.buf.bond_ys2, p.buf.bond_acc, tau);
  }

  // Lie-Trotter half sweep Phi_h(u) and its adjoint (see oracle/ttn.py)
  void phi(int u, double hh, bool flow_u) {
    for (int c : p.tree.children[u]) {
      qr(u, c);
      absorb(c, u);
      env(u, c);
      phi(c, hh, true);
      qr(c, u);
      env(c, u);
      bond_flow(c, u, -hh);
      absorb(u, c);
    }
    if (flow_u) node_flow(u, hh);
  }
  void phi_adj(int u, double hh, bool flow_u) {
    if (flow_u) node_flow(u, hh);
    const auto& ch = p.tree.children[u];
    for (auto it = ch.rbegin(); it != ch.rend(); ++it) {
      const int c = *it;
      qr(u, c);
      env(u, c);
      bond_flow(u, c, -hh);
      absorb(c, u);
      phi_adj(c, hh, true);
      qr(c, u);
      env(c, u);
      absorb(u, c);
    }
  }
  void drive(double t) {
    if (h->drive_list.empty()) return;
    DriveArgs g{};
    for (size_t d = 0; d < h->drives.size() && d < (size_t)kMaxDrives; ++d)
      g.g[d] = h->drives[d].fn ? h->drives[d].fn(t, h->drives[d].user) : 0.0;
    float2* const* m32 = h->prec == PREC_F32 ? (float2* const*)h->Tlo.mats : nullptr;
    run(3, 0.0, [&] {
      launch_drive((double2* const*)h->T.mats, m32, h->drive_list_dev, (int)h->drive_list.size(), g, s);
    });
    if (h->tc_pool_on) {
      std::vector<TcEmbedJob> jobs;
      for (const DriveMat& dm : h->drive_list)
        if (h->tc_off[dm.cur] >= 0) jobs.push_back(TcEmbedJob{dm.cur, dm.d, h->tc_off[dm.cur]});
      run(3, 0.0, [&] { launch_tc_embed(h->Tlo.mats, jobs.data(), (int)jobs.size(), h->tc_pool, s); });
    }
  }
  void step_ps1(double dt, double t0) {
    const double hh = 0.5 * dt;
    if (p.n_drives == 0) {
      phi(0, hh, false);
      node_flow(0, dt);
      phi_adj(0, hh, false);
    } else {
      drive(t0 + 0.25 * dt);
      phi(0, hh, true);
      drive(t0 + 0.75 * dt);
      phi_adj(0, hh, true);
    }
  }
  // ---- ps2 (adaptive rank): see oracle/ttn.py psi / psi_adj / two_site ----
  cudaError_t err = cudaSuccess;
  void note(cudaError_t e) {
    if (e != cudaSuccess && err == cudaSuccess) err = e;
  }
  // a failure found on the host during a ps2 split (SVD not converged, a grid
  // wait that gave up): the split is abandoned and ttn_step returns it
  ttn_status fail_st = TTN_OK;
  std::string fail_msg;
  void fail(ttn_status st, const std::string& m) {
    if (fail_st == TTN_OK) {
      fail_st = st;
      fail_msg = m;
    }
  }
  uint64_t wait_ns() const { return (uint64_t)(h->params.wait_s * 1e9); }
  // launch the Jacobi SVD (one CTA or the whole GPU) and read back sigma; false
  // (with fail_st set) when it did not converge or a grid wait gave up
  bool jacobi(const double2* theta, int m, int n, std::vector<double>& sig) {
    const int nc = std::min(m, n);
    run(2, 0.0, [&] {
      if (!launch_jacobi_svd_grid(theta, m, n, h->svd_A, h->svd_V, h->svd_sigma, h->svd_info, h->svd_sync,
                                  h->flag_dev, wait_ns(), s))
        {
          const cudaError_t e = cudaGetLastError();
          note(e != cudaSuccess ? e : cudaErrorLaunchFailure);
        }
    });
    sig.assign(nc, 0.0);
    int info[2] = {0, 0}, flag = 0;
    note(cudaMemcpyAsync(sig.data(), h->svd_sigma, nc * sizeof(double), cudaMemcpyDeviceToHost, s));
    note(cudaMemcpyAsync(info, h->svd_info, sizeof(info), cudaMemcpyDeviceToHost, s));
    note(cudaMemcpyAsync(&flag, h->flag_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    note(cudaStreamSynchronize(s));
    if (err != cudaSuccess) return false;
    if (flag & 16) {
      fail(TTN_ETIMEOUT, "a grid barrier of the Jacobi SVD gave up after wait_s");
      return false;
    }
    if (info[0] >= kJacMaxSweeps) {
      fail(TTN_ENUMERIC, "Jacobi SVD of a " + std::to_string(m) + " x " + std::to_string(n) +
                             " two-site matrix did not converge in " + std::to_string(kJacMaxSweeps) + " sweeps");
      return false;
    }
    const int nr = std::max(m, n);
    h->n_flops[2] += 8.0 * 4.0 * info[0] * 0.5 * nc * (nc - 1) * (double)(nr + nc);
    return true;
  }
  // new dims -> job lists rebuilt on the host and re-uploaded (queued kernels
  // still read the old tables, so the stream is drained first)
  void upload_jobs() {
    note(cudaStreamSynchronize(s));
    note(cudaMemcpy((void*)h->T.terms, p.ap_terms.data(), p.ap_terms.size() * sizeof(ApTerm), cudaMemcpyHostToDevice));
    note(cudaMemcpy((void*)h->T.outs, p.ap_outs.data(), p.ap_outs.size() * sizeof(ApOut), cudaMemcpyHostToDevice));
    if (!p.pj_outs.empty())
      note(cudaMemcpy((void*)h->T.pjs, p.pj_outs.data(), p.pj_outs.size() * sizeof(PjOut), cudaMemcpyHostToDevice));
    h->drop_graph();
  }
  void set_rank(int child, int r) {
    if (p.ranks[child] == r) return;
    p.ranks[child] = r;
    p.update_dims();
    p.build_jobs();
    upload_jobs();
  }
  void two_site(int first, int second, double hh, int centre_to) {
    if (err != cudaSuccess || fail_st != TTN_OK) return;
    const int lf = p.tree.leg_index(first, second), ls = p.tree.leg_index(second, first);
    const int fd[3] = {p.dims[first][0], p.dims[first][1], p.dims[first][2]};
    const int sd[3] = {p.dims[second][0], p.dims[second][1], p.dims[second][2]};
    const std::array<int, 4> td = p.theta_dims(first, second);
    const int m = td[0] * td[1], n = td[2] * td[3];
    const int tl = p.buf.th_y;
    run(3, 0.0, [&] {
      launch_merge(h->h_bufs[first], fd, lf, h->h_bufs[second], sd, ls, h->h_bufs[tl], lo_copy(tl), s);
    });
    rk4(p.two_site[p.dir_id(first, second)], tl, p.buf.th_ys, p.buf.th_ys2, p.buf.th_acc, hh);
    const int nc = std::min(m, n);
    const int child = p.tree.parent[first] == second ? first : second;
    const int r_cur = p.ranks[child];
    const int cap = std::min(h->params.max_rank, nc);
    // features of this split (history of the bond), computed before any SVD
    float f[24];
    {
      const auto& es = h->edge_sig[child];
      for (int i = 0; i < 16; ++i)
        f[i] = i < (int)es.size() ? (float)(std::log10(std::max(es[i], 1e-16)) / 16.0) : -1.f;
      f[16] = (float)r_cur / (float)cap;
      const auto& ed = h->edge_disc[child];
      for (int i = 0; i < 4; ++i)
        f[17 + i] = i < (int)ed.size() ? (float)(std::log10(std::max(ed[i], 1e-20)) / 20.0) : -1.f;
      f[21] = (float)(std::log10(std::max(h->params.ps2_atol, 1e-300)) / 10.0);
      f[22] = (float)(h->params.ps2_ratio / 4.0);
      f[23] = 1.f;
    }
    const bool iso_first = centre_to == second;
    const int rows_iso = iso_first ? m : n;
    std::vector<double> sig;
    std::vector<int> perm;
    int r = 0, g = 0;
    bool accepted = false;
    if (h->proposer) {  // proposal -> randomised truncated factorisation, checked exactly
      ++h->n_proposed;
      float logits[13];
      note(cudaMemcpyAsync(h->mlp_x, f, sizeof(f), cudaMemcpyHostToDevice, s));
      run(3, 0.0, [&] { launch_mlp_forward(h->proposer, h->mlp_x, 1, h->mlp_ws, h->mlp_logits, s); });
      note(cudaMemcpyAsync(logits, h->mlp_logits, sizeof(logits), cudaMemcpyDeviceToHost, s));
      note(cudaStreamSynchronize(s));
      int best = 0;
      for (int o = 1; o < 13; ++o)
        if (logits[o] > logits[best]) best = o;
      const int r_prop = std::max(1, std::min(cap, r_cur + best - 4));
      const int kk = std::min(r_prop + 8, nc);
      if (kk < nc && err == cudaSuccess) {
        run(3, 0.0, [&] { launch_gauss(h->rs_omega, (int64_t)n * kk, 0x5eedull + 7919ull * h->n_splits, s); });
        run(2, 8.0 * m * n * kk, [&] { launch_zgemm(h->h_bufs[tl], h->rs_omega, h->rs_Y, m, kk, n, false, s); });
        run(2, 16.0 * (2.0 * m * kk * kk - 2.0 * kk * kk * kk / 3.0), [&] {
          launch_qr(h->rs_Y, m, 1, kk, 2, h->params.qr_tol, h->qr_work, h->qr_elems, h->h_bufs[p.buf.tmp], h->svd_V, h->flag_dev,
                    nullptr, nullptr, s);
        });
        run(2, 8.0 * m * n * kk, [&] { launch_zgemm(h->rs_Y, h->h_bufs[tl], h->rs_B, kk, n, m, true, s); });
        run(3, 0.0, [&] { launch_norm2(h->h_bufs[tl], (int64_t)m * n, h->rs_norm, s); });
        std::vector<double> sb;
        if (!jacobi(h->rs_B, kk, n, sb)) return;
        double tot = 0.0;
        note(cudaMemcpyAsync(&tot, h->rs_norm, sizeof(double), cudaMemcpyDeviceToHost, s));
        note(cudaStreamSynchronize(s));
        std::vector<int> pb(kk);
        for (int i = 0; i < kk; ++i) pb[i] = i;
        std::stable_sort(pb.begin(), pb.end(), [&](int a, int b) { return sb[a] > sb[b]; });
        int r0b = 0;
        for (int i = 0; i < kk; ++i) r0b += sb[i] > h->params.ps2_atol ? 1 : 0;
        const int rb = std::min(cap, std::max(1, (int)std::ceil(h->params.ps2_ratio * r0b - 1e-9)));
        double kept = 0.0;
        for (int i = 0; i < rb; ++i) kept += sb[pb[i]] * sb[pb[i]];
        // accept only if the cut is resolved inside the sketch and the exact discarded
        // weight ||Theta||_F^2 - sum_{i<r} sigma_i^2 is within ps2_atol^2
        if (rb < kk && tot - kept <= h->params.ps2_atol * h->params.ps2_atol) {
          accepted = true;
          ++h->n_accepted;
          r = rb;
          const double smax = sb[pb[0]];
          while (g < r && smax > 0 && sb[pb[g]] > h->params.svd_tol * smax) ++g;
          h->discarded.push_back(std::sqrt(std::max(tot - kept, 0.0)));
          sig.assign(sb.begin(), sb.end());
          perm = pb;
          note(cudaMemcpy(h->svd_perm, perm.data(), r * sizeof(int), cudaMemcpyHostToDevice));
          run(3, 0.0, [&] {
            launch_rsvd_vecs(h->rs_Y, m, kk, h->svd_A, h->svd_V, h->svd_sigma, n, h->svd_perm, r, g, iso_first,
                             h->svd_Z, h->svd_Zg, h->svd_C, s);
          });
        }
      }
    }
    if (!accepted) {
      if (!jacobi(h->h_bufs[tl], m, n, sig)) return;
      // truncation (host): r0 = #{sigma > ps2_atol}, r = min(cap, max(1, ceil(ratio r0)))
      perm.resize(nc);
      for (int i = 0; i < nc; ++i) perm[i] = i;
      std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return sig[a] > sig[b]; });
      int r0 = 0;
      for (int i = 0; i < nc; ++i) r0 += sig[i] > h->params.ps2_atol ? 1 : 0;
      r = std::min(cap, std::max(1, (int)std::ceil(h->params.ps2_ratio * r0 - 1e-9)));
      const double smax = sig[perm[0]];
      while (g < r && smax > 0 && sig[perm[g]] > h->params.svd_tol * smax) ++g;
      double disc = 0.0;
      for (int i = r; i < nc; ++i) disc += sig[perm[i]] * sig[perm[i]];
      h->discarded.push_back(std::sqrt(disc));
      // training record: features and the rank change the SVD rule chose
      for (int i = 0; i < 24; ++i) h->log_feats.push_back(f[i]);
      h->log_labels.push_back(std::max(-4, std::min(8, r - r_cur)) + 4);
      note(cudaMemcpy(h->svd_perm, perm.data(), r * sizeof(int), cudaMemcpyHostToDevice));
      run(3, 0.0, [&] {
        launch_svd_vecs(h->svd_A, h->svd_V, h->svd_sigma, m, n, h->svd_perm, r, g, iso_first, h->svd_Z,
                        h->svd_Zg, h->svd_C, s);
      });
    }
    ++h->n_splits;
    {  // bond history for the next split's features
      auto& es = h->edge_sig[child];
      es.clear();
      const double s1 = sig.empty() ? 0.0 : sig[perm[0]];
      for (int i = 0; i < 16 && i < (int)perm.size(); ++i) es.push_back(s1 > 0 ? sig[perm[i]] / s1 : 0.0);
      auto& ed = h->edge_disc[child];
      ed.insert(ed.begin(), h->discarded.back());
      if (ed.size() > 4) ed.resize(4);
    }
    if (g < r) {  // deterministic completion of the undetermined directions (Householder, tol 0)
      run(2, 0.0, [&] {
        launch_qr(h->svd_Z, rows_iso, 1, r, 2, 0.0, h->qr_work, h->qr_elems, h->h_bufs[p.buf.tmp], h->svd_V, h->flag_dev,
                  nullptr, nullptr, s);
      });
      run(3, 0.0, [&] { launch_restore_cols(h->svd_Z, h->svd_Zg, rows_iso, r, g, s); });
    }
    set_rank(child, r);
    const int nfd[3] = {p.dims[first][0], p.dims[first][1], p.dims[first][2]};
    const int nsd[3] = {p.dims[second][0], p.dims[second][1], p.dims[second][2]};
    run(3, 0.0, [&] {
      launch_write_pair(h->h_bufs[first], lo_copy(first), nfd, lf, h->h_bufs[second], lo_copy(second), nsd, ls,
                        h->svd_Z, h->svd_C, r, iso_first, s);
    });
  }
  void psi(int u, double hh, bool last) {
    const auto& ch = p.tree.children[u];
    for (size_t idx = 0; idx < ch.size(); ++idx) {
      const int c = ch[idx];
      qr(u, c);
      absorb(c, u);
      env(u, c);
      psi(c, hh, false);
      two_site(c, u, hh, u);
      env(c, u);
      if (!(last && idx + 1 == ch.size())) node_flow(u, -hh);
    }
  }
  void psi_adj(int u, double hh, bool first_call) {
    const auto& ch = p.tree.children[u];
    for (size_t k = 0; k < ch.size(); ++k) {
      const int c = ch[ch.size() - 1 - k];
      if (!(first_call && k == 0)) node_flow(u, -hh);
      two_site(u, c, hh, c);
      env(u, c);
      psi_adj(c, hh, false);
      qr(c, u);
      env(c, u);
      absorb(u, c);
    }
  }
  void step_ps2(double dt, double t0) {
    const double hh = 0.5 * dt;
    drive(t0 + 0.25 * dt);
    psi(0, hh, true);
    drive(t0 + 0.75 * dt);
    psi_adj(0, hh, true);
  }

  // ---- vmf (direct integration): see oracle/ttn.py vmf_rhs / step_vmf ----
  void copy64(double2* dst, const double2* src, int64_t n) {
    run(3, 0.0, [&] { launch_copy(dst, nullptr, src, n, s); });
  }
  // node derivative of u into K (flat layout); root: H A, others: the
  // projected, regularised equation (vmf.cu)
  void vmf_node(int u, double2* K) {
    double2* Ku = K + h->node_off[u];
    store(0, p.node_flow[u].first[0]);
    apply(0, p.node_flow[u].combine[0],
          Epi{EPI_RK1, h->h_bufs[u], h->h_bufs_lo[u], h->h_bufs_lo[p.buf.ys], Ku, 0.0});
    if (u == 0) return;
    apply(0, p.node_down[u], Epi{EPI_RK1, h->h_bufs[u], h->h_bufs_lo[u], h->h_bufs_lo[p.buf.ys], h->h_bufs[p.buf.acc], 0.0});
    const int r = p.dims[u][0];
    const int64_t nc = p.P[u] / r;
    run(3, 0.0, [&] {
      launch_vmf_finish(Ku, h->h_bufs[p.buf.acc], h->vmf_dmi, h->h_bufs[u], r, nc, h->vmf_x, s);
    });
  }
  // buffer pn holds the gauge-moved V_pn (the parent edge's class slots the
  // isometric environments); every child edge gets its isometric environments
  // and its R, then each child (its own V absorbed) recursively, then the
  // child's edge is transformed and the child's derivative computed
  void vmf_walk(int pn, double2* K) {
    const auto& ch = p.tree.children[pn];
    for (int c : ch) {
      copy64(h->vmf_tmp, h->h_bufs[pn], p.P[pn]);
      qr(pn, c);
      env(pn, c);
      copy64(h->vmf_r + h->vmf_r_off[c], h->h_bufs[p.buf.bond_y], (int64_t)p.ranks[c] * p.ranks[c]);
      copy64(h->h_bufs[pn], h->vmf_tmp, p.P[pn]);
    }
    for (int c : ch) {
      copy64(h->vmf_save + h->node_off[c], h->h_bufs[c], p.P[c]);
      copy64(h->h_bufs[p.buf.bond_y], h->vmf_r + h->vmf_r_off[c], (int64_t)p.ranks[c] * p.ranks[c]);
      absorb(c, pn);
      vmf_walk(c, K);
      copy64(h->h_bufs[c], h->vmf_save + h->node_off[c], p.P[c]);
      const int e = p.dir_id(pn, c);
      const int nk = h->vmf_slot_off[e + 1] - h->vmf_slot_off[e];
      run(3, 0.0, [&] {
        launch_vmf_edge((double2* const*)h->T.mats, h->vmf_slots + h->vmf_slot_off[e], nk, h->vmf_r + h->vmf_r_off[c],
                        p.ranks[c], h->params.vmf_atol, h->vmf_aug, h->vmf_dmi, h->vmf_ctmp, s);
      });
      vmf_node(c, K);
    }
  }
  // K := F(t, y) for the stage state in the node buffers
  void vmf_rhs(double t, double2* K) {
    drive(t);
    for (int c : p.tree.postorder)
      if (c != 0) env(c, p.tree.parent[c]);
    vmf_node(0, K);
    vmf_walk(0, K);
  }

  void rebuild_envs() {
    drive(h->t);
    for (int c : p.tree.postorder)
      if (c != 0) env(c, p.tree.parent[c]);
  }
  void rdm(double2* out) {
    for (int u : p.tree.postorder) {
      const auto& d = p.dims[u];
      const double2* w[3] = {nullptr, nullptr, nullptr};
      for (int li = (u == 0 ? 2 : 1); li < 3; ++li) {
        const Leg& L = p.tree.legs[u][li];
        if (L.kind == 'n') w[li] = h->rdm_vec + h->rdm_off[L.v];
      }
      run(3, 0.0, [&] {
        launch_rdm_node(h->h_bufs[u], d[0], d[1], d[2], u == 0, w[1], w[2],
                        u == 0 ? out : h->rdm_vec + h->rdm_off[u], s);
      });
    }
  }
};


// Capture one ps1 step of h as a CUDA graph (autonomous generator, non-default
// stream, not profiling). Returns whether h->graph is usable for dt.
bool ensure_graph(ttn_t h, double dt) {
  const bool graphable =
      h->plan.n_drives == 0 && h->prof_mode != 1 && h->stream != nullptr && !h->graph_disabled;
  if (!graphable) return false;
  if (h->graph && h->graph_dt == dt && h->graph_prof == h->prof_mode) return true;
  h->drop_graph();
  Exec ex(h);
  int64_t l0[4];
  double f0[4];
  for (int c = 0; c < 4; ++c) {
    l0[c] = h->n_launch[c];
    f0[c] = h->n_flops[c];
  }
  cudaGraph_t g = nullptr;
  bool ok = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    h->capturing = h->prof_mode == 2;
    ex.step_ps1(dt, h->t);
    h->capturing = false;
    ok = cudaStreamEndCapture(h->stream, &g) == cudaSuccess && g != nullptr;
  }
  if (ok) ok = cudaGraphInstantiate(&h->graph, g, 0) == cudaSuccess;
  for (int c = 0; c < 4; ++c) {  // the captured launches did not run
    h->graph_launch[c] = h->n_launch[c] - l0[c];
    h->graph_flops[c] = h->n_flops[c] - f0[c];
    h->n_launch[c] = l0[c];
    h->n_flops[c] = f0[c];
  }
  if (!ok) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    h->drop_graph();
    h->graph_disabled = true;
    return false;
  }
  h->graph_src = g;
  h->graph_dt = dt;
  h->graph_prof = h->prof_mode;
  return true;
}

template <typename F>
ttn_status guarded(ttn_t h, F&& f) {
  if (!h) return TTN_EINVAL;
  try {
    return f();
  } catch (const std::bad_alloc&) {
    return h->fail(TTN_ENOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return h->fail(TTN_EINVAL, e.what());
  }
}

ttn_status status_of(const std::string& e) {
  if (e.rfind("UNSUPPORTED", 0) == 0) return TTN_EUNSUPPORTED;
  return TTN_EINVAL;
}

// Copy n complex values to an FP64 device buffer and, in FP32 mode, to its shadow.
ttn_status upload_pair(ttn_t h, double2* dst, void* dst_lo, const double2* src, size_t n) {
  cudaStream_t s = h->stream;
  CUDA_TRY(h, cudaMemcpyAsync(dst, src, n * sizeof(double2), cudaMemcpyHostToDevice, s));
  if (h->prec == PREC_F32 && dst_lo && dst_lo != (void*)dst) {
    std::vector<float2> lo(n);
    for (size_t i = 0; i < n; ++i) lo[i] = make_float2((float)src[i].x, (float)src[i].y);
    CUDA_TRY(h, cudaMemcpyAsync(dst_lo, lo.data(), n * sizeof(float2), cudaMemcpyHostToDevice, s));
    CUDA_TRY(h, cudaStreamSynchronize(s));
  }
  CUDA_TRY(h, cudaStreamSynchronize(s));
  return TTN_OK;
}

ttn_status upload_initial(ttn_t h, const double* rho0) {
  Plan& p = h->plan;
  if (!h->init_ranks.empty() && p.ranks != h->init_ranks) {  // ps2 changed them
    Exec ex(h);
    p.ranks = h->init_ranks;
    p.update_dims();
    p.build_jobs();
    ex.upload_jobs();
    if (ex.err != cudaSuccess) return cuda_fail(h, ex.err, "job upload");
  }
  const int M = p.leg_dims[0];
  cudaStream_t s = h->stream;
  for (int u = 0; u < p.tree.n_nodes; ++u) {
    std::vector<double2> T((size_t)p.P[u], make_double2(0.0, 0.0));
    const auto& d = p.dims[u];
    if (u == 0) {
      // legs 0, 1 (i, j) come first in the root's canonical order
      for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j)
          T[((size_t)i * d[1] + j) * d[2]] = make_double2(rho0[2 * (i * M + j)], rho0[2 * (i * M + j) + 1]);
    } else {
      const int64_t cols = (int64_t)d[1] * d[2];
      for (int a = 0; a < d[0]; ++a) T[(size_t)a * cols + a] = make_double2(1.0, 0.0);
    }
    ttn_status st = upload_pair(h, h->h_bufs[u], h->h_bufs_lo[u], T.data(), T.size());
    if (st != TTN_OK) return st;
  }
  (void)s;
  h->envs_dirty = true;
  h->t = 0.0;
  h->vmf_h = 0.0;
  h->mix_switched = false;
  return TTN_OK;
}

ttn_status ensure_envs(ttn_t h) {
  if (!h->envs_dirty) return TTN_OK;
  Exec ex(h);
  ex.rebuild_envs();
  CUDA_TRY(h, cudaGetLastError());
  h->envs_dirty = false;
  return TTN_OK;
}

}  // namespace

extern "C" {

ttn_status ttn_create(const ttn_tree* tree, const int32_t* leg_dims, const int32_t* ranks,
                      int32_t precision, ttn_t* out) {
  if (!out) return TTN_EINVAL;
  *out = nullptr;
  if (!tree || !leg_dims || !ranks) return TTN_EINVAL;
  if (precision != TTN_FP64 && precision != TTN_MIXED_FP32) return TTN_EINVAL;
  ttn_t h = new (std::nothrow) ttn_ctx();
  if (!h) return TTN_ENOMEM;
  std::string e;
  {  // SM count sizes the per-tile CTA split of the job lists; keep the default without a device
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
      h->plan.sm_count = sms;
    else
      cudaGetLastError();
  }
  try {
    e = h->plan.build(tree->n_nodes, tree->parent, tree->n_legs, tree->leg_node, leg_dims, ranks);
  } catch (...) {
    e = "tree construction failed";
  }
  if (!e.empty()) {
    ttn_status st = status_of(e);
    delete h;
    return st;
  }
  h->precision = precision;
  h->prec = precision == TTN_MIXED_FP32 ? PREC_F32 : PREC_F64;
  *out = h;
  return TTN_OK;
}

ttn_status ttn_set_params(ttn_t h, const ttn_params* prm) {
  return guarded(h, [&]() -> ttn_status {
    if (!prm) return h->fail(TTN_EINVAL, "null params");
    if (!(prm->qr_tol >= 0) || !(prm->kappa > 0) || !(prm->ps2_atol >= 0) || !(prm->ps2_ratio >= 1) ||
        prm->max_rank < 1 || !(prm->svd_tol >= 0) || prm->max_split < 1 || prm->max_split > kMaxSplit ||
        (prm->tensor_cores < 0 || prm->tensor_cores > 2) || !(prm->wait_s >= 0.0 && prm->wait_s <= 60.0) ||
        !(prm->ode_rtol > 0.0) || !(prm->ode_atol > 0.0) || !(prm->vmf_atol >= 0.0) ||
        !(prm->tile_warps == 0 || prm->tile_warps == 2 || prm->tile_warps == 4 || prm->tile_warps == 8))
      return h->fail(TTN_EINVAL, "parameter out of range");
    if (h->ws_bound && prm->max_rank != h->params.max_rank)
      return h->fail(TTN_ESTATE, "max_rank must be set before the workspace is bound");
    if (prm->max_rank != h->plan.cap_rank) {
      h->plan.set_caps(prm->max_rank);
      if (h->plan.r_cap_max > 256) return h->fail(TTN_EUNSUPPORTED, "bond ranks above 256");
      if (h->sop_loaded) {
        std::string e = h->plan.rebuild_classes();
        if (!e.empty()) return h->fail(TTN_EINVAL, e);
      }
    }
    if (prm->max_split != h->params.max_split || prm->tile_warps != h->params.tile_warps)
      h->plan.set_split(prm->max_split, prm->tile_warps);
    h->params = *prm;
    h->drop_graph();  // substep counts, tolerances and launch shapes are baked into a captured step
    return TTN_OK;
  });
}

ttn_status ttn_get_params(ttn_t h, ttn_params* prm) {
  if (!h || !prm) return TTN_EINVAL;
  *prm = h->params;
  return TTN_OK;
}

ttn_status sop_load(ttn_t h, int32_t n_ops, const int32_t* op_leg, const int64_t* op_offset,
                    const double* op_data, int32_t n_terms, const int32_t* term_offsets,
                    const int32_t* term_ops, const double* coef, const int32_t* coef_drive) {
  return guarded(h, [&]() -> ttn_status {
    if (h->ws_bound) return h->fail(TTN_ESTATE, "sop_load after the workspace was bound");
    std::string e = h->plan.load_sop(n_ops, op_leg, op_offset, op_data, n_terms, term_offsets, term_ops,
                                     coef, coef_drive);
    if (!e.empty()) {
      h->sop_loaded = false;
      return h->fail(status_of(e), e);
    }
    if (h->plan.n_drives > kMaxDrives) return h->fail(TTN_EUNSUPPORTED, "at most 8 drives");
    if ((int)h->drives.size() < h->plan.n_drives) h->drives.resize(h->plan.n_drives);
    for (int d = 0; d < h->plan.n_drives; ++d) h->plan.drive_bound[d] = h->drives[d].bound;
    h->plan.compute_lambda();
    e = h->plan.build_jobs();
    if (!e.empty()) return h->fail(TTN_EINVAL, e);
    h->sop_loaded = true;
    return TTN_OK;
  });
}

ttn_status ttn_set_drive(ttn_t h, int32_t id, ttn_drive_fn g, void* user, double g_bound) {
  return guarded(h, [&]() -> ttn_status {
    if (id < 0 || id >= kMaxDrives) return h->fail(TTN_EINVAL, "drive id out of range");
    if (!g || !(g_bound >= 0) || !std::isfinite(g_bound)) return h->fail(TTN_EINVAL, "bad drive");
    if (h->ws_bound) return h->fail(TTN_ESTATE, "ttn_set_drive after the workspace was bound");
    if ((int)h->drives.size() <= id) h->drives.resize(id + 1);
    h->drives[id] = DriveSlot{g, user, g_bound};
    if ((int)h->plan.drive_bound.size() <= id) h->plan.drive_bound.resize(id + 1, 1.0);
    h->plan.drive_bound[id] = g_bound;
    if (h->sop_loaded) h->plan.compute_lambda();
    return TTN_OK;
  });
}

ttn_status ttn_workspace_size(ttn_t h, size_t* bytes) {
  return guarded(h, [&]() -> ttn_status {
    if (!bytes) return h->fail(TTN_EINVAL, "null bytes");
    if (!h->sop_loaded) return h->fail(TTN_ESTATE, "sop_load first");
    *bytes = layout_of(h->plan, h->prec).total;
    return TTN_OK;
  });
}

ttn_status ttn_set_stream(ttn_t h, void* stream) {
  if (!h) return TTN_EINVAL;
  cudaStream_t ns = (cudaStream_t)stream;
  if (h->ws_bound && ns != h->stream) {  // order the new stream after work queued on the old one
    cudaEvent_t ev;
    CUDA_TRY(h, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CUDA_TRY(h, cudaEventRecord(ev, h->stream));
    CUDA_TRY(h, cudaStreamWaitEvent(ns, ev, 0));
    cudaEventDestroy(ev);
  }
  h->stream = ns;
  h->drop_graph();
  return TTN_OK;
}

ttn_status ttn_set_workspace(ttn_t h, void* dptr, size_t bytes) {
  return guarded(h, [&]() -> ttn_status {
    if (!h->sop_loaded) return h->fail(TTN_ESTATE, "sop_load first");
    if (!dptr || ((uintptr_t)dptr % kAlign) != 0) return h->fail(TTN_EINVAL, "workspace must be 256-byte aligned");
    for (int d = 0; d < h->plan.n_drives; ++d)
      if (!h->drives[d].fn) return h->fail(TTN_ESTATE, "a drive used by the SOP has no function");
    allow_wide_splits();
    Plan& p = h->plan;
    Layout L = layout_of(p, h->prec);
    if (bytes < L.total) return h->fail(TTN_ENOMEM, "workspace smaller than ttn_workspace_size");
    char* base = (char*)dptr;
    h->ws = base;
    h->ws_bytes = bytes;
    // buffer table
    h->h_bufs.assign(p.buf.n_bufs, nullptr);
    double2* nodes = (double2*)(base + L.nodes);
    for (int u = 0; u < p.tree.n_nodes; ++u) h->h_bufs[u] = nodes + L.node_off[u];
    double2* scr = (double2*)(base + L.scratch);
    int64_t o = 0;
    auto nxt = [&](int64_t n) {
      double2* q = scr + o;
      o += n;
      return q;
    };
    const int64_t S = std::max(p.P_cap_max, p.theta_cap);
    h->h_bufs[p.buf.ys] = nxt(S);
    h->h_bufs[p.buf.ys2] = nxt(S);
    h->h_bufs[p.buf.acc] = nxt(S);
    h->h_bufs[p.buf.tmp] = nxt(S);
    for (int i = 0; i < p.buf.n_t; ++i) h->h_bufs[p.buf.t0 + i] = nxt(S);
    for (int i = 0; i < p.buf.n_w; ++i) h->h_bufs[p.buf.w0 + i] = nxt(S);
    h->h_bufs[p.buf.th_y] = nxt(p.theta_cap);
    h->h_bufs[p.buf.th_ys] = nxt(p.theta_cap);
    h->h_bufs[p.buf.th_ys2] = nxt(p.theta_cap);
    h->h_bufs[p.buf.th_acc] = nxt(p.theta_cap);
    h->svd_A = nxt(p.theta_cap);
    h->svd_V = nxt(p.theta_cap);
    h->svd_Z = nxt(p.theta_cap);
    h->svd_Zg = nxt(p.theta_cap);
    h->svd_C = nxt(p.theta_cap);
    h->svd_sigma = (double*)(base + L.svd_small);
    h->svd_perm = (int*)(h->svd_sigma + p.theta_cap);
    h->svd_info = h->svd_perm + p.theta_cap;
    h->svd_sync = (unsigned*)(h->svd_info + 4);
    h->rs_omega = (double2*)(base + L.rsvd);
    h->rs_Y = h->rs_omega + p.theta_cap;
    h->rs_B = h->rs_Y + p.theta_cap;
    h->rs_norm = (double*)(base + L.mlp);
    h->mlp_x = (float*)(h->rs_norm + 2);
    h->mlp_logits = h->mlp_x + 24;
    h->mlp_ws = h->mlp_logits + 16;
    h->edge_sig.assign(p.tree.n_nodes, {});
    h->edge_disc.assign(p.tree.n_nodes, {});
    const int64_t r2 = (int64_t)p.r_cap_max * p.r_cap_max;
    h->h_bufs[p.buf.bond_y] = nxt(r2);
    h->h_bufs[p.buf.bond_ys] = nxt(r2);
    h->h_bufs[p.buf.bond_ys2] = nxt(r2);
    h->h_bufs[p.buf.bond_acc] = nxt(r2);
    h->pool = (double2*)(base + L.pool);
    h->h_mats.assign(p.mats.size(), nullptr);
    for (size_t i = 0; i < p.mats.size(); ++i)
      h->h_mats[i] = p.mats[i].off >= 0 ? h->pool + p.mats[i].off : nullptr;
    h->h_mats[p.bond_mat] = h->h_bufs[p.buf.bond_y];
    h->qr_work = (double2*)(base + L.qr);
    h->qr_elems = L.qr_elems;
    h->rdm_vec = (double2*)(base + L.rdm);
    h->rdm_off = L.rdm_off;
    h->rho_dev = (double2*)(base + L.rho);
    h->flag_dev = (int*)(base + L.flag);
    h->node_off = L.node_off;
    if (h->prec == PREC_F64) {
      h->vmf_n = L.nodes_elems;
      h->vmf_y = (double2*)(base + L.vmf_y);
      h->vmf_save = (double2*)(base + L.vmf_save);
      for (int k = 0; k < 7; ++k) h->vmf_k[k] = (double2*)(base + L.vmf_k) + (int64_t)k * L.nodes_elems;
      h->vmf_tmp = (double2*)(base + L.vmf_tmp);
      h->vmf_r = (double2*)(base + L.vmf_r);
      h->vmf_aug = (double2*)(base + L.vmf_aug);
      h->vmf_dmi = (double2*)(base + L.vmf_dmi);
      h->vmf_x = (double2*)(base + L.vmf_x);
      h->vmf_ctmp = (double2*)(base + L.vmf_ctmp);
      h->vmf_slots = (int*)(base + L.vmf_slots);
      h->vmf_err = (double*)(base + L.vmf_err);
      h->vmf_r_off = L.vmf_r_off;
      h->vmf_slot_off = L.vmf_slot_off;
      if (!L.vmf_slot_host.empty())
        CUDA_TRY(h, cudaMemcpy(h->vmf_slots, L.vmf_slot_host.data(), L.vmf_slot_host.size() * sizeof(int),
                               cudaMemcpyHostToDevice));
    }
    h->T.bufs = (void* const*)(base + L.bufs_tab);
    h->T.mats = (void* const*)(base + L.mats_tab);
    h->T.terms = (const ApTerm*)(base + L.terms);
    h->T.outs = (const ApOut*)(base + L.outs);
    h->T.pjs = (const PjOut*)(base + L.pjs);
    h->drive_list_dev = (DriveMat*)(base + L.drives);
    // contraction-type view: FP64 mode aliases the FP64 buffers
    h->h_bufs_lo.assign(h->h_bufs.begin(), h->h_bufs.end());
    h->h_mats_lo.assign(h->h_mats.begin(), h->h_mats.end());
    h->Tlo = h->T;
    if (h->prec == PREC_F32) {
      float2* n32 = (float2*)(base + L.nodes32);
      for (int u = 0; u < p.tree.n_nodes; ++u) h->h_bufs_lo[u] = n32 + L.node_off[u];
      float2* sc = (float2*)(base + L.scratch32);
      int64_t o32 = 0;
      auto nx = [&](int64_t n) {
        float2* q = sc + o32;
        o32 += n;
        return (void*)q;
      };
      h->h_bufs_lo[p.buf.ys] = nx(S);
      h->h_bufs_lo[p.buf.ys2] = nx(S);
      for (int i = 0; i < p.buf.n_t; ++i) h->h_bufs_lo[p.buf.t0 + i] = nx(S);
      for (int i = 0; i < p.buf.n_w; ++i) h->h_bufs_lo[p.buf.w0 + i] = nx(S);
      h->h_bufs_lo[p.buf.th_y] = nx(p.theta_cap);
      h->h_bufs_lo[p.buf.th_ys] = nx(p.theta_cap);
      h->h_bufs_lo[p.buf.th_ys2] = nx(p.theta_cap);
      h->h_bufs_lo[p.buf.th_acc] = nullptr;
      h->h_bufs_lo[p.buf.bond_y] = nx(r2);
      h->h_bufs_lo[p.buf.bond_ys] = nx(r2);
      h->h_bufs_lo[p.buf.bond_ys2] = nx(r2);
      h->h_bufs_lo[p.buf.acc] = nullptr;       // accumulators stay FP64 (epilogue pointers)
      h->h_bufs_lo[p.buf.bond_acc] = nullptr;
      h->h_bufs_lo[p.buf.tmp] = nullptr;       // absorb runs in FP64
      float2* p32 = (float2*)(base + L.pool32);
      for (size_t i = 0; i < p.mats.size(); ++i)
        h->h_mats_lo[i] = p.mats[i].off >= 0 ? (void*)(p32 + p.mats[i].off) : nullptr;
      h->h_mats_lo[p.bond_mat] = h->h_bufs_lo[p.buf.bond_y];
      h->tc_acc = (float2*)(base + L.tc_acc);
      h->tc_acc_elems = 3 * S;
      h->tc_pool = (float*)(base + L.tc_pool);
      h->tc_off_dev = (int64_t*)(base + L.tc_off);
      h->tc_off = L.tc_off_host;
      h->tc_bsplit = (float*)(base + L.tc_bsplit);
      h->tc_bsplit_floats = L.tc_bsplit_floats;
      h->tc_pool_on = false;
      for (const ApList& al : p.ap_lists)
        h->tc_pool_on = h->tc_pool_on || (al.n_tiles > 0 && tc_applicable(al, p.ap_outs.data(), p.ap_terms.data()));
      h->Tlo.bufs = (void* const*)(base + L.bufs_tab_lo);
      h->Tlo.mats = (void* const*)(base + L.mats_tab_lo);
    }
    cudaStream_t s = h->stream;
    CUDA_TRY(h, cudaMemcpyAsync((void*)h->T.bufs, h->h_bufs.data(), h->h_bufs.size() * sizeof(double2*),
                                cudaMemcpyHostToDevice, s));
    CUDA_TRY(h, cudaMemcpyAsync((void*)h->T.mats, h->h_mats.data(), h->h_mats.size() * sizeof(double2*),
                                cudaMemcpyHostToDevice, s));
    if (h->prec == PREC_F32) {
      CUDA_TRY(h, cudaMemcpyAsync((void*)h->Tlo.bufs, h->h_bufs_lo.data(), h->h_bufs_lo.size() * sizeof(void*),
                                  cudaMemcpyHostToDevice, s));
      CUDA_TRY(h, cudaMemcpyAsync((void*)h->Tlo.mats, h->h_mats_lo.data(), h->h_mats_lo.size() * sizeof(void*),
                                  cudaMemcpyHostToDevice, s));
      CUDA_TRY(h, cudaMemcpyAsync(h->tc_off_dev, h->tc_off.data(), h->tc_off.size() * sizeof(int64_t),
                                  cudaMemcpyHostToDevice, s));
      CUDA_TRY(h, cudaStreamSynchronize(s));
    }
    if (!p.ap_terms.empty())
      CUDA_TRY(h, cudaMemcpyAsync((void*)h->T.terms, p.ap_terms.data(), p.ap_terms.size() * sizeof(ApTerm),
                                  cudaMemcpyHostToDevice, s));
    if (!p.ap_outs.empty())
      CUDA_TRY(h, cudaMemcpyAsync((void*)h->T.outs, p.ap_outs.data(), p.ap_outs.size() * sizeof(ApOut),
                                  cudaMemcpyHostToDevice, s));
    if (!p.pj_outs.empty())
      CUDA_TRY(h, cudaMemcpyAsync((void*)h->T.pjs, p.pj_outs.data(), p.pj_outs.size() * sizeof(PjOut),
                                  cudaMemcpyHostToDevice, s));
    // open-leg matrices: current = static part at g = 0; drive parts
    h->drive_list.clear();
    std::vector<double2> tmp;
    std::vector<float2> tmp32;
    auto put = [&](int slot, const std::vector<cd>& m) -> cudaError_t {
      tmp.resize(m.size());
      for (size_t i = 0; i < m.size(); ++i) tmp[i] = make_double2(m[i].real(), m[i].imag());
      cudaError_t e = cudaMemcpyAsync(h->h_mats[slot], tmp.data(), tmp.size() * sizeof(double2),
                                      cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess && h->prec == PREC_F32 && h->h_mats_lo[slot] != (void*)h->h_mats[slot]) {
        tmp32.resize(m.size());
        for (size_t i = 0; i < m.size(); ++i) tmp32[i] = make_float2((float)m[i].real(), (float)m[i].imag());
        e = cudaMemcpyAsync(h->h_mats_lo[slot], tmp32.data(), tmp32.size() * sizeof(float2),
                            cudaMemcpyHostToDevice, s);
      }
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      return e;
    };
    for (const LocalMat& lm : p.locals) {
      CUDA_TRY(h, put(lm.slot, lm.stat));
      if (lm.time_dependent) {
        CUDA_TRY(h, put(lm.slot_stat, lm.stat));
        DriveMat dm{};
        dm.d = p.leg_dims[lm.leg];
        dm.cur = lm.slot;
        dm.stat = lm.slot_stat;
        for (int d = 0; d < kMaxDrives; ++d) dm.part[d] = -1;
        for (int d = 0; d < p.n_drives; ++d)
          if (lm.slot_drive[d] >= 0) {
            CUDA_TRY(h, put(lm.slot_drive[d], lm.drive[d]));
            dm.part[d] = lm.slot_drive[d];
          }
        h->drive_list.push_back(dm);
      }
    }
    if (!h->drive_list.empty())
      CUDA_TRY(h, cudaMemcpyAsync(h->drive_list_dev, h->drive_list.data(), h->drive_list.size() * sizeof(DriveMat),
                                  cudaMemcpyHostToDevice, s));
    CUDA_TRY(h, cudaMemsetAsync(h->flag_dev, 0, sizeof(int), s));
    if (h->tc_pool_on) {  // pool copies of the open-leg operators (classes follow with every env update)
      std::vector<TcEmbedJob> jobs;
      for (const LocalMat& lm : p.locals)
        if (h->tc_off[lm.slot] >= 0) jobs.push_back(TcEmbedJob{lm.slot, p.leg_dims[lm.leg], h->tc_off[lm.slot]});
      launch_tc_embed(h->Tlo.mats, jobs.data(), (int)jobs.size(), h->tc_pool, s);
      CUDA_TRY(h, cudaGetLastError());
    }
    CUDA_TRY(h, cudaStreamSynchronize(s));
    h->ws_bound = true;
    h->init_ranks = p.ranks;
    const int M = p.leg_dims[0];
    std::vector<double> rho0(2 * M * M, 0.0);
    rho0[0] = 1.0;
    ttn_status st = upload_initial(h, rho0.data());
    if (st != TTN_OK) return st;
    return ensure_envs(h);
  });
}

ttn_status ttn_set_rdo0(ttn_t h, const double* rho0) {
  return guarded(h, [&]() -> ttn_status {
    if (!h->ws_bound) return h->fail(TTN_ESTATE, "bind the workspace first");
    if (!rho0) return h->fail(TTN_EINVAL, "null rho0");
    const int M = h->plan.leg_dims[0];
    for (int i = 0; i < 2 * M * M; ++i)
      if (!std::isfinite(rho0[i])) return h->fail(TTN_EINVAL, "non-finite rho0");
    ttn_status st = upload_initial(h, rho0);
    if (st != TTN_OK) return st;
    CUDA_TRY(h, cudaMemsetAsync(h->flag_dev, 0, sizeof(int), h->stream));
    return ensure_envs(h);
  });
}

}  // extern "C"

namespace {

// Dormand-Prince 5(4) (Dormand & Prince 1980), the tableau and controller of
// oracle/ttn.py dopri5: err = sqrt(sum |e / (atol + rtol max(|y|, |y5|))|^2 / n)
// over the active entries, accept when err <= 1, next trial step
// h * min(5, max(0.2, 0.9 err^(-1/5))), a shortened landing step keeps the
// longer trial step.
constexpr double kDpC[7] = {0.0, 1.0 / 5, 3.0 / 10, 4.0 / 5, 8.0 / 9, 1.0, 1.0};
constexpr double kDpA[7][6] = {{0, 0, 0, 0, 0, 0},
                               {1.0 / 5, 0, 0, 0, 0, 0},
                               {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
                               {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
                               {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
                               {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
                               {35.0 / 384, 0.0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};
constexpr double kDpB5[7] = {35.0 / 384, 0.0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84, 0.0};
constexpr double kDpB4[7] = {5179.0 / 57600, 0.0, 7571.0 / 16695, 393.0 / 640, -92097.0 / 339200, 187.0 / 2100,
                             1.0 / 40};

ttn_status vmf_steps(ttn_t h, double dt, int n_steps) {
  if (h->prec != PREC_F64) return h->fail(TTN_EUNSUPPORTED, "vmf runs in the FP64 form only");
  Plan& p = h->plan;
  cudaStream_t s = h->stream;
  ttn_status st = ensure_envs(h);
  if (st != TTN_OK) return st;
  Exec ex(h);
  double2* nodes = h->h_bufs[0];
  const int n = p.tree.n_nodes;
  // inactive tails of the capacity slots stay zero in every flat vector
  for (int u = 0; u < n; ++u) {
    const int64_t slot = (u + 1 < n ? h->node_off[u + 1] : h->vmf_n) - h->node_off[u];
    if (slot > p.P[u])
      CUDA_TRY(h, cudaMemsetAsync(nodes + h->node_off[u] + p.P[u], 0, (slot - p.P[u]) * sizeof(double2), s));
  }
  for (int k = 0; k < 7; ++k) CUDA_TRY(h, cudaMemsetAsync(h->vmf_k[k], 0, h->vmf_n * sizeof(double2), s));
  int64_t cnt = 0;
  for (int u = 0; u < n; ++u) cnt += p.P[u];
  double2* K[7];
  for (int k = 0; k < 7; ++k) K[k] = h->vmf_k[k];
  const double rtol = h->params.ode_rtol, atol = h->params.ode_atol;
  for (int step = 0; step < n_steps; ++step) {
    const double t0 = h->t, t1 = t0 + dt;
    double t = t0, h_try = h->vmf_h > 0.0 ? h->vmf_h : dt;
    ex.copy64(h->vmf_y, nodes, h->vmf_n);
    ex.vmf_rhs(t, K[0]);
    int guard = 0;
    while (t1 - t > 1e-13 * std::max(1.0, std::fabs(t1))) {
      if (++guard > 100000) return h->fail(TTN_ENUMERIC, "vmf: dopri5 step limit reached");
      const bool last = h_try >= t1 - t;
      const double hh = last ? t1 - t : h_try;
      for (int i = 1; i < 7; ++i) {
        VmfComb cb{};
        cb.n = i;
        for (int l = 0; l < i; ++l) {
          cb.c[l] = hh * kDpA[i][l];
          cb.K[l] = K[l];
        }
        ex.run(3, 0.0, [&] { launch_vmf_stage(nodes, h->vmf_y, cb, h->vmf_n, s); });
        ex.vmf_rhs(t + kDpC[i] * hh, K[i]);
      }
      VmfComb ce{};
      ce.n = 7;
      for (int l = 0; l < 7; ++l) {
        ce.c[l] = hh * (kDpB5[l] - kDpB4[l]);
        ce.K[l] = K[l];
      }
      ex.run(3, 0.0, [&] {
        launch_vmf_err(h->vmf_y, nodes, ce, rtol, atol, h->vmf_n, h->vmf_err, h->vmf_err + 1024, s);
      });
      double sum = 0.0;
      CUDA_TRY(h, cudaMemcpyAsync(&sum, h->vmf_err + 1024, sizeof(double), cudaMemcpyDeviceToHost, s));
      CUDA_TRY(h, cudaStreamSynchronize(s));
      if (ex.err != cudaSuccess) return cuda_fail(h, ex.err, "vmf step");
      const double err = std::sqrt(sum / (double)std::max<int64_t>(cnt, 1));
      if (!std::isfinite(err) && !(hh > 1e-12 * dt))
        return h->fail(TTN_ENUMERIC, "vmf: non-finite error estimate at the smallest step");
      const double fac = !std::isfinite(err) ? 0.2
                         : err == 0.0       ? 5.0
                                            : std::min(5.0, std::max(0.2, 0.9 * std::pow(err, -0.2)));
      if (err <= 1.0) {
        t = last ? t1 : t + hh;
        ex.copy64(h->vmf_y, nodes, h->vmf_n);  // y5, already in the node buffers
        std::swap(K[0], K[6]);
        ++h->vmf_acc;
        h_try = last ? std::max(h_try, hh * fac) : hh * fac;
      } else {
        ++h->vmf_rej;
        h_try = hh * fac;
        if (!(h_try > 1e-12 * dt)) return h->fail(TTN_ENUMERIC, "vmf: dopri5 step size underflow");
      }
    }
    ex.copy64(nodes, h->vmf_y, h->vmf_n);
    h->vmf_h = h_try;
    h->t = t1;
  }
  for (int k = 0; k < 7; ++k) h->vmf_k[k] = K[k];
  h->envs_dirty = true;  // the top-down class slots hold the transformed environments
  ex.run(3, 0.0, [&] { launch_check_finite(h->h_bufs[0], h->plan.P[0], h->flag_dev, h->stream); });
  CUDA_TRY(h, cudaGetLastError());
  return TTN_OK;
}

}  // namespace

extern "C" {

static ttn_status step_impl(ttn_t h, double dt, int32_t scheme, int32_t n_steps) {
  return guarded(h, [&]() -> ttn_status {
    if (!h->ws_bound) return h->fail(TTN_ESTATE, "bind the workspace first");
    if (!(std::isfinite(dt)) || dt <= 0 || n_steps < 0) return h->fail(TTN_EINVAL, "bad dt or n_steps");
    if (scheme != TTN_PS1 && scheme != TTN_PS2 && scheme != TTN_VMF && scheme != TTN_MIX)
      return h->fail(TTN_EINVAL, "unknown scheme");
    if (scheme == TTN_VMF) return vmf_steps(h, dt, n_steps);
    if (scheme == TTN_MIX) {  // ps2 until a bond reaches max_rank, then vmf at those ranks
      for (int k = 0; k < n_steps; ++k) {
        if (h->mix_switched) {
          ttn_status st = vmf_steps(h, dt, 1);
          if (st != TTN_OK) return st;
          continue;
        }
        ttn_status st = step_impl(h, dt, TTN_PS2, 1);
        if (st != TTN_OK) return st;
        int rmax = 0;
        for (int u = 1; u < h->plan.tree.n_nodes; ++u) rmax = std::max(rmax, h->plan.ranks[u]);
        if (rmax >= h->params.max_rank) h->mix_switched = true;
      }
      return TTN_OK;
    }
    if (scheme == TTN_PS2) {
      ttn_status st = ensure_envs(h);
      if (st != TTN_OK) return st;
      Exec ex(h);
      for (int k = 0; k < n_steps; ++k) {
        ex.step_ps2(dt, h->t);
        if (ex.err != cudaSuccess || ex.fail_st != TTN_OK) cudaStreamSynchronize(h->stream);  // drain what was issued
        if (ex.err != cudaSuccess) return cuda_fail(h, ex.err, "ps2 step");
        if (ex.fail_st != TTN_OK) return h->fail(ex.fail_st, ex.fail_msg);
        h->t += dt;
      }
      ex.run(3, 0.0, [&] { launch_check_finite(h->h_bufs[0], h->plan.P[0], h->flag_dev, h->stream); });
      CUDA_TRY(h, cudaGetLastError());
      return TTN_OK;
    }
    if (h->plan.n_sub(dt, h->params.kappa) > (1 << 20))
      return h->fail(TTN_EINVAL, "dt * Lambda needs more than 2^20 RK4 substeps");
    ttn_status st = ensure_envs(h);
    if (st != TTN_OK) return st;
    Exec ex(h);
    int k = 0;
    const bool graphable = ensure_graph(h, dt);
    if (graphable && h->graph) {
      for (; k < n_steps; ++k) {
        CUDA_TRY(h, cudaGraphLaunch(h->graph, h->stream));
        if (h->graph_prof == 2) CUDA_TRY(h, h->read_graph_marks());
        for (int c = 0; c < 4; ++c) {
          h->n_launch[c] += h->graph_launch[c];
          h->n_flops[c] += h->graph_flops[c];
        }
        h->t += dt;
      }
    }
    for (; k < n_steps; ++k) {
      ex.step_ps1(dt, h->t);
      h->t += dt;
    }
    ex.run(3, 0.0, [&] { launch_check_finite(h->h_bufs[0], h->plan.P[0], h->flag_dev, h->stream); });
    CUDA_TRY(h, cudaGetLastError());
    return TTN_OK;
  });
}

// ps2, vmf and mix run under host control (they synchronise at every split or
// step attempt): a call that fails part-way with TTN_ETIMEOUT or TTN_ENUMERIC
// puts the handle back to the state it had before the call (time, ranks and
// node tensors from a checkpoint blob taken at its start). ps1 steps are
// asynchronous, so their failures are reported by a later call.
ttn_status ttn_step(ttn_t h, double dt, int32_t scheme, int32_t n_steps) {
  if (!h) return TTN_EINVAL;
  const bool sync_scheme = scheme == TTN_PS2 || scheme == TTN_VMF || scheme == TTN_MIX;
  if (!sync_scheme || !h->ws_bound || !h->sop_loaded || n_steps <= 0) return step_impl(h, dt, scheme, n_steps);
  std::vector<char> snap;
  size_t bytes = 0;
  if (ttn_checkpoint_size(h, &bytes) == TTN_OK) {
    snap.resize(bytes);
    if (ttn_checkpoint_save(h, snap.data(), bytes) != TTN_OK) snap.clear();
  }
  const bool mix0 = h->mix_switched;
  const ttn_status st = step_impl(h, dt, scheme, n_steps);
  if ((st == TTN_ETIMEOUT || st == TTN_ENUMERIC) && !snap.empty()) {
    const std::string msg = h->err;
    cudaStreamSynchronize(h->stream);
    if (ttn_checkpoint_load(h, snap.data(), snap.size()) == TTN_OK) {
      h->mix_switched = mix0;
      h->err = msg + " (state put back to the start of the call)";
    } else {
      h->err = msg + " (the state could not be put back: " + h->err + ")";
    }
  }
  return st;
}

static ttn_status check_flag(ttn_t h) {
  int flag = 0;
  CUDA_TRY(h, cudaMemcpyAsync(&flag, h->flag_dev, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  if (flag & 2) return h->fail(TTN_ETIMEOUT, "a cluster or grid exchange of the QR kernels gave up");
  if (flag & 8) return h->fail(TTN_ETIMEOUT, "a tensor-core MMA wait gave up after 1 s");
  if (flag & 16) return h->fail(TTN_ETIMEOUT, "a grid barrier of the Jacobi SVD gave up after wait_s");
  if (flag) return h->fail(TTN_ENUMERIC, "non-finite amplitude in the root tensor");
  return TTN_OK;
}

ttn_status ttn_rdm_device(ttn_t h, void* rho_dev) {
  return guarded(h, [&]() -> ttn_status {
    if (!h->ws_bound) return h->fail(TTN_ESTATE, "bind the workspace first");
    if (!rho_dev) return h->fail(TTN_EINVAL, "null output");
    Exec ex(h);
    ex.rdm((double2*)rho_dev);
    CUDA_TRY(h, cudaGetLastError());
    return TTN_OK;
  });
}

ttn_status ttn_rdm(ttn_t h, double* rho_out) {
  return guarded(h, [&]() -> ttn_status {
    if (!h->ws_bound) return h->fail(TTN_ESTATE, "bind the workspace first");
    if (!rho_out) return h->fail(TTN_EINVAL, "null output");
    Exec ex(h);
    ex.rdm(h->rho_dev);
    const int M = h->plan.leg_dims[0];
    CUDA_TRY(h, cudaGetLastError());
    CUDA_TRY(h, cudaMemcpyAsync(rho_out, h->rho_dev, (size_t)M * M * sizeof(double2), cudaMemcpyDeviceToHost,
                                h->stream));
    return check_flag(h);
  });
}

ttn_status ttn_get_ranks(ttn_t h, int32_t* ranks_out) {
  if (!h || !ranks_out) return TTN_EINVAL;
  for (int u = 0; u < h->plan.tree.n_nodes; ++u) ranks_out[u] = u == 0 ? 0 : h->plan.ranks[u];
  return TTN_OK;
}

ttn_status ttn_node_shape(ttn_t h, int32_t u, int32_t* dims3) {
  if (!h || !dims3) return TTN_EINVAL;
  if (u < 0 || u >= h->plan.tree.n_nodes) return h->fail(TTN_EINVAL, "node out of range");
  for (int i = 0; i < 3; ++i) dims3[i] = h->plan.dims[u][i];
  return TTN_OK;
}

ttn_status ttn_get_node(ttn_t h, int32_t u, double* host_out) {
  return guarded(h, [&]() -> ttn_status {
    if (!h->ws_bound) return h->fail(TTN_ESTATE, "bind the workspace first");
    if (u < 0 || u >= h->plan.tree.n_nodes || !host_out) return h->fail(TTN_EINVAL, "bad node or output");
    CUDA_TRY(h, cudaMemcpyAsync(host_out, h->h_bufs[u], h->plan.P[u] * sizeof(double2), cudaMemcpyDeviceToHost,
                                h->stream));
    return check_flag(h);
  });
}

ttn_status ttn_set_node(ttn_t h, int32_t u, const double* host_in) {
  return guarded(h, [&]() -> ttn_status {
    if (!h->ws_bound) return h->fail(TTN_ESTATE, "bind the workspace first");
    if (u < 0 || u >= h->plan.tree.n_nodes || !host_in) return h->fail(TTN_EINVAL, "bad node or input");
    for (int64_t i = 0; i < 2 * h->plan.P[u]; ++i)
      if (!std::isfinite(host_in[i])) return h->fail(TTN_EINVAL, "non-finite node entry");
    ttn_status st = upload_pair(h, h->h_bufs[u], h->h_bufs_lo[u], (const double2*)host_in, (size_t)h->plan.P[u]);
    if (st != TTN_OK) return st;
    h->envs_dirty = true;
    return TTN_OK;
  });
}

ttn_status ttn_time(ttn_t h, double* t) {
  if (!h || !t) return TTN_EINVAL;
  *t = h->t;
  return TTN_OK;
}

}  // extern "C"

namespace {

// Checkpoint blob: header, the topology and generator fingerprint that a
// loading handle must match, the time, the effective ranks, then every node
// tensor (complex128, canonical layout) in node order.
constexpr char kCkptMagic[8] = {'T', 'T', 'N', 'C', 'K', 'P', 'T', '1'};
struct CkptHead {
  char magic[8];
  int32_t version, n_nodes, n_legs, precision;
  uint64_t sop_hash;
  double t;
};

// FNV-1a over the loaded generator: operators (leg, entries), terms
// (coefficient, drive, factors), drive bounds.
uint64_t sop_fingerprint(const Plan& p) {
  uint64_t hsh = 1469598103934665603ull;
  auto mix = [&](const void* data, size_t n) {
    const unsigned char* b = (const unsigned char*)data;
    for (size_t i = 0; i < n; ++i) {
      hsh ^= b[i];
      hsh *= 1099511628211ull;
    }
  };
  for (size_t k = 0; k < p.ops.size(); ++k) {
    mix(&p.op_leg[k], sizeof(int));
    mix(p.ops[k].data(), p.ops[k].size() * sizeof(cd));
  }
  for (const RawTerm& t : p.terms) {
    mix(&t.coef, sizeof(cd));
    mix(&t.drive, sizeof(int));
    for (const Factor& f : t.f) {
      mix(&f.leg, sizeof(int));
      mix(&f.op, sizeof(int));
    }
  }
  mix(p.drive_bound.data(), p.drive_bound.size() * sizeof(double));
  return hsh;
}

size_t ckpt_bytes(const Plan& p) {
  size_t n = sizeof(CkptHead) + sizeof(int32_t) * (2 * p.tree.n_nodes + 2 * p.tree.n_legs);
  for (int u = 0; u < p.tree.n_nodes; ++u) n += (size_t)p.P[u] * sizeof(double2);
  return n;
}

}  // namespace

extern "C" {

ttn_status ttn_checkpoint_size(ttn_t h, size_t* bytes) {
  if (!h || !bytes) return TTN_EINVAL;
  if (!h->ws_bound) return h->fail(TTN_ESTATE, "bind the workspace first");
  *bytes = ckpt_bytes(h->plan);
  return TTN_OK;
}

ttn_status ttn_checkpoint_save(ttn_t h, void* host_buf, size_t bytes) {
  return guarded(h, [&]() -> ttn_status {
    if (!h->ws_bound) return h->fail(TTN_ESTATE, "bind the workspace first");
    const Plan& p = h->plan;
    if (!host_buf || bytes < ckpt_bytes(p)) return h->fail(TTN_EINVAL, "checkpoint buffer missing or too small");
    char* o = (char*)host_buf;
    CkptHead hd{};
    std::memcpy(hd.magic, kCkptMagic, 8);
    hd.version = 1;
    hd.n_nodes = p.tree.n_nodes;
    hd.n_legs = p.tree.n_legs;
    hd.precision = h->precision;
    hd.sop_hash = sop_fingerprint(p);
    hd.t = h->t;
    std::memcpy(o, &hd, sizeof(hd));
    o += sizeof(hd);
    auto put_ints = [&](const std::vector<int>& v) {
      for (int x : v) {
        const int32_t y = x;
        std::memcpy(o, &y, sizeof(y));
        o += sizeof(y);
      }
    };
    put_ints(p.tree.parent);
    put_ints(p.tree.leg_node);
    put_ints(p.leg_dims);
    put_ints(p.ranks);
    for (int u = 0; u < p.tree.n_nodes; ++u) {
      CUDA_TRY(h, cudaMemcpyAsync(o, h->h_bufs[u], (size_t)p.P[u] * sizeof(double2), cudaMemcpyDeviceToHost,
                                  h->stream));
      o += (size_t)p.P[u] * sizeof(double2);
    }
    return check_flag(h);
  });
}

ttn_status ttn_checkpoint_load(ttn_t h, const void* host_buf, size_t bytes) {
  return guarded(h, [&]() -> ttn_status {
    if (!h->ws_bound) return h->fail(TTN_ESTATE, "bind the workspace first");
    Plan& p = h->plan;
    const int n = p.tree.n_nodes, nl = p.tree.n_legs;
    const size_t fixed = sizeof(CkptHead) + sizeof(int32_t) * (2 * n + 2 * nl);
    if (!host_buf || bytes < fixed) return h->fail(TTN_EINVAL, "checkpoint too short");
    const char* in = (const char*)host_buf;
    CkptHead hd;
    std::memcpy(&hd, in, sizeof(hd));
    in += sizeof(hd);
    if (std::memcmp(hd.magic, kCkptMagic, 8) != 0 || hd.version != 1)
      return h->fail(TTN_EINVAL, "not a TTN checkpoint (magic / version)");
    if (hd.n_nodes != n || hd.n_legs != nl) return h->fail(TTN_EINVAL, "checkpoint tree size differs");
    if (hd.sop_hash != sop_fingerprint(p))
      return h->fail(TTN_EINVAL, "checkpoint was written under another generator (operators, terms or drives)");
    if (!std::isfinite(hd.t)) return h->fail(TTN_EINVAL, "non-finite checkpoint time");
    auto get_ints = [&](int k) {
      std::vector<int> v(k);
      for (int i = 0; i < k; ++i) {
        int32_t y;
        std::memcpy(&y, in, sizeof(y));
        in += sizeof(y);
        v[i] = y;
      }
      return v;
    };
    const std::vector<int> parent = get_ints(n), leg_node = get_ints(nl), dims = get_ints(nl), ranks = get_ints(n);
    if (parent != p.tree.parent || leg_node != p.tree.leg_node || dims != p.leg_dims)
      return h->fail(TTN_EINVAL, "checkpoint topology or leg dimensions differ");
    for (int u = 1; u < n; ++u)
      if (ranks[u] < 1 || ranks[u] > p.caps[u])
        return h->fail(TTN_EINVAL, "checkpoint rank beyond this handle's capacity (max_rank)");
    // adopt the saved ranks (as a ps2 rank change does), then the tensors
    if (ranks != p.ranks) {
      Exec ex(h);
      p.ranks = ranks;
      p.update_dims();
      p.build_jobs();
      ex.upload_jobs();
      if (ex.err != cudaSuccess) return cuda_fail(h, ex.err, "job upload");
    }
    size_t need = fixed;
    for (int u = 0; u < n; ++u) need += (size_t)p.P[u] * sizeof(double2);
    if (bytes < need) return h->fail(TTN_EINVAL, "checkpoint truncated");
    const double* vals = (const double*)in;
    for (size_t i = 0; i < (need - fixed) / sizeof(double); ++i)
      if (!std::isfinite(vals[i])) return h->fail(TTN_EINVAL, "non-finite checkpoint entry");
    for (int u = 0; u < n; ++u) {
      ttn_status st = upload_pair(h, h->h_bufs[u], h->h_bufs_lo[u], (const double2*)in, (size_t)p.P[u]);
      if (st != TTN_OK) return st;
      in += (size_t)p.P[u] * sizeof(double2);
    }
    h->t = hd.t;
    h->envs_dirty = true;
    h->drop_graph();
    CUDA_TRY(h, cudaMemsetAsync(h->flag_dev, 0, sizeof(int), h->stream));
    return ensure_envs(h);
  });
}

ttn_status ttn_substeps(ttn_t h, double tau, int32_t* m) {
  if (!h || !m) return TTN_EINVAL;
  if (!h->sop_loaded) return h->fail(TTN_ESTATE, "sop_load first");
  *m = h->plan.n_sub(tau, h->params.kappa);
  return TTN_OK;
}

ttn_status ttn_batch_step(ttn_t* hs, int32_t n, double dt, int32_t scheme, int32_t n_steps) {
  if (!hs || n < 0) return TTN_EINVAL;
  if (n == 0 || n_steps == 0) return TTN_OK;
  for (int i = 0; i < n; ++i)
    if (!hs[i]) return TTN_EINVAL;
  ttn_t h0 = hs[0];
  return guarded(h0, [&]() -> ttn_status {
    if (!(std::isfinite(dt)) || dt <= 0 || n_steps < 0) return h0->fail(TTN_EINVAL, "bad dt or n_steps");
    for (int i = 0; i < n; ++i) {
      for (int j = 0; j < i; ++j)
        if (hs[j] == hs[i]) return h0->fail(TTN_EINVAL, "a handle appears twice in the batch");
      if (!hs[i]->ws_bound) return h0->fail(TTN_ESTATE, "a handle in the batch has no workspace");
    }
    // every member as one concurrent branch of a parent graph (ps1, autonomous)
    bool all_graphs = scheme == TTN_PS1;
    for (int i = 0; i < n && all_graphs; ++i) {
      ttn_status st = ensure_envs(hs[i]);
      if (st != TTN_OK) return h0->fail(st, std::string("batch member: ") + hs[i]->err);
      if (hs[i]->plan.n_sub(dt, hs[i]->params.kappa) > (1 << 20)) return h0->fail(TTN_EINVAL, "dt too large");
      all_graphs = hs[i]->prof_mode == 0 && ensure_graph(hs[i], dt);
    }
    if (!all_graphs) {  // drives, default streams or profiling: one handle after another
      for (int i = 0; i < n; ++i) {
        ttn_status st = ttn_step(hs[i], dt, scheme, n_steps);
        if (st != TTN_OK) return h0->fail(st, std::string("batch member: ") + hs[i]->err);
      }
      return TTN_OK;
    }
    bool same = h0->batch_exec && h0->batch_dt == dt && (int)h0->batch_members.size() == n;
    for (int i = 0; same && i < n; ++i)
      same = h0->batch_members[i] == hs[i] && h0->batch_member_graphs[i] == hs[i]->graph;
    if (!same) {
      h0->drop_batch();
      cudaGraph_t parent = nullptr;
      CUDA_TRY(h0, cudaGraphCreate(&parent, 0));
      for (int i = 0; i < n; ++i) {
        cudaGraphNode_t node;
        cudaError_t e = cudaGraphAddChildGraphNode(&node, parent, nullptr, 0, hs[i]->graph_src);
        if (e != cudaSuccess) {
          cudaGraphDestroy(parent);
          return cuda_fail(h0, e, "cudaGraphAddChildGraphNode");
        }
      }
      cudaError_t e = cudaGraphInstantiate(&h0->batch_exec, parent, 0);
      cudaGraphDestroy(parent);
      if (e != cudaSuccess) return cuda_fail(h0, e, "cudaGraphInstantiate (batch)");
      h0->batch_dt = dt;
      for (int i = 0; i < n; ++i) {
        h0->batch_members.push_back(hs[i]);
        h0->batch_member_graphs.push_back(hs[i]->graph);
      }
    }
    // order the batch after earlier work on every member stream, and later work after it
    cudaStream_t s0 = h0->stream;
    std::vector<cudaEvent_t> evs;
    for (int i = 1; i < n; ++i)
      if (hs[i]->stream != s0) {
        cudaEvent_t ev;
        CUDA_TRY(h0, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        evs.push_back(ev);
        CUDA_TRY(h0, cudaEventRecord(ev, hs[i]->stream));
        CUDA_TRY(h0, cudaStreamWaitEvent(s0, ev, 0));
      }
    for (int k = 0; k < n_steps; ++k) CUDA_TRY(h0, cudaGraphLaunch(h0->batch_exec, s0));
    for (int i = 0; i < n; ++i) {
      ttn_t h = hs[i];
      for (int c = 0; c < 4; ++c) {
        h->n_launch[c] += (int64_t)n_steps * h->graph_launch[c];
        h->n_flops[c] += n_steps * h->graph_flops[c];
      }
      h->t += n_steps * dt;
      launch_check_finite(h->h_bufs[0], h->plan.P[0], h->flag_dev, s0);
    }
    cudaEvent_t done;
    CUDA_TRY(h0, cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
    CUDA_TRY(h0, cudaEventRecord(done, s0));
    for (int i = 1; i < n; ++i)
      if (hs[i]->stream != s0) CUDA_TRY(h0, cudaStreamWaitEvent(hs[i]->stream, done, 0));
    cudaEventDestroy(done);  // destruction is deferred until the event completes
    for (auto ev : evs) cudaEventDestroy(ev);
    CUDA_TRY(h0, cudaGetLastError());
    return TTN_OK;
  });
}

ttn_status ttn_batch_autotune(ttn_t* hs, int32_t n, double dt, int32_t reps, int32_t* warps_out, float* ms_out) {
  if (!hs || n < 1 || reps < 1 || reps > 100) return TTN_EINVAL;
  for (int i = 0; i < n; ++i)
    if (!hs[i]) return TTN_EINVAL;
  ttn_t h0 = hs[0];
  return guarded(h0, [&]() -> ttn_status {
    if (!(std::isfinite(dt)) || dt <= 0) return h0->fail(TTN_EINVAL, "bad dt");
    // every member's state and statistics, to be put back after the timed steps
    std::vector<std::vector<char>> saved(n);
    std::vector<std::array<int64_t, 4>> saved_launch(n);
    std::vector<std::array<double, 4>> saved_flops(n);
    for (int i = 0; i < n; ++i)
      for (int c = 0; c < 4; ++c) {
        saved_launch[i][c] = hs[i]->n_launch[c];
        saved_flops[i][c] = hs[i]->n_flops[c];
      }
    for (int i = 0; i < n; ++i) {
      size_t b = 0;
      ttn_status st = ttn_checkpoint_size(hs[i], &b);
      if (st == TTN_OK) {
        saved[i].resize(b);
        st = ttn_checkpoint_save(hs[i], saved[i].data(), b);
      }
      if (st != TTN_OK) return h0->fail(st, std::string("batch member: ") + hs[i]->err);
    }
    auto set_warps = [&](int w) -> ttn_status {
      for (int i = 0; i < n; ++i) {
        ttn_params q = hs[i]->params;
        q.tile_warps = w;
        ttn_status st = ttn_set_params(hs[i], &q);
        if (st != TTN_OK) return h0->fail(st, std::string("batch member: ") + hs[i]->err);
      }
      return TTN_OK;
    };
    cudaEvent_t e0, e1;
    CUDA_TRY(h0, cudaEventCreate(&e0));
    CUDA_TRY(h0, cudaEventCreate(&e1));
    const int cand[3] = {8, 4, 2};
    int best = 8;
    float tb = 3.4e38f;
    ttn_status st = TTN_OK;
    for (int c = 0; c < 3 && st == TTN_OK; ++c) {
      st = set_warps(cand[c]);
      if (st == TTN_OK) st = ttn_batch_step(hs, n, dt, TTN_PS1, 1);  // capture + warm-up
      if (st != TTN_OK) break;
      cudaEventRecord(e0, h0->stream);
      st = ttn_batch_step(hs, n, dt, TTN_PS1, reps);
      cudaEventRecord(e1, h0->stream);
      if (st != TTN_OK || cudaEventSynchronize(e1) != cudaSuccess) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms_out) ms_out[c] = ms / reps;
      if (ms < 0.97f * tb) {  // the planned shape first: another must win by 3 %
        tb = ms;
        best = cand[c];
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != TTN_OK) return st;
    CUDA_TRY(h0, cudaGetLastError());
    st = set_warps(best);
    for (int i = 0; i < n && st == TTN_OK; ++i) {
      st = ttn_checkpoint_load(hs[i], saved[i].data(), saved[i].size());
      if (st != TTN_OK) return h0->fail(st, std::string("batch member: ") + hs[i]->err);
      for (int c = 0; c < 4; ++c) {
        hs[i]->n_launch[c] = saved_launch[i][c];
        hs[i]->n_flops[c] = saved_flops[i][c];
      }
    }
    if (warps_out) *warps_out = best;
    return st;
  });
}

ttn_status ttn_stats(ttn_t h, int32_t kind, int64_t* launches, double* flops) {
  if (!h || kind < 0 || kind > 4) return TTN_EINVAL;
  if (kind == 4) {
    if (launches) *launches = h->n_ring;
    if (flops) *flops = 0.0;
    return TTN_OK;
  }
  if (launches) *launches = h->n_launch[kind];
  if (flops) *flops = h->n_flops[kind];
  return TTN_OK;
}

ttn_status ttn_profile(ttn_t h, int32_t on) {
  if (!h) return TTN_EINVAL;
  if (on < 0 || on > 2) return TTN_EINVAL;
  h->prof_mode = on;
  h->profiling = on == 1;
  return TTN_OK;
}

ttn_status ttn_profile_read(ttn_t h, int32_t kind, double* ms) {
  if (!h || kind < 0 || kind > 3 || !ms) return TTN_EINVAL;
  CUDA_TRY(h, h->drain_marks());
  *ms = h->prof_ms[kind];
  return TTN_OK;
}

namespace {
using TuneKey = std::array<int32_t, 9>;
TuneKey ap_key(const Plan& p, const ApList& L, int prec) {
  const ApOut& o = p.ap_outs[L.out_begin];
  const int nt = p.ap_outs[L.out_end - 1].term_end - o.term_begin;
  return {0, prec, o.d0, o.d1, o.d2, o.d3, L.out_end - L.out_begin, nt, L.n_tiles};
}
TuneKey pj_key(const Plan& p, const PjList& L, int prec) {
  const PjOut& o = p.pj_outs[L.out_begin];
  return {1, prec, o.d0, o.d1, o.d2, o.leg, L.out_end - L.out_begin, 0, L.n_tiles};
}
// precision each apply list runs in (absorb lists are FP64 in both forms)
std::vector<int> ap_precs(const Plan& p, int prec) {
  std::vector<int> pr(p.ap_lists.size(), prec);
  for (const auto& a : p.absorb)
    for (int id : a)
      if (id >= 0) pr[id] = PREC_F64;
  return pr;
}
}  // namespace

ttn_status ttn_autotune(ttn_t h, int32_t reps) {
  return guarded(h, [&]() -> ttn_status {
    if (!h->ws_bound) return h->fail(TTN_ESTATE, "bind the workspace first");
    if (reps < 1 || reps > 100) return h->fail(TTN_EINVAL, "reps must be 1..100");
    Plan& p = h->plan;
    cudaStream_t s = h->stream;
    std::vector<char> f64(p.ap_lists.size(), 0);  // absorb lists run in FP64 in both forms
    for (const auto& a : p.absorb)
      for (int id : a)
        if (id >= 0) f64[id] = 1;
    cudaEvent_t e0, e1;
    CUDA_TRY(h, cudaEventCreate(&e0));
    CUDA_TRY(h, cudaEventCreate(&e1));
    auto time_of = [&](auto&& launch) -> float {
      launch();  // warm
      cudaEventRecord(e0, s);
      for (int r = 0; r < reps; ++r) launch();
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      return ms;
    };
    // lists writing scratch outputs run as they are; lists with an RK
    // epilogue run as stage 1 into scratch (tmp read, acc / ys2 written), so
    // the state is untouched; the environment matrices the projections
    // overwrite are rebuilt before the next step
    const Epi store{EPI_STORE, nullptr, nullptr, nullptr, nullptr, 0.0};
    const Epi rk1{EPI_RK1, h->h_bufs[p.buf.tmp], h->h_bufs_lo[p.buf.tmp], h->h_bufs_lo[p.buf.ys2],
                  h->h_bufs[p.buf.acc], 0.0};
    const int cap = std::min(kMaxSplit, h->params.max_split);
    std::map<TuneKey, std::pair<int, int>> done;  // shape chosen per list key
    for (size_t i = 0; i < p.ap_lists.size(); ++i) {
      ApList& L = p.ap_lists[i];
      if (L.n_tiles <= 0) continue;
      const int prec = f64[i] ? PREC_F64 : h->prec;
      const DevTables& T = f64[i] ? h->T : h->Tlo;
      if (!f64[i] && h->prec == PREC_F32 && h->params.tensor_cores &&
          tc_applicable(L, p.ap_outs.data(), p.ap_terms.data()))
        continue;
      const bool epi = p.ap_outs[L.out_begin].dst < 0;
      const TuneKey key = ap_key(p, L, prec);
      auto seen = done.find(key);
      if (seen != done.end()) {  // lists of one shape share one tuning
        L.w = seen->second.first;
        L.k = seen->second.second;
        L.useful = (L.units + L.w - 1) / L.w;
        continue;
      }
      int best_w = kSplitWarps, best_k = 1;
      float tb = 3.4e38f;
      for (int w : {8, 4, 2}) {  // the planned shape first: another must win by 3 %
        const int useful = (L.units + w - 1) / w;
        // splits only pay below a few CTAs per SM: larger lists keep one CTA per tile
        const int kmax = std::max(1, std::min(std::min(useful, cap), (32 / w) * p.sm_count / L.n_tiles));
        for (int k = 1; k <= kmax; ++k) {
          ApList L2 = L;
          L2.w = w;
          L2.k = k;
          L2.useful = useful;
          const float t = time_of([&] { launch_apply(prec, T, L2, epi ? rk1 : store, s); });
          if (t < 0.97f * tb) {
            tb = t;
            best_w = w;
            best_k = k;
          }
        }
      }
      L.w = best_w;
      L.k = best_k;
      L.useful = (L.units + best_w - 1) / best_w;
      done.emplace(key, std::make_pair(best_w, best_k));
    }
    for (PjList& L : p.pj_lists) {
      if (L.n_tiles <= 0) continue;
      const TuneKey key = pj_key(p, L, h->prec);
      auto seen = done.find(key);
      if (seen != done.end()) {
        L.k = seen->second.second;
        continue;
      }
      int best = L.k;
      float tb = 3.4e38f;
      const int kmax = std::max(1, std::min(std::min(L.useful, cap), 4 * p.sm_count / L.n_tiles));
      if (kmax == 1) {
        L.k = 1;
        done.emplace(key, std::make_pair(kSplitWarps, 1));
        continue;
      }
      for (int k = 1; k <= kmax; ++k) {
        PjList L2 = L;
        L2.k = k;
        const float t = time_of([&] { launch_project(h->prec, h->Tlo, L2, s); });
        if (t < 0.97f * tb) {
          tb = t;
          best = k;
        }
      }
      L.k = best;
      done.emplace(key, std::make_pair(kSplitWarps, best));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CUDA_TRY(h, cudaGetLastError());
    h->envs_dirty = true;
    h->drop_graph();
    return TTN_OK;
  });
}


ttn_status ttn_tuning_get(ttn_t h, int32_t* rows, int32_t max_rows, int32_t* n_rows) {
  if (!h || !n_rows || max_rows < 0 || (max_rows > 0 && !rows)) return TTN_EINVAL;
  return guarded(h, [&]() -> ttn_status {
    if (!h->sop_loaded) return h->fail(TTN_ESTATE, "sop_load first");
    const Plan& p = h->plan;
    const std::vector<int> pr = ap_precs(p, h->prec);
    int n = 0;
    auto put = [&](const TuneKey& k, int w, int kk) {
      if (n < max_rows) {
        int32_t* r = rows + (size_t)n * TTN_TUNING_COLS;
        for (int i = 0; i < 9; ++i) r[i] = k[i];
        r[9] = w;
        r[10] = kk;
      }
      ++n;
    };
    for (size_t i = 0; i < p.ap_lists.size(); ++i) put(ap_key(p, p.ap_lists[i], pr[i]), p.ap_lists[i].w, p.ap_lists[i].k);
    for (const PjList& L : p.pj_lists) put(pj_key(p, L, h->prec), kSplitWarps, L.k);
    *n_rows = n;
    return TTN_OK;
  });
}

ttn_status ttn_tuning_set(ttn_t h, const int32_t* rows, int32_t n_rows, int32_t* n_applied) {
  if (!h || n_rows < 0 || (n_rows > 0 && !rows)) return TTN_EINVAL;
  return guarded(h, [&]() -> ttn_status {
    if (!h->sop_loaded) return h->fail(TTN_ESTATE, "sop_load first");
    const int cap = std::min(kMaxSplit, h->params.max_split);
    std::map<TuneKey, std::pair<int, int>> shape;
    for (int i = 0; i < n_rows; ++i) {
      const int32_t* r = rows + (size_t)i * TTN_TUNING_COLS;
      const int w = r[9], k = r[10];
      const bool w_ok = r[0] == 0 ? (w == 2 || w == 4 || w == 8) : (r[0] == 1 && w == kSplitWarps);
      if (!w_ok || k < 1 || k > cap) return h->fail(TTN_EINVAL, "tuning row " + std::to_string(i) + " out of range");
      TuneKey key;
      for (int j = 0; j < 9; ++j) key[j] = r[j];
      shape.emplace(key, std::make_pair(w, k));  // the first row of a key wins
    }
    Plan& p = h->plan;
    const std::vector<int> pr = ap_precs(p, h->prec);
    int applied = 0;
    for (size_t i = 0; i < p.ap_lists.size(); ++i) {
      ApList& L = p.ap_lists[i];
      auto it = shape.find(ap_key(p, L, pr[i]));
      if (it == shape.end()) continue;
      L.w = it->second.first;
      L.k = it->second.second;
      L.useful = (L.units + L.w - 1) / L.w;
      ++applied;
    }
    for (PjList& L : p.pj_lists) {
      auto it = shape.find(pj_key(p, L, h->prec));
      if (it == shape.end()) continue;
      L.k = it->second.second;
      ++applied;
    }
    if (n_applied) *n_applied = applied;
    h->drop_graph();
    return TTN_OK;
  });
}

ttn_status ttn_stats_reset(ttn_t h) {
  if (!h) return TTN_EINVAL;
  CUDA_TRY(h, h->drain_marks());
  h->n_ring = 0;
  for (int k = 0; k < 4; ++k) {
    h->n_launch[k] = 0;
    h->n_flops[k] = 0;
    h->prof_ms[k] = 0;
  }
  return TTN_OK;
}

ttn_status ttn_split_log(ttn_t h, float* feats, int32_t* labels, int32_t max, int32_t* n_total) {
  if (!h || !n_total || max < 0) return TTN_EINVAL;
  const int n = (int)h->log_labels.size();
  *n_total = n;
  const int k = std::min(n, (int)max);
  if (feats && k > 0) std::memcpy(feats, h->log_feats.data(), (size_t)k * 24 * sizeof(float));
  if (labels && k > 0) std::memcpy(labels, h->log_labels.data(), (size_t)k * sizeof(int32_t));
  return TTN_OK;
}

ttn_status ttn_split_log_clear(ttn_t h) {
  if (!h) return TTN_EINVAL;
  h->log_feats.clear();
  h->log_labels.clear();
  return TTN_OK;
}

ttn_status ttn_set_rank_proposer(ttn_t h, const float* params_dev) {
  if (!h) return TTN_EINVAL;
  h->proposer = params_dev;
  return TTN_OK;
}

ttn_status ttn_proposer_stats(ttn_t h, int64_t* proposed, int64_t* accepted) {
  if (!h) return TTN_EINVAL;
  if (proposed) *proposed = h->n_proposed;
  if (accepted) *accepted = h->n_accepted;
  return TTN_OK;
}

const char* ttn_last_error(ttn_t h) { return h ? h->err.c_str() : "null handle"; }

void ttn_destroy(ttn_t h) { delete h; }

}  // extern "C"
