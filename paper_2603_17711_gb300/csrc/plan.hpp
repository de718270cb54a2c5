// Host-side planning for the TTN-HEOM library: tree canonicalisation, bond-rank
// caps, SOP merging into per-bond operator classes, and the static job lists
// that the CUDA kernels execute. Pure C++17 (no CUDA), so it is testable on
// any host.
#pragma once

#include <array>
#include <complex>
#include <cstdint>
#include <string>
#include <vector>

namespace ttn {

using cd = std::complex<double>;

// Leg of a node in canonical order: 'p' parent bond, 'n' child node, 'o' open leg.
struct Leg {
  char kind;
  int v;
};

struct Tree {
  int n_nodes = 0, n_legs = 0;
  std::vector<int> parent, leg_node;
  std::vector<std::vector<int>> children;  // child nodes in canonical leg order
  std::vector<std::vector<Leg>> legs;      // canonical leg order per node
  std::vector<std::vector<char>> below;    // below[u][l] = open leg l lies under u
  std::vector<int> postorder;
  // returns "" on success, else an error message
  std::string build(int n_nodes, const int32_t* parent, int n_legs, const int32_t* leg_node);
  int leg_index(int u, int v) const;  // leg of u facing neighbour node v
};

// Effective bond ranks: min(requested, product of the other leg dims at either
// end), iterated to a fixed point. r[0] = 0.
std::vector<int> effective_ranks(const Tree& t, const std::vector<int>& leg_dims,
                                 const std::vector<int>& requested);

// One SOP term after validation.
struct Factor {
  int leg;
  int op;  // index into the operator table
};
struct RawTerm {
  cd coef;
  int drive;  // -1 static
  std::vector<Factor> f;
};

// ||M||_2 of a d x d complex matrix (cyclic Jacobi on M^H M).
double spectral_norm(const cd* M, int d);

// ---------------------------------------------------------------------------
// Operator classes. Every directed edge e (behind-set T) carries
//   S        : sum of all terms supported inside T            (kind 0)
//   X(key)   : the key factor, for keys inside T whose partners are not all in T   (kind 1)
//   P(key)   : sum of coef*partner factors inside T, for keys outside T            (kind 2)
// A "site" is either a directed bond (a -> b, behind = subtree behind a) or an
// open leg (behind = {leg}).
// ---------------------------------------------------------------------------
struct Key {
  int leg, op;
};

struct ClassId {
  int kind;  // 0 S, 1 X, 2 P
  int key;   // -1 for S
  bool operator==(const ClassId& o) const { return kind == o.kind && key == o.key; }
};

// A matrix slot: d x d complex in the device pool.
struct MatSlot {
  int d;
  int64_t off;  // complex elements from the pool base
};

// Local (open-leg) matrix with optional drive components.
struct LocalMat {
  int leg;
  ClassId cls;
  std::vector<cd> stat;                 // d*d static part
  std::vector<std::vector<cd>> drive;   // per drive id: d*d part (empty if none)
  bool time_dependent = false;
  int slot = -1;        // current matrix slot
  int slot_stat = -1;   // static part slot (time-dependent only)
  std::vector<int> slot_drive;  // per drive (time-dependent only, -1 if none)
};

// Term of a "sum of mode products" job: out += M x_leg src (M = -1: identity).
struct ApTerm {
  int32_t mat;
  int32_t leg;
  int32_t src;  // buffer id
  int32_t pad;
};
// One output tensor of an apply job list.
struct ApOut {
  int32_t d0, d1, d2;
  int32_t term_begin, term_end;
  int32_t dst;      // buffer id (STORE epilogue) or -1 (epilogue from kernel args)
  int32_t tile0;    // first global tile of this output
  int32_t d3;       // fourth leg (two-site tensors); 1 for node tensors
};
struct ApList {
  int32_t out_begin, out_end;  // into the global ApOut table
  int32_t n_tiles;
  int32_t k = 1;       // CTAs sharing one output tile (thread-block cluster size, 1..16)
  int32_t useful = 1;  // largest split that still gives every warp work (for w warps per CTA)
  int32_t w = 8;       // warps per CTA (2, 4 or 8): with k, the tile shape of the launch
  int32_t units = 1;   // work units of the list's largest output tile
  int32_t tpo = 0;     // tiles per output when every output has as many (tile -> output by one division), else 0
  double flops;        // algorithmic: 8 * P * d_leg per non-identity term and output
};
// Projection job: E[x',x] = sum_r conj(U[.. x' at leg ..]) W[.. x at leg ..].
struct PjOut {
  int32_t d0, d1, d2;
  int32_t leg;
  int32_t u_buf, w_buf;
  int32_t dst_mat;
  int32_t tile0;
};
struct PjList {
  int32_t out_begin, out_end;
  int32_t n_tiles;
  int32_t k = 1;       // CTAs sharing one output tile (thread-block cluster size, 1..16)
  int32_t useful = 1;  // largest split that still gives every warp >= 4 positions
  int32_t tpo = 0;     // tiles per output when every output has as many, else 0
  double flops;        // 8 * P * d_leg per output
};

// Buffer ids used by job lists. Node slots come first (0..n_nodes-1).
// The RK4 stage input is double-buffered (ys, ys2): a combine kernel reads its
// stage input along whole legs in other CTAs while its epilogue writes the next
// stage input, so the two must never be the same buffer.
struct BufIds {
  int ys, ys2, acc, tmp;  // node-sized scratch
  int t0, n_t;            // pair intermediates T_0..T_{n_t-1}
  int w0, n_w;            // env class outputs W_0..W_{n_w-1}
  int bond_y, bond_ys, bond_ys2, bond_acc;  // bond matrices as (1, d, d) tensors
  int th_y, th_ys, th_ys2, th_acc;          // two-site tensor Theta (ps2)
  int n_bufs;
};

// Job lists of one node flow / bond flow, per source: 0 = the state, 1 = ys, 2 = ys2.
struct FlowLists {
  int first[3] = {-1, -1, -1};    // ApList ids (pairs' first mode products), -1 if no pairs
  int combine[3] = {-1, -1, -1};  // ApList ids (sum with RK4 epilogue)
};
struct EnvLists {
  int first = -1;    // ApList id
  int classes = -1;  // ApList id producing W_c
  int project = -1;  // PjList id
};

struct Plan {
  // inputs
  Tree tree;
  std::vector<int> leg_dims, ranks;  // effective ranks
  std::vector<std::vector<cd>> ops;  // operator table (d*d each)
  std::vector<int> op_leg;
  std::vector<RawTerm> terms;
  int n_drives = 0;
  std::vector<double> drive_bound;
  double lambda = 0.0;

  // keys of two-factor terms
  std::vector<Key> keys;
  std::vector<int> term_key;      // key of a two-factor term (-1 otherwise)
  std::vector<int> term_partner;  // index of the partner factor in the term

  // node dims (3 legs) and sizes at the current ranks
  std::vector<std::array<int, 3>> dims;
  std::vector<int64_t> P;
  int64_t P_max = 0;
  int r_max = 0;
  // capacity (workspace sizing): ranks capped at max(requested, max_rank)
  std::vector<int> req, caps;
  std::vector<std::array<int, 3>> cap_dims;
  std::vector<int64_t> P_cap;
  int64_t P_cap_max = 0, theta_cap = 0;
  int r_cap_max = 1;
  int cap_rank = 32;
  int sm_count = 152;  // SMs of the device: sizes the per-tile CTA split of the job lists
  int max_split = 16;  // upper bound of that split (ttn_params.max_split; kMaxSplit below)
  int tile_warps = 0;  // warps per CTA of new apply lists (ttn_params.tile_warps; 0: kSplitWarps)

  // classes
  std::vector<std::vector<ClassId>> dir_classes;  // per directed bond id
  std::vector<std::vector<int>> dir_slots;        // matching matrix slots
  std::vector<LocalMat> locals;                   // open-leg matrices
  std::vector<MatSlot> mats;                      // all matrix slots in the pool
  int64_t mat_pool = 0;                           // complex elements
  int bond_mat = -1;                              // matrix id aliasing the bond buffer

  // job lists
  BufIds buf;
  std::vector<ApTerm> ap_terms;
  std::vector<ApOut> ap_outs;
  std::vector<ApList> ap_lists;
  std::vector<PjOut> pj_outs;
  std::vector<PjList> pj_lists;
  std::vector<FlowLists> node_flow;          // per node
  // per non-root node: the combine list of node_flow (source = the node) kept
  // to the terms with no factor on the parent leg (singles on the other legs,
  // pairs between the other legs; T_g as written by node_flow.first[0]); the
  // direct integration (vmf) weights these terms separately
  std::vector<int> node_down;
  std::vector<FlowLists> bond_flow;          // per directed bond (from -> to)
  std::vector<EnvLists> env;                 // per directed bond
  std::vector<std::array<int, 3>> absorb;    // per node: ApList id for R on leg li
  // ps2 two-site flows: per directed bond (first -> second), Theta legs = first's
  // other legs then second's other legs (canonical order, bond removed)
  std::vector<FlowLists> two_site;

  int dir_id(int a, int b) const;                 // a, b adjacent nodes
  std::vector<char> behind(int u, int li) const;  // open legs behind leg li of node u
  int slot_of(int u, int li, ClassId c) const;    // -1 if absent

  std::string build(int n_nodes, const int32_t* parent, int n_legs, const int32_t* leg_node,
                    const int32_t* leg_dims, const int32_t* ranks);
  std::string load_sop(int n_ops, const int32_t* op_leg, const int64_t* op_offset,
                       const double* op_data, int n_terms, const int32_t* term_offsets,
                       const int32_t* term_ops, const double* coef, const int32_t* coef_drive);
  void compute_lambda();
  void set_caps(int max_rank);  // capacity ranks; rebuild classes afterwards
  std::string rebuild_classes();  // after set_caps: classes, lambda, job lists
  void update_dims();           // dims/P/P_max/r_max from ranks
  std::array<int, 4> theta_dims(int first, int second) const;
  int n_sub(double tau, double kappa) const;
  bool built_jobs = false;
  std::string build_jobs();
  // recompute the tile shape of every job list: tile_warps warps per CTA of the
  // apply lists (0: kSplitWarps) and the planned split below max_split
  void set_split(int max_split, int tw = 0);

 private:
  std::string build_classes();
  int new_mat(int d);
  int add_list(const std::vector<ApOut>& outs, const std::vector<std::vector<ApTerm>>& terms);
  int add_pj_list(const std::vector<PjOut>& outs);
  int split_factor(int tiles, int useful) const;
  void node_terms(int u, int src, int t_base, std::vector<ApTerm>& singles,
                  std::vector<std::array<int, 4>>& pairs) const;
  // operator terms on an arbitrary list of (node, leg) "virtual legs"
  void vl_terms(const std::vector<std::pair<int, int>>& vl, int src, std::vector<ApTerm>& singles,
                std::vector<std::array<int, 4>>& pairs) const;
};

constexpr int kApTile = 32;   // output elements per CTA of the apply kernel
constexpr int kPjTile = 32;   // output entries per CTA of the projection kernel
constexpr int kApChunk = 4;   // leg positions per work unit of the apply kernel
constexpr int kSplitWarps = 8;  // warps per CTA of the apply / projection kernels
constexpr int kMaxSplit = 16;   // at most this many CTAs (one cluster, non-portable above 8) share an output tile

}  // namespace ttn
