// Host-side planning: see plan.hpp.
#include "plan.hpp"

#include <climits>

#include <algorithm>
#include <cmath>
#include <map>
#include <sstream>

namespace ttn {

// ---------------------------------------------------------------------------
// Tree
// ---------------------------------------------------------------------------
std::string Tree::build(int n, const int32_t* par, int nl, const int32_t* ln) {
  if (n < 1 || !par) return "tree: need at least one node";
  if (nl < 2 || !ln) return "tree: need at least the two system legs";
  n_nodes = n;
  n_legs = nl;
  parent.assign(par, par + n);
  leg_node.assign(ln, ln + nl);
  if (parent[0] != -1) return "tree: node 0 must be the root (parent -1)";
  children.assign(n, {});
  std::vector<std::vector<int>> ch(n);
  for (int u = 1; u < n; ++u) {
    if (parent[u] < 0 || parent[u] >= n || parent[u] == u) return "tree: bad parent index";
    ch[parent[u]].push_back(u);
  }
  for (int u = 0; u < n; ++u) {  // every node must reach the root
    int v = u, steps = 0;
    while (v != 0) {
      v = parent[v];
      if (++steps > n) return "tree: parent array contains a cycle";
    }
  }
  std::vector<std::vector<int>> open(n);
  for (int l = 0; l < nl; ++l) {
    if (leg_node[l] < 0 || leg_node[l] >= n) return "tree: leg attached to no node";
    open[leg_node[l]].push_back(l);
  }
  if (leg_node[0] != 0 || leg_node[1] != 0) return "tree: system legs 0 and 1 must sit on the root";
  // postorder
  postorder.clear();
  std::vector<std::pair<int, int>> stack{{0, 0}};
  while (!stack.empty()) {
    auto& top = stack.back();
    if (top.second < (int)ch[top.first].size()) {
      int c = ch[top.first][top.second++];
      stack.push_back({c, 0});
    } else {
      postorder.push_back(top.first);
      stack.pop_back();
    }
  }
  below.assign(n, std::vector<char>(nl, 0));
  std::vector<int> min_leg(n, 1 << 30);
  for (int u : postorder) {
    for (int l : open[u]) below[u][l] = 1;
    for (int c : ch[u])
      for (int l = 0; l < nl; ++l) below[u][l] |= below[c][l];
    for (int l = 0; l < nl; ++l)
      if (below[u][l]) {
        min_leg[u] = l;
        break;
      }
    if (min_leg[u] == (1 << 30)) return "tree: a node has no open leg below it";
  }
  legs.assign(n, {});
  for (int u = 0; u < n; ++u) {
    std::vector<std::pair<int, Leg>> items;
    for (int l : open[u]) items.push_back({l, Leg{'o', l}});
    for (int c : ch[u]) items.push_back({min_leg[c], Leg{'n', c}});
    std::sort(items.begin(), items.end(),
              [](const std::pair<int, Leg>& a, const std::pair<int, Leg>& b) { return a.first < b.first; });
    if (u != 0) legs[u].push_back(Leg{'p', parent[u]});
    for (auto& it : items) legs[u].push_back(it.second);
    for (auto& it : items)
      if (it.second.kind == 'n') children[u].push_back(it.second.v);
    if (legs[u].size() != 3) return "UNSUPPORTED: only nodes with exactly three legs are supported";
  }
  // recompute postorder with canonical child order (deterministic sweeps)
  postorder.clear();
  std::vector<std::pair<int, int>> st2{{0, 0}};
  while (!st2.empty()) {
    auto& top = st2.back();
    if (top.second < (int)children[top.first].size()) {
      int c = children[top.first][top.second++];
      st2.push_back({c, 0});
    } else {
      postorder.push_back(top.first);
      st2.pop_back();
    }
  }
  return "";
}

int Tree::leg_index(int u, int v) const {
  for (int i = 0; i < (int)legs[u].size(); ++i) {
    const Leg& L = legs[u][i];
    if ((L.kind == 'p' || L.kind == 'n') && L.v == v) return i;
  }
  return -1;
}

std::vector<int> effective_ranks(const Tree& t, const std::vector<int>& leg_dims,
                                 const std::vector<int>& req) {
  std::vector<int> r(t.n_nodes, 0);
  for (int u = 1; u < t.n_nodes; ++u) r[u] = req[u];
  auto dim = [&](int u, const Leg& L) -> long long {
    if (L.kind == 'p') return r[u];
    if (L.kind == 'n') return r[L.v];
    return leg_dims[L.v];
  };
  bool changed = true;
  while (changed) {
    changed = false;
    for (int c = 1; c < t.n_nodes; ++c) {
      int u = t.parent[c];
      long long pc = 1, pu = 1;
      for (const Leg& L : t.legs[c])
        if (L.kind != 'p') pc = std::min<long long>(pc * dim(c, L), 1LL << 40);
      for (const Leg& L : t.legs[u])
        if (!(L.kind == 'n' && L.v == c)) pu = std::min<long long>(pu * dim(u, L), 1LL << 40);
      long long nw = std::min<long long>({(long long)r[c], pc, pu});
      if (nw != r[c]) {
        r[c] = (int)nw;
        changed = true;
      }
    }
  }
  return r;
}

// ||M||_2 = sqrt(lambda_max(M^H M)); the Hermitian H = A + iB is embedded as the
// real symmetric [[A, -B], [B, A]] (same eigenvalues, each twice) and
// diagonalised by the cyclic Jacobi method (Rutishauser's rotation formulas).
double spectral_norm(const cd* M, int d) {
  std::vector<cd> H(d * d, cd(0));
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      cd s = 0;
      for (int k = 0; k < d; ++k) s += std::conj(M[k * d + i]) * M[k * d + j];
      H[i * d + j] = s;
    }
  int n = 2 * d;
  std::vector<double> S(n * n);
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      double a = H[i * d + j].real(), b = H[i * d + j].imag();
      S[i * n + j] = a;
      S[(i + d) * n + (j + d)] = a;
      S[i * n + (j + d)] = -b;
      S[(i + d) * n + j] = b;
    }
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0, diag = 0;
    for (int p = 0; p < n; ++p)
      for (int q = 0; q < n; ++q) (p == q ? diag : off) += S[p * n + q] * S[p * n + q];
    if (off <= 1e-32 * diag || off == 0) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = S[p * n + q];
        if (apq == 0) continue;
        double tau = (S[q * n + q] - S[p * n + p]) / (2 * apq);
        double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1 + tau * tau));
        double c = 1 / std::sqrt(1 + t * t), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          double skp = S[k * n + p], skq = S[k * n + q];
          S[k * n + p] = c * skp - s * skq;
          S[k * n + q] = s * skp + c * skq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          double spk = S[p * n + k], sqk = S[q * n + k];
          S[p * n + k] = c * spk - s * sqk;
          S[q * n + k] = s * spk + c * sqk;
        }
      }
  }
  double lmax = 0;
  for (int i = 0; i < n; ++i) lmax = std::max(lmax, S[i * n + i]);
  return std::sqrt(std::max(lmax, 0.0));
}

// ---------------------------------------------------------------------------
// Plan
// ---------------------------------------------------------------------------
std::string Plan::build(int n_nodes, const int32_t* parent, int n_legs, const int32_t* leg_node,
                        const int32_t* ld, const int32_t* rk) {
  std::string e = tree.build(n_nodes, parent, n_legs, leg_node);
  if (!e.empty()) return e;
  if (!ld || !rk) return "null leg_dims or ranks";
  leg_dims.assign(ld, ld + n_legs);
  for (int l = 0; l < n_legs; ++l)
    if (leg_dims[l] < 1) return "leg dimension < 1";
  if (leg_dims[0] != leg_dims[1]) return "legs 0 and 1 (system ket/bra) must have equal dimension";
  req.assign(rk, rk + n_nodes);
  req[0] = 0;
  for (int u = 1; u < n_nodes; ++u)
    if (req[u] < 1) return "rank < 1";
  ranks = effective_ranks(tree, leg_dims, req);
  update_dims();
  set_caps(cap_rank);
  if (r_cap_max > 256) return "UNSUPPORTED: bond ranks above 256 (QR kernel limit)";
  return "";
}

void Plan::update_dims() {
  const int n = tree.n_nodes;
  dims.assign(n, {0, 0, 0});
  P.assign(n, 0);
  P_max = 0;
  r_max = 1;
  for (int u = 0; u < n; ++u) {
    int64_t p = 1;
    for (int i = 0; i < 3; ++i) {
      const Leg& L = tree.legs[u][i];
      int d = L.kind == 'p' ? ranks[u] : L.kind == 'n' ? ranks[L.v] : leg_dims[L.v];
      dims[u][i] = d;
      p *= d;
    }
    P[u] = p;
    P_max = std::max(P_max, p);
  }
  for (int u = 1; u < n; ++u) r_max = std::max(r_max, ranks[u]);
}

void Plan::set_caps(int max_rank) {
  const int n = tree.n_nodes;
  cap_rank = max_rank;
  std::vector<int> want(n, 0);
  for (int u = 1; u < n; ++u) want[u] = std::max(req[u], max_rank);
  caps = effective_ranks(tree, leg_dims, want);
  for (int u = 1; u < n; ++u) caps[u] = std::max(caps[u], ranks[u]);
  cap_dims.assign(n, {0, 0, 0});
  P_cap.assign(n, 0);
  P_cap_max = 0;
  r_cap_max = 1;
  for (int u = 0; u < n; ++u) {
    int64_t p = 1;
    for (int i = 0; i < 3; ++i) {
      const Leg& L = tree.legs[u][i];
      int d = L.kind == 'p' ? caps[u] : L.kind == 'n' ? caps[L.v] : leg_dims[L.v];
      cap_dims[u][i] = d;
      p *= d;
    }
    P_cap[u] = p;
    P_cap_max = std::max(P_cap_max, p);
  }
  for (int u = 1; u < n; ++u) r_cap_max = std::max(r_cap_max, caps[u]);
  theta_cap = 1;
  for (int c = 1; c < n; ++c) {  // merged pair (c, parent) at capacity: P_c * P_p / r_cap^2
    const int p = tree.parent[c];
    theta_cap = std::max(theta_cap, P_cap[c] / caps[c] * (P_cap[p] / caps[c]));
  }
}

int Plan::dir_id(int a, int b) const {
  if (tree.parent[a] == b) return a;            // up edge a -> parent
  if (tree.parent[b] == a) return tree.n_nodes + b;  // down edge parent -> b
  return -1;
}

std::vector<char> Plan::behind(int u, int li) const {
  const Leg& L = tree.legs[u][li];
  std::vector<char> out(tree.n_legs, 0);
  if (L.kind == 'o') {
    out[L.v] = 1;
  } else if (L.kind == 'n') {
    out = tree.below[L.v];
  } else {
    for (int l = 0; l < tree.n_legs; ++l) out[l] = !tree.below[u][l];
  }
  return out;
}

int Plan::slot_of(int u, int li, ClassId c) const {
  const Leg& L = tree.legs[u][li];
  if (L.kind == 'o') {
    for (const LocalMat& m : locals)
      if (m.leg == L.v && m.cls == c) return m.slot;
    return -1;
  }
  int e = dir_id(L.v, u);
  const auto& cl = dir_classes[e];
  for (size_t i = 0; i < cl.size(); ++i)
    if (cl[i] == c) return dir_slots[e][i];
  return -1;
}

static bool finite_c(double a, double b) { return std::isfinite(a) && std::isfinite(b); }

std::string Plan::load_sop(int n_ops, const int32_t* opl, const int64_t* opo, const double* opd,
                           int n_terms, const int32_t* toff, const int32_t* tops, const double* coef,
                           const int32_t* cdrive) {
  if (n_ops < 0 || n_terms < 0) return "negative counts";
  if ((n_ops > 0 && (!opl || !opo || !opd)) || (n_terms > 0 && (!toff || !tops || !coef)))
    return "null SOP array";
  ops.assign(n_ops, {});
  op_leg.assign(n_ops, 0);
  for (int k = 0; k < n_ops; ++k) {
    int l = opl[k];
    if (l < 0 || l >= tree.n_legs) return "operator on a non-existent leg";
    int d = leg_dims[l];
    if (opo[k] < 0) return "negative operator offset";
    op_leg[k] = l;
    ops[k].resize((size_t)d * d);
    for (int i = 0; i < d * d; ++i) {
      double re = opd[2 * (opo[k] + i)], im = opd[2 * (opo[k] + i) + 1];
      if (!finite_c(re, im)) return "non-finite operator entry";
      ops[k][i] = cd(re, im);
    }
  }
  terms.assign(n_terms, {});
  n_drives = 0;
  if (toff && toff[0] != 0) return "term_offsets[0] must be 0";
  for (int m = 0; m < n_terms; ++m) {
    RawTerm& t = terms[m];
    if (!finite_c(coef[2 * m], coef[2 * m + 1])) return "non-finite coefficient";
    t.coef = cd(coef[2 * m], coef[2 * m + 1]);
    t.drive = cdrive ? cdrive[m] : -1;
    if (t.drive < -1) return "bad drive id";
    int b = toff[m], e = toff[m + 1];
    if (e - b < 1 || e - b > 2) return "UNSUPPORTED: terms must have one or two factors";
    for (int i = b; i < e; ++i) {
      int op = tops[i];
      if (op < 0 || op >= n_ops) return "term references a non-existent operator";
      t.f.push_back(Factor{op_leg[op], op});
    }
    if (t.f.size() == 2 && t.f[0].leg == t.f[1].leg) return "two factors of one term on the same leg";
    if (t.drive >= 0) {
      n_drives = std::max(n_drives, t.drive + 1);
      for (const Factor& f : t.f)
        if (tree.leg_node[f.leg] != 0) return "UNSUPPORTED: driven terms may only act on legs of the root";
    }
  }
  if ((int)drive_bound.size() < n_drives) drive_bound.resize(n_drives, 1.0);
  std::string e = build_classes();
  if (!e.empty()) return e;
  compute_lambda();
  built_jobs = false;
  return "";
}

std::string Plan::rebuild_classes() {
  std::string e = build_classes();
  if (!e.empty()) return e;
  compute_lambda();
  return build_jobs();
}

void Plan::compute_lambda() {
  std::vector<double> opn(ops.size());
  for (size_t k = 0; k < ops.size(); ++k) opn[k] = spectral_norm(ops[k].data(), leg_dims[op_leg[k]]);
  lambda = 0;
  for (const RawTerm& t : terms) {
    double v = std::abs(t.coef);
    if (t.drive >= 0) v *= (t.drive < (int)drive_bound.size() ? drive_bound[t.drive] : 1.0);
    for (const Factor& f : t.f) v *= opn[f.op];
    lambda += v;
  }
}

int Plan::n_sub(double tau, double kappa) const {
  double x = std::fabs(tau) * lambda / kappa - 1e-9;
  if (!(x < 1e9)) return 1 << 30;  // caller rejects absurd substep counts
  int m = (int)std::ceil(x);
  return std::max(1, m);
}

int Plan::new_mat(int d) {
  mats.push_back(MatSlot{d, mat_pool});
  mat_pool += (int64_t)d * d;
  return (int)mats.size() - 1;
}

std::string Plan::build_classes() {
  const int n = tree.n_nodes, nl = tree.n_legs;
  // keys: the factor shared by more two-factor terms (ties: lower leg)
  std::map<std::pair<int, int>, int> count;
  for (const RawTerm& t : terms)
    if (t.f.size() == 2)
      for (const Factor& f : t.f) count[{f.leg, f.op}]++;
  keys.clear();
  std::map<std::pair<int, int>, int> key_id;
  term_key.assign(terms.size(), -1);
  term_partner.assign(terms.size(), -1);
  for (size_t m = 0; m < terms.size(); ++m) {
    const RawTerm& t = terms[m];
    if (t.f.size() != 2) continue;
    int c0 = count[{t.f[0].leg, t.f[0].op}], c1 = count[{t.f[1].leg, t.f[1].op}];
    int ki = (c0 > c1 || (c0 == c1 && t.f[0].leg < t.f[1].leg)) ? 0 : 1;
    std::pair<int, int> kk{t.f[ki].leg, t.f[ki].op};
    auto it = key_id.find(kk);
    if (it == key_id.end()) {
      key_id[kk] = (int)keys.size();
      keys.push_back(Key{kk.first, kk.second});
    }
    term_key[m] = key_id[kk];
    term_partner[m] = 1 - ki;
  }
  const int nk = (int)keys.size();
  // partner legs of every key
  std::vector<std::vector<char>> partner_on(nk, std::vector<char>(nl, 0));
  for (size_t m = 0; m < terms.size(); ++m)
    if (term_key[m] >= 0) partner_on[term_key[m]][terms[m].f[term_partner[m]].leg] = 1;

  mats.clear();
  mat_pool = 0;
  dir_classes.assign(2 * n, {});
  dir_slots.assign(2 * n, {});
  for (int c = 1; c < n; ++c) {
    int p = tree.parent[c];
    for (int dir = 0; dir < 2; ++dir) {
      int e = dir == 0 ? dir_id(c, p) : dir_id(p, c);
      std::vector<char> T(nl);
      for (int l = 0; l < nl; ++l) T[l] = dir == 0 ? tree.below[c][l] : !tree.below[c][l];
      auto& cls = dir_classes[e];
      bool has_s = false;
      for (const RawTerm& t : terms) {
        bool in = true;
        for (const Factor& f : t.f) in = in && T[f.leg];
        has_s = has_s || in;
      }
      if (has_s) cls.push_back(ClassId{0, -1});
      for (int k = 0; k < nk; ++k) {
        bool a_in = T[keys[k].leg];
        bool p_in = false, p_out = false;
        for (int l = 0; l < nl; ++l)
          if (partner_on[k][l]) (T[l] ? p_in : p_out) = true;
        if (a_in && p_out) cls.push_back(ClassId{1, k});
        if (!a_in && p_in) cls.push_back(ClassId{2, k});
      }
      for (size_t i = 0; i < cls.size(); ++i) dir_slots[e].push_back(new_mat(caps[c]));
    }
  }
  // open-leg matrices
  locals.clear();
  auto local_for = [&](int leg, ClassId c) -> LocalMat& {
    for (LocalMat& m : locals)
      if (m.leg == leg && m.cls == c) return m;
    LocalMat m;
    m.leg = leg;
    m.cls = c;
    int d = leg_dims[leg];
    m.stat.assign((size_t)d * d, cd(0));
    m.drive.assign(n_drives, {});
    locals.push_back(m);
    return locals.back();
  };
  auto add_into = [&](LocalMat& lm, int drive, cd coef, const std::vector<cd>& op) {
    std::vector<cd>& dst = drive < 0 ? lm.stat : lm.drive[drive];
    if (dst.empty()) dst.assign(op.size(), cd(0));
    for (size_t i = 0; i < op.size(); ++i) dst[i] += coef * op[i];
    if (drive >= 0) lm.time_dependent = true;
  };
  for (size_t m = 0; m < terms.size(); ++m) {
    const RawTerm& t = terms[m];
    if (t.f.size() == 1) {
      add_into(local_for(t.f[0].leg, ClassId{0, -1}), t.drive, t.coef, ops[t.f[0].op]);
    } else {
      int k = term_key[m];
      const Factor& pf = t.f[term_partner[m]];
      add_into(local_for(pf.leg, ClassId{2, k}), t.drive, t.coef, ops[pf.op]);
    }
  }
  for (int k = 0; k < nk; ++k) add_into(local_for(keys[k].leg, ClassId{1, k}), -1, cd(1), ops[keys[k].op]);
  for (LocalMat& lm : locals) {
    int d = leg_dims[lm.leg];
    lm.slot = new_mat(d);
    if (lm.time_dependent) {
      lm.slot_stat = new_mat(d);
      lm.slot_drive.assign(n_drives, -1);
      for (int dr = 0; dr < n_drives; ++dr)
        if (!lm.drive[dr].empty()) lm.slot_drive[dr] = new_mat(d);
    }
  }
  bond_mat = (int)mats.size();  // alias of the bond buffer (no pool storage)
  mats.push_back(MatSlot{r_cap_max, -1});
  return "";
}

// ---------------------------------------------------------------------------
// Job lists
// ---------------------------------------------------------------------------
// CTAs per output tile: the smallest k <= min(useful, kMaxSplit) that brings
// tiles * k to two CTAs per SM (1 when the list alone fills the device).
int Plan::split_factor(int tiles, int useful) const {
  const int target = 2 * sm_count;
  int k = 1;
  const int kmax = std::max(1, std::min(std::min(useful, kMaxSplit), max_split));
  while (k < kmax && tiles * k < target) ++k;
  return k;
}

void Plan::set_split(int m, int tw) {
  max_split = m;
  tile_warps = tw;
  const int w = tw > 0 ? tw : kSplitWarps;
  for (ApList& L : ap_lists) {
    L.w = w;
    L.useful = (L.units + w - 1) / w;
    L.k = split_factor(L.n_tiles, L.useful);
  }
  for (PjList& L : pj_lists) L.k = split_factor(L.n_tiles, L.useful);
}

int Plan::add_list(const std::vector<ApOut>& outs, const std::vector<std::vector<ApTerm>>& tl) {
  ApList L;
  L.out_begin = (int)ap_outs.size();
  L.flops = 0;
  int tiles = 0;
  for (size_t i = 0; i < outs.size(); ++i) {
    ApOut o = outs[i];
    o.term_begin = (int)ap_terms.size();
    if (o.d3 < 1) o.d3 = 1;
    const int dd[4] = {o.d0, o.d1, o.d2, o.d3};
    for (const ApTerm& t : tl[i]) {
      ap_terms.push_back(t);
      if (t.mat >= 0) L.flops += 8.0 * o.d0 * o.d1 * o.d2 * o.d3 * dd[t.leg];
    }
    o.term_end = (int)ap_terms.size();
    o.tile0 = tiles;
    int64_t p = (int64_t)o.d0 * o.d1 * o.d2 * o.d3;
    const int nt = (int)((p + kApTile - 1) / kApTile);
    L.tpo = i == 0 ? nt : (L.tpo == nt ? nt : 0);
    tiles += nt;
    ap_outs.push_back(o);
  }
  L.out_end = (int)ap_outs.size();
  L.n_tiles = tiles;
  // Work units of an output tile: one per identity term, ceil(d_leg / kApChunk)
  // per mode product. Split a tile over k CTAs (one cluster) while the grid is
  // below two CTAs per SM and every warp still gets a unit.
  int units_max = 1;
  for (size_t i = 0; i < outs.size(); ++i) {
    const int dd[4] = {outs[i].d0, outs[i].d1, outs[i].d2, outs[i].d3 < 1 ? 1 : outs[i].d3};
    int u = 0;
    for (const ApTerm& t : tl[i]) u += t.mat < 0 ? 1 : (dd[t.leg] + kApChunk - 1) / kApChunk;
    units_max = std::max(units_max, u);
  }
  L.units = units_max;
  L.w = tile_warps > 0 ? tile_warps : kSplitWarps;
  L.useful = (units_max + L.w - 1) / L.w;
  L.k = split_factor(tiles, L.useful);
  ap_lists.push_back(L);
  return (int)ap_lists.size() - 1;
}

int Plan::add_pj_list(const std::vector<PjOut>& outs) {
  PjList L;
  L.out_begin = (int)pj_outs.size();
  L.flops = 0;
  int tiles = 0;
  for (size_t i = 0; i < outs.size(); ++i) {
    PjOut o = outs[i];
    o.tile0 = tiles;
    int d = o.leg == 0 ? o.d0 : o.leg == 1 ? o.d1 : o.d2;
    L.flops += 8.0 * o.d0 * o.d1 * o.d2 * d;
    const int nt = (d * d + kPjTile - 1) / kPjTile;
    L.tpo = i == 0 ? nt : (L.tpo == nt ? nt : 0);
    tiles += nt;
    pj_outs.push_back(o);
  }
  L.out_end = (int)pj_outs.size();
  L.n_tiles = tiles;
  // split the reduction range so that each warp keeps at least 4 positions
  int64_t rest_min = INT64_MAX;
  for (const PjOut& o : outs) {
    const int d = o.leg == 0 ? o.d0 : o.leg == 1 ? o.d1 : o.d2;
    rest_min = std::min<int64_t>(rest_min, (int64_t)o.d0 * o.d1 * o.d2 / d);
  }
  if (outs.empty()) rest_min = 1;
  L.useful = (int)std::min<int64_t>(kMaxSplit, std::max<int64_t>(1, rest_min / (4 * kSplitWarps)));
  L.k = split_factor(tiles, L.useful);
  pj_lists.push_back(L);
  return (int)pj_lists.size() - 1;
}

// Operator on a list of virtual legs (node, leg index): singles {S on each leg}
// and pairs (X slot, leg a, P slot, leg b) for every key whose factor lies
// behind leg a and whose partners lie behind leg b. The legs' behind-sets must
// partition the open legs (one node's three legs, or a merged pair's four).
void Plan::vl_terms(const std::vector<std::pair<int, int>>& vl, int src, std::vector<ApTerm>& singles,
                    std::vector<std::array<int, 4>>& pairs) const {
  singles.clear();
  pairs.clear();
  const int nv = (int)vl.size();
  std::vector<std::vector<char>> B(nv);
  for (int a = 0; a < nv; ++a) B[a] = behind(vl[a].first, vl[a].second);
  for (int a = 0; a < nv; ++a) {
    int s = slot_of(vl[a].first, vl[a].second, ClassId{0, -1});
    if (s >= 0) singles.push_back(ApTerm{s, a, src, 0});
  }
  std::vector<std::vector<char>> partner_on(keys.size(), std::vector<char>(tree.n_legs, 0));
  for (size_t m = 0; m < terms.size(); ++m)
    if (term_key[m] >= 0) partner_on[term_key[m]][terms[m].f[term_partner[m]].leg] = 1;
  for (size_t k = 0; k < keys.size(); ++k) {
    int l1 = -1;
    for (int a = 0; a < nv; ++a)
      if (B[a][keys[k].leg]) l1 = a;
    for (int l2 = 0; l2 < nv; ++l2) {
      if (l2 == l1) continue;
      bool any = false;
      for (int l = 0; l < tree.n_legs; ++l) any = any || (partner_on[k][l] && B[l2][l]);
      if (!any) continue;
      int xs = slot_of(vl[l1].first, vl[l1].second, ClassId{1, (int)k});
      int ps = slot_of(vl[l2].first, vl[l2].second, ClassId{2, (int)k});
      pairs.push_back({xs, l1, ps, l2});
    }
  }
}

void Plan::node_terms(int u, int src, int, std::vector<ApTerm>& singles,
                      std::vector<std::array<int, 4>>& pairs) const {
  vl_terms({{u, 0}, {u, 1}, {u, 2}}, src, singles, pairs);
}

std::array<int, 4> Plan::theta_dims(int first, int second) const {
  std::array<int, 4> d{1, 1, 1, 1};
  int k = 0;
  const int lf = tree.leg_index(first, second), ls = tree.leg_index(second, first);
  for (int i = 0; i < 3; ++i)
    if (i != lf) d[k++] = dims[first][i];
  for (int i = 0; i < 3; ++i)
    if (i != ls) d[k++] = dims[second][i];
  return d;
}

std::string Plan::build_jobs() {
  const int n = tree.n_nodes;
  ap_terms.clear();
  ap_outs.clear();
  ap_lists.clear();
  pj_outs.clear();
  pj_lists.clear();
  // buffer ids
  buf.ys = n;
  buf.ys2 = n + 1;
  buf.acc = n + 2;
  buf.tmp = n + 3;
  buf.bond_y = n + 4;
  buf.bond_ys = n + 5;
  buf.bond_ys2 = n + 6;
  buf.bond_acc = n + 7;
  buf.th_y = n + 8;
  buf.th_ys = n + 9;
  buf.th_ys2 = n + 10;
  buf.th_acc = n + 11;
  buf.t0 = n + 12;
  // count pairs / classes to size T and W
  int max_pairs = 0, max_classes = 0;
  std::vector<ApTerm> singles;
  std::vector<std::array<int, 4>> pairs;
  for (int u = 0; u < n; ++u) {
    node_terms(u, u, 0, singles, pairs);
    max_pairs = std::max(max_pairs, (int)pairs.size());
  }
  for (auto& cl : dir_classes) max_classes = std::max(max_classes, (int)cl.size());
  // bond pairs
  auto bond_terms = [&](int a, int b, int src, std::vector<ApTerm>& sg, std::vector<std::array<int, 4>>& pr) {
    sg.clear();
    pr.clear();
    int e1 = dir_id(a, b), e2 = dir_id(b, a);
    auto find = [&](int e, ClassId c) {
      for (size_t i = 0; i < dir_classes[e].size(); ++i)
        if (dir_classes[e][i] == c) return dir_slots[e][i];
      return -1;
    };
    int s1 = find(e1, ClassId{0, -1}), s2 = find(e2, ClassId{0, -1});
    if (s1 >= 0) sg.push_back(ApTerm{s1, 1, src, 0});
    if (s2 >= 0) sg.push_back(ApTerm{s2, 2, src, 0});
    for (size_t k = 0; k < keys.size(); ++k) {
      int x1 = find(e1, ClassId{1, (int)k}), p2 = find(e2, ClassId{2, (int)k});
      if (x1 >= 0 && p2 >= 0) pr.push_back({x1, 1, p2, 2});
      int p1 = find(e1, ClassId{2, (int)k}), x2 = find(e2, ClassId{1, (int)k});
      if (p1 >= 0 && x2 >= 0) pr.push_back({p1, 1, x2, 2});
    }
  };
  for (int c = 1; c < n; ++c) {
    int p = tree.parent[c];
    for (int dir = 0; dir < 2; ++dir) {
      bond_terms(dir ? p : c, dir ? c : p, 0, singles, pairs);
      max_pairs = std::max(max_pairs, (int)pairs.size());
    }
  }
  for (int c = 1; c < n; ++c) {  // two-site operators have more pairs (four legs)
    int p = tree.parent[c];
    std::vector<std::pair<int, int>> vl;
    const int lf = tree.leg_index(c, p), ls = tree.leg_index(p, c);
    for (int i = 0; i < 3; ++i)
      if (i != lf) vl.push_back({c, i});
    for (int i = 0; i < 3; ++i)
      if (i != ls) vl.push_back({p, i});
    vl_terms(vl, 0, singles, pairs);
    max_pairs = std::max(max_pairs, (int)pairs.size());
  }
  buf.n_t = std::max(max_pairs, 1);
  buf.w0 = buf.t0 + buf.n_t;
  buf.n_w = std::max(max_classes, 1);
  buf.n_bufs = buf.w0 + buf.n_w;

  // node flows
  node_flow.assign(n, {});
  node_down.assign(n, -1);
  for (int u = 0; u < n; ++u) {
    for (int var = 0; var < 3; ++var) {
      int src = var == 0 ? u : var == 1 ? buf.ys : buf.ys2;
      node_terms(u, src, 0, singles, pairs);
      ApOut base{dims[u][0], dims[u][1], dims[u][2], 0, 0, -1, 0, 0};
      if (!pairs.empty()) {
        std::vector<ApOut> outs;
        std::vector<std::vector<ApTerm>> tl;
        for (size_t g = 0; g < pairs.size(); ++g) {
          ApOut o = base;
          o.dst = buf.t0 + (int)g;
          outs.push_back(o);
          tl.push_back({ApTerm{pairs[g][2], pairs[g][3], src, 0}});
        }
        node_flow[u].first[var] = add_list(outs, tl);
      }
      std::vector<ApTerm> all = singles;
      for (size_t g = 0; g < pairs.size(); ++g) all.push_back(ApTerm{pairs[g][0], pairs[g][1], buf.t0 + (int)g, 0});
      node_flow[u].combine[var] = add_list({base}, {all});
      if (var == 0 && u != 0) {
        std::vector<ApTerm> down;
        for (const ApTerm& t : singles)
          if (t.leg != 0) down.push_back(t);
        for (size_t g = 0; g < pairs.size(); ++g)
          if (pairs[g][1] != 0 && pairs[g][3] != 0) down.push_back(ApTerm{pairs[g][0], pairs[g][1], buf.t0 + (int)g, 0});
        node_down[u] = add_list({base}, {down});
      }
    }
  }
  // bond flows (R as a (1, r, r) tensor: leg 1 = from side, leg 2 = to side)
  bond_flow.assign(2 * n, {});
  for (int c = 1; c < n; ++c) {
    int p = tree.parent[c];
    for (int dir = 0; dir < 2; ++dir) {
      int a = dir ? p : c, b = dir ? c : p;
      int e = dir_id(a, b);
      int r = ranks[c];
      for (int var = 0; var < 3; ++var) {
        int src = var == 0 ? buf.bond_y : var == 1 ? buf.bond_ys : buf.bond_ys2;
        bond_terms(a, b, src, singles, pairs);
        ApOut base{1, r, r, 0, 0, -1, 0, 0};
        if (!pairs.empty()) {
          std::vector<ApOut> outs;
          std::vector<std::vector<ApTerm>> tl;
          for (size_t g = 0; g < pairs.size(); ++g) {
            ApOut o = base;
            o.dst = buf.t0 + (int)g;
            outs.push_back(o);
            tl.push_back({ApTerm{pairs[g][2], pairs[g][3], src, 0}});
          }
          bond_flow[e].first[var] = add_list(outs, tl);
        }
        std::vector<ApTerm> all = singles;
        for (size_t g = 0; g < pairs.size(); ++g)
          all.push_back(ApTerm{pairs[g][0], pairs[g][1], buf.t0 + (int)g, 0});
        bond_flow[e].combine[var] = add_list({base}, {all});
      }
    }
  }
  // two-site flows (ps2): Theta of the merged pair (first, second)
  two_site.assign(2 * n, {});
  for (int c = 1; c < n; ++c) {
    int p = tree.parent[c];
    for (int dir = 0; dir < 2; ++dir) {
      int first = dir ? p : c, second = dir ? c : p;
      int e = dir_id(first, second);
      std::vector<std::pair<int, int>> vl;
      const int lf = tree.leg_index(first, second), ls = tree.leg_index(second, first);
      for (int i = 0; i < 3; ++i)
        if (i != lf) vl.push_back({first, i});
      for (int i = 0; i < 3; ++i)
        if (i != ls) vl.push_back({second, i});
      const std::array<int, 4> td = theta_dims(first, second);
      for (int var = 0; var < 3; ++var) {
        int src = var == 0 ? buf.th_y : var == 1 ? buf.th_ys : buf.th_ys2;
        vl_terms(vl, src, singles, pairs);
        ApOut base{td[0], td[1], td[2], 0, 0, -1, 0, td[3]};
        if (!pairs.empty()) {
          std::vector<ApOut> outs;
          std::vector<std::vector<ApTerm>> tl;
          for (size_t g = 0; g < pairs.size(); ++g) {
            ApOut o = base;
            o.dst = buf.t0 + (int)g;
            outs.push_back(o);
            tl.push_back({ApTerm{pairs[g][2], pairs[g][3], src, 0}});
          }
          two_site[e].first[var] = add_list(outs, tl);
        }
        std::vector<ApTerm> all = singles;
        for (size_t g = 0; g < pairs.size(); ++g)
          all.push_back(ApTerm{pairs[g][0], pairs[g][1], buf.t0 + (int)g, 0});
        two_site[e].combine[var] = add_list({base}, {all});
      }
    }
  }
  // environment updates a -> b
  env.assign(2 * n, {});
  for (int c = 1; c < n; ++c) {
    int p = tree.parent[c];
    for (int dir = 0; dir < 2; ++dir) {
      int a = dir ? p : c, b = dir ? c : p;
      int e = dir_id(a, b);
      int lb = tree.leg_index(a, b);
      node_terms(a, a, 0, singles, pairs);
      std::vector<std::array<int, 4>> inner;
      for (auto& pr : pairs)
        if (pr[1] != lb && pr[3] != lb) inner.push_back(pr);
      ApOut base{dims[a][0], dims[a][1], dims[a][2], 0, 0, -1, 0, 0};
      if (!inner.empty()) {
        std::vector<ApOut> outs;
        std::vector<std::vector<ApTerm>> tl;
        for (size_t g = 0; g < inner.size(); ++g) {
          ApOut o = base;
          o.dst = buf.t0 + (int)g;
          outs.push_back(o);
          tl.push_back({ApTerm{inner[g][2], inner[g][3], a, 0}});
        }
        env[e].first = add_list(outs, tl);
      }
      std::array<std::vector<char>, 3> B;
      for (int li = 0; li < 3; ++li) B[li] = behind(a, li);
      std::vector<std::vector<char>> partner_on(keys.size(), std::vector<char>(tree.n_legs, 0));
      for (size_t m = 0; m < terms.size(); ++m)
        if (term_key[m] >= 0) partner_on[term_key[m]][terms[m].f[term_partner[m]].leg] = 1;
      std::vector<ApOut> outs;
      std::vector<std::vector<ApTerm>> tl;
      std::vector<PjOut> pj;
      for (size_t ci = 0; ci < dir_classes[e].size(); ++ci) {
        ClassId cl = dir_classes[e][ci];
        std::vector<ApTerm> t;
        if (cl.kind == 0) {
          for (auto& s : singles)
            if (s.leg != lb) t.push_back(s);
          for (size_t g = 0; g < inner.size(); ++g) t.push_back(ApTerm{inner[g][0], inner[g][1], buf.t0 + (int)g, 0});
        } else if (cl.kind == 1) {
          for (int li = 0; li < 3; ++li)
            if (li != lb && B[li][keys[cl.key].leg]) t.push_back(ApTerm{slot_of(a, li, cl), li, a, 0});
        } else {
          for (int li = 0; li < 3; ++li) {
            if (li == lb) continue;
            bool any = false;
            for (int l = 0; l < tree.n_legs; ++l) any = any || (partner_on[cl.key][l] && B[li][l]);
            if (any) t.push_back(ApTerm{slot_of(a, li, cl), li, a, 0});
          }
        }
        for (auto& x : t)
          if (x.mat < 0) return "internal: missing operator class";
        ApOut o = base;
        o.dst = buf.w0 + (int)ci;
        outs.push_back(o);
        tl.push_back(t);
        pj.push_back(PjOut{dims[a][0], dims[a][1], dims[a][2], lb, a, buf.w0 + (int)ci, dir_slots[e][ci], 0});
      }
      if (!outs.empty()) {
        env[e].classes = add_list(outs, tl);
        env[e].project = add_pj_list(pj);
      }
    }
  }
  // absorb R into node v at leg li: tmp = R x_li U_v
  absorb.assign(n, {-1, -1, -1});
  for (int v = 0; v < n; ++v)
    for (int li = 0; li < 3; ++li) {
      if (tree.legs[v][li].kind == 'o') continue;
      ApOut o{dims[v][0], dims[v][1], dims[v][2], 0, 0, buf.tmp, 0, 0};
      absorb[v][li] = add_list({o}, {{ApTerm{bond_mat, li, v, 0}}});
    }
  // every term of every list must reference an existing matrix
  for (const ApTerm& t : ap_terms)
    if (t.mat < -1 || t.mat >= (int)mats.size()) return "internal: bad matrix id";
  built_jobs = true;
  return "";
}

}  // namespace ttn
