// Host-side model builder and step compiler.
//
// Hamiltonian: the star Hamiltonian of Eq. 2 with bosons truncated to Fock
// states 0..d-1 and the system Hamiltonian shifted by -tr(H_S)/n_el (a global
// phase).  Every term is an on-site operator or a product of two single-node
// operators; the coefficient of a two-node term sits on its first factor.
//
// Tree (Results, "TTNS for vibronic quantum dynamics"; Methods, "Tensor Network
// States"): the electronic node is the root; with the star form every chain's
// first site hangs off the root, with the ER form a balanced binary tree of
// third-order entanglement-renormalisation nodes sits between them (each lowest
// ER node carries two chains).  Leg order of every tensor: [parent] +
// [children in order] + [physical]; row-major storage.
//
// Step (one-site TDVP, the paper's time integrator; projector-splitting
// ordering): S(tau) = visit(root), visit(v) = forward-evolve v, then for each
// child c: QR toward c, environment v->c, backward-evolve the bond, absorb it in
// c, visit(c), QR of c toward v, environment c->v, absorb R in v.  The second
// half-step S*(tau) runs the same operations in reverse order (bond evolution on
// the way up, the node's forward evolution last).  One step = S(dt/2) S*(dt/2).
#include "model.h"

#include <algorithm>
#include <cmath>
#include <functional>
#include <map>
#include <stdexcept>
#include <string>

namespace ttns {

std::vector<int> HostTree::legs(int v) const {
  std::vector<int> d;
  if (parent[v] >= 0) d.push_back(bond[v]);
  for (int c : children[v]) d.push_back(bond[c]);
  if (phys[v] > 0) d.push_back(phys[v]);
  return d;
}

int HostTree::leg_of(int v, int u) const {
  if (parent[v] == u) return 0;
  int off = parent[v] >= 0 ? 1 : 0;
  for (size_t k = 0; k < children[v].size(); ++k)
    if (children[v][k] == u) return off + (int)k;
  throw std::logic_error("leg_of: not a neighbour");
}

int HostTree::phys_leg(int v) const { return (int)legs(v).size() - 1; }

std::vector<int> HostTree::neighbours(int v) const {
  std::vector<int> nb;
  if (parent[v] >= 0) nb.push_back(parent[v]);
  for (int c : children[v]) nb.push_back(c);
  return nb;
}

// ---------------------------------------------------------------------------
// chain maps
// ---------------------------------------------------------------------------

void chain_ohmic(double alpha, double omega_c, int L, double* rc, double* onsite, double* hop) {
  // Laguerre weight x exp(-x) (parameter 1): monic recurrence a_n = 2n+2, b_n = n(n+1)
  *rc = 2.0 * omega_c * std::sqrt(alpha);
  for (int n = 0; n < L; ++n) onsite[n] = omega_c * (2.0 * n + 2.0);
  for (int n = 0; n + 1 < L; ++n) hop[n] = omega_c * std::sqrt((n + 1.0) * (n + 2.0));
}

bool chain_from_modes(int K, const double* omega, const double* lam, int L, double* rc, double* onsite,
                      double* hop) {
  if (L > K || L < 1) return false;
  double nrm = 0;
  for (int k = 0; k < K; ++k) nrm += lam[k] * lam[k];
  nrm = std::sqrt(nrm);
  *rc = nrm;
  if (nrm == 0.0) {
    std::vector<double> w(omega, omega + K);
    std::sort(w.begin(), w.end());
    for (int n = 0; n < L; ++n) onsite[n] = w[n];
    for (int n = 0; n + 1 < L; ++n) hop[n] = 0.0;
    return true;
  }
  // Lanczos on diag(omega) from lam/||lam||, re-orthogonalised twice against all vectors
  std::vector<double> V((size_t)K * L, 0.0);  // column n at V[n*K ...]
  for (int k = 0; k < K; ++k) V[k] = lam[k] / nrm;
  std::vector<double> w(K);
  for (int n = 0; n < L; ++n) {
    const double* q = &V[(size_t)n * K];
    double a = 0;
    for (int k = 0; k < K; ++k) { w[k] = omega[k] * q[k]; a += q[k] * w[k]; }
    onsite[n] = a;
    for (int k = 0; k < K; ++k) w[k] -= a * q[k];
    if (n > 0) {
      const double* qp = &V[(size_t)(n - 1) * K];
      for (int k = 0; k < K; ++k) w[k] -= hop[n - 1] * qp[k];
    }
    for (int pass = 0; pass < 2; ++pass) {
      for (int i = 0; i <= n; ++i) {
        const double* qi = &V[(size_t)i * K];
        double c = 0;
        for (int k = 0; k < K; ++k) c += qi[k] * w[k];
        for (int k = 0; k < K; ++k) w[k] -= c * qi[k];
      }
    }
    if (n + 1 < L) {
      double b = 0;
      for (int k = 0; k < K; ++k) b += w[k] * w[k];
      b = std::sqrt(b);
      hop[n] = b;
      if (b == 0.0) return false;
      double* qn = &V[(size_t)(n + 1) * K];
      for (int k = 0; k < K; ++k) qn[k] = w[k] / b;
    }
  }
  return true;
}

// ---------------------------------------------------------------------------
// tree
// ---------------------------------------------------------------------------

static void clamp_bonds(HostTree& t, std::vector<long long>& D) {
  const int n = t.n();
  bool changed = true;
  while (changed) {
    changed = false;
    for (int u = 0; u < n; ++u) {
      if (t.parent[u] < 0) continue;
      int v = t.parent[u];
      long long lim_u = std::max(t.phys[u], 1);
      for (int c : t.children[u]) lim_u = std::min<long long>(lim_u * D[c], 1LL << 40);
      long long lim_v = std::max(t.phys[v], 1);
      if (t.parent[v] >= 0) lim_v = std::min<long long>(lim_v * D[v], 1LL << 40);
      for (int c : t.children[v])
        if (c != u) lim_v = std::min<long long>(lim_v * D[c], 1LL << 40);
      long long nd = std::min(D[u], std::min(lim_u, lim_v));
      if (nd != D[u]) { D[u] = nd; changed = true; }
    }
  }
}

HostTree build_host_tree(const TreeInput& in) {
  HostTree t;
  t.n_el = in.n_el;
  std::vector<long long> req;
  auto add = [&](int p, int ph, int kind, long long D) {
    int v = t.n();
    t.parent.push_back(p);
    t.children.emplace_back();
    t.phys.push_back(ph);
    t.kind.push_back(kind);
    req.push_back(D);
    if (p >= 0) t.children[p].push_back(v);
    return v;
  };
  const int root = add(-1, in.n_el, 0, 0);
  std::vector<int> attach;
  if (in.er_tree) {
    int top = add(root, 0, 1, in.D_er);
    std::vector<int> level{top};
    while (2 * (int)level.size() < in.n_env) {
      std::vector<int> nxt;
      for (int p : level) {
        nxt.push_back(add(p, 0, 1, in.D_er));
        nxt.push_back(add(p, 0, 1, in.D_er));
      }
      level.swap(nxt);
    }
    for (int p : level) { attach.push_back(p); attach.push_back(p); }
  } else {
    attach.assign(in.n_env, root);
  }
  for (int i = 0; i < in.n_env; ++i) {
    std::vector<int> nodes;
    int p = attach[i];
    const int obb = (int)in.obb.size() > i ? in.obb[i] : 0;
    for (int s = 0; s < in.L[i]; ++s) {
      if (obb > 0) {
        // optimised boson basis: the site tensor keeps the chain bonds and a bond of dimension
        // obb to a leaf holding the Fock leg, on which the site's operators act
        int v = add(p, 0, 2, in.D[i]);
        nodes.push_back(add(v, in.d[i], 3, obb));
        p = v;
      } else {
        int v = add(p, in.d[i], 2, in.D[i]);
        nodes.push_back(v);
        p = v;
      }
    }
    t.chain_nodes.push_back(nodes);
  }
  if (!in.bond_req.empty()) {
    if ((int)in.bond_req.size() != t.n()) throw std::invalid_argument("bond requests do not match the tree's nodes");
    for (int v = 1; v < t.n(); ++v) {
      if (in.bond_req[v] < 1) throw std::invalid_argument("bond request below 1");
      req[v] = in.bond_req[v];
    }
  }
  // requested bond dimensions (any size: a request beyond the Hilbert space asks for the full
  // bond) are clamped first; what remains must fit the device code's leg limit
  clamp_bonds(t, req);
  t.bond.assign(t.n(), 0);
  for (int v = 1; v < t.n(); ++v) {
    if (req[v] > TTNS_MAX_D)
      throw std::invalid_argument("bond dimension " + std::to_string(req[v]) + " of node " + std::to_string(v) +
                                  " exceeds " + std::to_string(TTNS_MAX_D) + " after the Hilbert-space clamp");
    t.bond[v] = (int)req[v];
  }

  // on-site operators
  t.onsite.assign(t.n(), {});
  const int ne = in.n_el;
  double tr = 0;
  for (int s = 0; s < ne; ++s) tr += in.H_S[s * ne + s].real();
  t.onsite[root] = in.H_S;
  for (int s = 0; s < ne; ++s) t.onsite[root][s * ne + s] -= tr / ne;
  for (int i = 0; i < in.n_env; ++i) {
    const int d = in.d[i];
    std::vector<cplx> a(d * d, 0.0), ad(d * d, 0.0), apad(d * d, 0.0);
    for (int s = 1; s < d; ++s) {
      a[(s - 1) * d + s] = std::sqrt((double)s);   // a|s> = sqrt(s)|s-1>
      ad[s * d + (s - 1)] = std::sqrt((double)s);
    }
    for (int k = 0; k < d * d; ++k) apad[k] = a[k] + ad[k];
    const auto& nodes = t.chain_nodes[i];
    for (int s = 0; s < in.L[i]; ++s) {
      std::vector<cplx> num(d * d, 0.0);
      for (int q = 0; q < d; ++q) num[q * d + q] = in.omega[i][s] * q;
      t.onsite[nodes[s]] = num;
    }
    // system-RC coupling Wbar_i ||lambda_i|| / sqrt(2) (x) (a + a^+)
    std::vector<cplx> Wc(ne * ne);
    for (int k = 0; k < ne * ne; ++k) Wc[k] = in.W[i][k] * (in.rc[i] / std::sqrt(2.0));
    t.coups.push_back({root, Wc, nodes[0], apad});
    for (int s = 0; s + 1 < in.L[i]; ++s) {
      std::vector<cplx> tad(d * d), ta(d * d);
      for (int k = 0; k < d * d; ++k) { tad[k] = in.hop[i][s] * ad[k]; ta[k] = in.hop[i][s] * a[k]; }
      t.coups.push_back({nodes[s], tad, nodes[s + 1], a});
      t.coups.push_back({nodes[s], ta, nodes[s + 1], ad});
    }
  }
  t.psi_el = in.psi_el;
  return t;
}

HostTree kinetic_tree(const HostTree& h, const TreeInput& in) {
  HostTree k = h;
  k.onsite.assign(h.n(), {});
  k.coups.clear();
  for (int i = 0; i < in.n_env; ++i) {
    const int d = in.d[i];
    // P = a^+ - a and P^2 (products of the truncated matrices)
    std::vector<cplx> P(d * d, 0.0), P2(d * d, 0.0);
    for (int s = 1; s < d; ++s) {
      P[s * d + (s - 1)] = std::sqrt((double)s);
      P[(s - 1) * d + s] = -std::sqrt((double)s);
    }
    for (int r = 0; r < d; ++r)
      for (int c = 0; c < d; ++c) {
        cplx acc = 0.0;
        for (int q = 0; q < d; ++q) acc += P[r * d + q] * P[q * d + c];
        P2[r * d + c] = acc;
      }
    const auto& nodes = h.chain_nodes[i];
    for (int s = 0; s < in.L[i]; ++s) {
      std::vector<cplx> on(d * d);
      for (int q = 0; q < d * d; ++q) on[q] = -0.25 * in.omega[i][s] * P2[q];
      k.onsite[nodes[s]] = on;
    }
    for (int s = 0; s + 1 < in.L[i]; ++s) {
      std::vector<cplx> pa(d * d);
      for (int q = 0; q < d * d; ++q) pa[q] = -0.5 * in.hop[i][s] * P[q];
      k.coups.push_back({nodes[s], pa, nodes[s + 1], P});
    }
  }
  return k;
}

// ---------------------------------------------------------------------------
// compilation
// ---------------------------------------------------------------------------

namespace {

struct EnvInfo {
  long long off = -1;      // pool offset of the H block; channel b at off + (1+b) D^2
  int D = 0;
  std::vector<int> chans;  // coupling ids, ascending
};

struct TreeCompiler {
  const HostTree& t;
  Compiled& C;
  int tree_idx;
  int node0;                            // global node id of node 0
  std::vector<std::vector<char>> sub;   // subtree membership
  std::map<std::pair<int, int>, EnvInfo> env;
  std::vector<long long> opa_off, opb_off, onsite_off;
  std::map<long long, std::pair<int, long long>> sparse_of;  // constant matrix offset -> (nnz, table offset)
  long long bond_off = 0;
  std::map<std::pair<int, int>, int> bond_node;   // (u, w) -> global pseudo-node id of bond X[i_u, i_w]
  std::map<std::pair<int, int>, int> bond_list;   // (u, w) -> term list index
  std::map<int, int> heff_list;                   // v -> term list
  std::map<std::pair<int, int>, int> envh_list;   // (u, v) -> term list of the H block
  std::map<std::pair<int, int>, std::pair<int, int>> env_chan;  // (u, v) -> (first, count) in chans
  std::map<std::pair<int, int>, int> hist_slot;
  bool batched;
  int grid_threshold;
  int qr_grid_threshold;

  TreeCompiler(const HostTree& t_, Compiled& C_, int idx, bool b, int gt, int qgt)
      : t(t_), C(C_), tree_idx(idx), batched(b), grid_threshold(gt), qr_grid_threshold(qgt) {}

  long long push_matrix(const std::vector<cplx>& m) {
    long long off = (long long)C.pool_init.size();
    for (const cplx& z : m) C.pool_init.push_back(make_double2(z.real(), z.imag()));
    return off;
  }
  // constant operator: a dense matrix in the current region; when every row has few
  // nonzeros, a row-sparse table is also built (placed at the end of the region, see
  // finish_sparse)
  std::vector<std::pair<long long, std::vector<cplx>>> pending_sparse;
  long long push_operator(const std::vector<cplx>& m) {
    const long long off = push_matrix(m);
    pending_sparse.push_back({off, m});
    return off;
  }
  void finish_sparse() {
    for (auto& pr : pending_sparse) {
      const long long off = pr.first;
      const std::vector<cplx>& m = pr.second;
      const int D = (int)std::lround(std::sqrt((double)m.size()));
      int nnz = 0;
      for (int i = 0; i < D; ++i) {
        int c = 0;
        for (int k = 0; k < D; ++k) c += std::abs(m[i * D + k]) > 0.0 ? 1 : 0;
        nnz = std::max(nnz, c);
      }
      if (nnz >= 1 && nnz <= TTNS_SPARSE_MAX && nnz < D) {
        const long long sp = (long long)C.pool_init.size();
        C.pool_init.resize(C.pool_init.size() + 2LL * D * nnz, make_double2(0.0, 0.0));
        for (int i = 0; i < D; ++i) {
          int e = 0;
          for (int k = 0; k < D; ++k) {
            if (std::abs(m[i * D + k]) > 0.0) {
              C.pool_init[sp + (long long)i * nnz + e] = make_double2(m[i * D + k].real(), m[i * D + k].imag());
              C.pool_init[sp + (long long)D * nnz + (long long)i * nnz + e] = make_double2((double)k, 0.0);
              ++e;
            }
          }
        }
        sparse_of[off] = {nnz, sp};
      }
    }
    pending_sparse.clear();
  }
  Factor with_sparse(Factor f) const {
    f.nnz = 0;
    f.sp = 0;
    auto it = sparse_of.find(f.mat);
    if (it != sparse_of.end()) { f.nnz = it->second.first; f.sp = it->second.second; }
    return f;
  }
  long long push_zeros(long long n) {
    long long off = (long long)C.pool_init.size();
    C.pool_init.resize(C.pool_init.size() + n, make_double2(0.0, 0.0));
    return off;
  }

  bool in_piece(int u, int v, int x) const {  // x on u's side of edge (u, v)
    if (t.parent[u] == v) return sub[u][x] != 0;
    return sub[v][x] == 0;
  }
  int toward(int v, int x) const {
    for (int c : t.children[v])
      if (sub[c][x]) return c;
    return t.parent[v];
  }
  // factor of coupling k's end e seen from node u
  Factor end_factor(int u, int k, int e) const {
    const Coupling& cp = t.coups[k];
    if (e == u) return with_sparse(Factor{t.phys_leg(u), e == cp.va ? opa_off[k] : opb_off[k], 0, 0});
    int w = toward(u, e);
    const EnvInfo& E = env.at({w, u});
    int pos = (int)(std::find(E.chans.begin(), E.chans.end(), k) - E.chans.begin());
    if (pos >= (int)E.chans.size()) throw std::logic_error("channel not found");
    return Factor{t.leg_of(u, w), E.off + (long long)(1 + pos) * E.D * E.D, 0, 0};
  }
  int slot(int v, int x) const { return x == v ? -1 : toward(v, x); }

  // terms of node u restricted to all neighbours except `excl` (-1: none)
  // A two-factor term is evaluated directly (one pass, no temporary) when one factor is
  // row-sparse and the direct cost nnz * D_dense is at most twice the two-stage cost.
  static int direct_factor(const Term& T, const NodeDesc& nd) {
    for (int f = 0; f < 2; ++f) {
      const Factor& s_ = T.f[f];
      const Factor& d_ = T.f[1 - f];
      if (s_.nnz > 0 && d_.nnz == 0) {
        const int Dd = nd.dims[d_.leg], Ds = nd.dims[s_.leg];
        if (s_.nnz * Dd <= 2 * (Dd + Ds)) return f;
      }
    }
    return -1;
  }

  int node_terms(int u, int excl) {
    std::vector<Term> one, direct, two;
    const NodeDesc& nd = C.nodes[node0 + u];
    if (!t.onsite[u].empty())
      one.push_back(Term{1, {with_sparse(Factor{t.phys_leg(u), onsite_off[u], 0, 0}), Factor{0, 0, 0, 0}}, -1});
    for (int w : t.neighbours(u)) {
      if (w == excl) continue;
      const EnvInfo& E = env.at({w, u});
      one.push_back(Term{1, {Factor{t.leg_of(u, w), E.off, 0, 0}, Factor{0, 0, 0, 0}}, -1});
    }
    for (int k = 0; k < (int)t.coups.size(); ++k) {
      const Coupling& cp = t.coups[k];
      if (excl >= 0 && (!in_piece(u, excl, cp.va) || !in_piece(u, excl, cp.vb))) continue;
      if (slot(u, cp.va) == slot(u, cp.vb)) continue;
      Term T{2, {end_factor(u, k, cp.va), end_factor(u, k, cp.vb)}, -1};
      T.sparse_f = direct_factor(T, nd);
      (T.sparse_f >= 0 ? direct : two).push_back(T);
    }
    TermList L;
    L.first = (int)C.terms.size();
    L.count = (int)(one.size() + direct.size() + two.size());
    L.n2 = (int)two.size();
    L.nd = (int)direct.size();
    for (auto& x : one) C.terms.push_back(x);
    for (auto& x : direct) C.terms.push_back(x);
    for (auto& x : two) C.terms.push_back(x);
    C.max_tmp = std::max(C.max_tmp, L.n2);
    C.lists.push_back(L);
    return (int)C.lists.size() - 1;
  }

  double list_flops(int li, const NodeDesc& nd) const {
    const TermList& L = C.lists[li];
    double f = 0;
    for (int k = 0; k < L.count; ++k) {
      const Term& T = C.terms[L.first + k];
      for (int j = 0; j < T.nf; ++j) f += 8.0 * nd.size * (T.f[j].nnz > 0 ? T.f[j].nnz : nd.dims[T.f[j].leg]);
    }
    return f;
  }

  NodeDesc make_desc(const std::vector<int>& dims, long long off) {
    NodeDesc d{};
    d.nl = (int)dims.size();
    int s = 1;
    for (int k = d.nl - 1; k >= 0; --k) { d.dims[k] = dims[k]; d.strides[k] = s; s *= dims[k]; }
    d.size = s;
    d.off = off;
    d.reg_off = 0;
    d.reg_len = 0;
    for (int k = 0; k < TTNS_MAX_LEGS; ++k) {
      d.inv_dims[k] = k < d.nl ? 1.0f / (float)d.dims[k] : 0.0f;
      d.inv_strides[k] = k < d.nl ? 1.0f / (float)d.strides[k] : 0.0f;
    }
    return d;
  }

  int team_for(int size, bool qr = false) const {
    if (batched) return TEAM_CLUSTER;
    return size >= (qr ? qr_grid_threshold : grid_threshold) ? TEAM_GRID : TEAM_CLUSTER;
  }

  // Environment pass of a second operator on the tree of an already compiled tree (its
  // nodes node0_existing ..): environment blocks toward the root only, the operator's
  // constant matrices, one instruction per edge in post-order, and the root's term list.
  // Returns (first instruction, count, root term list).
  std::vector<long long> op_reg_off, op_reg_len;
  void compile_operator(int node0_existing, int* first, int* count, int* root_terms) {
    const int n = t.n();
    sub.assign(n, std::vector<char>(n, 0));
    for (int v = n - 1; v >= 0; --v) {
      sub[v][v] = 1;
      for (int c : t.children[v])
        for (int x = 0; x < n; ++x)
          if (sub[c][x]) sub[v][x] = 1;
    }
    node0 = node0_existing;
    onsite_off.assign(n, -1);
    opa_off.assign(t.coups.size(), -1);
    opb_off.assign(t.coups.size(), -1);
    op_reg_off.assign(n, 0);
    op_reg_len.assign(n, 0);
    for (int v = 0; v < n; ++v) {
      const long long reg0 = (long long)C.pool_init.size();
      for (int w : t.children[v]) {
        EnvInfo E;
        E.D = t.bond[w];
        for (int k = 0; k < (int)t.coups.size(); ++k) {
          bool a = in_piece(w, v, t.coups[k].va), b = in_piece(w, v, t.coups[k].vb);
          if (a != b) E.chans.push_back(k);
        }
        E.off = push_zeros((long long)(1 + E.chans.size()) * E.D * E.D);
        env[{w, v}] = E;
      }
      if (!t.onsite[v].empty()) onsite_off[v] = push_operator(t.onsite[v]);
      for (int k = 0; k < (int)t.coups.size(); ++k) {
        if (t.coups[k].va == v) opa_off[k] = push_operator(t.coups[k].opa);
        if (t.coups[k].vb == v) opb_off[k] = push_operator(t.coups[k].opb);
      }
      finish_sparse();
      op_reg_off[v] = reg0;
      op_reg_len[v] = (long long)C.pool_init.size() - reg0;
    }
    std::vector<int> post;
    std::function<void(int)> rec = [&](int v) {
      for (int c : t.children[v]) rec(c);
      post.push_back(v);
    };
    rec(0);
    *first = (int)C.prog.size();
    for (int v : post)
      if (t.parent[v] >= 0) {
        emit_env(v, t.parent[v]);
        Instr& I = C.prog.back();
        I.rega_off = op_reg_off[v];
        I.rega_len = (int)op_reg_len[v];
      }
    *count = (int)C.prog.size() - *first;
    *root_terms = node_terms(0, -1);
  }

  void compile() {
    const int n = t.n();
    sub.assign(n, std::vector<char>(n, 0));
    for (int v = n - 1; v >= 0; --v) {
      sub[v][v] = 1;
      for (int c : t.children[v])
        for (int x = 0; x < n; ++x)
          if (sub[c][x]) sub[v][x] = 1;
    }
    // node tensors with the initial isometric state
    node0 = (int)C.nodes.size();
    for (int v = 0; v < n; ++v) {
      std::vector<int> dims = t.legs(v);
      long long size = 1;
      for (int x : dims) size *= x;
      long long off = push_zeros(size);
      if (t.parent[v] < 0) {
        // root: psi_el on the physical leg, index 0 on every bond
        for (int s = 0; s < t.n_el; ++s) C.pool_init[off + s] = make_double2(t.psi_el[s].real(), t.psi_el[s].imag());
      } else {
        long long rest = size / dims[0];
        for (int k = 0; k < dims[0]; ++k) C.pool_init[off + k * rest + k] = make_double2(1.0, 0.0);
      }
      C.nodes.push_back(make_desc(dims, off));
      C.max_node = std::max<int>(C.max_node, (int)size);
      for (int x : dims) C.max_D = std::max(C.max_D, x);
    }
    // operator regions: for every node v, the environment blocks flowing into v (one
    // directed edge w -> v per neighbour) followed by v's constant operators, contiguous so
    // that an op on v stages them with one copy
    onsite_off.assign(n, -1);
    opa_off.assign(t.coups.size(), -1);
    opb_off.assign(t.coups.size(), -1);
    for (int v = 0; v < n; ++v) {
      const long long reg0 = (long long)C.pool_init.size();
      for (int w : t.neighbours(v)) {
        EnvInfo E;
        E.D = (t.parent[w] == v) ? t.bond[w] : t.bond[v];
        for (int k = 0; k < (int)t.coups.size(); ++k) {
          bool a = in_piece(w, v, t.coups[k].va), b = in_piece(w, v, t.coups[k].vb);
          if (a != b) E.chans.push_back(k);
        }
        E.off = push_zeros((long long)(1 + E.chans.size()) * E.D * E.D);
        env[{w, v}] = E;
      }
      if (!t.onsite[v].empty()) onsite_off[v] = push_operator(t.onsite[v]);
      for (int k = 0; k < (int)t.coups.size(); ++k) {
        if (t.coups[k].va == v) opa_off[k] = push_operator(t.coups[k].opa);
        if (t.coups[k].vb == v) opb_off[k] = push_operator(t.coups[k].opb);
      }
      finish_sparse();  // the node's row-sparse tables close its region (staged with it)
      C.nodes[node0 + v].reg_off = reg0;
      C.nodes[node0 + v].reg_len = (int)((long long)C.pool_init.size() - reg0);
    }
    bond_off = push_zeros((long long)TTNS_MAX_D * TTNS_MAX_D);
    // pseudo nodes for bond matrices
    for (int u = 0; u < n; ++u)
      for (int w : t.neighbours(u)) {
        int D = env[{u, w}].D;
        bond_node[{u, w}] = (int)C.nodes.size();
        C.nodes.push_back(make_desc({D, D}, bond_off));
        C.nodes.back().reg_off = 0;
        C.nodes.back().reg_len = 0;
      }
    // trajectory
    TreeDesc td{};
    td.n_nodes = n;
    td.node0 = node0;
    td.n_el = t.n_el;
    td.root_off = C.nodes[node0].off;
    td.root_phys_leg = t.phys_leg(0);
    td.bond_off = bond_off;
    td.max_node = 0;
    for (int v = 0; v < n; ++v) td.max_node = std::max(td.max_node, C.nodes[node0 + v].size);
    int ns = 0;
    for (auto& c : t.chain_nodes) ns += (int)c.size();
    td.n_sites = ns;

    // initial environment pass: env(c -> parent) in post-order
    std::vector<int> post;
    std::function<void(int)> rec = [&](int v) {
      for (int c : t.children[v]) rec(c);
      post.push_back(v);
    };
    rec(0);
    td.init_first = (int)C.prog.size();
    for (int v : post)
      if (t.parent[v] >= 0) emit_env(v, t.parent[v]);
    td.init_count = (int)C.prog.size() - td.init_first;

    // one step
    td.prog_first = (int)C.prog.size();
    visit(0);
    visit_adj(0);
    Instr r{};
    r.op = OP_RECORD;
    r.team = team_for(C.nodes[node0].size);
    r.tree = tree_idx;
    r.node = node0;
    C.prog.push_back(r);
    td.prog_count = (int)C.prog.size() - td.prog_first;
    td.traj_off = 0;  // assigned later
    C.trees.push_back(td);
    std::vector<int> sites;
    for (auto& c : t.chain_nodes)
      for (int v : c) sites.push_back(node0 + v);
    C.site_nodes.push_back(sites);
  }

  int hist(int a, int b) {
    auto key = std::make_pair(a, b);
    auto it = hist_slot.find(key);
    if (it != hist_slot.end()) return it->second;
    int h = C.n_hist++;
    hist_slot[key] = h;
    return h;
  }

  void emit_fwd(int v) {
    auto it = heff_list.find(v);
    int li = it == heff_list.end() ? (heff_list[v] = node_terms(v, -1)) : it->second;
    Instr I{};
    I.op = OP_FWD;
    I.tree = tree_idx;
    I.node = node0 + v;
    I.team = team_for(C.nodes[I.node].size);
    I.terms = li;
    I.hist = hist(v, -1);
    I.sign = 1.0;
    I.flops = list_flops(li, C.nodes[I.node]);
    set_regions(I, v, -1);
    C.prog.push_back(I);
  }
  void set_regions(Instr& I, int a, int b) {
    I.rega_off = C.nodes[node0 + a].reg_off;
    I.rega_len = C.nodes[node0 + a].reg_len;
    I.regb_off = b >= 0 ? C.nodes[node0 + b].reg_off : 0;
    I.regb_len = b >= 0 ? C.nodes[node0 + b].reg_len : 0;
  }
  void emit_qr(int v, int u) {
    Instr I{};
    I.op = OP_QR;
    I.tree = tree_idx;
    I.node = node0 + v;
    I.team = team_for(C.nodes[I.node].size, true);
    I.leg = t.leg_of(v, u);
    I.D = C.nodes[I.node].dims[I.leg];
    C.prog.push_back(I);
  }
  void emit_env(int u, int v) {
    auto key = std::make_pair(u, v);
    auto it = envh_list.find(key);
    int li;
    if (it == envh_list.end()) {
      li = node_terms(u, v);
      envh_list[key] = li;
      const EnvInfo& E = env.at(key);
      int first = (int)C.chans.size();
      for (int k : E.chans) {
        const Coupling& cp = t.coups[k];
        int e = in_piece(u, v, cp.va) ? cp.va : cp.vb;
        C.chans.push_back(end_factor(u, k, e));
      }
      env_chan[key] = {first, (int)E.chans.size()};
    } else {
      li = it->second;
    }
    const EnvInfo& E = env.at(key);
    Instr I{};
    I.op = OP_ENV;
    I.tree = tree_idx;
    I.node = node0 + u;
    I.team = team_for(C.nodes[I.node].size);
    I.leg = t.leg_of(u, v);
    I.terms = li;
    I.chan_first = env_chan[key].first;
    I.nchan = env_chan[key].second;
    I.env_out = E.off;
    I.D = E.D;
    I.flops = list_flops(li, C.nodes[I.node]) + 8.0 * C.nodes[I.node].size * E.D * (1 + E.chans.size());
    set_regions(I, u, -1);
    C.prog.push_back(I);
  }
  void emit_bond(int u, int w) {
    auto key = std::make_pair(u, w);
    auto it = bond_list.find(key);
    int li;
    if (it == bond_list.end()) {
      const EnvInfo& Eu = env.at({u, w});
      const EnvInfo& Ew = env.at({w, u});
      TermList L;
      L.first = (int)C.terms.size();
      C.terms.push_back(Term{1, {Factor{0, Eu.off, 0, 0}, Factor{0, 0, 0, 0}}, -1});
      C.terms.push_back(Term{1, {Factor{1, Ew.off, 0, 0}, Factor{0, 0, 0, 0}}, -1});
      int n2 = 0;
      for (size_t a = 0; a < Eu.chans.size(); ++a) {
        int k = Eu.chans[a];
        size_t b = std::find(Ew.chans.begin(), Ew.chans.end(), k) - Ew.chans.begin();
        if (b >= Ew.chans.size()) throw std::logic_error("bond channel mismatch");
        C.terms.push_back(Term{2, {Factor{0, Eu.off + (long long)(1 + a) * Eu.D * Eu.D, 0, 0},
                                   Factor{1, Ew.off + (long long)(1 + b) * Ew.D * Ew.D, 0, 0}}, -1});
        ++n2;
      }
      L.count = 2 + n2;
      L.n2 = n2;
      L.nd = 0;
      C.max_tmp = std::max(C.max_tmp, n2);
      C.lists.push_back(L);
      li = (int)C.lists.size() - 1;
      bond_list[key] = li;
    } else {
      li = it->second;
    }
    Instr I{};
    I.op = OP_BOND;
    I.tree = tree_idx;
    I.node = bond_node[key];
    I.team = TEAM_CLUSTER;
    I.terms = li;
    I.D = C.nodes[I.node].dims[0];
    I.D2 = C.nodes[I.node].dims[1];
    I.hist = hist(u, w + 1000000);
    I.sign = -1.0;
    I.flops = list_flops(li, C.nodes[I.node]);
    set_regions(I, u, w);
    if (!batched) I.team = TEAM_CLUSTER;
    C.prog.push_back(I);
  }
  void emit_absorb(int u, int v) {
    Instr I{};
    I.op = OP_ABSORB;
    I.tree = tree_idx;
    I.node = node0 + u;
    I.team = team_for(C.nodes[I.node].size);
    I.leg = t.leg_of(u, v);
    I.D = C.nodes[I.node].dims[I.leg];
    C.prog.push_back(I);
  }

  void visit(int v) {
    emit_fwd(v);
    for (int c : t.children[v]) {
      emit_qr(v, c);
      emit_env(v, c);
      emit_bond(v, c);
      emit_absorb(c, v);
      visit(c);
      emit_qr(c, v);
      emit_env(c, v);
      emit_absorb(v, c);
    }
  }
  void visit_adj(int v) {
    for (auto it = t.children[v].rbegin(); it != t.children[v].rend(); ++it) {
      int c = *it;
      emit_qr(v, c);
      emit_env(v, c);
      emit_absorb(c, v);
      visit_adj(c);
      emit_qr(c, v);
      emit_env(c, v);
      emit_bond(c, v);
      emit_absorb(v, c);
    }
    emit_fwd(v);
  }
};

}  // namespace

Compiled compile_trees(const std::vector<TreeInput>& inputs, bool batched, int grid_threshold,
                       int qr_grid_threshold, int max_record, int record) {
  Compiled C;
  for (size_t i = 0; i < inputs.size(); ++i) {
    C.host.push_back(build_host_tree(inputs[i]));
  }
  for (size_t i = 0; i < inputs.size(); ++i) {
    TreeCompiler tc(C.host[i], C, (int)i, batched, grid_threshold, qr_grid_threshold);
    tc.compile();
    TreeDesc& td = C.trees.back();
    td.heff_terms = tc.heff_list.at(0);
    // the chains' kinetic energy on the same tree (energy surfaces): its environment pass
    // reads the node tensors of this tree
    const HostTree kin = kinetic_tree(C.host[i], inputs[i]);
    TreeCompiler kc(kin, C, (int)i, batched, grid_threshold, qr_grid_threshold);
    kc.compile_operator(td.node0, &td.obs_first, &td.obs_count, &td.teff_terms);
  }
  // trajectory buffers at the end of the pool
  for (auto& td : C.trees) {
    if (record) {
      td.traj_off = (long long)C.pool_init.size();
      C.pool_init.resize(C.pool_init.size() + (size_t)max_record * td.n_el * td.n_el, make_double2(0, 0));
    } else {
      td.traj_off = -1;
    }
  }
  C.pool_size = (long long)C.pool_init.size();
  return C;
}

}  // namespace ttns
