// C ABI of the TTNS sweep library (declarations and contracts in include/ttns.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ttns.h"
#include "internal.h"
#include "model.h"

namespace ttns {
cudaError_t launch_sweep(const KernelParams& P, int phase, int grid, int cluster, int cooperative,
                         cudaStream_t stream);
cudaError_t max_grid_for(int cluster, long long smem_bytes, int* grid);
cudaError_t launch_density(const double2* pool, const NodeDesc& nd, int l, const double2* rho_in, double2* xbuf,
                           double* partials,
                           int nblocks, double* out, cudaStream_t st);
cudaError_t launch_energy(const KernelParams& P, int node, int terms, int n2, double* partials, int nblocks,
                          double* out, cudaStream_t st);
cudaError_t launch_occ(const double2* dens, int d, double* out, cudaStream_t st);
cudaError_t launch_wait_selftest(Ctl* ctl, long long spin_limit, int skip, cudaStream_t st);
cudaError_t launch_apply_x(const KernelParams& P, int node, int terms, int n2, const double2* x, double2* y,
                           int nblocks, cudaStream_t st);
cudaError_t launch_herm_jacobi(const double2* base, const long long* offs, const int* ns, const int* lds, int count,
                               int n_max, double* evals, double2* evecs, cudaStream_t st);
cudaError_t launch_bath_states(const double2* A, long long R, int n_el, const double2* U, const double* sig, int nb,
                               double2* Phi, cudaStream_t st);
cudaError_t launch_build_x(const double2* Phi, int k, int l, long long R, int n_el, double2* X, cudaStream_t st);
cudaError_t launch_project(const double2* y, const double2* Phi, long long R, int n_el, int nb, double* partials,
                           int nblocks, double* out, cudaStream_t st);
cudaError_t launch_sub(const double* a, const double* b, double* c, int n, cudaStream_t st);
cudaError_t launch_mirror32(const double2* pool, float2* pool32, long long n, cudaStream_t st);
cudaError_t launch_pad_copy(const double2* src_pool, const NodeDesc& so, double2* dst_pool, const NodeDesc& dn,
                            cudaStream_t st);
}  // namespace ttns

using namespace ttns;

static thread_local std::string g_err;

namespace ttns {
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace ttns

static ttns_status fail(ttns_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

struct ttns_tree {
  Compiled C;
  std::vector<TreeInput> inputs;  // validated problems (written into checkpoints)
  ttns_options opt{};
  bool batched = false;
  int grid = 0, cluster = 16;
  cudaStream_t stream = nullptr;
  // device buffers
  double2* pool = nullptr;
  float2* pool32 = nullptr;  // FP32 mirror of the pool (mixed modes)
  NodeDesc* d_nodes = nullptr;
  Term* d_terms = nullptr;
  TermList* d_lists = nullptr;
  Factor* d_chans = nullptr;
  Instr* d_prog = nullptr;
  TreeDesc* d_trees = nullptr;
  Ctl* ctl = nullptr;
  double2* work = nullptr;
  double* red = nullptr;
  double* red_grid = nullptr;
  double2* cta_scratch = nullptr;
  int* mhist = nullptr;
  int* traj_count = nullptr;
  double* obs = nullptr;        // observable scratch (partials + outputs)
  long long obs_size = 0;
  // regions of obs (doubles)
  long long o_bond = 0, o_site = 0, o_occ = 0, o_rho = 0, o_en = 0;
  KernelParams P{};
  std::vector<void*> allocs;
  double t_fs = 0.0;
  // step launches not yet confirmed by a synchronising call (dt, n), and how often a launch
  // was repeated as a plain cluster launch (see run_launch)
  std::vector<std::pair<double, int>> pending;
  long long launch_fallbacks = 0;
  // scratch of the energy surfaces and bond entropies (allocated on first use)
  double* surf = nullptr;
  long long surf_size = 0;
};

// Launch of the persistent kernel with the tree set's launch options.  launch_flags bit 1 is a
// host-side fault injection for tests: step launches get clusters of one CTA (as a profiler
// that drops the cluster shape of cooperative launches would give them) until the library has
// switched to plain cluster launches; the kernel's launch check refuses each before any
// barrier or distributed-shared-memory access.
static cudaError_t launch_persistent(ttns_tree* t, const ttns::KernelParams& P, int phase) {
  const bool inject = (t->opt.launch_flags & 2) && !(t->opt.launch_flags & 1) && phase == 1;
  return ttns::launch_sweep(P, phase, t->grid, inject ? 1 : t->cluster, !(t->opt.launch_flags & 1), t->stream);
}

static const char* kStatusNames[] = {"ok", "invalid", "oom", "cuda", "not converged", "timeout", "nonfinite", "io"};

extern "C" const char* ttns_last_error(void) { return g_err.c_str(); }

static std::string status_text(const Ctl& h) {
  if (h.err_where == 300)
    return std::string(kStatusNames[h.status]) + ": the persistent kernel ran with a cluster of " +
           std::to_string(h.err_node) + " CTAs or less dynamic shared memory than planned";
  return std::string(kStatusNames[h.status]) + " (op " + std::to_string(h.err_where) + ", node " +
         std::to_string(h.err_node) + ")";
}

#define CUDA_TRY(x)                                                                          \
  do {                                                                                       \
    cudaError_t e_ = (x);                                                                    \
    if (e_ != cudaSuccess) return fail(TTNS_E_CUDA, std::string(#x ": ") + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
static ttns_status dalloc(ttns_tree* t, T** p, size_t count) {
  void* q = nullptr;
  size_t bytes = std::max<size_t>(count * sizeof(T), 16);
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(TTNS_E_OOM, std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
  }
  t->allocs.push_back(q);
  *p = (T*)q;
  return TTNS_OK;
}

template <typename T>
static ttns_status upload(ttns_tree* t, T** p, const std::vector<T>& h) {
  ttns_status s = dalloc(t, p, h.size());
  if (s != TTNS_OK) return s;
  if (!h.empty()) CUDA_TRY(cudaMemcpyAsync(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, t->stream));
  return TTNS_OK;
}

static bool hermitian(const double* M, int n) {
  double scale = 0;
  for (int k = 0; k < 2 * n * n; ++k) scale = std::max(scale, std::fabs(M[k]));
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const double* a = M + 2 * (i * n + j);
      const double* b = M + 2 * (j * n + i);
      if (std::fabs(a[0] - b[0]) > 1e-12 * (1 + scale) || std::fabs(a[1] + b[1]) > 1e-12 * (1 + scale)) return false;
    }
  return true;
}

static ttns_status validate(const ttns_problem* p, const ttns_options* opt, TreeInput* in) {
  if (!p) return fail(TTNS_E_INVALID, "problem is NULL");
  if (p->n_el < 1 || p->n_el > TTNS_MAX_D) return fail(TTNS_E_INVALID, "n_el out of range");
  if (!p->H_S || !p->W_bar || !p->rc_coupling || !p->chain_len || !p->chain_omega || !p->local_dim || !p->bond_dim)
    return fail(TTNS_E_INVALID, "NULL array in problem");
  if (p->n_env < 1 || p->n_env > 64) return fail(TTNS_E_INVALID, "n_env out of range");
  const int er = opt ? opt->er_tree : 0;
  if (er && (p->n_env < 2 || (p->n_env & (p->n_env - 1)) != 0))
    return fail(TTNS_E_INVALID, "er_tree needs a power-of-two number of environments >= 2");
  if (er && opt->D_er < 1) return fail(TTNS_E_INVALID, "D_er must be >= 1");
  const int ne = p->n_el;
  if (!hermitian(p->H_S, ne)) return fail(TTNS_E_INVALID, "H_S is not Hermitian");
  in->n_el = ne;
  in->n_env = p->n_env;
  in->H_S.resize(ne * ne);
  for (int k = 0; k < ne * ne; ++k) in->H_S[k] = cplx(p->H_S[2 * k], p->H_S[2 * k + 1]);
  for (int i = 0; i < p->n_env; ++i) {
    const double* W = p->W_bar + (size_t)2 * ne * ne * i;
    if (!hermitian(W, ne)) return fail(TTNS_E_INVALID, "W_bar[" + std::to_string(i) + "] is not Hermitian");
    std::vector<cplx> w(ne * ne);
    for (int k = 0; k < ne * ne; ++k) w[k] = cplx(W[2 * k], W[2 * k + 1]);
    in->W.push_back(w);
    const int L = p->chain_len[i], d = p->local_dim[i], D = p->bond_dim[i];
    if (L < 1 || L > 4096) return fail(TTNS_E_INVALID, "chain_len out of range");
    if (d < 2 || d > TTNS_MAX_D) return fail(TTNS_E_INVALID, "local_dim out of range (2..64)");
    if (D < 1) return fail(TTNS_E_INVALID, "bond_dim must be >= 1");
    if (!std::isfinite(p->rc_coupling[i])) return fail(TTNS_E_INVALID, "rc_coupling not finite");
    if (!p->chain_omega[i]) return fail(TTNS_E_INVALID, "chain_omega entry is NULL");
    if (L > 1 && (!p->chain_hop || !p->chain_hop[i])) return fail(TTNS_E_INVALID, "chain_hop entry is NULL");
    in->rc.push_back(p->rc_coupling[i]);
    in->omega.emplace_back(p->chain_omega[i], p->chain_omega[i] + L);
    if (L > 1)
      in->hop.emplace_back(p->chain_hop[i], p->chain_hop[i] + (L - 1));
    else
      in->hop.emplace_back();
    in->L.push_back(L);
    in->d.push_back(d);
    in->D.push_back(D);
    const int obb = p->obb_dim ? p->obb_dim[i] : 0;
    if (obb < 0) return fail(TTNS_E_INVALID, "obb_dim must be >= 0");
    in->obb.push_back(obb);
  }
  in->er_tree = er;
  in->D_er = er ? opt->D_er : 0;
  in->psi_el.assign(ne, cplx(0, 0));
  if (opt && opt->psi_el) {
    double nn = 0;
    for (int s = 0; s < ne; ++s) {
      in->psi_el[s] = cplx(opt->psi_el[2 * s], opt->psi_el[2 * s + 1]);
      nn += std::norm(in->psi_el[s]);
    }
    if (!(nn > 0) || !std::isfinite(nn)) return fail(TTNS_E_INVALID, "psi_el is zero or not finite");
  } else {
    const int s0 = opt ? opt->init_state : 0;
    if (s0 < 0 || s0 >= ne) return fail(TTNS_E_INVALID, "init_state out of range");
    in->psi_el[s0] = 1.0;
  }
  return TTNS_OK;
}

// Checks every offset of the compiled tables against the buffers they index, so that a
// malformed table is reported on the host instead of reaching the device.
static ttns_status check_tables(const Compiled& C, int mmax, long long kvec, long long per_cta, int n_tmp) {
  auto in_pool = [&](long long off, long long n) { return off >= 0 && n >= 0 && off + n <= C.pool_size; };
  for (size_t i = 0; i < C.nodes.size(); ++i) {
    const NodeDesc& nd = C.nodes[i];
    if (nd.nl < 1 || nd.nl > TTNS_MAX_LEGS) return fail(TTNS_E_INVALID, "table: leg count");
    long long sz = 1;
    for (int k = 0; k < nd.nl; ++k) {
      if (nd.dims[k] < 1 || nd.dims[k] > TTNS_MAX_D) return fail(TTNS_E_INVALID, "table: dim out of range");
      sz *= nd.dims[k];
    }
    if (sz != nd.size || !in_pool(nd.off, nd.size) || nd.size > kvec) return fail(TTNS_E_INVALID, "table: node extent");
    if (nd.size >= (1 << 24)) return fail(TTNS_E_INVALID, "table: a tensor has 2^24 or more elements");
  }
  auto check_factor = [&](const Factor& f, const NodeDesc& nd) {
    if (f.leg < 0 || f.leg >= nd.nl) return false;
    const long long D = nd.dims[f.leg];
    if (f.nnz < 0 || f.nnz > TTNS_SPARSE_MAX) return false;
    if (f.nnz > 0) {
      if (!in_pool(f.sp, 2 * D * f.nnz)) return false;
      for (long long e = 0; e < D * f.nnz; ++e) {
        const double c = C.pool_init[f.sp + D * f.nnz + e].x;
        if (!(c >= 0.0 && c < (double)D)) return false;  // column index in range
      }
    }
    return in_pool(f.mat, D * D);
  };
  for (const Instr& I : C.prog) {
    if (I.node < 0 || I.node >= (int)C.nodes.size()) return fail(TTNS_E_INVALID, "table: instruction node");
    if (I.tree < 0 || I.tree >= (int)C.trees.size()) return fail(TTNS_E_INVALID, "table: instruction tree");
    const NodeDesc& nd = C.nodes[I.node];
    const TreeDesc& td = C.trees[I.tree];
    if (!in_pool(td.bond_off, (long long)TTNS_MAX_D * TTNS_MAX_D)) return fail(TTNS_E_INVALID, "table: bond buffer");
    if (I.op == OP_FWD || I.op == OP_BOND || I.op == OP_ENV) {
      if (I.terms < 0 || I.terms >= (int)C.lists.size()) return fail(TTNS_E_INVALID, "table: term list");
      const TermList& L = C.lists[I.terms];
      if (L.first < 0 || L.first + L.count > (int)C.terms.size() || L.n2 > n_tmp || L.n2 > L.count ||
          L.count > TTNS_MAX_TERMS)
        return fail(TTNS_E_INVALID, "table: term range");
      const int n1 = L.count - L.n2 - L.nd;
      if (n1 < 0 || L.nd < 0) return fail(TTNS_E_INVALID, "table: term counts");
      for (int k = 0; k < L.count; ++k) {
        const Term& T = C.terms[L.first + k];
        const bool two = k >= n1;
        if (T.nf != (two ? 2 : 1)) return fail(TTNS_E_INVALID, "table: term order");
        const bool direct = k >= n1 && k < n1 + L.nd;
        if (direct && (T.sparse_f < 0 || T.sparse_f > 1 || T.f[T.sparse_f].nnz <= 0))
          return fail(TTNS_E_INVALID, "table: direct term without a sparse factor");
        for (int j = 0; j < T.nf; ++j)
          if (!check_factor(T.f[j], nd)) return fail(TTNS_E_INVALID, "table: factor");
      }
      if (I.op != OP_ENV && (I.hist < 0 || I.hist >= std::max(C.n_hist, 1))) return fail(TTNS_E_INVALID, "table: hist");
    }
    if (I.op == OP_ENV) {
      if (I.leg < 0 || I.leg >= nd.nl || I.D != nd.dims[I.leg]) return fail(TTNS_E_INVALID, "table: env leg");
      if (I.chan_first < 0 || I.chan_first + I.nchan > (int)C.chans.size() || I.nchan > 16)
        return fail(TTNS_E_INVALID, "table: chans");
      for (int b = 0; b < I.nchan; ++b)
        if (!check_factor(C.chans[I.chan_first + b], nd)) return fail(TTNS_E_INVALID, "table: channel factor");
      if (!in_pool(I.env_out, (long long)(1 + I.nchan) * I.D * I.D)) return fail(TTNS_E_INVALID, "table: env out");
      if (1 + I.nchan > mmax || 2LL * (1 + I.nchan) * I.D * I.D > per_cta) return fail(TTNS_E_INVALID, "table: env size");
    }
    if (I.op == OP_QR || I.op == OP_ABSORB) {
      if (I.leg < 0 || I.leg >= nd.nl || I.D != nd.dims[I.leg]) return fail(TTNS_E_INVALID, "table: qr leg");
      if (nd.size / I.D < I.D) return fail(TTNS_E_INVALID, "table: qr needs rows >= cols");
      if (2LL * I.D * I.D > per_cta) return fail(TTNS_E_INVALID, "table: qr partials");
    }
    if (I.op == OP_BOND) {
      if (nd.off != td.bond_off || nd.nl != 2) return fail(TTNS_E_INVALID, "table: bond node");
    }
    if (I.op == OP_RECORD) {
      if (td.n_el * td.n_el * 2LL > per_cta) return fail(TTNS_E_INVALID, "table: record partials");
      if (td.traj_off >= 0 && !in_pool(td.traj_off, 0)) return fail(TTNS_E_INVALID, "table: trajectory");
    }
  }
  return TTNS_OK;
}

struct Sizes {
  int mmax;
  long long kvec, work_stride, per_cta;
  int maxchan;
};

static ttns_status plan_sizes(const Compiled& C, const ttns_options& o, Sizes* z) {
  z->mmax = std::min(o.krylov_mmax > 0 ? o.krylov_mmax : 30, TTNS_KMAX);
  z->maxchan = 0;
  for (const Instr& I : C.prog) z->maxchan = std::max(z->maxchan, I.nchan);
  if (1 + z->maxchan > z->mmax) return fail(TTNS_E_INVALID, "too many coupling channels for krylov_mmax");
  if (C.max_D > TTNS_MAX_D) return fail(TTNS_E_INVALID, "a bond dimension exceeds 64");
  z->kvec = ((long long)C.max_node + 31) / 32 * 32;
  // Krylov vectors, two-factor temporaries, the compute-type shadow and a spare slot, and eight
  // slots for the tensor-core partial results (up to sixteen compute-type vectors)
  z->work_stride = (long long)(z->mmax + std::max(C.max_tmp, 1) + 2 + 8) * z->kvec;
  long long per_cta = 8;
  per_cta = std::max<long long>(per_cta, 2LL * C.max_D * C.max_D);
  per_cta = std::max<long long>(per_cta, 2LL * (1 + z->maxchan) * C.max_D * C.max_D);
  per_cta = std::max<long long>(per_cta, 2LL * TTNS_MAX_D);
  per_cta = std::max<long long>(per_cta, 2LL * (TTNS_KMAX + 1));  // reorthogonalisation dots
  z->per_cta = per_cta;
  return check_tables(C, z->mmax, z->kvec, per_cta, std::max(C.max_tmp, 1));
}

// A persistent launch refused by the kernel's own launch check: it returned before any work
// because it did not get the planned cluster shape (a profiler re-launches a cooperative
// cluster launch with clusters of one CTA).
static bool launch_refused(const Ctl& h) { return h.status == TTNS_E_CUDA && h.err_where == 300; }

// Waits for the tree's stream and reads the device status word.  Launches that the kernel's
// launch check refused are repeated once, in order, as plain cluster launches (launch_flags
// bit 0), which keep their cluster shape under such tools: the initial environment pass when
// `phase0`, then every step launched since the last check.  Nothing ran in the refused
// launches, so the repeat is the computation that was asked for.
static ttns_status wait_and_check(ttns_tree* t, bool phase0, const char* what) {
  CUDA_TRY(cudaStreamSynchronize(t->stream));
  Ctl h;
  CUDA_TRY(cudaMemcpy(&h, t->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  if (launch_refused(h) && !(t->opt.launch_flags & 1)) {
    t->opt.launch_flags |= 1;
    ++t->launch_fallbacks;
    h.status = 0;
    h.err_where = 0;
    h.err_node = 0;
    CUDA_TRY(cudaMemcpy(t->ctl, &h, sizeof(Ctl), cudaMemcpyHostToDevice));
    if (phase0) {
      KernelParams P0 = t->P;
      P0.dt = 0.0;
      P0.n_steps = 1;
      CUDA_TRY(launch_sweep(P0, 0, t->grid, t->cluster, 0, t->stream));
    }
    for (const auto& pr : t->pending) {
      t->P.dt = pr.first;
      t->P.n_steps = pr.second;
      CUDA_TRY(launch_sweep(t->P, 1, t->grid, t->cluster, 0, t->stream));
    }
    CUDA_TRY(cudaStreamSynchronize(t->stream));
    CUDA_TRY(cudaMemcpy(&h, t->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  }
  t->pending.clear();
  if (h.status != 0) return fail((ttns_status)h.status, std::string(what) + status_text(h));
  return TTNS_OK;
}

static ttns_status device_init(ttns_tree* t) {
  Compiled& C = t->C;
  const ttns_options& o = t->opt;
  Sizes z;
  ttns_status s = plan_sizes(C, o, &z);
  if (s != TTNS_OK) return s;
  const int mmax = z.mmax;
  const long long kvec = z.kvec, work_stride = z.work_stride, per_cta = z.per_cta;
  t->cluster = o.cluster_ctas > 0 ? o.cluster_ctas : 16;
  if (t->cluster > 16) return fail(TTNS_E_INVALID, "cluster_ctas must be <= 16");
  int maxgrid = 0;
  const long long smem_bytes = 200 * 1024;
  // the QR keeps three reduction buffers of 2 n^2 doubles (n <= TTNS_MAX_D) in it
  static_assert(3LL * 2 * TTNS_MAX_D * TTNS_MAX_D * 8 <= 200 * 1024, "QR reduction buffers exceed the shared memory");
  CUDA_TRY(max_grid_for(t->cluster, smem_bytes, &maxgrid));
  if (maxgrid < t->cluster) return fail(TTNS_E_CUDA, "no co-resident cluster of the requested size");
  int grid = o.grid_ctas > 0 ? o.grid_ctas : maxgrid;
  grid = std::min(grid, maxgrid);
  grid = (grid / t->cluster) * t->cluster;
  if (grid < t->cluster) grid = t->cluster;
  bool any_grid = false;
  for (const Instr& I : C.prog) any_grid = any_grid || I.team == TEAM_GRID;
  if (!t->batched && !any_grid) grid = t->cluster;  // one cluster does everything
  t->grid = grid;
  const int n_clusters = grid / t->cluster;
  const int n_workers = t->batched ? n_clusters : 1;
  if ((s = dalloc(t, &t->pool, C.pool_size)) != TTNS_OK) return s;
  CUDA_TRY(cudaMemcpyAsync(t->pool, C.pool_init.data(), C.pool_size * sizeof(double2), cudaMemcpyHostToDevice, t->stream));
  if (o.precision != TTNS_FP64) {
    if ((s = dalloc(t, &t->pool32, C.pool_size)) != TTNS_OK) return s;
    CUDA_TRY(launch_mirror32(t->pool, t->pool32, C.pool_size, t->stream));
  }
  if ((s = upload(t, &t->d_nodes, C.nodes)) != TTNS_OK) return s;
  if ((s = upload(t, &t->d_terms, C.terms)) != TTNS_OK) return s;
  if ((s = upload(t, &t->d_lists, C.lists)) != TTNS_OK) return s;
  if ((s = upload(t, &t->d_chans, C.chans)) != TTNS_OK) return s;
  if ((s = upload(t, &t->d_prog, C.prog)) != TTNS_OK) return s;
  if ((s = upload(t, &t->d_trees, C.trees)) != TTNS_OK) return s;
  if ((s = dalloc(t, &t->ctl, 1)) != TTNS_OK) return s;
  CUDA_TRY(cudaMemsetAsync(t->ctl, 0, sizeof(Ctl), t->stream));
  if ((s = dalloc(t, &t->work, (size_t)n_workers * work_stride)) != TTNS_OK) return s;
  CUDA_TRY(cudaMemsetAsync(t->work, 0, (size_t)n_workers * work_stride * sizeof(double2), t->stream));
  const long long red_stride = (long long)t->cluster * per_cta;
  if ((s = dalloc(t, &t->red, (size_t)n_clusters * 2 * red_stride)) != TTNS_OK) return s;
  const long long red_stride_grid = (long long)grid * per_cta;
  if ((s = dalloc(t, &t->red_grid, (size_t)2 * red_stride_grid)) != TTNS_OK) return s;
  const long long scr = 3LL * TTNS_MAX_D * TTNS_MAX_D;
  if ((s = dalloc(t, &t->cta_scratch, (size_t)grid * scr)) != TTNS_OK) return s;
  if ((s = dalloc(t, &t->mhist, std::max(C.n_hist, 1))) != TTNS_OK) return s;
  CUDA_TRY(cudaMemsetAsync(t->mhist, 0, std::max(C.n_hist, 1) * sizeof(int), t->stream));
  if ((s = dalloc(t, &t->traj_count, C.trees.size())) != TTNS_OK) return s;
  CUDA_TRY(cudaMemsetAsync(t->traj_count, 0, C.trees.size() * sizeof(int), t->stream));
  // observables scratch: partials for up to 1024 blocks of 2*maxD^2 doubles + densities per node
  const long long nn = (long long)C.nodes.size();
  const long long d2 = 2LL * C.max_D * C.max_D;
  t->o_bond = 1024LL * d2;
  t->o_site = t->o_bond + nn * d2;
  t->o_occ = t->o_site + nn * d2;
  // rho_S is read as complex (16-byte loads) by the eigen kernels: 256-byte aligned
  t->o_rho = (t->o_occ + nn + 64 + 31) & ~31LL;
  t->o_en = t->o_rho + 2 * 64 * 64;
  t->obs_size = t->o_en + 16;
  if ((s = dalloc(t, &t->obs, t->obs_size)) != TTNS_OK) return s;

  KernelParams& P = t->P;
  P.pool = t->pool;
  P.pool32 = t->pool32;
  P.nodes = t->d_nodes;
  P.terms = t->d_terms;
  P.lists = t->d_lists;
  P.chans = t->d_chans;
  P.prog = t->d_prog;
  P.trees = t->d_trees;
  P.n_trees = (int)C.trees.size();
  P.batched = t->batched ? 1 : 0;
  P.ctl = t->ctl;
  P.work = t->work;
  P.work_stride = work_stride;
  P.kvec = (int)kvec;
  P.n_tmp = std::max(C.max_tmp, 1);
  P.red = t->red;
  P.red_stride = red_stride;
  P.red_grid = t->red_grid;
  P.red_stride_grid = red_stride_grid;
  P.cta_scratch = t->cta_scratch;
  P.cta_scratch_stride = scr;
  P.mhist = t->mhist;
  P.traj_count = t->traj_count;
  P.max_record = o.max_record > 0 ? o.max_record : 4096;
  P.record = o.record;
  P.dt = 0.0;
  P.n_steps = 1;
  P.precision = o.precision;
  P.tol = o.krylov_tol > 0 ? o.krylov_tol : 1e-12;
  P.mmax = mmax;
  P.cluster_ctas = t->cluster;
  P.spin_limit = o.spin_limit > 0 ? o.spin_limit : 20LL * 1000 * 1000 * 1000;  // SM clock cycles (~10 s)
  P.profile = o.profile;
  P.smem_bytes = smem_bytes;
  P.cluster_resident = 1;
  P.qr_cutoff = o.qr_cutoff > 0.0 ? o.qr_cutoff : 1e-8;
  // initial environment pass
  CUDA_TRY(launch_persistent(t, P, 0));
  return wait_and_check(t, true, "device status after the initial pass: ");
}

static ttns_status check_options(const ttns_options& o) {
  if (o.precision < TTNS_FP64 || o.precision > TTNS_FP32) return fail(TTNS_E_INVALID, "unknown precision");
  if (o.krylov_mmax < 0 || o.krylov_mmax > TTNS_KMAX) return fail(TTNS_E_INVALID, "krylov_mmax out of range (0..32)");
  if (o.krylov_tol < 0) return fail(TTNS_E_INVALID, "krylov_tol < 0");
  if (o.max_record < 0) return fail(TTNS_E_INVALID, "max_record < 0");
  if (o.grid_threshold < 0 || o.qr_grid_threshold < 0 || o.spin_limit < 0)
    return fail(TTNS_E_INVALID, "negative grid_threshold, qr_grid_threshold or spin_limit");
  if (!(o.qr_cutoff >= 0.0 && o.qr_cutoff < 1.0)) return fail(TTNS_E_INVALID, "qr_cutoff must be in [0, 1)");
  return TTNS_OK;
}

// Builds the host model and the compiled step of validated inputs into t.
static ttns_status compile_inputs(std::vector<TreeInput> ins, const ttns_options& o, ttns_tree* t) {
  ttns_status s = check_options(o);
  if (s != TTNS_OK) return s;
  t->opt = o;
  t->opt.psi_el = nullptr;
  t->batched = ins.size() > 1;
  t->stream = (cudaStream_t)o.cuda_stream;
  try {
    t->C = compile_trees(ins, t->batched, o.grid_threshold > 0 ? o.grid_threshold : 16384,
                         o.qr_grid_threshold > 0 ? o.qr_grid_threshold : 65536, o.max_record > 0 ? o.max_record : 4096,
                         o.record);
  } catch (const std::exception& e) {
    return fail(TTNS_E_INVALID, std::string("model: ") + e.what());
  }
  t->inputs = std::move(ins);
  return TTNS_OK;
}

static ttns_status compile_only(int n_trees, const ttns_problem* probs, const ttns_options* opt, ttns_tree* t) {
  ttns_options o{};
  if (opt) o = *opt;
  ttns_status s = check_options(o);
  if (s != TTNS_OK) return s;
  std::vector<TreeInput> ins(n_trees);
  for (int i = 0; i < n_trees; ++i) {
    s = validate(&probs[i], &o, &ins[i]);
    if (s != TTNS_OK) return s;
  }
  return compile_inputs(std::move(ins), o, t);
}

extern "C" ttns_status ttns_plan(int n_trees, const ttns_problem* problems, const ttns_options* opt,
                                 ttns_plan_info* info) {
  if (!info) return fail(TTNS_E_INVALID, "info is NULL");
  if (n_trees < 1 || !problems) return fail(TTNS_E_INVALID, "no problems");
  ttns_tree t;
  ttns_status s = compile_only(n_trees, problems, opt, &t);
  if (s != TTNS_OK) return s;
  Sizes z;
  if ((s = plan_sizes(t.C, t.opt, &z)) != TTNS_OK) return s;
  std::memset(info, 0, sizeof(*info));
  info->n_nodes = 0;
  for (const TreeDesc& td : t.C.trees) info->n_nodes += td.n_nodes;
  info->pool_complex = t.C.pool_size;
  info->max_node = t.C.max_node;
  info->max_bond = t.C.max_D;
  info->instructions_per_step = 0;
  for (const TreeDesc& td : t.C.trees) info->instructions_per_step += td.prog_count;
  info->work_complex_per_worker = z.work_stride;
  const HostTree& h = t.C.host[0];
  for (int v = 0; v < h.n() && v < 4096; ++v) info->bonds[v] = h.bond[v];
  info->n_bonds_written = std::min(h.n(), 4096);
  // useful flops of one step if every exponential took one Krylov iteration (scale by the counted iterations)
  double fexp = 0, fenv = 0;
  long long nexp = 0, nenv = 0;
  for (const Instr& I : t.C.prog) {
    if (I.op == OP_FWD || I.op == OP_BOND) { fexp += I.flops; ++nexp; }
    if (I.op == OP_ENV) { fenv += I.flops; ++nenv; }
  }
  info->apply_flops_per_step = fexp;
  info->env_flops_per_step = fenv;
  info->exponentials_per_step = nexp;
  info->env_updates_per_step = nenv;
  return TTNS_OK;
}

static ttns_status finish_build(ttns_tree* t, ttns_tree** out) {
  ttns_status s = device_init(t);
  if (s != TTNS_OK) {
    std::string keep = g_err;
    ttns_free(t);
    g_err = keep;
    return s;
  }
  *out = t;
  return TTNS_OK;
}

static ttns_status build(int n_trees, const ttns_problem* probs, const ttns_options* opt, ttns_tree** out) {
  if (!out) return fail(TTNS_E_INVALID, "out is NULL");
  *out = nullptr;
  if (n_trees < 1 || !probs) return fail(TTNS_E_INVALID, "no problems");
  ttns_tree* t = new ttns_tree();
  ttns_status s0 = compile_only(n_trees, probs, opt, t);
  if (s0 != TTNS_OK) {
    delete t;
    return s0;
  }
  return finish_build(t, out);
}

static ttns_status build_inputs(std::vector<TreeInput> ins, const ttns_options& o, ttns_tree** out) {
  ttns_tree* t = new ttns_tree();
  ttns_status s0 = compile_inputs(std::move(ins), o, t);
  if (s0 != TTNS_OK) {
    delete t;
    return s0;
  }
  return finish_build(t, out);
}

// Autotuner of the team shape: for each candidate number of CTAs per cluster team, build the
// same tree set, run one warm-up step and time one step with CUDA events on the options'
// stream, free it; report the fastest.  The state evolves differently only by rounding, so
// any candidate gives a valid run; the choice is purely a performance one.
extern "C" ttns_status ttns_autotune(int n_trees, const ttns_problem* problems, const ttns_options* opt, double dt_fs,
                                     int n_candidates, const int* candidates, int* best_cluster_ctas,
                                     double* best_seconds_per_step) {
  if (!best_cluster_ctas) return fail(TTNS_E_INVALID, "best_cluster_ctas is NULL");
  if (!std::isfinite(dt_fs) || dt_fs == 0.0) return fail(TTNS_E_INVALID, "dt must be finite and nonzero");
  static const int kDefault[3] = {16, 8, 4};
  if (n_candidates < 0 || (n_candidates > 0 && !candidates)) return fail(TTNS_E_INVALID, "bad candidate list");
  const int nc = n_candidates > 0 ? n_candidates : 3;
  const int* cand = n_candidates > 0 ? candidates : kDefault;
  for (int k = 0; k < nc; ++k)
    if (cand[k] < 1 || cand[k] > 16) return fail(TTNS_E_INVALID, "cluster candidates must be in 1..16");
  ttns_options base{};
  if (opt) base = *opt;
  base.record = 0;
  base.profile = 0;
  int best = 0;
  double best_s = 0.0;
  std::string last_err;
  for (int k = 0; k < nc; ++k) {
    ttns_options o = base;
    o.cluster_ctas = cand[k];
    ttns_tree* t = nullptr;
    if (build(n_trees, problems, &o, &t) != TTNS_OK) {
      last_err = g_err;
      continue;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = -1.0f;
    bool ok = ttns_step(t, dt_fs, 1) == TTNS_OK && ttns_sync(t) == TTNS_OK;
    ok = ok && cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
    ok = ok && cudaEventRecord(e0, t->stream) == cudaSuccess && ttns_step(t, dt_fs, 1) == TTNS_OK &&
         cudaEventRecord(e1, t->stream) == cudaSuccess && ttns_sync(t) == TTNS_OK &&
         cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    if (!ok) last_err = g_err;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    ttns_free(t);
    if (ok && ms >= 0.0f && (best == 0 || ms * 1e-3 < best_s)) {
      best = cand[k];
      best_s = ms * 1e-3;
    }
  }
  if (best == 0) return fail(TTNS_E_CUDA, "autotune: no candidate ran (" + last_err + ")");
  *best_cluster_ctas = best;
  if (best_seconds_per_step) *best_seconds_per_step = best_s;
  return TTNS_OK;
}

extern "C" ttns_status ttns_build_tree(const ttns_problem* problem, const ttns_options* opt, ttns_tree** out) {
  return build(1, problem, opt, out);
}

extern "C" ttns_status ttns_build_batch(int n_trees, const ttns_problem* problems, const ttns_options* opt,
                                        ttns_tree** out) {
  return build(n_trees, problems, opt, out);
}

extern "C" ttns_status ttns_step(ttns_tree* t, double dt_fs, int n_steps) {
  if (!t) return fail(TTNS_E_INVALID, "tree is NULL");
  if (n_steps < 0) return fail(TTNS_E_INVALID, "n_steps < 0");
  if (!std::isfinite(dt_fs)) return fail(TTNS_E_INVALID, "dt not finite");
  if (n_steps == 0) return TTNS_OK;
  t->P.dt = dt_fs;
  t->P.n_steps = n_steps;
  CUDA_TRY(launch_persistent(t, t->P, 1));
  t->pending.emplace_back(dt_fs, n_steps);
  t->t_fs += dt_fs * n_steps;
  return TTNS_OK;
}

extern "C" ttns_status ttns_sync(ttns_tree* t) {
  if (!t) return fail(TTNS_E_INVALID, "tree is NULL");
  return wait_and_check(t, false, "device status: ");
}

static int find_root_fwd_terms(ttns_tree* t, int tree_idx, int* n2) {
  const TreeDesc& td = t->C.trees[tree_idx];
  for (int k = 0; k < td.prog_count; ++k) {
    const Instr& I = t->C.prog[td.prog_first + k];
    if (I.op == OP_FWD && I.node == td.node0) {
      *n2 = t->C.lists[I.terms].n2;
      return I.terms;
    }
  }
  return -1;
}

// root densities: rho_S (phys leg) into obs + off
static ttns_status density(ttns_tree* t, int node, int leg, const double2* rho_in, double* out) {
  const NodeDesc& nd = t->C.nodes[node];
  const int D = nd.dims[leg];
  // about eight rows per block; rho_in applied once per element into the worker workspace
  int nblocks = (int)std::min<long long>(1024, std::max<long long>(1, nd.size / D / 8));
  CUDA_TRY(launch_density(t->pool, nd, leg, rho_in, t->work, t->obs, nblocks, out, t->stream));
  return TTNS_OK;
}

extern "C" ttns_status ttns_reduced_density_matrix(ttns_tree* t, int tree_idx, double* rho_out) {
  if (!t || !rho_out) return fail(TTNS_E_INVALID, "NULL argument");
  if (tree_idx < 0 || tree_idx >= (int)t->C.trees.size()) return fail(TTNS_E_INVALID, "tree_idx out of range");
  ttns_status s = ttns_sync(t);
  if (s != TTNS_OK) return s;
  const TreeDesc& td = t->C.trees[tree_idx];
  double* out = t->obs + t->o_rho;
  if ((s = density(t, td.node0, td.root_phys_leg, nullptr, out)) != TTNS_OK) return s;
  CUDA_TRY(cudaMemcpyAsync(rho_out, out, sizeof(double) * 2 * td.n_el * td.n_el, cudaMemcpyDeviceToHost, t->stream));
  CUDA_TRY(cudaStreamSynchronize(t->stream));
  return TTNS_OK;
}

// Downward pass of bond densities from the root (the centre): the parent-bond density of
// every non-root node v at obs + o_bond + v * 2 maxD^2 (D_v x D_v, row-major); with sites,
// also every chain site's local density and <n> (occupations).
static ttns_status downward_pass(ttns_tree* t, int tree_idx, bool sites);

extern "C" ttns_status ttns_occupations(ttns_tree* t, int tree_idx, double* occ_out) {
  if (!t || !occ_out) return fail(TTNS_E_INVALID, "NULL argument");
  if (tree_idx < 0 || tree_idx >= (int)t->C.trees.size()) return fail(TTNS_E_INVALID, "tree_idx out of range");
  ttns_status s = ttns_sync(t);
  if (s != TTNS_OK) return s;
  if ((s = downward_pass(t, tree_idx, true)) != TTNS_OK) return s;
  const TreeDesc& td = t->C.trees[tree_idx];
  CUDA_TRY(cudaMemcpyAsync(occ_out, t->obs + t->o_occ, sizeof(double) * td.n_sites, cudaMemcpyDeviceToHost, t->stream));
  CUDA_TRY(cudaStreamSynchronize(t->stream));
  return TTNS_OK;
}

static ttns_status downward_pass(ttns_tree* t, int tree_idx, bool sites) {
  ttns_status s;
  const HostTree& h = t->C.host[tree_idx];
  const TreeDesc& td = t->C.trees[tree_idx];
  const int maxD = t->C.max_D;
  // per node: incoming parent-bond density at dens + v * 2 maxD^2
  double* dens = t->obs + t->o_bond;
  double* occ_dev = t->obs + t->o_occ;
  // preorder walk
  std::vector<int> order;
  std::vector<int> stack{0};
  while (!stack.empty()) {
    int v = stack.back();
    stack.pop_back();
    order.push_back(v);
    for (auto it = h.children[v].rbegin(); it != h.children[v].rend(); ++it) stack.push_back(*it);
  }
  std::vector<int> site_pos(h.n(), -1);
  {
    int k = 0;
    for (auto& c : h.chain_nodes)
      for (int v : c) site_pos[v] = k++;
  }
  double* site_dens = t->obs + t->o_site;  // 2*maxD^2 per site
  for (int v : order) {
    const int gv = td.node0 + v;
    const double2* rin = h.parent[v] >= 0 ? (const double2*)(dens + (long long)v * 2 * maxD * maxD) : nullptr;
    for (int c : h.children[v]) {
      if ((s = density(t, gv, h.leg_of(v, c), rin, dens + (long long)c * 2 * maxD * maxD)) != TTNS_OK) return s;
    }
    if (sites && h.parent[v] >= 0 && h.phys[v] > 0 && site_pos[v] >= 0) {
      double* sd = site_dens + (long long)site_pos[v] * 2 * maxD * maxD;
      if ((s = density(t, gv, h.phys_leg(v), rin, sd)) != TTNS_OK) return s;
      CUDA_TRY(launch_occ((const double2*)sd, h.phys[v], occ_dev + site_pos[v], t->stream));
    }
  }
  return TTNS_OK;
}

static ttns_status surface_scratch(ttns_tree* t, long long doubles) {
  if (t->surf_size >= doubles) return TTNS_OK;
  ttns_status s = dalloc(t, &t->surf, (size_t)doubles);
  if (s != TTNS_OK) return s;
  t->surf_size = doubles;
  return TTNS_OK;
}

// Batched Hermitian eigenvalues (and optionally vectors) of count matrices in device memory.
static ttns_status eig_batch(ttns_tree* t, const double2* base, const std::vector<long long>& offs,
                             const std::vector<int>& ns, double* d_evals, double2* d_evecs, long long* d_offs,
                             int* d_ns) {
  const int count = (int)offs.size();
  int n_max = 1;
  for (int n : ns) n_max = std::max(n_max, n);
  if (n_max > 64) return fail(TTNS_E_INVALID, "eigenproblem larger than 64");
  CUDA_TRY(cudaMemcpyAsync(d_offs, offs.data(), sizeof(long long) * count, cudaMemcpyHostToDevice, t->stream));
  CUDA_TRY(cudaMemcpyAsync(d_ns, ns.data(), sizeof(int) * count, cudaMemcpyHostToDevice, t->stream));
  CUDA_TRY(cudaMemcpyAsync(d_ns + count, ns.data(), sizeof(int) * count, cudaMemcpyHostToDevice, t->stream));
  CUDA_TRY(launch_herm_jacobi(base, d_offs, d_ns, d_ns + count, count, n_max, d_evals, d_evecs, t->stream));
  return TTNS_OK;
}

// The environment pass of the chains' kinetic energy (persistent kernel, phase 2), repeated as
// a plain cluster launch if the launch check refused it.
// One launch of a single-pass phase of the persistent kernel (2: the kinetic operator's
// environment pass, 3: the completion of grown bonds, 0: the environment pass), with the
// repeat of a refused launch as a plain cluster launch (nothing ran in the refused one).
static ttns_status run_phase(ttns_tree* t, int phase, const char* what) {
  KernelParams Pp = t->P;
  Pp.dt = 0.0;
  Pp.n_steps = 1;
  CUDA_TRY(launch_sweep(Pp, phase, t->grid, t->cluster, !(t->opt.launch_flags & 1), t->stream));
  CUDA_TRY(cudaStreamSynchronize(t->stream));
  Ctl h;
  CUDA_TRY(cudaMemcpy(&h, t->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  if (launch_refused(h) && !(t->opt.launch_flags & 1)) {
    t->opt.launch_flags |= 1;
    ++t->launch_fallbacks;
    h.status = h.err_where = h.err_node = 0;
    CUDA_TRY(cudaMemcpy(t->ctl, &h, sizeof(Ctl), cudaMemcpyHostToDevice));
    CUDA_TRY(launch_sweep(Pp, phase, t->grid, t->cluster, 0, t->stream));
    CUDA_TRY(cudaStreamSynchronize(t->stream));
    CUDA_TRY(cudaMemcpy(&h, t->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  }
  if (h.status != 0) return fail((ttns_status)h.status, std::string(what) + status_text(h));
  return TTNS_OK;
}

static ttns_status kinetic_envs(ttns_tree* t) { return run_phase(t, 2, "kinetic environment pass: "); }

extern "C" ttns_status ttns_energy_surfaces(ttns_tree* t, int tree_idx, double sigma_tol, double* tes, double* pes,
                                            double* sigma, int* n_bath) {
  if (!t || !tes || !pes || !sigma || !n_bath) return fail(TTNS_E_INVALID, "NULL argument");
  if (tree_idx < 0 || tree_idx >= (int)t->C.trees.size()) return fail(TTNS_E_INVALID, "tree_idx out of range");
  if (!(sigma_tol >= 0.0)) return fail(TTNS_E_INVALID, "sigma_tol must be >= 0");
  ttns_status s = ttns_sync(t);
  if (s != TTNS_OK) return s;
  const TreeDesc& td = t->C.trees[tree_idx];
  const int ne = td.n_el;
  if (ne > 16) return fail(TTNS_E_INVALID, "energy surfaces need n_el <= 16");
  const NodeDesc& rootd = t->C.nodes[td.node0];
  const long long R = rootd.size / ne;
  // scratch: evals (2 x 64), evecs (64 x 64 complex), U and sigma of the kept states, H / T / V
  // (32 x 32 complex each), projection partials (256 blocks x 2 x 32), offsets and sizes
  const long long o_ev = 0, o_vec = 128, o_u = o_vec + 2 * 64 * 64, o_sig = o_u + 2 * 16 * 16,
                  o_h = o_sig + 64, o_t = o_h + 2 * 32 * 32, o_v = o_t + 2 * 32 * 32, o_part = o_v + 2 * 32 * 32,
                  o_offs = o_part + 256 * 2 * 32, o_ns = o_offs + 8, total = o_ns + 8;
  if ((s = surface_scratch(t, total)) != TTNS_OK) return s;
  double* sc = t->surf;
  // 1. environment blocks of the kinetic energy at the current state
  if ((s = kinetic_envs(t)) != TTNS_OK) return s;
  // 2. Schmidt decomposition through rho_S = A^T conj(A): eigenvectors and values
  double* rho = t->obs + t->o_rho;
  if ((s = density(t, td.node0, td.root_phys_leg, nullptr, rho)) != TTNS_OK) return s;
  if ((s = eig_batch(t, (const double2*)rho, {0}, {ne}, sc + o_ev, (double2*)(sc + o_vec), (long long*)(sc + o_offs),
                     (int*)(sc + o_ns))) != TTNS_OK)
    return s;
  std::vector<double> ev(64);
  std::vector<double2> vec(64 * 64);
  CUDA_TRY(cudaMemcpyAsync(ev.data(), sc + o_ev, sizeof(double) * 64, cudaMemcpyDeviceToHost, t->stream));
  CUDA_TRY(cudaMemcpyAsync(vec.data(), sc + o_vec, sizeof(double2) * 64 * 64, cudaMemcpyDeviceToHost, t->stream));
  CUDA_TRY(cudaStreamSynchronize(t->stream));
  std::vector<int> keep;
  for (int k = ne - 1; k >= 0; --k) {
    const double sg = std::sqrt(std::max(ev[k], 0.0));
    sigma[ne - 1 - k] = sg;
    if (sg > sigma_tol) keep.push_back(k);
  }
  const int nb = (int)keep.size();
  const int nv = nb * ne;
  if (nv > 32) return fail(TTNS_E_INVALID, "energy surfaces need (bath states) x n_el <= 32");
  *n_bath = nb;
  if (nb == 0) return fail(TTNS_E_INVALID, "no Schmidt value above sigma_tol");
  std::vector<double2> U(ne * nb);
  std::vector<double> sg(nb);
  for (int k = 0; k < nb; ++k) {
    sg[k] = std::sqrt(std::max(ev[keep[k]], 0.0));
    for (int q = 0; q < ne; ++q) U[q * nb + k] = vec[q * 64 + keep[k]];
  }
  CUDA_TRY(cudaMemcpyAsync(sc + o_u, U.data(), sizeof(double2) * U.size(), cudaMemcpyHostToDevice, t->stream));
  CUDA_TRY(cudaMemcpyAsync(sc + o_sig, sg.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, t->stream));
  // 3. bath states and the projected H_eff(root), T_eff(root) in the basis |phi_k, l>
  const long long kv = t->P.kvec;
  double2* slot = t->work + (long long)(t->P.mmax + t->P.n_tmp + 2) * kv;
  double2 *Phi = slot, *X = slot + kv, *Y = slot + 2 * kv;
  const double2* A = t->pool + rootd.off;
  CUDA_TRY(launch_bath_states(A, R, ne, (const double2*)(sc + o_u), sc + o_sig, nb, Phi, t->stream));
  const int nbl = (int)std::min<long long>(1024, (rootd.size + 255) / 256);
  const int npb = (int)std::min<long long>(256, R / 64 + 1);
  const int n2h = t->C.lists[td.heff_terms].n2, n2t = t->C.lists[td.teff_terms].n2;
  for (int c = 0; c < nv; ++c) {
    CUDA_TRY(launch_build_x(Phi, c / ne, c % ne, R, ne, X, t->stream));
    CUDA_TRY(launch_apply_x(t->P, td.node0, td.heff_terms, n2h, X, Y, nbl, t->stream));
    CUDA_TRY(launch_project(Y, Phi, R, ne, nb, sc + o_part, npb, sc + o_h + 2LL * c * nv, t->stream));
    CUDA_TRY(launch_apply_x(t->P, td.node0, td.teff_terms, n2t, X, Y, nbl, t->stream));
    CUDA_TRY(launch_project(Y, Phi, R, ne, nb, sc + o_part, npb, sc + o_t + 2LL * c * nv, t->stream));
  }
  // 4. V = H - T and the eigenvalues of both (the matrices are stored by columns: their
  //    transposes, conj(H) and conj(V), have the same eigenvalues)
  CUDA_TRY(launch_sub(sc + o_h, sc + o_t, sc + o_v, 2 * nv * nv, t->stream));
  if ((s = eig_batch(t, (const double2*)sc, {o_h / 2, o_v / 2}, {nv, nv}, sc + o_ev, nullptr,
                     (long long*)(sc + o_offs), (int*)(sc + o_ns))) != TTNS_OK)
    return s;
  std::vector<double> ev2(128);
  CUDA_TRY(cudaMemcpyAsync(ev2.data(), sc + o_ev, sizeof(double) * 128, cudaMemcpyDeviceToHost, t->stream));
  CUDA_TRY(cudaStreamSynchronize(t->stream));
  for (int k = 0; k < nv; ++k) {
    tes[k] = ev2[k];
    pes[k] = ev2[64 + k];
  }
  return TTNS_OK;
}

// Spectra of rho_S (node 0) and of every non-root node's parent-bond density matrix: the
// downward pass of bond densities and the batched Hermitian Jacobi; ev holds 64 values per
// node (the first ns[v] are the eigenvalues of node v's matrix).
static ttns_status bond_spectra(ttns_tree* t, int tree_idx, std::vector<double>* ev, std::vector<int>* ns_out) {
  ttns_status s = ttns_sync(t);
  if (s != TTNS_OK) return s;
  const TreeDesc& td = t->C.trees[tree_idx];
  const HostTree& h = t->C.host[tree_idx];
  const int n = h.n();
  const int maxD = t->C.max_D;
  if ((s = downward_pass(t, tree_idx, false)) != TTNS_OK) return s;
  double* rho = t->obs + t->o_rho;
  if ((s = density(t, td.node0, td.root_phys_leg, nullptr, rho)) != TTNS_OK) return s;
  // matrices: rho_S (root), then every node's parent-bond density
  const long long o_ev = 0, o_offs = 64LL * n, o_ns = o_offs + n + 8, total = o_ns + n + 8;
  if ((s = surface_scratch(t, std::max<long long>(total, 1))) != TTNS_OK) return s;
  // rho_S and the bond densities live in one buffer (obs): offsets relative to obs as double2
  std::vector<long long> offs(n);
  std::vector<int>& ns = *ns_out;
  ns.assign(n, 0);
  offs[0] = (t->o_rho) / 2;
  ns[0] = td.n_el;
  for (int v = 1; v < n; ++v) {
    offs[v] = (t->o_bond + (long long)v * 2 * maxD * maxD) / 2;
    ns[v] = h.bond[v];
  }
  double* sc = t->surf;
  if ((s = eig_batch(t, (const double2*)t->obs, offs, ns, sc + o_ev, nullptr, (long long*)(sc + o_offs),
                     (int*)(sc + o_ns))) != TTNS_OK)
    return s;
  ev->assign(64LL * n, 0.0);
  CUDA_TRY(cudaMemcpyAsync(ev->data(), sc + o_ev, sizeof(double) * 64 * n, cudaMemcpyDeviceToHost, t->stream));
  CUDA_TRY(cudaStreamSynchronize(t->stream));
  return TTNS_OK;
}

extern "C" ttns_status ttns_bond_entropies(ttns_tree* t, int tree_idx, double* S_out) {
  if (!t || !S_out) return fail(TTNS_E_INVALID, "NULL argument");
  if (tree_idx < 0 || tree_idx >= (int)t->C.trees.size()) return fail(TTNS_E_INVALID, "tree_idx out of range");
  std::vector<double> ev;
  std::vector<int> ns;
  ttns_status s = bond_spectra(t, tree_idx, &ev, &ns);
  if (s != TTNS_OK) return s;
  for (int v = 0; v < (int)ns.size(); ++v) {
    double S = 0.0;
    for (int a = 0; a < ns[v]; ++a) {
      const double l = ev[(long long)v * 64 + a];
      if (l > 1e-300) S -= l * std::log(l);
    }
    S_out[v] = S;
  }
  return TTNS_OK;
}

// Adaptive bond dimension: the tree is rebuilt with the larger bonds, every tensor copied
// with zero slices on the grown legs, and the completion program (children first: the QR of
// each grown child toward its parent, whose zero columns get the identity reflector, and the
// absorb of R into the parent) runs before a fresh environment pass; the new tree set takes
// the place of the old one in the same handle.
extern "C" ttns_status ttns_grow_bonds(ttns_tree* t, const int* new_bond, int n_nodes, int* n_grown) {
  if (!t || !new_bond) return fail(TTNS_E_INVALID, "NULL argument");
  if (n_grown) *n_grown = 0;
  if (t->C.trees.size() != 1) return fail(TTNS_E_INVALID, "bond growth works on a single-tree set");
  const HostTree h = t->C.host[0];
  if (n_nodes != h.n()) return fail(TTNS_E_INVALID, "n_nodes does not match the tree");
  ttns_status s = ttns_sync(t);
  if (s != TTNS_OK) return s;
  TreeInput in = t->inputs[0];
  in.bond_req.assign(h.n(), 0);
  for (int v = 1; v < h.n(); ++v) in.bond_req[v] = std::max(h.bond[v], new_bond[v]);
  ttns_tree* t2 = new ttns_tree();
  std::vector<TreeInput> ins{in};
  if ((s = compile_inputs(std::move(ins), t->opt, t2)) != TTNS_OK) {
    delete t2;
    return s;
  }
  const HostTree& h2 = t2->C.host[0];
  std::vector<int> grown;
  for (int v = 1; v < h2.n(); ++v)
    if (h2.bond[v] > h.bond[v]) grown.push_back(v);
  if (grown.empty()) {
    delete t2;
    return TTNS_OK;
  }
  // the completion program, children first
  {
    Compiled& C2 = t2->C;
    TreeDesc& td2 = C2.trees[0];
    const long long gthr = t->opt.grid_threshold > 0 ? t->opt.grid_threshold : 16384;
    const long long qthr = t->opt.qr_grid_threshold > 0 ? t->opt.qr_grid_threshold : 65536;
    td2.grow_first = (int)C2.prog.size();
    for (auto it = grown.rbegin(); it != grown.rend(); ++it) {
      const int v = *it, p = h2.parent[v];
      Instr Q{};
      Q.op = OP_QR;
      Q.tree = 0;
      Q.node = td2.node0 + v;
      Q.leg = h2.leg_of(v, p);
      Q.D = C2.nodes[Q.node].dims[Q.leg];
      Q.team = C2.nodes[Q.node].size >= qthr ? TEAM_GRID : TEAM_CLUSTER;
      C2.prog.push_back(Q);
      Instr A{};
      A.op = OP_ABSORB;
      A.tree = 0;
      A.node = td2.node0 + p;
      A.leg = h2.leg_of(p, v);
      A.D = C2.nodes[A.node].dims[A.leg];
      A.team = C2.nodes[A.node].size >= gthr ? TEAM_GRID : TEAM_CLUSTER;
      C2.prog.push_back(A);
    }
    td2.grow_count = (int)C2.prog.size() - td2.grow_first;
  }
  if ((s = device_init(t2)) != TTNS_OK) {
    std::string keep = g_err;
    ttns_free(t2);
    g_err = keep;
    return s;
  }
  auto abort_with = [&](ttns_status st) {
    std::string keep = g_err;
    ttns_free(t2);
    g_err = keep;
    return st;
  };
  // the state, the trajectory record, the Krylov history and the counters
  const TreeDesc& td = t->C.trees[0];
  const TreeDesc& td2 = t2->C.trees[0];
  for (int v = 0; v < h.n(); ++v) {
    const NodeDesc& so = t->C.nodes[td.node0 + v];
    const NodeDesc& dn = t2->C.nodes[td2.node0 + v];
    bool shapes = so.nl == dn.nl && so.off + so.size <= t->C.pool_size && dn.off + dn.size <= t2->C.pool_size;
    for (int l = 0; shapes && l < so.nl; ++l) shapes = so.dims[l] <= dn.dims[l];
    if (!shapes) return abort_with(fail(TTNS_E_INVALID, "grown tree does not contain the old tensor shapes"));
    cudaError_t e = launch_pad_copy(t->pool, so, t2->pool, dn, t2->stream);
    if (e != cudaSuccess) return abort_with(fail(TTNS_E_CUDA, std::string("pad copy: ") + cudaGetErrorString(e)));
  }
  // the trajectory record exists only when recording is on (traj_off < 0 otherwise); both
  // trees have the same recording settings and electronic dimension
  if (td.traj_off >= 0 && td2.traj_off >= 0 && t->P.max_record == t2->P.max_record && td.n_el == td2.n_el) {
    const size_t traj = (size_t)t->P.max_record * td.n_el * td.n_el;
    if (td.traj_off + (long long)traj > t->C.pool_size || td2.traj_off + (long long)traj > t2->C.pool_size)
      return abort_with(fail(TTNS_E_INVALID, "trajectory region outside the pool"));
    if (cudaMemcpyAsync(t2->pool + td2.traj_off, t->pool + td.traj_off, traj * sizeof(double2),
                        cudaMemcpyDeviceToDevice, t2->stream) != cudaSuccess ||
        cudaMemcpyAsync(t2->traj_count, t->traj_count, sizeof(int), cudaMemcpyDeviceToDevice, t2->stream) != cudaSuccess)
      return abort_with(fail(TTNS_E_CUDA, "trajectory copy failed"));
  }
  if (t2->C.n_hist == t->C.n_hist &&
      cudaMemcpyAsync(t2->mhist, t->mhist, sizeof(int) * std::max(t->C.n_hist, 1), cudaMemcpyDeviceToDevice,
                      t2->stream) != cudaSuccess)
    return abort_with(fail(TTNS_E_CUDA, "history copy failed"));
  Ctl hc;
  if (cudaMemcpy(&hc, t->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost) != cudaSuccess)
    return abort_with(fail(TTNS_E_CUDA, "control block read failed"));
  hc.bar_count = 0;
  hc.bar_gen = 0;
  hc.status = hc.err_where = hc.err_node = 0;
  if (cudaMemcpy(t2->ctl, &hc, sizeof(Ctl), cudaMemcpyHostToDevice) != cudaSuccess)
    return abort_with(fail(TTNS_E_CUDA, "control block write failed"));
  if ((s = run_phase(t2, 3, "completion of grown bonds: ")) != TTNS_OK) return abort_with(s);
  if ((s = run_phase(t2, 0, "environment pass after growth: ")) != TTNS_OK) return abort_with(s);
  t2->t_fs = t->t_fs;
  t2->launch_fallbacks += t->launch_fallbacks;
  std::swap(*t, *t2);
  ttns_free(t2);  // the old tree set
  if (n_grown) *n_grown = (int)grown.size();
  return TTNS_OK;
}

extern "C" ttns_status ttns_adapt_bonds(ttns_tree* t, double eps, int step, int d_max, int* n_grown) {
  if (!t) return fail(TTNS_E_INVALID, "NULL argument");
  if (n_grown) *n_grown = 0;
  if (!(eps >= 0.0) || step < 1 || d_max < 1) return fail(TTNS_E_INVALID, "eps >= 0, step >= 1 and d_max >= 1 required");
  if (t->C.trees.size() != 1) return fail(TTNS_E_INVALID, "bond growth works on a single-tree set");
  std::vector<double> ev;
  std::vector<int> ns;
  ttns_status s = bond_spectra(t, 0, &ev, &ns);
  if (s != TTNS_OK) return s;
  const HostTree& h = t->C.host[0];
  std::vector<int> req(h.n(), 0);
  bool any = false;
  for (int v = 1; v < h.n(); ++v) {
    double lo = 1e300;
    for (int a = 0; a < ns[v]; ++a) lo = std::min(lo, ev[(long long)v * 64 + a]);
    if (h.bond[v] < d_max && lo > eps) {
      req[v] = std::min(h.bond[v] + step, d_max);
      any = true;
    }
  }
  if (!any) return TTNS_OK;
  return ttns_grow_bonds(t, req.data(), h.n(), n_grown);
}

extern "C" ttns_status ttns_observables(ttns_tree* t, int tree_idx, double* norm, double* energy) {
  if (!t || !norm || !energy) return fail(TTNS_E_INVALID, "NULL argument");
  if (tree_idx < 0 || tree_idx >= (int)t->C.trees.size()) return fail(TTNS_E_INVALID, "tree_idx out of range");
  ttns_status s = ttns_sync(t);
  if (s != TTNS_OK) return s;
  if (t->batched) {
    // the temporaries of worker 0 are used: fine outside a sweep
  }
  int n2 = 0;
  int li = find_root_fwd_terms(t, tree_idx, &n2);
  if (li < 0) return fail(TTNS_E_INVALID, "no root operator");
  double* out = t->obs + t->o_en;
  const int nb = 256;
  CUDA_TRY(launch_energy(t->P, t->C.trees[tree_idx].node0, li, n2, t->obs, nb, out, t->stream));
  double h[2];
  CUDA_TRY(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, t->stream));
  CUDA_TRY(cudaStreamSynchronize(t->stream));
  *norm = std::sqrt(h[1]);
  *energy = h[1] > 0 ? h[0] / h[1] : 0.0;
  return TTNS_OK;
}

extern "C" ttns_status ttns_trajectory(ttns_tree* t, int tree_idx, double* out, int max_steps, int* n_written) {
  if (!t || !out || !n_written) return fail(TTNS_E_INVALID, "NULL argument");
  if (tree_idx < 0 || tree_idx >= (int)t->C.trees.size()) return fail(TTNS_E_INVALID, "tree_idx out of range");
  if (!t->opt.record) return fail(TTNS_E_INVALID, "the tree was built without record=1");
  ttns_status s = ttns_sync(t);
  if (s != TTNS_OK) return s;
  int cnt = 0;
  CUDA_TRY(cudaMemcpy(&cnt, t->traj_count + tree_idx, sizeof(int), cudaMemcpyDeviceToHost));
  const TreeDesc& td = t->C.trees[tree_idx];
  cnt = std::min(cnt, std::min(max_steps, t->P.max_record));
  if (cnt > 0)
    CUDA_TRY(cudaMemcpy(out, t->pool + td.traj_off, sizeof(double2) * (size_t)cnt * td.n_el * td.n_el,
                        cudaMemcpyDeviceToHost));
  *n_written = cnt;
  return TTNS_OK;
}

extern "C" ttns_status ttns_populations_device(ttns_tree* t, double* dev_out) {
  if (!t || !dev_out) return fail(TTNS_E_INVALID, "NULL argument");
  ttns_status s;
  int off = 0;
  for (size_t k = 0; k < t->C.trees.size(); ++k) {
    const TreeDesc& td = t->C.trees[k];
    double* tmp = t->obs + t->o_rho;
    if ((s = density(t, td.node0, td.root_phys_leg, nullptr, tmp)) != TTNS_OK) return s;
    // diagonal (real parts) -> dev_out
    for (int q = 0; q < td.n_el; ++q)
      CUDA_TRY(cudaMemcpyAsync(dev_out + off + q, tmp + 2 * (q * td.n_el + q), sizeof(double), cudaMemcpyDeviceToDevice,
                               t->stream));
    off += td.n_el;
  }
  return TTNS_OK;
}

extern "C" ttns_status ttns_get_counters(ttns_tree* t, ttns_counters* out) {
  if (!t || !out) return fail(TTNS_E_INVALID, "NULL argument");
  CUDA_TRY(cudaStreamSynchronize(t->stream));
  Ctl h;
  CUDA_TRY(cudaMemcpy(&h, t->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  out->krylov_iters = (long long)h.krylov_iters;
  out->applies = (long long)h.applies;
  out->contraction_flops = h.flops;
  out->not_converged = (long long)h.not_converged;
  out->steps = (long long)h.steps;
  int khz = 0;
  cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, 0);
  const double hz = khz > 0 ? khz * 1e3 : 1.9e9;
  for (int op = 0; op < 6; ++op)
    for (int k = 0; k < 2; ++k) {
      out->op_seconds[op][k] = h.prof_cycles[op][k] / hz;
      out->op_count[op][k] = (long long)h.prof_count[op][k];
    }
  for (int k = 0; k < 8; ++k) out->expm_phase_seconds[k] = h.phase_cycles[k] / hz;
  for (int k = 0; k < 8; ++k) out->qr_phase_seconds[k] = h.phase_cycles[8 + k] / hz;
  for (int k = 0; k < 8; ++k) out->expm_phase_seconds_grid[k] = h.phase_cycles_grid[k] / hz;
  for (int k = 0; k < 8; ++k) out->qr_phase_seconds_grid[k] = h.phase_cycles_grid[8 + k] / hz;
  for (int k = 0; k < 4; ++k) {
    out->env_phase_seconds[0][k] = h.phase_cycles[16 + k] / hz;
    out->env_phase_seconds[1][k] = h.phase_cycles_grid[16 + k] / hz;
    out->tc_phase_seconds[k] = h.phase_cycles_grid[20 + k] / hz;
  }
  out->launch_fallbacks = t->launch_fallbacks;
  return TTNS_OK;
}

extern "C" ttns_status ttns_node_info(ttns_tree* t, int tree_idx, int node, int* n_legs, int* dims, int* n_nodes) {
  if (!t) return fail(TTNS_E_INVALID, "tree is NULL");
  if (tree_idx < 0 || tree_idx >= (int)t->C.trees.size()) return fail(TTNS_E_INVALID, "tree_idx out of range");
  const TreeDesc& td = t->C.trees[tree_idx];
  if (n_nodes) *n_nodes = td.n_nodes;
  if (node < 0) return TTNS_OK;
  if (node >= td.n_nodes) return fail(TTNS_E_INVALID, "node out of range");
  const NodeDesc& nd = t->C.nodes[td.node0 + node];
  if (n_legs) *n_legs = nd.nl;
  if (dims)
    for (int k = 0; k < nd.nl; ++k) dims[k] = nd.dims[k];
  return TTNS_OK;
}

extern "C" ttns_status ttns_get_node(ttns_tree* t, int tree_idx, int node, double* out, size_t n_complex) {
  if (!t || !out) return fail(TTNS_E_INVALID, "NULL argument");
  if (tree_idx < 0 || tree_idx >= (int)t->C.trees.size()) return fail(TTNS_E_INVALID, "tree_idx out of range");
  const TreeDesc& td = t->C.trees[tree_idx];
  if (node < 0 || node >= td.n_nodes) return fail(TTNS_E_INVALID, "node out of range");
  const NodeDesc& nd = t->C.nodes[td.node0 + node];
  if (n_complex < (size_t)nd.size) return fail(TTNS_E_INVALID, "output buffer too small");
  ttns_status s = ttns_sync(t);
  if (s != TTNS_OK) return s;
  CUDA_TRY(cudaMemcpy(out, t->pool + nd.off, sizeof(double2) * nd.size, cudaMemcpyDeviceToHost));
  return TTNS_OK;
}

// Checkpoint format (little-endian host types):
//   "TTNSCKP3", int64 n_trees, every tree's problem (TreeInput: n_el, shifted-free H_S,
//   patterns, chains, dims, requested bonds, ER layout, initial amplitudes, the per-node bond
//   requests of a grown tree), int32 record and
//   max_record, then int64 {pool size, history slots, trees, 0}, double t_fs, the complex pool
//   (tensors, environment blocks, trajectory), the Krylov-length history, the trajectory
//   counters and the device control block.
static const char kMagic[8] = {'T', 'T', 'N', 'S', 'C', 'K', 'P', '3'};

namespace {
struct Writer {
  FILE* f;
  bool ok = true;
  template <typename T> void put(const T& x) { ok = ok && std::fwrite(&x, sizeof(T), 1, f) == 1; }
  template <typename T> void put_vec(const std::vector<T>& v) {
    put((long long)v.size());
    if (!v.empty()) ok = ok && std::fwrite(v.data(), sizeof(T), v.size(), f) == v.size();
  }
};
struct Reader {
  FILE* f;
  bool ok = true;
  template <typename T> void get(T& x) { ok = ok && std::fread(&x, sizeof(T), 1, f) == 1; }
  template <typename T> void get_vec(std::vector<T>& v, long long max_n) {
    long long n = -1;
    get(n);
    if (!ok || n < 0 || n > max_n) { ok = false; return; }
    v.resize(n);
    if (n > 0) ok = ok && std::fread(v.data(), sizeof(T), n, f) == (size_t)n;
  }
};
const long long kMaxVec = 1LL << 26;

void write_input(Writer& w, const TreeInput& in) {
  w.put(in.n_el);
  w.put_vec(in.H_S);
  w.put(in.n_env);
  w.put((long long)in.W.size());
  for (const auto& x : in.W) w.put_vec(x);
  w.put_vec(in.rc);
  w.put((long long)in.omega.size());
  for (const auto& x : in.omega) w.put_vec(x);
  w.put((long long)in.hop.size());
  for (const auto& x : in.hop) w.put_vec(x);
  w.put_vec(in.L);
  w.put_vec(in.d);
  w.put_vec(in.D);
  w.put_vec(in.obb);
  w.put(in.er_tree);
  w.put(in.D_er);
  w.put_vec(in.psi_el);
  w.put_vec(in.bond_req);
}

bool read_input(Reader& r, TreeInput& in) {
  long long n = 0;
  r.get(in.n_el);
  r.get_vec(in.H_S, kMaxVec);
  r.get(in.n_env);
  r.get(n);
  if (!r.ok || n < 0 || n > 4096) return false;
  in.W.resize(n);
  for (auto& x : in.W) r.get_vec(x, kMaxVec);
  r.get_vec(in.rc, kMaxVec);
  r.get(n);
  if (!r.ok || n < 0 || n > 4096) return false;
  in.omega.resize(n);
  for (auto& x : in.omega) r.get_vec(x, kMaxVec);
  r.get(n);
  if (!r.ok || n < 0 || n > 4096) return false;
  in.hop.resize(n);
  for (auto& x : in.hop) r.get_vec(x, kMaxVec);
  r.get_vec(in.L, kMaxVec);
  r.get_vec(in.d, kMaxVec);
  r.get_vec(in.D, kMaxVec);
  r.get_vec(in.obb, kMaxVec);
  r.get(in.er_tree);
  r.get(in.D_er);
  r.get_vec(in.psi_el, kMaxVec);
  r.get_vec(in.bond_req, kMaxVec);
  if (!r.ok) return false;
  // the shapes must agree with each other (the values were validated when the file was written)
  const size_t ne = (size_t)in.n_env;
  if (in.n_el < 1 || in.n_el > TTNS_MAX_D || in.n_env < 1 || in.H_S.size() != (size_t)in.n_el * in.n_el ||
      in.W.size() != ne || in.rc.size() != ne || in.omega.size() != ne || in.hop.size() != ne || in.L.size() != ne ||
      in.d.size() != ne || in.D.size() != ne || in.obb.size() != ne || in.psi_el.size() != (size_t)in.n_el)
    return false;
  for (size_t i = 0; i < ne; ++i) {
    if (in.W[i].size() != (size_t)in.n_el * in.n_el || in.L[i] < 1 || in.L[i] > 4096 ||
        in.omega[i].size() != (size_t)in.L[i] || in.hop[i].size() != (size_t)std::max(in.L[i] - 1, 0) ||
        in.d[i] < 2 || in.d[i] > TTNS_MAX_D || in.D[i] < 1)
      return false;
  }
  return true;
}

// Reads the problem section of a checkpoint; leaves the file at the state section.
ttns_status read_header(FILE* f, std::vector<TreeInput>* ins, int* record, int* max_record) {
  char magic[8];
  Reader r{f};
  if (std::fread(magic, 1, 8, f) != 8 || std::memcmp(magic, kMagic, 8) != 0)
    return fail(TTNS_E_IO, "not a TTNS checkpoint (bad magic)");
  long long nt = 0;
  r.get(nt);
  if (!r.ok || nt < 1 || nt > (1 << 20)) return fail(TTNS_E_IO, "checkpoint: bad tree count");
  ins->resize(nt);
  for (auto& in : *ins)
    if (!read_input(r, in)) return fail(TTNS_E_IO, "checkpoint: truncated or malformed problem section");
  r.get(*record);
  r.get(*max_record);
  if (!r.ok) return fail(TTNS_E_IO, "checkpoint truncated");
  return TTNS_OK;
}

// Reads the state section into an existing tree set of the same shape.
ttns_status read_state(ttns_tree* t, FILE* f) {
  long long hdr[4];
  double tf = 0;
  Reader r{f};
  r.get(hdr);
  r.get(tf);
  if (!r.ok || hdr[0] != t->C.pool_size || hdr[1] != (long long)std::max(t->C.n_hist, 1) ||
      hdr[2] != (long long)t->C.trees.size())
    return fail(TTNS_E_IO, "checkpoint does not match this tree (or is truncated)");
  std::vector<double2> pool(hdr[0]);
  std::vector<int> mh(hdr[1]), tc(hdr[2]);
  Ctl h;
  bool ok = std::fread(pool.data(), sizeof(double2), pool.size(), f) == pool.size() &&
            std::fread(mh.data(), sizeof(int), mh.size(), f) == mh.size() &&
            std::fread(tc.data(), sizeof(int), tc.size(), f) == tc.size() && std::fread(&h, sizeof(Ctl), 1, f) == 1;
  if (!ok) return fail(TTNS_E_IO, "checkpoint truncated");
  // the tensors are not validated here: a non-finite entry is reported by the next step
  // (TTNS_E_NONFINITE from the Krylov norm)
  h.bar_count = 0;
  h.bar_gen = 0;
  h.status = 0;
  h.err_where = 0;
  h.err_node = 0;
  CUDA_TRY(cudaMemcpy(t->pool, pool.data(), pool.size() * sizeof(double2), cudaMemcpyHostToDevice));
  if (t->pool32) {
    CUDA_TRY(launch_mirror32(t->pool, t->pool32, (long long)pool.size(), t->stream));
    CUDA_TRY(cudaStreamSynchronize(t->stream));
  }
  CUDA_TRY(cudaMemcpy(t->mhist, mh.data(), mh.size() * sizeof(int), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(t->traj_count, tc.data(), tc.size() * sizeof(int), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(t->ctl, &h, sizeof(Ctl), cudaMemcpyHostToDevice));
  t->t_fs = tf;
  return TTNS_OK;
}
}  // namespace

extern "C" ttns_status ttns_save(ttns_tree* t, const char* path) {
  if (!t || !path) return fail(TTNS_E_INVALID, "NULL argument");
  ttns_status s = ttns_sync(t);
  if (s != TTNS_OK) return s;
  std::vector<double2> pool(t->C.pool_size);
  std::vector<int> mh(std::max(t->C.n_hist, 1)), tc(t->C.trees.size());
  Ctl h;
  CUDA_TRY(cudaMemcpy(pool.data(), t->pool, pool.size() * sizeof(double2), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemcpy(mh.data(), t->mhist, mh.size() * sizeof(int), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemcpy(tc.data(), t->traj_count, tc.size() * sizeof(int), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemcpy(&h, t->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(TTNS_E_IO, std::string("cannot open ") + path);
  Writer w{f};
  w.ok = std::fwrite(kMagic, 1, 8, f) == 8;
  w.put((long long)t->inputs.size());
  for (const TreeInput& in : t->inputs) write_input(w, in);
  w.put((int)t->opt.record);
  w.put((int)t->P.max_record);
  long long hdr[4] = {(long long)pool.size(), (long long)mh.size(), (long long)tc.size(), 0};
  w.put(hdr);
  w.put(t->t_fs);
  bool ok = w.ok && std::fwrite(pool.data(), sizeof(double2), pool.size(), f) == pool.size() &&
            std::fwrite(mh.data(), sizeof(int), mh.size(), f) == mh.size() &&
            std::fwrite(tc.data(), sizeof(int), tc.size(), f) == tc.size() && std::fwrite(&h, sizeof(Ctl), 1, f) == 1;
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return fail(TTNS_E_IO, std::string("write failed: ") + path);
  return TTNS_OK;
}

extern "C" ttns_status ttns_load_state(ttns_tree* t, const char* path) {
  if (!t || !path) return fail(TTNS_E_INVALID, "NULL argument");
  ttns_status s = ttns_sync(t);
  if (s != TTNS_OK) return s;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(TTNS_E_IO, std::string("cannot open ") + path);
  std::vector<TreeInput> ins;
  int record = 0, max_record = 0;
  s = read_header(f, &ins, &record, &max_record);
  if (s == TTNS_OK) s = read_state(t, f);
  std::fclose(f);
  return s;
}

static ttns_status build_inputs(std::vector<TreeInput> ins, const ttns_options& o, ttns_tree** out);

extern "C" ttns_status ttns_load(const char* path, const ttns_options* opt, ttns_tree** out) {
  if (!path || !out) return fail(TTNS_E_INVALID, "NULL argument");
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(TTNS_E_IO, std::string("cannot open ") + path);
  std::vector<TreeInput> ins;
  int record = 0, max_record = 0;
  ttns_status s = read_header(f, &ins, &record, &max_record);
  if (s != TTNS_OK) {
    std::fclose(f);
    return s;
  }
  ttns_options o{};
  if (opt) o = *opt;
  // the tree layout and the trajectory buffer come from the file (the pool must match)
  o.er_tree = ins[0].er_tree;
  o.D_er = ins[0].D_er;
  o.psi_el = nullptr;
  o.record = record;
  o.max_record = max_record;
  ttns_tree* t = nullptr;
  s = build_inputs(std::move(ins), o, &t);
  if (s == TTNS_OK) s = read_state(t, f);
  std::fclose(f);
  if (s != TTNS_OK) {
    std::string keep = g_err;
    ttns_free(t);
    g_err = keep;
    return s;
  }
  *out = t;
  return TTNS_OK;
}

extern "C" void ttns_free(ttns_tree* t) {
  if (!t) return;
  if (t->stream) cudaStreamSynchronize(t->stream); else cudaDeviceSynchronize();
  for (void* p : t->allocs) cudaFree(p);
  delete t;
}

extern "C" ttns_status ttns_chain_ohmic(double alpha, double omega_c, int L, double* rc, double* onsite, double* hop) {
  if (L < 1 || !rc || !onsite || (L > 1 && !hop)) return fail(TTNS_E_INVALID, "bad arguments");
  if (!(alpha >= 0) || !(omega_c > 0)) return fail(TTNS_E_INVALID, "alpha must be >= 0 and omega_c > 0");
  chain_ohmic(alpha, omega_c, L, rc, onsite, hop);
  return TTNS_OK;
}

extern "C" ttns_status ttns_chain_from_modes(int n_modes, const double* omega, const double* lambda, int L, double* rc,
                                             double* onsite, double* hop) {
  if (n_modes < 1 || !omega || !lambda || !rc || !onsite || (L > 1 && !hop)) return fail(TTNS_E_INVALID, "bad arguments");
  if (L < 1 || L > n_modes) return fail(TTNS_E_INVALID, "L must be in 1..n_modes");
  if (!chain_from_modes(n_modes, omega, lambda, L, rc, onsite, hop))
    return fail(TTNS_E_INVALID, "Lanczos breakdown: fewer distinct modes than sites");
  return TTNS_OK;
}

extern "C" ttns_status ttns_selftest_wait_timeout(long long spin_limit, int* device_status) {
  if (!device_status) return fail(TTNS_E_INVALID, "NULL argument");
  Ctl* ctl = nullptr;
  CUDA_TRY(cudaMalloc(&ctl, sizeof(Ctl)));
  cudaError_t e = cudaMemset(ctl, 0, sizeof(Ctl));
  const int skip = spin_limit > 0 ? 1 : 0;
  if (e == cudaSuccess) e = launch_wait_selftest(ctl, spin_limit > 0 ? spin_limit : 2000000000LL, skip, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  Ctl h{};
  if (e == cudaSuccess) e = cudaMemcpy(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost);
  cudaFree(ctl);
  if (e != cudaSuccess) return fail(TTNS_E_CUDA, cudaGetErrorString(e));
  *device_status = h.status;
  return TTNS_OK;
}
