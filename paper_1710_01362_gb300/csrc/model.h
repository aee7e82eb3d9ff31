// Host-side model: the star Hamiltonian of Eq. 2 on a tree, the bond-dimension
// clamp, the isometric initial state, and the compilation of one TDVP step
// into device instructions.
#pragma once
#include <complex>
#include <string>
#include <vector>

#include "internal.h"

namespace ttns {

using cplx = std::complex<double>;

struct Coupling {
  int va;
  std::vector<cplx> opa;   // on va's physical leg (coefficient included)
  int vb;
  std::vector<cplx> opb;
};

// One tree: nodes in creation order, the root is node 0.
struct HostTree {
  int n_el = 0;
  std::vector<int> parent;
  std::vector<std::vector<int>> children;
  std::vector<int> phys;             // 0 = no physical leg
  std::vector<int> kind;             // 0 electronic, 1 ER, 2 chain site, 3 Fock leaf of a site (OBB)
  std::vector<int> bond;             // bond to parent (root: 0)
  std::vector<std::vector<cplx>> onsite;
  std::vector<Coupling> coups;
  std::vector<std::vector<int>> chain_nodes;  // nodes holding each chain's Fock legs, site order
  std::vector<cplx> psi_el;

  int n() const { return (int)parent.size(); }
  std::vector<int> legs(int v) const;
  int leg_of(int v, int u) const;    // leg of v pointing to neighbour u
  int phys_leg(int v) const;
  std::vector<int> neighbours(int v) const;
};

// Inputs of one tree (already validated).
struct TreeInput {
  int n_el;
  std::vector<cplx> H_S;
  int n_env;
  std::vector<std::vector<cplx>> W;  // per env, n_el^2
  std::vector<double> rc;
  std::vector<std::vector<double>> omega, hop;
  std::vector<int> L, d, D;
  std::vector<int> obb;              // per env: optimised boson basis dimension (0: none)
  int er_tree = 0;
  int D_er = 0;
  std::vector<cplx> psi_el;
  // requested parent-bond dimension of every node (node order of the built tree; the root's
  // entry unused), replacing the per-chain and ER requests when not empty: a tree whose bonds
  // were grown during the run
  std::vector<int> bond_req;
};

HostTree build_host_tree(const TreeInput& in);

// The same tree with the chains' nuclear kinetic energy as its operator:
//   T = -(1/4) sum_m w_m (a^+ - a)_m^2 - (1/2) sum_m t_m (a^+ - a)_m (a^+ - a)_{m+1}
// per chain (w_m onsite energies, t_m hoppings of the chain map): the kinetic energy of the
// normal modes, sum_n w_n p_n^2 / 2, written in the chain basis.
HostTree kinetic_tree(const HostTree& h, const TreeInput& in);

// Flattened device tables for a set of trees.
struct Compiled {
  std::vector<NodeDesc> nodes;
  std::vector<Term> terms;
  std::vector<TermList> lists;
  std::vector<Factor> chans;
  std::vector<Instr> prog;
  std::vector<TreeDesc> trees;
  std::vector<int> init_first, init_count;   // per tree: initial environment pass
  std::vector<double2> pool_init;            // initial complex pool contents
  long long pool_size = 0;
  int max_node = 0;          // largest tensor
  int max_tmp = 0;           // largest number of two-factor terms
  int max_D = 0;
  int n_hist = 0;
  std::vector<HostTree> host;
  std::vector<std::vector<int>> site_nodes;  // per tree: global node ids of chain sites, output order
  std::vector<double> flops_per_instr;       // useful flops of one apply of each instruction's operator
};

// grid_threshold: tensors at least this large use the whole-grid team (single-tree mode) for
// Krylov exponentials, environment updates and absorbs; qr_grid_threshold the same for QRs.
Compiled compile_trees(const std::vector<TreeInput>& inputs, bool batched, int grid_threshold,
                       int qr_grid_threshold, int max_record,
                       int record);

void chain_ohmic(double alpha, double omega_c, int L, double* rc, double* onsite, double* hop);
bool chain_from_modes(int K, const double* omega, const double* lam, int L, double* rc, double* onsite,
                      double* hop);

}  // namespace ttns
