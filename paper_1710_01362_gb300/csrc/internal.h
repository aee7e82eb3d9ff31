// Internal descriptors shared by the host model builder and the device sweep.
//
// Device memory of one tree set lives in one workspace:
//   cplx pool   node tensors, operator matrices, environment blocks, bond
//               matrices (FP64 complex, double2)
//   work        per worker (cluster team) Krylov basis, term temporaries,
//               QR work arrays, reduction partials
//   tables      node / term / instruction descriptors (this header)
#pragma once
#include <cstdint>
#include <vector_types.h>

#define TTNS_MAX_LEGS 8
#define TTNS_KMAX 32          // largest Krylov dimension
#define TTNS_MAX_TERMS 64     // terms of one local operator
#define TTNS_MAX_D 64         // largest bond / physical dimension handled by the QR

namespace ttns {

enum TeamKind : int { TEAM_GRID = 0, TEAM_CLUSTER = 1 };

enum OpCode : int {
  OP_FWD = 0,     // A_v <- exp(-i tau H_eff(v)) A_v
  OP_QR = 1,      // A_v <- Q (isometry toward leg), bond <- R
  OP_ENV = 2,     // env(u -> v) blocks from A_u
  OP_BOND = 3,    // bond <- exp(+i tau H_bond) bond
  OP_ABSORB = 4,  // A_u <- bond applied on leg
  OP_RECORD = 5   // rho_S -> trajectory slot (centre at the root)
};

struct NodeDesc {
  int nl;                        // number of legs
  int dims[TTNS_MAX_LEGS];
  int strides[TTNS_MAX_LEGS];    // row-major strides
  int size;                      // product of dims
  long long off;                 // offset of the tensor in the complex pool
  long long reg_off;             // operator region: the environment blocks flowing into this node
  int reg_len;                   // and its constant operators, contiguous (staged together)
  float inv_dims[TTNS_MAX_LEGS];     // 1/dims and 1/strides for exact fast index division
  float inv_strides[TTNS_MAX_LEGS];  // (indices stay below 2^24)
};

#define TTNS_SPARSE_MAX 4  // nonzeros per row of a constant operator stored in row-sparse form

struct Factor {
  int leg;        // leg of the tensor the matrix acts on
  long long mat;  // offset of a dims[leg] x dims[leg] row-major matrix in the complex pool
  int nnz;        // 0: dense; else row-sparse with nnz entries per row (constant operators only)
  long long sp;   // row-sparse table: dims*nnz values, then dims*nnz column indices (in .x)
};

struct Term {
  int nf;         // 1 or 2 factors
  Factor f[2];
  int sparse_f;   // two-factor terms evaluated directly: index of the sparse factor
};

// A list of terms in the global term table, ordered
//   [one-factor terms][direct two-factor terms][two-stage two-factor terms]
// Direct terms (one factor row-sparse) are evaluated in one pass from the input;
// two-stage terms go through a temporary (first factor, barrier, second factor).
struct TermList {
  int first;
  int count;
  int n2;         // two-stage two-factor terms (the last n2 entries)
  int nd;         // direct two-factor terms (before the two-stage ones)
};

struct Instr {
  int op;
  int team;        // TeamKind
  int tree;        // tree index
  int node;        // tensor the op works on (node id, or -1 for the bond matrix)
  int leg;         // leg of `node` toward the neighbour (QR, ENV, ABSORB)
  int terms;       // index into the TermList table (FWD, ENV H-block, BOND)
  int chan_first;  // ENV: first channel Factor in the factor table
  int nchan;       // ENV: number of channel blocks
  long long env_out;  // ENV: offset of the (1 + nchan) output blocks, each D x D
  int D;           // ENV / BOND / QR: dimension of the bond
  int D2;          // BOND: second dimension of the bond matrix
  int hist;        // Krylov-length history slot (FWD, BOND)
  double sign;     // FWD +1, BOND -1 (sign of the time argument)
  double flops;    // useful flops of one application of this op's operator
  long long rega_off, regb_off;  // operator regions staged in shared memory for this op
  int rega_len, regb_len;
};

// Per-tree description used by the device.
struct TreeDesc {
  int n_nodes;
  int node0;          // first node in the global node table
  int n_el;
  long long root_off; // offset of the root tensor (== node table entry node0)
  int root_phys_leg;
  long long bond_off; // bond matrix buffer (TTNS_MAX_D^2 complex)
  int prog_first;     // first instruction of one step
  int prog_count;
  int init_first;     // initial environment pass
  int init_count;
  long long traj_off; // trajectory buffer offset (complex), n_el^2 per step
  int max_node;       // largest tensor (complex elements)
  int n_sites;        // chain sites (occupation outputs)
  int obs_first;      // environment pass of the chains' kinetic-energy operator (energy surfaces)
  int obs_count;
  int heff_terms;     // term list of H_eff(root) and of T_eff(root)
  int teff_terms;
  int grow_first;     // completion of grown bonds (QR of each grown child, absorb into its parent)
  int grow_count;
};

// Device-side control block (status word, barrier, counters).
struct Ctl {
  unsigned bar_count;
  unsigned bar_gen;
  int status;          // ttns_status of the device
  int pad0;
  unsigned long long krylov_iters;
  unsigned long long applies;
  double flops;        // accumulated by team rank 0 only
  unsigned long long not_converged;
  unsigned long long steps;
  int err_where;       // op code of the first failure
  int err_node;
  unsigned long long prof_cycles[8][2];  // per op code and team kind (rank-0 CTA clock cycles)
  unsigned long long prof_count[8][2];
  unsigned long long phase_cycles[24];   // phases of the Krylov exponential (0-7), QR (8-15), env (16-19), cluster team
  unsigned long long phase_cycles_grid[24];  // the same for grid-team ops
  unsigned progress;                     // bumped after every cluster-team instruction
  unsigned pad1;
};

struct KernelParams {
  double2* pool;           // complex pool
  float2* pool32;          // FP32 mirror of the pool's operator data (mixed modes; else null):
                           // written with every operator, read by the compute-type contractions
  const NodeDesc* nodes;
  const Term* terms;
  const TermList* lists;
  const Factor* chans;
  const Instr* prog;
  const TreeDesc* trees;
  int n_trees;
  int batched;             // 1: each cluster runs whole trees; 0: one tree, mixed teams
  Ctl* ctl;
  // per-worker workspace
  double2* work;           // n_workers * work_stride complex
  long long work_stride;
  int kvec;                // complex elements per Krylov vector slot
  int n_tmp;               // two-factor temporaries per worker
  double* red;             // reduction partials: n_workers * 2 * red_stride doubles (grid: red_grid)
  long long red_stride;
  double* red_grid;        // grid-team reduction partials: 2 * red_stride_grid doubles
  long long red_stride_grid;
  double2* cta_scratch;    // per CTA (blockIdx.x) small-matrix scratch
  long long cta_scratch_stride;
  int* mhist;              // Krylov length history (per slot)
  int* traj_count;         // per tree
  int max_record;
  int record;
  // run parameters
  double dt;
  int n_steps;
  int precision;           // 0 FP64, 1 MIXED
  double tol;
  int mmax;
  int cluster_ctas;
  long long spin_limit;
  int profile;
  long long smem_bytes;    // dynamic shared memory per CTA (operator matrices of one op)
  int cluster_resident;    // 1: small-node Krylov exponentials kept in the cluster's shared memory
  double qr_cutoff;        // relative null threshold of the QR
};

}  // namespace ttns
